"""gwas_estimate (step 1: per-trait h^2, sigma^2 by ML or REML) on the GPU against the FP64
oracle (oracle/estimate.py), through the C ABI.

Both sides maximise the same criterion over [0, 0.999]; the maximum itself is well conditioned,
the maximiser less so where the criterion is flat.  The checks: the GPU's maximum equals the
oracle's to 1e-8 (relative), the oracle's own criterion at the GPU's h^2 is as high (the GPU found
a maximiser, not just a value), sigma^2 is the oracle's profiled sigma^2 at that h^2, and h^2
agrees with the oracle's to 1e-4 where the criterion is curved enough to fix it."""
import numpy as np
import pytest

import synth
from oracle import estimate as est

pytestmark = pytest.mark.gpu
RTOL = 1e-8


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


def _check(g, c, method, h_tol=1e-4):
    m = est.ML if method == "ml" else est.REML
    h2, s2, ll, ms = g.gwas_estimate(c.Phi, c.XL, c.Y, method=method)
    h2r, s2r, llr = est.estimate(c.Phi, c.XL, c.Y, m)
    for j in range(c.Y.shape[1]):
        assert abs(ll[j] - llr[j]) <= RTOL * abs(llr[j]), (j, ll[j], llr[j])
        crit, s2_at, _ = est.profile(c.Phi, c.XL, c.Y[:, j], h2[j], m)
        assert crit >= llr[j] - RTOL * abs(llr[j]), (j, h2[j], h2r[j])
        assert abs(s2[j] - s2_at) <= 1e-8 * s2_at, (j, s2[j], s2_at)
        assert 0.0 <= h2[j] <= est.H2_MAX
        if h_tol is not None:
            assert abs(h2[j] - h2r[j]) <= h_tol, (j, h2[j], h2r[j])
    assert ms[0] > 0 and ms[1] > 0
    return h2


@pytest.mark.parametrize("method", ["ml", "reml"])
@pytest.mark.parametrize("n,q,t", [(200, 3, 9), (97, 1, 5), (300, 7, 4)])
def test_estimate_matches_oracle(g, method, n, q, t):
    c = synth.small_problem(101 + n + q, n=n, q=q, m=1, t=t)
    _check(g, c, method)


def test_estimate_null_traits_reach_the_boundary(g):
    """Traits with no kinship component: the maximiser is often h^2 = 0 exactly (the grid's first
    point beats every interior point); both sides agree there too."""
    c = synth.small_problem(7, n=150, q=3, m=1, t=6, h2=np.zeros(6))
    h2 = _check(g, c, "ml")
    assert np.any(h2 < 1e-6)


def test_estimate_workload2_traits(g):
    """n = 1,000 individuals, the kinship and covariates of the many-trait workload, 4 traits."""
    c = synth.make_cohort(2, m=0, t=4, with_genotypes=False)
    for method in ("ml", "reml"):
        _check(g, c, method)


def test_estimate_identity_kinship_and_exact_fit(g):
    """Phi = I: the criterion is flat in h^2, sigma^2 is the OLS residual variance.  A trait in
    the span of X_L: NaN h^2 and criterion, sigma^2 = 0."""
    c = synth.small_problem(9, n=120, q=3, m=1, t=3)
    n = c.XL.shape[0]
    Y = c.Y.copy()
    Y[:, 2] = c.XL @ np.array([1.0, 0.5, -2.0])
    h2, s2, ll, _ = g.gwas_estimate(np.eye(n), c.XL, Y, method="ml")
    for j in range(2):
        rss = np.linalg.lstsq(c.XL, Y[:, j], rcond=None)[1][0]
        assert abs(s2[j] - rss / n) <= 1e-10 * rss / n
    assert np.isnan(h2[2]) and s2[2] == 0.0 and np.isnan(ll[2])


def test_estimate_near_exact_fit_is_finite(g):
    """A trait with R^2 = 1 - 1e-10 is above the exact-fit threshold (1e-12): a finite estimate,
    with Phi = I the OLS residual variance to the accuracy the small residual allows."""
    c = synth.small_problem(10, n=120, q=3, m=1, t=1)
    n = c.XL.shape[0]
    rs = np.random.default_rng(12)
    fit = c.XL @ np.array([1.0, 0.5, -2.0])
    e = rs.standard_normal(n)
    e -= c.XL @ np.linalg.lstsq(c.XL, e, rcond=None)[0]
    e *= np.sqrt(1e-10 * (fit @ fit) / (e @ e))
    h2, s2, ll, _ = g.gwas_estimate(np.eye(n), c.XL, (fit + e)[:, None], method="ml")
    assert np.isfinite(h2[0]) and np.isfinite(ll[0])
    assert abs(s2[0] - (e @ e) / n) <= 1e-4 * (e @ e) / n


def test_estimate_feeds_setup(g):
    """The estimates are valid gwas_setup parameters (h^2 < 1, sigma^2 > 0)."""
    c = synth.small_problem(12, n=128, q=3, m=64, t=3)
    h2, s2, _, _ = g.gwas_estimate(c.Phi, c.XL, c.Y, method="reml")
    h = g.gwas_setup(c.Phi, c.XL, c.Y, h2, s2, algo="eig", precision="fp64")
    g.gwas_destroy(h)
