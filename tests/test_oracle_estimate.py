"""Pins of the step-1 oracle (oracle/estimate.py) against what probability and linear algebra fix
independently of it: the multivariate normal density (scipy.stats), the density of REML error
contrasts built from an explicit null-space basis, ordinary least squares when Phi = I, brute
force over a dense grid, and invariances of the model.  A planted mistake in the criterion is
caught by one of them."""
import numpy as np
import pytest
from scipy.linalg import null_space
from scipy.stats import multivariate_normal

import synth
from oracle import estimate as est


def _problem(seed=3, n=60, q=3, t=3):
    return synth.small_problem(seed, n=n, q=q, m=1, t=t)


def _ml_matches_density(profile_fn, c, h):
    """ML criterion at h == the N(X_L beta, s2 H(h)) log-density of y at the profiled beta, s2."""
    y = c.Y[:, 0]
    crit, s2, beta = profile_fn(c.Phi, c.XL, y, h, est.ML)
    ref = multivariate_normal.logpdf(y, mean=c.XL @ beta, cov=s2 * est.kinship_cov(c.Phi, h))
    return abs(crit - ref) <= 1e-9 * abs(ref)


def _reml_matches_contrasts(profile_fn, c, h):
    """REML criterion at h == log-density of the error contrasts A^T y, A an orthonormal basis of
    the null space of X_L^T, at the profiled s2 (Harville's restricted likelihood)."""
    y = c.Y[:, 0]
    crit, s2, _ = profile_fn(c.Phi, c.XL, y, h, est.REML)
    A = null_space(c.XL.T)
    cov = s2 * A.T @ est.kinship_cov(c.Phi, h) @ A
    ref = multivariate_normal.logpdf(A.T @ y, mean=np.zeros(A.shape[1]), cov=cov)
    return abs(crit - ref) <= 1e-9 * abs(ref)


def _profiled_values_are_maximal(profile_fn, c, h):
    """At fixed h, no other (beta, s2) gives a higher ML density than the profiled ones."""
    y = c.Y[:, 0]
    crit, s2, beta = profile_fn(c.Phi, c.XL, y, h, est.ML)
    H = est.kinship_cov(c.Phi, h)
    base = multivariate_normal.logpdf(y, mean=c.XL @ beta, cov=s2 * H)
    rs = np.random.default_rng(0)
    for _ in range(6):
        b2 = beta + 1e-3 * rs.standard_normal(beta.shape)
        if multivariate_normal.logpdf(y, mean=c.XL @ b2, cov=s2 * H) > base:
            return False
    for f in (0.99, 1.01):
        if multivariate_normal.logpdf(y, mean=c.XL @ beta, cov=f * s2 * H) > base:
            return False
    return True


PINS = [_ml_matches_density, _reml_matches_contrasts, _profiled_values_are_maximal]


@pytest.mark.parametrize("h", [0.0, 0.3, 0.77, est.H2_MAX])
def test_criteria_match_gaussian_densities(h):
    c = _problem()
    for pin in PINS:
        assert pin(est.profile, c, h), (pin.__name__, h)


@pytest.mark.parametrize("method", [est.ML, est.REML])
def test_estimate_is_the_maximum_over_a_dense_grid(method):
    """Brute force: the criterion at the estimate is at least its value at 2001 points."""
    c = _problem(seed=11, n=50, t=2)
    h2, s2, ll = est.estimate(c.Phi, c.XL, c.Y, method)
    for j in range(c.Y.shape[1]):
        dense = [est.profile(c.Phi, c.XL, c.Y[:, j], h, method)[0]
                 for h in np.linspace(0.0, est.H2_MAX, 2001)]
        assert ll[j] >= max(dense) - 1e-9 * abs(ll[j])
        assert 0.0 <= h2[j] <= est.H2_MAX
        crit, s2_j, _ = est.profile(c.Phi, c.XL, c.Y[:, j], h2[j], method)
        assert np.isclose(crit, ll[j], rtol=1e-12) and np.isclose(s2_j, s2[j], rtol=1e-12)


def test_identity_kinship_is_ols():
    """Phi = I makes H(h) = I for every h: the criterion is flat in h and sigma^2 is the OLS
    residual variance (RSS / n for ML, RSS / (n - q) for REML; numpy.linalg.lstsq)."""
    c = _problem(seed=5, n=80)
    n, q = c.XL.shape
    Phi = np.eye(n)
    for j in range(c.Y.shape[1]):
        y = c.Y[:, j]
        rss = np.linalg.lstsq(c.XL, y, rcond=None)[1][0]
        vals = [est.profile(Phi, c.XL, y, h, est.ML)[0] for h in (0.0, 0.4, 0.9)]
        assert np.allclose(vals, vals[0], rtol=1e-12)
        _, s2, _ = est.estimate(Phi, c.XL, y[:, None], est.ML)
        assert np.isclose(s2[0], rss / n, rtol=1e-10)
        _, s2r, _ = est.estimate(Phi, c.XL, y[:, None], est.REML)
        assert np.isclose(s2r[0], rss / (n - q), rtol=1e-10)


def test_scale_and_shift_invariance():
    """y -> c y scales sigma^2 by c^2 and leaves h^2; y -> y + X_L g leaves both."""
    c = _problem(seed=8, n=70, t=2)
    rs = np.random.default_rng(1)
    for method in (est.ML, est.REML):
        h2, s2, _ = est.estimate(c.Phi, c.XL, c.Y, method)
        h2c, s2c, _ = est.estimate(c.Phi, c.XL, 3.0 * c.Y, method)
        h2s, s2s, _ = est.estimate(c.Phi, c.XL, c.Y + c.XL @ rs.standard_normal((c.XL.shape[1], 2)),
                                   method)
        assert np.allclose(h2c, h2, atol=1e-7) and np.allclose(s2c, 9.0 * s2, rtol=1e-6)
        assert np.allclose(h2s, h2, atol=1e-7) and np.allclose(s2s, s2, rtol=1e-6)


def test_exact_fit_is_nan():
    """A trait lying in the span of X_L has no finite estimate."""
    c = _problem(seed=2, n=40, t=1)
    y = c.XL @ np.array([1.0, -2.0, 0.5])
    h2, s2, ll = est.estimate(c.Phi, c.XL, y[:, None])
    assert np.isnan(h2[0]) and s2[0] == 0.0 and np.isnan(ll[0])


def test_near_exact_fit_is_finite():
    """The exact-fit threshold (r^T H^-1 r <= 1e-12 y^T H^-1 y) only catches traits X_L fits to
    rounding: a trait with R^2 = 1 - 1e-10 (residual fraction 1e-10, two orders above the
    threshold) still gets a finite estimate -- with Phi = I the OLS residual variance, RSS / n."""
    c = _problem(seed=4, n=40, t=1)
    n = c.XL.shape[0]
    rs = np.random.default_rng(11)
    fit = c.XL @ np.array([1.0, -2.0, 0.5])
    e = rs.standard_normal(n)
    e -= c.XL @ np.linalg.lstsq(c.XL, e, rcond=None)[0]  # residual orthogonal to X_L
    e *= np.sqrt(1e-10 * (fit @ fit) / (e @ e))
    y = fit + e
    frac = float(e @ e) / float(y @ y)
    assert 0.9e-10 < frac < 1.1e-10
    for method in (est.ML, est.REML):
        h2, s2, ll = est.estimate(np.eye(n), c.XL, y[:, None], method)
        assert np.isfinite(h2[0]) and np.isfinite(ll[0])
        dof = n if method == est.ML else n - c.XL.shape[1]
        assert abs(s2[0] - (e @ e) / dof) <= 1e-6 * (e @ e) / dof
    h2, s2, ll = est.estimate(c.Phi, c.XL, y[:, None], est.REML)
    assert np.isfinite(h2[0]) and s2[0] > 0 and np.isfinite(ll[0])


def _mutant(kind):
    """The oracle's criterion with one plausible mistake planted."""
    def profile(Phi, XL, y, h, method=est.ML):
        n, q = XL.shape
        Hm = {"h swapped": est.kinship_cov(Phi, 1.0 - h)}.get(kind, est.kinship_cov(Phi, h))
        L = np.linalg.cholesky(Hm)
        Xw = np.linalg.solve(L, XL)
        yw = np.linalg.solve(L, y)
        S = Xw.T @ Xw
        beta = np.linalg.solve(S, Xw.T @ yw)
        r = yw - Xw @ beta
        Q = float(r @ r)
        ldH = 2 * np.sum(np.log(np.diag(L))) if kind != "log|H| dropped" else 0.0
        if method == est.ML:
            s2 = Q / (n - q if kind == "ML divides by n - q" else n)
            return -0.5 * (n * np.log(2 * np.pi * s2) + ldH + n), s2, beta
        s2 = Q / (n - q)
        ldS = np.linalg.slogdet(S)[1] if kind != "REML log|X^T H^-1 X| dropped" else 0.0
        ldX = np.linalg.slogdet(XL.T @ XL)[1]
        return -0.5 * ((n - q) * np.log(2 * np.pi * s2) + ldH + ldS - ldX + (n - q)), s2, beta
    return profile


@pytest.mark.parametrize("kind", ["h swapped", "log|H| dropped", "ML divides by n - q",
                                  "REML log|X^T H^-1 X| dropped"])
def test_planted_mistakes_are_caught(kind):
    c = _problem(seed=4)
    assert all(pin(_mutant("none"), c, 0.3) for pin in PINS)  # the mutant frame itself is right
    assert not all(pin(_mutant(kind), c, 0.3) for pin in PINS), kind
