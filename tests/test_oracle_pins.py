"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties the oracle to something it does not compute itself: exact rational arithmetic,
closed forms (exact recovery, OLS), invariances of the GLS (Eq. "GLS"), agreement of the two
independent formulations (Algorithms 1/3 vs Algorithms 2/4), and the null distribution of the
Wald statistic.  A dropped term, wrong sign, wrong index or transposed operand anywhere in
oracle/gls.py breaks at least one of them (test_planted_mistakes_are_caught checks a few).
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.stats

import synth
from oracle import gls
from oracle.exact import gls_exact, grid_exact


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


# --------------------------------------------------------------------------- exact arithmetic

def test_golden_pedigree_definition(golden_pedigree):
    g = golden_pedigree
    B, W, Vd = gls.gls_grid(g["Phi"], g["XL"], g["XR"], g["Y"], g["h2"], g["s2"])
    assert _rel(B, g["B"]) < 1e-12
    assert _rel(Vd, g["Vd"]) < 1e-12
    assert _rel(W, g["W"]) < 1e-12


def test_golden_pedigree_sequences(golden_pedigree):
    g = golden_pedigree
    Be, We, Vde = gls.eig_sequence(g["Phi"], g["XL"], g["XR"], g["Y"], g["h2"], g["s2"])
    assert _rel(Be, g["B"]) < 1e-11 and _rel(We, g["W"]) < 1e-11 and _rel(Vde, g["Vd"]) < 1e-11
    for j in range(g["Y"].shape[1]):
        Bc, Wc, Vdc = gls.chol_sequence(g["Phi"], g["XL"], g["XR"], g["Y"][:, j], g["h2"][j], g["s2"][j])
        assert _rel(Bc, g["B"][:, j]) < 1e-12 and _rel(Wc, g["W"][:, j]) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_rational_problems(seed):
    r = np.random.default_rng(seed)
    n, p = 7, 3
    # Phi = A A^T / 8 + I/4 with small-integer A: rational SPD
    A = r.integers(-2, 3, size=(n, n))
    Phi = [[Fraction(int((A @ A.T)[i, j]), 8) + (Fraction(1, 4) if i == j else 0) for j in range(n)] for i in range(n)]
    X = [[Fraction(1)] + [Fraction(int(v), 4) for v in r.integers(-6, 7, size=p - 2)] + [Fraction(int(r.integers(0, 3)))] for _ in range(n)]
    y = [Fraction(int(v), 3) for v in r.integers(-9, 10, size=n)]
    h2, s2 = Fraction(int(r.integers(1, 9)), 10), Fraction(int(r.integers(1, 7)), 4)
    b_ex, V_ex = gls_exact(Phi, X, y, h2, s2)
    f = lambda M: np.array([[float(v) for v in row] for row in M])
    Phif, Xf, yf = f(Phi), f(X), np.array([float(v) for v in y])
    b_ex = np.array([float(v) for v in b_ex]); V_ex = f(V_ex)
    for fn in (gls.gls_chol, gls.gls_eig):
        b, V = fn(Phif, Xf, yf, float(h2), float(s2))
        assert _rel(b, b_ex) < 1e-11, fn.__name__
        assert _rel(V, V_ex) < 1e-11, fn.__name__


def test_form_M_entries():
    Phi = np.array([[1.0, 0.5], [0.5, 1.0]])
    M = gls.form_M(Phi, 0.25, 2.0)
    # 2 * (0.25 * Phi + 0.75 I)
    assert np.array_equal(M, np.array([[2.0, 0.25], [0.25, 2.0]]))


# --------------------------------------------------------------------------- closed forms

def _problem(seed=3, n=40, q=3, m=25, t=3, **kw):
    return synth.small_problem(seed, n=n, q=q, m=m, t=t, **kw)


def test_exact_recovery_null_model():
    c = _problem()
    beta = np.array([[1.5, -0.5, 2.0], [0.25, 1.0, -3.0], [-2.0, 0.0, 0.5]])
    Y = c.XL @ beta
    B, W, _ = gls.gls_grid(c.Phi, c.XL, c.XR, Y, c.h2, c.s2)
    assert np.max(np.abs(B[:, :, :3] - beta.T[None])) < 1e-9
    assert np.max(np.abs(B[:, :, 3])) < 1e-9
    assert np.max(W) < 1e-15


def test_exact_recovery_snp_effect():
    c = _problem()
    i0, gamma = 7, -1.25
    beta = np.array([0.5, -1.0, 2.0])
    y = c.XL @ beta + gamma * c.XR[i0].astype(float)
    B, _, _ = gls.gls_grid(c.Phi, c.XL, c.XR, y[:, None], c.h2[:1], c.s2[:1], snps=[i0])
    assert np.max(np.abs(B[0, 0] - np.r_[beta, gamma])) < 1e-9


def test_ols_when_h2_is_zero():
    c = _problem(t=2, h2=0.0, s2=[1.7, 0.6])
    B, W, Vd = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    for i in range(c.m):
        X = np.c_[c.XL, c.XR[i].astype(float)]
        XtXi = np.linalg.inv(X.T @ X)
        for j in range(c.t):
            b = np.linalg.lstsq(X, c.Y[:, j], rcond=None)[0]
            assert np.max(np.abs(B[i, j] - b)) < 1e-10 * max(1.0, np.max(np.abs(b)))
            assert _rel(Vd[i, j], c.s2[j] * np.diag(XtXi)) < 1e-10


def test_full_var_matches_exact_rational_and_ols():
    """The whole Var(b) = (X^T M^-1 X)^-1 of every pair (Eq. "probDef"): equal to Gauss-Jordan in
    rational arithmetic (oracle.exact) on a tiny problem, and to sigma^2 (X^T X)^-1 when h2 = 0."""
    from fractions import Fraction
    from oracle import exact
    rs = np.random.default_rng(5)
    n, q, m, t = 7, 2, 3, 2
    A = rs.integers(-3, 4, size=(n, n))
    Phi = [[Fraction(int(v), 9) for v in row] for row in (A @ A.T + 9 * np.eye(n, dtype=int))]
    XL = [[1, int(rs.integers(-2, 3))] for _ in range(n)]
    XR = [[int(v) for v in rs.integers(0, 3, size=n)] for _ in range(m)]
    Y = [[int(v) for v in rs.integers(-5, 6, size=t)] for _ in range(n)]
    h2, s2 = [Fraction(1, 3), Fraction(3, 5)], [Fraction(2), Fraction(1, 2)]
    _, Ve, _ = exact.grid_exact(Phi, XL, XR, Y, h2, s2)
    f = lambda x: np.array(x, dtype=np.float64)
    B, W, Vd, V = gls.gls_grid(f([[float(v) for v in r] for r in Phi]), f(XL), np.array(XR, np.int8),
                               f(Y), f([float(v) for v in h2]), f([float(v) for v in s2]),
                               full_var=True)
    for i in range(m):
        for j in range(t):
            ref = np.array([[float(v) for v in row] for row in Ve[i][j]])
            assert np.max(np.abs(V[i, j] - ref)) <= 1e-12 * np.max(np.abs(ref))
            assert np.allclose(np.diagonal(V[i, j]), Vd[i, j], rtol=0, atol=0)
    c = _problem(t=2, h2=0.0, s2=[1.7, 0.6])
    _, _, _, V = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, full_var=True)
    for i in range(c.m):
        X = np.c_[c.XL, c.XR[i].astype(float)]
        XtXi = np.linalg.inv(X.T @ X)
        for j in range(c.t):
            assert np.max(np.abs(V[i, j] - c.s2[j] * XtXi)) <= 1e-10 * np.max(np.abs(c.s2[j] * XtXi))


def test_ols_when_phi_is_identity():
    c = _problem(t=2)
    I = np.eye(c.n)
    B, _, _ = gls.gls_grid(I, c.XL, c.XR, c.Y, c.h2, c.s2)
    for i in range(0, c.m, 5):
        X = np.c_[c.XL, c.XR[i].astype(float)]
        for j in range(c.t):
            b = np.linalg.lstsq(X, c.Y[:, j], rcond=None)[0]
            assert np.max(np.abs(B[i, j] - b)) < 1e-10 * max(1.0, np.max(np.abs(b)))


# --------------------------------------------------------------------------- two formulations

def test_definition_chol_sequence_eig_sequence_agree():
    c = _problem(n=64, m=30, t=4)
    B, W, Vd = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    Be, We, Vde = gls.eig_sequence(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    assert np.max(gls.rel_err_b(Be, B, Vd)) < 1e-10
    assert np.max(gls.rel_err_wald(We, W)) < 1e-10
    for j in range(c.t):
        Bc, Wc, _ = gls.chol_sequence(c.Phi, c.XL, c.XR, c.Y[:, j], c.h2[j], c.s2[j])
        assert np.max(gls.rel_err_b(Bc, B[:, j], Vd[:, j])) < 1e-10
        assert np.max(gls.rel_err_wald(Wc, W[:, j])) < 1e-10


def test_single_gls_chol_equals_eig():
    c = _problem(n=50, m=3, t=1)
    X = np.c_[c.XL, c.XR[1].astype(float)]
    b1, V1 = gls.gls_chol(c.Phi, X, c.Y[:, 0], c.h2[0], c.s2[0])
    b2, V2 = gls.gls_eig(c.Phi, X, c.Y[:, 0], c.h2[0], c.s2[0])
    assert _rel(b2, b1) < 1e-10 and _rel(V2, V1) < 1e-10


# --------------------------------------------------------------------------- invariances

def test_sigma2_scaling():
    c = _problem(t=1)
    B1, W1, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B2, W2, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, 3.0 * c.s2)
    assert _rel(B2, B1) < 1e-10
    assert _rel(W2, W1 / 3.0) < 1e-10


def test_allele_coding_flip():
    c = _problem(t=2)
    B1, W1, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B2, W2, _ = gls.gls_grid(c.Phi, c.XL, (2 - c.XR).astype(np.int8), c.Y, c.h2, c.s2)
    assert np.max(np.abs(B2[..., 3] + B1[..., 3])) < 1e-10
    assert np.max(np.abs(B2[..., 0] - (B1[..., 0] + 2 * B1[..., 3]))) < 1e-9
    assert _rel(W2, W1) < 1e-8


def test_permutation_of_individuals():
    c = _problem(t=2)
    perm = np.random.default_rng(5).permutation(c.n)
    B1, W1, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B2, W2, _ = gls.gls_grid(c.Phi[np.ix_(perm, perm)], c.XL[perm], c.XR[:, perm], c.Y[perm], c.h2, c.s2)
    assert np.max(np.abs(B2 - B1)) < 1e-9 and _rel(W2, W1) < 1e-8


def test_covariate_scaling():
    c = _problem(t=1)
    XL2 = c.XL.copy()
    XL2[:, 1] *= 4.0
    B1, W1, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B2, W2, _ = gls.gls_grid(c.Phi, XL2, c.XR, c.Y, c.h2, c.s2)
    assert _rel(B2[..., 1], B1[..., 1] / 4.0) < 1e-9
    assert np.max(np.abs(B2[..., 3] - B1[..., 3])) < 1e-10 and _rel(W2, W1) < 1e-8


def test_eigenvector_signs_do_not_matter():
    c = _problem(t=3)
    w, Z = np.linalg.eigh(c.Phi)
    flip = np.where(np.random.default_rng(9).random(c.n) < 0.5, -1.0, 1.0)
    B1, W1, _ = gls.eig_sequence(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, Z=Z, w=w)
    B2, W2, _ = gls.eig_sequence(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, Z=Z * flip, w=w)
    assert np.max(np.abs(B2 - B1)) < 1e-10 and _rel(W2, W1) < 1e-8


# --------------------------------------------------------------------------- statistics, edge cases

def test_null_wald_is_chi2_1():
    c = synth.make_cohort(0, m=4000)
    B, W, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    w = W[:, 0]
    assert abs(w.mean() - 1.0) < 0.1
    assert scipy.stats.kstest(w, scipy.stats.chi2(1).cdf).pvalue > 1e-3


def test_monomorphic_snp_is_nan():
    c = _problem(t=2)
    XR = c.XR.copy()
    XR[4] = 1  # constant column, collinear with the intercept
    B, W, Vd = gls.gls_grid(c.Phi, c.XL, XR, c.Y, c.h2, c.s2)
    assert np.all(np.isnan(B[4])) and np.all(np.isnan(W[4]))
    assert np.all(np.isfinite(B[np.arange(c.m) != 4]))


def test_pairs_match_grid():
    c = _problem(t=5)
    pairs = np.array([[3, 1], [0, 4], [3, 4], [24, 0], [11, 1]])
    B, W, Vd = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    Bp, Wp, Vp = gls.gls_pairs(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, pairs)
    assert np.array_equal(Bp, B[pairs[:, 0], pairs[:, 1]])
    assert np.array_equal(Wp, W[pairs[:, 0], pairs[:, 1]])


# --------------------------------------------------------------------------- the pins have teeth

MUTATIONS = {
    "sign of (1-h2)": lambda Phi, h2, s2: s2 * (h2 * Phi + (1.0 + h2) * np.eye(Phi.shape[0])),
    "h2 and 1-h2 swapped": lambda Phi, h2, s2: s2 * ((1.0 - h2) * Phi + h2 * np.eye(Phi.shape[0])),
    "dropped sigma2": lambda Phi, h2, s2: (h2 * Phi + (1.0 - h2) * np.eye(Phi.shape[0])),
    "off-diagonal kinship halved": lambda Phi, h2, s2: s2 * (
        h2 * 0.5 * (Phi + np.diag(np.diag(Phi))) + (1.0 - h2) * np.eye(Phi.shape[0])),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistakes_are_caught(name, golden_pedigree, monkeypatch):
    """Plant a mistake in the oracle (CPU only) and check that a pin rejects it."""
    monkeypatch.setattr(gls, "form_M", MUTATIONS[name])
    failed = []
    for pin in (test_golden_pedigree_definition, ):
        try:
            pin(golden_pedigree)
        except AssertionError:
            failed.append(pin.__name__)
    try:
        test_sigma2_scaling()
    except AssertionError:
        failed.append("sigma2")
    assert failed, f"mutation {name!r} survived every pin"


def test_error_measures_on_hand_computed_values():
    """The error measures every parity check uses, against values worked out by hand: a large
    coefficient is compared relatively, one near zero in units of its standard error sqrt(Var)
    (not Var), and the Wald statistic relatively above 1 and absolutely below."""
    b = np.array([[1.0, 0.002]])
    b_ref = np.array([[1.1, 0.0]])
    vd_ref = np.array([[0.04, 1e-4]])       # standard errors 0.2 and 0.01
    eb = gls.rel_err_b(b, b_ref, vd_ref)
    assert np.allclose(eb, [[0.1 / 1.1, 0.002 / 0.01]], rtol=1e-12, atol=0)
    ew = gls.rel_err_wald(np.array([4.0, 0.3]), np.array([5.0, 0.1]))
    assert np.allclose(ew, [1.0 / 5.0, 0.2 / 1.0], rtol=1e-12, atol=0)
    assert gls.max_rel_errors(b, np.array([4.0]), b_ref, np.array([5.0]), vd_ref) == \
        pytest.approx((0.2, 0.2), rel=1e-12)


def test_max_rel_errors_rejects_nan_where_the_reference_is_finite():
    """A pair left unwritten in a NaN-filled output buffer (or written as a spurious NaN) is an
    infinite error; NaN on both sides (a singular GLS) is left out of the maxima."""
    rs = np.random.default_rng(0)
    b_ref = rs.standard_normal((6, 3, 4))
    w_ref = rs.random((6, 3)) * 5
    vd_ref = rs.random((6, 3, 4)) + 0.1
    b, w = b_ref * (1 + 1e-6), w_ref * (1 + 1e-6)
    eb, ew = gls.max_rel_errors(b, w, b_ref, w_ref, vd_ref)
    assert eb < 2e-6 and ew < 2e-6
    planted = b.copy()
    planted[4, 1] = np.nan                      # one pair overwritten by NaN on the output side
    assert gls.max_rel_errors(planted, w, b_ref, w_ref, vd_ref) == (np.inf, np.inf)
    wp = w.copy()
    wp[2, 2] = np.nan
    assert gls.max_rel_errors(b, wp, b_ref, w_ref, vd_ref) == (np.inf, np.inf)
    # a pair the reference calls singular must be NaN in the output too
    b_ref2, w_ref2 = b_ref.copy(), w_ref.copy()
    b_ref2[0, 0] = np.nan
    w_ref2[0, 0] = np.nan
    assert gls.max_rel_errors(b, w, b_ref2, w_ref2, vd_ref) == (np.inf, np.inf)
    b2, w2 = b.copy(), w.copy()
    b2[0, 0] = np.nan
    w2[0, 0] = np.nan
    eb, ew = gls.max_rel_errors(b2, w2, b_ref2, w_ref2, vd_ref)
    assert eb < 2e-6 and ew < 2e-6
