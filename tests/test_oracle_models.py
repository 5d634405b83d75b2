"""Pins of the oracle's genetic models (CPU only).

Table 1 sets p, the width of X, by the covariates and "the genetic model assumed": a SNP
contributes a block X_R,i of p_R columns (here: additive x; dominant [x >= 1]; recessive [x = 2];
additive and dominance [x, x = 1]), and the test of the SNP is the joint Wald statistic of the
block, b_R^T Var(b)_RR^-1 b_R with p_R degrees of freedom.  Each pin ties the oracle to something
it does not compute itself: exact rational Gauss-Jordan on a design these tests build by hand,
the drop in the generalised residual sum of squares (the Wald statistic with a known covariance
equals it), ordinary least squares when h^2 = 0, the invariance of the joint test under a
reparametrisation of the block, and Algorithms 3 and 4 with a bordered p_R x p_R block.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import gls
from oracle.exact import gls_exact

# the designs, written out here independently of oracle.gls.GENETIC_MODELS
HAND = {
    "additive": lambda x: [x],
    "dominant": lambda x: [1 if x >= 1 else 0],
    "recessive": lambda x: [1 if x == 2 else 0],
    "add_dom": lambda x: [x, 1 if x == 1 else 0],
}


def _rational_problem(seed, n=7, q=2, m=3, t=2):
    r = np.random.default_rng(seed)
    A = r.integers(-2, 3, size=(n, n))
    Phi = [[Fraction(int((A @ A.T)[i, j]), 8) + (Fraction(1, 4) if i == j else 0) for j in range(n)]
           for i in range(n)]
    XL = [[Fraction(1)] + [Fraction(int(v), 4) for v in r.integers(-6, 7, size=q - 1)] for _ in range(n)]
    # every SNP carries all three genotypes, so that each model's block has full column rank
    XR = [[int(v) for v in r.permutation([0, 1, 2] + [int(v) for v in r.integers(0, 3, size=n - 3)])]
          for _ in range(m)]
    Y = [[Fraction(int(v), 3) for v in r.integers(-9, 10, size=t)] for _ in range(n)]
    h2 = [Fraction(int(v), 10) for v in r.integers(1, 9, size=t)]
    s2 = [Fraction(int(v), 4) for v in r.integers(1, 7, size=t)]
    return Phi, XL, XR, Y, h2, s2


def _f(M):
    return np.array([[float(v) for v in row] for row in M])


@pytest.mark.parametrize("model", list(HAND))
@pytest.mark.parametrize("seed", [0, 1])
def test_models_match_exact_rational(model, seed):
    Phi, XL, XR, Y, h2, s2 = _rational_problem(seed)
    n, q, m, t = len(Phi), len(XL[0]), len(XR), len(Y[0])
    p_r = len(HAND[model](0))
    B, W, Vd = gls.gls_grid(_f(Phi), _f(XL), np.array(XR, dtype=np.int8), _f(Y),
                            np.array([float(v) for v in h2]), np.array([float(v) for v in s2]),
                            model=model)
    assert B.shape == (m, t, q + p_r)
    for i in range(m):
        X = [list(XL[r]) + HAND[model](XR[i][r]) for r in range(n)]
        for j in range(t):
            b, V = gls_exact(Phi, X, [Y[r][j] for r in range(n)], h2[j], s2[j])
            # joint Wald statistic of the genetic block, by hand: b_R^T Var_RR^-1 b_R
            VR = _f([row[q:] for row in V[q:]])
            bR = np.array([float(v) for v in b[q:]])
            w = float(bR @ np.linalg.solve(VR, bR))
            bf = np.array([float(v) for v in b])
            assert np.max(np.abs(B[i, j] - bf) / np.maximum(np.abs(bf), 1e-300)) < 1e-11
            assert np.max(np.abs(Vd[i, j] - np.diag(_f(V))) / np.diag(_f(V))) < 1e-11
            assert abs(W[i, j] - w) <= 1e-11 * abs(w)


@pytest.mark.parametrize("model", list(HAND))
def test_wald_is_the_drop_in_generalised_rss(model):
    """With M known, the Wald statistic of the block equals r0^T M^-1 r0 - r1^T M^-1 r1, the
    residuals of the GLS fits without and with the block (here with M^-1 by a plain inverse)."""
    c = synth.small_problem(71, n=60, q=3, m=20, t=2)
    B, W, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=model)
    for j in range(c.t):
        Mi = np.linalg.inv(gls.form_M(c.Phi, c.h2[j], c.s2[j]))
        y = c.Y[:, j]

        def grss(X):
            b = np.linalg.solve(X.T @ Mi @ X, X.T @ Mi @ y)
            r = y - X @ b
            return r @ Mi @ r

        r0 = grss(c.XL)
        for i in range(c.m):
            cols = np.array([HAND[model](int(x)) for x in c.XR[i]], dtype=np.float64)
            X = np.hstack([c.XL, cols])
            if np.linalg.matrix_rank(X) < X.shape[1]:  # e.g. no homozygote for "recessive"
                assert np.isnan(W[i, j]) and np.all(np.isnan(B[i, j]))
                continue
            drop = r0 - grss(X)
            assert abs(W[i, j] - drop) <= 1e-8 * max(drop, 1.0), (i, j, W[i, j], drop)


@pytest.mark.parametrize("model", list(HAND))
def test_ols_when_h2_is_zero(model):
    """h^2 = 0: M = s2 I, so b is the least-squares fit (numpy.linalg.lstsq), Var = s2 (X^T X)^-1,
    and the Wald statistic is (RSS_without - RSS_with) / s2."""
    c = synth.small_problem(72, n=50, q=2, m=12, t=1, h2=0.0, s2=1.7)
    B, W, Vd = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=model)
    y = c.Y[:, 0]
    rss0 = np.linalg.lstsq(c.XL, y, rcond=None)[1][0]
    for i in range(c.m):
        X = np.hstack([c.XL, np.array([HAND[model](int(x)) for x in c.XR[i]], dtype=np.float64)])
        if np.linalg.matrix_rank(X) < X.shape[1]:
            assert np.isnan(W[i, 0]) and np.all(np.isnan(B[i, 0]))
            continue
        b, rss1 = np.linalg.lstsq(X, y, rcond=None)[:2]
        assert np.allclose(B[i, 0], b, rtol=1e-10, atol=1e-12)
        assert np.allclose(Vd[i, 0], 1.7 * np.diag(np.linalg.inv(X.T @ X)), rtol=1e-10)
        assert abs(W[i, 0] - (rss0 - rss1[0]) / 1.7) <= 1e-8 * max(W[i, 0], 1.0)


def test_joint_test_is_invariant_to_reparametrisation():
    """[x, x = 1] and the genotype indicators [x = 1, x = 2] span the same columns: the same fit,
    the same joint Wald statistic, and coefficients related by x = I1 + 2 I2, d = I1."""
    c = synth.small_problem(73, n=80, q=3, m=25, t=3)
    Ba, Wa, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model="add_dom")
    Bg, Wg, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=((0, 1, 0), (0, 0, 1)))
    # a SNP missing a genotype class is singular in both parametrisations
    assert np.array_equal(np.isnan(Wa), np.isnan(Wg)) and not np.all(np.isnan(Wa))
    assert np.allclose(Wa, Wg, rtol=1e-9, equal_nan=True)
    q = c.q
    assert np.allclose(Bg[..., q], Ba[..., q] + Ba[..., q + 1], rtol=1e-9, atol=1e-12, equal_nan=True)
    assert np.allclose(Bg[..., q + 1], 2 * Ba[..., q], rtol=1e-9, atol=1e-12, equal_nan=True)
    assert np.allclose(Bg[..., :q], Ba[..., :q], rtol=1e-9, atol=1e-12, equal_nan=True)


def test_degenerate_blocks_are_nan():
    """A SNP with no heterozygote has an all-zero dominance column (add_dom singular); one with no
    non-carrier makes the dominant column the intercept, and x + d = 2 under add_dom (both
    singular): NaN, not an error."""
    c = synth.small_problem(74, n=40, q=2, m=4, t=1)
    XR = c.XR.copy()
    XR[1] = np.where(XR[1] == 1, 2, XR[1])   # no heterozygote
    XR[2] = np.maximum(XR[2], 1)             # everyone carries
    XR[2, :5] = 2
    Bd, Wd, _ = gls.gls_grid(c.Phi, c.XL, XR, c.Y, c.h2, c.s2, model="add_dom")
    assert np.all(np.isnan(Bd[[1, 2]])) and np.all(np.isnan(Wd[[1, 2]]))
    assert np.all(np.isfinite(Bd[[0, 3]]))
    Bm, Wm, _ = gls.gls_grid(c.Phi, c.XL, XR, c.Y, c.h2, c.s2, model="dominant")
    assert np.all(np.isnan(Bm[2])) and np.isnan(Wm[2, 0])


@pytest.mark.parametrize("model", ["add_dom", "recessive"])
def test_sequences_match_the_definition(model):
    """Algorithm 3 and Algorithm 4 with the bordered p_R x p_R block equal Eq. "probDef"."""
    c = synth.small_problem(75, n=70, q=3, m=30, t=4)
    B, W, Vd = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=model)
    Be, We, Vde = gls.eig_sequence(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=model)
    assert max(gls.max_rel_errors(Be, We, B, W, Vd)) < 1e-10
    for j in range(c.t):
        Bc, Wc, _ = gls.chol_sequence(c.Phi, c.XL, c.XR, c.Y[:, j], c.h2[j], c.s2[j], model=model)
        assert max(gls.max_rel_errors(Bc, Wc, B[:, j], W[:, j], Vd[:, j])) < 1e-10


def test_additive_model_is_the_single_snp_column():
    """The default model reproduces the one-column results (the same W as b^2 / Var)."""
    c = synth.small_problem(76, n=50, q=3, m=20, t=3)
    B, W, Vd = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model="additive")
    assert np.allclose(W, gls.wald_from(B, Vd), rtol=1e-12)


@pytest.mark.parametrize("mistake", ["diag_only_wald", "dom_as_recessive", "block_transposed"])
def test_planted_model_mistakes_are_caught(mistake, monkeypatch):
    """A plausible mistake in the model code of the oracle fails one of the pins above."""
    if mistake == "diag_only_wald":
        def bad(b, Var, p_r):
            return np.sum(b[..., -p_r:] ** 2 / np.diagonal(Var, axis1=-2, axis2=-1)[..., -p_r:], axis=-1)
        monkeypatch.setattr(gls, "wald_block", bad)
        with pytest.raises(AssertionError):
            test_wald_is_the_drop_in_generalised_rss("add_dom")
    elif mistake == "dom_as_recessive":
        monkeypatch.setitem(gls.GENETIC_MODELS, "add_dom", ((0, 1, 2), (0, 0, 1)))
        with pytest.raises(AssertionError):
            test_models_match_exact_rational("add_dom", 0)
    else:
        orig = gls.genetic_columns

        def swapped(XR_rows, model="additive"):
            return orig(XR_rows, model)[..., ::-1]
        monkeypatch.setattr(gls, "genetic_columns", swapped)
        with pytest.raises(AssertionError):
            test_models_match_exact_rational("add_dom", 1)
