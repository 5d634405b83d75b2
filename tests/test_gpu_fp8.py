"""Parity of the SPLIT_FP8 CHOL path with the FP64 oracle.

SPLIT_FP8 splits the augmented L_j^-1 into an FP16 hi piece and an E4M3 lo piece: the hi product
takes the centred genotypes in FP16 (kind::f16), the lo product the uncentred codes in E4M3
(kind::f8f6f4), both accumulating into one TMEM accumulator; the epilogue subtracts the
centring term the lo product misses (mu times each row's sum of lo), and each row group is
scaled by a power of two into FP16 range.  Tolerance 1e-4 in oracle.gls's error measure, as for
SPLIT_BF16.

Cases: n on every side of the 64-column K step (62, 63, 64, 97, 130, 256, 300, 520), ragged SNP
counts, q from 1 to 7, several traits (each its own scales), the workload-1 shape with every SNP
checked, the golden pedigree, genetic models (one and two columns), all output modes, no
intercept (no centring), sigma^2 far from 1 (the power-of-two scaling), singular SNPs, the
host-streaming ring, a badly conditioned trait (three BF16 pieces beside FP8 traits), and EIG,
which runs exactly as SPLIT_BF16.
"""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import run, max_errors

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


def _fp8_traits(g, c, algo="chol", precision="split_fp8"):
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision=precision)
    try:
        return g.gwas_fp8_traits(h), g.gwas_split_pieces(h)
    finally:
        g.gwas_destroy(h)


@pytest.mark.parametrize("n,q,m,t", [(256, 3, 1000, 1), (62, 1, 131, 1), (63, 2, 200, 1),
                                     (64, 3, 129, 2), (97, 1, 131, 1), (130, 7, 257, 1),
                                     (520, 2, 129, 3), (64, 3, 1, 1), (300, 5, 384, 1)])
def test_fp8_ragged(g, n, q, m, t):
    c = synth.small_problem(5 * n + q + m, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, nsing = run(g, c, "chol", "split_fp8")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)
    assert nsing == 0
    assert _fp8_traits(g, c) == (t, 2)


def test_fp8_golden_pedigree(g, golden_pedigree):
    gp = golden_pedigree
    for j in range(2):
        c = synth.Cohort(Phi=gp["Phi"], XL=gp["XL"], Y=gp["Y"][:, j:j + 1], h2=gp["h2"][j:j + 1],
                         s2=gp["s2"][j:j + 1], XR=gp["XR"], beta=None)
        B, W, _ = run(g, c, "chol", "split_fp8")
        eb, ew = max_errors(B, W, gp["B"][:, j:j + 1], gp["W"][:, j:j + 1], gp["Vd"][:, j:j + 1])
        assert eb < TOL and ew < TOL, (eb, ew)


def test_fp8_workload1_slice(g):
    """Workload 1's shape (n = 1000, h2 = 0.5) on 3,000 SNPs, every SNP checked."""
    c = synth.make_cohort(1, m=3000)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "chol", "split_fp8", packed=True)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


@pytest.mark.parametrize("s2", [1e-6, 1.0, 3e5])
def test_fp8_scales(g, s2):
    """sigma^2 far from 1 moves L^-1 by 1/sqrt(sigma^2): the power-of-two row scaling keeps the
    FP16 piece in range, and the estimates do not depend on sigma^2."""
    c = synth.small_problem(77, n=200, q=3, m=300, t=2)
    # the traits' residuals rescaled to the new sigma^2, so that they still follow the model
    resid = c.Y - c.XL @ c.beta
    c.Y = c.XL @ c.beta + resid * np.sqrt(s2 / c.s2)
    c.s2[:] = s2
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "chol", "split_fp8")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def test_fp8_no_intercept(g):
    """Without an intercept column the SNPs are not centred: the lo product's codes need no
    correction (mu = 0)."""
    c = synth.small_problem(78, n=180, q=3, m=260, t=1)
    rs = np.random.default_rng(5)
    c.XL[:, 0] = rs.standard_normal(c.n)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "chol", "split_fp8")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


@pytest.mark.parametrize("model", ["dominant", "recessive", "add_dom"])
@pytest.mark.parametrize("n,q,m,t", [(97, 1, 131, 1), (200, 3, 300, 2), (256, 7, 140, 1)])
def test_fp8_models(g, model, n, q, m, t):
    c = synth.small_problem(11 * n + q + m, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=model)
    B, W, _ = run(g, c, "chol", "split_fp8", model=model, packed=True)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def _unpack_upper(flat, p):
    V = np.empty(flat.shape[:-1] + (p, p))
    e = 0
    for r in range(p):
        for c in range(r, p):
            V[..., r, c] = V[..., c, r] = flat[..., e]
            e += 1
    return V


def test_fp8_output_modes_and_singular(g):
    c = synth.small_problem(79, n=250, q=3, m=400, t=1)
    c.XR[[0, 200]] = 1  # monomorphic: singular
    p = c.p
    Bref, Wref, Vref, Vfull = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, full_var=True)
    Bf, Wf, sf = run(g, c, "chol", "split_fp8")
    assert sf == 2
    eb, ew = max_errors(Bf, Wf, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)
    Bs, Ws, _ = run(g, c, "chol", "split_fp8", out_mode="snp")
    assert np.array_equal(Ws, Wf, equal_nan=True)
    assert np.array_equal(Bs[..., 0], Bf[..., p - 1], equal_nan=True)
    se_ref = np.sqrt(Vref[..., p - 1])
    ok = ~np.isnan(se_ref)
    assert np.array_equal(ok, ~np.isnan(Bs[..., 1]))
    assert np.max(np.abs(Bs[..., 1][ok] - se_ref[ok]) / se_ref[ok]) < TOL
    Bv, Wv, _ = run(g, c, "chol", "split_fp8", out_mode="var")
    assert np.array_equal(Bv[..., :p], Bf, equal_nan=True)
    V = _unpack_upper(Bv[..., p:], p)
    okm = np.ones(c.m, bool)
    okm[[0, 200]] = False
    assert np.all(np.isnan(V[~okm]))
    d = np.sqrt(np.diagonal(Vfull[okm], axis1=2, axis2=3))
    err = np.abs(V[okm] - Vfull[okm]) / (d[..., :, None] * d[..., None, :])
    assert np.max(err) < TOL, np.max(err)


def test_fp8_streamed_equals_device(g):
    c = synth.small_problem(80, n=300, q=3, m=1100, t=1)
    Bd, Wd, _ = run(g, c, "chol", "split_fp8")
    Bh, Wh, _ = run(g, c, "chol", "split_fp8", device=False, block_snps=256)
    assert np.array_equal(Bd, Bh, equal_nan=True) and np.array_equal(Wd, Wh, equal_nan=True)


def test_fp8_badly_conditioned_trait_takes_three_bf16_pieces(g):
    """A trait with h2 = 0.999 on a kinship of 200 SNPs for 500 individuals (kappa ~ 3000) is split
    into three BF16 pieces; its neighbour with h2 = 0.5 (kappa ~ 7) keeps the FP8 split."""
    rs = np.random.default_rng(12)
    n, q, t = 500, 3, 2
    Phi = synth.kinship(synth.kinship_factor(rs, n, n_snps=200))
    XL = synth.covariates(rs, n, q)
    h2 = np.array([0.999, 0.5])
    s2 = np.array([1.3, 0.7])
    Y = XL @ rs.standard_normal((q, t)) + rs.standard_normal((n, t))
    XR = synth.genotypes(rs, n, 300)
    c = synth.Cohort(Phi=Phi, XL=XL, Y=Y, h2=h2, s2=s2, XR=XR, beta=None)
    assert _fp8_traits(g, c) == (1, 3)
    Bref, Wref, Vref = gls.gls_grid(Phi, XL, XR, Y, h2, s2)
    B, W, _ = run(g, c, "chol", "split_fp8", packed=True)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def test_fp8_eig_runs_as_split_bf16(g):
    """EIG has no FP8 variant: SPLIT_FP8 scans it exactly as SPLIT_BF16 (same bits)."""
    c = synth.small_problem(81, n=200, q=3, m=300, t=9)
    B8, W8, _ = run(g, c, "eig", "split_fp8")
    Bb, Wb, _ = run(g, c, "eig", "split_bf16")
    assert np.array_equal(B8, Bb, equal_nan=True) and np.array_equal(W8, Wb, equal_nan=True)
    assert _fp8_traits(g, c, algo="eig") == (0, 2)
