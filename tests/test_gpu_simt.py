"""Parity of the plain CUDA-core paths (FP64 and FP32, CHOL and EIG) with the FP64 oracle.

The FP64 paths must match to 1e-6 in the error measure of oracle.gls (relative error, or error in
standard-error units where the coefficient is near zero); FP32 to 2e-3.  Sizes span several
64-wide tiles plus ragged tails; edge cases cover tiny n, p = 2 and p = 8, singular SNPs,
invalid genotypes, non-SPD covariances and collinear covariates.
"""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import run, max_errors

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-6, "fp32": 2e-3}


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


@pytest.mark.parametrize("algo", ["chol", "eig"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_golden_pedigree(g, golden_pedigree, algo, prec):
    gp = golden_pedigree
    c = synth.Cohort(Phi=gp["Phi"], XL=gp["XL"], Y=gp["Y"], h2=gp["h2"], s2=gp["s2"], XR=gp["XR"], beta=None)
    B, W, _ = run(g, c, algo, prec, f64=(prec == "fp64"))
    eb, ew = max_errors(B, W, gp["B"], gp["W"], gp["Vd"])
    tol = 1e-10 if prec == "fp64" else TOL[prec]
    assert eb < tol and ew < tol, (eb, ew)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chol_workload0_all_snps(g, prec):
    c = synth.make_cohort(0)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, nsing = run(g, c, "chol", prec, f64=(prec == "fp64"))
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL[prec] and ew < TOL[prec], (eb, ew)
    assert nsing == 0


@pytest.mark.parametrize("n,q,m,t", [(97, 1, 131, 1), (200, 3, 300, 3), (130, 7, 70, 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chol_ragged(g, n, q, m, t, prec):
    c = synth.small_problem(n + q + m, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "chol", prec, f64=(prec == "fp64"))
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL[prec] and ew < TOL[prec], (eb, ew)


@pytest.mark.parametrize("n,q,m,t", [(97, 1, 131, 5), (200, 3, 300, 37), (130, 7, 70, 17), (64, 2, 64, 16)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eig_ragged(g, n, q, m, t, prec):
    c = synth.small_problem(7 * n + q + m, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "eig", prec, f64=(prec == "fp64"))
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL[prec] and ew < TOL[prec], (eb, ew)


def test_eig_workload2_sampled(g):
    """Workload 2's shape (n=1000, t=1000) on a 2,000-SNP slice; oracle on sampled pairs."""
    c = synth.make_cohort(2, m=2000)
    B, W, _ = run(g, c, "eig", "fp64", f64=True)
    rs = np.random.default_rng(0)
    pairs = np.c_[rs.integers(0, c.m, 60), rs.integers(0, c.t, 60)]
    Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, pairs)
    eb, ew = max_errors(B[pairs[:, 0], pairs[:, 1]], W[pairs[:, 0], pairs[:, 1]], Bref, Wref, Vref)
    assert eb < 1e-6 and ew < 1e-6, (eb, ew)


@pytest.mark.parametrize("algo", ["chol", "eig"])
def test_streamed_host_buffers_match_device(g, algo):
    import torch
    c = synth.small_problem(11, n=150, q=3, m=517, t=3)
    Bd, Wd, _ = run(g, c, algo, "fp64", f64=True)
    Bh, Wh, _ = run(g, c, algo, "fp64", f64=True, device=False, block_snps=64)
    assert np.array_equal(Bd, Bh) and np.array_equal(Wd, Wh)
    # pinned host input, device output
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision="fp64", block_snps=100)
    try:
        xr = torch.from_numpy(c.XR).pin_memory()
        B = torch.zeros((c.m, c.t, c.p), dtype=torch.float64, device="cuda")
        W = torch.zeros((c.m, c.t), dtype=torch.float64, device="cuda")
        g.gwas_scan_f64(h, xr, B, W)
        torch.cuda.synchronize()
        assert np.array_equal(B.cpu().numpy(), Bd) and np.array_equal(W.cpu().numpy(), Wd)
    finally:
        g.gwas_destroy(h)


@pytest.mark.parametrize("algo", ["chol", "eig"])
def test_singular_snps_are_nan_and_counted(g, algo):
    c = synth.small_problem(12, n=80, q=2, m=40, t=2)
    XR = c.XR.copy()
    XR[[3, 17]] = 1
    B, W, nsing = run(g, c, algo, "fp64", XR=XR, f64=True)
    assert np.all(np.isnan(B[[3, 17]])) and np.all(np.isnan(W[[3, 17]]))
    mask = np.ones(c.m, bool); mask[[3, 17]] = False
    assert np.all(np.isfinite(B[mask]))
    assert nsing == 2 * c.t


def test_invalid_genotype_is_reported(g):
    import torch
    c = synth.small_problem(13, n=50, q=2, m=10, t=1)
    XR = c.XR.copy()
    XR[4, 7] = 3
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo="chol", precision="fp64", validate_genotypes=1)
    try:
        B = torch.zeros((c.m, 1, c.p), dtype=torch.float32, device="cuda")
        with pytest.raises(g.GwasError) as ei:
            g.gwas_scan(h, torch.from_numpy(XR).cuda(), B)
        assert ei.value.status == -6
        g.gwas_scan(h, torch.from_numpy(c.XR).cuda(), B)  # handle still usable after the error
    finally:
        g.gwas_destroy(h)


@pytest.mark.parametrize("algo", ["chol", "eig"])
def test_not_spd_is_reported(g, algo):
    n = 20
    Phi = -np.eye(n)
    XL = np.ones((n, 1))
    with pytest.raises(g.GwasError) as ei:
        g.gwas_setup(Phi, XL, np.zeros((n, 2)), [0.9, 0.9], [1.0, 1.0], algo=algo, precision="fp64")
    assert ei.value.status == -2


@pytest.mark.parametrize("algo", ["chol", "eig"])
def test_collinear_covariates_are_reported(g, algo):
    c = synth.small_problem(14, n=40, q=3, m=5, t=2)
    XL = c.XL.copy()
    XL[:, 2] = 2.0 * XL[:, 1]
    with pytest.raises(g.GwasError) as ei:
        g.gwas_setup(c.Phi, XL, c.Y, c.h2, c.s2, algo=algo, precision="fp64")
    assert ei.value.status == -8


def test_setup_timing_and_info(g):
    c = synth.small_problem(15, n=64, q=2, m=5, t=3)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, precision="fp64")
    try:
        assert g.gwas_setup_timing(h) > 0
        info = g.gwas_info(h)
        assert info == dict(n=64, q=2, t=3, p=3, p_r=1, algo=2, precision=0)
    finally:
        g.gwas_destroy(h)


def test_empty_scan_is_ok(g):
    import torch
    c = synth.small_problem(16, n=32, q=1, m=1, t=1)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, precision="fp64")
    try:
        B = torch.zeros((1, 1, 2), device="cuda")
        g.gwas_scan(h, torch.zeros((0, 32), dtype=torch.int8, device="cuda"), B, m=0)
    finally:
        g.gwas_destroy(h)
