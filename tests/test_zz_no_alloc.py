"""gwas_scan_static: the scan entry point that allocates no device memory (its scratch is a
fixed 16 MiB device array in the library).  It exists for callers that cannot have a library
call cudaMalloc in the middle of their work: latency-critical loops, which cudaMalloc's implicit
device synchronisation would stall, and applications whose device memory belongs to their own
allocator or budget.

Checked through the C ABI, on two calls in a row (the second finds the first call's data in the
shared array), against the FP64 oracle (coefficients, Wald statistics and, in the VAR output
mode, the whole Var(b)) and against gwas_scan on the same handle, in the error measure and
tolerances of every other CUDA-core parity test; also its rejection of blocks larger than the
array and of other handles, and its genotype check.

This file is collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import max_errors

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-6, "fp32": 2e-3}


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


def _unpack_upper(flat, p):
    """(..., p(p+1)/2) packed upper triangle, row by row -> (..., p, p) symmetric."""
    V = np.empty(flat.shape[:-1] + (p, p))
    e = 0
    for r in range(p):
        for c in range(r, p):
            V[..., r, c] = V[..., c, r] = flat[..., e]
            e += 1
    return V


def _static(g, h, xr, m, B, W):
    """One gwas_scan_static call through the C ABI (device pointers, the current stream)."""
    import torch
    st = g.lib.gwas_scan_static(h, xr.data_ptr(), m, B.data_ptr(),
                                W.data_ptr() if W is not None else None,
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("prec,out_mode", [("fp64", "full"), ("fp32", "full"), ("fp64", "var")])
def test_static_scan_matches_oracle_and_gwas_scan(g, prec, out_mode):
    import torch
    c = synth.small_problem(41, n=300, q=3, m=500, t=23)
    XR = c.XR.copy()
    XR[257] = 1  # monomorphic: a singular pair for every trait, NaN on both sides
    p = c.p
    Bref, Wref, Vref, Vfull = gls.gls_grid(c.Phi, c.XL, XR, c.Y, c.h2, c.s2, full_var=True)
    pw = p + p * (p + 1) // 2 if out_mode == "var" else p
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo="eig", precision=prec, out_mode=out_mode)
    try:
        xr = torch.from_numpy(XR).cuda()
        # the existing entry point on the same handle
        B0 = torch.full((c.m, c.t, pw), float("nan"), device="cuda")
        W0 = torch.full((c.m, c.t), float("nan"), device="cuda")
        g.gwas_scan(h, xr, B0, W0)
        torch.cuda.synchronize()
        B0 = B0.cpu().numpy().astype(np.float64)
        W0 = W0.cpu().numpy().astype(np.float64)
        for call in range(2):
            B1 = torch.full((c.m, c.t, pw), float("nan"), device="cuda")
            W1 = torch.full((c.m, c.t), float("nan"), device="cuda")
            assert _static(g, h, xr, c.m, B1, W1) == 0, g.gwas_last_error()
            B1 = B1.cpu().numpy().astype(np.float64)
            W1 = W1.cpu().numpy().astype(np.float64)
            eb, ew = max_errors(B1[..., :p], W1, Bref, Wref, Vref)
            assert eb < TOL[prec] and ew < TOL[prec], ("oracle", call, eb, ew)
            eb, ew = max_errors(B1[..., :p], W1, B0[..., :p], W0, Vref)
            assert eb < TOL[prec] and ew < TOL[prec], ("gwas_scan", call, eb, ew)
            if out_mode == "var":
                V = _unpack_upper(B1[..., p:], p)
                assert np.all(np.isnan(V[257]))
                ok = np.ones(c.m, bool)
                ok[257] = False
                d = np.sqrt(np.diagonal(Vfull[ok], axis1=2, axis2=3))
                err = np.abs(V[ok] - Vfull[ok]) / (d[..., :, None] * d[..., None, :])
                assert np.max(err) < TOL[prec], ("var", call, np.max(err))
    finally:
        g.gwas_destroy(h)


def test_static_scan_rejects_oversize_and_other_handles(g):
    import torch
    c = synth.small_problem(42, n=1000, q=2, m=3000, t=3)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo="eig", precision="fp64")
    try:
        xr = torch.from_numpy(c.XR).cuda()
        B = torch.zeros((c.m, c.t, c.p), device="cuda")
        # 3000 SNPs x 1024 x 8 bytes > 16 MiB
        assert _static(g, h, xr, c.m, B, None) == -1
        assert "static scratch" in g.gwas_last_error()
        # 2048 SNPs x 1024 x 8 bytes = 16 MiB: the largest block this handle may pass
        B = torch.full((2048, c.t, c.p), float("nan"), device="cuda")
        W = torch.full((2048, c.t), float("nan"), device="cuda")
        assert _static(g, h, xr, 2048, B, W) == 0, g.gwas_last_error()
        sel = np.arange(0, 2048, 97)
        Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, snps=sel)
        eb, ew = max_errors(B.cpu().numpy().astype(np.float64)[sel],
                            W.cpu().numpy().astype(np.float64)[sel], Bref, Wref, Vref)
        assert eb < TOL["fp64"] and ew < TOL["fp64"], (eb, ew)
    finally:
        g.gwas_destroy(h)
    h = g.gwas_setup(c.Phi, c.XL, c.Y[:, :1], c.h2[:1], c.s2[:1], algo="chol", precision="fp64")
    try:
        B = torch.zeros((10, 1, c.p), device="cuda")
        assert _static(g, h, xr, 10, B, None) == -5
    finally:
        g.gwas_destroy(h)


def test_static_scan_validates_genotypes(g):
    """A handle set up with validate_genotypes rejects a code outside {0, 1, 2} here too, and a
    clean block afterwards passes (each call reports only its own genotypes)."""
    import torch
    c = synth.small_problem(43, n=130, q=2, m=90, t=5)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo="eig", precision="fp32",
                     validate_genotypes=1)
    try:
        bad = c.XR.copy()
        bad[40, 17] = 3
        B = torch.zeros((c.m, c.t, c.p), device="cuda")
        W = torch.zeros((c.m, c.t), device="cuda")
        assert _static(g, h, torch.from_numpy(bad).cuda(), c.m, B, W) == -6
        assert _static(g, h, torch.from_numpy(c.XR).cuda(), c.m, B, W) == 0, g.gwas_last_error()
        Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
        eb, ew = max_errors(B.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64),
                            Bref, Wref, Vref)
        assert eb < TOL["fp32"] and ew < TOL["fp32"], (eb, ew)
    finally:
        g.gwas_destroy(h)
