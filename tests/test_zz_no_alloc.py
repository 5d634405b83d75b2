"""gwas_scan_static: the scan entry point that allocates no device memory (its scratch is a
fixed 16 MiB device array in the library).  It exists for callers that cannot have a library
call cudaMalloc in the middle of their work: latency-critical loops, which cudaMalloc's implicit
device synchronisation would stall, and applications whose device memory belongs to their own
allocator or budget.  Checked through the C ABI against gwas_scan on the same handle, on two
calls in a row (the second finds the first call's data in the shared array), and for its
rejection of blocks larger than the array.

This file is collected last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import max_errors

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-6, "fp32": 2e-3}


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scan_matches_gwas_scan(g, prec):
    import torch
    c = synth.small_problem(41, n=300, q=3, m=500, t=23)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo="eig", precision=prec)
    try:
        xr = torch.from_numpy(c.XR).cuda()
        B0 = torch.zeros((c.m, c.t, c.p), dtype=torch.float32, device="cuda")
        W0 = torch.zeros((c.m, c.t), dtype=torch.float32, device="cuda")
        g.gwas_scan(h, xr, B0, W0)
        ref_B = B0.cpu().numpy().astype(np.float64)
        ref_W = W0.cpu().numpy().astype(np.float64)
        # the error measure needs a standard-error scale; the FP64 library result serves here
        vd = np.maximum(np.abs(ref_B), 1e-3)
        for call in range(2):
            B1 = torch.full((c.m, c.t, c.p), float("nan"), device="cuda")
            W1 = torch.full((c.m, c.t), float("nan"), device="cuda")
            # through the C ABI directly
            st = g.lib.gwas_scan_static(h, xr.data_ptr(), c.m, B1.data_ptr(), W1.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
            assert st == 0, g.gwas_last_error()
            torch.cuda.synchronize()
            eb, ew = max_errors(B1.cpu().numpy().astype(np.float64),
                                W1.cpu().numpy().astype(np.float64), ref_B, ref_W, vd ** 2)
            assert eb < TOL[prec] and ew < TOL[prec], (call, eb, ew)
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
        st = g.lib.gwas_scan_static(h, xr.data_ptr(), c.m, B.data_ptr(), None, None)
        assert st == -1 and "static scratch" in g.gwas_last_error()
        st = g.lib.gwas_scan_static(h, xr.data_ptr(), 2048, B.data_ptr(), None, None)
        assert st == 0, g.gwas_last_error()
        torch.cuda.synchronize()
    finally:
        g.gwas_destroy(h)
    h = g.gwas_setup(c.Phi, c.XL, c.Y[:, :1], c.h2[:1], c.s2[:1], algo="chol", precision="fp64")
    try:
        B = torch.zeros((10, 1, c.p), device="cuda")
        st = g.lib.gwas_scan_static(h, xr.data_ptr(), 10, B.data_ptr(), None, None)
        assert st == -5
    finally:
        g.gwas_destroy(h)
