"""The packed 2-bit genotype format (gwas_scan_packed, gwas_pack_genotypes) on the GPU.

Packing is a storage format: a scan of packed rows must give exactly the results of the int8
scan of the same genotypes on every path (the tensor-core kernels read packed rows either way;
the CUDA-core kernels unpack them), and the split-BF16 results stay within the oracle tolerance.
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


def _same(a, b):
    return np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


@pytest.mark.parametrize("n", [1, 97, 1000])
def test_device_packing_matches_host(g, n):
    import torch
    rs = np.random.default_rng(n + 5)
    X = rs.integers(0, 3, size=(1031, n)).astype(np.int8)
    X[3, 0] = 5   # invalid values: code 3 on both sides
    X[7, n - 1] = -2
    Gh = np.zeros((1031, g.gwas_packed_row_bytes(n)), np.uint8)
    st = g.lib.gwas_pack_genotypes(X.ctypes.data, X.shape[0], n, Gh.ctypes.data, 0, None)
    assert st == -6
    Gd = g.gwas_pack_genotypes(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(Gd.cpu().numpy(), Gh)


@pytest.mark.parametrize("algo,prec,n,q,m,t", [
    ("chol", "split_bf16", 97, 1, 131, 1), ("chol", "split_bf16", 200, 3, 300, 2),
    ("eig", "split_bf16", 130, 7, 70, 17), ("eig", "split_bf16", 300, 3, 257, 45),
    ("chol", "fp32", 97, 2, 131, 2), ("eig", "fp64", 130, 3, 70, 5)])
def test_packed_scan_equals_int8_scan(g, algo, prec, n, q, m, t):
    c = synth.small_problem(7 * n + q + m + t, n=n, q=q, m=m, t=t)
    B8, W8, s8 = run(g, c, algo, prec)
    Bp, Wp, sp = run(g, c, algo, prec, packed=True)
    assert _same(B8, Bp) and _same(W8, Wp) and s8 == sp
    if prec == "split_bf16":
        Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
        eb, ew = max_errors(Bp, Wp, Bref, Wref, Vref)
        assert eb < TOL and ew < TOL, (eb, ew)


@pytest.mark.parametrize("algo", ["chol", "eig"])
def test_packed_host_streamed(g, algo):
    c = synth.small_problem(31, n=300, q=3, m=700, t=1 if algo == "chol" else 20)
    Bd, Wd, _ = run(g, c, algo, "split_bf16", packed=True)
    Bh, Wh, _ = run(g, c, algo, "split_bf16", packed=True, device=False, block_snps=256)
    assert _same(Bd, Bh) and _same(Wd, Wh)


@pytest.mark.parametrize("prec,packed", [("split_bf16", True), ("fp64", False), ("fp32", False)])
def test_chol_streamed_two_lanes_many_blocks(g, prec, packed):
    """Host-streamed CHOL scans that use no scratch (tensor cores on packed rows, CUDA cores on
    int8 rows) alternate their blocks between two compute streams through a ring of four device
    buffers: 11 blocks of 256 SNPs (every buffer reused, a ragged last block) must give exactly
    the results of one device-resident scan."""
    c = synth.small_problem(33, n=257, q=2, m=2700, t=1)
    f64 = prec == "fp64"
    Bd, Wd, _ = run(g, c, "chol", prec, packed=packed, f64=f64)
    Bh, Wh, _ = run(g, c, "chol", prec, packed=packed, f64=f64, device=False, block_snps=256)
    assert _same(Bd, Bh) and _same(Wd, Wh)


@pytest.mark.parametrize("algo,prec", [("chol", "split_bf16"), ("eig", "split_bf16"),
                                       ("eig", "fp32"), ("chol", "fp64")])
def test_pinned_host_buffers_streamed(g, algo, prec):
    """Page-locked host buffers (asynchronous copies through the handle's ring): with host input
    and with device input, over several streamed blocks, the host outputs are exactly those of
    the device-resident scan."""
    import torch
    c = synth.small_problem(35, n=200, q=3, m=1500, t=1 if algo == "chol" else 17)
    f64 = prec == "fp64"
    dt = torch.float64 if f64 else torch.float32
    Bd, Wd, _ = run(g, c, algo, prec, f64=f64)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision=prec, block_snps=256)
    try:
        scan = g.gwas_scan_f64 if f64 else g.gwas_scan
        X = torch.from_numpy(c.XR).pin_memory()
        for xr in (X, X.cuda()):
            B = torch.full((c.m, c.t, c.p), float("nan"), dtype=dt).pin_memory()
            W = torch.full((c.m, c.t), float("nan"), dtype=dt).pin_memory()
            scan(h, xr, B, W)
            torch.cuda.synchronize()
            assert _same(B.numpy().astype(np.float64), Bd) and _same(W.numpy().astype(np.float64), Wd)
    finally:
        g.gwas_destroy(h)


@pytest.mark.parametrize("algo,prec", [("chol", "split_bf16"), ("eig", "split_bf16"),
                                       ("eig", "fp32")])
def test_packed_validation(g, algo, prec):
    import torch
    c = synth.small_problem(32, n=70, q=2, m=40, t=3)
    G = g.gwas_pack_genotypes(np.ascontiguousarray(c.XR))
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision=prec, validate_genotypes=1)
    try:
        B = torch.zeros((c.m, c.t, c.p), dtype=torch.float32, device="cuda")
        bad3 = G.copy()
        bad3[5, 2] |= 0x30               # genotype 10 of SNP 5 -> code 3
        pad = G.copy()
        pad[9, 17] |= 0x10              # genotype 70, past n = 70: byte 17, bits 4-5
        for bad in (bad3, pad):
            with pytest.raises(g.GwasError) as ei:
                g.gwas_scan_packed(h, torch.from_numpy(bad).cuda(), B)
            assert ei.value.status == -6
        g.gwas_scan_packed(h, torch.from_numpy(G).cuda(), B)  # valid rows pass
        X = c.XR.copy()
        X[2, 3] = 4
        with pytest.raises(g.GwasError) as ei:
            g.gwas_scan(h, torch.from_numpy(X).cuda(), B)
        assert ei.value.status == -6
    finally:
        g.gwas_destroy(h)


def test_packed_unaligned_device_pointer_is_rejected(g):
    import torch
    c = synth.small_problem(33, n=64, q=2, m=10, t=1)
    G = g.gwas_pack_genotypes(np.ascontiguousarray(c.XR))
    rb = G.shape[1]
    buf = torch.zeros(G.size + 16, dtype=torch.uint8, device="cuda")
    Gu = buf[1:1 + G.size].view(c.m, rb)
    Gu.copy_(torch.from_numpy(G).reshape(c.m, rb))
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo="chol", precision="split_bf16")
    try:
        B = torch.zeros((c.m, 1, c.p), dtype=torch.float32, device="cuda")
        with pytest.raises(g.GwasError) as ei:
            g.gwas_scan_packed(h, Gu, B)
        assert ei.value.status == -1
    finally:
        g.gwas_destroy(h)
