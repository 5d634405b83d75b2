"""The host-streaming pipeline ("Sequences of GLS'": blocks of SNPs moved to the device while the
previous ones are scanned): the block size chosen by timing when setup gets block_snps = 0, and
the device work of every full block replayed from a CUDA graph captured per ring slot.  Whatever
the block size and whether a block ran from a graph, the outputs are those of the device-resident
scan bit for bit (the same kernels on the same SNPs); across formats and output modes the graphs
are recaptured when their buffers or shapes change."""
import numpy as np
import pytest

import synth
from gpu_util import run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


def _scan(g, h, c, X, packed, device, p):
    import torch
    dev = "cuda" if device else "cpu"
    xr = torch.from_numpy(X).to(dev)
    if not device:
        xr = xr.pin_memory()
    B = torch.full((c.m, c.t, p), float("nan"), device=dev)
    W = torch.full((c.m, c.t), float("nan"), device=dev)
    if not device:
        B, W = B.pin_memory(), W.pin_memory()
    (g.gwas_scan_packed if packed else g.gwas_scan)(h, xr, B, W)
    if device:
        torch.cuda.synchronize()
    return B.cpu().numpy(), W.cpu().numpy()


@pytest.mark.parametrize("algo,prec,packed,m,t", [("chol", "split_bf16", True, 200_000, 1),
                                                  ("chol", "split_bf16", False, 70_000, 1),
                                                  ("eig", "split_bf16", True, 40_000, 64),
                                                  ("eig", "fp32", False, 30_000, 16)])
def test_block_size_by_timing(g, algo, prec, packed, m, t):
    c = synth.small_problem(51 + m, n=640, q=3, m=m, t=t)
    X = g.gwas_pack_genotypes(c.XR) if packed else c.XR
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision=prec, block_snps=0)
    try:
        assert not g.gwas_stream_info(h)["tuned"]
        Bd, Wd = _scan(g, h, c, X, packed, True, c.p)
        assert not g.gwas_stream_info(h)["tuned"]  # device buffers: nothing streamed
        Bh, Wh = _scan(g, h, c, X, packed, False, c.p)
        info = g.gwas_stream_info(h)
        assert info["tuned"] and info["block_snps"] in info["candidates"], info
        assert all(v[1] > 0 for v in info["candidates"].values())
        assert np.array_equal(Bd, Bh, equal_nan=True) and np.array_equal(Wd, Wh, equal_nan=True)
        if m > info["block_snps"]:
            assert info["graph_launches"] >= m // info["block_snps"] - 0
        # a second streamed call reuses the size and replays the graphs
        n0 = info["graph_launches"]
        Bh2, Wh2 = _scan(g, h, c, X, packed, False, c.p)
        assert np.array_equal(Bh2, Bh, equal_nan=True) and np.array_equal(Wh2, Wh, equal_nan=True)
        assert g.gwas_stream_info(h)["graph_launches"] == n0 + m // info["block_snps"]
    finally:
        g.gwas_destroy(h)


@pytest.mark.parametrize("algo,prec", [("chol", "split_bf16"), ("eig", "split_bf16"),
                                       ("eig", "fp64"), ("chol", "fp32")])
def test_graph_replays_across_formats(g, algo, prec):
    """One handle, blocks of 256 SNPs: int8 then packed host input (the tensor-core scans convert
    int8 on the device, the CUDA-core ones packed), every full block from a graph, the last
    partial one launched directly; all equal to the device-resident scan."""
    c = synth.small_problem(52, n=300, q=2, m=1300, t=9 if algo == "eig" else 1)
    ref_B, ref_W, _ = run(g, c, algo, prec)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision=prec, block_snps=256)
    try:
        for packed in (False, True, False):
            X = g.gwas_pack_genotypes(c.XR) if packed else c.XR
            n0 = g.gwas_stream_info(h)["graph_launches"]
            B, W = _scan(g, h, c, X, packed, False, c.p)
            assert np.array_equal(B, ref_B.astype(np.float32), equal_nan=True)
            assert np.array_equal(W, ref_W.astype(np.float32), equal_nan=True)
            assert g.gwas_stream_info(h)["graph_launches"] == n0 + 1300 // 256
    finally:
        g.gwas_destroy(h)
