"""Batched cohorts (gwas_setup_batch / gwas_scan_batch): one graph over cohorts of different
n, q and t gives every cohort exactly the results of its own scan, whatever launch plan the
autotuner picked, and stays within the oracle tolerance."""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import max_errors

pytestmark = pytest.mark.gpu
TOL = 1e-4
# (n, q, m, t): CHOL (t = 1) and EIG cohorts, ragged sizes, q from 1 to 7
COHORTS = [(97, 1, 700, 1), (256, 3, 1500, 5), (300, 7, 257, 17), (520, 2, 1029, 40),
           (130, 4, 64, 1), (200, 3, 900, 120)]


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


@pytest.fixture(scope="module")
def cohorts():
    return [synth.small_problem(60 + i, n=n, q=q, m=m, t=t) for i, (n, q, m, t) in enumerate(COHORTS)]


def _blocks(g, cs, fill=np.nan):
    import torch
    out = []
    for c in cs:
        G = g.gwas_pack_genotypes(torch.from_numpy(np.ascontiguousarray(c.XR)).cuda())
        B = torch.full((c.m, c.t, c.p), fill, dtype=torch.float32, device="cuda")
        W = torch.full((c.m, c.t), fill, dtype=torch.float32, device="cuda")
        out.append((G, B, W))
    return out


def _single(g, c):
    import torch
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, precision="split_bf16")
    try:
        G = g.gwas_pack_genotypes(torch.from_numpy(np.ascontiguousarray(c.XR)).cuda())
        B = torch.empty((c.m, c.t, c.p), dtype=torch.float32, device="cuda")
        W = torch.empty((c.m, c.t), dtype=torch.float32, device="cuda")
        g.gwas_scan_packed(h, G, B, W)
        torch.cuda.synchronize()
        return B.cpu().numpy(), W.cpu().numpy()
    finally:
        g.gwas_destroy(h)


def test_batch_equals_single_scans(g, cohorts):
    import torch
    b = g.gwas_setup_batch([(c.Phi, c.XL, c.Y, c.h2, c.s2) for c in cohorts])
    try:
        blocks = _blocks(g, cohorts)
        g.gwas_scan_batch(b, blocks)          # tunes the plan
        torch.cuda.synchronize()
        plan, ms = g.gwas_batch_plan(b)
        assert plan in (0, 1, 2, 3) and all(x > 0 for x in ms), (plan, ms)
        for c, (G, B, W) in zip(cohorts, blocks):
            Bs, Ws = _single(g, c)
            assert np.array_equal(B.cpu().numpy(), Bs) and np.array_equal(W.cpu().numpy(), Ws)
        # same sizes, new buffers: the chosen graph replayed on them
        blocks2 = _blocks(g, cohorts, fill=-7.0)
        g.gwas_scan_batch(b, blocks2)
        torch.cuda.synchronize()
        for (G, B, W), (G2, B2, W2) in zip(blocks, blocks2):
            assert torch.equal(B, B2) and torch.equal(W, W2)
        assert g.gwas_batch_plan(b)[0] == plan
        # the tuner's table: 3 EIG chunk sizes x 4 plans, the chosen pair its fastest entry
        tun = g.gwas_batch_tuning(b)
        assert tun["plan"] == plan and tun["chunk_div"] in (0, 1, 2)
        ms_all = np.array(tun["ms"])
        assert ms_all.shape == (3, 4) and np.all(ms_all > 0)
        assert ms_all[tun["chunk_div"], plan] == ms_all.min()
        assert list(ms) == list(ms_all[tun["chunk_div"]])
        for i, c in enumerate(cohorts):
            ck = g.gwas_eig_chunk(g.gwas_batch_handle(b, i))
            assert (ck == 0) if c.t == 1 else (ck > 0 and ck % 128 == 0)
    finally:
        g.gwas_destroy_batch(b)


def test_batch_tuned_chunk_equals_single_scan(g):
    """An EIG cohort longer than the smallest candidate chunk: whatever chunk the tuner keeps,
    the batch gives exactly the results of the cohort's own scan (each SNP's arithmetic does not
    depend on the chunk it falls in), and the chunk is capacity >> chunk_div."""
    import torch
    cs = [synth.small_problem(71, n=150, q=3, m=20000, t=9),
          synth.small_problem(72, n=97, q=1, m=300, t=1)]
    b = g.gwas_setup_batch([(c.Phi, c.XL, c.Y, c.h2, c.s2) for c in cs])
    try:
        blocks = _blocks(g, cs)
        g.gwas_scan_batch(b, blocks)
        torch.cuda.synchronize()
        tun = g.gwas_batch_tuning(b)
        h_single = g.gwas_setup(cs[0].Phi, cs[0].XL, cs[0].Y, cs[0].h2, cs[0].s2,
                                precision="split_bf16")
        try:
            cap = g.gwas_eig_chunk(h_single)
        finally:
            g.gwas_destroy(h_single)
        assert g.gwas_eig_chunk(g.gwas_batch_handle(b, 0)) == cap >> tun["chunk_div"]
        for c, (G, B, W) in zip(cs, blocks):
            Bs, Ws = _single(g, c)
            assert np.array_equal(B.cpu().numpy(), Bs) and np.array_equal(W.cpu().numpy(), Ws)
    finally:
        g.gwas_destroy_batch(b)


def test_batch_parity_and_skipped_cohort(g, cohorts):
    import torch
    cs = cohorts[:4]
    b = g.gwas_setup_batch([(c.Phi, c.XL, c.Y, c.h2, c.s2) for c in cs])
    try:
        blocks = _blocks(g, cs)
        G1, B1, W1 = blocks[1]
        blocks[1] = (G1[:0], B1, W1)          # m = 0: cohort 1 is skipped
        g.gwas_scan_batch(b, blocks)
        torch.cuda.synchronize()
        assert torch.isnan(B1).all()
        for i in (0, 2, 3):
            c = cs[i]
            Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
            eb, ew = max_errors(blocks[i][1].cpu().numpy().astype(np.float64),
                                blocks[i][2].cpu().numpy().astype(np.float64), Bref, Wref, Vref)
            assert eb < TOL and ew < TOL, (i, eb, ew)
        h0 = g.gwas_batch_handle(b, 0)
        assert g.gwas_info(h0)["n"] == cs[0].n and g.gwas_singular_count(h0) == 0
    finally:
        g.gwas_destroy_batch(b)


def test_batch_split_fp8_equals_single_scans(g, cohorts):
    """A batch set up with SPLIT_FP8 (its CHOL cohorts on the FP16 + E4M3 split, its EIG cohorts as
    SPLIT_BF16) gives every cohort exactly the results of its own SPLIT_FP8 scan, within 1e-4 of
    the oracle."""
    import torch
    cs = cohorts[:3]
    b = g.gwas_setup_batch([(c.Phi, c.XL, c.Y, c.h2, c.s2) for c in cs], precision="split_fp8")
    try:
        blocks = _blocks(g, cs)
        g.gwas_scan_batch(b, blocks)
        torch.cuda.synchronize()
        for i, (c, (G, B, W)) in enumerate(zip(cs, blocks)):
            h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, precision="split_fp8")
            try:
                assert g.gwas_fp8_traits(g.gwas_batch_handle(b, i)) == g.gwas_fp8_traits(h)
                Bs = torch.empty_like(B)
                Ws = torch.empty_like(W)
                g.gwas_scan_packed(h, G, Bs, Ws)
                torch.cuda.synchronize()
            finally:
                g.gwas_destroy(h)
            assert torch.equal(B, Bs) and torch.equal(W, Ws), i
            Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
            eb, ew = max_errors(B.cpu().numpy().astype(np.float64),
                                W.cpu().numpy().astype(np.float64), Bref, Wref, Vref)
            assert eb < TOL and ew < TOL, (i, eb, ew)
    finally:
        g.gwas_destroy_batch(b)
