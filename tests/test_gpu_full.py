"""Tensor-core parity at the benchmark's full sizes and launch configuration, and with many
work items per persistent CTA.

Full sizes (2,000,000 SNPs for the single-trait CHOL scan, 100,000 SNPs x 1,000 traits and one
32 Ki-SNP block of 30,000 traits for EIG) are checked on sampled (SNP, trait) pairs that the
oracle solves one by one, through the same calls and packed device-resident input as the bench.
The smaller cases give every CTA several work items (several SNP tiles, or several column
blocks of one tile), with every pair checked.  The largest n that setup accepts (16384) is
checked for the CHOL scan in both split precisions, and n = 4500 for EIG, every pair checked.
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


@pytest.mark.parametrize("n,m,t", [(1000, 5000, 5), (300, 40000, 3), (640, 20000, 2)])
def test_eig_split_many_items_per_cta(g, n, m, t):
    """Rotation work items (tile, 256-column block) outnumber the SMs: each CTA converts the
    genotype slices of several tiles through its shared-memory ring."""
    c = synth.small_problem(40 + n, n=n, q=3, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    for packed in (False, True):
        B, W, nsing = run(g, c, "eig", "split_bf16", packed=packed)
        eb, ew = max_errors(B, W, Bref, Wref, Vref)
        assert eb < TOL and ew < TOL, (packed, eb, ew)
        assert nsing == 0


def test_chol_split_many_tiles_per_cta(g):
    c = synth.small_problem(41, n=1000, q=3, m=40000, t=1)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "chol", "split_bf16", packed=True)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def _full_sampled(g, idx, m, pairs_count, algo):
    import torch
    c = synth.make_cohort(idx, m=0, with_genotypes=False)
    c.XR = synth.workload_genotypes(idx, m)
    mm, t, p = c.m, c.t, c.p
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision="split_bf16")
    try:
        G = g.gwas_pack_genotypes(torch.from_numpy(c.XR).cuda())
        B = torch.empty((mm, t, p), dtype=torch.float32, device="cuda")
        W = torch.empty((mm, t), dtype=torch.float32, device="cuda")
        g.gwas_scan_packed(h, G, B, W)
        torch.cuda.synchronize()
        del G
        rs = np.random.default_rng(idx)
        snps = np.sort(rs.choice(mm, size=pairs_count, replace=False))
        snps[-1] = mm - 1  # the ragged last tile
        traits = rs.integers(0, t, size=pairs_count)
        sel = torch.from_numpy(snps).cuda()
        Bs = B[sel].cpu().numpy()[np.arange(pairs_count), traits].astype(np.float64)
        Ws = W[sel].cpu().numpy()[np.arange(pairs_count), traits].astype(np.float64)
    finally:
        g.gwas_destroy(h)
    Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, np.c_[snps, traits])
    return max_errors(Bs, Ws, Bref, Wref, Vref)


def test_chol_workload1_full_size_sampled(g):
    """n = 1,000, p = 4, m = 2,000,000 in one launch; 256 sampled SNPs."""
    eb, ew = _full_sampled(g, 1, None, 256, "chol")
    assert eb < TOL and ew < TOL, (eb, ew)


def test_eig_workload2_full_size_sampled(g):
    """n = 1,000, t = 1,000, m = 100,000 (four 32 Ki-SNP chunks); 300 sampled pairs."""
    eb, ew = _full_sampled(g, 2, None, 300, "eig")
    assert eb < TOL and ew < TOL, (eb, ew)


def test_eig_workload3_block_sampled(g):
    """n = 1,000, t = 30,000, one 32,768-SNP block (the bench's block); 200 sampled pairs."""
    eb, ew = _full_sampled(g, 3, 32768, 200, "eig")
    assert eb < TOL and ew < TOL, (eb, ew)


@pytest.fixture(scope="module")
def max_n_cohort():
    """n = 16384, the largest n that gwas_setup accepts.  The kinship comes from 256 standardised
    SNPs (plus the ridge), so that building it stays cheap on the host; its non-zero eigenvalues
    sit near n / 256, which at h2 = 0.5 keeps lam_max / lam_min of M below 100 (two pieces, and
    the FP8 split)."""
    rs = np.random.default_rng(16384)
    n, q, m = 16384, 3, 300
    Gs = synth.kinship_factor(rs, n, n_snps=256)
    Phi = synth.kinship(Gs)
    XL = synth.covariates(rs, n, q)
    h2, s2 = np.array([0.5]), np.array([1.3])
    Y, beta = synth.traits(rs, XL, Gs, h2, s2)
    c = synth.Cohort(Phi=Phi, XL=XL, Y=Y, h2=h2, s2=s2, XR=synth.genotypes(rs, n, m), beta=beta)
    return c, gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)


@pytest.mark.parametrize("prec", ["split_bf16", "split_fp8"])
def test_chol_split_max_n(g, max_n_cohort, prec):
    """The CHOL tensor-core scan at n = 16384: 65 blocks of 256 rows of the augmented L^-1 per
    SNP tile, K ranges up to 16,384; every SNP checked against the oracle."""
    c, (Bref, Wref, Vref) = max_n_cohort
    B, W, nsing = run(g, c, "chol", prec, packed=True)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)
    assert nsing == 0


def test_eig_split_large_n(g):
    """EIG at n = 4500 (the eigendecomposition of a full-rank kinship, 71 K steps, 18 row blocks
    of Z^T in the rotation), several traits, every pair checked."""
    c = synth.small_problem(4500, n=4500, q=3, m=400, t=5)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, nsing = run(g, c, "eig", "split_bf16", packed=True)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)
    assert nsing == 0
