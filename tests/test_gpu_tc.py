"""Parity of the split-BF16 tensor-core path (tcgen05) with the FP64 oracle.

Tolerance 1e-4 in the error measure of oracle.gls (relative error, or error in standard-error
units where the coefficient is near zero), the bound the split path is specified to meet.
Shapes cover several 128-SNP tiles with ragged tails, n not a multiple of 8 / 64 / 256, p from 2
to 8, more than one trait, the full workload-1 size on a slice, and singular SNPs.
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


def test_chol_golden_pedigree(g, golden_pedigree):
    gp = golden_pedigree
    for j in range(2):
        c = synth.Cohort(Phi=gp["Phi"], XL=gp["XL"], Y=gp["Y"][:, j:j + 1], h2=gp["h2"][j:j + 1],
                         s2=gp["s2"][j:j + 1], XR=gp["XR"], beta=None)
        B, W, _ = run(g, c, "chol", "split_bf16")
        eb, ew = max_errors(B, W, gp["B"][:, j:j + 1], gp["W"][:, j:j + 1], gp["Vd"][:, j:j + 1])
        assert eb < TOL and ew < TOL, (eb, ew)


@pytest.mark.parametrize("n,q,m,t", [(256, 3, 1000, 1), (97, 1, 131, 1), (200, 3, 300, 2),
                                     (130, 7, 257, 1), (520, 2, 129, 1), (64, 3, 1, 1)])
def test_chol_split_ragged(g, n, q, m, t):
    c = synth.small_problem(3 * n + q + m, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, nsing = run(g, c, "chol", "split_bf16")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)
    assert nsing == 0


def test_chol_split_workload0(g):
    c = synth.make_cohort(0)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "chol", "split_bf16")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def test_chol_split_workload1_slice(g):
    """Workload 1's shape (n = 1000, h2 = 0.5) on 3,000 SNPs, every SNP checked."""
    c = synth.make_cohort(1, m=3000)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "chol", "split_bf16")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def test_chol_split_singular_and_streamed(g):
    c = synth.small_problem(21, n=300, q=3, m=700, t=1)
    XR = c.XR.copy()
    XR[[0, 255, 699]] = 2
    Bd, Wd, nsing = run(g, c, "chol", "split_bf16", XR=XR)
    assert nsing == 3
    assert np.all(np.isnan(Bd[[0, 255, 699]])) and np.all(np.isnan(Wd[[0, 255, 699]]))
    Bh, Wh, _ = run(g, c, "chol", "split_bf16", XR=XR, device=False, block_snps=256)
    assert np.array_equal(np.isnan(Bd), np.isnan(Bh))
    ok = ~np.isnan(Bd)
    assert np.array_equal(Bd[ok], Bh[ok])


# ------------------------------------------------------------------------------------------ EIG

def test_eig_golden_pedigree(g, golden_pedigree):
    gp = golden_pedigree
    c = synth.Cohort(Phi=gp["Phi"], XL=gp["XL"], Y=gp["Y"], h2=gp["h2"], s2=gp["s2"], XR=gp["XR"], beta=None)
    B, W, _ = run(g, c, "eig", "split_bf16")
    eb, ew = max_errors(B, W, gp["B"], gp["W"], gp["Vd"])
    assert eb < TOL and ew < TOL, (eb, ew)


@pytest.mark.parametrize("n,q,m,t", [(97, 1, 131, 5), (200, 3, 300, 37), (130, 7, 70, 17),
                                     (64, 2, 64, 16), (300, 3, 257, 300), (520, 4, 129, 70),
                                     (256, 5, 200, 51), (333, 6, 150, 40)])
def test_eig_split_ragged(g, n, q, m, t):
    c = synth.small_problem(5 * n + q + m + t, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, nsing = run(g, c, "eig", "split_bf16")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)
    assert nsing == 0


def test_eig_split_workload2_slice(g):
    """Workload 2's shape (n = 1000, t = 1000, h2 up to 0.95) on 1,500 SNPs; 300 sampled pairs."""
    c = synth.make_cohort(2, m=1500)
    B, W, _ = run(g, c, "eig", "split_bf16")
    rs = np.random.default_rng(3)
    pairs = np.c_[rs.integers(0, c.m, 300), rs.integers(0, c.t, 300)]
    Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, pairs)
    eb, ew = max_errors(B[pairs[:, 0], pairs[:, 1]], W[pairs[:, 0], pairs[:, 1]], Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def test_eig_split_singular_and_streamed(g):
    c = synth.small_problem(22, n=300, q=3, m=700, t=45)
    XR = c.XR.copy()
    XR[[1, 128, 699]] = 0
    Bd, Wd, nsing = run(g, c, "eig", "split_bf16", XR=XR)
    assert nsing == 3 * c.t
    assert np.all(np.isnan(Bd[[1, 128, 699]])) and np.all(np.isnan(Wd[[1, 128, 699]]))
    Bh, Wh, _ = run(g, c, "eig", "split_bf16", XR=XR, device=False, block_snps=256)
    ok = ~np.isnan(Bd)
    assert np.array_equal(np.isnan(Bd), np.isnan(Bh)) and np.array_equal(Bd[ok], Bh[ok])


@pytest.mark.parametrize("algo,t", [("chol", 1), ("eig", 9)])
def test_split_without_intercept(g, algo, t):
    """X_L of zero-mean covariates and no all-ones column: the tensor-core path does not centre
    the SNPs (centring is exact only when the intercept is in the model)."""
    c = synth.small_problem(23, n=300, q=3, m=400, t=t)
    c.XL = c.XL.copy()
    c.XL[:, 0] = np.random.default_rng(5).standard_normal(c.n)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, algo, "split_bf16")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL and ew < TOL, (eb, ew)


def _near_one_cohort(t):
    """A kinship from 200 SNPs for n = 500 (300 eigenvalues at the 1e-3 ridge), h2 = 0.999 on the
    first half of the traits, U(0.9, 0.995) on the rest, and SNPs nearly collinear with the
    covariates (half their values copied from covariate 1's sign)."""
    rs = np.random.default_rng(12)
    n, q = 500, 3
    Phi = synth.kinship(synth.kinship_factor(rs, n, n_snps=200))
    XL = synth.covariates(rs, n, q)
    h2 = np.full(t, 0.999) if t == 1 else np.r_[np.full(t // 2, 0.999), rs.uniform(0.9, 0.995, t - t // 2)]
    s2 = rs.uniform(0.5, 2.0, t)
    Y = XL @ rs.standard_normal((q, t)) + rs.standard_normal((n, t))
    XR = synth.genotypes(rs, n, 400)
    lead = np.flatnonzero(XL[:, 1] > 0)
    for i in range(0, 40, 4):  # genotype tracks covariate 1 on half the individuals
        XR[i, lead] = np.where(rs.random(lead.size) < 0.9, 2, XR[i, lead])
    return synth.Cohort(Phi=Phi, XL=XL, Y=Y, h2=h2, s2=s2, XR=XR, beta=None)


def _kappa(Phi, h2):
    w = np.linalg.eigvalsh(Phi)
    return (h2 * w.max() + 1 - h2) / (h2 * w.min() + 1 - h2)


@pytest.mark.parametrize("algo,t", [("chol", 1), ("eig", 24)])
def test_split_near_one_heritability(g, algo, t):
    """h2 up to 0.999 on a kinship from 200 SNPs for n = 500: 300 eigenvalues at the 1e-3 ridge,
    so M_j^-1 weights those coordinates up to ~1000 times the others (lam_max / lam_min of M_j
    near 3000 at h2 = 0.999, near 500 at 0.995), the hardest case the split operands meet; some
    SNPs are nearly collinear with the covariates so that sigma = s - a^T P a cancels.  Setup takes
    a third BF16 piece of L_j^-1 / U_j here (two would give 1.3e-4 / 2.9e-4).  CHOL meets 1e-4 on
    every output at h2 = 0.999.  On its own the EIG contraction reaches its FP32 accumulation floor
    there (~1e-4 on the SNP effect, 1.2e-4 on the intercept): an EIG handle scans each trait with
    lam_max / lam_min above 500 with the CHOL kernel as well, so every output of every trait
    meets 1e-4, and the singular pairs are counted once."""
    c = _near_one_cohort(t)
    c.XR[7] = 1  # monomorphic: one singular pair per trait
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    for packed, device in ((True, True), (False, False)):
        B, W, nsing = run(g, c, algo, "split_bf16", packed=packed, device=device, block_snps=128)
        eb, ew = max_errors(B, W, Bref, Wref, Vref)
        assert eb < TOL and ew < TOL, (packed, device, eb, ew)
        assert nsing == t
    # this cohort's M is conditioned ~3000: setup chose the three-piece split and, for EIG, the
    # CHOL route of the traits past kappa 500; a well conditioned one (h2 = 0.5 on the same
    # kinship, kappa ~ 7) keeps two pieces and no route
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision="split_bf16")
    try:
        assert g.gwas_split_pieces(h) == 3
        routed = int(np.sum(_kappa(c.Phi, c.h2) > 500)) if algo == "eig" else 0
        assert g.gwas_chol_routed_traits(h) == routed
        assert algo == "chol" or routed >= t // 2
    finally:
        g.gwas_destroy(h)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, np.full(t, 0.5), c.s2, algo=algo, precision="split_bf16")
    try:
        assert g.gwas_split_pieces(h) == 2
        assert g.gwas_chol_routed_traits(h) == 0
    finally:
        g.gwas_destroy(h)


def test_eig_chol_route_in_every_output_mode(g):
    """The traits an EIG handle routes through the CHOL kernel write the same outputs the CHOL
    kernel writes for them alone, in the SNP and VAR modes too, and the other traits are those of
    the EIG kernels (a handle without the routed traits gives them bit for bit)."""
    c = _near_one_cohort(10)
    kap = _kappa(c.Phi, c.h2)
    rt = np.flatnonzero(kap > 500)
    keep = np.flatnonzero(kap <= 500)
    assert rt.size and keep.size
    for mode in ("full", "snp", "var"):
        B, W, _ = run(g, c, "eig", "split_bf16", out_mode=mode)
        for j in rt[:2]:
            cj = synth.Cohort(Phi=c.Phi, XL=c.XL, Y=c.Y[:, j:j + 1], h2=c.h2[j:j + 1],
                              s2=c.s2[j:j + 1], XR=c.XR, beta=None)
            Bj, Wj, _ = run(g, cj, "chol", "split_bf16", out_mode=mode)
            assert np.array_equal(B[:, j], Bj[:, 0], equal_nan=True), (mode, j)
            assert np.array_equal(W[:, j], Wj[:, 0], equal_nan=True), (mode, j)
        ck = synth.Cohort(Phi=c.Phi, XL=c.XL, Y=c.Y[:, keep], h2=c.h2[keep], s2=c.s2[keep],
                          XR=c.XR, beta=None)
        Bk, Wk, _ = run(g, ck, "eig", "split_bf16", out_mode=mode)
        assert np.array_equal(B[:, keep], Bk, equal_nan=True), mode
        assert np.array_equal(W[:, keep], Wk, equal_nan=True), mode


@pytest.mark.parametrize("algo,prec", [("chol", "split_bf16"), ("chol", "split_fp8"),
                                       ("eig", "split_bf16"), ("chol", "fp32"), ("eig", "fp64")])
@pytest.mark.parametrize("device,packed", [(True, False), (True, True), (False, False), (False, True)])
def test_empty_scan_every_path(g, algo, prec, device, packed):
    """m = 0 SNPs is a valid call on every path: nothing is written, nothing is counted."""
    import torch
    c = synth.small_problem(17, n=70, q=2, m=1, t=1 if algo == "chol" else 3)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision=prec)
    try:
        dev = "cuda" if device else "cpu"
        cols = g.gwas_packed_row_bytes(c.n) if packed else c.n
        X = torch.zeros((0, cols), dtype=torch.uint8 if packed else torch.int8, device=dev)
        B = torch.full((1, c.t, c.p), 7.0, device=dev)
        W = torch.full((1, c.t), 7.0, device=dev)
        (g.gwas_scan_packed if packed else g.gwas_scan)(h, X, B, W, m=0)
        torch.cuda.synchronize()
        assert torch.all(B == 7.0) and torch.all(W == 7.0)
        assert g.gwas_singular_count(h) == 0
    finally:
        g.gwas_destroy(h)
