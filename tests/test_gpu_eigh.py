"""The setup's FP64 eigendecomposition of the kinship matrix (Householder reduction, multisection,
inverse iteration with cluster-separated shifts, Cholesky QR) on kinships whose spectra have large
exactly degenerate eigenspaces -- a genomic kinship from fewer SNPs than individuals (the ridge
eigenvalue repeated n - #SNPs times) and a pedigree of full sibships (two distinct eigenvalues) --
seen through everything that uses it: the CLAK-Eig scans against the FP64 oracle and step 1's
estimates against the step-1 oracle.  Two more: unrelated individuals (Phi = I, one n-fold
eigenvalue) and a weak chain of relatives (Phi = I + 1e-3 on the first off-diagonals, n even), whose
spectrum is symmetric about 1 so that the Sturm count is taken at a shift equal to the diagonal --
an exactly zero pivot, which has to be counted the way the rest of the recurrence uses it.  Last,
a Wilkinson-type kinship (tridiagonal, diagonal |k - i| for n = 2k + 1, off-diagonals 1, shifted
and scaled to be positive definite): its largest eigenvalues come in pairs that agree to about
1e-13 relative without being equal, the close-but-distinct clusters on which a Sturm count that
is not monotone in the shift would lose or repeat an eigenvalue."""
import numpy as np
import pytest

import synth
from oracle import estimate as est
from oracle import gls
from gpu_util import max_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


KINDS = ["few_snps", "sibships", "unrelated", "chain", "wilkinson"]


def _cohort(kind, n=300, q=3, m=200, t=6):
    rs = np.random.default_rng(12072169 + KINDS.index(kind) + 1)
    if kind == "wilkinson":
        n = 301
        k = n // 2
        W = np.diag(np.abs(k - np.arange(n)).astype(np.float64))
        W += np.eye(n, k=1) + np.eye(n, k=-1)
        Phi = (W + 2.0 * np.eye(n)) / (k + 3.0)
    elif kind == "few_snps":
        Phi = synth.kinship(synth.kinship_factor(rs, n, n_snps=40))
    elif kind == "unrelated":
        Phi = np.eye(n)
    elif kind == "chain":
        Phi = np.eye(n) + 1e-3 * (np.eye(n, k=1) + np.eye(n, k=-1))
    else:
        Phi = np.eye(n)
        for f in range(0, n, 4):  # families of four full sibs: relationship 1/2
            blk = slice(f, min(f + 4, n))
            Phi[blk, blk] = 0.5
            np.fill_diagonal(Phi[blk, blk], 1.0)
    XL = synth.covariates(rs, n, q)
    Y = XL @ rs.standard_normal((q, t)) + rs.standard_normal((n, t))
    h2 = rs.uniform(0.1, 0.9, t)
    s2 = rs.uniform(0.5, 2.0, t)
    XR = synth.genotypes(rs, n, m)
    return Phi, XL, Y, h2, s2, XR


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("split_bf16", 1e-4)])
def test_eig_scan_on_degenerate_kinships(g, kind, prec, tol):
    import torch
    Phi, XL, Y, h2, s2, XR = _cohort(kind)
    m, t, p = XR.shape[0], Y.shape[1], XL.shape[1] + 1
    h = g.gwas_setup(Phi, XL, Y, h2, s2, algo="eig", precision=prec)
    try:
        B = torch.empty((m, t, p), dtype=torch.float32, device="cuda")
        W = torch.empty((m, t), dtype=torch.float32, device="cuda")
        g.gwas_scan(h, torch.from_numpy(XR).cuda(), B, W)
        torch.cuda.synchronize()
    finally:
        g.gwas_destroy(h)
    Bref, Wref, Vref = gls.gls_grid(Phi, XL, XR, Y, h2, s2)
    eb, ew = max_errors(B.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64),
                        Bref, Wref, Vref)
    assert eb < tol and ew < tol, (eb, ew)


@pytest.mark.parametrize("kind", KINDS)
def test_estimate_on_degenerate_kinships(g, kind):
    Phi, XL, Y, _, _, _ = _cohort(kind, t=3)
    h2, s2, ll, _ = g.gwas_estimate(Phi, XL, Y, method="reml")
    _, _, llr = est.estimate(Phi, XL, Y, est.REML)
    assert np.all(np.abs(ll - llr) <= 1e-8 * np.abs(llr)), (ll, llr)
