"""Output modes: GWAS_OUT_SNP writes (b_snp, standard error) per pair -- the SNP effect equal to
the full scan's last coefficient, the standard error sqrt(Var(b)[p-1][p-1]) from the oracle --
and p-values of the Wald statistics match the chi-square(1) upper tail."""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


@pytest.mark.parametrize("algo,prec,n,q,m,t", [
    ("chol", "split_bf16", 200, 3, 300, 1), ("eig", "split_bf16", 300, 3, 257, 45),
    ("eig", "split_bf16", 130, 6, 140, 12), ("chol", "fp32", 97, 2, 131, 2),
    ("eig", "fp64", 130, 3, 70, 5)])
def test_snp_mode(g, algo, prec, n, q, m, t):
    c = synth.small_problem(81 + n + t, n=n, q=q, m=m, t=t)
    Bf, Wf, sf = run(g, c, algo, prec)
    Bs, Ws, ss = run(g, c, algo, prec, out_mode="snp")
    assert Bs.shape == (m, t, 2) and ss == sf
    assert np.array_equal(Bs[:, :, 0], Bf[:, :, -1]) and np.array_equal(Ws, Wf)
    _, _, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    se_ref = np.sqrt(Vref[:, :, -1])
    tol = 1e-6 if prec == "fp64" else 1e-4
    assert np.nanmax(np.abs(Bs[:, :, 1] - se_ref) / se_ref) < tol


def test_snp_mode_streamed_and_pvalues(g):
    import torch
    from scipy.stats import chi2
    c = synth.small_problem(91, n=300, q=3, m=700, t=20)
    Bd, Wd, _ = run(g, c, "eig", "split_bf16", out_mode="snp", packed=True)
    Bh, Wh, _ = run(g, c, "eig", "split_bf16", out_mode="snp", packed=True, device=False,
                    block_snps=256)
    assert np.array_equal(Bd, Bh) and np.array_equal(Wd, Wh)
    w = torch.from_numpy(Wd.astype(np.float32)).cuda()
    pv = g.gwas_wald_pvalues(w)
    torch.cuda.synchronize()
    ref = chi2.sf(Wd, 1)
    assert np.allclose(pv.cpu().numpy(), ref, rtol=2e-5, atol=1e-30)
