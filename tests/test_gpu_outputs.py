"""Output modes: GWAS_OUT_SNP writes (b_snp, standard error) per pair -- the SNP effect equal to
the full scan's last coefficient, the standard error sqrt(Var(b)[p-1][p-1]) from the oracle --;
GWAS_OUT_VAR writes the coefficients and the whole Var(b); p-values of the Wald statistics match
the chi-square(1) upper tail."""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import run, max_errors

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
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    tol = 1e-6 if prec == "fp64" else 1e-4
    eb, ew = max_errors(Bf, Wf, Bref, Wref, Vref)
    assert eb < tol and ew < tol, (eb, ew)
    # NaN exactly where the oracle has none (an unwritten pair stays NaN and fails here)
    se_ref = np.sqrt(Vref[:, :, -1])
    assert np.array_equal(np.isnan(Bs[:, :, 1]), np.isnan(se_ref))
    ok = ~np.isnan(se_ref)
    assert np.max(np.abs(Bs[:, :, 1][ok] - se_ref[ok]) / se_ref[ok]) < tol


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


def _unpack_upper(flat, p):
    """(..., p(p+1)/2) packed upper triangle, row by row -> (..., p, p) symmetric."""
    V = np.empty(flat.shape[:-1] + (p, p))
    e = 0
    for r in range(p):
        for c in range(r, p):
            V[..., r, c] = V[..., c, r] = flat[..., e]
            e += 1
    return V


@pytest.mark.parametrize("algo,prec,n,q,m,t,packed", [
    ("chol", "split_bf16", 200, 3, 300, 1, False), ("eig", "split_bf16", 300, 3, 257, 45, True),
    ("eig", "split_bf16", 130, 6, 140, 12, False), ("eig", "split_bf16", 150, 1, 90, 9, True),
    ("chol", "split_bf16", 256, 7, 160, 1, True), ("chol", "fp32", 97, 2, 131, 2, False),
    ("eig", "fp64", 130, 3, 70, 5, False), ("chol", "fp64", 120, 4, 64, 1, False)])
def test_var_mode(g, algo, prec, n, q, m, t, packed):
    """GWAS_OUT_VAR: per pair the p coefficients (exactly those of the full scan), then the whole
    Var(b) = (X_i^T M_j^-1 X_i)^-1 of Eq. "probDef" against the FP64 oracle, entry by entry on
    the scale of sqrt(Var_rr Var_cc); a monomorphic SNP gives NaN throughout."""
    c = synth.small_problem(181 + n + t, n=n, q=q, m=m, t=t)
    c.XR[m // 2] = 1  # monomorphic: singular pair
    p = q + 1
    Bf, Wf, sf = run(g, c, algo, prec, packed=packed)
    Bv, Wv, sv = run(g, c, algo, prec, packed=packed, out_mode="var")
    assert Bv.shape == (m, t, p + p * (p + 1) // 2) and sv == sf
    assert np.array_equal(Bv[:, :, :p], Bf, equal_nan=True) and np.array_equal(Wv, Wf, equal_nan=True)
    _, _, _, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, full_var=True)
    V = _unpack_upper(Bv[:, :, p:], p)
    assert np.all(np.isnan(V[m // 2]))
    ok = np.ones(m, bool)
    ok[m // 2] = False
    d = np.sqrt(np.diagonal(Vref[ok], axis1=2, axis2=3))
    err = np.abs(V[ok] - Vref[ok]) / (d[..., :, None] * d[..., None, :])
    tol = 1e-6 if prec == "fp64" else 1e-4
    assert np.max(err) < tol, np.max(err)


def test_var_mode_streamed(g):
    """GWAS_OUT_VAR through the host-streaming path equals the device-resident scan."""
    c = synth.small_problem(93, n=200, q=3, m=600, t=7)
    Bd, Wd, _ = run(g, c, "eig", "split_bf16", out_mode="var", packed=True)
    Bh, Wh, _ = run(g, c, "eig", "split_bf16", out_mode="var", packed=True, device=False,
                    block_snps=256)
    assert np.array_equal(Bd, Bh) and np.array_equal(Wd, Wh)


@pytest.mark.parametrize("out_mode,t", [("full", 64), ("snp", 64), ("snp", 65)])
def test_unaligned_outputs(g, out_mode, t):
    """Output buffers the C ABI allows -- float-aligned, not 16-byte aligned -- and an odd trait
    count in SNP mode get the same values as 16-byte-aligned ones (the kernel's vector stores
    are used only where the alignment allows them)."""
    import torch
    c = synth.small_problem(95, n=200, q=3, m=300, t=t)
    pw = 2 if out_mode == "snp" else c.p
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo="eig", precision="split_bf16",
                     out_mode=out_mode)
    try:
        xr = torch.from_numpy(c.XR).cuda()
        outs = []
        for shift in (0, 1):
            Bbuf = torch.full((c.m * c.t * pw + 4,), float("nan"), device="cuda")
            Wbuf = torch.full((c.m * c.t + 4,), float("nan"), device="cuda")
            B = Bbuf[shift:shift + c.m * c.t * pw].view(c.m, c.t, pw)
            W = Wbuf[shift:shift + c.m * c.t].view(c.m, c.t)
            assert (B.data_ptr() % 16 == 0) == (shift == 0)
            g.gwas_scan(h, xr, B, W)
            torch.cuda.synchronize()
            outs.append((B.cpu().numpy(), W.cpu().numpy()))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        assert not np.isnan(outs[0][0]).any()
    finally:
        g.gwas_destroy(h)
