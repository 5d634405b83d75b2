"""Parity of the genetic models (p_R genetic columns per SNP; Table 1's "genetic model assumed")
with the FP64 oracle: additive, dominant, recessive and the two-column additive + dominance
model, whose test is the joint 2-d.o.f. Wald statistic of the block.

Every scan path -- CHOL and EIG on the CUDA cores in FP64 (1e-6) and FP32 (2e-3), and on the
tensor cores (split BF16, 1e-4) -- is compared element by element with oracle.gls.gls_grid(model)
on ragged shapes (SNP counts that leave partial 32- and 64-column tiles, n off every tile size,
q from 1 to 7, several traits), in all three output modes, through the host-streaming ring, and
with SNPs whose block is singular (no heterozygote: an all-zero dominance column)."""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import run, max_errors

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-6, "fp32": 2e-3, "split_bf16": 1e-4}
MODELS = ["dominant", "recessive", "add_dom"]


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("algo,n,q,m,t", [("chol", 97, 1, 131, 1), ("chol", 200, 3, 300, 2),
                                          ("eig", 97, 1, 131, 5), ("eig", 130, 7, 70, 17),
                                          ("eig", 200, 3, 300, 37)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_models_ragged(g, model, algo, n, q, m, t, prec):
    c = synth.small_problem(11 * n + q + m + t, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=model)
    B, W, nsing = run(g, c, algo, prec, f64=(prec == "fp64"), model=model)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL[prec] and ew < TOL[prec], (eb, ew)
    assert nsing == int(np.isnan(Wref).sum())


@pytest.mark.parametrize("algo,t", [("chol", 1), ("eig", 9)])
def test_add_dom_singular_snps(g, algo, t):
    """SNPs with no heterozygote (all-zero dominance column) or no homozygote of one kind: NaN in
    every output of the pair and counted, exactly where the oracle's Cholesky fails."""
    c = synth.small_problem(31, n=150, q=3, m=100, t=t)
    XR = c.XR.copy()
    XR[5] = np.where(XR[5] == 1, 0, XR[5])
    XR[77] = np.where(XR[77] == 1, 2, XR[77])
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, XR, c.Y, c.h2, c.s2, model="add_dom")
    assert np.all(np.isnan(Wref[[5, 77]]))
    B, W, nsing = run(g, c, algo, "fp64", XR=XR, f64=True, model="add_dom")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < 1e-6 and ew < 1e-6, (eb, ew)
    assert nsing == int(np.isnan(Wref).sum()) >= 2 * t


@pytest.mark.parametrize("algo,t,prec", [("chol", 1, "fp64"), ("chol", 1, "fp32"),
                                         ("eig", 11, "fp64"), ("eig", 11, "fp32"),
                                         ("chol", 1, "split_bf16"), ("eig", 11, "split_bf16")])
def test_add_dom_output_modes(g, algo, t, prec):
    """SNP mode: (b_x, b_d, se_x, se_d) per pair; VAR mode: the p coefficients, then the whole
    Var(b) = (X_i^T M_j^-1 X_i)^-1 (p = q + 2) against the oracle entry by entry."""
    c = synth.small_problem(32, n=140, q=2, m=90, t=t)
    p = c.q + 2
    _, _, Vd, V = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, full_var=True, model="add_dom")
    Bref, Wref, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model="add_dom")
    tol = TOL[prec]
    Bs, Ws, _ = run(g, c, algo, prec, model="add_dom", out_mode="snp")
    assert Bs.shape == (c.m, t, 4)
    eb, ew = max_errors(Bs[..., :2], Ws, Bref[..., c.q:], Wref, Vd[..., c.q:])
    assert eb < tol and ew < tol, (eb, ew)
    se = np.sqrt(Vd[..., c.q:])
    ok = np.isfinite(se)
    assert np.array_equal(np.isnan(Bs[..., 2:]), ~ok)
    assert np.max(np.abs(Bs[..., 2:][ok] - se[ok]) / se[ok]) < tol
    Bv, Wv, _ = run(g, c, algo, prec, model="add_dom", out_mode="var")
    assert Bv.shape == (c.m, t, p + p * (p + 1) // 2)
    eb, ew = max_errors(Bv[..., :p], Wv, Bref, Wref, Vd)
    assert eb < tol and ew < tol, (eb, ew)
    Vg = np.empty(Bv.shape[:2] + (p, p))
    e = p
    for r in range(p):
        for cc in range(r, p):
            Vg[..., r, cc] = Vg[..., cc, r] = Bv[..., e]
            e += 1
    fin = np.all(np.isfinite(V), axis=(-1, -2))
    assert np.array_equal(np.all(np.isnan(Vg), axis=(-1, -2)), ~fin)
    d = np.sqrt(np.diagonal(V[fin], axis1=-2, axis2=-1))
    err = np.abs(Vg[fin] - V[fin]) / (d[..., :, None] * d[..., None, :])
    assert np.max(err) < tol, np.max(err)


@pytest.mark.parametrize("algo,t", [("chol", 2), ("eig", 13)])
def test_add_dom_streamed_equals_device(g, algo, t):
    """Host buffers through the streaming ring give the device-resident scan's outputs bit for
    bit (blocks of 96 SNPs: partial tiles at every block end)."""
    c = synth.small_problem(33, n=120, q=3, m=500, t=t)
    Bd, Wd, _ = run(g, c, algo, "fp64", f64=True, model="add_dom")
    Bh, Wh, _ = run(g, c, algo, "fp64", f64=True, model="add_dom", device=False, block_snps=96)
    assert np.array_equal(Bd, Bh, equal_nan=True) and np.array_equal(Wd, Wh, equal_nan=True)


# ------------------------------------------------------------------------------- tensor cores

@pytest.mark.parametrize("model", ["dominant", "recessive"])
@pytest.mark.parametrize("algo,n,q,m,t", [("chol", 97, 1, 131, 1), ("chol", 256, 3, 700, 1),
                                          ("eig", 200, 3, 300, 37), ("eig", 130, 7, 70, 17)])
@pytest.mark.parametrize("packed", [False, True])
def test_split_single_column_models(g, model, algo, n, q, m, t, packed):
    """One-column codings on the tensor cores: each row's byte table maps the hard calls to the
    model's values (centred by the multiple of 1/64 nearest the coded column's mean)."""
    c = synth.small_problem(13 * n + q + m + t, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model=model)
    B, W, nsing = run(g, c, algo, "split_bf16", model=model, packed=packed)
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < 1e-4 and ew < 1e-4, (eb, ew)
    assert nsing == int(np.isnan(Wref).sum())


@pytest.mark.parametrize("n,q,m,t", [(97, 1, 131, 1), (256, 3, 700, 1), (520, 7, 300, 2),
                                     (64, 2, 1, 1), (1000, 3, 1500, 1)])
def test_split_chol_add_dom(g, n, q, m, t):
    """The two-column model on the CHOL tensor-core kernel: 64 SNPs per tile, a SNP's two working
    columns 16 TMEM lanes apart, their cross product summed with a lane shuffle, the 2 x 2 Schur
    solve in FP64; ragged tails, one SNP, q up to 7, the n = 1000 shape."""
    c = synth.small_problem(17 * n + q + m, n=n, q=q, m=m, t=t, h2=0.5 if n == 1000 else None)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model="add_dom")
    for packed in (False, True):
        B, W, nsing = run(g, c, "chol", "split_bf16", model="add_dom", packed=packed)
        eb, ew = max_errors(B, W, Bref, Wref, Vref)
        assert eb < 1e-4 and ew < 1e-4, (packed, eb, ew)
        assert nsing == int(np.isnan(Wref).sum())


@pytest.mark.parametrize("algo,t", [("chol", 1), ("eig", 21)])
def test_split_add_dom_streamed_and_without_intercept(g, algo, t):
    """Host buffers through the streaming ring equal the device-resident scan.  Without an
    intercept column the tensor-core setup refuses the two-column model (its working columns
    are centred through the intercept), and the CUDA-core paths take it."""
    c = synth.small_problem(35 if algo == "chol" else 36, n=300, q=3, m=700, t=t)
    Bd, Wd, _ = run(g, c, algo, "split_bf16", model="add_dom", packed=True)
    Bh, Wh, _ = run(g, c, algo, "split_bf16", model="add_dom", packed=True, device=False,
                    block_snps=256)
    assert np.array_equal(Bd, Bh, equal_nan=True) and np.array_equal(Wd, Wh, equal_nan=True)
    c.XL = c.XL.copy()
    c.XL[:, 0] = np.random.default_rng(6).standard_normal(c.n)
    with pytest.raises(g.GwasError) as e:
        run(g, c, algo, "split_bf16", model="add_dom")
    assert e.value.status == -5 and "intercept" in str(e.value)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model="add_dom")
    B, W, _ = run(g, c, algo, "fp32", model="add_dom")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < TOL["fp32"] and ew < TOL["fp32"], (eb, ew)


@pytest.mark.parametrize("n,q,m,t", [(97, 1, 131, 5), (200, 3, 300, 37), (130, 7, 70, 17),
                                     (300, 3, 257, 300), (64, 2, 1, 3)])
def test_split_eig_add_dom(g, n, q, m, t):
    """The two-column model on the EIG tensor-core kernels: ROT writes three squared planes per
    SNP (x0 x0, x0 x1, x1 x1; 64 SNPs per tile, a SNP's columns 16 lanes apart), SQ contracts
    every plane row with d_j, and AC solves each pair's 2 x 2 Schur complement in FP32 from the
    partner lane's a and c; several trait blocks, ragged tails, one SNP, q up to 7."""
    c = synth.small_problem(19 * n + q + m + t, n=n, q=q, m=m, t=t)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, model="add_dom")
    for packed in (False, True):
        B, W, nsing = run(g, c, "eig", "split_bf16", model="add_dom", packed=packed)
        eb, ew = max_errors(B, W, Bref, Wref, Vref)
        assert eb < 1e-4 and ew < 1e-4, (packed, eb, ew)
        assert nsing == int(np.isnan(Wref).sum())


def test_split_eig_add_dom_workload2_shape(g):
    """Workload 2's shape (n = 1000, t = 1000, h2 up to 0.95) on 700 SNPs; 300 sampled pairs."""
    c = synth.make_cohort(2, m=700)
    B, W, _ = run(g, c, "eig", "split_bf16", model="add_dom", packed=True)
    rs = np.random.default_rng(8)
    pairs = np.c_[rs.integers(0, c.m, 300), rs.integers(0, c.t, 300)]
    Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, pairs, model="add_dom")
    eb, ew = max_errors(B[pairs[:, 0], pairs[:, 1]], W[pairs[:, 0], pairs[:, 1]], Bref, Wref, Vref)
    assert eb < 1e-4 and ew < 1e-4, (eb, ew)


def test_add_dom_pvalues_on_device(g):
    """2-d.o.f. p-values of the joint statistics on the device: scipy's chi-square(2) tail of
    the same statistics; NaN for the singular pairs."""
    import torch
    from scipy.stats import chi2
    c = synth.small_problem(37, n=200, q=3, m=300, t=7)
    _, W, _ = run(g, c, "eig", "split_bf16", model="add_dom")
    w = torch.from_numpy(W.astype(np.float32)).cuda()
    pv = g.gwas_wald_pvalues_dof(w, 2).cpu().numpy()
    ref = chi2.sf(W.astype(np.float32).astype(np.float64), 2)
    assert np.array_equal(np.isnan(pv), np.isnan(W))
    ok = ~np.isnan(W)
    assert np.allclose(pv[ok], ref[ok], rtol=2e-5, atol=1e-30)
