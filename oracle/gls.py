"""Plain FP64 oracle for the GLS grid (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs import this
module.  It is slow on purpose: each problem is solved as the paper defines it, with no
blocking or fusion beyond what the cited algorithm states.  It shares no code with the CUDA
library.

Notation (Supplementary Note Section 1): n individuals, X_i = [X_L | x_i] with X_L = [1 | L]
(q = p - 1 columns, intercept first) and the SNP column last, y_j the j-th trait,
M_j = sigma_j^2 (h_j^2 Phi + (1 - h_j^2) I).

Readings where the paper is silent or garbled:
  * Var(b) = (X^T M^-1 X)^-1.  Eq. "probDef" multiplies by sigma^2 again although M already
    contains sigma^2; we take the standard GLS covariance (both coincide when sigma^2 = 1).
  * Wald statistic for the SNP effect: chi2 = b_snp^2 / Var(b)_snp,snp (the paper only says
    "p-values"); for a genetic model of p_R > 1 columns (e.g. additive and dominance codes),
    the joint statistic of the block, b_R^T Var(b)_RR^-1 b_R with p_R degrees of freedom.
  * Algorithm 2 / Eq. "Eig0": M^-1 = Z D Z^T with D = diag(1 / (sigma^2 (h^2 w_k + 1 - h^2))),
    K = D^(1/2) (the printed Z D^-1 Z^T double-inverts D).
  * A GLS whose p x p normal matrix S is numerically singular (a Cholesky pivot d_k with
    d_k <= tol * S_kk, e.g. a monomorphic SNP) yields NaN for b, Var and chi2.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

SINGULAR_TOL = 1e-12


def form_M(Phi: np.ndarray, h2: float, s2: float) -> np.ndarray:
    """Variance-components covariance, Supplementary Note Section 1 / Algorithm 1:
    M = sigma^2 (h^2 Phi + (1 - h^2) I)."""
    n = Phi.shape[0]
    return s2 * (h2 * Phi + (1.0 - h2) * np.eye(n))


def _small_cholesky(S: np.ndarray, tol: float = SINGULAR_TOL):
    """Cholesky of a batch of p x p SPD matrices S (N, p, p), column by column.

    Returns (L, ok): ok[k] is False where a pivot fell to <= tol * S_kk (singular GLS)."""
    N, p, _ = S.shape
    L = np.zeros_like(S)
    ok = np.ones(N, dtype=bool)
    for k in range(p):
        d = S[:, k, k] - np.sum(L[:, k, :k] ** 2, axis=1)
        ok &= d > tol * S[:, k, k]
        dk = np.sqrt(np.where(ok, d, 1.0))
        L[:, k, k] = dk
        for i in range(k + 1, p):
            L[:, i, k] = (S[:, i, k] - np.sum(L[:, i, :k] * L[:, k, :k], axis=1)) / dk
    return L, ok


def _small_spd_solve(S: np.ndarray, r: np.ndarray):
    """b = S^-1 r and Var = S^-1 for a batch, through S = L L^T (Algorithm 1, last two lines)."""
    N, p, _ = S.shape
    L, ok = _small_cholesky(S)
    # L^-1 by forward substitution on the identity, row by row.
    Linv = np.zeros_like(L)
    for i in range(p):
        Linv[:, i, i] = 1.0 / L[:, i, i]
        for j in range(i):
            Linv[:, i, j] = -np.sum(L[:, i, j:i] * Linv[:, j:i, j], axis=1) / L[:, i, i]
    Var = np.einsum("nki,nkj->nij", Linv, Linv)
    b = np.einsum("nij,nj->ni", Var, r)
    b[~ok] = np.nan
    Var[~ok] = np.nan
    return b, Var, ok


def wald_from(b: np.ndarray, var_diag: np.ndarray) -> np.ndarray:
    """Wald chi-square (1 d.o.f.) of the SNP coefficient (last): b_snp^2 / Var_snp,snp."""
    return b[..., -1] ** 2 / var_diag[..., -1]


# Genetic models.  Table 1's p, the width of X, is set by the covariates and by "the genetic
# model assumed": the block X_R,i a SNP contributes has one column per coding, a coding being
# the column's value for the hard calls x = 0, 1, 2.
GENETIC_MODELS = {
    "additive": ((0, 1, 2),),            # allele count
    "dominant": ((0, 1, 1),),            # carries at least one copy
    "recessive": ((0, 0, 1),),           # carries two copies
    "add_dom": ((0, 1, 2), (0, 1, 0)),   # allele count and heterozygosity (2 columns)
}


def codings_of(model):
    """The codings of a genetic model: a name of GENETIC_MODELS or a tuple of codings."""
    return GENETIC_MODELS[model] if isinstance(model, str) else tuple(tuple(c) for c in model)


def genetic_columns(XR_rows: np.ndarray, model="additive") -> np.ndarray:
    """X_R,i of k SNPs: (k, n) hard calls -> (n, k, p_R) float64, column c = coding c of x."""
    x = np.asarray(XR_rows).astype(np.int64)
    cols = [np.asarray(cd, dtype=np.float64)[x] for cd in codings_of(model)]
    return np.stack(cols, axis=-1).transpose(1, 0, 2)


def wald_block(b: np.ndarray, Var: np.ndarray, p_r: int) -> np.ndarray:
    """Wald statistic of the genetic block (the last p_r coefficients), b_R^T Var_RR^-1 b_R,
    chi-square with p_r d.o.f. (p_r = 1: b_snp^2 / Var_snp,snp).  NaN where Var is NaN."""
    bR = b[..., -p_r:]
    VR = Var[..., -p_r:, -p_r:]
    out = np.full(bR.shape[:-1], np.nan)
    ok = np.all(np.isfinite(VR), axis=(-1, -2)) & np.all(np.isfinite(bR), axis=-1)
    if np.any(ok):
        sol = np.linalg.solve(VR[ok], bR[ok][..., None])[..., 0]
        out[ok] = np.sum(bR[ok] * sol, axis=-1)
    return out


# ---------------------------------------------------------------------------------------------
# Single GLS (Supplementary Note Section 2)
# ---------------------------------------------------------------------------------------------

def gls_chol(Phi, X, y, h2, s2):
    """Algorithm 1 (CLAK-Chol, one GLS): M; L L^T = M; X := L^-1 X; y := L^-1 y;
    S := X^T X; b := X^T y; b := S^-1 b.  Returns (b, Var) with Var = S^-1."""
    M = form_M(Phi, h2, s2)
    L = np.linalg.cholesky(M)
    Xw = solve_triangular(L, X, lower=True)
    yw = solve_triangular(L, y, lower=True)
    S = Xw.T @ Xw
    r = Xw.T @ yw
    b, Var, _ = _small_spd_solve(S[None], r[None])
    return b[0], Var[0]


def gls_eig(Phi, X, y, h2, s2, Z=None, w=None):
    """Algorithm 2 (CLAK-Eig, one GLS): Z W Z^T = Phi; D := (sigma^2 (h^2 W + (1-h^2) I))^-1;
    K K^T = D; V := X^T Z K; S := V V^T; b := V K^T Z^T y; b := S^-1 b.
    An eigenbasis (Z, w) may be passed in to test that any orthonormal basis works."""
    if Z is None:
        w, Z = np.linalg.eigh(Phi)
    D = 1.0 / (s2 * (h2 * w + (1.0 - h2)))
    K = np.sqrt(D)
    V = (X.T @ Z) * K[None, :]
    S = V @ V.T
    r = V @ (K * (Z.T @ y))
    b, Var, _ = _small_spd_solve(S[None], r[None])
    return b[0], Var[0]


# ---------------------------------------------------------------------------------------------
# The 2-D problem (Eq. "probDef"), by definition
# ---------------------------------------------------------------------------------------------

def gls_grid(Phi, XL, XR, Y, h2, s2, snps=None, traits=None, chunk=512, full_var=False,
             model="additive"):
    """Eq. "probDef": for every (SNP i, trait j) solve b_ij = (X_i^T M_j^-1 X_i)^-1 X_i^T M_j^-1 y_j
    with X_i = [X_L | X_R,i], each problem by Algorithm 1.  X_R,i is the SNP's genotype column
    (model "additive") or the p_R columns of another genetic model (genetic_columns).

    XR is (m, n) int8 (SNP-major), Y is (n, t).  Forming and factoring M_j (Algorithm 1) and
    L_j^-1 y_j do not depend on i and are computed once per trait; Algorithm 1's whitening of
    X_i is one triangular solve for many SNPs' X_i.  Returns
    B (len(snps), len(traits), p), W (same, the Wald statistic of the genetic block, p_R
    d.o.f.) and Vd (same shape as B: diag of Var), p = q + p_R; with full_var also
    V (len(snps), len(traits), p, p), the whole Var(b) = (X_i^T M_j^-1 X_i)^-1 of
    Eq. "probDef"."""
    XL = np.asarray(XL, dtype=np.float64)
    n, q = XL.shape
    p_r = len(codings_of(model))
    p = q + p_r
    snps = np.arange(XR.shape[0]) if snps is None else np.asarray(snps)
    traits = np.arange(Y.shape[1]) if traits is None else np.asarray(traits)
    B = np.empty((len(snps), len(traits), p))
    W = np.empty((len(snps), len(traits)))
    Vd = np.empty((len(snps), len(traits), p))
    V = np.empty((len(snps), len(traits), p, p)) if full_var else None
    for jj, j in enumerate(traits):
        M = form_M(Phi, float(h2[j]), float(s2[j]))
        L = np.linalg.cholesky(M)
        yw = solve_triangular(L, Y[:, j], lower=True)
        for s0 in range(0, len(snps), chunk):
            idx = snps[s0:s0 + chunk]
            k = len(idx)
            X = np.empty((n, k, p))
            X[:, :, :q] = XL[:, None, :]
            X[:, :, q:] = genetic_columns(XR[idx], model)
            Xw = solve_triangular(L, X.reshape(n, k * p), lower=True).reshape(n, k, p)
            S = np.einsum("rki,rkj->kij", Xw, Xw)
            r = np.einsum("rki,r->ki", Xw, yw)
            b, Var, _ = _small_spd_solve(S, r)
            B[s0:s0 + k, jj] = b
            W[s0:s0 + k, jj] = wald_block(b, Var, p_r)
            Vd[s0:s0 + k, jj] = np.diagonal(Var, axis1=1, axis2=2)
            if full_var:
                V[s0:s0 + k, jj] = Var
    return (B, W, Vd, V) if full_var else (B, W, Vd)


def gls_pairs(Phi, XL, XR, Y, h2, s2, pairs, model="additive"):
    """Eq. "probDef" on a list of (i, j) pairs, grouped by trait so each M_j is factored once.
    Returns B (len(pairs), p), W, Vd in the order of `pairs`."""
    pairs = np.asarray(pairs).reshape(-1, 2)
    p = XL.shape[1] + len(codings_of(model))
    B = np.empty((len(pairs), p))
    W = np.empty(len(pairs))
    Vd = np.empty((len(pairs), p))
    for j in np.unique(pairs[:, 1]):
        sel = np.flatnonzero(pairs[:, 1] == j)
        b, w, v = gls_grid(Phi, XL, XR, Y, h2, s2, snps=pairs[sel, 0], traits=[j], model=model)
        B[sel] = b[:, 0]
        W[sel] = w[:, 0]
        Vd[sel] = v[:, 0]
    return B, W, Vd


# ---------------------------------------------------------------------------------------------
# Sequence algorithms, in the paper's order (Supplementary Note Section 3)
# ---------------------------------------------------------------------------------------------

def chol_sequence(Phi, XL, XR, y, h2, s2, model="additive"):
    """Algorithm 3 (CLAK-Chol, single trait): M; L L^T = M; X_L := L^-1 X_L; X_R := L^-1 X_R;
    y := L^-1 y; S_TL := X_L^T X_L; b_T := X_L^T y; then for each SNP i the bordered system
    S = [[S_TL, *], [X_Ri^T X_L, X_Ri^T X_Ri]], b_i = [b_T; X_Ri^T y], b_i := S^-1 b_i, with
    X_Ri the SNP's p_R columns of the genetic model.  Returns B (m, p), W (m,), Vd (m, p)."""
    n, q = XL.shape
    m = XR.shape[0]
    p_r = len(codings_of(model))
    M = form_M(Phi, h2, s2)
    L = np.linalg.cholesky(M)
    XLw = solve_triangular(L, XL, lower=True)
    XRw = solve_triangular(L, genetic_columns(XR, model).reshape(n, m * p_r),
                           lower=True).reshape(n, m, p_r)
    yw = solve_triangular(L, y, lower=True)
    S_TL = XLw.T @ XLw
    b_T = XLw.T @ yw
    S = np.empty((m, q + p_r, q + p_r))
    S[:, :q, :q] = S_TL
    S[:, q:, :q] = np.einsum("rmc,rk->mck", XRw, XLw)
    S[:, :q, q:] = np.transpose(S[:, q:, :q], (0, 2, 1))
    S[:, q:, q:] = np.einsum("rmc,rmd->mcd", XRw, XRw)
    rhs = np.empty((m, q + p_r))
    rhs[:, :q] = b_T
    rhs[:, q:] = np.einsum("rmc,r->mc", XRw, yw)
    b, Var, _ = _small_spd_solve(S, rhs)
    Vd = np.diagonal(Var, axis1=1, axis2=2).copy()
    return b, wald_block(b, Var, p_r), Vd


def eig_sequence(Phi, XL, XR, Y, h2, s2, Z=None, w=None, model="additive"):
    """Algorithm 4 (CLAK-Eig, many traits): Z W Z^T = Phi; X_L := Z^T X_L; X_R := Z^T X_R;
    Y := Z^T Y; for each trait j: D := (sigma_j^2 (h_j^2 W + (1-h_j^2) I))^-1, K K^T = D,
    Y_j := K^T Y_j, W_L := K^T X_L, S_TL := W_L^T W_L, b_T := W_L^T Y_j; for each SNP i:
    W_R := K^T X_Ri, S = [[S_TL, *], [W_R^T W_L, W_R^T W_R]], b_ij = [b_T; W_R^T Y_j],
    b_ij := S^-1 b_ij.  Returns B (m, t, p), W (m, t), Vd (m, t, p)."""
    if Z is None:
        w, Z = np.linalg.eigh(Phi)
    n, q = XL.shape
    m = XR.shape[0]
    t = Y.shape[1]
    p_r = len(codings_of(model))
    XLt = Z.T @ XL
    XRt = (Z.T @ genetic_columns(XR, model).reshape(n, m * p_r)).reshape(n, m, p_r)
    Yt = Z.T @ Y
    B = np.empty((m, t, q + p_r))
    W = np.empty((m, t))
    Vd = np.empty((m, t, q + p_r))
    for j in range(t):
        D = 1.0 / (s2[j] * (h2[j] * w + (1.0 - h2[j])))
        K = np.sqrt(D)
        yj = K * Yt[:, j]
        WL = K[:, None] * XLt
        S_TL = WL.T @ WL
        b_T = WL.T @ yj
        WR = K[:, None, None] * XRt  # n x m x p_R: all SNPs' W_R at once
        S = np.empty((m, q + p_r, q + p_r))
        S[:, :q, :q] = S_TL
        S[:, q:, :q] = np.einsum("rmc,rk->mck", WR, WL)
        S[:, :q, q:] = np.transpose(S[:, q:, :q], (0, 2, 1))
        S[:, q:, q:] = np.einsum("rmc,rmd->mcd", WR, WR)
        rhs = np.empty((m, q + p_r))
        rhs[:, :q] = b_T
        rhs[:, q:] = np.einsum("rmc,r->mc", WR, yj)
        b, Var, _ = _small_spd_solve(S, rhs)
        B[:, j] = b
        W[:, j] = wald_block(b, Var, p_r)
        Vd[:, j] = np.diagonal(Var, axis1=1, axis2=2)
    return B, W, Vd


# ---------------------------------------------------------------------------------------------
# Error measures used by every parity check
# ---------------------------------------------------------------------------------------------

def rel_err_b(b, b_ref, vd_ref):
    """Per-coefficient error |b - b_ref| / max(|b_ref|, sqrt(Var_ref,kk)): relative where the
    estimate is large, in standard-error units where it is near zero (SNP effects under the null)."""
    scale = np.maximum(np.abs(b_ref), np.sqrt(vd_ref))
    return np.abs(b - b_ref) / scale


def rel_err_wald(w, w_ref):
    """|chi2 - chi2_ref| / max(chi2_ref, 1)."""
    return np.abs(w - w_ref) / np.maximum(np.abs(w_ref), 1.0)


def max_rel_errors(b, w, b_ref, w_ref, vd_ref):
    """Largest rel_err_b and rel_err_wald over the checked pairs, for parity checks.

    A singular GLS is NaN on both sides, so NaN must sit exactly where the reference has it: an
    output that is NaN where the reference is finite (or finite where it is NaN) -- e.g. a pair
    a kernel never wrote into a NaN-filled buffer -- makes both errors infinite instead of being
    skipped.  Pairs NaN on both sides are left out of the maxima."""
    b, w = np.asarray(b, dtype=np.float64), np.asarray(w, dtype=np.float64)
    nb, nbr = np.isnan(b), np.isnan(b_ref)
    nw, nwr = np.isnan(w), np.isnan(w_ref)
    if nb.shape != nbr.shape or nw.shape != nwr.shape:
        raise ValueError("output and reference shapes differ")
    if not (np.array_equal(nb, nbr) and np.array_equal(nw, nwr)):
        return float("inf"), float("inf")
    eb = rel_err_b(b, b_ref, vd_ref)[~nbr]
    ew = rel_err_wald(w, w_ref)[~nwr]
    return (float(eb.max()) if eb.size else 0.0, float(ew.max()) if ew.size else 0.0)

