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
    "p-values").
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

def gls_grid(Phi, XL, XR, Y, h2, s2, snps=None, traits=None, chunk=512, full_var=False):
    """Eq. "probDef": for every (SNP i, trait j) solve b_ij = (X_i^T M_j^-1 X_i)^-1 X_i^T M_j^-1 y_j
    with X_i = [X_L | x_i], each problem by Algorithm 1.

    XR is (m, n) int8 (SNP-major), Y is (n, t).  Forming and factoring M_j (Algorithm 1) and
    L_j^-1 y_j do not depend on i and are computed once per trait; Algorithm 1's whitening of
    X_i is one triangular solve for many SNPs' X_i.  Returns
    B (len(snps), len(traits), p), W (same, chi2) and Vd (same shape as B: diag of Var); with
    full_var also V (len(snps), len(traits), p, p), the whole Var(b) = (X_i^T M_j^-1 X_i)^-1 of
    Eq. "probDef"."""
    XL = np.asarray(XL, dtype=np.float64)
    n, q = XL.shape
    p = q + 1
    snps = np.arange(XR.shape[0]) if snps is None else np.asarray(snps)
    traits = np.arange(Y.shape[1]) if traits is None else np.asarray(traits)
    B = np.empty((len(snps), len(traits), p))
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
            X[:, :, q] = XR[idx].T.astype(np.float64)
            Xw = solve_triangular(L, X.reshape(n, k * p), lower=True).reshape(n, k, p)
            S = np.einsum("rki,rkj->kij", Xw, Xw)
            r = np.einsum("rki,r->ki", Xw, yw)
            b, Var, _ = _small_spd_solve(S, r)
            B[s0:s0 + k, jj] = b
            Vd[s0:s0 + k, jj] = np.diagonal(Var, axis1=1, axis2=2)
            if full_var:
                V[s0:s0 + k, jj] = Var
    W = wald_from(B, Vd)
    return (B, W, Vd, V) if full_var else (B, W, Vd)


def gls_pairs(Phi, XL, XR, Y, h2, s2, pairs):
    """Eq. "probDef" on a list of (i, j) pairs, grouped by trait so each M_j is factored once.
    Returns B (len(pairs), p), W, Vd in the order of `pairs`."""
    pairs = np.asarray(pairs).reshape(-1, 2)
    q = XL.shape[1]
    B = np.empty((len(pairs), q + 1))
    Vd = np.empty((len(pairs), q + 1))
    for j in np.unique(pairs[:, 1]):
        sel = np.flatnonzero(pairs[:, 1] == j)
        b, _, v = gls_grid(Phi, XL, XR, Y, h2, s2, snps=pairs[sel, 0], traits=[j])
        B[sel] = b[:, 0]
        Vd[sel] = v[:, 0]
    return B, wald_from(B, Vd), Vd


# ---------------------------------------------------------------------------------------------
# Sequence algorithms, in the paper's order (Supplementary Note Section 3)
# ---------------------------------------------------------------------------------------------

def chol_sequence(Phi, XL, XR, y, h2, s2):
    """Algorithm 3 (CLAK-Chol, single trait): M; L L^T = M; X_L := L^-1 X_L; X_R := L^-1 X_R;
    y := L^-1 y; S_TL := X_L^T X_L; b_T := X_L^T y; then for each SNP i the bordered system
    S = [[S_TL, *], [X_Ri^T X_L, X_Ri^T X_Ri]], b_i = [b_T; X_Ri^T y], b_i := S^-1 b_i.
    Returns B (m, p), W (m,), Vd (m, p)."""
    n, q = XL.shape
    M = form_M(Phi, h2, s2)
    L = np.linalg.cholesky(M)
    XLw = solve_triangular(L, XL, lower=True)
    XRw = solve_triangular(L, XR.T.astype(np.float64), lower=True)  # n x m
    yw = solve_triangular(L, y, lower=True)
    S_TL = XLw.T @ XLw
    b_T = XLw.T @ yw
    m = XR.shape[0]
    S = np.empty((m, q + 1, q + 1))
    S[:, :q, :q] = S_TL
    S[:, q, :q] = XRw.T @ XLw
    S[:, :q, q] = S[:, q, :q]
    S[:, q, q] = np.sum(XRw * XRw, axis=0)
    rhs = np.empty((m, q + 1))
    rhs[:, :q] = b_T
    rhs[:, q] = XRw.T @ yw
    b, Var, _ = _small_spd_solve(S, rhs)
    Vd = np.diagonal(Var, axis1=1, axis2=2).copy()
    return b, wald_from(b, Vd), Vd


def eig_sequence(Phi, XL, XR, Y, h2, s2, Z=None, w=None):
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
    XLt = Z.T @ XL
    XRt = Z.T @ XR.T.astype(np.float64)  # n x m
    Yt = Z.T @ Y
    B = np.empty((m, t, q + 1))
    Vd = np.empty((m, t, q + 1))
    for j in range(t):
        D = 1.0 / (s2[j] * (h2[j] * w + (1.0 - h2[j])))
        K = np.sqrt(D)
        yj = K * Yt[:, j]
        WL = K[:, None] * XLt
        S_TL = WL.T @ WL
        b_T = WL.T @ yj
        WR = K[:, None] * XRt  # n x m: all SNPs' W_R at once
        S = np.empty((m, q + 1, q + 1))
        S[:, :q, :q] = S_TL
        S[:, q, :q] = WR.T @ WL
        S[:, :q, q] = S[:, q, :q]
        S[:, q, q] = np.sum(WR * WR, axis=0)
        rhs = np.empty((m, q + 1))
        rhs[:, :q] = b_T
        rhs[:, q] = WR.T @ yj
        b, Var, _ = _small_spd_solve(S, rhs)
        B[:, j] = b
        Vd[:, j] = np.diagonal(Var, axis1=1, axis2=2)
    return B, wald_from(B, Vd), Vd


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

