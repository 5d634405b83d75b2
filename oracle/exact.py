"""The GLS definition in exact rational arithmetic (test infrastructure only).

Only tests/ (and the committed script that writes tests/golden/) import this module.  It
solves Eq. "GLS" (Supplementary Note Section 1),
    b = (X^T M^-1 X)^-1 X^T M^-1 y,   Var = (X^T M^-1 X)^-1,   M = s2 (h2 Phi + (1 - h2) I),
with Python Fractions and Gauss-Jordan elimination: no Cholesky, no whitening, no eigenbasis,
no rounding.  It is meant for n <= 10.
"""
from __future__ import annotations

from fractions import Fraction


def _solve(A, B):
    """Exact A^-1 B for a square nonsingular rational A (list of rows) and B (list of rows)."""
    n = len(A)
    k = len(B[0])
    T = [list(A[i]) + list(B[i]) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if T[r][c] != 0)
        T[c], T[piv] = T[piv], T[c]
        inv = 1 / T[c][c]
        T[c] = [v * inv for v in T[c]]
        for r in range(n):
            if r != c and T[r][c] != 0:
                f = T[r][c]
                T[r] = [a - f * b for a, b in zip(T[r], T[c])]
    return [row[n:n + k] for row in T]


def gls_exact(Phi, X, y, h2, s2):
    """Exact (b, Var) of one GLS.  Phi: n x n, X: n x p, y: n (all Fractions or ints)."""
    n = len(Phi)
    p = len(X[0])
    h2 = Fraction(h2)
    s2 = Fraction(s2)
    M = [[s2 * (h2 * Fraction(Phi[i][j]) + ((1 - h2) if i == j else 0)) for j in range(n)]
         for i in range(n)]
    rhs = [[Fraction(X[i][c]) for c in range(p)] + [Fraction(y[i])] for i in range(n)]
    MinvXy = _solve(M, rhs)
    S = [[sum(Fraction(X[r][a]) * MinvXy[r][b] for r in range(n)) for b in range(p)]
         for a in range(p)]
    rr = [[sum(Fraction(X[r][a]) * MinvXy[r][p] for r in range(n))] for a in range(p)]
    eye = [[Fraction(int(a == b)) for b in range(p)] for a in range(p)]
    Var = _solve(S, eye)
    b = [sum(Var[a][c] * rr[c][0] for c in range(p)) for a in range(p)]
    return b, Var


def wald_exact(b, var, p_r):
    """b_R^T Var_RR^-1 b_R of the last p_r coefficients, exactly (p_r = 1: b^2 / Var)."""
    bR = b[-p_r:]
    VR = [row[-p_r:] for row in var[-p_r:]]
    sol = _solve(VR, [[v] for v in bR])
    return sum(bR[k] * sol[k][0] for k in range(p_r))


def grid_exact(Phi, XL, XR, Y, h2, s2, codings=((0, 1, 2),)):
    """Eq. "probDef" exactly: XL n x q, XR m x n (ints), Y n x t, h2/s2 length t.  The SNP's
    block X_R,i has one column per coding (the column's values for hard calls 0, 1, 2; the
    default is the genotype itself).  Returns B[i][j] (list of p Fractions), V[i][j] (p x p)
    and W[i][j] = b_R^T Var_RR^-1 b_R over the genetic block (b_snp^2 / Var_snp for one column)."""
    n = len(Phi)
    m = len(XR)
    t = len(Y[0])
    B, V, W = [], [], []
    for i in range(m):
        X = [list(XL[r]) + [cd[XR[i][r]] for cd in codings] for r in range(n)]
        Bi, Vi, Wi = [], [], []
        for j in range(t):
            b, var = gls_exact(Phi, X, [Y[r][j] for r in range(n)], h2[j], s2[j])
            Bi.append(b)
            Vi.append(var)
            Wi.append(wald_exact(b, var, len(codings)))
        B.append(Bi)
        V.append(Vi)
        W.append(Wi)
    return B, V, W
