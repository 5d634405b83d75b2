"""Plain FP64 oracle for step 1 of the two-step method (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs import this
module; it shares no code with the CUDA library.

The reduced model (Supplementary Note Section 1, "Mixed Models for GWAS"): y = X_L beta + R with
R ~ N(0, sigma^2 (h^2 Phi + (1 - h^2) I)), X_L = [1 | L].  Step 1 fits it per trait and returns
the estimates (h^2, sigma^2) that step 2 plugs into M_j.  The paper names Maximum Likelihood
(GenABEL, FaST-LMM) and Restricted Maximum Likelihood (EMMAX) as the criteria and an iterative
search as the method (Supplementary Note, "Time complexity"), without writing the likelihoods
out; the ones below are the standard Gaussian (restricted) log-likelihoods of that model.

Notation: h stands for h^2 and H(h) = h Phi + (1 - h) I, so M = sigma^2 H(h).

Readings where the paper leaves a choice open:
  * ML: sigma^2 and beta are profiled out; the criterion is the log-likelihood maximised over them,
      l(h) = -1/2 [ n log(2 pi s2(h)) + log|H(h)| + n ],  s2(h) = r^T H^-1 r / n,
    with r = y - X_L beta(h) the GLS residual.
  * REML: the log-density of the error contrasts (Harville 1974), with sigma^2 profiled out,
      l_R(h) = -1/2 [ (n-q) log(2 pi s2(h)) + log|H| + log|X_L^T H^-1 X_L| - log|X_L^T X_L| + (n-q) ],
      s2(h) = r^T H^-1 r / (n - q).
  * Search interval h in [0, H2_MAX] (the model allows [0, 1]; setup of step 2 needs h < 1):
    the criterion on the grid h_g = (g / GRID) H2_MAX, g = 0..GRID, then a bounded scalar search
    between the best grid point's neighbours; the better of the two is the estimate.
  * A trait fitted exactly by X_L has no finite estimate: NaN for h and the criterion, 0 for
    sigma^2.  "Exactly" is r^T H^-1 r <= 1e-12 y^T H^-1 y (R^2 within 1e-12 of 1), a margin
    above the rounding of FP64 sums of n products, so that a computation of r^T H^-1 r as
    y^T H^-1 y minus the fitted part reaches the same decision.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cho_solve, cholesky, solve_triangular
from scipy.optimize import minimize_scalar

H2_MAX = 0.999
GRID = 100
EXACT_FIT = 1e-12  # r^T H^-1 r at most this fraction of y^T H^-1 y: y lies in the span of X_L
ML, REML = 0, 1


def kinship_cov(Phi: np.ndarray, h: float) -> np.ndarray:
    """H(h) = h Phi + (1 - h) I, the covariance of R divided by sigma^2 (Section 1)."""
    n = Phi.shape[0]
    return h * Phi + (1.0 - h) * np.eye(n)


def profile(Phi, XL, y, h, method=ML):
    """Criterion at h with beta and sigma^2 profiled out, from the definition: H formed
    explicitly, factored H = L L^T, the GLS of y on X_L in the whitened space.

    Returns (criterion, sigma2_hat, beta_hat)."""
    n, q = XL.shape
    L = cholesky(kinship_cov(Phi, h), lower=True)
    Xw = solve_triangular(L, XL, lower=True)
    yw = solve_triangular(L, y, lower=True)
    S = Xw.T @ Xw
    Sc = cholesky(S, lower=True)
    beta = cho_solve((Sc, True), Xw.T @ yw)
    r = yw - Xw @ beta
    Q = float(r @ r)
    logdet_H = 2.0 * np.sum(np.log(np.diag(L)))
    if not Q > EXACT_FIT * float(yw @ yw):
        return np.nan, 0.0, beta
    if method == ML:
        s2 = Q / n
        crit = -0.5 * (n * np.log(2 * np.pi * s2) + logdet_H + n)
    else:
        s2 = Q / (n - q)
        logdet_S = 2.0 * np.sum(np.log(np.diag(Sc)))
        logdet_XtX = np.linalg.slogdet(XL.T @ XL)[1]
        crit = -0.5 * ((n - q) * np.log(2 * np.pi * s2) + logdet_H + logdet_S - logdet_XtX +
                       (n - q))
    return crit, s2, beta


def estimate(Phi, XL, Y, method=ML, grid=GRID, h_max=H2_MAX, xatol=1e-10):
    """Per trait (column of Y): (h2_hat, s2_hat, criterion) by grid + bounded scalar search.

    Returns three arrays of length t."""
    Y = np.asarray(Y, dtype=np.float64).reshape(Phi.shape[0], -1)
    t = Y.shape[1]
    hs = (np.arange(grid + 1) / grid) * h_max
    h2 = np.empty(t)
    s2 = np.empty(t)
    ll = np.empty(t)
    for j in range(t):
        y = Y[:, j]
        vals = np.array([profile(Phi, XL, y, h, method)[0] for h in hs])
        if np.all(np.isnan(vals)):
            h2[j], s2[j], ll[j] = np.nan, 0.0, np.nan
            continue
        g = int(np.nanargmax(vals))
        lo, hi = hs[max(g - 1, 0)], hs[min(g + 1, grid)]
        res = minimize_scalar(lambda h: -profile(Phi, XL, y, h, method)[0], bounds=(lo, hi),
                              method="bounded", options={"xatol": xatol})
        best_h, best = (res.x, -res.fun) if -res.fun >= vals[g] else (hs[g], vals[g])
        crit, s2_hat, _ = profile(Phi, XL, y, best_h, method)
        h2[j], s2[j], ll[j] = best_h, s2_hat, crit
    return h2, s2, ll
