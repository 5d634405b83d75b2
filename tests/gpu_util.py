"""Helpers shared by the GPU parity tests: run the library through its C ABI, compare with the
oracle using the error measures of oracle.gls (relative where large, in standard errors near 0)."""
import numpy as np

from oracle import gls


def run(g, c, algo, precision, XR=None, device=True, block_snps=0, f64=False, packed=False,
        validate=False, out_mode="full", model="additive"):
    """packed: pass the genotypes as packed rows (gwas_pack_genotypes on the host, then
    gwas_scan_packed) instead of int8 rows (gwas_scan).  model: the genetic model (p_R columns
    per SNP, p = q + p_R)."""
    import torch
    XR = c.XR if XR is None else XR
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, algo=algo, precision=precision,
                     block_snps=block_snps, validate_genotypes=int(validate), out_mode=out_mode,
                     genetic_model=model)
    try:
        pr = g.gwas_genetic_columns(h)
        pp = c.q + pr
        pv = pp + pp * (pp + 1) // 2
        m, t, p = XR.shape[0], c.t, {"snp": 2 * pr, "var": pv}.get(out_mode, pp)
        dt = torch.float64 if f64 else torch.float32
        dev = "cuda" if device else "cpu"
        X = np.ascontiguousarray(XR)
        if packed:
            X = g.gwas_pack_genotypes(X)
        xr = torch.from_numpy(X).to(dev)
        B = torch.full((m, t, p), float("nan"), dtype=dt, device=dev)
        W = torch.full((m, t), float("nan"), dtype=dt, device=dev)
        if packed:
            assert not f64
            g.gwas_scan_packed(h, xr, B, W)
        else:
            (g.gwas_scan_f64 if f64 else g.gwas_scan)(h, xr, B, W)
        if device:
            torch.cuda.synchronize()
        nsing = g.gwas_singular_count(h)
        return B.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64), nsing
    finally:
        g.gwas_destroy(h)


def max_errors(B, W, Bref, Wref, Vref):
    """Max errors; NaN must appear exactly where the oracle's (an unwritten pair of the
    NaN-filled buffers of run() is then an infinite error, not a skipped one)."""
    return gls.max_rel_errors(B, W, Bref, Wref, Vref)
