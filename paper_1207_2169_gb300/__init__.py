"""Python binding of libgwasgb.so (include/gwas.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no arithmetic of the
method: it checks shapes/dtypes, passes pointers (NumPy arrays or torch tensors, host or CUDA)
and raises GwasError on a non-zero status.  The library must have been built
(`python paper_1207_2169_gb300/_build.py` or __graft_entry__.build()); importing this module
without it raises ImportError -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgwasgb.so")

ALGO = {"auto": 0, "chol": 1, "eig": 2}
PRECISION = {"fp64": 0, "fp32": 1, "split_bf16": 2, "split_fp8": 3}
OUT_MODE = {"full": 0, "snp": 1, "var": 2}
GENETIC_MODEL = {"additive": 0, "dominant": 1, "recessive": 2, "add_dom": 3}
STATUS = {0: "GWAS_OK", -1: "GWAS_ERR_ARG", -2: "GWAS_ERR_NOT_SPD", -3: "GWAS_ERR_CUDA",
          -4: "GWAS_ERR_OOM", -5: "GWAS_ERR_UNSUPPORTED", -6: "GWAS_ERR_GENOTYPE",
          -7: "GWAS_ERR_TIMEOUT", -8: "GWAS_ERR_SINGULAR", -9: "GWAS_ERR_NOT_CONVERGED"}

# every symbol include/gwas.h declares
EXPORTS = ["gwas_default_options", "gwas_setup", "gwas_scan", "gwas_scan_f64",
           "gwas_packed_row_bytes", "gwas_pack_genotypes", "gwas_scan_packed", "gwas_shard",
           "gwas_setup_batch", "gwas_scan_batch", "gwas_batch_plan", "gwas_batch_handle",
           "gwas_destroy_batch", "gwas_sync", "gwas_selftest_timeout", "gwas_wald_pvalues",
           "gwas_wald_pvalues_dof",
           "gwas_estimate",
           "gwas_scan_static", "gwas_setup_timing", "gwas_info", "gwas_singular_count",
           "gwas_genetic_columns", "gwas_split_pieces", "gwas_fp8_traits", "gwas_eig_chunk",
           "gwas_chol_routed_traits",
           "gwas_batch_tuning", "gwas_stream_info",
           "gwas_stage_timing", "gwas_stage_times", "gwas_last_error", "gwas_destroy"]

STAGES = ["pack", "centres", "chol", "rot", "sq", "ac", "simt"]
NSTAGES = 8


class GwasError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class gwas_cohort(ctypes.Structure):
    _fields_ = [("Phi", ctypes.c_void_p), ("n", ctypes.c_int), ("XL", ctypes.c_void_p),
                ("q", ctypes.c_int), ("Y", ctypes.c_void_p), ("t", ctypes.c_int),
                ("h2", ctypes.c_void_p), ("s2", ctypes.c_void_p)]


class gwas_cohort_block(ctypes.Structure):
    _fields_ = [("G", ctypes.c_void_p), ("m", ctypes.c_int64), ("B", ctypes.c_void_p),
                ("wald", ctypes.c_void_p)]


class gwas_options(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("precision", ctypes.c_int), ("block_snps", ctypes.c_int),
                ("validate_genotypes", ctypes.c_int), ("device", ctypes.c_int),
                ("out_mode", ctypes.c_int), ("genetic_model", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python paper_1207_2169_gb300/_build.py` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    lib.gwas_default_options.argtypes = [ctypes.POINTER(gwas_options)]
    lib.gwas_default_options.restype = None
    lib.gwas_setup.argtypes = [vp, i32, vp, i32, vp, i32, vp, vp, ctypes.POINTER(gwas_options),
                               ctypes.POINTER(vp)]
    lib.gwas_setup.restype = i32
    for f in (lib.gwas_scan, lib.gwas_scan_f64, lib.gwas_scan_packed):
        f.argtypes = [vp, vp, i64, i32, vp, vp, i32, vp]
        f.restype = i32
    lib.gwas_estimate.argtypes = [vp, i32, vp, i32, vp, i32, i32, i32, vp, vp, vp, vp]
    lib.gwas_estimate.restype = i32
    lib.gwas_packed_row_bytes.argtypes = [i32]
    lib.gwas_packed_row_bytes.restype = i32
    lib.gwas_shard.argtypes = [i64, i32, i32, i64, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64)]
    lib.gwas_pack_genotypes.argtypes = [vp, i64, i32, vp, i32, vp]
    lib.gwas_pack_genotypes.restype = i32
    lib.gwas_setup_batch.argtypes = [i32, ctypes.POINTER(gwas_cohort), ctypes.POINTER(gwas_options),
                                     ctypes.POINTER(vp)]
    lib.gwas_setup_batch.restype = i32
    lib.gwas_scan_batch.argtypes = [vp, ctypes.POINTER(gwas_cohort_block), vp]
    lib.gwas_scan_batch.restype = i32
    lib.gwas_batch_plan.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp]
    lib.gwas_batch_plan.restype = i32
    lib.gwas_batch_handle.argtypes = [vp, i32]
    lib.gwas_batch_handle.restype = vp
    lib.gwas_destroy_batch.argtypes = [vp]
    lib.gwas_destroy_batch.restype = None
    lib.gwas_wald_pvalues.argtypes = [vp, i64, vp, i32, vp]
    lib.gwas_wald_pvalues.restype = i32
    lib.gwas_wald_pvalues_dof.argtypes = [vp, i64, i32, vp, i32, vp]
    lib.gwas_sync.argtypes = [vp]
    lib.gwas_sync.restype = i32
    lib.gwas_selftest_timeout.argtypes = [i32, i32]
    lib.gwas_selftest_timeout.restype = i32
    lib.gwas_scan_static.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.gwas_scan_static.restype = i32
    lib.gwas_setup_timing.argtypes = [vp, dp]
    lib.gwas_setup_timing.restype = i32
    ip = ctypes.POINTER(ctypes.c_int)
    lib.gwas_info.argtypes = [vp, ip, ip, ip, ip, ip]
    lib.gwas_info.restype = i32
    lib.gwas_stream_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(i64), ctypes.POINTER(i32),
                                     ctypes.POINTER(i64), dp]
    lib.gwas_stream_info.restype = i32
    lib.gwas_split_pieces.argtypes = [vp]
    lib.gwas_split_pieces.restype = i32
    lib.gwas_fp8_traits.argtypes = [vp]
    lib.gwas_fp8_traits.restype = i32
    lib.gwas_chol_routed_traits.argtypes = [vp]
    lib.gwas_chol_routed_traits.restype = i32
    lib.gwas_eig_chunk.argtypes = [vp]
    lib.gwas_eig_chunk.restype = i64
    lib.gwas_batch_tuning.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), dp]
    lib.gwas_batch_tuning.restype = i32
    lib.gwas_genetic_columns.argtypes = [vp]
    lib.gwas_genetic_columns.restype = i32
    lib.gwas_singular_count.argtypes = [vp]
    lib.gwas_singular_count.restype = i64
    lib.gwas_stage_timing.argtypes = [vp, i32]
    lib.gwas_stage_timing.restype = i32
    lib.gwas_stage_times.argtypes = [vp, dp, ctypes.POINTER(i64)]
    lib.gwas_stage_times.restype = i32
    lib.gwas_last_error.argtypes = []
    lib.gwas_last_error.restype = ctypes.c_char_p
    lib.gwas_destroy.argtypes = [vp]
    lib.gwas_destroy.restype = None
    return lib


lib = _load()


def _check(st: int, where: str):
    if st != 0:
        raise GwasError(st, where, gwas_last_error())


def _f64_fortran(x, shape, name):
    a = np.asfortranarray(np.asarray(x, dtype=np.float64))
    if a.shape != shape:
        raise ValueError(f"{name}: shape {a.shape}, expected {shape}")
    return a


def _ptr(x):
    """(address, on_device) of a NumPy array or torch tensor (must be C-contiguous)."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    raise TypeError(f"unsupported buffer type {type(x)}")


def gwas_default_options(**kw) -> gwas_options:
    o = gwas_options()
    lib.gwas_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "algo" and isinstance(v, str):
            v = ALGO[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "out_mode" and isinstance(v, str):
            v = OUT_MODE[v]
        if k == "genetic_model" and isinstance(v, str):
            v = GENETIC_MODEL[v]
        setattr(o, k, int(v))
    return o


def gwas_setup(Phi, XL, Y, h2, s2, options: gwas_options | None = None, **kw):
    """Returns an opaque handle (int).  Phi: n x n, XL: n x q, Y: n x t, h2/s2: t."""
    Phi = np.asarray(Phi, dtype=np.float64)
    n = Phi.shape[0]
    XL = np.asarray(XL, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    q, t = XL.shape[1], Y.shape[1]
    Phi = _f64_fortran(Phi, (n, n), "Phi")
    XL = _f64_fortran(XL, (n, q), "XL")
    Y = _f64_fortran(Y, (n, t), "Y")
    h2 = np.ascontiguousarray(np.broadcast_to(np.asarray(h2, dtype=np.float64), (t,)))
    s2 = np.ascontiguousarray(np.broadcast_to(np.asarray(s2, dtype=np.float64), (t,)))
    o = options if options is not None else gwas_default_options(**kw)
    h = ctypes.c_void_p()
    st = lib.gwas_setup(Phi.ctypes.data, n, XL.ctypes.data, q, Y.ctypes.data, t, h2.ctypes.data,
                        s2.ctypes.data, ctypes.byref(o), ctypes.byref(h))
    _check(st, "gwas_setup")
    return h.value


def _scan(fn, name, h, XR, m, B, wald, stream):
    xp, xdev = _ptr(XR)
    bp, bdev = _ptr(B)
    wp, wdev = _ptr(wald) if wald is not None else (0, bdev)
    if wald is not None and wdev != bdev:
        raise ValueError("B and wald must both be host or both be device buffers")
    if stream is None and (xdev or bdev):
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = fn(h, xp, int(m), xdev, bp, wp or None, bdev, stream or None)
    _check(st, name)


def gwas_scan(h, XR, B, wald=None, stream=None, m=None):
    """XR: (m, n) int8; B: (m, t, p) float32; wald: (m, t) float32 or None."""
    _scan(lib.gwas_scan, "gwas_scan", h, XR, XR.shape[0] if m is None else m, B, wald, stream)


def gwas_scan_f64(h, XR, B, wald=None, stream=None, m=None):
    """As gwas_scan with float64 B and wald."""
    _scan(lib.gwas_scan_f64, "gwas_scan_f64", h, XR, XR.shape[0] if m is None else m, B, wald, stream)


EST_METHOD = {"ml": 0, "reml": 1}


def gwas_estimate(Phi, XL, Y, method="ml", device=0):
    """Step 1: per trait, (h2, s2) maximising the ML or REML criterion of the reduced model.
    Phi: n x n, XL: n x q, Y: n x t (or n).  Returns (h2, s2, crit, ms), ms = device
    milliseconds of the eigendecomposition + rotation and of the search."""
    Phi = np.asarray(Phi, dtype=np.float64)
    n = Phi.shape[0]
    XL = np.asarray(XL, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    q, t = XL.shape[1], Y.shape[1]
    Phi = _f64_fortran(Phi, (n, n), "Phi")
    XL = _f64_fortran(XL, (n, q), "XL")
    Y = _f64_fortran(Y, (n, t), "Y")
    h2, s2, crit, ms = np.empty(t), np.empty(t), np.empty(t), np.empty(2)
    m = EST_METHOD[method] if isinstance(method, str) else int(method)
    st = lib.gwas_estimate(Phi.ctypes.data, n, XL.ctypes.data, q, Y.ctypes.data, t, m,
                           int(device), h2.ctypes.data, s2.ctypes.data, crit.ctypes.data,
                           ms.ctypes.data)
    _check(st, "gwas_estimate")
    return h2, s2, crit, ms


def gwas_packed_row_bytes(n: int) -> int:
    return int(lib.gwas_packed_row_bytes(int(n)))


def gwas_shard(m_total: int, rank: int, world: int, align: int = 1) -> tuple[int, int]:
    """(start, count): the SNP range of rank `rank` of `world` in a genome of m_total SNPs."""
    a, c = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.gwas_shard(int(m_total), int(rank), int(world), int(align), ctypes.byref(a),
                          ctypes.byref(c)), "gwas_shard")
    return a.value, c.value


def gwas_pack_genotypes(X, G=None, stream=None):
    """X: (m, n) int8, host array or CUDA tensor.  Returns G, (m, gwas_packed_row_bytes(n))
    uint8 in the same place as X (allocated here when G is None)."""
    m, n = X.shape
    rb = gwas_packed_row_bytes(n)
    xp, xdev = _ptr(X)
    if G is None:
        if xdev:
            import torch
            G = torch.empty((m, rb), dtype=torch.uint8, device=X.device)
        else:
            G = np.empty((m, rb), dtype=np.uint8)
    gp, gdev = _ptr(G)
    if gdev != xdev or tuple(G.shape) != (m, rb):
        raise ValueError(f"G must be a ({m}, {rb}) uint8 buffer beside X")
    if xdev and stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.gwas_pack_genotypes(xp, int(m), int(n), gp, xdev, stream or None),
           "gwas_pack_genotypes")
    return G


def gwas_scan_packed(h, G, B, wald=None, stream=None, m=None):
    """G: (m, gwas_packed_row_bytes(n)) uint8 packed rows; B, wald as gwas_scan."""
    _scan(lib.gwas_scan_packed, "gwas_scan_packed", h, G, G.shape[0] if m is None else m, B, wald,
          stream)


def gwas_scan_static(h, XR, B, wald=None, stream=None, m=None):
    """As gwas_scan on device buffers, without any device allocation (EIG CUDA-core handles;
    see include/gwas.h for the size limit and the rules on sharing its fixed scratch)."""
    xp, xdev = _ptr(XR)
    bp, bdev = _ptr(B)
    wp = _ptr(wald)[0] if wald is not None else 0
    if not (xdev and bdev):
        raise ValueError("gwas_scan_static takes device buffers only")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    m = XR.shape[0] if m is None else m
    _check(lib.gwas_scan_static(h, xp, int(m), bp, wp or None, stream or None), "gwas_scan_static")


def gwas_setup_batch(cohorts, options: gwas_options | None = None, **kw):
    """cohorts: sequence of (Phi, XL, Y, h2, s2).  Returns an opaque batch (int)."""
    keep, arr = [], (gwas_cohort * len(cohorts))()
    for i, (Phi, XL, Y, h2, s2) in enumerate(cohorts):
        Phi = np.asarray(Phi, dtype=np.float64)
        n = Phi.shape[0]
        XL = np.asarray(XL, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        if Y.ndim == 1:
            Y = Y[:, None]
        q, t = XL.shape[1], Y.shape[1]
        Phi = _f64_fortran(Phi, (n, n), "Phi")
        XL = _f64_fortran(XL, (n, q), "XL")
        Y = _f64_fortran(Y, (n, t), "Y")
        h2 = np.ascontiguousarray(np.broadcast_to(np.asarray(h2, dtype=np.float64), (t,)))
        s2 = np.ascontiguousarray(np.broadcast_to(np.asarray(s2, dtype=np.float64), (t,)))
        keep += [Phi, XL, Y, h2, s2]
        arr[i] = gwas_cohort(Phi.ctypes.data, n, XL.ctypes.data, q, Y.ctypes.data, t,
                             h2.ctypes.data, s2.ctypes.data)
    o = options if options is not None else gwas_default_options(**kw)
    b = ctypes.c_void_p()
    _check(lib.gwas_setup_batch(len(cohorts), arr, ctypes.byref(o), ctypes.byref(b)),
           "gwas_setup_batch")
    return b.value


def gwas_scan_batch(b, blocks, stream=None):
    """blocks: sequence of (G, B, wald) CUDA tensors per cohort (G packed rows; wald may be
    None; a G with 0 rows skips the cohort)."""
    arr = (gwas_cohort_block * len(blocks))()
    for i, (G, B, W) in enumerate(blocks):
        gp, gdev = _ptr(G)
        bp, bdev = _ptr(B)
        wp = _ptr(W)[0] if W is not None else 0
        if not (gdev and bdev):
            raise ValueError("gwas_scan_batch takes device buffers only")
        arr[i] = gwas_cohort_block(gp, int(G.shape[0]), bp, wp or None)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.gwas_scan_batch(b, arr, stream or None), "gwas_scan_batch")


def gwas_batch_plan(b):
    plan = ctypes.c_int()
    ms = (ctypes.c_double * 4)()
    _check(lib.gwas_batch_plan(b, ctypes.byref(plan), ms), "gwas_batch_plan")
    return plan.value, list(ms)


def gwas_batch_handle(b, i):
    return lib.gwas_batch_handle(b, int(i))


def gwas_destroy_batch(b) -> None:
    lib.gwas_destroy_batch(b)


def _pvalues(wald, pval, stream, dof):
    wp, wdev = _ptr(wald)
    if pval is None:
        pval = wald.clone() if wdev else np.empty_like(wald)
    pp, pdev = _ptr(pval)
    if pdev != wdev:
        raise ValueError("wald and pval must both be host or both be device arrays")
    if wdev and stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    count = int(np.prod(wald.shape))
    if dof is None:
        _check(lib.gwas_wald_pvalues(wp, count, pp, wdev, stream or None), "gwas_wald_pvalues")
    else:
        _check(lib.gwas_wald_pvalues_dof(wp, count, int(dof), pp, wdev, stream or None),
               "gwas_wald_pvalues_dof")
    return pval


def gwas_wald_pvalues(wald, pval=None, stream=None):
    """chi-square(1) upper-tail p-values of a float32 array or CUDA tensor of Wald statistics."""
    return _pvalues(wald, pval, stream, None)


def gwas_wald_pvalues_dof(wald, dof, pval=None, stream=None):
    """chi-square(dof) upper-tail p-values, dof = 1 or 2 (gwas_genetic_columns of the handle)."""
    return _pvalues(wald, pval, stream, dof)


def gwas_sync(h) -> None:
    _check(lib.gwas_sync(h), "gwas_sync")


def gwas_selftest_timeout(device: int = 0, limit_ms: int = 200) -> int:
    """Status of the bounded-wait self-test: -7 (GWAS_ERR_TIMEOUT) when the wait gave up."""
    return int(lib.gwas_selftest_timeout(int(device), int(limit_ms)))


def gwas_setup_timing(h) -> float:
    ms = ctypes.c_double()
    _check(lib.gwas_setup_timing(h, ctypes.byref(ms)), "gwas_setup_timing")
    return ms.value


def gwas_info(h) -> dict:
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib.gwas_info(h, *[ctypes.byref(x) for x in v]), "gwas_info")
    n, q, t, algo, prec = (x.value for x in v)
    pr = int(lib.gwas_genetic_columns(h))
    return dict(n=n, q=q, t=t, p=q + pr, p_r=pr, algo=algo, precision=prec)


def gwas_genetic_columns(h) -> int:
    return int(lib.gwas_genetic_columns(h))


def gwas_split_pieces(h) -> int:
    return int(lib.gwas_split_pieces(h))


def gwas_fp8_traits(h) -> int:
    return int(lib.gwas_fp8_traits(h))


def gwas_chol_routed_traits(h) -> int:
    return int(lib.gwas_chol_routed_traits(h))


def gwas_eig_chunk(h) -> int:
    return int(lib.gwas_eig_chunk(h))


def gwas_batch_tuning(b) -> dict:
    """The batch autotuner's choice for the last new block shape: plan, EIG chunk divisor and
    the time of every (divisor, plan) candidate (ms)."""
    plan, div = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_double * 12)()
    _check(lib.gwas_batch_tuning(b, ctypes.byref(plan), ctypes.byref(div), ms), "gwas_batch_tuning")
    return {"plan": plan.value, "chunk_div": div.value,
            "ms": [[ms[4 * d + i] for i in range(4)] for d in range(3)]}


def gwas_stream_info(h) -> dict:
    """Streaming block size in use, whether it was chosen by timing, graph replays, and the timed
    candidates {snps: (ms H2D, ms scan, ms D2H)}."""
    blk, tuned, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    gl = ctypes.c_int64()
    snps = (ctypes.c_int64 * 8)()
    ms = (ctypes.c_double * 24)()
    _check(lib.gwas_stream_info(h, ctypes.byref(blk), ctypes.byref(tuned), ctypes.byref(gl),
                                ctypes.byref(nc), snps, ms), "gwas_stream_info")
    return dict(block_snps=blk.value, tuned=bool(tuned.value), graph_launches=gl.value,
                candidates={int(snps[i]): tuple(ms[3 * i:3 * i + 3]) for i in range(nc.value)})


def gwas_singular_count(h) -> int:
    return int(lib.gwas_singular_count(h))


def gwas_stage_timing(h, enable=True) -> None:
    _check(lib.gwas_stage_timing(h, int(bool(enable))), "gwas_stage_timing")


def gwas_stage_times(h) -> dict:
    """{stage name: (milliseconds, timed launches)} since the last read, stages with launches."""
    ms = (ctypes.c_double * NSTAGES)()
    n = (ctypes.c_int64 * NSTAGES)()
    _check(lib.gwas_stage_times(h, ms, n), "gwas_stage_times")
    return {name: (ms[i], int(n[i])) for i, name in enumerate(STAGES) if n[i]}


def gwas_last_error() -> str:
    return lib.gwas_last_error().decode()


def gwas_destroy(h) -> None:
    lib.gwas_destroy(h)
