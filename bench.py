#!/usr/bin/env python
"""Throughput of the GLS grid scan on one GB300: (SNP x trait) GLS solves per second.

Headline workload: single-trait genome scan, CLAK-Chol with the split-BF16 tensor-core
whitening: n = 1,000 individuals, p = 4 (intercept, two covariates, SNP), m = 2,000,000 SNPs as
int8 hard calls, h2 = 0.5, s2 = 1.  One step = one gwas_scan over all m SNPs (every SNP's GLS
solved and its Wald statistic written).  `value` is measured with the genotypes already resident
in HBM (2 GB, larger than the 129 MB L2, so no flush is needed between steps); `e2e` is the same
metric through the same C call with pinned HOST genotype and output buffers (the library streams
64 Ki-SNP blocks with double-buffered copies).  The line also carries the many-trait CLAK-Eig
workload (n = 1,000, t = 1,000, m = 100,000) under "other_workloads", measured the same way.
`--impl reference` times the FP64 CPU oracle instead.

Launch: python bench.py [--gpus N --steps K --warmup W] [--workload 1|0|2] [--precision P]
Under torchrun (N > 1) every rank scans its own replica of the workload (weak scaling, no
collective on the data path); rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "(SNP x trait) GLS solves/s at <=1e-4 rel err vs FP64"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def make_inputs(idx: int, m: int | None = None):
    """Workload `idx` with its genotypes drawn block by block (each block its own stream)."""
    c = synth.make_cohort(idx, m=0, with_genotypes=False)
    c.XR = synth.workload_genotypes(idx, m)
    return c


def _row_bytes(n, fmt):
    return n if fmt == "int8" else -(-n // 64) * 16


L2_BYTES = 129e6
FLUSH_BYTES = 512 << 20  # written between timed steps when the inputs would fit in L2


def _flushes(s, m, fmt):
    """True when a step's genotype input is not well above the L2 size: the timed steps are then
    separated by a write of FLUSH_BYTES (outside the timed events)."""
    return m * _row_bytes(s["n"], fmt) < 2 * L2_BYTES


def _config(s, precision, m, fmt):
    gb = m * _row_bytes(s["n"], fmt) / 1e9
    if _flushes(s, m, fmt):
        l2 = ("inputs (%s genotypes, %.3f GB) fit in the 129 MB L2: L2 flushed between timed "
              "steps by a %d MB write, each step timed alone" % (fmt, gb, FLUSH_BYTES >> 20))
    else:
        l2 = ("inputs (%s genotypes, %.2f GB) exceed the 129 MB L2 and are streamed once per "
              "step; no flush" % (fmt, gb))
    return {"workload": s["name"], "n": s["n"], "p": s["q"] + 1, "m": m, "t": s["t"],
            "algo": s["algo"], "precision": precision, "block_snps": s["block"],
            "genotypes": fmt, "l2": l2}


# ------------------------------------------------------------------------------------------
# algorithmic work (per unit) and traffic of the dominant kernel
# ------------------------------------------------------------------------------------------

def algorithmic_flops(s, m):
    """Algorithmic FLOPs of one step.  CHOL: the lower-triangular whitening x' = L^-1 x costs
    n(n+1) flops per SNP, the reductions a, c, s 2n(q+2).  EIG: per pair 2n(q+2) for a, c, s,
    plus the rotation Z^T x (2n^2 per SNP)."""
    n, q, t = s["n"], s["q"], s["t"]
    if s["algo"] == "chol":
        return m * t * (n * (n + 1) + 2 * n * (q + 2))
    return m * t * 2 * n * (q + 2) + m * 2 * n * n


def executed_flops(s, m):
    """Tensor-core FLOPs the split kernels issue (padding and split products included)."""
    n, q, t = s["n"], s["q"], s["t"]
    kpad = -(-n // 64) * 64
    rpad = -(-n // 256) * 256
    if s["algo"] == "chol":
        # rows of L^-1 plus the q + 1 rows of M^-1 [X_L | r]; per block the live rows (16-row
        # MMA granularity), and on the diagonal only the rows a K step meets
        macs = 0
        for nb in range(-(-(n + q + 1) // 256)):
            ncols = min(256, -(-(n + q + 1 - 256 * nb) // 16) * 16)
            nk = min(4 * (nb + 1), kpad // 64)
            for ks in range(nk):
                macs += 64 * (ncols - 64 * max(0, ks - 4 * nb))
        return 2 * 2 * macs * m * t
    rot = 2 * 2 * rpad * kpad * m
    sq = 3 * 2 * kpad * t * m
    ac = 2 * 2 * kpad * (q + 1) * t * m
    return rot + sq + ac


def traffic_key(s):
    """Entry of profiles/traffic.json for a workload: CHOL, or EIG at its trait count."""
    return "chol" if s["algo"] == "chol" else f"eig_t{s['t']}"


def traffic_per_launch(key, m):
    """DRAM bytes of the dominant kernel (CHOL) or of the whole step (EIG) from the committed ncu
    summary, scaled to m SNPs, or None if there is no capture for this workload or the kernel
    source changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)[key]
        with open(os.path.join(ROOT, d["source"]), "rb") as f:
            sha = hashlib.sha1(f.read()).hexdigest()
        if sha != d["source_sha1"]:
            return None
        return d["dram_bytes_per_snp"] * m
    except (OSError, KeyError, ValueError):
        return None


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle, as it stands
# ------------------------------------------------------------------------------------------

def run_reference(args, ws, rank):
    if rank != 0:
        return
    from oracle import gls
    s = dict(synth.WORKLOADS[args.workload])
    sample = args.ref_sample
    c = make_inputs(args.workload, m=sample)
    pairs_per_step = sample * c.t

    def step():
        gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = pairs_per_step / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        # the same workload description as our arm's line (the oracle's own arithmetic is the
        # line's dtype and its sample)
        "data": "synthetic", "config": _config(s, args.precision, s["m"], args.format),
        "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"first {sample} SNPs x {c.t} trait(s) of the workload per step, "
                                   "FP64 oracle (Algorithm 1 per GLS on int8 genotypes)"},
        "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def cpu_baseline(idx: int, sample: int):
    from oracle import gls
    c = make_inputs(idx, m=sample)
    t0 = time.perf_counter()
    gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    dt = time.perf_counter() - t0
    return {"value": sample * c.t / dt, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {sample} SNPs x {c.t} trait(s) of the workload, FP64 oracle "
                      f"(Algorithm 1 per GLS, BLAS threads = all cores), {dt:.1f} s"}


def parity_sample(c, Bd, Wd, count=256):
    """Max errors of the run's own outputs against the oracle on sampled (SNP, trait) pairs."""
    from oracle import gls
    rs = np.random.default_rng(1)
    snps = np.sort(rs.choice(c.m, size=min(count, c.m), replace=False))
    traits = rs.integers(0, c.t, size=len(snps))
    pairs = np.c_[snps, traits]
    Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, pairs)
    B = Bd[snps, traits].astype(np.float64)
    W = Wd[snps, traits].astype(np.float64)
    return (float(np.nanmax(gls.rel_err_b(B, Bref, Vref))),
            float(np.nanmax(gls.rel_err_wald(W, Wref))), len(pairs))


def measure(args, idx, precision, steps, warmup, local, ws, m=None, e2e_steps=5, e2e=True,
            fmt="packed"):
    """Setup + timed device steps + end-to-end host steps + parity sample for one workload.
    fmt: the genotype input format, "packed" (2-bit rows, gwas_scan_packed) or "int8"
    (gwas_scan; the tensor-core path packs on the device inside the step)."""
    import torch
    import paper_1207_2169_gb300 as g
    s = dict(synth.WORKLOADS[idx])
    c = make_inputs(idx, m=m)
    mm, n, t, p = c.m, c.n, c.t, c.p
    opt = g.gwas_default_options(algo=s["algo"], precision=precision, device=local)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, options=opt)
    try:
        setup_ms = g.gwas_setup_timing(h)
        xr_d = torch.from_numpy(c.XR).cuda()
        scan = g.gwas_scan
        if fmt == "packed":  # packed once, outside the timed region: it is the input format
            xr_d = g.gwas_pack_genotypes(xr_d)
            torch.cuda.synchronize()
            scan = g.gwas_scan_packed
        B_d = torch.empty((mm, t, p), dtype=torch.float32, device="cuda")
        W_d = torch.empty((mm, t), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()

        def step():
            scan(h, xr_d, B_d, W_d, stream=stream.cuda_stream)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        flush = _flushes(s, mm, fmt)
        scratch = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda") if flush else None
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps if flush else 1)]
        with ClockSampler(local) as clk:
            _barrier(ws)
            torch.cuda.synchronize()
            if flush:
                for e0, e1 in evs:
                    scratch.fill_(1.0)  # evicts the previous step's lines from L2
                    e0.record(stream)
                    step()
                    e1.record(stream)
            else:
                evs[0][0].record(stream)
                for _ in range(steps):
                    step()
                evs[0][1].record(stream)
            torch.cuda.synchronize()
            _barrier(ws)
        ms = _max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in evs) / steps, ws)
        del scratch
        eb, ew, npairs = parity_sample(c, B_d.cpu().numpy(), W_d.cpu().numpy())
        # end to end: pinned host genotypes in, pinned host results out, through the same call
        e2e_s, same = None, None
        if e2e:
            xr_h = xr_d.cpu().pin_memory()
            del xr_d
            B_h = torch.empty((mm, t, p), dtype=torch.float32).pin_memory()
            W_h = torch.empty((mm, t), dtype=torch.float32).pin_memory()
            scan(h, xr_h, B_h, W_h)
            _barrier(ws)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                scan(h, xr_h, B_h, W_h)
            e2e_s = _max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)
            same = bool(torch.equal(B_h, B_d.cpu()))
    finally:
        g.gwas_destroy(h)
    pairs = mm * t
    res = {
        "s": s, "m": mm, "ms": ms, "value": pairs * ws / (ms * 1e-3), "setup_ms": setup_ms,
        "clocks": clk.summary(), "parity": {"max_rel_err_b": eb, "max_rel_err_wald": ew,
                                            "pairs_checked": npairs,
                                            "tolerance": 1e-4 if precision != "fp64" else 1e-6},
        "e2e": None if e2e_s is None else {
            "value": pairs * ws / e2e_s, "unit": "pairs/s",
            "h2d_bytes_per_step": mm * _row_bytes(n, fmt),
            "d2h_bytes_per_step": mm * t * (p + 1) * 4, "ms_per_step": e2e_s * 1e3,
            "matches_device_run": same},
    }
    return res


def roofline(res, precision):
    """Roofline entry of the step's dominant kernel.  For CHOL a step is exactly one launch of the
    whiten-and-reduce kernel, so the CUDA-event step time is that kernel's launch duration.  For
    EIG a step is four launches (centres, rotation, s, a/c+Schur); the entry then covers the
    whole step (labelled so)."""
    s, m, ms = res["s"], res["m"], res["ms"]
    peaks, kind = _peaks()
    alg = algorithmic_flops(s, m) / (ms * 1e-3) / 1e12
    if precision != "split_bf16":
        return {"bound": "alu", "achieved": alg, "unit": "TFLOP/s", "peak": None, "frac": None,
                "traffic": None, "kernel": s["algo"] + " CUDA-core scan",
                "note": "plain FP64/FP32 comparator; no tensor-core roofline"}
    peak = peaks["bf16_tflops_sustained"]
    exe = executed_flops(s, m) / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": alg, "peak": peak, "unit": "TFLOP/s",
            "frac": alg / peak, "traffic": traffic_per_launch(traffic_key(s), m),
            "kernel": "chol_tc_kernel (whiten + reduce + Schur)" if s["algo"] == "chol"
            else "whole EIG step (rotation, s, a/c + Schur)",
            "peak_source": f"bf16_tflops_sustained, {kind} (MEASURED_PEAKS.json)",
            "executed_tflops": exe, "executed_frac": exe / peak,
            "algorithmic_flops_per_launch": algorithmic_flops(s, m)}


def launches_per_scan(s, precision, m, fmt):
    """Kernels of ours per scan on device buffers (validation off).  Input in the other format
    than the kernels read (int8 for the tensor-core path, packed for the CUDA-core paths) is
    converted first, one launch per chunk of up to 1 GiB of converted rows."""
    n, t, blk = s["n"], s["t"], s["block"]
    tc = precision == "split_bf16"
    convert = (fmt == "int8") == tc
    row = _row_bytes(n, "packed") if tc else n
    cc = max(min(m, (1 << 30) // row), min(m, blk)) if convert else m

    def kernels(mm):
        if s["algo"] == "chol":
            return t
        if tc:
            return 4 * -(-mm // 32768)  # centres, rotation, s, a/c + Schur per 32 Ki SNPs
        return 2 * -(-mm // min(m, blk))

    return sum(int(convert) + kernels(min(cc, m - off)) for off in range(0, m, cc))


def measure_estimate(method="reml", sample=4):
    """Step 1 (gwas_estimate) on the many-trait workload's cohort: n = 1,000, q = 3, t = 1,000
    traits, h^2 and sigma^2 per trait by REML.  Device time from the call's own CUDA events: the
    eigendecomposition of Phi with the rotation of X_L and Y (once per cohort), then the
    per-trait search (168 evaluations of the criterion per trait).  The FP64 oracle runs on
    `sample` evenly spaced traits for parity and as the CPU baseline."""
    import paper_1207_2169_gb300 as g
    from oracle import estimate as est
    c = synth.make_cohort(2, m=0, with_genotypes=False)
    n, q = c.XL.shape
    t = c.Y.shape[1]
    g.gwas_estimate(c.Phi, c.XL, c.Y[:, :8], method=method)  # warm-up
    h2, s2, ll, ms = g.gwas_estimate(c.Phi, c.XL, c.Y, method=method)
    sel = np.linspace(0, t - 1, sample).astype(int)
    m = est.ML if method == "ml" else est.REML
    t0 = time.perf_counter()
    h2r, s2r, llr = est.estimate(c.Phi, c.XL, c.Y[:, sel], m)
    cpu_s = time.perf_counter() - t0
    total = float(ms[0] + ms[1])
    # algorithmic FP64 work of the search, per eigen-coordinate: the grid tables (101 points,
    # once) q(q+1)/2 multiply-adds, a reciprocal and a logarithm; per trait, 101 grid points of
    # q + 1 multiply-adds, then 2 + 64 + 1 search points of q(q+1)/2 + q + 1 multiply-adds, a
    # reciprocal and a logarithm (a multiply-add counted as 2 flops)
    full = 2 * (q * (q + 1) // 2 + q + 1) + 2
    flops = 101 * n * (q * (q + 1) + 2) + t * n * (101 * 2 * (q + 1) + 67 * full)
    fp64_peak = 1250.0  # GFLOP/s, GB300 FP64 (nominal; no measured FP64 peak on this machine)
    return {"config": {"workload": f"estimate_{method}_n{n}_t{t}", "n": n, "q": q, "t": t,
                       "method": method, "grid": 101, "search": "golden section, 64 steps"},
            "value": t / (total * 1e-3), "unit": "traits/s", "ms_per_step": total,
            "ms_eigendecomposition": float(ms[0]), "ms_search": float(ms[1]),
            "parity": {"max_rel_err_crit": float(np.max(np.abs(ll[sel] - llr) / np.abs(llr))),
                       "max_abs_err_h2": float(np.max(np.abs(h2[sel] - h2r))),
                       "max_rel_err_s2": float(np.max(np.abs(s2[sel] - s2r) / s2r)),
                       "traits_checked": int(sample), "tolerance_crit": 1e-8},
            "roofline": {"bound": "alu", "kernel": "estimate_kernel (per-trait search)",
                         "achieved": flops / (ms[1] * 1e-3) / 1e9, "peak": fp64_peak,
                         "unit": "GFLOP/s", "frac": flops / (ms[1] * 1e-3) / 1e9 / fp64_peak,
                         "traffic": None, "peak_source": "nominal FP64 rate of GB300"},
            "cpu_baseline": {"value": sample / cpu_s, "unit": "traits/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{sample} of the {t} traits, FP64 oracle (H formed and "
                                       f"factored per evaluation), {cpu_s:.1f} s"}}


def run_ours(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    res = measure(args, args.workload, args.precision, args.steps, args.warmup, local, ws, m=args.m,
                  fmt=args.format)
    s = res["s"]
    other = []
    if not args.no_other and args.workload == 1 and args.m is None:
        # the many-trait EIG workloads: n=1000, t=1000, m=100,000 in full; and one 32 Ki-SNP
        # block of the omics workload (t=30,000; its full B for m=1,000,000 is 480 GB and is
        # consumed block by block), device-resident only
        for idx, m_other, with_e2e in ((2, None, True), (3, 32768, False)):
            k = max(3, args.steps // 2)
            o = measure(args, idx, args.precision, k, args.warmup, local, ws, m=m_other, e2e=with_e2e,
                        fmt=args.format)
            other.append({"config": _config(o["s"], args.precision, o["m"], args.format),
                          "value": o["value"],
                          "unit": "pairs/s", "ms_per_step": o["ms"], "e2e": o["e2e"],
                          "parity": o["parity"], "setup_ms": o["setup_ms"],
                          "roofline": roofline(o, args.precision),
                          "gpu_launches": k * launches_per_scan(o["s"], args.precision, o["m"],
                                                                args.format)})
        other.append(measure_estimate())
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": res["value"], "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"split_bf16": "bf16x2->f32", "fp32": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic", "config": _config(s, args.precision, res["m"], args.format),
        "e2e": res["e2e"],
        "gpu_launches": args.steps * launches_per_scan(s, args.precision, res["m"], args.format),
        "roofline": roofline(res, args.precision),
        "parity": res["parity"], "setup_ms": res["setup_ms"], "clocks": res["clocks"],
    }
    if other:
        line["other_workloads"] = other
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample)
    print(json.dumps(line), flush=True)


def run_batch(args, ws, rank, local):
    """Workload 4: 16 uneven cohorts scanned by one gwas_scan_batch (a CUDA graph whose launch
    plan the library picked by timing), against the same scans issued cohort by cohort."""
    import torch
    import paper_1207_2169_gb300 as g
    from oracle import gls
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    spec = synth.BATCH
    m = spec["m"] if args.m is None else args.m
    shapes = synth.batch_shapes()
    cohorts = [synth.batch_cohort(i, n, q, t) for i, (n, q, t) in enumerate(shapes)]
    t0 = time.perf_counter()
    opt = g.gwas_default_options(precision="split_bf16", device=local)
    b = g.gwas_setup_batch([(c.Phi, c.XL, c.Y, c.h2, c.s2) for c in cohorts], options=opt)
    setup_s = time.perf_counter() - t0
    try:
        blocks, samples = [], []
        rs = np.random.default_rng(4)
        for i, ((n, q, t), c) in enumerate(zip(shapes, cohorts)):
            X = synth.device_genotypes(i, n, m)
            snps = np.sort(rs.choice(m, size=4, replace=False))
            samples.append((snps, int(rs.integers(0, t)), X[torch.from_numpy(snps).cuda()].cpu().numpy()))
            G = g.gwas_pack_genotypes(X)
            del X
            B = torch.empty((m, t, q + 1), dtype=torch.float32, device="cuda")
            W = torch.empty((m, t), dtype=torch.float32, device="cuda")
            blocks.append((G, B, W))
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        g.gwas_scan_batch(b, blocks, stream=stream.cuda_stream)  # picks the launch plan
        plan, plan_ms = g.gwas_batch_plan(b)
        for _ in range(args.warmup):
            g.gwas_scan_batch(b, blocks, stream=stream.cuda_stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            _barrier(ws)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                g.gwas_scan_batch(b, blocks, stream=stream.cuda_stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            _barrier(ws)
        ms = _max_over_ranks(ev0.elapsed_time(ev1) / args.steps, ws)
        # the same work as separate per-cohort calls (each launch with every SM, one after another)
        handles = [g.gwas_batch_handle(b, i) for i in range(len(cohorts))]
        for _ in range(2):
            for h, (G, B, W) in zip(handles, blocks):
                g.gwas_scan_packed(h, G, B, W, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            for h, (G, B, W) in zip(handles, blocks):
                g.gwas_scan_packed(h, G, B, W, stream=stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_seq = _max_over_ranks(ev0.elapsed_time(ev1) / args.steps, ws)
        g.gwas_scan_batch(b, blocks, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        eb = ew = 0.0
        for (snps, j, Xs), c, (G, B, W) in zip(samples, cohorts, blocks):
            Bd = B[torch.from_numpy(snps).cuda(), j].cpu().numpy().astype(np.float64)
            Wd = W[torch.from_numpy(snps).cuda(), j].cpu().numpy().astype(np.float64)
            pairs = np.c_[np.arange(len(snps)), np.full(len(snps), j)]
            Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, Xs, c.Y, c.h2, c.s2, pairs)
            eb = max(eb, float(np.nanmax(gls.rel_err_b(Bd, Bref, Vref))))
            ew = max(ew, float(np.nanmax(gls.rel_err_wald(Wd, Wref))))
    finally:
        g.gwas_destroy_batch(b)
    if rank != 0:
        return
    pairs = m * sum(t for _, _, t in shapes)
    flops = 0.0
    for n, q, t in shapes:
        kp, rp = -(-n // 64) * 64, -(-n // 256) * 256
        flops += m * (4.0 * rp * kp + t * kp * (6.0 + 4.0 * (q + 1)))
    peaks, kind = _peaks()
    exe = flops / (ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": pairs * ws / (ms * 1e-3), "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x2->f32", "data": "synthetic",
        "config": {"workload": spec["name"], "cohorts": [dict(n=n, p=q + 1, t=t) for n, q, t in shapes],
                   "m": m, "genotypes": "packed", "algo": "eig (t > 1)",
                   "l2": "inputs (packed genotypes, %.2f GB) exceed the 129 MB L2; no flush" %
                         (m * sum(-(-n // 64) * 16 for n, _, _ in shapes) / 1e9)},
        "gpu_launches": args.steps * sum(launches_per_scan(dict(n=n, q=q, t=t, algo="eig", block=32768),
                                                           "split_bf16", m, "packed")
                                         for n, q, t in shapes),
        "batch": {"plan": plan, "plan_ms": plan_ms,
                  "plans": ["sequential", "concurrent, SM shares by work", "concurrent, all SMs",
                            "two lanes of half the SMs"],
                  "per_cohort_calls_ms": ms_seq, "speedup_vs_per_cohort_calls": ms_seq / ms},
        "roofline": {"bound": "tensor", "achieved": None, "executed_tflops": exe,
                     "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                     "executed_frac": exe / peaks["bf16_tflops_sustained"], "traffic": None,
                     "kernel": "whole batched step", "peak_source": f"bf16_tflops_sustained, {kind}"},
        "parity": {"max_rel_err_b": eb, "max_rel_err_wald": ew, "pairs_checked": 4 * len(shapes),
                   "tolerance": 1e-4},
        "setup_s": setup_s, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=1)
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "fp32", "fp64"])
    ap.add_argument("--format", default="packed", choices=["packed", "int8"],
                    help="genotype input format of the timed scans")
    ap.add_argument("--m", type=int, default=None, help="override the SNP count (profiling only)")
    ap.add_argument("--cpu-sample", type=int, default=400_000)
    ap.add_argument("--ref-sample", type=int, default=20_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip the EIG workload measurement")
    ap.add_argument("--only-estimate", action="store_true",
                    help="run only the step-1 (gwas_estimate) measurement and print its entry")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = _dist()
    if args.only_estimate:
        import torch
        torch.cuda.set_device(local)
        if rank == 0:
            print(json.dumps(measure_estimate()), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == 4:
        run_batch(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
