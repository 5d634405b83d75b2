#!/usr/bin/env python
"""Throughput of the GLS grid scan on one GB300: (SNP x trait) GLS solves per second.

Headline workload: single-trait genome scan, CLAK-Chol with the split-BF16 tensor-core
whitening: n = 1,000 individuals, p = 4 (intercept, two covariates, SNP), m = 2,000,000 SNPs,
h2 = 0.5, s2 = 1.  One step = one gwas_scan_packed over all m SNPs (every SNP's GLS solved and
its Wald statistic written).  `value` is measured with the genotypes already resident in HBM
(0.51 GB of 2-bit packed rows, larger than the 129 MB L2, so no flush is needed between steps);
`e2e` is the same metric through the same C call with pinned HOST genotype and output buffers
(the library streams 64 Ki-SNP blocks with double-buffered copies).

The same JSON line carries, under "other_workloads", every other workload measured the same way:
the headline with int8 genotypes as input, the plain FP32 CUDA-core form of the headline (and the
speedup of the tensor-core path over it at equal accuracy), the FP64 CHOL workload (n = 256,
m = 10^4, every SNP checked at 1e-6), the many-trait CLAK-Eig workload (n = 1,000, t = 1,000,
m = 100,000) with its FP32 and FP64 CUDA-core forms, the omics-scale CLAK-Eig workload streamed as
stated (t = 30,000, m = 10^6 in 32 Ki-SNP blocks, full and SNP-only outputs, device-resident and
end to end), the batch of 16 uneven cohorts (one graph-captured gwas_scan_batch), and step 1
(h2, s2 by REML).  Each carries its own parity sample against the FP64 oracle, per-kernel
rooflines from CUDA events recorded around each kernel on its stream (gwas_stage_timing), and
the count of kernels launched.  `--impl reference` times the FP64 CPU oracle instead.

Launch: python bench.py [--gpus N --steps K --warmup W] [--workload 0|1|2|3|4] [--precision P]
Under torchrun (N > 1) every rank scans its own SNP range of a genome N times the workload's
length (gwas_shard; weak scaling, the same cohort on every rank, no collective on the data
path); rank 0 prints the max-over-ranks time and value = all ranks' pairs / that time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
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
TOL = {"split_bf16": 1e-4, "split_fp8": 1e-4, "fp32": 1e-4, "fp64": 1e-6}
SPLIT = ("split_bf16", "split_fp8")
DTYPE = {"split_bf16": "bf16x2->f32", "split_fp8": "f16+e4m3->f32", "fp32": "f32", "fp64": "f64"}


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


_INPUTS = {}


def make_inputs(idx: int, m: int | None = None, shard: bool = False):
    """Workload `idx` with its genotypes drawn block by block (each block its own stream).  The
    last workload drawn is kept, so that its variants (input format, precision) reuse it.
    shard: under torchrun, this rank's own SNP range (gwas_shard) of a genome of WORLD_SIZE x m
    SNPs -- every rank scans m SNPs (weak scaling), different ones, with the same cohort."""
    ws, rank, _ = _dist()
    spec = synth.WORKLOADS[idx]
    m = spec["m"] if m is None else m
    start = 0
    if shard and ws > 1:
        import paper_1207_2169_gb300 as g
        start, m = g.gwas_shard(ws * m, rank, ws)
    key = (idx, m, start)
    if key not in _INPUTS:
        _INPUTS.clear()
        c = synth.make_cohort(idx, m=0, with_genotypes=False)
        c.XR = synth.workload_genotypes(idx, m, start=start)
        c.snp_start = start
        _INPUTS[key] = c
    return _INPUTS[key]


def _row_bytes(n, fmt):
    return n if fmt == "int8" else -(-n // 64) * 16


L2_BYTES = 129e6
FLUSH_BYTES = 512 << 20  # written between timed steps when the inputs would fit in L2


def _flushes(s, m, fmt):
    """True when a step's genotype input is not well above the L2 size: the timed steps are then
    separated by a write of FLUSH_BYTES (outside the timed events)."""
    return m * _row_bytes(s["n"], fmt) < 2 * L2_BYTES


def _config(s, precision, m, fmt, **extra):
    gb = m * _row_bytes(s["n"], fmt) / 1e9
    if _flushes(s, m, fmt):
        l2 = ("inputs (%s genotypes, %.3f GB) fit in the 129 MB L2: L2 flushed between timed "
              "steps by a %d MB write, each step timed alone" % (fmt, gb, FLUSH_BYTES >> 20))
    else:
        l2 = ("inputs (%s genotypes, %.2f GB) exceed the 129 MB L2 and are streamed once per "
              "step; no flush" % (fmt, gb))
    d = {"workload": s["name"], "n": s["n"], "p": s["q"] + 1, "m": m, "t": s["t"],
         "algo": s["algo"], "precision": precision, "block_snps": s["block"],
         "genotypes": fmt, "l2": l2}
    d.update(extra)
    return d


# ------------------------------------------------------------------------------------------
# algorithmic work (per unit), executed tensor work, and DRAM traffic of each kernel
# ------------------------------------------------------------------------------------------

def eig_ac_traits(q):
    """Traits per column block of the EIG a/c kernel (its 256 accumulator columns)."""
    qp = 4 if q + 1 <= 4 else 8
    return min(256 // (q + 1), (256 - qp) // (q + 1) + 1)


def stage_flops(s, m):
    """Algorithmic FLOPs of one step per kernel stage.  CHOL: the lower-triangular whitening
    x' = L^-1 x costs n(n+1) flops per SNP, the reductions a, c, s 2n(q+2).  EIG: the rotation
    Z^T x 2n^2 per SNP; s_ij 2n per pair; a_ij, c_ij 2n(q+1) per pair."""
    n, q, t = s["n"], s["q"], s["t"]
    if s["algo"] == "chol":
        return {"chol": m * t * (n * (n + 1) + 2 * n * (q + 2))}
    return {"rot": m * 2 * n * n, "sq": m * t * 2 * n, "ac": m * t * 2 * n * (q + 1)}


def algorithmic_flops(s, m):
    return sum(stage_flops(s, m).values())


def stage_executed(s, m, pieces=2, fp8=False):
    """Tensor-core FLOPs the split kernels issue per stage (split products, K and N padding);
    `pieces`: BF16 pieces of L^-1 (CHOL) or U (EIG's a/c kernel), 2 or 3.  fp8 (CHOL,
    SPLIT_FP8): an FP16 hi product and an E4M3 lo product over the same K steps, the
    lo product counted at half weight (the FP8 rate is twice the BF16 one): BF16-equivalent
    FLOPs, comparable with the BF16 peak."""
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
        return {"chol": (1.5 if fp8 else pieces) * 2 * macs * m * t}
    nac = -(-t // eig_ac_traits(q))
    return {"rot": 2 * 2 * rpad * kpad * m, "sq": 3 * 2 * kpad * (-(-t // 256) * 256) * m,
            "ac": pieces * 2 * kpad * 256 * nac * m}


def code_sha1(path):
    """SHA-1 of a source file with its comments and blank space removed, so that an edit to
    comments alone does not invalidate the DRAM counters taken on the kernel."""
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", " ", src).strip()
    return hashlib.sha1(src.encode()).hexdigest()


KERNEL_NAMES = {"chol": "chol_tc_kernel", "rot": "eig_tc_kernel<ROT>", "sq": "eig_tc_kernel<SQ>",
                "ac": "eig_tc_kernel<AC>"}


def traffic_per_unit(kernel):
    """(DRAM bytes per unit, unit) of a kernel from the committed ncu summary, or (None, None) if
    there is no capture or the kernel's code changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)[kernel]
        if code_sha1(os.path.join(ROOT, d["source"])) != d["code_sha1"]:
            return None, None
        return float(d["dram_bytes_per_unit"]), d["unit"]
    except (OSError, KeyError, ValueError):
        return None, None


def kernel_roofline(s, m, stage, ms_total, launches, peak_tf, peak_src, steps, pieces=2,
                    fp8=False):
    """Roofline entry of one kernel stage from its CUDA-event time over the timed region."""
    alg = stage_flops(s, m)[stage] * steps
    exe = stage_executed(s, m, pieces, fp8)[stage] * steps
    name = KERNEL_NAMES[stage] + ("<F8>" if fp8 else "")
    per, unit = traffic_per_unit(name)
    units = m * steps * (s["t"] if unit == "pair" else 1)
    sec = ms_total * 1e-3
    achieved = alg / sec / 1e12
    return {"bound": "tensor", "kernel": name,
            "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved / peak_tf,
            "traffic": None if per is None else per * units / launches,
            "peak_source": peak_src, "launches": launches, "ms_per_launch": ms_total / launches,
            "algorithmic_flops_per_launch": alg / launches,
            "executed_tflops": exe / sec / 1e12, "executed_frac": exe / sec / 1e12 / peak_tf}


def rooflines(s, m, stages, steps, precision, pieces=2, fp8=False):
    """Per-kernel roofline entries of a tensor-core scan and the dominant one (largest time).
    The step's kernels are each timed alone per launch (a few ms at most), so the burst BF16 peak
    applies (FP16 has the BF16 rate; with fp8 the E4M3 lo product is counted at half weight in
    the executed figure)."""
    if precision not in SPLIT:
        ms = stages.get("simt", (0.0, 0))[0]
        alg = algorithmic_flops(s, m) * steps / (ms * 1e-3) / 1e12 if ms else None
        return {"bound": "alu", "kernel": s["algo"] + " CUDA-core scan", "achieved": alg,
                "unit": "TFLOP/s", "peak": None, "frac": None, "traffic": None,
                "note": "plain FP64/FP32 comparator on the CUDA cores; no tensor-core roofline"}, []
    peaks, kind = _peaks()
    peak = peaks["bf16_tflops"]
    src = f"bf16_tflops (burst: each launch is timed alone), {kind} (MEASURED_PEAKS.json)"
    entries = [kernel_roofline(s, m, st, stages[st][0], stages[st][1], peak, src, steps, pieces,
                               fp8 and st == "chol")
               for st in (["chol"] if s["algo"] == "chol" else ["rot", "sq", "ac"]) if st in stages]
    if fp8:
        for e in entries:
            if e["kernel"] == "chol_tc_kernel<F8>":
                e["note"] = ("FP16 hi x FP16 centred genotypes plus E4M3 lo x E4M3 genotypes into "
                             "one accumulator; executed FLOPs count the E4M3 product at half "
                             "weight (its nominal rate is twice the BF16 one)")
    dom = max(entries, key=lambda e: e["ms_per_launch"] * e["launches"])
    return dom, entries


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle, as it stands
# ------------------------------------------------------------------------------------------

def run_reference(args, ws, rank):
    if rank != 0:
        return
    from oracle import gls
    idx = args.workload if args.workload in (0, 1, 2, 3) else 1
    s = dict(synth.WORKLOADS[idx])
    sample = args.ref_sample
    c = make_inputs(idx, m=sample)
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


def parity_sample(c, Bd, Wd, count=256, every=False):
    """Max errors of the run's own outputs against the oracle on sampled (SNP, trait) pairs (or
    on every pair); NaN must sit exactly where the oracle's is."""
    from oracle import gls
    if every:
        Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
        eb, ew = gls.max_rel_errors(Bd.astype(np.float64), Wd.astype(np.float64), Bref, Wref, Vref)
        return eb, ew, c.m * c.t
    rs = np.random.default_rng(1)
    snps = np.sort(rs.choice(c.m, size=min(count, c.m), replace=False))
    traits = rs.integers(0, c.t, size=len(snps))
    pairs = np.c_[snps, traits]
    Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, pairs)
    B = Bd[snps, traits].astype(np.float64)
    W = Wd[snps, traits].astype(np.float64)
    eb, ew = gls.max_rel_errors(B, W, Bref, Wref, Vref)
    return eb, ew, len(pairs)


def host_link():
    """Bandwidth of this GPU's host link, measured now: 256 MB copies between pinned host memory
    and the device, each direction alone (GB/s).  Several streams, or an SM copy kernel reading
    mapped host memory, reach the same rate on a GB300 machine, and the two directions share it
    (both at once add up to about the one-direction figure), so the e2e floor of a step is
    h2d_bytes / h2d_gbs + d2h_bytes / d2h_gbs.  The rate moves with the host's other load (the
    box shares its CPU memory with other tenants), so it is taken right after each e2e timing."""
    import torch
    nb = 256 << 20
    h = torch.empty(nb, dtype=torch.uint8).pin_memory()
    d = torch.empty(nb, dtype=torch.uint8, device="cuda")
    h.fill_(1)
    d.fill_(2)
    link = {}
    for key, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        link[key] = 5 * nb / (e0.elapsed_time(e1) * 1e-3) / 1e9
    return link


def link_roof(e2e, link):
    """The host-link floor of an e2e entry: the time its copies take at the link rate measured
    beside it, and that floor over the measured e2e step (1.0 = the step runs at the link's
    rate)."""
    floor = (e2e["h2d_bytes_per_step"] / link["h2d_gbs"] + e2e["d2h_bytes_per_step"] / link["d2h_gbs"]) / 1e6
    e2e["host_link"] = {"h2d_gbs": link["h2d_gbs"], "d2h_gbs": link["d2h_gbs"],
                        "copy_floor_ms_per_step": floor, "frac": floor / e2e["ms_per_step"],
                        "note": "pinned cudaMemcpyAsync rate measured right after this e2e "
                                "timing; the two directions share the link"}
    return e2e


def _timed(stream, steps, step, flush, scratch):
    """Device milliseconds of `steps` calls of step(), from CUDA events on `stream`."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps if flush else 1)]
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
    return sum(e0.elapsed_time(e1) for e0, e1 in evs)


def measure(idx, precision, steps, warmup, local, ws, m=None, e2e_steps=5, e2e=True,
            fmt="packed", c=None, every=False, parity_count=256):
    """Setup + timed device steps (per-kernel events on) + end-to-end host steps + parity for one
    workload.  fmt: the genotype input format, "packed" (2-bit rows, gwas_scan_packed) or
    "int8" (gwas_scan; the tensor-core path packs on the device inside the step)."""
    import torch
    import paper_1207_2169_gb300 as g
    s = dict(synth.WORKLOADS[idx])
    c = make_inputs(idx, m=m, shard=True) if c is None else c
    mm, n, t, p = c.m, c.n, c.t, c.p
    opt = g.gwas_default_options(algo=s["algo"], precision=precision, device=local)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, options=opt)
    try:
        setup_ms = g.gwas_setup_timing(h)
        pieces = max(g.gwas_split_pieces(h), 2)
        fp8 = g.gwas_fp8_traits(h) > 0
        xr_d = torch.from_numpy(c.XR).cuda()
        scan = g.gwas_scan
        if fmt == "packed":  # packed once, outside the timed region: it is the input format
            xr_d = g.gwas_pack_genotypes(xr_d)
            torch.cuda.synchronize()
            scan = g.gwas_scan_packed
        B_d = torch.full((mm, t, p), float("nan"), dtype=torch.float32, device="cuda")
        W_d = torch.full((mm, t), float("nan"), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()

        def step():
            scan(h, xr_d, B_d, W_d, stream=stream.cuda_stream)

        # parity on the outputs of the first call: every pair written (the buffers were NaN)
        step()
        torch.cuda.synchronize()
        eb, ew, npairs = parity_sample(c, B_d.cpu().numpy(), W_d.cpu().numpy(), count=parity_count,
                                       every=every)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        flush = _flushes(s, mm, fmt)
        scratch = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda") if flush else None
        g.gwas_stage_timing(h, True)
        with ClockSampler(local) as clk:
            _barrier(ws)
            ms = _timed(stream, steps, step, flush, scratch)
            _barrier(ws)
        stages = g.gwas_stage_times(h)
        g.gwas_stage_timing(h, False)
        ms = _max_over_ranks(ms / steps, ws)
        del scratch
        # end to end: pinned host genotypes in, pinned host results out, through the same call
        e2e_s, same, stream = None, None, None
        if e2e:
            xr_h = xr_d.cpu().pin_memory()
            del xr_d
            B_h = torch.empty((mm, t, p), dtype=torch.float32).pin_memory()
            W_h = torch.empty((mm, t), dtype=torch.float32).pin_memory()
            scan(h, xr_h, B_h, W_h)  # the first streamed call also picks the block size
            t0 = time.perf_counter()
            scan(h, xr_h, B_h, W_h)
            # enough steps for about half a second of host-timed work: a 3 ms step timed five
            # times is at the mercy of one late wake-up of the host thread
            e2e_steps = int(min(max(e2e_steps, 0.5 / max(time.perf_counter() - t0, 1e-6)), 200))
            e2e_steps = int(_max_over_ranks(e2e_steps, ws))
            info0 = g.gwas_stream_info(h)
            _barrier(ws)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                scan(h, xr_h, B_h, W_h)
            e2e_s = _max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)
            link = host_link()
            info1 = g.gwas_stream_info(h)
            stream = {"block_snps": info1["block_snps"], "block_chosen_by_timing": info1["tuned"],
                      "candidates_ms_h2d_scan_d2h": {str(k): v for k, v in info0["candidates"].items()},
                      "graph_replays_per_step": (info1["graph_launches"] - info0["graph_launches"]) / e2e_steps}
            same = bool(torch.equal(B_h, B_d.cpu()))
    finally:
        g.gwas_destroy(h)
    pairs = mm * t
    dom, kernels = rooflines(s, mm, stages, steps, precision, pieces, fp8)
    res = {
        "s": s, "m": mm, "ms": ms, "value": pairs * ws / (ms * 1e-3), "setup_ms": setup_ms,
        "split_pieces": pieces if precision in SPLIT else None,
        "clocks": clk.summary(), "parity": {"max_rel_err_b": eb, "max_rel_err_wald": ew,
                                            "pairs_checked": npairs, "tolerance": TOL[precision]},
        "e2e": None if e2e_s is None else link_roof({
            "value": pairs * ws / e2e_s, "unit": "pairs/s",
            "h2d_bytes_per_step": mm * _row_bytes(n, fmt),
            "d2h_bytes_per_step": mm * t * (p + 1) * 4, "ms_per_step": e2e_s * 1e3,
            "steps": e2e_steps, "matches_device_run": same, "streaming": stream}, link),
        "roofline": dom, "kernels": kernels,
        "gpu_launches": sum(v[1] for v in stages.values()),
        "stage_ms": {k: v[0] / steps for k, v in stages.items()},
    }
    return res


def entry(res, precision, fmt, steps, warmup, **extra):
    """A workload's entry under other_workloads."""
    d = {"config": _config(res["s"], precision, res["m"], fmt, **extra.pop("config", {})),
         "value": res["value"], "unit": "pairs/s", "ms_per_step": res["ms"], "steps": steps,
         "warmup": warmup, "e2e": res["e2e"], "parity": res["parity"],
         "setup_ms": res["setup_ms"],
         "roofline": res["roofline"], "gpu_launches": res["gpu_launches"],
         "stage_ms_per_step": res["stage_ms"], "clocks": res["clocks"],
         "split_pieces": res.get("split_pieces")}
    if res["kernels"] and len(res["kernels"]) > 1:
        d["kernel_rooflines"] = res["kernels"]
    d.update(extra)
    return d


def measure_stream3(local, ws, steps=2, warmup=1, m=None, out_mode="full", pinned=None):
    """The omics-scale CLAK-Eig workload as stated: n = 1,000, t = 30,000, m = 10^6 SNPs in
    32 Ki-SNP blocks.  One step = the whole genome, one gwas_scan_packed per block.  Device rate:
    packed genotypes resident, each block's results into one of two device buffers (a consumer
    takes each block's 1e9 pairs before the next but one).  End to end: pinned host genotypes,
    each block's results copied to one pinned host buffer (the consumer's, reused per block).
    Parity: 100 random traits x 100 random SNPs = 10,000 pairs grouped by trait."""
    import torch
    import paper_1207_2169_gb300 as g
    from oracle import gls
    s = dict(synth.WORKLOADS[3])
    blk = s["block"]
    c = make_inputs(3, m=m, shard=True)
    mm, n, t, p = c.m, c.n, c.t, c.p
    pw = 2 if out_mode == "snp" else p
    nblk = -(-mm // blk)
    opt = g.gwas_default_options(algo="eig", precision="split_bf16", device=local,
                                 out_mode=out_mode)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, options=opt)
    try:
        setup_ms = g.gwas_setup_timing(h)
        pieces = g.gwas_split_pieces(h)
        G = g.gwas_pack_genotypes(torch.from_numpy(c.XR).cuda())
        Bs = [torch.empty((blk, t, pw), dtype=torch.float32, device="cuda") for _ in range(2)]
        Ws = [torch.empty((blk, t), dtype=torch.float32, device="cuda") for _ in range(2)]
        stream = torch.cuda.current_stream()

        def step():
            for b in range(nblk):
                lo, hi = b * blk, min(mm, (b + 1) * blk)
                g.gwas_scan_packed(h, G[lo:hi], Bs[b & 1][:hi - lo], Ws[b & 1][:hi - lo],
                                   stream=stream.cuda_stream)

        for _ in range(warmup):
            step()
        g.gwas_stage_timing(h, True)
        with ClockSampler(local) as clk:
            _barrier(ws)
            ms = _timed(stream, steps, step, False, None)
            _barrier(ws)
        stages = g.gwas_stage_times(h)
        g.gwas_stage_timing(h, False)
        ms = _max_over_ranks(ms / steps, ws)
        # parity: sampled SNPs' rows of each block gathered after a scan of that block
        rs = np.random.default_rng(3)
        snps = np.sort(rs.choice(mm, size=100, replace=False))
        traits = np.sort(rs.choice(t, size=100, replace=False))
        Bsel = np.empty((100, 100, pw))
        Wsel = np.empty((100, 100))
        tr = torch.from_numpy(traits).cuda()
        for b in sorted(set(snps // blk)):
            lo, hi = b * blk, min(mm, (b + 1) * blk)
            Bs[0].fill_(float("nan"))
            Ws[0].fill_(float("nan"))
            g.gwas_scan_packed(h, G[lo:hi], Bs[0][:hi - lo], Ws[0][:hi - lo], stream=stream.cuda_stream)
            k = np.flatnonzero(snps // blk == b)
            loc = torch.from_numpy(snps[k] - lo).cuda()
            Bsel[k] = Bs[0][loc][:, tr].double().cpu().numpy()
            Wsel[k] = Ws[0][loc][:, tr].double().cpu().numpy()
        Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2, snps=snps, traits=traits)
        if out_mode == "snp":  # (b_snp, standard error): the last coefficient and sqrt(Var)
            eb, ew = gls.max_rel_errors(Bsel[..., :1], Wsel, Bref[..., -1:], Wref, Vref[..., -1:])
            se = np.abs(Bsel[..., 1] - np.sqrt(Vref[..., -1])) / np.sqrt(Vref[..., -1])
            eb = max(eb, float(np.max(se)) if np.all(np.isfinite(se)) else float("inf"))
        else:
            eb, ew = gls.max_rel_errors(Bsel, Wsel, Bref, Wref, Vref)
        del Bs, Ws
        torch.cuda.empty_cache()
        # end to end: host genotypes and host outputs, one call per block
        G_h = G.cpu().pin_memory()
        del G
        if pinned is None or pinned[0].numel() < blk * t * pw:
            pinned = (torch.empty(blk * t * pw, dtype=torch.float32, pin_memory=True),
                      torch.empty(blk * t, dtype=torch.float32, pin_memory=True))
        Bh, Wh = pinned

        call_ms = []

        def e2e_step():
            for b in range(nblk):
                lo, hi = b * blk, min(mm, (b + 1) * blk)
                t1 = time.perf_counter()
                g.gwas_scan_packed(h, G_h[lo:hi], Bh[:(hi - lo) * t * pw].view(hi - lo, t, pw),
                                   Wh[:(hi - lo) * t].view(hi - lo, t))
                call_ms.append((time.perf_counter() - t1) * 1e3)

        e2e_step()
        call_ms.clear()
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(steps):
            e2e_step()
        e2e_s = _max_over_ranks((time.perf_counter() - t0) / steps, ws)
        link = host_link()
        info = g.gwas_stream_info(h)
        full = sorted(x for i, x in enumerate(call_ms) if (i % nblk) != nblk - 1)
        stream_info = {"block_snps": info["block_snps"], "block_chosen_by_timing": info["tuned"],
                       "ms_per_32Ki_call": {"min": full[0], "median": full[len(full) // 2],
                                            "max": full[-1]}}
    finally:
        g.gwas_destroy(h)
    pairs = mm * t
    dom, kernels = rooflines(s, mm, stages, steps, "split_bf16", pieces)
    res = {"s": s, "m": mm, "ms": ms, "value": pairs * ws / (ms * 1e-3), "setup_ms": setup_ms,
           "split_pieces": pieces,
           "clocks": clk.summary(),
           "parity": {"max_rel_err_b": eb, "max_rel_err_wald": ew, "pairs_checked": 10000,
                      "tolerance": 1e-4,
                      "sample": "100 random traits x 100 random SNPs, grouped by trait"},
           "e2e": link_roof({"value": pairs * ws / e2e_s, "unit": "pairs/s",
                             "h2d_bytes_per_step": mm * _row_bytes(n, "packed"),
                             "d2h_bytes_per_step": mm * t * (pw + 1) * 4,
                             "ms_per_step": e2e_s * 1e3, "streaming": stream_info}, link),
           "roofline": dom, "kernels": kernels,
           "gpu_launches": sum(v[1] for v in stages.values()),
           "stage_ms": {k: v[0] / steps for k, v in stages.items()}}
    return res, pinned


def measure_batch(local, ws, steps, warmup, m=None):
    """Workload 4: 16 uneven cohorts scanned by one gwas_scan_batch (a CUDA graph whose launch
    plan the library picked by timing), against the same scans issued cohort by cohort."""
    import torch
    import paper_1207_2169_gb300 as g
    from oracle import gls
    spec = synth.BATCH
    m = spec["m"] if m is None else m
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
            B = torch.full((m, t, q + 1), float("nan"), dtype=torch.float32, device="cuda")
            W = torch.full((m, t), float("nan"), dtype=torch.float32, device="cuda")
            blocks.append((G, B, W))
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        g.gwas_scan_batch(b, blocks, stream=stream.cuda_stream)  # picks the launch plan
        plan, plan_ms = g.gwas_batch_plan(b)
        tuning = g.gwas_batch_tuning(b)
        torch.cuda.synchronize()
        eb = ew = 0.0
        for (snps, j, Xs), c, (G, B, W) in zip(samples, cohorts, blocks):
            Bd = B[torch.from_numpy(snps).cuda(), j].cpu().numpy().astype(np.float64)
            Wd = W[torch.from_numpy(snps).cuda(), j].cpu().numpy().astype(np.float64)
            pairs = np.c_[np.arange(len(snps)), np.full(len(snps), j)]
            Bref, Wref, Vref = gls.gls_pairs(c.Phi, c.XL, Xs, c.Y, c.h2, c.s2, pairs)
            e1, e2 = gls.max_rel_errors(Bd, Wd, Bref, Wref, Vref)
            eb, ew = max(eb, e1), max(ew, e2)
        for _ in range(warmup):
            g.gwas_scan_batch(b, blocks, stream=stream.cuda_stream)
        with ClockSampler(local) as clk:
            _barrier(ws)
            ms = _timed(stream, steps, lambda: g.gwas_scan_batch(b, blocks, stream=stream.cuda_stream),
                        False, None)
            _barrier(ws)
        ms = _max_over_ranks(ms / steps, ws)
        # the same work as separate per-cohort calls (each launch with every SM, one after another)
        handles = [g.gwas_batch_handle(b, i) for i in range(len(cohorts))]
        pieces = [g.gwas_split_pieces(h) for h in handles]

        def seq():
            for h, (G, B, W) in zip(handles, blocks):
                g.gwas_scan_packed(h, G, B, W, stream=stream.cuda_stream)

        for _ in range(2):
            seq()
        ms_seq = _max_over_ranks(_timed(stream, steps, seq, False, None) / steps, ws)
        # kernels per batched step: the same stages the per-cohort calls launch, counted by events
        for h in handles:
            g.gwas_stage_timing(h, True)
        seq()
        launches = 0
        for h in handles:
            launches += sum(v[1] for v in g.gwas_stage_times(h).values())
            g.gwas_stage_timing(h, False)
    finally:
        g.gwas_destroy_batch(b)
    pairs = m * sum(t for _, _, t in shapes)
    exe = sum(sum(stage_executed(dict(n=n, q=q, t=t, algo="eig"), m, pc).values())
              for (n, q, t), pc in zip(shapes, pieces))
    alg = sum(algorithmic_flops(dict(n=n, q=q, t=t, algo="eig"), m) for n, q, t in shapes)
    peaks, kind = _peaks()
    peak = peaks["bf16_tflops"]
    return {
        "value": pairs * ws / (ms * 1e-3), "unit": "pairs/s", "ms_per_step": ms, "steps": steps,
        "warmup": warmup,
        "config": {"workload": spec["name"], "cohorts": [dict(n=n, p=q + 1, t=t) for n, q, t in shapes],
                   "m": m, "genotypes": "packed", "algo": "eig (t > 1)", "precision": "split_bf16",
                   "l2": "inputs (packed genotypes, %.2f GB) exceed the 129 MB L2; no flush" %
                         (m * sum(-(-n // 64) * 16 for n, _, _ in shapes) / 1e9)},
        "gpu_launches": steps * launches,
        "batch": {"plan": plan, "plan_ms": plan_ms,
                  "plans": ["sequential", "concurrent, SM shares by work", "concurrent, all SMs",
                            "two lanes of half the SMs"],
                  "eig_chunk_div": tuning["chunk_div"],
                  "tuning_ms_by_chunk_div_and_plan": tuning["ms"],
                  "gain_of_chunk_tuning": min(tuning["ms"][0]) / min(min(r) for r in tuning["ms"]),
                  "per_cohort_calls_ms": ms_seq, "speedup_vs_per_cohort_calls": ms_seq / ms,
                  "split_pieces": pieces},
        "roofline": {"bound": "tensor", "kernel": "whole batched step (16 cohorts' EIG kernels)",
                     "achieved": alg / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": alg / (ms * 1e-3) / 1e12 / peak,
                     "executed_tflops": exe / (ms * 1e-3) / 1e12,
                     "executed_frac": exe / (ms * 1e-3) / 1e12 / peak, "traffic": None,
                     "peak_source": f"bf16_tflops (burst), {kind}"},
        "parity": {"max_rel_err_b": eb, "max_rel_err_wald": ew, "pairs_checked": 4 * len(shapes),
                   "tolerance": 1e-4},
        "setup_s": setup_s, "clocks": clk.summary(),
    }


def fp64_peak_tflops():
    """FP64 throughput of this GPU measured here (cuBLAS DGEMM 4096^3 through torch, best of 3):
    the denominator of the FP64 step-1 kernel's roofline."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * 4096 ** 3 / (best * 1e-3) / 1e12


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
    peak = fp64_peak_tflops() * 1e3
    return {"config": {"workload": f"estimate_{method}_n{n}_t{t}", "n": n, "q": q, "t": t,
                       "method": method, "grid": 101, "search": "golden section, 64 steps"},
            "value": t / (total * 1e-3), "unit": "traits/s", "ms_per_step": total,
            "ms_eigendecomposition": float(ms[0]), "ms_search": float(ms[1]),
            "parity": {"max_rel_err_crit": float(np.max(np.abs(ll[sel] - llr) / np.abs(llr))),
                       "max_abs_err_h2": float(np.max(np.abs(h2[sel] - h2r))),
                       "max_rel_err_s2": float(np.max(np.abs(s2[sel] - s2r) / s2r)),
                       "traits_checked": int(sample), "tolerance_crit": 1e-8},
            "roofline": {"bound": "alu", "kernel": "estimate_kernel (per-trait search)",
                         "achieved": flops / (ms[1] * 1e-3) / 1e9, "peak": peak,
                         "unit": "GFLOP/s", "frac": flops / (ms[1] * 1e-3) / 1e9 / peak,
                         "traffic": None,
                         "peak_source": "FP64 DGEMM (cuBLAS, 4096^3, best of 3) measured in this "
                                        "run; MEASURED_PEAKS.json has no FP64 figure"},
            "cpu_baseline": {"value": sample / cpu_s, "unit": "traits/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{sample} of the {t} traits, FP64 oracle (H formed and "
                                       f"factored per evaluation), {cpu_s:.1f} s"}}


def other_workloads(args, ws, local, head):
    """Every workload besides the headline, each as an entry of the headline's line."""
    out = []
    k = max(3, args.steps // 2)
    w = args.warmup

    def add(fn, *a, **kw):
        try:
            out.append(fn(*a, **kw))
        except Exception as e:  # one workload's failure must not lose the others' numbers
            out.append({"workload_error": f"{fn.__name__}: {type(e).__name__}: {e}"})
        print(f"# other workload {len(out)} done", file=sys.stderr, flush=True)

    # headline workload with int8 genotypes as input (packed on the device inside each step)
    def int8_head():
        r = measure(1, "split_bf16", k, w, local, ws, fmt="int8")
        return entry(r, "split_bf16", "int8", k, w)
    add(int8_head)

    # the headline workload with the FP16 hi + E4M3 lo split of L^-1 (SPLIT_FP8), oracle on 2,000
    # sampled SNPs, and its speedup over the split-BF16 headline
    def fp8_head():
        r = measure(1, "split_fp8", k, w, local, ws, parity_count=2000)
        e = entry(r, "split_fp8", "packed", k, w)
        if args.precision == "split_bf16":
            e["speedup_over_split_bf16"] = r["value"] / head["value"]
        return e
    add(fp8_head)

    # the plain FP32 CUDA-core form of the headline, and the speedup at equal accuracy
    def fp32_head():
        r = measure(1, "fp32", 3, w, local, ws, fmt="int8", e2e=False)
        e = entry(r, "fp32", "int8", 3, w)
        if r["parity"]["max_rel_err_b"] < 1e-4 and r["parity"]["max_rel_err_wald"] < 1e-4:
            e["speedup_of_split_bf16_at_equal_accuracy"] = head["value"] / r["value"]
        return e
    add(fp32_head)

    # workload 0 as stated (FP64 CUDA cores, every SNP checked), and on the tensor cores
    for prec in ("fp64", "split_bf16"):
        def w0(prec=prec):
            fmt = "int8" if prec == "fp64" else "packed"
            r = measure(0, prec, max(k, 10), w, local, ws, fmt=fmt, every=True)
            return entry(r, prec, fmt, max(k, 10), w)
        add(w0)

    # the many-trait EIG workload and its CUDA-core forms
    eig = {}

    def w2():
        r = measure(2, "split_bf16", k, w, local, ws)
        eig["split"] = r["value"]
        return entry(r, "split_bf16", "packed", k, w)
    add(w2)

    def w2_fp32():
        r = measure(2, "fp32", 3, w, local, ws, fmt="int8", e2e=False)
        e = entry(r, "fp32", "int8", 3, w)
        if "split" in eig and r["parity"]["max_rel_err_b"] < 1e-4:
            e["speedup_of_split_bf16_at_equal_accuracy"] = eig["split"] / r["value"]
        return e
    add(w2_fp32)

    def w2_fp64():
        r = measure(2, "fp64", 3, w, local, ws, m=20000, fmt="int8", e2e=False)
        return entry(r, "fp64", "int8", 3, w, note="first 20,000 SNPs of the workload (pairs/s "
                     "is independent of m at this size)")
    add(w2_fp64)

    # the omics-scale EIG workload streamed as stated, full and SNP-only outputs
    pinned = [None]
    for mode in ("full", "snp"):
        def w3(mode=mode):
            r, pinned[0] = measure_stream3(local, ws, steps=2, warmup=1, out_mode=mode,
                                           pinned=pinned[0])
            return entry(r, "split_bf16", "packed", 2, 1,
                         config={"out_mode": mode, "blocks": "31 calls of 32,768 SNPs (the last "
                                 "16,960) per step", "step": "the whole 10^6-SNP genome"})
        add(w3)
    pinned[0] = None

    # the batch of 16 uneven cohorts
    add(measure_batch, local, ws, 3, w)
    add(measure_estimate)
    return out


def run_ours(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.workload == 4:
        line = measure_batch(local, ws, args.steps, args.warmup, m=args.m)
        if rank == 0:
            line.update({"metric": METRIC, "n_gpus": ws, "higher_is_better": True,
                         "scaling": "weak", "vs_baseline": None, "dtype": "bf16x2->f32",
                         "data": "synthetic"})
            print(json.dumps(line), flush=True)
        return
    if args.workload == 3:
        res, _ = measure_stream3(local, ws, steps=args.steps, warmup=args.warmup, m=args.m,
                                 out_mode=args.out_mode)
        fmt = "packed"
    else:
        res = measure(args.workload, args.precision, args.steps, args.warmup, local, ws, m=args.m,
                      fmt=args.format, every=args.workload == 0,
                      parity_count=2000 if args.workload == 1 else 256)
        fmt = args.format
    s = res["s"]
    other = []
    if not args.no_other and args.workload == 1 and args.m is None:
        other = other_workloads(args, ws, local, res)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": res["value"], "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision],
        "data": "synthetic",
        "config": dict(_config(s, args.precision, res["m"], fmt),
                       **({"sharding": f"rank r scans SNPs [r*{res['m']}, (r+1)*{res['m']}) of a "
                                       f"{ws * res['m']}-SNP genome (gwas_shard)"} if ws > 1 else {})),
        "e2e": res["e2e"], "gpu_launches": res["gpu_launches"],
        "roofline": res["roofline"], "parity": res["parity"], "setup_ms": res["setup_ms"],
        "clocks": res["clocks"], "stage_ms_per_step": res["stage_ms"],
    }
    if len(res["kernels"]) > 1:
        line["kernel_rooflines"] = res["kernels"]
    if other:
        line["other_workloads"] = other
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload if args.workload in (0, 2) else 1,
                                            args.cpu_sample)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=1)
    ap.add_argument("--precision", default="split_bf16", choices=list(DTYPE))
    ap.add_argument("--format", default="packed", choices=["packed", "int8"],
                    help="genotype input format of the timed scans")
    ap.add_argument("--out-mode", default="full", choices=["full", "snp"],
                    help="output mode of workload 3")
    ap.add_argument("--m", type=int, default=None, help="override the SNP count (profiling only)")
    ap.add_argument("--cpu-sample", type=int, default=400_000)
    ap.add_argument("--ref-sample", type=int, default=20_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="measure the headline workload only")
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
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
