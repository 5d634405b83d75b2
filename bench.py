#!/usr/bin/env python
"""Throughput of the GLS grid scan on one GB300: (SNP x trait) GLS solves per second.

Default workload: single-trait genome scan, CLAK-Chol with the split-BF16 tensor-core whitening:
n = 1,000 individuals, p = 4 (intercept, two covariates, SNP), m = 2,000,000 SNPs as int8 hard
calls, h2 = 0.5, s2 = 1.  One step = one gwas_scan over all m SNPs (every SNP's GLS solved and
its Wald statistic written).  `value` is measured with the genotypes already resident in HBM
(2 GB, larger than L2, so no flush is needed between steps); `e2e` is the same metric through
the same C call with pinned HOST genotype and output buffers (the library streams 64 Ki-SNP
blocks with double-buffered copies).  `--impl reference` times the FP64 CPU oracle instead.

Launch: python bench.py [--gpus N --steps K --warmup W] [--workload 1|0|2] [--precision P]
Under torchrun (N > 1) every rank scans its own replica of the workload (weak scaling, no
collective on the data path); rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
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
            d = json.load(f)
        return d, "measured"
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
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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


def workload_spec(idx: int):
    s = dict(synth.WORKLOADS[idx])
    return s


def make_inputs(idx: int, m: int | None = None):
    s = workload_spec(idx)
    m = s["m"] if m is None else m
    c = synth.make_cohort(idx, m=0, with_genotypes=False)
    # genotypes in lazily drawn blocks (each block has its own seeded stream)
    blk = s["block"]
    XR = np.empty((m, s["n"]), dtype=np.int8)
    for b in range((m + blk - 1) // blk):
        lo, hi = b * blk, min(m, (b + 1) * blk)
        XR[lo:hi] = synth.snp_block(idx, s["n"], blk, b)[:hi - lo]
    c.XR = XR
    return c


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle, as it stands
# ------------------------------------------------------------------------------------------

def run_reference(args, ws, rank):
    if rank != 0:
        return
    from oracle import gls
    s = workload_spec(args.workload)
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
        "data": "synthetic", "config": _config(args, s),
        "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"first {sample} SNPs of the workload per step"},
        "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, s):
    return {"workload": s["name"], "n": s["n"], "p": s["q"] + 1, "m": s["m"], "t": s["t"],
            "algo": s["algo"], "precision": args.precision, "block_snps": s["block"],
            "l2": "inputs (m x n int8 = %.1f GB) exceed the 129 MB L2; no flush" % (s["m"] * s["n"] / 1e9)}


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
                      f"(Algorithm 1 per GLS), {dt:.1f} s"}


def parity_sample(g, h, c, Bd, Wd, count=256):
    """Max errors of the bench run's own outputs against the oracle on sampled pairs."""
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


def run_ours(args, ws, rank, local):
    import torch
    import paper_1207_2169_gb300 as g

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    s = workload_spec(args.workload)
    c = make_inputs(args.workload, m=args.m)
    m, n, t, p = c.m, c.n, c.t, c.p
    opt = g.gwas_default_options(algo=s["algo"], precision=args.precision, device=local)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, options=opt)
    setup_ms = g.gwas_setup_timing(h)
    xr_d = torch.from_numpy(c.XR).cuda()
    B_d = torch.empty((m, t, p), dtype=torch.float32, device="cuda")
    W_d = torch.empty((m, t), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        g.gwas_scan(h, xr_d, B_d, W_d, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        _barrier(ws)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        _barrier(ws)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = _max_over_ranks(ms, ws)
    pairs = m * t
    value = pairs * ws / (ms * 1e-3)
    clocks = clk.summary()
    eb, ew, npairs = parity_sample(g, h, c, B_d.cpu().numpy(), W_d.cpu().numpy())

    # end to end: pinned host genotypes in, pinned host results out, through the same call
    xr_h = torch.from_numpy(c.XR).pin_memory()
    B_h = torch.empty((m, t, p), dtype=torch.float32).pin_memory()
    W_h = torch.empty((m, t), dtype=torch.float32).pin_memory()
    g.gwas_scan(h, xr_h, B_h, W_h)  # warm the ring
    e2e_steps = max(1, min(args.steps, 5))
    _barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.gwas_scan(h, xr_h, B_h, W_h)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = _max_over_ranks(e2e_s, ws)
    same = bool(torch.equal(B_h, B_d.cpu()))

    peaks, peak_kind = _peaks()
    kinfo = g_kernel_info(args, s, m, t, ms)
    roof = None
    if kinfo:
        peak = peaks["bf16_tflops_sustained"] if kinfo["unit"] == "TFLOP/s" else peaks["hbm_gbs"]
        roof = {"bound": kinfo["bound"], "achieved": kinfo["achieved"], "peak": peak,
                "unit": kinfo["unit"], "frac": kinfo["achieved"] / peak, "traffic": kinfo.get("traffic"),
                "kernel": kinfo["kernel"], "peak_source": f"{peak_kind} (MEASURED_PEAKS.json)",
                "executed": kinfo.get("executed")}
    g.gwas_destroy(h)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"split_bf16": "bf16x2->f32", "fp32": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic", "config": _config(args, s),
        "e2e": {"value": pairs * ws / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": m * n,
                "d2h_bytes_per_step": m * t * (p + 1) * 4, "ms_per_step": e2e_s * 1e3,
                "matches_device_run": same},
        "gpu_launches": args.steps * launches_per_scan(args, s, m),
        "roofline": roof,
        "parity": {"max_rel_err_b": eb, "max_rel_err_wald": ew, "pairs_checked": npairs,
                   "tolerance": 1e-4 if args.precision != "fp64" else 1e-6},
        "setup_ms": setup_ms,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample)
    print(json.dumps(line), flush=True)


def launches_per_scan(args, s, m):
    if s["algo"] == "chol":
        return 1 if args.precision == "split_bf16" else 1
    return 2


def g_kernel_info(args, s, m, t, ms_step):
    """Algorithmic work of the dominant kernel per launch over its measured time.

    CHOL whitening + reduction: n(n+1) flops per SNP for X' = L^-1 x (a lower-triangular product)
    plus 2n(q+2) for the reductions.  The step is one launch of that kernel, so the step time
    bounds its duration from above."""
    n, q = s["n"], s["q"]
    if s["algo"] == "chol":
        flops = m * (n * (n + 1) + 2 * n * (q + 2))
        achieved = flops / (ms_step * 1e-3) / 1e12
        pieces = 2 if args.precision == "split_bf16" else 1
        return {"bound": "tensor" if args.precision == "split_bf16" else "alu", "unit": "TFLOP/s",
                "achieved": achieved, "kernel": "chol whiten+reduce",
                "executed": achieved * pieces}
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=1)
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "fp32", "fp64"])
    ap.add_argument("--m", type=int, default=None, help="override the SNP count (testing only)")
    ap.add_argument("--cpu-sample", type=int, default=100_000)
    ap.add_argument("--ref-sample", type=int, default=20_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
