"""The N > 1 host path on two gloo ranks on CPU: the SNP-range split (gwas_shard, host-only in
the C library) and bench.py's weak scaling with barrier + max-over-ranks timing.  No pair of
the grid depends on another, so each rank scans its own SNP range with no exchange on the data
path; here each rank solves its range with the FP64 oracle (the CPU stand-in for its GPU) and
the gathered ranges must equal the whole grid bit for bit.  Only the timing reduction and this
check cross ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench._barrier(ws)
    mx = bench._max_over_ranks(1.5 + rank, ws)  # rank-dependent "step time"
    out[rank] = mx
    bench._barrier(ws)
    dist.destroy_process_group()


def test_two_rank_max_timing():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_single_rank_is_identity():
    import bench
    assert bench._max_over_ranks(3.25, 1) == 3.25
    bench._barrier(1)


def test_work_accounting():
    """Algorithmic and executed FLOP counts used by the roofline."""
    import bench
    import synth
    s = dict(synth.WORKLOADS[1])
    n, q = s["n"], s["q"]
    assert bench.algorithmic_flops(s, 10) == 10 * (n * (n + 1) + 2 * n * (q + 2))
    # executed: 2 pieces x 2 flops x MACs: 64-column K steps over kpad = 1024; blocks of 256 rows
    # of the augmented L^-1 (1000 + q + 1 = 1004 rows: the last block has 240 live rows); on a
    # block's diagonal, step 4 nb + j meets rows 64 j onwards
    live = [256, 256, 256, 240]
    macs = sum(64 * (live[nb] - 64 * max(0, ks - 4 * nb)) for nb in range(4) for ks in range(4 * (nb + 1)))
    assert bench.stage_executed(s, 1) == {"chol": 4 * macs}
    assert bench.stage_executed(s, 1)["chol"] > 2 * bench.algorithmic_flops(s, 1)
    # EIG, per kernel: rotation 2 n^2 per SNP, s 2n per pair, a and c 2n(q+1) per pair
    e = dict(synth.WORKLOADS[2])
    n, q, t = e["n"], e["q"], e["t"]
    assert bench.stage_flops(e, 3) == {"rot": 3 * 2 * n * n, "sq": 3 * t * 2 * n,
                                       "ac": 3 * t * 2 * n * (q + 1)}
    # executed: rotation 2 pieces over 1024 x 1024 padded; s 3 products over 1024 traits (t
    # rounded up to 256-column blocks); a, c 2 products over 16 blocks of 64 traits x 256 columns
    assert bench.stage_executed(e, 1) == {"rot": 4 * 1024 * 1024, "sq": 6 * 1024 * 1024,
                                          "ac": 4 * 1024 * 256 * 16}
    assert bench.eig_ac_traits(3) == 64 and bench.eig_ac_traits(7) == 32


def test_code_hash_ignores_comments(tmp_path):
    """The DRAM counters of a kernel stay valid across comment-only edits of its source."""
    import bench
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) {  // doubles\n  return 2 * x; /* twice */\n}\n")
    b.write_text("// a header comment\nint f(int x) {\n  return 2 * x;\n}\n")
    assert bench.code_sha1(a) == bench.code_sha1(b)
    b.write_text("int f(int x) {\n  return 3 * x;\n}\n")
    assert bench.code_sha1(a) != bench.code_sha1(b)


def test_shard_ranges_cover_the_genome():
    """Contiguous, disjoint, ordered ranges covering [0, m); whole align-units except at the end;
    unit counts differing by at most one; bad arguments rejected."""
    import paper_1207_2169_gb300 as g
    for m in (0, 1, 7, 1000, 65535, 2_000_000):
        for world in (1, 2, 3, 8):
            for align in (1, 64, 65536):
                got = [g.gwas_shard(m, r, world, align) for r in range(world)]
                pos = 0
                units = []
                for start, count in got:
                    assert start == pos and count >= 0
                    pos += count
                    if start + count < m:
                        assert count % align == 0
                    units.append(-(-count // align))
                assert pos == m
                assert max(units) - min(units) <= 1
    for bad in ((-1, 0, 2, 1), (10, 2, 2, 1), (10, -1, 2, 1), (10, 0, 0, 1), (10, 0, 2, 0)):
        with pytest.raises(RuntimeError):
            g.gwas_shard(*bad)


def _shard_main(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import paper_1207_2169_gb300 as g
    import synth
    from oracle import gls
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = synth.small_problem(81, n=40, q=2, m=37, t=3)
    start, count = g.gwas_shard(c.m, rank, world)
    B, W, _ = gls.gls_grid(c.Phi, c.XL, c.XR[start:start + count], c.Y, c.h2, c.s2)
    parts = [None] * world
    dist.all_gather_object(parts, (start, B, W))
    if rank == 0:
        parts.sort(key=lambda x: x[0])
        Ball = np.concatenate([p[1] for p in parts])
        Wall = np.concatenate([p[2] for p in parts])
        Bref, Wref, _ = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
        out["ok"] = bool(np.array_equal(Ball, Bref, equal_nan=True)
                         and np.array_equal(Wall, Wref, equal_nan=True))
    # bench.py's inputs on this rank: its own range of a genome of world x m SNPs
    import bench
    x = bench.make_inputs(0, m=3000, shard=True).XR
    out[rank] = bool(np.array_equal(x, synth.workload_genotypes(0, 3000, start=3000 * rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_scan_their_own_snp_ranges():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    assert dict(out) == {"ok": True, 0: True, 1: True}
