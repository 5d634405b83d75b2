"""The N > 1 host path of bench.py (weak scaling, barrier + max-over-ranks timing) on two gloo
ranks on CPU.  The GPU work of each rank is an independent replica; only the timing reduction
crosses ranks, so that is what is exercised here."""
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
