"""The benchmark's multi-rank host logic on CPU: two gloo ranks agree on the
maximum time over ranks (what bench.py divides the whole-job bytes by)."""
import os
import socket



def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        t = bench.max_over_ranks(10.0 + 3.5 * rank, ws)
        bench.barrier(ws)
        q.put((rank, t))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 13.5, 1: 13.5}


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(7.25, 1) == 7.25


def _shard_worker(rank, ws, port, q):
    """Rank r takes its block of each array; its partial (the GPU's per-rank
    result, here the oracle's value over the same block on the CPU, which
    the GPU tests hold the library to) goes through the all-gather and the
    rank-order combine."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import numpy as np
    import torch.distributed as dist
    import oracle as O
    from paper_2106_03219_gb300 import inputs, sharded
    from paper_2106_03219_gb300 import omprt as R
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        out = {}
        n = 100003
        s, c = sharded.rank_block(n, ws, rank)
        f = inputs.f32_lognormal_signed(n, 3)
        i64 = inputs.int64_uniform(n, 4)
        i64[::97] = (1 << 62)  # partial sums past 2^63: the combine must wrap
        for name, a, op, integer in (("sum_f32", f, R.OP_SUM, False),
                                     ("max_f32", f, R.OP_MAX, False),
                                     ("min_f32", f, R.OP_MIN, False),
                                     ("sum_i64", i64, R.OP_SUM, True)):
            blk = a[s:s + c]
            if op == R.OP_SUM:
                v = O.sum_int(blk) if integer else O.exact_sum_f32(blk)
            else:
                v = O.max_min(blk, "max" if op == R.OP_MAX else "min")
            out[name] = sharded.combine(sharded.gather_partials(v, integer), op, integer)
        out["block"] = (s, c)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_sharded_reduce_two_gloo_ranks():
    """The rank blocks tile [0, n) in rank order (C1 with P = 2); every rank
    ends with the same combined value; integer sums and max / min equal the
    oracle's over the whole array exactly; the fp32 sum (two fp64 partials
    added in rank order) is within the reduction bound of the exact sum."""
    import numpy as np
    import torch.multiprocessing as mp
    import oracle as O
    from paper_2106_03219_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    n = 100003
    assert got[0]["block"] == (0, 50002) and got[1]["block"] == (50002, 50001)
    assert got[0]["block"] == O.static_nochunk(n, 2, 0)
    for k in ("sum_f32", "max_f32", "min_f32", "sum_i64"):
        assert got[0][k] == got[1][k], k
    f = inputs.f32_lognormal_signed(n, 3)
    i64 = inputs.int64_uniform(n, 4)
    i64[::97] = (1 << 62)
    assert got[0]["max_f32"] == O.max_min(f, "max")
    assert got[0]["min_f32"] == O.max_min(f, "min")
    assert got[0]["sum_i64"] == O.sum_int(i64)
    exact = O.exact_sum_f32(f)
    bound = 1e-6 * max(abs(exact), 2.0 ** -24 * O.exact_abs_sum_f32(f))
    assert abs(got[0]["sum_f32"] - exact) <= bound


def test_rank_blocks_and_combine_rules():
    """rank_block is C1 (the oracle's static split) for several world sizes;
    the combine adds in rank order (fp64), takes max / min exactly and wraps
    int64 sums modulo 2^64."""
    import oracle as O
    from paper_2106_03219_gb300 import sharded
    from paper_2106_03219_gb300 import omprt as R
    for n in (0, 1, 7, 1000, (1 << 28) + 5):
        for ws in (1, 2, 3, 8):
            assert [sharded.rank_block(n, ws, r) for r in range(ws)] == \
                [O.static_nochunk(n, ws, r) for r in range(ws)]
    assert sharded.combine([2.0 ** 53, 1.0, 1.0], R.OP_SUM, False) == 2.0 ** 53
    assert sharded.combine([1.0, 1.0, 2.0 ** 53], R.OP_SUM, False) == 2.0 ** 53 + 2
    assert sharded.combine([(1 << 63) - 1, 1], R.OP_SUM, True) == -(1 << 63)
    assert sharded.combine([3.5, -1.0, 7.25], R.OP_MAX, False) == 7.25
    assert sharded.combine([3, -9, 7], R.OP_MIN, True) == -9
