"""One loop sharded over GPUs: a distribute level above the teams.

Rank r of W gets the contiguous balanced block of the loop's n iterations
(C1 with P = W, the split level 1 gives teams), runs it through the library
on its own GPU, and a reduction's per-rank result (one 8-byte fp64 or int64
value) is exchanged with one all-gather of 8 bytes per rank and combined on
every rank in rank order: fp64 adds left to right for floating sums (the
same result on every rank and run for a fixed W), exact for max / min, and
int64 sums wrapping modulo 2^64.  No kernel reads another rank's memory;
the only data exchanged are the partials.

This is the multi-GPU form of the reduction the runtime finishes across teams
(partials, flush, last-team combine in team order, Sec. 3.1): the same
combine one level up, with ranks in place of teams.
"""
from . import omprt as R


def rank_block(n, world, rank):
    """(start, count) of rank's block: q + (rank < r) iterations from
    q * rank + min(rank, r), n = q * world + r."""
    q, r = divmod(int(n), int(world))
    return q * rank + min(rank, r), q + (1 if rank < r else 0)


def _wrap64(v):
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= (1 << 63) else v


def combine(parts, op, integer):
    """The rank-order combine of the per-rank partials (a list in rank order)."""
    if op == R.OP_MAX:
        return max(parts)
    if op == R.OP_MIN:
        return min(parts)
    if integer:
        return _wrap64(sum(int(p) for p in parts))
    s = 0.0
    for p in parts:  # Python floats are fp64: one rounding per add, left to right
        s = s + float(p)
    return s


def gather_partials(value, integer):
    """Every rank's 8-byte partial, in rank order (an all-gather; one rank: the
    value itself).  Uses the default process group, on its backend's device."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [value]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.int64 if integer else torch.float64, device=dev)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [o.item() for o in out]


def reduce_shard(rt, op, shard, precision=R.PREC_COMP_F64, teams=0, threads=0, stream=None):
    """This rank's partial: omprt_reduce over its own block (a device tensor),
    read back as a Python number (synchronises the stream)."""
    import torch
    integer = shard.dtype in (torch.int32, torch.int64)
    res = torch.zeros(1, dtype=torch.int64 if integer else torch.float64, device=shard.device)
    rt.reduce(op, shard, res, precision, teams, threads, stream=stream)
    return res.item(), integer


def sharded_reduce(rt, op, shard, precision=R.PREC_COMP_F64, teams=0, threads=0, stream=None):
    """reduction(op) over a loop whose blocks live on the ranks: this rank's
    partial on its GPU, then the all-gather and the rank-order combine.  Every
    rank returns the same value."""
    v, integer = reduce_shard(rt, op, shard, precision, teams, threads, stream)
    return combine(gather_partials(v, integer), op, integer)
