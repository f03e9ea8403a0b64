"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module draws random numbers and lays them out; it holds none of the
runtime's arithmetic (no schedule, body or reduction).  Both the CUDA path and
the CPU oracle receive the same bytes from here.

The paper measures on SPEC ACCEL and miniQMC (Sec. 4.3), which are not
available; these synthetic recipes stand in for them:
  * streaming loops over large fp32 / int32 arrays (the stencil-class codes),
  * thousands of short target regions of uneven length (miniQMC's many short
    region launches, Sec. 4.3 table).
RNG: numpy PCG64 via default_rng(seed); seed for the first operand, seed+1 for
the second, 1234 for metadata (trip counts, kinds, traces).
"""
import numpy as np

META_SEED = 1234


def rng(seed):
    return np.random.default_rng(seed)


def int32_uniform(n, seed, lo=-(1 << 20), hi=(1 << 20)):
    """int32 uniform in [lo, hi)."""
    return rng(seed).integers(lo, hi, size=n, dtype=np.int64).astype(np.int32)


def f32_uniform01(n, seed):
    """fp32 uniform in [0, 1)."""
    return rng(seed).random(n, dtype=np.float32)


def f32_uniform_pm1(n, seed):
    """fp32 uniform in [-1, 1] (drawn in fp64, rounded once to fp32)."""
    return rng(seed).uniform(-1.0, 1.0, size=n).astype(np.float32)


def f32_lognormal_signed(n, seed, sigma=3.0):
    """sign * exp(N(0, sigma^2)), sign a fair coin, rounded once to fp32."""
    g = rng(seed)
    mag = np.exp(g.normal(0.0, sigma, size=n))
    sign = np.where(g.random(n) < 0.5, -1.0, 1.0)
    return (sign * mag).astype(np.float32)


def bf16_bits_from_f32(a):
    """Round fp32 values to bf16 (nearest, ties to even); return uint16 patterns."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def bf16_uniform_pm1(n, seed):
    return bf16_bits_from_f32(f32_uniform_pm1(n, seed))


def int64_uniform(n, seed, lo=-(1 << 31), hi=(1 << 31)):
    return rng(seed).integers(lo, hi, size=n, dtype=np.int64)


def grid_f32(ny, nx, seed):
    return f32_uniform01(ny * nx, seed).reshape(ny, nx)


# -- batched regions -------------------------------------------------------------

KIND_AXPY, KIND_DOT, KIND_STENCIL1D = 0, 1, 2


def batched_regions(nregions=4096, seed=META_SEED, lo=100, hi=1_000_000,
                    median=1e4, log_sd=np.log(10.0)):
    """Trip counts round(exp(N(ln median, log_sd^2))) clipped to [lo, hi] and a
    kind drawn uniformly from {axpy, dot, stencil1d}.  Returns (n[int64],
    kind[int32], offset[int64]) where offset is each region's start in one
    packed fp32 allocation (regions are disjoint, starts 64-element aligned)."""
    g = rng(seed)
    n = np.rint(np.exp(g.normal(np.log(median), log_sd, size=nregions)))
    n = np.clip(n, lo, hi).astype(np.int64)
    kind = g.integers(0, 3, size=nregions).astype(np.int32)
    padded = (n + 63) // 64 * 64
    offset = np.concatenate([[0], np.cumsum(padded)[:-1]]).astype(np.int64)
    return n, kind, offset


# -- stack-allocator traces --------------------------------------------------------

def stack_trace(nops, seed=META_SEED, max_bytes=4096, p_free=0.45, bad_free=False):
    """A random alloc/free trace as int64 pairs (kind, arg): kind 0 allocates arg
    bytes, kind 1 frees allocation number arg.  Frees are LIFO over the live
    allocations unless bad_free, which makes some frees name a non-top block."""
    g = rng(seed)
    ops, live, nalloc = [], [], 0
    for _ in range(nops):
        if live and g.random() < p_free:
            if bad_free and len(live) > 1 and g.random() < 0.3:
                j = int(g.integers(0, len(live) - 1))
                ops.append((1, live.pop(j)))
            else:
                ops.append((1, live.pop()))
        else:
            ops.append((0, int(g.integers(0, max_bytes + 1))))
            live.append(nalloc)
            nalloc += 1
    return np.array(ops, dtype=np.int64).reshape(-1, 2)


# -- learned-schedule loop set ------------------------------------------------------

LOOP_KINDS = ("axpy", "dot", "stencil1d3", "stencil2d5", "reduce_sum")


def loop_set(count, seed, log2_lo=10, log2_hi=26):
    """count loops: kind uniform over LOOP_KINDS, trip count log-uniform in
    [2^log2_lo, 2^log2_hi].  Returns (kind[int32], n[int64])."""
    g = rng(seed)
    kind = g.integers(0, len(LOOP_KINDS), size=count).astype(np.int32)
    n = np.rint(np.exp2(g.uniform(log2_lo, log2_hi, size=count))).astype(np.int64)
    return kind, n


# -- counter-based values for loops too large to draw on the host -------------
# Value i of stream `seed` is a function of (i, seed) alone, so a device fill of
# billions of elements and a host evaluation of a few sampled indices give the
# same bytes.  The 32-bit mixer is the xor-shift-multiply integer hash with
# multiplier 0x45d9f3b (T. Mueller); with a multiplier below 2^27 every
# product of a 32-bit value stays below 2^59, so int64 arithmetic computes it
# exactly in numpy and in torch alike.

_M32 = 0xFFFFFFFF
_MUL = 0x45D9F3B


def _mix32(x):
    x = x ^ (x >> 16)
    x = (x * _MUL) & _M32
    x = x ^ (x >> 16)
    x = (x * _MUL) & _M32
    return x ^ (x >> 16)


def _hash_u32(i, seed):
    """32-bit hash of index i (int64 array or tensor, 0 <= i < 2^62) and seed."""
    hi = _mix32(((i >> 32) + 0x9E3779B9 * (seed + 1)) & _M32)
    return _mix32((i & _M32) ^ hi)


def counter_f32_01(idx, seed):
    """fp32 in [0, 1) with 24 random bits (exact in fp32), at int64 indices idx."""
    idx = np.asarray(idx, dtype=np.int64)
    return ((_hash_u32(idx, seed) >> 8).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def counter_f32_01_fill(t, seed, start=0, block=1 << 26):
    """Fill the 1-D fp32 tensor t (any device) with counter_f32_01(start + k,
    seed), k = 0 .. t.numel() - 1, in blocks of `block` elements."""
    import torch
    n = t.numel()
    for b in range(0, n, block):
        e = min(b + block, n)
        idx = torch.arange(start + b, start + e, dtype=torch.int64, device=t.device)
        t[b:e] = (_hash_u32(idx, seed) >> 8).to(torch.float32) * (2.0 ** -24)
    return t
