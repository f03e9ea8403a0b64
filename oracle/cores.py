"""Run oracle routines over disjoint slices on all host cores (TEST
INFRASTRUCTURE: the CPU-baseline timings of the benchmark).

Worker processes (started with `spawn`, so a parent that already uses CUDA is
never forked) map the parent's arrays (files in a temporary directory, mapped
shared) and each call one oracle routine on its own slice; nothing here does
any of the method's arithmetic.  Exact sums stay exact across slices: each
worker returns
its slice's exact sum as a non-overlapping expansion of doubles
(orc_exact_sum_*_terms) and the parent sums all terms with the oracle's exact
fp64 sum, which rounds once.  Timing is wall time from a common start (the
workers wait at a barrier) to the last worker's end, on the system-wide
monotonic clock.
"""
import multiprocessing as mp
import os
import shutil
import tempfile
import time

import numpy as np


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# -- worker side -------------------------------------------------------------------

_barrier = None


def _init(barrier):
    global _barrier
    _barrier = barrier


def _view(spec):
    path, shape, dtype = spec
    return np.memmap(path, dtype=np.dtype(dtype), mode="r+", shape=shape)


def _work(task):
    import oracle as O
    kind, specs, lo, hi, extra = task
    arrs = [_view(s) for s in specs]
    O.lib()  # loaded before the clock starts
    _barrier.wait(timeout=600)
    t0 = time.monotonic()
    out = None
    if kind == "axpy_f32":          # y[lo:hi] = fma(a, x, y) in place
        x, y = arrs
        y[lo:hi] = O.axpy_f32(extra, x[lo:hi], y[lo:hi])
    elif kind == "axpy_i32_sum":    # config 1: y = 3x + y (wrapping), then the int64 sum of y
        x, y = arrs
        y[lo:hi] = O.axpy_i32(extra, x[lo:hi], y[lo:hi])
        out = O.sum_int(y[lo:hi])
    elif kind == "stencil2d":       # output rows [lo, hi) from input rows lo-1 .. hi
        g, o = arrs
        a, b = max(lo - 1, 0), min(hi + 1, g.shape[0])
        res = O.stencil2d5(g[a:b])
        # the band's first / last row is a grid row only at the grid's edge;
        # otherwise it is a halo row, whose (copied) output is not kept
        o[lo:hi] = res[lo - a:lo - a + (hi - lo)]
    elif kind == "exact_terms":
        (a,) = arrs
        out = O.exact_sum_terms(a[lo:hi], bf16=bool(extra))
    elif kind == "plain_sum":
        (a,) = arrs
        out = O.plain_sum_f32(a[lo:hi])
    elif kind == "regions":         # batched regions lo .. hi-1 of a region table
        x, y, out_buf, table = arrs
        for r in range(lo, hi):
            kind_r, off, n = (int(v) for v in table[r])
            if kind_r == 0:
                y[off:off + n] = O.axpy_f32(3.0, x[off:off + n], y[off:off + n])
            elif kind_r == 1:
                O.exact_dot_f32(x[off:off + n], y[off:off + n])
            else:
                out_buf[off:off + n] = O.stencil1d3(x[off:off + n])
    else:
        raise ValueError(kind)
    t1 = time.monotonic()
    for a in arrs:
        a.flush()
    del arrs
    return t0, t1, out


class Cores:
    """A pool of `n` spawned workers (default: every host core)."""

    def __init__(self, n=None):
        self.n = n or host_cores()
        ctx = mp.get_context("spawn")
        self.barrier = ctx.Barrier(self.n)
        self.pool = ctx.Pool(self.n, initializer=_init, initargs=(self.barrier,))
        self.dir = tempfile.mkdtemp(prefix="oracle_cores_")
        self.count = 0

    def share(self, a):
        """Copy a into a file mapped by every worker; returns (spec, view)."""
        a = np.ascontiguousarray(a)
        path = os.path.join(self.dir, "a%d" % self.count)
        self.count += 1
        v = np.memmap(path, dtype=a.dtype, mode="w+", shape=a.shape if a.size else (1,))
        if a.size:
            v[...] = a
        v.flush()
        return (path, v.shape, a.dtype.str), v

    def run(self, kind, specs, total, extra=None, parts=None):
        """Split [0, total) into one contiguous part per worker (or `parts`,
        a list of (lo, hi)); returns (wall seconds, per-part results)."""
        if parts is None:
            cuts = [total * k // self.n for k in range(self.n + 1)]
            parts = list(zip(cuts[:-1], cuts[1:]))
        assert len(parts) == self.n
        res = self.pool.map(_work, [(kind, specs, lo, hi, extra) for lo, hi in parts],
                            chunksize=1)
        t0 = min(r[0] for r in res)
        t1 = max(r[1] for r in res)
        return t1 - t0, [r[2] for r in res]

    def close(self):
        self.pool.close()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)
