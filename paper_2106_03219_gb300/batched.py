"""Batched target regions: build the region set, run it as one persistent
kernel or as one launch per region, and time the forms against each other.

The region set stands in for an application that launches thousands of short
target regions of uneven length (the paper's miniQMC measurement, Sec. 4.3,
times two such regions launched tens of thousands of times).  Trip counts are
lognormal, clipped to [100, 10^6]; each region is an fp32 axpy, an fp32 dot
product with a sum reduction, or a 1-D 3-point stencil, on disjoint slices of
one allocation.
"""

from . import inputs
from . import omprt as R

BYTES_PER_ITER = {inputs.KIND_AXPY: 12, inputs.KIND_DOT: 8, inputs.KIND_STENCIL1D: 8}


class RegionSet:
    def __init__(self, nregions=4096, seed=inputs.META_SEED, alpha=3.0):
        import torch
        self.n, self.kind, self.offset = inputs.batched_regions(nregions, seed)
        total = int(self.offset[-1] + (self.n[-1] + 63) // 64 * 64)
        self.total = total
        self.x0 = inputs.f32_uniform01(total, 0)
        self.y0 = inputs.f32_uniform01(total, 1)
        self.x = torch.from_numpy(self.x0).cuda()
        self.y = torch.from_numpy(self.y0).cuda()
        self.out = torch.zeros(total, dtype=torch.float32, device="cuda")
        self.res = torch.zeros(nregions, dtype=torch.float64, device="cuda")
        self.alpha = alpha
        self.descs, self.reds = [], []
        for r in range(nregions):
            n, k, o = int(self.n[r]), int(self.kind[r]), int(self.offset[r])
            xs, ys, os_ = self.x[o:o + n], self.y[o:o + n], self.out[o:o + n]
            if k == inputs.KIND_AXPY:
                d = R.loop_desc(R.BODY_AXPY, n=n, x=xs, y=ys, alpha=alpha)
                red = R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, None)
            elif k == inputs.KIND_DOT:
                d = R.loop_desc(R.BODY_DOT, n=n, x=xs, y=ys)
                red = R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, self.res[r:r + 1].data_ptr())
            else:
                d = R.loop_desc(R.BODY_STENCIL1D3, n=n, x=xs, out=os_)
                red = R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, None)
            self.descs.append(d)
            self.reds.append(red)

    @property
    def nregions(self):
        return len(self.descs)

    def algorithmic_bytes(self):
        return int(sum(BYTES_PER_ITER[int(k)] * int(n) for k, n in zip(self.kind, self.n)))

    def reset(self):
        import torch
        self.y.copy_(torch.from_numpy(self.y0))
        self.out.zero_()
        self.res.zero_()

    def batch(self, rt, chunk_elems=0):
        return rt.batch_create(self.descs, self.reds, chunk_elems)

    def launch_per_region(self, rt, threads=256, stream=None):
        """One launch per region with the plain heuristic (auto mapping,
        runtime-chosen teams)."""
        for d, red in zip(self.descs, self.reds):
            rt.launch_region(d, R.SCHED_AUTO, 0, 0, threads,
                             red=red if red.result_dev else None, stream=stream)


def time_forms(rt, rs, reps=5, chunk_elems=0, threads=256):
    """Median device time (ms) of the per-region launch loop (eager and under a
    CUDA graph) and of the persistent kernel (eager and under a graph)."""
    import statistics
    import torch

    stream = torch.cuda.Stream()
    b = rs.batch(rt, chunk_elems)

    def timed(fn):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                fn()
                e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    per_region = lambda: rs.launch_per_region(rt, threads, stream=stream)
    persistent = lambda: b.launch(0, threads, stream=stream)
    per_region()
    persistent()
    torch.cuda.synchronize()
    out = {"per_region_eager_ms": timed(per_region), "persistent_eager_ms": timed(persistent)}
    for name, fn in (("per_region_graph_ms", per_region), ("persistent_graph_ms", persistent)):
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            fn()
        g.replay()
        torch.cuda.synchronize()
        out[name] = timed(g.replay)
    assert rt.sync_status() == 0
    items = b.items
    b.destroy()
    nbytes = rs.algorithmic_bytes()
    for k in list(out):
        out[k.replace("_ms", "_regions_per_s")] = rs.nregions / (out[k] * 1e-3)
        out[k.replace("_ms", "_GBps")] = nbytes / (out[k] * 1e-3) / 1e9
    out["regions"] = rs.nregions
    out["iterations"] = int(rs.n.sum())
    out["algorithmic_bytes"] = nbytes
    out["items"] = items
    out["chunk_elems"] = chunk_elems or 8192
    out["threads"] = threads
    return out
