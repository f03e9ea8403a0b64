"""Guard bands: every entry point writes only where it is told to.

Each output buffer is a slice of a larger allocation whose margins hold a
canary pattern; after the launch the margins must be unchanged.  Sizes are
odd and the slices start at misaligned offsets so the vector, head and tail
paths of every schedule run next to a margin.  (Stands in for an
out-of-bounds checker on this pool.)"""
import numpy as np
import pytest

from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu

MARGIN = 96


class Guarded:
    """A device buffer of n elements starting `offset` elements before a
    32-byte boundary, with canary bytes (0xA5) in margins on both sides."""

    def __init__(self, n, dtype, offset, fill=None):
        self.n = n
        self.lo = MARGIN - offset            # MARGIN elements of 4 or 8 bytes: 32-byte aligned
        base = np.zeros(n + 2 * MARGIN, dtype=dtype)
        base.view(np.uint8)[:] = 0xA5
        if fill is not None:
            base[self.lo:self.lo + n] = fill
        self.init = base
        self.buf = dev(base)
        self.view = self.buf[self.lo:self.lo + n]

    def check(self):
        got = host(self.buf)
        lo, hi = self.lo, self.lo + self.n
        assert np.array_equal(got[:lo].view(np.uint8), self.init[:lo].view(np.uint8)), "low margin"
        assert np.array_equal(got[hi:].view(np.uint8), self.init[hi:].view(np.uint8)), "high margin"


SCHEDS = [(R.SCHED_STATIC, 0), (R.SCHED_STATIC_CHUNKED, 1), (R.SCHED_STATIC_CHUNKED, 5),
          (R.SCHED_STATIC_CHUNKED, 64), (R.SCHED_DYNAMIC, 7), (R.SCHED_DYNAMIC, 256),
          (R.SCHED_DYNAMIC, 8), (R.SCHED_AUTO, 0), (R.SCHED_GUIDED, 3),
          (R.SCHED_NONMONOTONIC, 5), (R.SCHED_NONMONOTONIC, 64)]


@pytest.mark.parametrize("sched,chunk", SCHEDS)
@pytest.mark.parametrize("n,off", [(1, 1), (37, 3), (10007, 5), (65539, 7), (4099, 0),
                                   (65539, 0)])
def test_axpy_and_stencils_stay_in_bounds(rt, sched, chunk, n, off):
    x = inputs.f32_uniform01(n, 0)
    y = Guarded(n, np.float32, off, inputs.f32_uniform01(n, 1))
    xd = dev(x)
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=y.view), sched, chunk, 13, 64)
    y.check()
    out = Guarded(n, np.float32, off)
    rt.launch_region(R.loop_desc(R.BODY_STENCIL1D3, n=n, x=xd, out=out.view), sched, chunk, 7, 96)
    out.check()
    nx = 1 if n < 8 else 8 + off
    ny = n // nx
    out2 = Guarded(nx * ny, np.float32, off)
    g = dev(inputs.f32_uniform01(nx * ny, 2))
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=nx * ny, x=g, out=out2.view, nx=nx, ny=ny),
                     sched, chunk, 11, 128)
    out2.check()
    xi = dev(inputs.int32_uniform(n, 3))
    yi = Guarded(n, np.int32, off, inputs.int32_uniform(n, 4))
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xi, y=yi.view, alpha=3), sched, chunk, 5, 32)
    yi.check()
    assert rt.sync_status() == 0


@pytest.mark.parametrize("n", [0, 1, 1000, 40003])
def test_map_record_and_reductions_stay_in_bounds(rt, n):
    G, T = 9, 64
    owner = Guarded(max(n, 1), np.int32, 1)
    count = Guarded(max(n, 1), np.int32, 2, np.zeros(max(n, 1), np.int32))
    last = Guarded(G * T, np.int32, 3)
    for sched, chunk in SCHEDS:
        count.buf.copy_(dev(count.init))
        rt.launch_region(R.loop_desc(R.BODY_MAP_RECORD, n=n, x=last.view, y=count.view,
                                     out=owner.view, data_type=R.I32), sched, chunk, G, T)
        owner.check()
        count.check()
        last.check()
    res = Guarded(1, np.float64, 0)
    a = dev(inputs.f32_uniform_pm1(max(n, 1), 5))[:n]
    rt.reduce(R.OP_SUM, a, res.view, R.PREC_COMP_F64, 17, 96)
    res.check()
    resi = Guarded(1, np.int64, 0)
    b = dev(inputs.int64_uniform(max(n, 1), 6))[:n]
    rt.reduce(R.OP_SUM, b, resi.view, 0, 17, 96)
    resi.check()
    assert rt.sync_status() == 0


def test_dist_batch_generic_stay_in_bounds(rt):
    n, off = 30011, 3
    x = dev(inputs.f32_uniform01(n, 0))
    y = Guarded(n, np.float32, off, inputs.f32_uniform01(n, 1))
    for d, c in ((1024, 8), (128, 1), (1000, 0)):
        rt.launch_region_dist(R.loop_desc(R.BODY_AXPY, n=n, x=x, y=y.view), d,
                              R.SCHED_STATIC_CHUNKED if c else R.SCHED_STATIC, c, 7, 128)
        y.check()
    seg = dev(np.array([0, 100, 100, 5000, n], np.int64))
    res = Guarded(4, np.float64, 1)
    rt.launch_generic(seg, R.loop_desc(R.BODY_DOT, n=n, x=x, y=y.view), res.view, 3, 64)
    res.check()
    out = Guarded(n, np.float32, off)
    d1 = R.loop_desc(R.BODY_STENCIL1D3, n=n, x=x, out=out.view)
    d2 = R.loop_desc(R.BODY_AXPY, n=n, x=x, y=y.view)
    b = rt.batch_create([d1, d2], None, 256)
    b.launch(0, 128)
    b.destroy()
    out.check()
    y.check()
    assert rt.sync_status() == 0
