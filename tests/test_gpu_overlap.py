"""GPU parity: regions launched back to back on one stream, with launch
overlap on (the default: each kernel may be scheduled while the one before it
drains, and waits for it before touching memory) and off (plain launches).

Every launch of a chain reads what the launch before it wrote and overwrites
what that launch read, so a grid that touched memory before the grid ahead of
it had finished would change a result.  The chains cross the 2-D stencil's
forms (tensor tiles, bands, strips, slabs, the column ring, the row rings,
the plain region kernel), dynamic and guided counters, the int32 axpy with
and without its int64 sum, a library kernel in between and the reductions.
Results must equal the oracle applied in the same order: bit-exact, the
integer sums exactly, the fp32 sum within the reduction tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, fp_sum_ok, host

pytestmark = pytest.mark.gpu

ST, CH, DY, AU, GU = (R.SCHED_STATIC, R.SCHED_STATIC_CHUNKED, R.SCHED_DYNAMIC, R.SCHED_AUTO,
                      R.SCHED_GUIDED)

# the worksharing step's six schedules, with the (teams, threads) of the
# committed tuning table (4 teams a SM x 256 threads where it has none)
SCHED6 = [("static1", CH, 1), ("static8", CH, 8), ("static64", CH, 64), ("static", ST, 0),
          ("dynamic256", DY, 256), ("auto", AU, 0)]


def step_shape(body, label):
    from paper_2106_03219_gb300 import autotune
    table = autotune.load_sweep_table() or {}
    return tuple(table.get("%s/%s" % (body, label), (4 * 152, 256)))


# (sched, chunk, teams, threads) on the 4096 x 4096 grid: the step's six
# schedules, then forms the step does not use
STENCIL_CHAIN = [(sched, chunk) + step_shape("stencil2d", label)
                 for label, sched, chunk in SCHED6] + [
    (DY, 64, 1024, 128), (CH, 4, 512, 256), (CH, 3, 1000, 96), (GU, 16, 300, 128),
    (DY, 256, 4096, 256), (CH, 32, 2048, 128), (AU, 0, 152, 256), (ST, 0, 333, 160),
]


@pytest.fixture
def overlap_modes(rt):
    yield rt
    rt.set_launch_overlap(True)


@pytest.mark.parametrize("overlap", [True, False])
def test_stencil_chain_back_to_back(overlap_modes, overlap):
    import torch
    rt = overlap_modes
    rt.set_launch_overlap(overlap)
    ny = nx = 4096
    a = inputs.grid_f32(ny, nx, 61)
    bufs = [dev(a), torch.full((ny, nx), -5.0, device="cuda")]
    want = a
    torch.cuda.synchronize()
    for k, (sched, chunk, G, T) in enumerate(STENCIL_CHAIN):
        src, dst = bufs[k % 2], bufs[(k + 1) % 2]
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=src, out=dst, nx=nx, ny=ny),
                         sched, chunk, G, T)
        want = O.stencil2d5(want)
        if k == 6:
            dst.neg_()              # a library kernel between two regions
            want = -want
    K = len(STENCIL_CHAIN)
    assert np.array_equal(bits32(host(bufs[K % 2])), bits32(want))
    # one more region, then a reduction right behind it over what it wrote
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=bufs[K % 2],
                                 out=bufs[(K + 1) % 2], nx=nx, ny=ny), AU, 0, 1216, 1024)
    want = O.stencil2d5(want)
    rt.reduce(R.OP_SUM, bufs[(K + 1) % 2], res, R.PREC_COMP_F64)
    ok, err, bound = fp_sum_ok(float(host(res)[0]), O.exact_sum_f32(want),
                               O.exact_abs_sum_f32(want))
    assert ok, (err, bound)
    assert rt.sync_status() == 0


@pytest.mark.parametrize("overlap", [True, False])
def test_axpy_chain_with_sums(overlap_modes, overlap):
    """x and y swap roles every launch (y = 3x + y, then x = 3y + x, ...),
    some launches carrying an int64 sum of what they wrote; dynamic and
    guided launches reuse the context's counters one after another."""
    import torch
    rt = overlap_modes
    rt.set_launch_overlap(overlap)
    n = (1 << 24) + 7
    v = [inputs.int32_uniform(n, 62), inputs.int32_uniform(n, 63)]
    d = [dev(v[0]), dev(v[1])]
    chain = [(DY, 256, 8192, 32), (DY, 256, 8192, 32), (ST, 0, 16384, 256), (GU, 64, 700, 128),
             (CH, 1, 4096, 512), (DY, 1024, 300, 1024), (AU, 0, 0, 0), (CH, 8, 8192, 256)]
    sums = []
    for k, (sched, chunk, G, T) in enumerate(chain):
        src, dst = k % 2, (k + 1) % 2
        red = None
        if k % 3 == 1:
            res = torch.zeros(1, dtype=torch.int64, device="cuda")
            red = R.ReduceDesc(R.OP_SUM, 0, res.data_ptr())
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=d[src], y=d[dst], alpha=3), sched, chunk,
                         G, T, red=red)
        v[dst] = O.axpy_i32(3, v[src], v[dst])
        if red is not None:
            sums.append((res, O.sum_int(v[dst])))
    r64 = torch.zeros(1, dtype=torch.int64, device="cuda")
    rt.reduce(R.OP_SUM, d[len(chain) % 2], r64)
    assert np.array_equal(host(d[0]), v[0]) and np.array_equal(host(d[1]), v[1])
    for res, want in sums:
        assert int(host(res)[0]) == want
    assert int(host(r64)[0]) == O.sum_int(v[len(chain) % 2])
    assert rt.sync_status() == 0


def test_overlap_modes_agree_on_the_step(overlap_modes):
    """The worksharing step's twelve launches (axpy and stencil, six
    schedules) as one back-to-back sequence: the same bits with overlap on
    and off."""
    import torch
    rt = overlap_modes
    n = 1 << 26
    x = inputs.f32_uniform01(n, 0)
    y0 = inputs.f32_uniform01(n, 1)
    g = inputs.grid_f32(4096, 4096, 0)
    outs = []
    for on in (True, False):
        rt.set_launch_overlap(on)
        xd, yd, gd = dev(x), dev(y0), dev(g)
        od = torch.empty_like(gd)
        torch.cuda.synchronize()
        for i, (label, sched, chunk) in enumerate(SCHED6):
            G, T = step_shape("axpy", label)
            rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), sched, chunk,
                             G, T)
            G, T = step_shape("stencil2d", label)
            src, dst = (gd, od) if i % 2 == 0 else (od, gd)
            rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=src, out=dst,
                                         nx=4096, ny=4096), sched, chunk, G, T)
        outs.append((bits32(host(yd)), bits32(host(gd))))
        del xd, yd, gd, od
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    want, want_y = g, y0
    for _ in SCHED6:
        want = O.stencil2d5(want)
        want_y = O.axpy_f32(3.0, x, want_y)
    assert np.array_equal(outs[0][1], bits32(want))
    assert np.array_equal(outs[0][0], bits32(want_y))
    assert rt.sync_status() == 0
