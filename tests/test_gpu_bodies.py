"""GPU parity: loop bodies under every schedule, bit-exact against the oracle
(including misaligned pointers, ragged sizes and degenerate grids)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu

SCHEDS = [(R.SCHED_STATIC, 0), (R.SCHED_STATIC_CHUNKED, 1), (R.SCHED_STATIC_CHUNKED, 5),
          (R.SCHED_STATIC_CHUNKED, 8), (R.SCHED_STATIC_CHUNKED, 64), (R.SCHED_DYNAMIC, 7),
          (R.SCHED_DYNAMIC, 256), (R.SCHED_AUTO, 0)]
SHAPES = [(148, 256), (13, 96), (1184, 1024), (1, 32)]


@pytest.mark.parametrize("sched,chunk", SCHEDS)
@pytest.mark.parametrize("G,T", SHAPES)
def test_axpy_f32_bit_exact(rt, sched, chunk, G, T):
    n = (1 << 20) + 13
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    xd, yd = dev(x), dev(y)
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), sched, chunk, G, T)
    assert np.array_equal(bits32(host(yd)), bits32(O.axpy_f32(3.0, x, y)))


@pytest.mark.parametrize("sched,chunk", SCHEDS)
def test_axpy_f32_misaligned_and_ragged(rt, sched, chunk):
    import torch
    for n, off in ((0, 0), (1, 1), (7, 3), (1000, 1), (65543, 5)):
        yb0 = inputs.f32_uniform01(n + 8, 3)
        xb = dev(inputs.f32_uniform01(n + 8, 2))
        yb = dev(yb0)
        x, y = xb[off:off + n], yb[1:1 + n]       # different misalignments
        x0, y0 = host(x).copy(), host(y).copy()
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=x, y=y, alpha=-1.25), sched, chunk,
                         7, 64)
        assert np.array_equal(bits32(host(y)), bits32(O.axpy_f32(-1.25, x0, y0)))
        after = host(yb)
        assert after[0] == yb0[0] and np.array_equal(after[1 + n:], yb0[1 + n:])  # no stray writes


@pytest.mark.parametrize("sched,chunk", SCHEDS)
def test_axpy_i32_with_int64_sum(rt, sched, chunk):
    import torch
    n = (1 << 20) + 3
    x, y = inputs.int32_uniform(n, 0), inputs.int32_uniform(n, 1)
    x[:3] = [2 ** 31 - 1, -2 ** 31, 12345]          # wrap-around cases
    xd, yd = dev(x), dev(y)
    res = torch.zeros(1, dtype=torch.int64, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3),
                     sched, chunk, 37, 128, red=R.ReduceDesc(R.OP_SUM, 0, res.data_ptr()))
    ynew = O.axpy_i32(3, x, y)
    assert np.array_equal(host(yd), ynew)
    assert int(host(res)[0]) == O.sum_int(ynew)
    assert rt.sync_status() == 0


def test_single_region_config(rt):
    """teams distribute parallel for schedule(static), n = 2^20, int32 x, y
    uniform in [-2^20, 2^20) (seeds 0, 1), y = 3x + y, reduction(+) into
    int64; 4 teams x 128 threads."""
    import torch
    n = 1 << 20
    x, y = inputs.int32_uniform(n, 0), inputs.int32_uniform(n, 1)
    xd, yd = dev(x), dev(y)
    res = torch.zeros(1, dtype=torch.int64, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3), R.SCHED_STATIC, 0, 4,
                     128, red=R.ReduceDesc(R.OP_SUM, 0, res.data_ptr()))
    ynew = O.axpy_i32(3, x, y)
    assert np.array_equal(host(yd), ynew)
    assert int(host(res)[0]) == O.sum_int(ynew)


@pytest.mark.parametrize("sched,chunk", SCHEDS)
@pytest.mark.parametrize("n", [1, 2, 3, 9, 17, 1000, (1 << 18) + 5])
def test_stencil1d_bit_exact(rt, sched, chunk, n):
    import torch
    a = inputs.f32_uniform01(n, 4)
    ad = dev(a)
    out = torch.full((n,), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL1D3, n=n, x=ad, out=out), sched, chunk, 11, 64)
    assert np.array_equal(bits32(host(out)), bits32(O.stencil1d3(a)))


@pytest.mark.parametrize("sched,chunk", SCHEDS)
@pytest.mark.parametrize("ny,nx", [(1, 1), (1, 9), (9, 1), (2, 2), (3, 5), (64, 64),
                                   (129, 257), (67, 40), (1024, 1024), (5, 16), (9, 8), (2, 8),
                                   (1, 8), (17, 24)])
def test_stencil2d_bit_exact(rt, sched, chunk, ny, nx):
    import torch
    a = inputs.grid_f32(ny, nx, 6)
    ad = dev(a)
    out = torch.full((ny, nx), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                     sched, chunk, 23, 128)
    assert np.array_equal(bits32(host(out)), bits32(O.stencil2d5(a)))


def test_stencil2d_full_grid(rt):
    """The 4096 x 4096 fp32 grid of the worksharing sweep, static schedule."""
    import torch
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    out = torch.empty_like(ad)
    for sched, chunk in ((R.SCHED_STATIC, 0), (R.SCHED_AUTO, 0), (R.SCHED_DYNAMIC, 256)):
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                     ny=4096), sched, chunk, 592, 256)
        assert np.array_equal(bits32(host(out)), bits32(O.stencil2d5(a)))


def test_axpy_full_size_static(rt):
    """n = 2^26 fp32 axpy, the worksharing sweep's size, at one sweep point."""
    n = 1 << 26
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    xd, yd = dev(x), dev(y)
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), R.SCHED_STATIC, 0,
                     592, 256)
    assert np.array_equal(bits32(host(yd)), bits32(O.axpy_f32(3.0, x, y)))


@pytest.mark.parametrize("ny,nx", [(1, 4), (2, 8), (4, 4), (9, 8), (33, 132), (100, 260),
                                   (67, 40), (31, 4), (1024, 1024)])
@pytest.mark.parametrize("G,T", [(1, 32), (5, 64), (37, 96), (152, 128), (4096, 256),
                                 (64, 1024)])
def test_stencil2d_auto_tiles_bit_exact(rt, ny, nx, G, T):
    """schedule(auto) runs the 2-D stencil on tensor-copied tiles of 128 x 32
    when nx % 4 == 0: bit-exact at ragged tile edges, for 1, 2, 4 and 8 warps
    per team and more teams than tiles."""
    import torch
    a = inputs.grid_f32(ny, nx, 6)
    ad = dev(a)
    out = torch.full((ny, nx), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                     R.SCHED_AUTO, 0, G, T)
    assert np.array_equal(bits32(host(out)), bits32(O.stencil2d5(a)))
    assert rt.sync_status() == 0


def test_stencil2d_auto_fallbacks(rt):
    """Misaligned output, nx % 4 != 0 and a reduction run the strip-walking
    form; all bit-exact (the reduction within the sum bound)."""
    import torch
    from gpu_helpers import fp_sum_ok
    ny, nx = 70, 136
    a = inputs.grid_f32(ny, nx, 6)
    ad = dev(a)
    want = O.stencil2d5(a)
    buf = torch.full((ny * nx + 1,), -7.0, device="cuda")
    out = buf[1:]  # 4-byte aligned only
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                     R.SCHED_AUTO, 0, 17, 128)
    assert np.array_equal(bits32(host(out)), bits32(want.reshape(-1)))
    b = inputs.grid_f32(9, 10, 7)
    outb = torch.full((9, 10), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=90, x=dev(b), out=outb, nx=10, ny=9),
                     R.SCHED_AUTO, 0, 3, 64)
    assert np.array_equal(bits32(host(outb)), bits32(O.stencil2d5(b)))
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    out2 = torch.full((ny, nx), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out2, nx=nx, ny=ny),
                     R.SCHED_AUTO, 0, 17, 128,
                     red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, res.data_ptr()))
    assert np.array_equal(bits32(host(out2)), bits32(want))
    ok, err, bound = fp_sum_ok(float(host(res)[0]), O.exact_sum_f32(want.reshape(-1)),
                               O.exact_abs_sum_f32(want.reshape(-1)))
    assert ok, (err, bound)
    assert rt.sync_status() == 0


@pytest.mark.parametrize("chunk,G,T", [(1, 7, 64), (7, 148, 256), (256, 64, 32), (64, 13, 1024)])
def test_nonmonotonic_bodies_bit_exact(rt, chunk, G, T):
    """axpy and both stencils under schedule(nonmonotonic: dynamic, c)."""
    import torch
    n = (1 << 20) + 13
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    xd, yd = dev(x), dev(y)
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), R.SCHED_NONMONOTONIC,
                     chunk, G, T)
    assert np.array_equal(bits32(host(yd)), bits32(O.axpy_f32(3.0, x, y)))
    out = torch.full((n,), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL1D3, n=n, x=xd, out=out), R.SCHED_NONMONOTONIC,
                     chunk, G, T)
    assert np.array_equal(bits32(host(out)), bits32(O.stencil1d3(x)))
    a = inputs.grid_f32(129, 256, 6)
    out2 = torch.full((129, 256), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=129 * 256, x=dev(a), out=out2, nx=256,
                                 ny=129), R.SCHED_NONMONOTONIC, chunk, G, T)
    assert np.array_equal(bits32(host(out2)), bits32(O.stencil2d5(a)))
    assert rt.sync_status() == 0
