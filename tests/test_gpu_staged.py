"""GPU parity: the staged form of dynamic, static(c) and static schedules.

Chunks taken by a warp are moved through shared memory by bulk copies
(P chunks per pass); the owner of every iteration is unchanged.  Axpy results
must be bit-exact against the oracle with staging on (several pass sizes, from
32 chunks per pass down to one) and off; integer reductions exact; fp32 / bf16
sums within the reduction bound.  Cases cover ragged tails (a last chunk that is
not a whole 16-byte unit), team blocks that do not start on a 16-byte boundary
(those teams run the plain form inside the same launch), misaligned pointers
and chunks that are not a whole number of 16-byte units (plain form)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, fp_sum_ok, host

pytestmark = pytest.mark.gpu

DEFAULT_STAGE = 32768

# (chunk, threads): chunks per pass with the default 32 KiB for axpy (2 arrays)
CASES = [(256, 32),    # 16
         (64, 32),     # 32 (the whole claim in one pass)
         (64, 128),    # 16
         (128, 64),    # 16
         (68, 32),     # 30: a 272-byte chunk, not a power of two
         (256, 64),    # 8: plain form
         (8, 128),     # 32-byte chunks: plain form
         (6, 64),      # 24-byte chunks: plain form
         (1000, 32)]   # 4: plain form


@pytest.fixture
def staged(rt):
    yield rt
    rt.set_stage_bytes(DEFAULT_STAGE)


def _axpy(rt, n, G, T, chunk, x, y, alpha=3.0):
    xd, yd = dev(x), dev(y)
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=alpha), R.SCHED_DYNAMIC,
                     chunk, G, T)
    return host(yd)


@pytest.mark.parametrize("chunk,T", CASES)
@pytest.mark.parametrize("n", [0, 1, 5, 4099, 300007, (1 << 20) + 13])
def test_axpy_f32_staged_bit_exact(staged, chunk, T, n):
    rt = staged
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    want = bits32(O.axpy_f32(3.0, x, y))
    for G in (1, 7, 64):
        assert np.array_equal(bits32(_axpy(rt, n, G, T, chunk, x, y)), want), G
    for G in (1, 64):  # nonmonotonic dynamic takes the same staged path
        xd, yd = dev(x), dev(y)
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0),
                         R.SCHED_NONMONOTONIC, chunk, G, T)
        assert np.array_equal(bits32(host(yd)), want), ("nonmonotonic", G)
    rt.set_stage_bytes(0)  # plain form, same results
    assert np.array_equal(bits32(_axpy(rt, n, 7, T, chunk, x, y)), want)
    assert rt.sync_status() == 0


# static(c): warp w's k-th set of chunks is k*T + 32w + lane, one contiguous
# range; static without chunk is staged when n = G * T * c exactly.
@pytest.mark.parametrize("chunk,T", [(64, 32), (64, 128), (256, 32), (68, 64), (8, 512), (6, 64)])
@pytest.mark.parametrize("n", [1, 4099, 300007, (1 << 20) + 13])
def test_axpy_static_chunked_staged_bit_exact(staged, chunk, T, n):
    rt = staged
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    want = bits32(O.axpy_f32(3.0, x, y))
    for G in (1, 7, 64):
        xd, yd = dev(x), dev(y)
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0),
                         R.SCHED_STATIC_CHUNKED, chunk, G, T)
        assert np.array_equal(bits32(host(yd)), want), G
    assert rt.sync_status() == 0


@pytest.mark.parametrize("G,T,c", [(1, 32, 256), (16, 32, 64), (64, 128, 64), (8, 64, 128),
                                   (4, 256, 16), (2, 32, 68)])
def test_axpy_static_staged_bit_exact(staged, G, T, c):
    """n = G * T * c: every thread's block is one staged chunk; n + 4 and
    n - 4 (blocks of unequal size) run the plain form."""
    rt = staged
    for n in (G * T * c, G * T * c + 4, G * T * c - 4):
        x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
        xd, yd = dev(x), dev(y)
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), R.SCHED_STATIC, 0,
                         G, T)
        assert np.array_equal(bits32(host(yd)), bits32(O.axpy_f32(3.0, x, y))), n
        r = _res("i")
        xi, yi = inputs.int32_uniform(n, 3), inputs.int32_uniform(n, 4)
        yid = dev(yi)
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=dev(xi), y=yid, alpha=3), R.SCHED_STATIC,
                         0, G, T, red=R.ReduceDesc(R.OP_SUM, 0, r.data_ptr()))
        want = O.axpy_i32(3, xi, yi)
        assert np.array_equal(host(yid), want), n
        assert int(host(r)[0]) == O.sum_int(want), n
    assert rt.sync_status() == 0


@pytest.mark.parametrize("budget", [16, 2048, 16384, 32768, 65536, 131072])
def test_axpy_i32_staged_budgets(staged, budget):
    rt = staged
    rt.set_stage_bytes(budget)
    n = 200003
    x, y = inputs.int32_uniform(n, 3), inputs.int32_uniform(n, 4)
    want = O.axpy_i32(3, x, y)
    for chunk, T in ((64, 32), (256, 64), (8, 512), (256, 32), (64, 512)):
        xd, yd = dev(x), dev(y)
        r = _res("i")
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3), R.SCHED_DYNAMIC,
                         chunk, 19, T, red=R.ReduceDesc(R.OP_SUM, 0, r.data_ptr()))
        assert np.array_equal(host(yd), want), (chunk, T)
        assert int(host(r)[0]) == O.sum_int(want), (chunk, T)
    assert rt.sync_status() == 0


def test_misaligned_pointers_run_plain(staged):
    rt = staged
    n = 65537
    xb, yb = inputs.f32_uniform01(n + 8, 0), inputs.f32_uniform01(n + 8, 1)
    for ox, oy in ((1, 0), (0, 3), (2, 2)):
        xd, yd = dev(xb), dev(yb)
        x, y = xd[ox:ox + n], yd[oy:oy + n]
        x0, y0 = host(x).copy(), host(y).copy()
        rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=x, y=y, alpha=-0.5), R.SCHED_DYNAMIC,
                         256, 4, 32)
        assert np.array_equal(bits32(host(y)), bits32(O.axpy_f32(-0.5, x0, y0)))
        # elements outside the views are untouched
        yh = host(yd)
        assert np.array_equal(bits32(yh[:oy]), bits32(yb[:oy]))
        assert np.array_equal(bits32(yh[oy + n:]), bits32(yb[oy + n:]))


def _res(kind):
    import torch
    return torch.zeros(1, dtype=torch.float64 if kind == "f" else torch.int64, device="cuda")


# with a reduction: staged for P = 32 and at most 512 bytes of chunk over the
# arrays (dot c = 64 at T <= 64; sum c = 64 at T <= 128, c = 128 at T <= 64),
# plain otherwise
@pytest.mark.parametrize("chunk,T", [(64, 32), (64, 64), (64, 128), (128, 32), (256, 32),
                                     (1000, 64), (6, 64)])
@pytest.mark.parametrize("n", [1, 4099, (1 << 20) + 3])
def test_reductions_staged(staged, chunk, T, n):
    rt = staged
    import torch
    G = 11
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    r = _res("f")
    rt.launch_region(R.loop_desc(R.BODY_DOT, n=n, x=dev(x), y=dev(y)), R.SCHED_DYNAMIC, chunk,
                     G, T, red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
    exact = O.exact_dot_f32(x, y)
    assert fp_sum_ok(float(host(r)[0]), exact, exact)[0]
    a = inputs.f32_lognormal_signed(n, 2)
    rt.launch_region(R.loop_desc(R.BODY_NONE, n=n, x=dev(a), data_type=R.F32), R.SCHED_DYNAMIC,
                     chunk, G, T, red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
    ok, err, bound = fp_sum_ok(float(host(r)[0]), O.exact_sum_f32(a), O.exact_abs_sum_f32(a))
    assert ok, (err, bound)
    rt.launch_region(R.loop_desc(R.BODY_NONE, n=n, x=dev(a), data_type=R.F32), R.SCHED_DYNAMIC,
                     chunk, G, T, red=R.ReduceDesc(R.OP_MAX, 0, r.data_ptr()))
    assert host(r)[0] == O.max_min(a, "max")
    bits = inputs.bf16_uniform_pm1(n, 5)
    xb = dev(bits.view(np.int16)).view(torch.bfloat16)
    rt.launch_region(R.loop_desc(R.BODY_NONE, n=n, x=xb, data_type=R.BF16), R.SCHED_DYNAMIC,
                     chunk, G, T, red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
    vals = (bits.astype(np.uint32) << 16).view(np.float32)
    ok, err, bound = fp_sum_ok(float(host(r)[0]), O.exact_sum_bf16(bits),
                               O.exact_abs_sum_f32(vals))
    assert ok, (err, bound)
    ri = _res("i")
    for a in (inputs.int32_uniform(n, 3), inputs.int64_uniform(n, 4)):
        dt = R.I32 if a.dtype == np.int32 else R.I64
        rt.launch_region(R.loop_desc(R.BODY_NONE, n=n, x=dev(a), data_type=dt), R.SCHED_DYNAMIC,
                         chunk, G, T, red=R.ReduceDesc(R.OP_SUM, 0, ri.data_ptr()))
        assert int(host(ri)[0]) == O.sum_int(a)
    assert rt.sync_status() == 0


def test_full_size_axpy_staged(staged):
    """n = 2^26 at the launch shape of the dynamic(256) bench line family."""
    rt = staged
    n = 1 << 26
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    want = bits32(O.axpy_f32(3.0, x, y))
    for G, T in ((4096, 32), (2048, 64), (1024, 256)):
        assert np.array_equal(bits32(_axpy(rt, n, G, T, 256, x, y)), want), (G, T)
    assert rt.sync_status() == 0


def test_stage_bytes_validation(rt):
    with pytest.raises(R.OmprtError):
        rt.set_stage_bytes(-16)
    with pytest.raises(R.OmprtError):
        rt.set_stage_bytes(1 << 30)
    rt.set_stage_bytes(DEFAULT_STAGE)


# -- stencils: the pass's input window (one row / one element on each side)
# is staged with one bulk copy; outputs go back by one bulk store per pass.

STENCIL_SCHEDS = [(R.SCHED_DYNAMIC, 64), (R.SCHED_DYNAMIC, 256), (R.SCHED_STATIC_CHUNKED, 64),
                  (R.SCHED_STATIC_CHUNKED, 68), (R.SCHED_STATIC, 0)]


@pytest.mark.parametrize("sched,chunk", STENCIL_SCHEDS)
@pytest.mark.parametrize("ny,nx", [(64, 64), (67, 40), (4, 4), (9, 8), (130, 516), (33, 1028),
                                   (65, 42), (256, 256)])
@pytest.mark.parametrize("budget", [32768, 131072])
def test_stencil2d_staged_bit_exact(staged, sched, chunk, ny, nx, budget):
    """nx % 4 != 0 (42) runs the plain form."""
    import torch
    rt = staged
    rt.set_stage_bytes(budget)
    a = inputs.grid_f32(ny, nx, 6)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for G, T in ((1, 32), (3, 64), (16, 32), (64, 128)):
        out = torch.full((ny, nx), -7.0, device="cuda")
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                         sched, chunk, G, T)
        assert np.array_equal(bits32(host(out)), want), (G, T)
    assert rt.sync_status() == 0


@pytest.mark.parametrize("sched,chunk", STENCIL_SCHEDS)
@pytest.mark.parametrize("n", [4, 4096, 4100, 65536, 300000, 300001])
def test_stencil1d_staged_bit_exact(staged, sched, chunk, n):
    """n % 4 != 0 (300001) runs the plain form."""
    import torch
    rt = staged
    a = inputs.f32_uniform01(n, 4)
    ad = dev(a)
    want = bits32(O.stencil1d3(a))
    for G, T in ((1, 32), (7, 64), (64, 32)):
        out = torch.full((n,), -7.0, device="cuda")
        rt.launch_region(R.loop_desc(R.BODY_STENCIL1D3, n=n, x=ad, out=out), sched, chunk, G, T)
        assert np.array_equal(bits32(host(out)), want), (G, T)
    assert rt.sync_status() == 0


def test_stencil2d_staged_full_grid(staged):
    """The 4096 x 4096 grid of the worksharing sweep under large budgets: a
    pass would need two 16 KB halo rows, more than a quarter of the pass, so
    the host runs the plain form; results must not depend on the budget."""
    import torch
    rt = staged
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for budget in (65536, 196608):
        rt.set_stage_bytes(budget)
        for sched, chunk, G, T in ((R.SCHED_DYNAMIC, 256, 4096, 32), (R.SCHED_STATIC_CHUNKED, 64,
                                   2048, 64), (R.SCHED_STATIC, 0, 4096, 32)):
            out = torch.empty_like(ad)
            rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                         ny=4096), sched, chunk, G, T)
            assert np.array_equal(bits32(host(out)), want), (budget, sched, G, T)
    assert rt.sync_status() == 0


def test_staged_and_tiled_forms_in_a_cuda_graph(staged):
    """Staged dynamic / static launches, a staged 1-D stencil, the
    tensor-tiled 2-D stencil (its tensor map is a kernel parameter) and the
    static(64) row ring on 4096-wide rows (96 KB of shared memory, opted in
    at launch) captured in one CUDA graph: every replay reproduces the eager
    results bit for bit."""
    import torch
    rt = staged
    n = (1 << 20) + 12
    x = inputs.f32_uniform01(n, 0)
    y0 = inputs.f32_uniform01(n, 1)
    xd, yd = dev(x), dev(y0)
    a1 = inputs.f32_uniform01(1 << 20, 4)
    a1d = dev(a1)
    o1 = torch.empty_like(a1d)
    g2 = inputs.grid_f32(1000, 1028, 6)
    g2d = dev(g2)
    o2 = torch.empty_like(g2d)
    g3 = inputs.grid_f32(41, 4096, 7)
    g3d = dev(g3)
    o3 = torch.empty_like(g3d)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        d = R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0)
        rt.launch_region(d, R.SCHED_DYNAMIC, 256, 64, 32, stream=s)
        rt.launch_region(d, R.SCHED_STATIC_CHUNKED, 64, 16, 128, stream=s)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL1D3, n=1 << 20, x=a1d, out=o1),
                         R.SCHED_DYNAMIC, 64, 64, 32, stream=s)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=1000 * 1028, x=g2d, out=o2, nx=1028,
                                     ny=1000), R.SCHED_AUTO, 0, 152, 256, stream=s)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=41 * 4096, x=g3d, out=o3, nx=4096,
                                     ny=41), R.SCHED_STATIC_CHUNKED, 64, 9, 256, stream=s)
    want_y = O.axpy_f32(3.0, x, O.axpy_f32(3.0, x, y0))
    for _ in range(3):
        yd.copy_(dev(y0))
        o1.fill_(-7.0)
        o2.fill_(-7.0)
        o3.fill_(-7.0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(bits32(host(yd)), bits32(want_y))
        assert np.array_equal(bits32(host(o1)), bits32(O.stencil1d3(a1)))
        assert np.array_equal(bits32(host(o2)), bits32(O.stencil2d5(g2)))
        assert np.array_equal(bits32(host(o3)), bits32(O.stencil2d5(g3)))
    assert rt.sync_status() == 0


# -- static(c) 2-D stencil (c in [4, 8) and [32, 128]): the team walks its
# block in passes of rows staged through a ring in shared memory; every thread
# computes exactly its chunks, in 16-byte units where its piece allows.  The
# other chunk sizes (and static without chunk) take the plain form.

@pytest.mark.parametrize("ny,nx", [(1, 4), (2, 8), (9, 8), (33, 132), (67, 40), (100, 64),
                                   (5, 16), (300, 1028)])
@pytest.mark.parametrize("sched,chunk", [(R.SCHED_STATIC, 0), (R.SCHED_STATIC_CHUNKED, 1),
                                         (R.SCHED_STATIC_CHUNKED, 4), (R.SCHED_STATIC_CHUNKED, 5),
                                         (R.SCHED_STATIC_CHUNKED, 8),
                                         (R.SCHED_STATIC_CHUNKED, 33),
                                         (R.SCHED_STATIC_CHUNKED, 64),
                                         (R.SCHED_STATIC_CHUNKED, 128),
                                         (R.SCHED_STATIC_CHUNKED, 300)])
def test_stencil2d_row_ring_bit_exact(staged, ny, nx, sched, chunk):
    import torch
    rt = staged
    a = inputs.grid_f32(ny, nx, 6)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for G, T in ((1, 32), (3, 64), (7, 96), (64, 256), (500, 32), (13, 1024), (5, 480)):
        out = torch.full((ny, nx), -7.0, device="cuda")
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                         sched, chunk, G, T)
        assert np.array_equal(bits32(host(out)), want), (G, T)
    assert rt.sync_status() == 0


def test_stencil2d_row_ring_full_grid_and_off(staged):
    """4096^2 at bench-like shapes, with the row ring and with staging off."""
    import torch
    rt = staged
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for budget in (32768, 0):
        rt.set_stage_bytes(budget)
        for sched, chunk, G, T in ((R.SCHED_STATIC, 0, 8192, 128), (R.SCHED_STATIC_CHUNKED, 8,
                                   1024, 1024), (R.SCHED_STATIC_CHUNKED, 64, 4096, 128),
                                   (R.SCHED_STATIC_CHUNKED, 64, 2048, 128),
                                   (R.SCHED_STATIC_CHUNKED, 4, 152, 1024),
                                   (R.SCHED_STATIC_CHUNKED, 128, 456, 512)):
            out = torch.empty_like(ad)
            rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                         ny=4096), sched, chunk, G, T)
            assert np.array_equal(bits32(host(out)), want), (budget, sched, chunk, G, T)
    assert rt.sync_status() == 0
