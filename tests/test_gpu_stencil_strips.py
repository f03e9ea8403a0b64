"""GPU parity: static schedules of the 2-D stencil run as vertical strips
(k_stencil_strips.cu).

When every team's block is whole rows and the schedule's period divides nx,
each thread owns the same columns in every row (static(1) with T | nx,
static(4) / static(8) with cT | nx, static with one row per team and
nx / T in {1, 4, 8}) and walks them down the rows.  Results must be
bit-exact against the oracle, including grids of one to a few rows, teams
that cover one and several rows, all the column-per-thread counts, and
launches that do not have that form (they fall back to the other forms)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu

# (sched, chunk, T) with nx = T * M (static(1)), c T M (static(c)), or T p (static)
CASES = [(R.SCHED_STATIC_CHUNKED, 1, 32), (R.SCHED_STATIC_CHUNKED, 1, 64),
         (R.SCHED_STATIC_CHUNKED, 1, 128), (R.SCHED_STATIC_CHUNKED, 1, 256),
         (R.SCHED_STATIC_CHUNKED, 4, 32), (R.SCHED_STATIC_CHUNKED, 4, 64),
         (R.SCHED_STATIC_CHUNKED, 8, 32), (R.SCHED_STATIC_CHUNKED, 8, 64),
         (R.SCHED_STATIC, 0, 32), (R.SCHED_STATIC, 0, 64), (R.SCHED_STATIC, 0, 128),
         (R.SCHED_STATIC, 0, 256)]


@pytest.mark.parametrize("nx", [256, 512, 1024])
@pytest.mark.parametrize("ny", [1, 2, 3, 17, 64, 100])
def test_strips_bit_exact(rt, nx, ny):
    import torch
    a = inputs.grid_f32(ny, nx, 12)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for sched, chunk, T in CASES:
        for G in sorted({1, ny, max(1, ny // 2), 3, 7, 64}):
            out = torch.full((ny, nx), -7.0, device="cuda")
            rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx,
                                         ny=ny), sched, chunk, G, T)
            assert np.array_equal(bits32(host(out)), want), (sched, chunk, G, T)
    assert rt.sync_status() == 0


def test_strips_full_grid(rt):
    """4096^2 at the shapes the tuner may pick for static(1), static(8) and
    static."""
    import torch
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for sched, chunk, G, T in ((R.SCHED_STATIC_CHUNKED, 1, 4096, 512),
                               (R.SCHED_STATIC_CHUNKED, 1, 1024, 1024),
                               (R.SCHED_STATIC_CHUNKED, 1, 2048, 512),
                               (R.SCHED_STATIC_CHUNKED, 8, 4096, 512),
                               (R.SCHED_STATIC_CHUNKED, 8, 1024, 512),
                               (R.SCHED_STATIC_CHUNKED, 4, 2048, 1024),
                               (R.SCHED_STATIC, 0, 4096, 512), (R.SCHED_STATIC, 0, 4096, 1024)):
        out = torch.empty_like(ad)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                     ny=4096), sched, chunk, G, T)
        assert np.array_equal(bits32(host(out)), want), (sched, chunk, G, T)
    assert rt.sync_status() == 0


def test_strips_misaligned_views_fall_back(rt):
    """A view 4 bytes into its allocation cannot take the 32-byte strip
    vectors; the launch runs another form, bit-exact, and leaves the floats
    around the view untouched."""
    import torch
    ny, nx = 40, 512
    a = inputs.grid_f32(ny, nx, 13)
    buf = torch.zeros(ny * nx + 16, device="cuda")
    buf[1:1 + ny * nx] = torch.from_numpy(a.ravel()).cuda()
    obuf = torch.full((ny * nx + 16,), -3.0, device="cuda")
    x, out = buf[1:1 + ny * nx], obuf[1:1 + ny * nx]
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=x, out=out, nx=nx, ny=ny),
                     R.SCHED_STATIC_CHUNKED, 8, 40, 64)
    got = host(obuf)
    assert np.array_equal(bits32(got[1:1 + ny * nx]), bits32(O.stencil2d5(a).ravel()))
    assert got[0] == -3.0 and np.all(got[1 + ny * nx:] == -3.0)
    assert rt.sync_status() == 0
