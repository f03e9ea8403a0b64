"""GPU parity: dynamic(c) 2-D stencil with team blocks of whole rows,
streamed through a ring of row slots (k_stencil_rowring.cu), and static(c)
on the same shapes (the slab, strip and row-pass forms).

The ring applies when G divides ny and c and nx are multiples of 4 (and the
slab form does not).  Results must be bit-exact against the oracle for
grids of one to a few rows, rows that are not whole 128-byte lines, chunks
that cross row ends or cover the whole block, rings that hold only one
team's rows (one group per CTA) and the full ring, and launches outside the
form (they fall back to the other forms)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu

STATIC = R.SCHED_STATIC_CHUNKED
DYN = R.SCHED_DYNAMIC
SCHEDS = [(STATIC, 1), (STATIC, 4), (STATIC, 8), (STATIC, 12), (STATIC, 64), (STATIC, 256),
          (STATIC, 1 << 20), (DYN, 4), (DYN, 8), (DYN, 12), (DYN, 64), (DYN, 256),
          (DYN, 1 << 20)]


def _run(rt, ad, ny, nx, sched, chunk, G, T):
    import torch
    out = torch.full((ny, nx), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                     sched, chunk, G, T)
    return bits32(host(out))


@pytest.mark.parametrize("nx", [4, 36, 100, 256, 1024])
@pytest.mark.parametrize("ny", [1, 2, 3, 12, 64])
def test_rowring_bit_exact(rt, nx, ny):
    a = inputs.grid_f32(ny, nx, 21)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    teams = sorted({g for g in (1, 2, 3, 4, 6, ny // 2, ny) if g >= 1 and ny % g == 0})
    for sched, chunk in SCHEDS:
        for G in teams:
            for T in (32, 64, 160, 512):
                got = _run(rt, ad, ny, nx, sched, chunk, G, T)
                assert np.array_equal(got, want), (sched, chunk, G, T)
    assert rt.sync_status() == 0


@pytest.mark.parametrize("budget", [4 * 4096 * 4 + 256, 8 * 4096 * 4 + 256, 226 * 1024])
def test_rowring_ring_sizes(rt, budget):
    """A ring of 4 rows (R + 3 with one-row blocks: one group a CTA), of 8
    rows, and the default; 4096-wide rows, 96 and 256 rows."""
    rt.set_stencil_stage_bytes(budget)
    try:
        for ny in (96, 256):
            a = inputs.grid_f32(ny, 4096, 22)
            ad = dev(a)
            want = bits32(O.stencil2d5(a))
            for sched, chunk in ((STATIC, 1), (STATIC, 64), (DYN, 256), (DYN, 64)):
                for G, T in ((ny, 32), (ny, 64), (ny, 256), (ny // 2, 32), (ny // 4, 128)):
                    got = _run(rt, ad, ny, 4096, sched, chunk, G, T)
                    assert np.array_equal(got, want), (budget, ny, sched, chunk, G, T)
    finally:
        rt.set_stencil_stage_bytes(226 * 1024)
    assert rt.sync_status() == 0


def test_rowring_full_grid(rt):
    """4096^2 at the shapes the tuner may pick."""
    import torch
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for sched, chunk, G, T in ((DYN, 256, 4096, 32), (DYN, 256, 2048, 32), (DYN, 256, 4096, 64),
                               (STATIC, 64, 4096, 64), (STATIC, 64, 4096, 32),
                               (STATIC, 64, 2048, 64), (STATIC, 1, 4096, 256),
                               (STATIC, 1, 4096, 128), (STATIC, 8, 4096, 128),
                               (STATIC, 4, 4096, 256)):
        out = torch.empty_like(ad)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                     ny=4096), sched, chunk, G, T)
        assert np.array_equal(bits32(host(out)), want), (sched, chunk, G, T)
    assert rt.sync_status() == 0


def test_rowring_outside_the_form_falls_back(rt):
    """Teams not dividing ny, c = 2, dynamic(1), nx not a multiple of 4 and
    teams of 1024 threads take other forms, bit-exact."""
    for ny, nx, sched, chunk, G, T in ((30, 256, STATIC, 64, 7, 64), (30, 256, STATIC, 2, 6, 64),
                                       (30, 256, DYN, 1, 6, 64), (20, 102, DYN, 4, 5, 32),
                                       (20, 102, STATIC, 1, 4, 32), (16, 2048, DYN, 64, 4, 1024)):
        a = inputs.grid_f32(ny, nx, 23)
        got = _run(rt, dev(a), ny, nx, sched, chunk, G, T)
        assert np.array_equal(got, bits32(O.stencil2d5(a))), (ny, nx, sched, chunk, G, T)
    assert rt.sync_status() == 0


def test_rowring_misaligned_views_fall_back(rt):
    """A view 4 bytes into its allocation cannot take bulk copies; the launch
    runs another form, bit-exact, and leaves the floats around the view
    untouched."""
    import torch
    ny, nx = 40, 512
    a = inputs.grid_f32(ny, nx, 24)
    buf = torch.zeros(ny * nx + 16, device="cuda")
    buf[1:1 + ny * nx] = torch.from_numpy(a.ravel()).cuda()
    obuf = torch.full((ny * nx + 16,), -3.0, device="cuda")
    x, out = buf[1:1 + ny * nx], obuf[1:1 + ny * nx]
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=x, out=out, nx=nx, ny=ny),
                     DYN, 64, 40, 64)
    got = host(obuf)
    assert np.array_equal(bits32(got[1:1 + ny * nx].reshape(ny, nx)),
                          bits32(O.stencil2d5(a)))
    assert got[0] == -3.0 and (got[1 + ny * nx:] == -3.0).all()
    assert rt.sync_status() == 0
