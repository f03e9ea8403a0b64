"""GPU parity: static(c) and dynamic(c) 2-D stencil whose warps take their
chunks slab by slab from swizzled tensor copies (k_stencil_slabs.cu).

The form applies when c is a multiple of the slab line (16 or 32 floats)
dividing nx, G divides ny and m = nx / c is a multiple or a divisor of 32.
Results must be bit-exact
against the oracle for one-row to many-row blocks, chunks of one to many
slabs, a warp's 32 chunks spanning one row, part of a row, or several rows,
blocks with fewer than 32 chunks (lanes without a chunk), and launches
outside the form (they fall back to the other forms)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu

STATIC = R.SCHED_STATIC_CHUNKED
DYN = R.SCHED_DYNAMIC


def _run(rt, ad, ny, nx, sched, chunk, G, T):
    import torch
    out = torch.full((ny, nx), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                     sched, chunk, G, T)
    return bits32(host(out))


SHAPES = [(16, 2), (16, 3), (16, 4), (32, 2), (32, 3), (32, 4)]


@pytest.mark.parametrize("nx", [32, 128, 1024, 2048])
@pytest.mark.parametrize("ny", [1, 2, 3, 8, 33])
def test_slabs_bit_exact(rt, nx, ny):
    """Every slab shape (floats a line, buffers a warp)."""
    a = inputs.grid_f32(ny, nx, 31)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    chunks = [c for c in (16, 32, 64, 96, 256, 1024, 2048) if nx % c == 0 and
              ((nx // c) % 32 == 0 or 32 % (nx // c) == 0)]
    teams = sorted({g for g in (1, 3, ny // 2, ny) if g >= 1 and ny % g == 0})
    try:
        for X, NB in SHAPES:
            rt.set_stencil_slab_shape(X, NB)
            for sched in (STATIC, DYN):
                for c in chunks:
                    for G in teams:
                        for T in (32, 64, 96, 512):
                            got = _run(rt, ad, ny, nx, sched, c, G, T)
                            assert np.array_equal(got, want), (X, NB, sched, c, G, T)
    finally:
        rt.set_stencil_slab_shape(0, 0)
    assert rt.sync_status() == 0


@pytest.mark.parametrize("X,NB", SHAPES)
def test_slabs_full_grid(rt, X, NB):
    """4096^2 at the shapes the tuner may pick."""
    import torch
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    rt.set_stencil_slab_shape(X, NB)
    for sched, chunk, G, T in ((DYN, 256, 4096, 32), (DYN, 256, 2048, 32), (DYN, 256, 1024, 64),
                               (DYN, 64, 4096, 64), (STATIC, 64, 4096, 64),
                               (STATIC, 64, 4096, 32), (STATIC, 64, 2048, 128),
                               (STATIC, 64, 1024, 256), (STATIC, 32, 4096, 128),
                               (STATIC, 4096, 4096, 32)):
        out = torch.empty_like(ad)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                     ny=4096), sched, chunk, G, T)
        assert np.array_equal(bits32(host(out)), want), (sched, chunk, G, T)
    rt.set_stencil_slab_shape(0, 0)
    assert rt.sync_status() == 0


def test_slab_shape_arguments(rt):
    for X, NB in ((8, 2), (64, 2), (16, 1), (32, 5), (-1, 0)):
        with pytest.raises(R.OmprtError):
            rt.set_stencil_slab_shape(X, NB)
    rt.set_stencil_slab_shape(0, 0)


def test_slabs_outside_the_form_falls_back(rt):
    """c = 40 (not a multiple of 16), m = 3 / 24 (neither a divisor nor a
    multiple of 32), teams not dividing ny, teams of 1024 threads: other
    forms, bit-exact."""
    for ny, nx, sched, chunk, G, T in ((12, 160, STATIC, 40, 6, 64), (12, 96, DYN, 32, 4, 32),
                                       (12, 768, STATIC, 32, 12, 64), (30, 256, DYN, 64, 7, 64),
                                       (16, 2048, STATIC, 64, 4, 1024)):
        a = inputs.grid_f32(ny, nx, 32)
        got = _run(rt, dev(a), ny, nx, sched, chunk, G, T)
        assert np.array_equal(got, bits32(O.stencil2d5(a))), (ny, nx, sched, chunk, G, T)
    assert rt.sync_status() == 0


def test_slabs_misaligned_views_fall_back(rt):
    """A view 4 bytes into its allocation cannot be a tensor copy's source;
    the launch runs another form, bit-exact, and leaves the floats around the
    view untouched."""
    import torch
    ny, nx = 40, 512
    a = inputs.grid_f32(ny, nx, 33)
    buf = torch.zeros(ny * nx + 16, device="cuda")
    buf[1:1 + ny * nx] = torch.from_numpy(a.ravel()).cuda()
    obuf = torch.full((ny * nx + 16,), -3.0, device="cuda")
    x, out = buf[1:1 + ny * nx], obuf[1:1 + ny * nx]
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=x, out=out, nx=nx, ny=ny),
                     STATIC, 64, 40, 64)
    got = host(obuf)
    assert np.array_equal(bits32(got[1:1 + ny * nx].reshape(ny, nx)),
                          bits32(O.stencil2d5(a)))
    assert got[0] == -3.0 and (got[1 + ny * nx:] == -3.0).all()
    assert rt.sync_status() == 0
