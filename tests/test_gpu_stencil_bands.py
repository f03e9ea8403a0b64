"""GPU parity: static(1) 2-D stencil whose warps take their strips a band of
rows at a time from tensor copies (k_stencil_bands.cu).

The form applies when the team size divides nx (at least 40 wide), teams
divide ny and the input is 16-byte aligned.  Results must be bit-exact
against the oracle for one-row to many-row grids, one to many strips a
thread, bands shorter than a team's block and longer, every buffer count,
and launches outside the form (they fall back to the other forms)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu

STATIC = R.SCHED_STATIC_CHUNKED


def _run(rt, ad, ny, nx, G, T):
    import torch
    out = torch.full((ny, nx), -7.0, device="cuda")
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx, ny=ny),
                     STATIC, 1, G, T)
    return bits32(host(out))


@pytest.mark.parametrize("nx", [64, 96, 256, 1024])
@pytest.mark.parametrize("ny", [1, 2, 3, 17, 64])
def test_bands_bit_exact(rt, nx, ny):
    a = inputs.grid_f32(ny, nx, 51)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    teams = sorted({g for g in (1, 2, ny // 2, ny) if g >= 1 and ny % g == 0})
    try:
        for NB in (2, 3, 4):
            rt.set_stencil_slab_shape(0, NB)
            for G in teams:
                for T in (32, 64, 128, 512, 1024):
                    if nx % T:
                        continue
                    got = _run(rt, ad, ny, nx, G, T)
                    assert np.array_equal(got, want), (NB, G, T)
    finally:
        rt.set_stencil_slab_shape(0, 0)
    assert rt.sync_status() == 0


def test_bands_full_grid(rt):
    """4096^2 at the shapes the tuner may pick."""
    import torch
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for G, T in ((4096, 1024), (4096, 512), (2048, 1024), (1024, 256), (512, 128)):
        out = torch.empty_like(ad)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                     ny=4096), STATIC, 1, G, T)
        assert np.array_equal(bits32(host(out)), want), (G, T)
    assert rt.sync_status() == 0


def test_bands_outside_the_form_falls_back(rt):
    """A team size not dividing nx, teams not dividing ny, a grid narrower
    than a box row, a misaligned input view: other forms, bit-exact, and the
    floats around the view untouched."""
    import torch
    for ny, nx, G, T in ((12, 192, 4, 128), (12, 256, 5, 64), (9, 32, 3, 32)):
        a = inputs.grid_f32(ny, nx, 52)
        got = _run(rt, dev(a), ny, nx, G, T)
        assert np.array_equal(got, bits32(O.stencil2d5(a))), (ny, nx, G, T)
    ny, nx = 40, 512
    a = inputs.grid_f32(ny, nx, 53)
    buf = torch.zeros(ny * nx + 16, device="cuda")
    buf[1:1 + ny * nx] = torch.from_numpy(a.ravel()).cuda()
    obuf = torch.full((ny * nx + 16,), -3.0, device="cuda")
    x, out = buf[1:1 + ny * nx], obuf[1:1 + ny * nx]
    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=x, out=out, nx=nx, ny=ny),
                     STATIC, 1, 40, 128)
    got = host(obuf)
    assert np.array_equal(bits32(got[1:1 + ny * nx].reshape(ny, nx)), bits32(O.stencil2d5(a)))
    assert got[0] == -3.0 and (got[1 + ny * nx:] == -3.0).all()
    assert rt.sync_status() == 0
