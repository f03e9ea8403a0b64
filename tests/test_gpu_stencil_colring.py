"""GPU parity: static(c) and dynamic(c) 2-D stencil with teams of one warp
whose blocks are the 32 / m rows that hold 32 chunks, the CTA's warps
playing adjacent teams from one tensor copy a step (k_stencil_colring.cu).

The form applies when T = 32, c is a multiple of 32, m = nx / c divides 32
with m < 32, and ny / G = 32 / m; the same launches with m >= 32 (one-row
blocks) take the per-warp slabs.  Results must be bit-exact against the
oracle for every m from 1 to 16 with one to many slabs a chunk (the words
across a chunk boundary come from the neighbouring lanes, the chunk's first
sector is stored at its last slab), CTAs with fewer teams than warps (idle
warps in the last round), CTAs that play their rounds in reverse, every
buffer count, and the full grid."""
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


@pytest.mark.parametrize("nx,c", [(32, 32), (64, 32), (256, 64), (1024, 32), (1024, 64),
                                  (1024, 256), (2048, 1024), (2048, 64), (4096, 128),
                                  (64, 64), (256, 256), (256, 32), (512, 64), (128, 32)])
@pytest.mark.parametrize("G", [1, 2, 7, 40, 300])
def test_colring_bit_exact(rt, nx, c, G):
    m = nx // c
    rows = 32 // min(m, 32)
    ny = G * rows
    a = inputs.grid_f32(ny, nx, 61)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    try:
        for NB in (2, 3, 4):
            rt.set_stencil_slab_shape(0, NB)
            for sched in (STATIC, DYN):
                got = _run(rt, ad, ny, nx, sched, c, G, 32)
                assert np.array_equal(got, want), (NB, sched)
    finally:
        rt.set_stencil_slab_shape(0, 0)
    assert rt.sync_status() == 0


def test_colring_full_grid(rt):
    import torch
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for sched, chunk, G in ((STATIC, 64, 4096), (DYN, 64, 4096), (DYN, 256, 2048),
                            (STATIC, 256, 2048), (STATIC, 32, 4096), (DYN, 1024, 512)):
        out = torch.empty_like(ad)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                     ny=4096), sched, chunk, G, 32)
        assert np.array_equal(bits32(host(out)), want), (sched, chunk, G)
    assert rt.sync_status() == 0
