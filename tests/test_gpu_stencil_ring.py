"""GPU parity: the 2-D stencil's streamed-ring form (dynamic(c) and
static(1); k_stencil_owner.cu).

Each CTA streams its teams' rows through a ring of row-sized segments in
shared memory, a producer warp refilling slots that every team group has
released; groups of thread_limit threads each play one team at a time and
every thread runs exactly its own iterations.  Results must be bit-exact
against the oracle for ragged grids (down to 1 x 4), one to thousands of
teams, teams of 32 to 512 threads (1024 falls back to the plain form), chunk
sizes that do and do not divide the rows, ring budgets from a few segments to
the whole shared memory, the 4096^2 grid at the benchmark's shapes, and under
CUDA-graph replay."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu

DEFAULT_BUDGET = 226 * 1024


@pytest.fixture
def ring(rt):
    yield rt
    rt.set_stencil_stage_bytes(DEFAULT_BUDGET)


SCHEDS = [(R.SCHED_DYNAMIC, 1), (R.SCHED_DYNAMIC, 4), (R.SCHED_DYNAMIC, 64),
          (R.SCHED_DYNAMIC, 68), (R.SCHED_DYNAMIC, 256), (R.SCHED_DYNAMIC, 1000),
          (R.SCHED_STATIC_CHUNKED, 1)]


@pytest.mark.parametrize("ny,nx", [(1, 4), (2, 8), (9, 8), (33, 132), (67, 40), (100, 64),
                                   (5, 16), (300, 1028), (41, 4096)])
@pytest.mark.parametrize("budget", [DEFAULT_BUDGET, 65536, 16384])
def test_ring_bit_exact(ring, ny, nx, budget):
    import torch
    rt = ring
    rt.set_stencil_stage_bytes(budget)
    a = inputs.grid_f32(ny, nx, 9)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for sched, chunk in SCHEDS:
        for G, T in ((1, 32), (3, 64), (7, 96), (64, 256), (500, 32), (13, 512), (5, 480),
                     (13, 1024), (4096, 32)):
            out = torch.full((ny, nx), -7.0, device="cuda")
            rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx,
                                         ny=ny), sched, chunk, G, T)
            assert np.array_equal(bits32(host(out)), want), (sched, chunk, G, T)
    assert rt.sync_status() == 0


def test_ring_full_grid(ring):
    """4096^2 at the benchmark's shapes and around them."""
    import torch
    rt = ring
    a = inputs.grid_f32(4096, 4096, 0)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for sched, chunk, G, T in ((R.SCHED_DYNAMIC, 256, 4096, 32), (R.SCHED_DYNAMIC, 256, 2048, 64),
                               (R.SCHED_DYNAMIC, 256, 1024, 128), (R.SCHED_DYNAMIC, 256, 8192, 32),
                               (R.SCHED_DYNAMIC, 64, 4096, 64),
                               (R.SCHED_STATIC_CHUNKED, 1, 4096, 128),
                               (R.SCHED_STATIC_CHUNKED, 1, 2048, 256),
                               (R.SCHED_STATIC_CHUNKED, 1, 152, 512)):
        out = torch.empty_like(ad)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=4096 * 4096, x=ad, out=out, nx=4096,
                                     ny=4096), sched, chunk, G, T)
        assert np.array_equal(bits32(host(out)), want), (sched, chunk, G, T)
    assert rt.sync_status() == 0


def test_ring_in_a_cuda_graph(ring):
    """Ring launches captured in a CUDA graph: every replay reproduces the
    oracle's output bit for bit (the counters and barriers need no reset)."""
    import torch
    rt = ring
    g1 = inputs.grid_f32(300, 1028, 3)
    g2 = inputs.grid_f32(64, 4096, 4)
    d1, d2 = dev(g1), dev(g2)
    o1, o2 = torch.empty_like(d1), torch.empty_like(d2)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=300 * 1028, x=d1, out=o1, nx=1028,
                                     ny=300), R.SCHED_DYNAMIC, 64, 600, 32, stream=s)
        rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=64 * 4096, x=d2, out=o2, nx=4096,
                                     ny=64), R.SCHED_STATIC_CHUNKED, 1, 64, 128, stream=s)
    for _ in range(3):
        o1.fill_(-7.0)
        o2.fill_(-7.0)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(bits32(host(o1)), bits32(O.stencil2d5(g1)))
        assert np.array_equal(bits32(host(o2)), bits32(O.stencil2d5(g2)))
    assert rt.sync_status() == 0


def test_stencil_stage_bytes_validation(rt):
    with pytest.raises(R.OmprtError):
        rt.set_stencil_stage_bytes(-16)
    with pytest.raises(R.OmprtError):
        rt.set_stencil_stage_bytes(1 << 30)
    rt.set_stencil_stage_bytes(DEFAULT_BUDGET)


@pytest.mark.parametrize("stage", [32768, 0])
def test_every_schedule_without_the_stencil_budget(ring, stage):
    """With the stencil stage budget at 0 the ring, slab, band and column forms
    are off: every schedule takes the strips, the row passes or (with the
    staged-region budget also 0) the plain region kernel, bit-exact."""
    import torch
    rt = ring
    rt.set_stencil_stage_bytes(0)
    rt.set_stage_bytes(stage)
    try:
        for ny, nx in ((40, 512), (33, 4096), (7, 100)):
            a = inputs.grid_f32(ny, nx, 19)
            ad = dev(a)
            want = bits32(O.stencil2d5(a))
            for sched, chunk in ((R.SCHED_STATIC, 0), (R.SCHED_STATIC_CHUNKED, 1),
                                 (R.SCHED_STATIC_CHUNKED, 8), (R.SCHED_STATIC_CHUNKED, 64),
                                 (R.SCHED_DYNAMIC, 64), (R.SCHED_DYNAMIC, 256),
                                 (R.SCHED_AUTO, 0)):
                for G, T in ((ny, 32), (ny, 64), (1, 512), (5, 128)):
                    out = torch.full((ny, nx), -7.0, device="cuda")
                    rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out,
                                                 nx=nx, ny=ny), sched, chunk, G, T)
                    assert np.array_equal(bits32(host(out)), want), (ny, nx, sched, chunk, G, T)
    finally:
        rt.set_stage_bytes(32768)
    assert rt.sync_status() == 0
