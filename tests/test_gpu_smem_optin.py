"""GPU: launches whose shared memory, static and dynamic together, just
passes the 48 KB a kernel gets without its opt-in.

Each of these ran into a launch error while the opt-in was only taken for
more than 48 KB of dynamic memory: the row-pass ring of a 2048-wide static(c)
stencil (exactly 48 KB of rows), a reduction whose team stack is 44 KB (the
region kernels carry several KB of their own), a generic-mode region with a
48 KB stack, and the stack test kernel at 48 KB."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu


def test_rows_ring_of_48k(rt):
    import torch
    ny, nx = 33, 2048
    a = inputs.grid_f32(ny, nx, 41)
    ad = dev(a)
    want = bits32(O.stencil2d5(a))
    for chunk in (32, 64, 128):
        for G, T in ((1, 512), (1, 256), (3, 512)):
            out = torch.full((ny, nx), -7.0, device="cuda")
            rt.launch_region(R.loop_desc(R.BODY_STENCIL2D5, n=ny * nx, x=ad, out=out, nx=nx,
                                         ny=ny), R.SCHED_STATIC_CHUNKED, chunk, G, T)
            assert np.array_equal(bits32(host(out)), want), (chunk, G, T)
    assert rt.sync_status() == 0


@pytest.mark.parametrize("stack", [40 * 1024, 44 * 1024, 48 * 1024])
def test_reduction_with_large_stack(rt, stack):
    import torch
    a = inputs.int64_uniform(1 << 20, 42)
    rt.alloc_shared(stack)
    try:
        r = torch.zeros(1, dtype=torch.int64, device="cuda")
        rt.reduce(R.OP_SUM, dev(a), r, 0, 152, 256)
        assert int(host(r)[0]) == int(a.sum(dtype=np.int64))
    finally:
        rt.alloc_shared(4096)
    assert rt.sync_status() == 0


def test_generic_with_48k_stack(rt):
    import torch
    seg = np.array([0, 1000, 1000, 5000, 20000], dtype=np.int64)
    n = int(seg[-1])
    x, y = inputs.f32_uniform01(n, 3), inputs.f32_uniform01(n, 4)
    rt.alloc_shared(48 * 1024)
    try:
        res = torch.full((len(seg) - 1,), -1.0, dtype=torch.float64, device="cuda")
        rt.launch_generic(dev(seg), R.loop_desc(R.BODY_DOT, n=n, x=dev(x), y=dev(y)), res, 4, 128)
        got = host(res)
    finally:
        rt.alloc_shared(4096)
    assert rt.sync_status() == 0
    for s in range(len(seg) - 1):
        exact = O.exact_dot_f32(x[seg[s]:seg[s + 1]], y[seg[s]:seg[s + 1]])
        assert abs(got[s] - exact) <= 1e-6 * max(abs(exact), 1e-300), s


def test_stack_kernel_at_48k(rt):
    import torch
    ops = inputs.stack_trace(200, seed=5, max_bytes=700, bad_free=False)
    S = 48 * 1024
    ref, ref_st = O.stack_replay(S, 1024, ops)
    out = torch.zeros((2, len(ops), 2), dtype=torch.int64, device="cuda")
    st = torch.zeros(2, dtype=torch.int64, device="cuda")
    from test_gpu_runtime import _gpu_trace
    rt.test_stack(2, S, 1024, dev(_gpu_trace(ops)), out, st)
    got = host(out)
    for g in range(2):
        assert np.array_equal(got[g], ref), g
    assert np.all(host(st) == ref_st)
    rt.sync_status()
