"""GPU parity: generic-mode (non-SPMD) regions over segments: the main
thread's sequential code, the worker hand-over, the globalised variable on
the team stack and the nested parallel for with reduction.  Dot results
within 1e-6 of the exact sums, axpy outputs bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, dev, host

pytestmark = pytest.mark.gpu


def _segments(nseg, seed, max_len=5000):
    g = np.random.default_rng(seed)
    lens = np.rint(np.exp(g.normal(np.log(300), 1.5, size=nseg))).astype(np.int64)
    lens = np.clip(lens, 0, max_len)
    lens[::7] = 0                                     # some empty segments
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


@pytest.mark.parametrize("nseg,G,T", [(1, 1, 32), (37, 7, 256), (4096, 152, 256),
                                      (500, 3, 1024), (64, 200, 64)])
def test_generic_dot_segments(rt, nseg, G, T):
    import torch
    seg = _segments(nseg, nseg)
    n = int(seg[-1])
    x, y = inputs.f32_uniform01(max(n, 1), 0)[:n], inputs.f32_uniform01(max(n, 1), 1)[:n]
    res = torch.full((nseg,), -1.0, dtype=torch.float64, device="cuda")
    xd, yd, segd = dev(x), dev(y), dev(seg)
    desc = R.loop_desc(R.BODY_DOT, n=n, x=xd, y=yd)
    rt.launch_generic(segd, desc, res, G, T)
    assert rt.sync_status() == 0
    got = host(res)
    for s in range(nseg):
        a, b = seg[s], seg[s + 1]
        exact = O.exact_dot_f32(x[a:b], y[a:b])
        assert abs(got[s] - exact) <= 1e-6 * max(abs(exact), 1e-300), s


def test_generic_axpy_segments(rt):
    import torch
    nseg = 300
    seg = _segments(nseg, 5)
    n = int(seg[-1])
    x, y = inputs.f32_uniform01(n, 2), inputs.f32_uniform01(n, 3)
    xd, yd = dev(x), dev(y)
    res = torch.zeros(nseg, dtype=torch.float64, device="cuda")
    rt.launch_generic(dev(seg), R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), res, 13, 128)
    ynew = O.axpy_f32(3.0, x, y)
    assert np.array_equal(bits32(host(yd)), bits32(ynew))
    got = host(res)
    for s in range(nseg):
        exact = O.exact_sum_f32(ynew[seg[s]:seg[s + 1]])
        assert abs(got[s] - exact) <= 1e-6 * max(abs(exact), 1e-300)


def test_generic_bad_offsets_flagged(rt):
    import torch
    seg = np.array([0, 10, 5, 20], np.int64)           # decreasing: invalid
    x = torch.zeros(20, device="cuda")
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    rt.launch_generic(dev(seg), R.loop_desc(R.BODY_DOT, n=20, x=x, y=x), res, 1, 32)
    assert rt.sync_status() & R.DEV_BAD_ARG


@pytest.mark.parametrize("nseg,G,T", [(1, 1, 32), (37, 7, 256), (4096, 152, 256),
                                      (500, 3, 1024), (64, 200, 64)])
def test_generic_two_regions_per_segment(rt, nseg, G, T):
    """Program DOT_AXPY: per segment the main thread runs region 1
    (v = x . y), computes a = (float)v * alpha from its result, and runs region
    2 (y = a x + y, w = sum of the new y) with that value.  v and w are
    globalised on the team stack.  v and w within the C7 bound of the exact
    sums; a is the fp32 product of v rounded to fp32 and alpha; y bit-exact
    against the oracle's axpy with each segment's a."""
    import torch
    seg = _segments(nseg, nseg + 1000)
    n = int(seg[-1])
    alpha = 1.0 / 64
    x, y = inputs.f32_uniform01(max(n, 1), 4)[:n], inputs.f32_uniform01(max(n, 1), 5)[:n]
    xd, yd = dev(x), dev(y)
    res = torch.full((3 * nseg,), -1.0, dtype=torch.float64, device="cuda")
    desc = R.loop_desc(R.BODY_DOT, n=n, x=xd, y=yd, alpha=alpha)
    rt.launch_generic(dev(seg), desc, res, G, T, program=R.GENERIC_DOT_AXPY)
    assert rt.sync_status() == 0
    got = host(res).reshape(nseg, 3)
    ynew = y.copy()
    for s in range(nseg):
        lo, hi = seg[s], seg[s + 1]
        v, a, w = got[s]
        exact = O.exact_dot_f32(x[lo:hi], y[lo:hi])
        assert abs(v - exact) <= 1e-6 * max(abs(exact), 1e-300), s
        assert a == float(np.float32(np.float32(v) * np.float32(alpha))), s
        ynew[lo:hi] = O.axpy_f32(np.float32(a), x[lo:hi], y[lo:hi])
        wexact = O.exact_sum_f32(ynew[lo:hi])
        assert abs(w - wexact) <= 1e-6 * max(abs(wexact), 1e-300), s
    assert np.array_equal(bits32(host(yd)), bits32(ynew))


def test_generic_out_of_stack_flagged(rt):
    """The team stack holds the runtime's reduction scratch and the
    globalised variables; with no shared-memory stack (S = 0) they go to the
    team's pool slice, which exists for teams below MAX_RED_TEAMS only.  A
    launch with more teams than that: the teams with a slice compute their
    segments, the others set STACK_NOMEM and write nothing."""
    import torch
    G = R.MAX_RED_TEAMS + 8
    nseg = G
    seg = np.arange(nseg + 1, dtype=np.int64) * 64
    n = int(seg[-1])
    x, y = inputs.f32_uniform01(n, 6), inputs.f32_uniform01(n, 7)
    res = torch.full((3 * nseg,), -1.0, dtype=torch.float64, device="cuda")
    rt.alloc_shared(0)
    try:
        rt.launch_generic(dev(seg), R.loop_desc(R.BODY_DOT, n=n, x=dev(x), y=dev(y), alpha=0.5),
                          res, G, 32, program=R.GENERIC_DOT_AXPY)
        bits = rt.sync_status()
    finally:
        rt.alloc_shared(4096)
    assert bits & R.DEV_STACK_NOMEM
    got = host(res).reshape(nseg, 3)
    ok = R.MAX_RED_TEAMS
    assert np.all(got[ok:] == -1.0)                   # no pool slice: nothing written
    for s in (0, 1, ok // 2, ok - 1):
        exact = O.exact_dot_f32(x[seg[s]:seg[s + 1]], y[seg[s]:seg[s + 1]])
        assert abs(got[s, 0] - exact) <= 1e-6 * abs(exact)
    # the stack is clean again for the next launch
    res2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    rt.launch_generic(dev(seg[:2]), R.loop_desc(R.BODY_DOT, n=n, x=dev(x), y=dev(y), alpha=0.5),
                      res2, 1, 32, program=R.GENERIC_DOT_AXPY)
    assert rt.sync_status() == 0
