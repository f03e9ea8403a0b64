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
