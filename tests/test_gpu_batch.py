"""GPU parity: the batched persistent executor.  Every region's output
matches the oracle (axpy and stencil bit-exact, dot within 1e-6 of the exact
sum), matches the one-launch-per-region form, and stays right on CUDA-graph
replay (queue head and tickets reset themselves)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import batched, inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import bits32, host

pytestmark = pytest.mark.gpu


def check_against_oracle(rs, y, out, res, rounds=1):
    for r in range(rs.nregions):
        n, k, o = int(rs.n[r]), int(rs.kind[r]), int(rs.offset[r])
        xs, ys = rs.x0[o:o + n], rs.y0[o:o + n]
        if k == inputs.KIND_AXPY:
            ref = ys
            for _ in range(rounds):
                ref = O.axpy_f32(rs.alpha, xs, ref)
            assert np.array_equal(bits32(y[o:o + n]), bits32(ref)), r
        elif k == inputs.KIND_DOT:
            exact = O.exact_dot_f32(xs, ys)
            assert abs(res[r] - exact) <= 1e-6 * abs(exact), r
        else:
            assert np.array_equal(bits32(out[o:o + n]), bits32(O.stencil1d3(xs))), r


@pytest.mark.parametrize("chunk,threads", [(256, 64), (2048, 256), (8192, 512), (65536, 1024)])
def test_batch_small_set_vs_oracle(rt, chunk, threads):
    rs = batched.RegionSet(nregions=300, seed=7)
    b = rs.batch(rt, chunk)
    b.launch(0, threads)
    assert rt.sync_status() == 0
    check_against_oracle(rs, host(rs.y), host(rs.out), host(rs.res))
    b.destroy()


def test_batch_matches_per_region_and_replays(rt):
    import torch
    rs = batched.RegionSet(nregions=4096)
    rs.launch_per_region(rt)
    y1, o1, r1 = host(rs.y).copy(), host(rs.out).copy(), host(rs.res).copy()
    check_against_oracle(rs, y1, o1, r1)
    rs.reset()
    b = rs.batch(rt)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.launch(0, 256, stream=s)
    g.replay()
    torch.cuda.synchronize()
    y2, o2, r2 = host(rs.y).copy(), host(rs.out).copy(), host(rs.res).copy()
    assert np.array_equal(bits32(y1), bits32(y2))
    assert np.array_equal(bits32(o1), bits32(o2))
    dot = rs.kind == inputs.KIND_DOT
    assert np.all(np.abs(r2[dot] - r1[dot]) <= 1e-6 * np.abs(r1[dot]))
    # replay twice more: axpy regions advance, dot results repeat bit for bit
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    check_against_oracle(rs, host(rs.y), host(rs.out), host(rs.res), rounds=3)
    assert np.array_equal(host(rs.res)[dot], r2[dot])
    assert rt.sync_status() == 0
    b.destroy()


def test_batch_rejects_bad_regions(rt):
    import torch
    x = torch.zeros(1000, device="cuda")
    y = torch.zeros(1000, device="cuda")
    good = R.loop_desc(R.BODY_AXPY, n=1000, x=x, y=y)
    bad = [R.loop_desc(R.BODY_AXPY, lb=5, ub=100, x=x, y=y),            # lb != 0
           R.loop_desc(R.BODY_DOT, n=1000, x=x, y=y),                     # dot without result
           R.loop_desc(R.BODY_STENCIL2D5, n=1000, x=x, out=y, nx=10, ny=100)]
    for d in bad:
        with pytest.raises(R.OmprtError):
            rt.batch_create([good, d])
    with pytest.raises(R.OmprtError):
        rt.batch_create([good], chunk_elems=100)
