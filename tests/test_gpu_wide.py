"""Loops past 2^32 iterations (GPU): the 64-bit index paths.

Below 2^32 the runtime maps a logical index to its stencil row with one
multiply-high; from 2^32 on every team block, chunk, claim and row is
computed in 64 bits, and the tiled and row-ring stencil forms check their
32-bit limits before they take a launch.  These tests run the bodies at
n = 2^32 + a few thousand under the level-2 schedules.  The inputs are
counter-based (a function of the index and a seed), so the oracle checks
sampled outputs: every team-block boundary, the indices around 2^31 and 2^32,
both ends and a random sample.  About 40 GB of device memory per test."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import host

pytestmark = pytest.mark.gpu

N_WIDE = (1 << 32) + 4100
GIB = 1 << 30


def need_gib(g):
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < g * GIB:
        pytest.skip("needs %d GiB free on the device" % g)


@pytest.fixture(scope="module")
def rt():
    r = R.Runtime(0)
    yield r
    r.close()


def team_blocks(n, G):
    return [O.static_nochunk(n, G, g) for g in range(G)]


def probes(n, Gs, seed=0, k=2000, extra=()):
    idx = {0, 1, n - 1, n - 2, n - 4100, (1 << 31) - 1, 1 << 31, (1 << 31) + 1}
    idx.update(range((1 << 32) - 8, (1 << 32) + 8))
    idx.update(extra)
    for G in Gs:
        for bs, bn in team_blocks(n, G):
            if bn:
                idx.update((bs, bs + 1, bs + bn - 2, bs + bn - 1))
    idx.update(int(v) for v in np.random.default_rng(seed).integers(0, n, size=k))
    return np.array(sorted(i for i in idx if 0 <= i < n), dtype=np.int64)


def gather(t, idx):
    import torch
    return host(t[torch.from_numpy(idx).cuda()])


AXPY_RUNS = [(R.SCHED_STATIC, 0, 1184, 256), (R.SCHED_STATIC_CHUNKED, 8, 8192, 256),
             (R.SCHED_STATIC_CHUNKED, 1, 4096, 256), (R.SCHED_STATIC_CHUNKED, 64, 2048, 128),
             (R.SCHED_DYNAMIC, 256, 8192, 32), (R.SCHED_NONMONOTONIC, 256, 4096, 64),
             (R.SCHED_GUIDED, 64, 1184, 256), (R.SCHED_AUTO, 0, 1184, 1024)]
AXPY_DIST_RUNS = [(2048, R.SCHED_STATIC_CHUNKED, 8, 4096, 256),   # d = 8T, static(8)
                  (256, R.SCHED_STATIC_CHUNKED, 1, 4096, 256),    # d = T, static(1)
                  (1 << 20, R.SCHED_STATIC, 0, 1000, 512)]


def test_axpy_past_2_32(rt):
    """y = 3x + y in place, bit-exact at every probe after every launch."""
    import torch
    need_gib(40)
    n = N_WIDE
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    inputs.counter_f32_01_fill(x, 0)
    inputs.counter_f32_01_fill(y, 1)
    idx = probes(n, sorted({G for *_, G, _ in AXPY_RUNS}))
    xs = inputs.counter_f32_01(idx, 0)
    want = inputs.counter_f32_01(idx, 1)
    desc = R.loop_desc(R.BODY_AXPY, n=n, x=x, y=y, alpha=3.0)
    for sched, chunk, G, T in AXPY_RUNS:
        rt.launch_region(desc, sched, chunk, G, T)
        want = O.axpy_f32(3.0, xs, want)
        got = gather(y, idx)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (sched, chunk, G, T)
    for d, sched, chunk, G, T in AXPY_DIST_RUNS:
        rt.launch_region_dist(desc, d, sched, chunk, G, T)
        want = O.axpy_f32(3.0, xs, want)
        got = gather(y, idx)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (d, sched, chunk, G, T)
    assert rt.sync_status() == 0
    del x, y
    torch.cuda.empty_cache()


def static_owner(n, G, T, chunk, idx):
    """g * T + t of the thread that owns each index under static (chunk 0) or
    static(chunk), from the oracle's level-1 blocks and level-2 ranges."""
    blocks = team_blocks(n, G)
    starts = np.array([b[0] for b in blocks], dtype=np.int64)
    out = np.empty(idx.size, dtype=np.int64)
    for k, i in enumerate(idx.tolist()):
        g = int(np.searchsorted(starts, i, side="right")) - 1
        bs, bn = blocks[g]
        assert bs <= i < bs + bn
        loc = i - bs
        if chunk == 0:
            lo, hi = 0, T - 1
            while lo < hi:
                mid = (lo + hi + 1) // 2
                if O.static_nochunk(bn, T, mid)[0] <= loc:
                    lo = mid
                else:
                    hi = mid - 1
            s, c = O.static_nochunk(bn, T, lo)
            assert s <= loc < s + c
            t = lo
        else:
            t = (loc // chunk) % T
            LB, _, st, _ = O.for_static_init(0, bn - 1, 1, "i64", T, t, chunk)
            assert loc >= LB and (loc - LB) % st < chunk
        out[k] = g * T + t
    return out


MAP_STATIC_RUNS = [(0, 1000, 256), (7, 777, 128), (1, 2048, 1024), (64, 152, 512)]


def test_map_record_past_2_32(rt):
    """Every iteration runs exactly once; under static / static(c) its owner is
    the oracle's; under dynamic(c) it stays in its team's block and a chunk
    has one owner; the last-iteration flag is set once, on the owner of n - 1."""
    import torch
    need_gib(40)
    n = (1 << 32) + 5
    owner = torch.empty(n, dtype=torch.int32, device="cuda")
    count = torch.empty(n, dtype=torch.int32, device="cuda")

    def run(sched, chunk, G, T):
        owner.fill_(-1)
        count.zero_()
        last = torch.full((G * T,), -1, dtype=torch.int32, device="cuda")
        desc = R.loop_desc(R.BODY_MAP_RECORD, n=n, x=last, y=count, out=owner, data_type=R.I32)
        rt.launch_region(desc, sched, chunk, G, T)
        assert rt.sync_status() == 0
        assert int((count != 1).sum().item()) == 0, (sched, chunk, G, T)
        lf = host(last)
        assert int((lf == 1).sum()) == 1
        assert lf[int(gather(owner, np.array([n - 1]))[0])] == 1

    for chunk, G, T in MAP_STATIC_RUNS:
        run(R.SCHED_STATIC_CHUNKED if chunk else R.SCHED_STATIC, chunk, G, T)
        idx = probes(n, [G], seed=chunk)
        got = gather(owner, idx).astype(np.int64)
        assert np.array_equal(got, static_owner(n, G, T, chunk, idx)), (chunk, G, T)

    c, G, T = 100, 1500, 64
    run(R.SCHED_DYNAMIC, c, G, T)
    blocks = team_blocks(n, G)
    starts = np.array([b[0] for b in blocks], dtype=np.int64)
    for i in probes(n, [G], seed=9, k=300).tolist():
        g = int(np.searchsorted(starts, i, side="right")) - 1
        bs, bn = blocks[g]
        cs = bs + (i - bs) // c * c
        ce = min(cs + c, bs + bn)
        own = host(owner[cs:ce])
        assert np.all(own == own[0]) and own[0] // T == g, (i, g)
    del owner, count
    torch.cuda.empty_cache()


STENCIL_RUNS = [(R.SCHED_AUTO, 0, 1184, 256), (R.SCHED_STATIC_CHUNKED, 64, 1024, 512),
                (R.SCHED_STATIC_CHUNKED, 8, 4096, 256), (R.SCHED_STATIC, 0, 8192, 128),
                (R.SCHED_DYNAMIC, 256, 4096, 32)]


def test_stencil2d_past_2_32(rt):
    """65536 x 65540 grid (row 65536 starts at index 2^32), bit-exact at every
    probe, including the rows and columns around the 2^32 crossing."""
    import torch
    need_gib(40)
    nx, ny = 65536, 65540
    n = nx * ny
    a = torch.empty(n, dtype=torch.float32, device="cuda")
    inputs.counter_f32_01_fill(a, 6)
    out = torch.empty_like(a)
    cross = [(1 << 32) + d for d in (-nx - 1, -nx, -2, -1, 0, 1, nx - 1, nx, nx + 1)]
    edges = [65536 * nx - 1, 65536 * nx + nx - 1, 65535 * nx, (ny - 1) * nx + 5, 3 * nx + nx - 1]
    idx = probes(n, sorted({G for *_, G, _ in STENCIL_RUNS}), seed=6, extra=cross + edges)
    # the oracle on each probe's 3 x 3 neighbourhood; boundary points copy
    want = np.empty(idx.size, dtype=np.float32)
    for k, i in enumerate(idx.tolist()):
        r, c = divmod(i, nx)
        if r == 0 or c == 0 or r == ny - 1 or c == nx - 1:
            want[k] = inputs.counter_f32_01(np.array([i]), 6)[0]
        else:
            nb = np.array([[(r + dr) * nx + c + dc for dc in (-1, 0, 1)] for dr in (-1, 0, 1)])
            patch = inputs.counter_f32_01(nb.reshape(-1), 6).reshape(3, 3)
            want[k] = O.stencil2d5(patch)[1, 1]
    desc = R.loop_desc(R.BODY_STENCIL2D5, n=n, x=a, out=out, nx=nx, ny=ny)
    for sched, chunk, G, T in STENCIL_RUNS:
        out.fill_(-7.0)
        rt.launch_region(desc, sched, chunk, G, T)
        got = gather(out, idx)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (sched, chunk, G, T)
    assert rt.sync_status() == 0
    del a, out
    torch.cuda.empty_cache()
