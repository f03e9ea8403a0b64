"""GPU parity: runtime atomics (closed forms of Sec. 3.1), barriers, the team
shared-memory stack (trace replay vs the oracle), argument errors, the stack
fallback pool and graph replay of self-resetting state."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import inputs
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


def test_atomics_closed_forms(rt):
    import torch
    G, T, reps, e = 6, 128, 4, 11
    N = G * T * reps                           # 3072, a multiple of e + 1
    words = torch.tensor([5, 0, 3, 7, 11], dtype=torch.int32, device="cuda")
    ret = torch.zeros(N, dtype=torch.int32, device="cuda")
    rt.test_atomics(G, T, reps, e, words, ret)
    w = host(words).view(np.uint32)
    assert rt.sync_status() == 0
    assert w[0] == 5 + N                       # add
    assert w[1] == N % (e + 1) == 0            # inc wraps: K mod (e+1) from 0
    vals = host(ret).view(np.uint32)           # each residue returned K/(e+1) times
    assert np.array_equal(np.bincount(vals, minlength=e + 1), np.full(e + 1, N // (e + 1)))
    assert w[2] == G * T - 1                   # max of all thread ids
    assert 0 <= w[3] < G * T                   # some thread's id was exchanged in last
    assert w[4] == 11 + N                      # cas-loop counter


@pytest.mark.parametrize("T,sub", [(32, 0), (256, 32), (1024, 128), (960, 64)])
def test_barrier(rt, T, sub):
    import torch
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rt.test_barrier(8, T, sub, 6, err)
    assert int(host(err)[0]) == 0


def _gpu_trace(ops):
    """Oracle trace (free names an allocation number) -> device trace (free
    names the op index of that allocation)."""
    g = ops.copy()
    alloc_ops = [i for i in range(len(ops)) if ops[i, 0] == 0]
    for i in range(len(ops)):
        if ops[i, 0] == 1:
            g[i, 1] = alloc_ops[ops[i, 1]] if ops[i, 1] < len(alloc_ops) else -1
    return g


@pytest.mark.parametrize("S,Q,seed,bad", [(1024, 2048, 0, False), (64, 0, 1, False),
                                          (0, 4096, 2, False), (512, 512, 3, True),
                                          (200 * 1024, 4096, 4, False)])
def test_stack_trace_vs_oracle(rt, S, Q, seed, bad):
    import torch
    ops = inputs.stack_trace(600, seed=seed, max_bytes=700, bad_free=bad)
    ref, ref_st = O.stack_replay(S, Q, ops)
    teams = 3
    out = torch.zeros((teams, len(ops), 2), dtype=torch.int64, device="cuda")
    st = torch.zeros(teams, dtype=torch.int64, device="cuda")
    rt.test_stack(teams, S, Q, dev(_gpu_trace(ops)), out, st)
    got = host(out)
    for g in range(teams):
        assert np.array_equal(got[g], ref), g
    assert np.all(host(st) == ref_st)
    rt.sync_status()  # clear the bits the trace raised


def test_stack_golden_trace(rt):
    import os
    import torch
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "stack_trace.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append([int(v) for v in line.split()])
    S, Q = rows[0]
    ops = np.array([r[:2] for r in rows[1:-1]], np.int64)
    out = torch.zeros((1, len(ops), 2), dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int64, device="cuda")
    rt.test_stack(1, S, Q, dev(_gpu_trace(ops)), out, st)
    assert host(out)[0].tolist() == [r[2:4] for r in rows[1:-1]]
    assert int(host(st)[0]) == rows[-1][0]
    assert rt.sync_status() == R.DEV_STACK_NOMEM | R.DEV_STACK_ORDER


def test_invalid_arguments_launch_nothing(rt):
    import torch
    x = torch.zeros(64, device="cuda")
    y = torch.zeros(64, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    good = R.loop_desc(R.BODY_AXPY, n=64, x=x, y=y)
    bad_cases = [
        (dict(incr=0), {}), ({}, dict(threads=48)), ({}, dict(threads=2048)),
        ({}, dict(teams=-1)), ({}, dict(sched=R.SCHED_STATIC_CHUNKED, chunk=0)),
        ({}, dict(sched=R.SCHED_DYNAMIC, chunk=0)), ({}, dict(sched=9)),
        ({}, dict(teams=R.MAX_RED_TEAMS + 1, red=R.ReduceDesc(R.OP_SUM, 0, res.data_ptr()))),
        (dict(idx_type=R.I32, ub=1 << 31), {}), (dict(reserved=1), {}),
    ]
    for dpatch, kpatch in bad_cases:
        d = R.LoopDesc.from_buffer_copy(good)
        for k, v in dpatch.items():
            setattr(d, k, v)
        kw = dict(sched=R.SCHED_STATIC, chunk=0, teams=4, threads=64)
        kw.update(kpatch)
        with pytest.raises(R.OmprtError) as ei:
            rt.launch_region(d, **kw)
        assert ei.value.status in (R.ERR_INVALID, R.ERR_UNSUPPORTED)
    assert float(host(y).sum()) == 0.0
    with pytest.raises(R.OmprtError):
        rt.alloc_shared(300 * 1024)
    st = R.loop_desc(R.BODY_STENCIL2D5, n=64, x=x, out=x, nx=8, ny=8)
    with pytest.raises(R.OmprtError):
        rt.launch_region(st)                      # in place is rejected


def test_stack_fallback_pool_keeps_results(rt):
    """With a zero-byte shared stack the reduction's scratch comes from the
    global fallback pool; the result is unchanged and no status is raised."""
    a = inputs.f32_uniform_pm1(1 << 20, 9)
    ad = dev(a)
    import torch
    r1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    r2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    rt.reduce(R.OP_SUM, ad, r1, R.PREC_COMP_F64, 200, 256)
    rt.alloc_shared(0)
    try:
        rt.reduce(R.OP_SUM, ad, r2, R.PREC_COMP_F64, 200, 256)
        assert rt.sync_status() == 0
    finally:
        rt.alloc_shared(4096)
    assert host(r1)[0] == host(r2)[0]


def test_graph_replay_self_resetting(rt):
    """A reduction and a dynamic-schedule launch captured in a CUDA graph give
    the eager result on every replay (tickets and counters reset themselves)."""
    import torch
    n = (1 << 20) + 7
    x = inputs.f32_uniform01(n, 0)
    xd = dev(x)
    y0 = inputs.f32_uniform01(n, 1)
    yd = dev(y0)
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rt.launch_region(R.loop_desc(R.BODY_DOT, n=n, x=xd, y=yd), R.SCHED_DYNAMIC, 256, 148, 256,
                         red=R.ReduceDesc(R.OP_SUM, 0, r.data_ptr()), stream=s)
    exact = O.exact_dot_f32(x, y0)
    seen = set()
    for _ in range(4):
        r.zero_()
        g.replay()
        torch.cuda.synchronize()
        v = float(host(r)[0])
        seen.add(v)
        assert abs(v - exact) <= 1e-6 * abs(exact)
    assert len(seen) == 1


def test_bounded_wait_times_out_and_context_survives(rt):
    """A wait on a flag that nothing sets gives up after its limit, reports
    OMPRT_DEV_TIMEOUT through the status word, and later launches work."""
    import torch
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    rt.test_wait(4, flag, 1, 2000, out)                  # nobody ever writes 1
    assert rt.sync_status() == R.DEV_TIMEOUT
    assert host(out).tolist() == [0, 0, 0, 0]
    flag.fill_(7)
    rt.test_wait(2, flag, 7, 2000, out)                  # already set: returns at once
    assert rt.sync_status() == 0
    assert host(out)[:2].tolist() == [1, 1]
    a = torch.arange(1000, dtype=torch.int64, device="cuda")
    r = torch.zeros(1, dtype=torch.int64, device="cuda")
    rt.reduce(R.OP_SUM, a, r, 0, 4, 64)
    assert int(host(r)[0]) == 999 * 1000 // 2
