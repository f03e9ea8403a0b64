"""GPU parity: worksharing maps (static tables and owner maps bit-exact
against the oracle; dynamic and auto schedules by invariants)."""
import numpy as np
import pytest

import oracle as O
from paper_2106_03219_gb300 import omprt as R
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu

BOUNDS = [("i64", 0, 1), ("i32", -5, 3), ("i64", 100, -7), ("u32", 4000000000, -2),
          ("u64", (1 << 64) - 60000, 1), ("i32", (1 << 31) - 200000, 1)]


@pytest.mark.parametrize("t,lb,incr", BOUNDS)
def test_static_init_table_bit_exact(rt, t, lb, incr):
    import torch
    for n in (0, 1, 5, 17, 1000, 123457):
        if t in ("u64", "i32") and n * abs(incr) > 190000:
            continue
        ub = lb + (n - 1) * incr if n else lb - incr
        desc = R.loop_desc(R.BODY_NONE, lb=lb, ub=ub, incr=incr, idx_type=R.TYPE_CODES[t],
                           data_type=R.F32)
        for G, T in ((1, 1), (3, 32), (7, 96), (152, 1024)):
            for c in (0, 1, 3, 8, 64):
                tab = torch.empty((G * T, 8), dtype=torch.int64, device="cuda")
                rt.static_init_table(desc, c, G, T, tab)
                ref = O.composite_table(lb, ub, incr, t, G, T, c)
                assert np.array_equal(host(tab), ref), (n, G, T, c)


def _map_record(rt, n, G, T, sched, chunk, with_seq=False):
    import torch
    owner = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros((max(n, 1),), dtype=torch.int32, device="cuda")
    last = torch.full((G * T,), -1, dtype=torch.int32, device="cuda")
    seq = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda") if with_seq else None
    desc = R.loop_desc(R.BODY_MAP_RECORD, n=n, x=last, y=count, out=owner, data_type=R.I32,
                       seq=seq)
    rt.launch_region(desc, sched, chunk, G, T)
    assert rt.sync_status() == 0
    if with_seq:
        return host(owner)[:n], host(count)[:n], host(last), host(seq)[:n]
    return host(owner)[:n], host(count)[:n], host(last)


def _run_order(owner, seq):
    """Per thread: its iterations in the order it ran them (sorted by seq).
    Checks that every thread's seq values are exactly 0 .. k-1."""
    order = np.lexsort((seq, owner))          # by owner, then by seq
    own, sq = owner[order], seq[order]
    starts = np.flatnonzero(np.r_[True, own[1:] != own[:-1]])
    rank = np.arange(owner.size) - np.repeat(starts, np.diff(np.r_[starts, owner.size]))
    assert np.array_equal(sq, rank), "a thread's ordinals are not 0 .. k-1"
    return order, own


CASES = [(0, 4, 32), (1, 1, 32), (31, 4, 32), (1000, 13, 128), (100003, 148, 256),
         ((1 << 20) + 7, 1184, 1024), (5000, 3, 1024)]


@pytest.mark.parametrize("n,G,T", CASES)
@pytest.mark.parametrize("chunk", [0, 1, 5, 8, 64])
def test_static_owner_map_bit_exact(rt, n, G, T, chunk):
    sched = R.SCHED_STATIC if chunk == 0 else R.SCHED_STATIC_CHUNKED
    owner, count, last = _map_record(rt, n, G, T, sched, chunk)
    assert np.array_equal(owner, O.owner_map(n, G, T, chunk))
    assert np.all(count == 1)
    assert int((last == 1).sum()) == (1 if n else 0)
    if n:
        assert last[owner[n - 1]] == 1


@pytest.mark.parametrize("n,G,T", CASES)
@pytest.mark.parametrize("chunk", [1, 7, 256])
def test_dynamic_invariants(rt, n, G, T, chunk):
    """C4: (1) every iteration runs exactly once; (2) each thread runs whole
    chunks of its own team's block; (3) every thread runs its chunks, and the
    iterations inside them, in increasing order (the claim counter only
    grows); (4) the claims: team g's ceil(n_g / c) chunks are handed out in
    groups of 32 consecutive chunks (one atomic add per warp), chunk j of a
    group going to lane j mod 32 of one warp, so the team makes
    ceil(ceil(n_g / c) / 32) warp claims that get work; (5) exactly one
    thread is last."""
    owner, count, last, seq = _map_record(rt, n, G, T, R.SCHED_DYNAMIC, chunk, with_seq=True)
    assert np.all(count == 1)                         # every iteration exactly once
    assert int((last == 1).sum()) == (1 if n else 0)  # exactly one thread is last
    if n:
        assert last[owner[n - 1]] == 1
        order, own = _run_order(owner, seq)
        same_thread = own[1:] == own[:-1]
        assert np.all(np.diff(order)[same_thread] > 0)  # (3) increasing, per thread
    for g in range(G):
        bs, bn = O.static_nochunk(n, G, g)            # level 1 stays static
        blk = owner[bs:bs + bn]
        assert np.all(blk // T == g)                  # iterations stay in the team
        idx = np.arange(bn)
        same = (idx[1:] // chunk) == (idx[:-1] // chunk)   # neighbours in one chunk
        assert np.all(blk[1:][same] == blk[:-1][same])      # each chunk has one owner
        if bn:
            nch = (bn - 1) // chunk + 1
            cown = blk[::chunk]                       # owner of each chunk
            assert cown.size == nch                   # (4) ceil(n_g / c) chunk claims
            j = np.arange(nch)
            assert np.all((cown % T) % 32 == j % 32)  # lane j mod 32 runs chunk j
            warp = (cown % T) // 32
            grp = j // 32
            first = np.r_[True, grp[1:] != grp[:-1]]
            assert np.all(warp == np.repeat(warp[first], np.diff(np.r_[np.flatnonzero(first),
                                                                       nch])))
            assert int(first.sum()) == (nch + 31) // 32   # warp claims with work


@pytest.mark.parametrize("n,G,T", [(1000, 13, 128), (100003, 148, 256), (5000, 3, 1024),
                                   ((1 << 20) + 7, 64, 512)])
@pytest.mark.parametrize("chunk", [1, 16, 256])
def test_guided_claims_in_order_and_shrinking(rt, n, G, T, chunk):
    """schedule(guided) is monotonic too: each thread runs its chunks in
    increasing order, and along the team's block the chunk sizes never grow
    except where the last chunk is cut short by the block's end."""
    owner, count, last, seq = _map_record(rt, n, G, T, R.SCHED_GUIDED, chunk, with_seq=True)
    assert np.all(count == 1)
    order, own = _run_order(owner, seq)
    assert np.all(np.diff(order)[own[1:] == own[:-1]] > 0)
    for g in range(G):
        bs, bn = O.static_nochunk(n, G, g)
        starts = O.guided_chunks(bn, T, chunk)
        sizes = np.diff(np.r_[starts, bn])
        assert np.all(np.diff(sizes[:-1]) <= 0) if sizes.size > 2 else True
        blk = owner[bs:bs + bn]
        for a, e in zip(starts, np.r_[starts[1:], bn]):
            assert np.all(blk[a:e] == blk[a])         # one owner per chunk


@pytest.mark.parametrize("n,G,T", CASES)
@pytest.mark.parametrize("chunk", [1, 7, 64, 256])
def test_nonmonotonic_invariants(rt, n, G, T, chunk):
    """schedule(nonmonotonic: dynamic, c): the same invariants as dynamic
    (every iteration once, whole chunks, chunks in the team, one last), with
    no order required of a thread's chunks."""
    owner, count, last = _map_record(rt, n, G, T, R.SCHED_NONMONOTONIC, chunk)
    assert np.all(count == 1)
    assert int((last == 1).sum()) == (1 if n else 0)
    if n:
        assert last[owner[n - 1]] == 1
    for g in range(G):
        bs, bn = O.static_nochunk(n, G, g)
        blk = owner[bs:bs + bn]
        assert np.all(blk // T == g)
        idx = np.arange(bn)
        same = (idx[1:] // chunk) == (idx[:-1] // chunk)
        assert np.all(blk[1:][same] == blk[:-1][same])
        # a claim is a group of 32 chunks, lane l of the claiming warp runs chunk
        # 32 g + l: the owning lane of chunk j is j mod 32
        if bn:
            j = idx[::chunk] // chunk
            assert np.all((blk[::chunk] % T) % 32 == j % 32)


def test_nonmonotonic_warps_take_their_own_range_first(rt):
    """One team of 8 warps and 8 * 32 groups of chunks, split evenly: a warp
    claims from its own range first, so (unless it was scheduled so late that
    another warp ran through a whole range first) the first group of range w
    goes to warp w.  Required of at least half the warps."""
    T, c = 256, 4
    n = 8 * 32 * 32 * c
    owner, count, last = _map_record(rt, n, 1, T, R.SCHED_NONMONOTONIC, c)
    assert np.all(count == 1)
    ng = n // (32 * c)
    own = sum(int(owner[w * (ng // 8) * 32 * c] // 32 == w) for w in range(T // 32))
    assert own >= 4, own


@pytest.mark.parametrize("n,G,T", CASES)
def test_auto_invariants(rt, n, G, T):
    owner, count, last = _map_record(rt, n, G, T, R.SCHED_AUTO, 0)
    assert np.all(count == 1)
    assert np.all((owner >= 0) & (owner < G * T))
    assert int((last == 1).sum()) == (1 if n else 0)


def test_dynamic_counters_reset_between_launches(rt):
    # a second launch on the same slots must see zeroed counters
    for _ in range(2 * R.SLOTS + 3):
        owner, count, last = _map_record(rt, 4099, 9, 64, R.SCHED_DYNAMIC, 16)
        assert np.all(count == 1)


# -- dist_schedule(static, d) composite ---------------------------------------------

DIST_CASES = [  # n, G, T, d, c  (d = c*T with c % 8 == 0 takes the vector fast path)
    (0, 4, 32, 32, 1), (1, 3, 32, 32, 1), (10000, 7, 32, 32, 1), ((1 << 20) + 5, 148, 256, 256, 1),
    ((1 << 20) + 5, 148, 256, 2048, 8), ((1 << 20), 148, 256, 2048, 8), (100003, 13, 96, 768, 8),
    (100003, 13, 128, 8192, 64), (100003, 5, 64, 1000, 0), (100003, 5, 64, 1000, 3),
    (77777, 9, 1024, 8192, 8), (5000, 200, 32, 256, 8)]


@pytest.mark.parametrize("n,G,T,d,c", DIST_CASES)
def test_dist_owner_map_bit_exact(rt, n, G, T, d, c):
    import torch
    owner = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros((max(n, 1),), dtype=torch.int32, device="cuda")
    last = torch.full((G * T,), -1, dtype=torch.int32, device="cuda")
    desc = R.loop_desc(R.BODY_MAP_RECORD, n=n, x=last, y=count, out=owner, data_type=R.I32)
    rt.launch_region_dist(desc, d, R.SCHED_STATIC_CHUNKED if c else R.SCHED_STATIC, c, G, T)
    assert rt.sync_status() == 0
    own = host(owner)[:n]
    assert np.array_equal(own, O.owner_map_dist(n, G, T, d, c))
    assert np.all(host(count)[:n] == 1)
    lf = host(last)
    assert int((lf == 1).sum()) == (1 if n else 0)
    if n:
        assert lf[own[n - 1]] == 1


@pytest.mark.parametrize("n,G,T,d,c", DIST_CASES)
def test_dist_axpy_and_sum(rt, n, G, T, d, c):
    import torch
    from paper_2106_03219_gb300 import inputs
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    xd, yd = dev(x), dev(y)
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    rt.launch_region_dist(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), d,
                          R.SCHED_STATIC_CHUNKED if c else R.SCHED_STATIC, c, G, T,
                          red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
    ynew = O.axpy_f32(3.0, x, y)
    assert np.array_equal(host(yd).view(np.uint32), ynew.view(np.uint32))
    exact = O.exact_sum_f32(ynew)
    assert abs(float(host(r)[0]) - exact) <= 1e-6 * max(abs(exact), 1e-30)


def test_dist_rejects(rt):
    import torch
    x = torch.zeros(64, device="cuda")
    d = R.loop_desc(R.BODY_AXPY, n=64, x=x, y=x.clone())
    for kw in (dict(dist_chunk=0), dict(dist_chunk=8, sched=R.SCHED_DYNAMIC, chunk=4),
               dict(dist_chunk=8, sched=R.SCHED_AUTO)):
        with pytest.raises(R.OmprtError):
            rt.launch_region_dist(d, teams=2, threads=32, **kw)


# -- schedule(guided, c) --------------------------------------------------------------

GUIDED_CASES = [(0, 3, 32, 1), (1, 1, 32, 1), (1000, 4, 32, 1), (100003, 13, 128, 1),
                (100003, 13, 128, 16), ((1 << 20) + 7, 148, 256, 1), ((1 << 20) + 7, 148, 256, 64),
                (5000, 7, 1024, 3)]


@pytest.mark.parametrize("n,G,T,c", GUIDED_CASES)
def test_guided_partition_bit_exact(rt, n, G, T, c):
    import torch
    owner = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros((max(n, 1),), dtype=torch.int32, device="cuda")
    last = torch.full((G * T,), -1, dtype=torch.int32, device="cuda")
    desc = R.loop_desc(R.BODY_MAP_RECORD, n=n, x=last, y=count, out=owner, data_type=R.I32)
    rt.launch_region(desc, R.SCHED_GUIDED, c, G, T)
    assert rt.sync_status() == 0
    own, cnt, lf = host(owner)[:n], host(count)[:n], host(last)
    assert np.all(cnt == 1)
    assert int((lf == 1).sum()) == (1 if n else 0)
    if n:
        assert lf[own[n - 1]] == 1
    for g in range(G):
        bs, bn = O.static_nochunk(n, G, g)
        blk = own[bs:bs + bn]
        assert np.all(blk // T == g)
        # chunk boundaries = where the owner changes; must be the oracle's starts
        if bn:
            changes = np.flatnonzero(np.diff(blk) != 0) + 1
            starts = np.concatenate([[0], changes])
            assert np.array_equal(starts, O.guided_chunks(bn, T, c)), g


@pytest.mark.parametrize("n,G,T,c", GUIDED_CASES)
def test_guided_axpy_and_dot(rt, n, G, T, c):
    import torch
    from paper_2106_03219_gb300 import inputs
    x, y = inputs.f32_uniform01(n, 0), inputs.f32_uniform01(n, 1)
    xd, yd = dev(x), dev(y)
    rt.launch_region(R.loop_desc(R.BODY_AXPY, n=n, x=xd, y=yd, alpha=3.0), R.SCHED_GUIDED, c, G, T)
    assert np.array_equal(host(yd).view(np.uint32), O.axpy_f32(3.0, x, y).view(np.uint32))
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    xs, ys = dev(x), dev(y)
    rt.launch_region(R.loop_desc(R.BODY_DOT, n=n, x=xs, y=ys), R.SCHED_GUIDED, c, G, T,
                     red=R.ReduceDesc(R.OP_SUM, R.PREC_COMP_F64, r.data_ptr()))
    exact = O.exact_dot_f32(x, y)
    assert abs(float(host(r)[0]) - exact) <= 1e-6 * max(abs(exact), 1e-30)
    assert rt.sync_status() == 0
