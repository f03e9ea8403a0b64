"""Pins for the oracle's trip count and static worksharing (C0-C3).

The oracle's closed forms (q = n / P, r = n % P, ...) are checked against
brute-force enumeration written from the OpenMP schedule rules themselves:
iterations are dealt out one at a time, and user indices are produced by
actually stepping the loop variable with Python integers (no overflow).
The paper places this routine in the runtime (Sec. 1, Sec. 2) without
specifying it; the rules are OpenMP's loop-schedule semantics.
"""
import itertools

import numpy as np
import pytest

import oracle as O

M64 = 1 << 64


def wrap64(v):
    v %= M64
    return v - M64 if v >= (1 << 63) else v


def brute_trip(lb, ub, incr):
    n, v = 0, lb
    while (v <= ub) if incr > 0 else (v >= ub):
        n += 1
        v += incr
        assert n < 10 ** 6
    return n


def brute_nochunk(n, P):
    """Deal iterations round-robin to count each entity's share, then lay the
    shares out contiguously in entity order."""
    counts = [0] * P
    for j in range(n):
        counts[j % P] += 1
    starts = [sum(counts[:k]) for k in range(P)]
    return starts, counts


def brute_pieces(n, P, c):
    """Per entity, its list of pieces [a, e) in logical index space."""
    pieces = [[] for _ in range(P)]
    if c == 0:
        starts, counts = brute_nochunk(n, P)
        for k in range(P):
            if counts[k]:
                pieces[k].append((starts[k], starts[k] + counts[k]))
        return pieces
    i, j = 0, 0
    while i < n:
        pieces[j % P].append((i, min(i + c, n)))
        i += c
        j += 1
    return pieces


# -- C0 ------------------------------------------------------------------------

TYPES = {"i32": (-(1 << 31), (1 << 31) - 1), "u32": (0, (1 << 32) - 1),
         "i64": (-(1 << 63), (1 << 63) - 1), "u64": (0, (1 << 64) - 1)}


@pytest.mark.parametrize("t", list(TYPES))
def test_trip_count_small_ranges(t):
    lo = 0 if t[0] == "u" else -7
    for lb in range(lo, lo + 12):
        for ub in range(lo, lo + 12):
            for incr in (-3, -2, -1, 1, 2, 3, 5):
                assert O.trip_count(lb, ub, incr, t) == brute_trip(lb, ub, incr)


@pytest.mark.parametrize("t", list(TYPES))
def test_trip_count_near_type_limits(t):
    tmin, tmax = TYPES[t]
    for incr in (1, 2, 3, 7):
        for d in range(0, 9):
            assert O.trip_count(tmax - d, tmax, incr, t) == brute_trip(tmax - d, tmax, incr)
            assert O.trip_count(tmin + d, tmin, -incr, t) == brute_trip(tmin + d, tmin, -incr)
    # full-range spans with a large step: the distance must not overflow
    big = (tmax - tmin) // 4 + 1
    assert O.trip_count(tmin, tmax, big, t) == brute_trip(tmin, tmax, big)
    assert O.trip_count(tmax, tmin, -big, t) == brute_trip(tmax, tmin, -big)


def test_trip_count_rejects():
    with pytest.raises(O.OracleError):
        O.trip_count(0, 10, 0, "i64")
    with pytest.raises(O.OracleError):
        O.trip_count(0, 1 << 31, 1, "i32")          # bound outside int32
    with pytest.raises(O.OracleError):
        O.trip_count(-1, 5, 1, "u32")               # bound outside uint32
    with pytest.raises(O.OracleError):
        O.trip_count(0, (1 << 64) - 1, 1, "u64")    # 2^64 iterations


@pytest.mark.parametrize("t", ["i32", "u32"])
def test_trip_count_increment_must_fit_the_index_type(t):
    """A 32-bit loop variable cannot step by an increment its type cannot hold
    (its negation too, for a decreasing loop): |incr| <= 2^31 - 1 is a loop,
    2^31 is rejected either way; the 64-bit types take any non-zero increment."""
    lo, hi = (-(1 << 31), (1 << 31) - 1) if t == "i32" else (0, (1 << 32) - 1)
    for incr in (1 << 31, -(1 << 31), 1 << 40, -(1 << 40)):
        with pytest.raises(O.OracleError):
            O.trip_count(lo if incr > 0 else hi, hi if incr > 0 else lo, incr, t)
    big = (1 << 31) - 1
    assert O.trip_count(lo, hi, big, t) == brute_trip(lo, hi, big)
    assert O.trip_count(hi, lo, -big, t) == brute_trip(hi, lo, -big)
    for t64 in ("i64", "u64"):
        assert O.trip_count(0, 1 << 40, 1 << 31, t64) == brute_trip(0, 1 << 40, 1 << 31)


# -- C1 / C2 -----------------------------------------------------------------------

def test_static_nochunk_vs_dealing():
    for n in range(0, 70):
        for P in range(1, 12):
            starts, counts = brute_nochunk(n, P)
            for k in range(P):
                assert O.static_nochunk(n, P, k) == (starts[k], counts[k])


def test_static_nochunk_invariants_large():
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(0, 1 << 40))
        P = int(rng.integers(1, 5000))
        prev_end, sizes = 0, []
        for k in list(range(min(P, 3))) + [P - 1]:
            s, c = O.static_nochunk(n, P, k)
            sizes.append(c)
        # contiguity of consecutive entities and exact cover at the end
        for k in range(min(P, 50)):
            s, c = O.static_nochunk(n, P, k)
            assert s == prev_end
            prev_end = s + c
        s, c = O.static_nochunk(n, P, P - 1)
        assert s + c == n
        assert max(sizes) - min(sizes) <= 1


def test_worked_example_ten_over_four():
    # 10 iterations over 4 threads: shares 3,3,2,2 in thread order
    assert [O.static_nochunk(10, 4, k) for k in range(4)] == [(0, 3), (3, 3), (6, 2), (8, 2)]
    # chunk 1 reduces to owner(i) = i mod P
    own = O.owner_map(10, 1, 4, chunk=1)
    assert own.tolist() == [i % 4 for i in range(10)]


@pytest.mark.parametrize("t,lb,incr", [("i64", 0, 1), ("i32", -5, 3), ("i64", 100, -7),
                                       ("u32", 4000000000, -2), ("u64", (1 << 64) - 50, 1),
                                       ("i32", (1 << 31) - 40, 1)])
def test_for_static_init_vs_brute(t, lb, incr):
    for n in range(0, 30):
        ub = lb + (n - 1) * incr if n > 0 else lb - incr
        tmin, tmax = TYPES[t]
        if not (tmin <= ub <= tmax):
            continue
        assert O.trip_count(lb, ub, incr, t) == n
        for P in range(1, 7):
            for c in (0, 1, 2, 3, 5):
                pieces = brute_pieces(n, P, c)
                for k in range(P):
                    LB, UB, st, last = O.for_static_init(lb, ub, incr, t, P, k, c)
                    if pieces[k]:
                        a, e = pieces[k][0]
                        assert LB == wrap64(lb + a * incr)
                        assert UB == wrap64(lb + (e - 1) * incr)
                    else:
                        assert LB == wrap64(lb + n * incr)
                        assert UB == wrap64(lb + (n - 1) * incr)
                    if c == 0:
                        assert st == wrap64(n * incr)
                    else:
                        if len(pieces[k]) > 1:
                            assert st == wrap64((pieces[k][1][0] - pieces[k][0][0]) * incr)
                        assert st == wrap64(P * c * incr)
                    owns_last = any(e == n for (_, e) in pieces[k]) and n > 0
                    assert last == int(owns_last)


# -- C3 ------------------------------------------------------------------------

def brute_owner(n, G, T, c):
    owner = [-1] * n
    tstarts, tcounts = brute_nochunk(n, G)
    for g in range(G):
        bs, bn = tstarts[g], tcounts[g]
        for t, plist in enumerate(brute_pieces(bn, T, c)):
            for a, e in plist:
                for i in range(a, e):
                    assert owner[bs + i] == -1
                    owner[bs + i] = g * T + t
    return owner


def test_owner_map_vs_brute():
    for n, G, T, c in itertools.product(range(0, 65, 3), range(1, 6), range(1, 10),
                                        (0, 1, 2, 3, 4, 7, 9)):
        own = O.owner_map(n, G, T, c)
        assert own.tolist() == brute_owner(n, G, T, c)


def test_owner_map_vs_brute_random_larger():
    """Seeded random launches well past the exhaustive range: thousands of
    iterations, hundreds of teams, up to 1024 threads, chunks up to 300
    (many threads and teams end up empty or with a partial last chunk)."""
    rng = np.random.default_rng(11)
    for _ in range(25):
        n = int(rng.integers(0, 10000))
        G = int(rng.integers(1, 300))
        T = int(rng.choice([1, 32, 96, 256, 1024]))
        c = int(rng.choice([0, 1, 2, 7, 64, 300]))
        assert O.owner_map(n, G, T, c).tolist() == brute_owner(n, G, T, c), (n, G, T, c)


@pytest.mark.parametrize("t,lb,incr", [("i64", 3, 2), ("i32", 50, -3), ("u64", 7, 1)])
def test_composite_table_vs_brute(t, lb, incr):
    for n, G, T, c in itertools.product((0, 1, 5, 17, 40), (1, 2, 3, 5), (1, 4, 9),
                                        (0, 1, 3, 8)):
        ub = lb + (n - 1) * incr if n > 0 else lb - incr
        tab = O.composite_table(lb, ub, incr, t, G, T, c)
        tstarts, tcounts = brute_nochunk(n, G)
        for g in range(G):
            bs, bn = tstarts[g], tcounts[g]
            pieces = brute_pieces(bn, T, c)
            for tt in range(T):
                row = tab[g * T + tt]
                # level 1: the team's block
                if bn:
                    assert row[0] == wrap64(lb + bs * incr)
                    assert row[1] == wrap64(lb + (bs + bn - 1) * incr)
                else:
                    assert row[0] == wrap64(lb + n * incr)
                assert row[2] == wrap64(n * incr)
                assert row[3] == int(bn > 0 and bs + bn == n)
                # level 2: the thread's first piece inside the block
                if pieces[tt]:
                    a, e = pieces[tt][0]
                    assert row[4] == wrap64(lb + (bs + a) * incr)
                    assert row[5] == wrap64(lb + (bs + e - 1) * incr)
                else:
                    assert row[4] == wrap64(lb + (bs + bn) * incr)
                    assert row[5] == wrap64(lb + (bs + bn - 1) * incr)
                assert row[6] == wrap64((bn if c == 0 else T * c) * incr)
                assert row[7] == int(any(e == bn for (_, e) in pieces[tt]) and bn > 0)


# -- dist_schedule(static, d) ------------------------------------------------------

def brute_owner_dist(n, G, T, d, c):
    """Deal distribute chunks of d round-robin to teams; inside each, deal
    the threads' pieces as for a loop of that length."""
    owner = [-1] * n
    j = 0
    for bs in range(0, n, d):
        g = j % G
        bn = min(d, n - bs)
        for t, plist in enumerate(brute_pieces(bn, T, c)):
            for a, e in plist:
                for i in range(a, e):
                    assert owner[bs + i] == -1
                    owner[bs + i] = g * T + t
        j += 1
    return owner


def test_owner_map_dist_vs_brute():
    for n, G, T, d, c in itertools.product((0, 1, 7, 40, 97), (1, 2, 3, 5), (1, 3, 8),
                                           (1, 4, 8, 13), (0, 1, 3)):
        assert O.owner_map_dist(n, G, T, d, c).tolist() == brute_owner_dist(n, G, T, d, c)


def test_owner_map_dist_vs_brute_random_larger():
    rng = np.random.default_rng(12)
    for _ in range(20):
        n = int(rng.integers(0, 10000))
        G = int(rng.integers(1, 200))
        T = int(rng.choice([1, 32, 128, 512]))
        d = int(rng.choice([1, T, 8 * T, 1000, 4099]))
        c = int(rng.choice([0, 1, 3, 8, 64]))
        assert O.owner_map_dist(n, G, T, d, c).tolist() == brute_owner_dist(n, G, T, d, c), \
            (n, G, T, d, c)


def test_owner_map_dist_spmd_closed_form():
    # dist_schedule(static, T) with schedule(static, 1): i -> team (i/T) mod G, thread i mod T
    n, G, T = 10000, 7, 32
    own = O.owner_map_dist(n, G, T, T, 1)
    i = np.arange(n)
    assert np.array_equal(own, ((i // T) % G) * T + i % T)
    # one distribute chunk per team covering the whole loop reduces to C3
    assert np.array_equal(O.owner_map_dist(n, 1, T, n, 0), O.owner_map(n, 1, T, 0))


# -- schedule(guided, c) -----------------------------------------------------------

@pytest.mark.parametrize("bn,T,c", [(0, 4, 1), (1, 4, 1), (100, 4, 1), (1000, 8, 3),
                                    (12345, 32, 16), (113359, 256, 1), (7, 100, 5)])
def test_guided_partition_invariants(bn, T, c):
    st = O.guided_chunks(bn, T, c).tolist()
    sizes = [b - a for a, b in zip(st, st[1:] + [bn])]
    assert sum(sizes) == bn
    if bn:
        assert st[0] == 0
        assert sizes[0] == min(bn, max(c, -(-bn // (2 * T))))   # first request sees all of bn
    assert all(s1 >= s2 for s1, s2 in zip(sizes, sizes[1:]))   # never growing
    assert all(s >= c for s in sizes[:-1])                      # only the last may be short
    # each size is what a request would take from the remainder at that point
    r = bn
    for s in sizes:
        assert s == min(r, max(c, -(-r // (2 * T))))
        r -= s


def test_guided_degenerates():
    # with c at least the block, one chunk
    assert O.guided_chunks(500, 4, 500).tolist() == [0]
    # one thread: chunks of ceil(r/2) down to c
    assert O.guided_chunks(16, 1, 1).tolist() == [0, 8, 12, 14, 15]
