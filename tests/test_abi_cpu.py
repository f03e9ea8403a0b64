"""The C-ABI library builds, loads and exports every entry point the header
declares; host-side logic that needs no device is checked against the
oracle.  No compute call is made (no GPU here)."""
import ctypes as C
import os
import re

import pytest

import oracle as O
from paper_2106_03219_gb300 import build_lib
from paper_2106_03219_gb300 import omprt as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build_lib.build()
    return R.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "omprt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(omprt_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("omprt_init", "omprt_finalize", "omprt_launch_region", "omprt_reduce",
                 "omprt_alloc_shared", "omprt_launch_batch", "omprt_sync_status"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert missing == []


def test_status_strings(L):
    assert R.status_str(R.OK) == "ok"
    assert R.status_str(R.ERR_INVALID) == "invalid argument"
    assert R.status_str(999) == "unknown status"


def test_null_context_is_rejected(L):
    d = R.LoopDesc()
    assert L.omprt_launch_region(None, C.byref(d), 0, 0, 1, 32, None, None) == R.ERR_NOT_INIT
    assert L.omprt_reduce(None, 0, R.F32, 0, None, 0, None, 0, 0, None) == R.ERR_NOT_INIT
    assert L.omprt_alloc_shared(None, 16) == R.ERR_NOT_INIT
    assert L.omprt_set_stage_bytes(None, 16) == R.ERR_NOT_INIT
    assert L.omprt_set_stencil_stage_bytes(None, 16) == R.ERR_NOT_INIT
    assert L.omprt_set_stencil_slab_shape(None, 0, 0) == R.ERR_NOT_INIT
    assert L.omprt_set_launch_overlap(None, 1) == R.ERR_NOT_INIT
    assert L.omprt_launch_generic(None, None, 0, C.byref(d), 0, None, 0, 0, None) == \
        R.ERR_NOT_INIT
    assert L.omprt_finalize(None) == R.ERR_NOT_INIT
    assert L.omprt_sm_count(None) == 0


def test_learned_config_table(L):
    cfgs = R.learned_configs()
    assert len(cfgs) == 12
    assert len(set(cfgs)) == 12
    for sched, chunk, tps, thr in cfgs:
        assert sched in (R.SCHED_STATIC, R.SCHED_STATIC_CHUNKED, R.SCHED_DYNAMIC, R.SCHED_AUTO)
        assert tps in (1, 4) and thr in (256, 1024)


TYPES = {"i32": (-(1 << 31), (1 << 31) - 1), "u32": (0, (1 << 32) - 1),
         "i64": (-(1 << 63), (1 << 63) - 1), "u64": (0, (1 << 64) - 1)}


@pytest.mark.parametrize("t", list(TYPES))
def test_host_trip_count_matches_oracle(L, t):
    tmin, tmax = TYPES[t]
    cases = []
    lo = 0 if t[0] == "u" else -5
    for lb in range(lo, lo + 9):
        for ub in range(lo, lo + 9):
            for incr in (-3, -1, 1, 2, 5):
                cases.append((lb, ub, incr))
    for incr in (1, 3, 1 << 20):
        cases += [(tmax - 10, tmax, incr), (tmin + 10, tmin, -incr), (tmin, tmax, incr * 97)]
    # increments at and past what a 32-bit index type holds
    for incr in ((1 << 31) - 1, 1 << 31, 1 << 40):
        cases += [(tmin, tmax, incr), (tmax, tmin, -incr)]
    for lb, ub, incr in cases:
        d = R.loop_desc(R.BODY_NONE, lb=lb, ub=ub, incr=incr, idx_type=R.TYPE_CODES[t],
                        data_type=R.F32)
        try:
            ref = O.trip_count(lb, ub, incr, t)
        except O.OracleError:
            ref = None
        if ref is None or ref >= (1 << 63):
            with pytest.raises(R.OmprtError):
                R.loop_trip_count(d)
        else:
            assert R.loop_trip_count(d) == ref, (lb, ub, incr)


def test_host_trip_count_rejects(L):
    for lb, ub, incr, t in [(0, 5, 0, R.I64), (0, 1 << 31, 1, R.I32), (-1, 4, 1, R.U32),
                            (0, 4, 1 << 31, R.I32)]:
        d = R.loop_desc(R.BODY_NONE, lb=lb, ub=ub, incr=incr, idx_type=t, data_type=R.F32)
        with pytest.raises(R.OmprtError):
            R.loop_trip_count(d)


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without the built library every call raises a clear error."""
    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R, "lib_path", lambda: "/nonexistent/libomprt.so")
    with pytest.raises(R.LibraryMissing, match="libomprt.so missing"):
        R.lib()
    with pytest.raises(R.LibraryMissing):
        R.Runtime(0)
