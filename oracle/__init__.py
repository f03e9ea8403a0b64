"""CPU oracle for the OpenMP device-runtime hot path (TEST INFRASTRUCTURE).

Only tests/, the smoke check and bench.py's CPU-baseline leg use this
package.  It wraps oracle/omp_oracle.c (built with gcc on first use) through
ctypes and adds nothing of the method's arithmetic itself: every function here
marshals numpy arrays and forwards to the C routine that states the reading
of the paper it follows.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

I32, U32, I64, U64 = 0, 1, 2, 3
TYPE_NAMES = {"i32": I32, "u32": U32, "i64": I64, "u64": U64}


def lib():
    """The built oracle.  OMPRT_ORACLE_LIB names another build of the same
    source to load instead: the mutation tests load copies with one planted
    mistake each and check that the pins fail on them."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("OMPRT_ORACLE_LIB") or _build.build())
        _declare(_lib)
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _declare(L):
    i64, u64, i32, dbl, vp = C.c_int64, C.c_uint64, C.c_int, C.c_double, C.c_void_p
    sig = {
        "orc_trip_count": (i32, [i64, i64, i64, i32, C.POINTER(u64)]),
        "orc_static_nochunk": (None, [u64, u64, u64, C.POINTER(u64), C.POINTER(u64)]),
        "orc_for_static_init": (i32, [i64, i64, i64, i32, u64, u64, u64, C.POINTER(i64),
                                      C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]),
        "orc_composite_table": (i32, [i64, i64, i64, i32, u64, u64, u64, vp]),
        "orc_owner_map": (i32, [u64, u64, u64, u64, vp]),
        "orc_owner_map_dist": (i32, [u64, u64, u64, u64, u64, vp]),
        "orc_guided_chunks": (u64, [u64, u64, u64, vp, u64]),
        "orc_axpy_i32": (None, [u64, C.c_int32, vp, vp]),
        "orc_axpy_f32": (None, [u64, C.c_float, vp, vp]),
        "orc_stencil1d3_f32": (None, [u64, C.c_float, C.c_float, vp, vp]),
        "orc_stencil2d5_f32": (None, [u64, u64, C.c_float, C.c_float, vp, vp]),
        "orc_sum_i64": (i64, [u64, vp]),
        "orc_sum_i32": (i64, [u64, vp]),
        "orc_max_f32": (dbl, [u64, vp]),
        "orc_min_f32": (dbl, [u64, vp]),
        "orc_max_i64": (i64, [u64, vp]),
        "orc_min_i64": (i64, [u64, vp]),
        "orc_max_i32": (i64, [u64, vp]),
        "orc_min_i32": (i64, [u64, vp]),
        "orc_exact_sum_f32": (dbl, [u64, vp]),
        "orc_exact_sum_bf16": (dbl, [u64, vp]),
        "orc_exact_dot_f32": (dbl, [u64, vp, vp]),
        "orc_exact_sum_f64": (dbl, [u64, vp]),
        "orc_exact_abs_sum_f32": (dbl, [u64, vp]),
        "orc_plain_sum_f32": (dbl, [u64, vp]),
        "orc_exact_sum_f32_terms": (i32, [u64, vp, vp, i32]),
        "orc_exact_sum_bf16_terms": (i32, [u64, vp, vp, i32]),
        "orc_atomic_inc": (C.c_uint32, [C.POINTER(C.c_uint32), C.c_uint32]),
        "orc_stack_replay": (i64, [u64, u64, u64, vp, vp]),
        "orc_mlp_nparam": (i32, []),
        "orc_mlp_forward": (None, [vp, u64, vp, vp]),
        "orc_mlp_loss_grad": (dbl, [vp, u64, vp, vp, vp]),
        "orc_adam_step": (None, [u64, vp, vp, vp, vp, u64, dbl, dbl, dbl, dbl]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


class OracleError(ValueError):
    pass


def _t(t):
    return TYPE_NAMES[t] if isinstance(t, str) else int(t)


def _as_i64(v):
    """A bound or increment as a signed 64-bit pattern (u64 values wrap)."""
    v = int(v)
    return v - (1 << 64) if v >= (1 << 63) else v


# -- C0..C3: trip count and static worksharing -------------------------------

def trip_count(lb, ub, incr, idx_type="i64"):
    n = C.c_uint64()
    rc = lib().orc_trip_count(_as_i64(lb), _as_i64(ub), _as_i64(incr), _t(idx_type), C.byref(n))
    if rc:
        raise OracleError("invalid loop")
    return n.value


def static_nochunk(n, P, k):
    s, c = C.c_uint64(), C.c_uint64()
    lib().orc_static_nochunk(n, P, k, C.byref(s), C.byref(c))
    return s.value, c.value


def for_static_init(lb, ub, incr, idx_type, P, k, chunk=0):
    LB, UB, st, last = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int()
    rc = lib().orc_for_static_init(_as_i64(lb), _as_i64(ub), _as_i64(incr), _t(idx_type),
                                   P, k, chunk, C.byref(LB), C.byref(UB), C.byref(st),
                                   C.byref(last))
    if rc:
        raise OracleError("invalid loop")
    return LB.value, UB.value, st.value, last.value


def composite_table(lb, ub, incr, idx_type, G, T, chunk=0):
    out = np.zeros((G * T, 8), dtype=np.int64)
    rc = lib().orc_composite_table(_as_i64(lb), _as_i64(ub), _as_i64(incr), _t(idx_type),
                                   G, T, chunk, _p(out))
    if rc:
        raise OracleError("invalid loop")
    return out


def owner_map(n, G, T, chunk=0):
    out = np.full(n, -1, dtype=np.int32)
    if lib().orc_owner_map(n, G, T, chunk, _p(out)):
        raise OracleError("invalid")
    return out


def owner_map_dist(n, G, T, dist_chunk, chunk=0):
    out = np.full(n, -1, dtype=np.int32)
    if lib().orc_owner_map_dist(n, G, T, dist_chunk, chunk, _p(out)):
        raise OracleError("invalid")
    return out


def guided_chunks(bn, T, chunk):
    """Chunk starts, in hand-out order, of schedule(guided, chunk) over bn."""
    k = lib().orc_guided_chunks(bn, T, chunk, None, 0)
    out = np.zeros(max(k, 1), dtype=np.uint64)
    lib().orc_guided_chunks(bn, T, chunk, _p(out), k)
    return out[:k].astype(np.int64)


# -- C6: bodies ----------------------------------------------------------------

def axpy_i32(alpha, x, y):
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.array(y, dtype=np.int32, copy=True)
    lib().orc_axpy_i32(x.size, int(alpha), _p(x), _p(y))
    return y


def axpy_f32(alpha, x, y):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.array(y, dtype=np.float32, copy=True)
    lib().orc_axpy_f32(x.size, float(alpha), _p(x), _p(y))
    return y


STENCIL_C0 = 0.5
STENCIL_C1 = 0.125


def stencil1d3(a, c0=STENCIL_C0, c1=STENCIL_C1):
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty_like(a)
    lib().orc_stencil1d3_f32(a.size, c0, c1, _p(a), _p(out))
    return out


def stencil2d5(a, c0=STENCIL_C0, c1=STENCIL_C1):
    a = np.ascontiguousarray(a, dtype=np.float32)
    ny, nx = a.shape
    out = np.empty_like(a)
    lib().orc_stencil2d5_f32(nx, ny, c0, c1, _p(a), _p(out))
    return out


# -- C7: reductions ------------------------------------------------------------

def sum_int(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.int32:
        return lib().orc_sum_i32(a.size, _p(a))
    a = a.astype(np.int64, copy=False)
    return lib().orc_sum_i64(a.size, _p(a))


def max_min(a, op):
    a = np.ascontiguousarray(a)
    name = {np.dtype(np.float32): "f32", np.dtype(np.int64): "i64",
            np.dtype(np.int32): "i32"}[a.dtype]
    return getattr(lib(), "orc_%s_%s" % (op, name))(a.size, _p(a))


def exact_sum_f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return lib().orc_exact_sum_f32(a.size, _p(a))


def exact_sum_bf16(bits):
    """bits: uint16 array holding bf16 patterns."""
    a = np.ascontiguousarray(bits, dtype=np.uint16)
    return lib().orc_exact_sum_bf16(a.size, _p(a))


def exact_dot_f32(x, y):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    return lib().orc_exact_dot_f32(x.size, _p(x), _p(y))


def exact_sum_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_exact_sum_f64(a.size, _p(a))


def exact_abs_sum_f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return lib().orc_exact_abs_sum_f32(a.size, _p(a))


def exact_sum_terms(a, bf16=False, cap=16):
    """The exact sum of a (fp32 values, or bf16 patterns when bf16) as a
    non-overlapping expansion of doubles, largest first."""
    out = np.zeros(cap)
    if bf16:
        a = np.ascontiguousarray(a, dtype=np.uint16)
        k = lib().orc_exact_sum_bf16_terms(a.size, _p(a), _p(out), cap)
    else:
        a = np.ascontiguousarray(a, dtype=np.float32)
        k = lib().orc_exact_sum_f32_terms(a.size, _p(a), _p(out), cap)
    if k > cap:
        raise OracleError("expansion longer than %d terms" % cap)
    return out[:k].copy()


def plain_sum_f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return lib().orc_plain_sum_f32(a.size, _p(a))


# -- C8: atomic inc ------------------------------------------------------------

def atomic_inc_sequence(x0, e, k):
    """Apply inc(x, e) k times sequentially; return (returned values, final x)."""
    x = C.c_uint32(x0)
    vals = [lib().orc_atomic_inc(C.byref(x), e) for _ in range(k)]
    return vals, x.value


# -- C10: shared-memory stack ----------------------------------------------------

def stack_replay(S, Q, ops):
    """ops: int64 array [nops, 2] of (kind, arg).  Returns (out [nops,2], status)."""
    ops = np.ascontiguousarray(ops, dtype=np.int64).reshape(-1, 2)
    out = np.zeros_like(ops)
    st = lib().orc_stack_replay(S, Q, ops.shape[0], _p(ops), _p(out))
    return out, st


# -- C12: MLP --------------------------------------------------------------------

def mlp_nparam():
    return lib().orc_mlp_nparam()


def mlp_forward(p, X):
    p = np.ascontiguousarray(p, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.zeros((X.shape[0], 12))
    lib().orc_mlp_forward(_p(p), X.shape[0], _p(X), _p(Y))
    return Y


def mlp_loss_grad(p, X, Yt):
    p = np.ascontiguousarray(p, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Yt = np.ascontiguousarray(Yt, dtype=np.float64)
    g = np.zeros_like(p)
    loss = lib().orc_mlp_loss_grad(_p(p), X.shape[0], _p(X), _p(Yt), _p(g))
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays p, m, v."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam_step(p.size, _p(p), _p(g), _p(m), _p(v), t, lr, b1, b2, eps)
