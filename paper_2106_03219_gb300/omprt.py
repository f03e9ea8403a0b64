"""Python binding of libomprt.so (argument marshalling only).

Every function here forwards to the C entry point of the same name declared
in include/omprt.h; all loop, reduction, dispatch and stack work runs in the
library's CUDA kernels.  Torch tensors supply device memory and the current
CUDA stream.  There is no fallback: if the library is missing or a call
fails, an OmprtError is raised.
"""
import ctypes as C
import os

from . import build_lib

# -- enums (mirrors of include/omprt.h) ----------------------------------------
OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_NOT_INIT, ERR_DEVICE = \
    range(8)
DEV_STACK_NOMEM, DEV_STACK_ORDER, DEV_TIMEOUT, DEV_BAD_ARG = 0x1, 0x2, 0x4, 0x8
SCHED_STATIC, SCHED_STATIC_CHUNKED, SCHED_DYNAMIC, SCHED_AUTO, SCHED_LEARNED, SCHED_GUIDED, \
    SCHED_NONMONOTONIC = range(7)
I32, U32, I64, U64, F32, BF16, F64 = range(7)
OP_SUM, OP_MAX, OP_MIN = range(3)
PREC_COMP_F64, PREC_COMP_F32, PREC_NAIVE_F32 = range(3)
BODY_MAP_RECORD, BODY_AXPY, BODY_STENCIL1D3, BODY_STENCIL2D5, BODY_DOT, BODY_NONE = range(6)
SLOTS = 64
MAX_RED_TEAMS = 16384
POOL_BYTES_PER_TEAM = 4096
MLP_IN, MLP_HID, MLP_OUT, MLP_NPARAM = 16, 64, 12, 6028
NOALLOC_MAX_TEAMS = 4096
GENERIC_REDUCE, GENERIC_DOT_AXPY = 0, 1

TYPE_CODES = {"i32": I32, "u32": U32, "i64": I64, "u64": U64}


class OmprtError(RuntimeError):
    """A non-OK omprt_status from the library; .status holds the code."""
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_str(status), status))


class LibraryMissing(RuntimeError):
    """libomprt.so has not been built: there is no fallback."""


class LoopDesc(C.Structure):
    """omprt_loop_desc (include/omprt.h): loop bounds, index type, body, data pointers."""
    _fields_ = [("lb", C.c_int64), ("ub", C.c_int64), ("incr", C.c_int64),
                ("idx_type", C.c_int32), ("body", C.c_int32), ("data_type", C.c_int32),
                ("reserved", C.c_int32), ("x", C.c_void_p), ("y", C.c_void_p),
                ("out", C.c_void_p), ("alpha", C.c_double), ("c0", C.c_double),
                ("c1", C.c_double), ("nx", C.c_int64), ("ny", C.c_int64),
                ("seq", C.c_void_p)]


class ReduceDesc(C.Structure):
    """omprt_reduce_desc: reduction op, precision and the device result pointer."""
    _fields_ = [("op", C.c_int32), ("precision", C.c_int32), ("result_dev", C.c_void_p)]


_lib = None


def _declare(L):
    vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
    st = C.c_int
    sig = {
        "omprt_init": (st, [C.c_int, C.POINTER(vp)]),
        "omprt_finalize": (st, [vp]),
        "omprt_alloc_shared": (st, [vp, C.c_size_t]),
        "omprt_set_stage_bytes": (st, [vp, i64]),
        "omprt_set_stencil_stage_bytes": (st, [vp, i64]),
        "omprt_set_stencil_slab_shape": (st, [vp, i32, i32]),
        "omprt_set_launch_overlap": (st, [vp, i32]),
        "omprt_launch_region": (st, [vp, C.POINTER(LoopDesc), i32, i64, i32, i32,
                                     C.POINTER(ReduceDesc), vp]),
        "omprt_launch_region_dist": (st, [vp, C.POINTER(LoopDesc), i64, i32, i64, i32, i32,
                                          C.POINTER(ReduceDesc), vp]),
        "omprt_launch_generic": (st, [vp, vp, i64, C.POINTER(LoopDesc), i32, vp, i32, i32, vp]),
        "omprt_reduce": (st, [vp, i32, i32, i32, vp, i64, vp, i32, i32, vp]),
        "omprt_reduce_noalloc": (st, [i32, i32, i32, vp, i64, vp, i32, i32, vp]),
        "omprt_static_init_table": (st, [vp, C.POINTER(LoopDesc), i64, i32, i32, vp, vp]),
        "omprt_sync_status": (st, [vp, vp, C.POINTER(u32)]),
        "omprt_loop_trip_count": (st, [C.POINTER(LoopDesc), C.POINTER(C.c_uint64)]),
        "omprt_status_str": (C.c_char_p, [st]),
        "omprt_sm_count": (i32, [vp]),
        "omprt_batch_create": (st, [vp, C.POINTER(LoopDesc), C.POINTER(ReduceDesc), i32, i64,
                                    C.POINTER(vp)]),
        "omprt_launch_batch": (st, [vp, i32, i32, vp]),
        "omprt_batch_destroy": (st, [vp]),
        "omprt_batch_items": (i64, [vp]),
        "omprt_test_atomics": (st, [vp, i32, i32, i32, u32, vp, vp, vp]),
        "omprt_test_barrier": (st, [vp, i32, i32, i32, i32, vp, vp]),
        "omprt_test_stack": (st, [vp, i32, i64, i64, vp, i64, vp, vp, vp]),
        "omprt_test_wait": (st, [vp, i32, vp, u32, i64, vp, vp]),
        "omprt_mlp_forward": (st, [vp, vp, vp, i32, vp, vp]),
        "omprt_mlp_loss_grad": (st, [vp, vp, vp, vp, i32, vp, vp, vp]),
        "omprt_mlp_adam": (st, [vp, vp, vp, vp, vp, i32, i32, C.c_float, C.c_float, C.c_float,
                                C.c_float, vp]),
        "omprt_learned_configs": (st, [vp, vp, vp, vp]),
        "omprt_set_cost_model": (st, [vp, vp, vp, vp]),
        "omprt_loop_features": (st, [vp, C.POINTER(LoopDesc), i32, vp]),
        "omprt_choose_config": (st, [vp, C.POINTER(LoopDesc), i32, C.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def lib_path():
    """Path of the in-tree libomprt.so that lib() loads."""
    return build_lib.LIB


def lib():
    """The loaded library.  Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise LibraryMissing("libomprt.so missing at %s; run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def loop_trip_count(desc):
    """Trip count of a loop descriptor, computed by the library on the host."""
    n = C.c_uint64()
    check(lib().omprt_loop_trip_count(C.byref(desc), C.byref(n)), "omprt_loop_trip_count")
    return n.value


def status_str(s):
    """omprt_status_str: the library's text for a status code."""
    try:
        return lib().omprt_status_str(s).decode()
    except OmprtError:
        return "status %d" % s


def check(status, what="omprt"):
    """Raise OmprtError unless status is OMPRT_OK."""
    if status != OK:
        raise OmprtError(status, what)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype_code(t):
    import torch
    return {torch.float32: F32, torch.bfloat16: BF16, torch.int32: I32, torch.int64: I64,
            torch.int16: BF16, torch.uint16: BF16}[t.dtype]


def loop_desc(body, n=None, x=None, y=None, out=None, *, lb=0, ub=None, incr=1, idx_type=I64,
              data_type=None, alpha=3.0, c0=0.5, c1=0.125, nx=0, ny=0, seq=None):
    """Build an omprt_loop_desc.  Give either n (then lb=0, incr=1) or lb/ub/incr.
    seq (map record only): int32 device tensor of per-iteration ordinals."""
    if ub is None:
        ub = lb + (n - 1) * incr
    if data_type is None:
        ref = x if x is not None else (y if y is not None else out)
        data_type = _dtype_code(ref) if ref is not None else I32
    ub_i = int(ub)
    lb_i = int(lb)
    to64 = lambda v: v - (1 << 64) if v >= (1 << 63) else v
    d = LoopDesc(to64(lb_i), to64(ub_i), int(incr), int(idx_type), int(body), int(data_type), 0,
                 None if x is None else x.data_ptr(), None if y is None else y.data_ptr(),
                 None if out is None else out.data_ptr(), float(alpha), float(c0), float(c1),
                 int(nx), int(ny), None if seq is None else seq.data_ptr())
    # the descriptor holds raw device pointers: keep the tensors alive with it
    d._keep = (x, y, out, seq)
    return d


class Runtime:
    """An omprt context on one CUDA device."""

    def __init__(self, device=0):
        ctx = C.c_void_p()
        check(lib().omprt_init(int(device), C.byref(ctx)), "omprt_init")
        self.ctx = ctx
        self.device = device

    def close(self):
        """omprt_finalize: free the context (streams must be synchronised)."""
        if self.ctx:
            check(lib().omprt_finalize(self.ctx), "omprt_finalize")
            self.ctx = None

    def __del__(self):
        try:
            if self.ctx:
                lib().omprt_finalize(self.ctx)
        except Exception:
            pass

    @property
    def sm_count(self):
        """omprt_sm_count: SMs of the context's device."""
        return lib().omprt_sm_count(self.ctx)

    def alloc_shared(self, nbytes):
        """omprt_alloc_shared: per-team shared-memory stack capacity for later launches."""
        check(lib().omprt_alloc_shared(self.ctx, int(nbytes)), "omprt_alloc_shared")

    def set_stage_bytes(self, nbytes):
        """Per-team shared memory for staged dynamic schedules (0: plain form)."""
        check(lib().omprt_set_stage_bytes(self.ctx, int(nbytes)), "omprt_set_stage_bytes")

    def set_stencil_slab_shape(self, slab_floats=0, buffers=0):
        """omprt_set_stencil_slab_shape: floats a slab line (16 / 32) and slabs a
        warp (2 .. 4) of the 2-D stencil's slab form; 0 the default."""
        check(lib().omprt_set_stencil_slab_shape(self.ctx, int(slab_floats), int(buffers)),
              "omprt_set_stencil_slab_shape")

    def set_launch_overlap(self, on=True):
        """omprt_set_launch_overlap: launch regions so that each may start while
        the kernel before it on the stream drains (True, the default) or as
        plain launches (False)."""
        check(lib().omprt_set_launch_overlap(self.ctx, 1 if on else 0), "omprt_set_launch_overlap")

    def set_stencil_stage_bytes(self, nbytes):
        """omprt_set_stencil_stage_bytes: per-CTA shared memory for the staged 2-D
        stencil windows under static / static(c) / dynamic(c) (0: off)."""
        check(lib().omprt_set_stencil_stage_bytes(self.ctx, int(nbytes)),
              "omprt_set_stencil_stage_bytes")

    def launch_region(self, desc, sched=SCHED_STATIC, chunk=0, teams=0, threads=0, red=None,
                      stream=None):
        """omprt_launch_region: run desc's loop under sched / chunk on teams x threads
        (0: defaults); red (ReduceDesc) adds a reduction.  Asynchronous on stream."""
        rd = None if red is None else C.byref(red)
        check(lib().omprt_launch_region(self.ctx, C.byref(desc), int(sched), int(chunk),
                                        int(teams), int(threads), rd, _stream(stream)),
              "omprt_launch_region")

    def launch_region_dist(self, desc, dist_chunk, sched=SCHED_STATIC, chunk=0, teams=0,
                           threads=0, red=None, stream=None):
        """omprt_launch_region_dist: dist_schedule(static, dist_chunk) at the team
        level, sched / chunk inside each distribute chunk."""
        rd = None if red is None else C.byref(red)
        check(lib().omprt_launch_region_dist(self.ctx, C.byref(desc), int(dist_chunk), int(sched),
                                             int(chunk), int(teams), int(threads), rd,
                                             _stream(stream)), "omprt_launch_region_dist")

    def launch_generic(self, seg, desc, result, teams=0, threads=0, stream=None,
                       program=GENERIC_REDUCE):
        """omprt_launch_generic: generic-mode regions over segments.  seg: int64
        device tensor of nseg + 1 offsets; result: float64[nseg] (GENERIC_REDUCE)
        or float64[3 * nseg] (GENERIC_DOT_AXPY: v, a, w per segment)."""
        nseg = max(int(seg.numel()) - 1, 0)
        check(lib().omprt_launch_generic(self.ctx, _ptr(seg), nseg, C.byref(desc), int(program),
                                         _ptr(result), int(teams), int(threads),
                                         _stream(stream)), "omprt_launch_generic")

    def reduce(self, op, data, result, precision=PREC_COMP_F64, teams=0, threads=0, dtype=None,
               stream=None):
        """omprt_reduce: reduction(op) over the device tensor data into result
        (float64[1] for fp32 / bf16 data, int64[1] for integers)."""
        dt = _dtype_code(data) if dtype is None else dtype
        check(lib().omprt_reduce(self.ctx, int(op), int(dt), int(precision), _ptr(data),
                                 int(data.numel()), _ptr(result), int(teams), int(threads),
                                 _stream(stream)), "omprt_reduce")

    def static_init_table(self, desc, chunk, teams, threads, table, stream=None):
        """omprt_static_init_table: table (int64 device tensor [G*T][8]) gets every
        thread's static worksharing tuple."""
        check(lib().omprt_static_init_table(self.ctx, C.byref(desc), int(chunk), int(teams),
                                            int(threads), _ptr(table), _stream(stream)),
              "omprt_static_init_table")

    def sync_status(self, stream=None):
        """Synchronise and return the device status bits (cleared)."""
        bits = C.c_uint32(0)
        s = lib().omprt_sync_status(self.ctx, _stream(stream), C.byref(bits))
        if s not in (OK, ERR_DEVICE):
            raise OmprtError(s, "omprt_sync_status")
        return bits.value

    # -- self-tests -------------------------------------------------------
    def test_atomics(self, teams, threads, reps, e, words, returned=None, stream=None):
        """omprt_test_atomics: device self-test of the runtime atomics (tensors on device)."""
        check(lib().omprt_test_atomics(self.ctx, teams, threads, reps, e, _ptr(words),
                                       _ptr(returned), _stream(stream)), "omprt_test_atomics")

    def test_barrier(self, teams, threads, sub, rounds, errors, stream=None):
        """omprt_test_barrier: device self-test of team and sub-team barriers."""
        check(lib().omprt_test_barrier(self.ctx, teams, threads, sub, rounds, _ptr(errors),
                                       _stream(stream)), "omprt_test_barrier")

    def test_wait(self, teams, flag, expect, timeout_us, out, stream=None):
        """omprt_test_wait: bounded device wait on flag (device tensor); out[g] = seen."""
        check(lib().omprt_test_wait(self.ctx, teams, _ptr(flag), int(expect), int(timeout_us),
                                    _ptr(out), _stream(stream)), "omprt_test_wait")

    def test_stack(self, teams, stack_bytes, pool_bytes, ops, out, status, stream=None):
        """omprt_test_stack: replay an alloc/free trace on the team stack (device tensors)."""
        nops = ops.shape[0] if ops is not None else 0
        check(lib().omprt_test_stack(self.ctx, teams, int(stack_bytes), int(pool_bytes),
                                     _ptr(ops), nops, _ptr(out), _ptr(status), _stream(stream)),
              "omprt_test_stack")

    # -- batch ----------------------------------------------------------------
    def batch_create(self, descs, reds=None, chunk_elems=0):
        """omprt_batch_create: a persistent batch of regions; returns a Batch."""
        n = len(descs)
        arr = (LoopDesc * n)(*descs)
        rarr = None if reds is None else (ReduceDesc * n)(*reds)
        b = C.c_void_p()
        check(lib().omprt_batch_create(self.ctx, arr, rarr, n, int(chunk_elems), C.byref(b)),
              "omprt_batch_create")
        return Batch(b)

    # -- MLP --------------------------------------------------------------------
    def mlp_forward(self, params, x, y, stream=None):
        """omprt_mlp_forward: y[B][12] = model(x[B][16]) (device tensors)."""
        check(lib().omprt_mlp_forward(self.ctx, _ptr(params), _ptr(x), int(x.shape[0]), _ptr(y),
                                      _stream(stream)), "omprt_mlp_forward")

    def mlp_loss_grad(self, params, x, target, grad, loss=None, stream=None):
        """omprt_mlp_loss_grad: grad = d loss / d params; loss[1] if given (device tensors)."""
        check(lib().omprt_mlp_loss_grad(self.ctx, _ptr(params), _ptr(x), _ptr(target),
                                        int(x.shape[0]), _ptr(grad), _ptr(loss),
                                        _stream(stream)), "omprt_mlp_loss_grad")

    def mlp_adam(self, params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                 stream=None):
        """omprt_mlp_adam: one bias-corrected Adam step on params (device tensors)."""
        check(lib().omprt_mlp_adam(self.ctx, _ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                                   int(params.numel()), int(t), lr, beta1, beta2, eps,
                                   _stream(stream)), "omprt_mlp_adam")

    def set_cost_model(self, params=None, mean=None, std=None):
        """params/mean/std: host float32 numpy arrays, or None to remove."""
        if params is None:
            check(lib().omprt_set_cost_model(self.ctx, None, None, None))
            return
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(std, dtype=np.float32)
        check(lib().omprt_set_cost_model(self.ctx, p.ctypes.data, m.ctypes.data, s.ctypes.data),
              "omprt_set_cost_model")

    def loop_features(self, desc, has_reduction):
        """omprt_loop_features: the 16 features the cost model sees (numpy float32)."""
        import numpy as np
        f = np.zeros(MLP_IN, dtype=np.float32)
        check(lib().omprt_loop_features(self.ctx, C.byref(desc), int(bool(has_reduction)),
                                        f.ctypes.data), "omprt_loop_features")
        return f

    def choose_config(self, desc, has_reduction):
        """omprt_choose_config: the configuration index the model (or heuristic) picks."""
        k = C.c_int32()
        check(lib().omprt_choose_config(self.ctx, C.byref(desc), int(bool(has_reduction)),
                                        C.byref(k)), "omprt_choose_config")
        return k.value


class Batch:
    """A batch handle from Runtime.batch_create (omprt_batch)."""
    def __init__(self, handle):
        self.handle = handle

    @property
    def items(self):
        """omprt_batch_items: work items (chunks) in the batch."""
        return lib().omprt_batch_items(self.handle)

    def launch(self, num_ctas=0, threads=0, stream=None):
        """omprt_launch_batch: run every region in one persistent launch."""
        check(lib().omprt_launch_batch(self.handle, int(num_ctas), int(threads), _stream(stream)),
              "omprt_launch_batch")

    def destroy(self):
        """omprt_batch_destroy: free the batch (streams must be synchronised)."""
        if self.handle:
            check(lib().omprt_batch_destroy(self.handle), "omprt_batch_destroy")
            self.handle = None


def reduce_noalloc(op, data, result, precision=PREC_COMP_F64, teams=0, threads=0, dtype=None,
                   stream=None):
    """omprt_reduce_noalloc: the reduction of Runtime.reduce with its scratch in
    a fixed array inside the library; needs no context and allocates nothing."""
    dt = _dtype_code(data) if dtype is None else dtype
    check(lib().omprt_reduce_noalloc(int(op), int(dt), int(precision), _ptr(data),
                                     int(data.numel()), _ptr(result), int(teams), int(threads),
                                     _stream(stream)), "omprt_reduce_noalloc")


def learned_configs():
    """The 12 learned-schedule configurations: list of (sched, chunk, teams_per_sm, threads)."""
    import numpy as np
    s = np.zeros(12, np.int32)
    c = np.zeros(12, np.int64)
    t = np.zeros(12, np.int32)
    h = np.zeros(12, np.int32)
    check(lib().omprt_learned_configs(s.ctypes.data, c.ctypes.data, t.ctypes.data, h.ctypes.data))
    return [(int(s[k]), int(c[k]), int(t[k]), int(h[k])) for k in range(12)]
