// The C ABI (include/omprt.h): context, argument validation, schedule
// resolution and kernel dispatch.  Host code only; every step of the loop
// itself runs in the executor kernels.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "api_internal.h"

using namespace rt;

namespace {

constexpr size_t kTicketBytes = 256;
constexpr size_t kPartialBytes = 16ull * OMPRT_MAX_RED_TEAMS;
constexpr size_t kDynBytes = 8ull * OMPRT_MAX_RED_TEAMS;
constexpr size_t kSlotBytes = kTicketBytes + kPartialBytes + kDynBytes;
constexpr uint32_t kMaxStackBytes = 200u * 1024u;
// shared memory per CTA for the staged 2-D stencil windows (two windows)
constexpr uint32_t kStencilStageDefault = 226u * 1024u;

bool is_int_type(int32_t t) { return t >= OMPRT_I32 && t <= OMPRT_U64; }

}  // namespace

DeviceGuard::DeviceGuard(int dev) {
  if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
    if (cudaSetDevice(dev) == cudaSuccess) changed = true;
  }
}
DeviceGuard::~DeviceGuard() {
  if (changed) cudaSetDevice(prev);
}

ScratchSlot ctx_next_slot(omprt_ctx* ctx) {
  const uint32_t s = ctx->next_slot.fetch_add(1) % OMPRT_SLOTS;
  unsigned char* base = ctx->slots_dev + (size_t)s * kSlotBytes;
  ScratchSlot r;
  r.ticket = (uint32_t*)base;
  r.partials = base + kTicketBytes;
  r.dyn_next = (unsigned long long*)(base + kTicketBytes + kPartialBytes);
  return r;
}

// C0 of the loop semantics: trip count in the loop variable's type; bounds
// compare in its signedness, the distance in unsigned 64-bit arithmetic.
omprt_status loop_trip_count(const omprt_loop_desc* d, uint64_t* n, int64_t* wide_lb) {
  const int32_t t = d->idx_type;
  if (!is_int_type(t) || d->incr == 0 || d->incr == INT64_MIN) return OMPRT_ERR_INVALID;
  int64_t lb = d->lb, ub = d->ub;
  if (t == OMPRT_I32) {
    if (lb != (int64_t)(int32_t)lb || ub != (int64_t)(int32_t)ub) return OMPRT_ERR_INVALID;
  } else if (t == OMPRT_U32) {
    if (lb != (int64_t)(uint32_t)lb || ub != (int64_t)(uint32_t)ub) return OMPRT_ERR_INVALID;
  }
  if ((t == OMPRT_I32 || t == OMPRT_U32) && (d->incr > INT32_MAX || d->incr < -INT32_MAX))
    return OMPRT_ERR_INVALID;
  const bool sgn = t == OMPRT_I32 || t == OMPRT_I64;
  const bool up = d->incr > 0;
  bool empty;
  if (sgn)
    empty = up ? ub < lb : ub > lb;
  else
    empty = up ? (uint64_t)ub < (uint64_t)lb : (uint64_t)ub > (uint64_t)lb;
  *wide_lb = lb;
  if (empty) {
    *n = 0;
    return OMPRT_OK;
  }
  const uint64_t span = up ? (uint64_t)ub - (uint64_t)lb : (uint64_t)lb - (uint64_t)ub;
  const uint64_t step = up ? (uint64_t)d->incr : 0ull - (uint64_t)d->incr;
  const uint64_t q = span / step;
  if (q >= (uint64_t)INT64_MAX) return OMPRT_ERR_UNSUPPORTED;  // 2^63 iterations or more
  *n = q + 1;
  return OMPRT_OK;
}

static omprt_status validate_body(const omprt_loop_desc* d, uint64_t n) {
  if (d->reserved != 0) return OMPRT_ERR_INVALID;
  if (d->seq && d->body != OMPRT_BODY_MAP_RECORD) return OMPRT_ERR_INVALID;
  switch (d->body) {
    case OMPRT_BODY_MAP_RECORD:
      if (!d->out && n) return OMPRT_ERR_INVALID;
      return OMPRT_OK;
    case OMPRT_BODY_AXPY:
      if (d->data_type != OMPRT_F32 && d->data_type != OMPRT_I32) return OMPRT_ERR_UNSUPPORTED;
      if ((!d->x || !d->y) && n) return OMPRT_ERR_INVALID;
      if (d->data_type == OMPRT_I32 &&
          (d->alpha != std::floor(d->alpha) || std::fabs(d->alpha) > 2147483647.0))
        return OMPRT_ERR_INVALID;
      return OMPRT_OK;
    case OMPRT_BODY_STENCIL1D3:
    case OMPRT_BODY_STENCIL2D5:
      if (d->data_type != OMPRT_F32) return OMPRT_ERR_UNSUPPORTED;
      if ((!d->x || !d->out) && n) return OMPRT_ERR_INVALID;
      if (d->x == d->out && n) return OMPRT_ERR_INVALID;  // out of place only
      if (d->body == OMPRT_BODY_STENCIL2D5) {
        if (d->nx < 1 || d->ny < 1) return OMPRT_ERR_INVALID;
        if ((uint64_t)d->nx > (uint64_t)INT64_MAX / (uint64_t)d->ny) return OMPRT_ERR_INVALID;
        if ((uint64_t)d->nx * (uint64_t)d->ny != n) return OMPRT_ERR_INVALID;
      }
      return OMPRT_OK;
    case OMPRT_BODY_DOT:
      if (d->data_type != OMPRT_F32) return OMPRT_ERR_UNSUPPORTED;
      if ((!d->x || !d->y) && n) return OMPRT_ERR_INVALID;
      return OMPRT_OK;
    case OMPRT_BODY_NONE:
      if (d->data_type != OMPRT_F32 && d->data_type != OMPRT_BF16 && d->data_type != OMPRT_I32 &&
          d->data_type != OMPRT_I64)
        return OMPRT_ERR_UNSUPPORTED;
      if (!d->x && n) return OMPRT_ERR_INVALID;
      return OMPRT_OK;
  }
  return OMPRT_ERR_INVALID;
}

// Accumulator kind for a body's reduction operand.
static omprt_status pick_acc(const omprt_loop_desc* d, const omprt_reduce_desc* red, int* acc) {
  if (!red) {
    if (d->body == OMPRT_BODY_DOT || d->body == OMPRT_BODY_NONE) return OMPRT_ERR_INVALID;
    *acc = kAccNone;
    return OMPRT_OK;
  }
  if (!red->result_dev) return OMPRT_ERR_INVALID;
  if (d->body == OMPRT_BODY_MAP_RECORD) return OMPRT_ERR_INVALID;
  const bool integer = d->data_type == OMPRT_I32 || d->data_type == OMPRT_I64;
  switch (red->op) {
    case OMPRT_OP_SUM:
      if (integer) {
        *acc = kAccSumI64;
      } else if (red->precision == OMPRT_PREC_COMP_F64 || red->precision == OMPRT_PREC_COMP_F32) {
        *acc = kAccCompF32;
      } else if (red->precision == OMPRT_PREC_NAIVE_F32) {
        *acc = kAccNaiveF32;
      } else {
        return OMPRT_ERR_INVALID;
      }
      return OMPRT_OK;
    case OMPRT_OP_MAX:
      *acc = integer ? kAccMaxI64 : kAccMaxF32;
      return OMPRT_OK;
    case OMPRT_OP_MIN:
      *acc = integer ? kAccMinI64 : kAccMinF32;
      return OMPRT_OK;
  }
  return OMPRT_ERR_INVALID;
}

static omprt_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return OMPRT_OK;
  if (e == cudaErrorNotSupported) return OMPRT_ERR_UNSUPPORTED;
  cudaGetLastError();  // clear a non-sticky launch error
  return OMPRT_ERR_CUDA;
}

extern "C" {

const char* omprt_status_str(omprt_status s) {
  switch (s) {
    case OMPRT_OK: return "ok";
    case OMPRT_ERR_INVALID: return "invalid argument";
    case OMPRT_ERR_NOMEM: return "out of device memory";
    case OMPRT_ERR_CUDA: return "CUDA runtime error";
    case OMPRT_ERR_TIMEOUT: return "bounded device wait timed out";
    case OMPRT_ERR_UNSUPPORTED: return "unsupported request";
    case OMPRT_ERR_NOT_INIT: return "context not initialised";
    case OMPRT_ERR_DEVICE: return "device reported an error";
  }
  return "unknown status";
}

omprt_status omprt_init(int device, omprt_ctx** out) {
  if (!out) return OMPRT_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return OMPRT_ERR_CUDA;
  DeviceGuard guard(device);
  omprt_ctx* c = new (std::nothrow) omprt_ctx();
  if (!c) return OMPRT_ERR_NOMEM;
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, device);
  cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  c->stack_bytes = 4096;
  c->stencil_stage_bytes = kStencilStageDefault;
  bool ok = cudaMalloc(&c->status_dev, 256) == cudaSuccess &&
            cudaMalloc(&c->slots_dev, kSlotBytes * OMPRT_SLOTS) == cudaSuccess &&
            cudaMalloc(&c->pool_dev, (size_t)OMPRT_MAX_RED_TEAMS * OMPRT_POOL_BYTES_PER_TEAM) ==
                cudaSuccess &&
            cudaMalloc(&c->mlp_rows_dev, sizeof(float) * kMlpMaxBatch * kMlpRowFloats) ==
                cudaSuccess;
  ok = ok && cudaMemset(c->status_dev, 0, 256) == cudaSuccess &&
       cudaMemset(c->slots_dev, 0, kSlotBytes * OMPRT_SLOTS) == cudaSuccess &&
       cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaFree(c->status_dev);
    cudaFree(c->slots_dev);
    cudaFree(c->pool_dev);
    cudaFree(c->mlp_rows_dev);
    cudaGetLastError();
    delete c;
    return OMPRT_ERR_NOMEM;
  }
  *out = c;
  return OMPRT_OK;
}

omprt_status omprt_finalize(omprt_ctx* c) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  DeviceGuard guard(c->device);
  cudaFree(c->status_dev);
  cudaFree(c->slots_dev);
  cudaFree(c->pool_dev);
  cudaFree(c->mlp_rows_dev);
  delete c;
  return OMPRT_OK;
}

int32_t omprt_sm_count(const omprt_ctx* c) { return c ? c->sm_count : 0; }

omprt_status omprt_alloc_shared(omprt_ctx* c, size_t bytes) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (bytes > kMaxStackBytes || (int64_t)((bytes + 15) & ~size_t(15)) > c->max_smem_optin)
    return OMPRT_ERR_INVALID;
  c->stack_bytes = (uint32_t)((bytes + 15) & ~size_t(15));
  return OMPRT_OK;
}

omprt_status omprt_set_stage_bytes(omprt_ctx* c, int64_t bytes) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (bytes < 0 || bytes > (int64_t)c->max_smem_optin) return OMPRT_ERR_INVALID;
  c->stage_bytes = (uint32_t)(bytes & ~int64_t(15));
  return OMPRT_OK;
}

omprt_status omprt_set_stencil_slab_shape(omprt_ctx* c, int32_t slab_floats, int32_t buffers) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if ((slab_floats != 0 && slab_floats != 16 && slab_floats != 32) ||
      (buffers != 0 && (buffers < 2 || buffers > 4)))
    return OMPRT_ERR_INVALID;
  c->slab_floats = (uint32_t)slab_floats;
  c->slab_buffers = (uint32_t)buffers;
  return OMPRT_OK;
}

omprt_status omprt_set_launch_overlap(omprt_ctx* c, int32_t on) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  c->launch_overlap = on != 0;
  return OMPRT_OK;
}

omprt_status omprt_set_stencil_stage_bytes(omprt_ctx* c, int64_t bytes) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (bytes < 0 || bytes > (int64_t)c->max_smem_optin) return OMPRT_ERR_INVALID;
  c->stencil_stage_bytes = (uint32_t)(bytes & ~int64_t(15));
  return OMPRT_OK;
}

}  // extern "C"

// Arrays a body moves per iteration and their element size, for the staged
// form of schedules (0 arrays: the body is not staged); halo: elements its
// input window reaches beyond a pass on each side (the stencils).
struct StageShape {
  uint32_t arrays, elem;
  uint64_t halo;
};
static StageShape stage_shape(const omprt_loop_desc* d, uint64_t n) {
  switch (d->body) {
    case OMPRT_BODY_AXPY:
      return {2u, 4u, 0};  // f32 or i32: x, y (y written back)
    case OMPRT_BODY_DOT:
      return {2u, 4u, 0};
    case OMPRT_BODY_NONE:
      if (d->data_type == OMPRT_F32 || d->data_type == OMPRT_I32) return {1u, 4u, 0};
      if (d->data_type == OMPRT_BF16) return {1u, 2u, 0};
      if (d->data_type == OMPRT_I64) return {1u, 8u, 0};
      return {0u, 0u, 0};
    case OMPRT_BODY_STENCIL1D3:  // the window is read in 16-byte units
      return n % 4 == 0 ? StageShape{1u, 4u, 1} : StageShape{0u, 0u, 0};
    case OMPRT_BODY_STENCIL2D5:  // and a unit must not straddle two rows
      return n % 4 == 0 && d->nx % 4 == 0 ? StageShape{1u, 4u, (uint64_t)d->nx}
                                          : StageShape{0u, 0u, 0};
    default:
      return {0u, 0u, 0};
  }
}

// Staged pass size for a dynamic(c) / static(c) / static launch: the largest
// P <= 32 chunks whose buffers (every warp: P chunks of every array) fit the
// context's per-team staging bytes, or 0 for the plain form.  Measured on
// GB300 (n = 2^26): chunks below 256 bytes are already coalesced in the plain
// form and lose to the per-pass overhead (static(8) axpy 0.94 staged against
// 1.02 plain); without a reduction staging wins from P >= 16 (dynamic(256)
// 0.97 against 0.64, static(64) 1.02 against 0.97) and loses below
// (dynamic(1024): P <= 8); with a (compensated) reduction the per-element
// work needs many warps per SM, and staging wins only with all 32 lanes busy
// on chunks of at most 512 bytes over all arrays (dot dynamic(64) +16%, sum
// +9%; dynamic(256) loses).
struct StagePlan {
  uint32_t chunks;      // P; 0: the plain form
  uint32_t warp_bytes;  // shared memory per warp
};
static StagePlan stage_plan(const omprt_ctx* c, const StageShape& sh, uint64_t chunk,
                            uint32_t threads, size_t smem_base, bool reduction) {
  const StagePlan none = {0u, 0u};
  if (!sh.arrays || c->stage_bytes == 0) return none;
  const uint64_t cb = chunk * sh.elem;
  if (cb % 16 || cb < 256 || cb > c->stage_bytes) return none;
  const uint64_t warps = threads / 32, per_warp = c->stage_bytes / warps;
  uint64_t P;
  if (sh.halo) {
    // window of at most P c + 2 halo + 6 elements (16-byte widened), then P
    // chunks of output.  The halo is re-read from L2 by every pass, so it
    // must stay small against the pass: at most a quarter of it (a 2-D grid
    // of 4096-wide rows needs two 16 KB halo rows per pass, and measured
    // slower staged: 0.21 against 0.25 for dynamic(256)).  A stencil unit
    // costs an owner lane several times an axpy unit, so long chunks walked
    // by one lane lose (1-D, n = 2^26: c = 64 0.94 staged against 0.69,
    // c = 128 0.74 against 0.65, c = 256 0.59 against 0.68): chunks of at
    // most 512 bytes.
    if (reduction || cb > 512) return none;
    const uint64_t fixed = (2 * sh.halo + 8) * sh.elem;
    P = per_warp > fixed ? (per_warp - fixed) / (2 * cb) : 0;
    if (P > 32) P = 32;
    if (P == 0 || 8 * sh.halo * sh.elem > P * cb) return none;
  } else {
    P = per_warp / (sh.arrays * cb);
    if (P > 32) P = 32;
    if (reduction ? (P < 32 || sh.arrays * cb > 512) : P < 16) return none;
  }
  // equal passes: a claim of 32 chunks in ceil(32 / P) passes of (nearly)
  // the same size, not P, P, ..., remainder
  P = (32 + (32 + P - 1) / P - 1) / ((32 + P - 1) / P);
  const uint64_t wb = sh.halo ? ((P * chunk + 2 * sh.halo + 8) * sh.elem + 15) / 16 * 16 + P * cb
                              : P * sh.arrays * cb;
  // leave room for the kernel's static shared memory
  if (smem_base + warps * wb + 2048 > (uint64_t)c->max_smem_optin) return none;
  return {(uint32_t)P, (uint32_t)wb};
}

static omprt_status launch_region_impl(omprt_ctx* c, const omprt_loop_desc* d, int64_t dist_chunk,
                                       int32_t sched, int64_t chunk, int32_t teams,
                                       int32_t threads, const omprt_reduce_desc* red,
                                       void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!d) return OMPRT_ERR_INVALID;
  uint64_t n;
  int64_t lb;
  omprt_status s = loop_trip_count(d, &n, &lb);
  if (s) return s;
  if ((s = validate_body(d, n))) return s;
  int acc;
  if ((s = pick_acc(d, red, &acc))) return s;
  if (sched == OMPRT_SCHED_LEARNED) {
    int32_t k;
    if ((s = omprt_choose_config(c, d, red != nullptr, &k))) return s;
    LearnedConfig cfg = learned_config(k);
    sched = cfg.sched;
    chunk = cfg.chunk;
    teams = cfg.teams_per_sm * c->sm_count;
    threads = cfg.threads;
  }
  if (chunk < 0 || threads < 0 || threads > 1024 || threads % 32 || teams < 0 || dist_chunk < 0)
    return OMPRT_ERR_INVALID;
  int ksched;
  if (dist_chunk > 0) {
    if (sched != OMPRT_SCHED_STATIC && sched != OMPRT_SCHED_STATIC_CHUNKED)
      return OMPRT_ERR_UNSUPPORTED;
    if (sched == OMPRT_SCHED_STATIC_CHUNKED && chunk < 1) return OMPRT_ERR_INVALID;
    ksched = kDist;
  } else switch (sched) {
    case OMPRT_SCHED_STATIC: ksched = chunk ? kChunked : kStatic; break;
    case OMPRT_SCHED_STATIC_CHUNKED:
      if (chunk < 1) return OMPRT_ERR_INVALID;
      ksched = kChunked;
      break;
    case OMPRT_SCHED_DYNAMIC:
      if (chunk < 1) return OMPRT_ERR_INVALID;
      ksched = kDynamic;
      break;
    case OMPRT_SCHED_AUTO: ksched = kAuto; break;
    case OMPRT_SCHED_GUIDED: ksched = kGuided; break;
    case OMPRT_SCHED_NONMONOTONIC:
      if (chunk < 1) return OMPRT_ERR_INVALID;
      ksched = kNonmono;
      break;
    default: return OMPRT_ERR_INVALID;
  }
  if (threads == 0) threads = 256;
  if (teams == 0) {
    const uint64_t want = (n + (uint64_t)threads - 1) / (uint64_t)threads;
    const uint64_t cap = 4ull * (uint64_t)c->sm_count;
    teams = (int32_t)(want < 1 ? 1 : (want > cap ? cap : want));
  }
  const bool counters = ksched == kDynamic || ksched == kGuided;
  if ((acc != kAccNone || counters) && teams > OMPRT_MAX_RED_TEAMS) return OMPRT_ERR_INVALID;

  DeviceGuard guard(c->device);
  rt::OverlapScope overlap(c->launch_overlap, (size_t)c->smem_per_sm);
  RegionArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.chunk = (uint64_t)chunk;
  a.dist_chunk = (uint64_t)dist_chunk;
  a.x = d->x;
  a.y = d->y;
  a.out = d->out;
  a.seq = d->seq;
  a.alpha_f = (float)d->alpha;
  a.alpha_i = d->data_type == OMPRT_I32 ? (int32_t)d->alpha : 0;
  a.c0 = (float)d->c0;
  a.c1 = (float)d->c1;
  a.nx = (uint64_t)d->nx;
  a.ny = (uint64_t)d->ny;
  a.nx_magic = a.nx >= 2 ? (~0ull) / a.nx + 1 : 0;
  a.small_index = (n < (1ull << 32) && a.nx < (1ull << 32)) ? 1u : 0u;
  a.prec = red ? (uint32_t)red->precision : 0u;
  a.stack_bytes = c->stack_bytes;
  a.pool_bytes = OMPRT_POOL_BYTES_PER_TEAM;
  a.pool = c->pool_dev;
  a.pool_teams = OMPRT_MAX_RED_TEAMS;
  a.result = red ? red->result_dev : nullptr;
  a.status = c->status_dev;
  if (acc != kAccNone || counters) {
    ScratchSlot sl = ctx_next_slot(c);
    a.partials = sl.partials;
    a.ticket = sl.ticket;
    a.dyn_next = sl.dyn_next;
  }
  size_t smem = acc != kAccNone ? c->stack_bytes : 0;
  // staged forms of dynamic(c), static(c) and static: the chunk a warp's
  // lanes own (static without chunk: one block of n / (G T) per thread, used
  // only when that division is exact, so every team's block is T of them)
  uint64_t stage_c = 0;
  if (ksched == kDynamic || ksched == kChunked || ksched == kNonmono) stage_c = (uint64_t)chunk;
  if (ksched == kStatic && n % ((uint64_t)teams * (uint64_t)threads) == 0)
    stage_c = n / ((uint64_t)teams * (uint64_t)threads);
  if (stage_c) {
    const StagePlan sp = stage_plan(c, stage_shape(d, n), stage_c, (uint32_t)threads, smem,
                                    acc != kAccNone);
    if (sp.chunks) {
      a.stage_chunks = sp.chunks;
      a.stage_warp_bytes = sp.warp_bytes;
      a.stage_off = (uint32_t)smem;
      if (ksched == kStatic) a.chunk = stage_c;
      smem += (size_t)(threads / 32) * sp.warp_bytes;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (d->body == OMPRT_BODY_STENCIL2D5 && ksched == kAuto && acc == kAccNone &&
      d->data_type == OMPRT_F32) {
    e = launch_stencil2d_tiles(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny,
                               (float)d->c0, (float)d->c1, (unsigned)teams, (unsigned)threads,
                               c->status_dev, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  // teams of one warp whose blocks are several rows of one 32-chunk group
  // (m = nx / c < 32): the CTA's warps on adjacent teams, one tensor copy a
  // step for all of them (4096^2 dynamic(256): 0.68 against 0.65 in slabs)
  if (d->body == OMPRT_BODY_STENCIL2D5 && acc == kAccNone && d->data_type == OMPRT_F32 &&
      (ksched == kDynamic || ksched == kChunked) && c->stencil_stage_bytes != 0) {
    e = launch_stencil2d_colring(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny, ksched,
                                 (uint64_t)chunk, (float)d->c0, (float)d->c1, (unsigned)teams,
                                 (unsigned)threads, c->slab_buffers, c->sm_count,
                                 c->max_smem_optin, c->status_dev, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  // static(c) and dynamic(c) with c a multiple of 16 dividing nx and team
  // blocks of whole rows: each warp's chunks in swizzled tensor-copied slabs
  // (4096^2, alone: static(64) 0.73 of the copy rate, dynamic(64) 0.70,
  // dynamic(256) 0.62, against 0.46 / - / 0.44 in the forms below)
  if (d->body == OMPRT_BODY_STENCIL2D5 && acc == kAccNone && d->data_type == OMPRT_F32 &&
      (ksched == kDynamic || ksched == kChunked) && c->stencil_stage_bytes != 0) {
    e = launch_stencil2d_slabs(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny, ksched,
                               (uint64_t)chunk, (float)d->c0, (float)d->c1, (unsigned)teams,
                               (unsigned)threads, c->slab_floats, c->slab_buffers, c->sm_count,
                               c->max_smem_optin, c->status_dev, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  // static(1), team size dividing nx: each warp's strips a band of rows at a
  // time from tensor copies (4096^2, alone: 0.68 of the copy rate, against
  // 0.57 in the register strips below)
  if (d->body == OMPRT_BODY_STENCIL2D5 && acc == kAccNone && d->data_type == OMPRT_F32 &&
      ksched == kChunked && chunk == 1 && c->stencil_stage_bytes != 0) {
    e = launch_stencil2d_bands(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny,
                               (float)d->c0, (float)d->c1, (unsigned)teams, (unsigned)threads,
                               c->slab_buffers, c->sm_count, c->max_smem_optin, c->status_dev, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  // static schedules of the 2-D stencil whose owner map repeats row by row:
  // vertical strips, rows above / at / below in registers (4096^2, alone:
  // static(8) 0.73 of the copy rate, static 0.73, static(4) 0.67, static(1)
  // 0.55, against 0.55 / 0.61 / - / 0.42 in the other forms)
  if (d->body == OMPRT_BODY_STENCIL2D5 && acc == kAccNone && d->data_type == OMPRT_F32 &&
      (ksched == kStatic || ksched == kChunked)) {
    e = launch_stencil2d_strips(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny, ksched,
                                (uint64_t)chunk, (float)d->c0, (float)d->c1, (unsigned)teams,
                                (unsigned)threads, c->sm_count, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  // dynamic(c) outside the slab form, team blocks of whole rows: the row
  // ring (4096^2 dynamic(256): 0.47 of the copy rate against 0.44 in the
  // streamed ring below)
  if (d->body == OMPRT_BODY_STENCIL2D5 && acc == kAccNone && d->data_type == OMPRT_F32 &&
      ksched == kDynamic && c->stencil_stage_bytes != 0) {
    e = launch_stencil2d_rowring(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny, ksched,
                                 (uint64_t)chunk, (float)d->c0, (float)d->c1, (unsigned)teams,
                                 (unsigned)threads, c->stencil_stage_bytes, c->sm_count,
                                 c->max_smem_optin, c->status_dev, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  // the streamed ring form of the 2-D stencil where it beats the others
  // (measured at 4096^2, best teams x threads of each form): dynamic(256)
  // 0.44 of the copy rate against 0.25 plain; static(1) launches that are not
  // row-periodic 0.42 against 0.40; static and static(c > 1) stay with their
  // own forms (plain static 0.59 against 0.51 in the ring, static(8) 0.53
  // against 0.52, static(64) 0.45 in the row ring against 0.44)
  if (d->body == OMPRT_BODY_STENCIL2D5 && acc == kAccNone && d->data_type == OMPRT_F32 &&
      (ksched == kDynamic || (ksched == kChunked && chunk == 1)) &&
      c->stencil_stage_bytes != 0) {
    e = launch_stencil2d_owner(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny, ksched,
                               (uint64_t)chunk, (float)d->c0, (float)d->c1, (unsigned)teams,
                               (unsigned)threads, c->stencil_stage_bytes, c->sm_count,
                               c->max_smem_optin, c->status_dev, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  if (d->body == OMPRT_BODY_STENCIL2D5 && ksched == kChunked && acc == kAccNone &&
      d->data_type == OMPRT_F32 && c->stage_bytes != 0) {
    e = launch_stencil2d_rows(d->x, (float*)d->out, (uint64_t)d->nx, (uint64_t)d->ny,
                              (uint64_t)chunk, (float)d->c0, (float)d->c1, (unsigned)teams,
                              (unsigned)threads, c->max_smem_optin, c->status_dev, st);
    if (e != cudaErrorNotSupported) return from_cuda(e);
    cudaGetLastError();
  }
  const bool f32path = d->data_type == OMPRT_F32 || d->data_type == OMPRT_BF16;
  if (d->body == OMPRT_BODY_MAP_RECORD || !f32path)
    e = launch_region_int(d->body, d->data_type, acc, ksched, (unsigned)teams, (unsigned)threads,
                          smem, st, a);
  else
    e = launch_region_f32(d->body, d->data_type, acc, ksched, (unsigned)teams, (unsigned)threads,
                          smem, st, a);
  return from_cuda(e);
}

extern "C" {

omprt_status omprt_launch_region(omprt_ctx* c, const omprt_loop_desc* d, int32_t sched,
                                 int64_t chunk, int32_t teams, int32_t threads,
                                 const omprt_reduce_desc* red, void* stream) {
  return launch_region_impl(c, d, 0, sched, chunk, teams, threads, red, stream);
}

omprt_status omprt_launch_region_dist(omprt_ctx* c, const omprt_loop_desc* d, int64_t dist_chunk,
                                      int32_t sched, int64_t chunk, int32_t teams,
                                      int32_t threads, const omprt_reduce_desc* red,
                                      void* stream) {
  if (dist_chunk < 1) return c ? OMPRT_ERR_INVALID : OMPRT_ERR_NOT_INIT;
  return launch_region_impl(c, d, dist_chunk, sched, chunk, teams, threads, red, stream);
}

omprt_status omprt_reduce(omprt_ctx* c, int32_t op, int32_t dtype, int32_t precision,
                          const void* data, int64_t n, void* result, int32_t teams,
                          int32_t threads, void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (n < 0 || !result) return OMPRT_ERR_INVALID;
  omprt_loop_desc d;
  std::memset(&d, 0, sizeof(d));
  d.lb = 0;
  d.ub = n - 1;
  d.incr = 1;
  d.idx_type = OMPRT_I64;
  d.body = OMPRT_BODY_NONE;
  d.data_type = dtype;
  d.x = const_cast<void*>(data);
  omprt_reduce_desc r;
  r.op = op;
  r.precision = precision;
  r.result_dev = result;
  // two teams of 512 a SM: the value bodies' registers leave room for two
  // such CTAs an SM, so every team is resident at once and the launch is one
  // wave (n = 2^28: bf16 sum 0.96 of the copy rate against 0.94 with four
  // teams a SM in two waves, fp32 sum 1.04 against 1.02)
  if (teams == 0) teams = 2 * c->sm_count;
  if (threads == 0) threads = 512;
  return omprt_launch_region(c, &d, OMPRT_SCHED_AUTO, 0, teams, threads, &r, stream);
}

omprt_status omprt_static_init_table(omprt_ctx* c, const omprt_loop_desc* d, int64_t chunk,
                                     int32_t teams, int32_t threads, int64_t* table,
                                     void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!d || !table || chunk < 0 || teams < 1 || threads < 1 || threads > 1024)
    return OMPRT_ERR_INVALID;
  if ((uint64_t)teams * (uint64_t)threads > (1ull << 26)) return OMPRT_ERR_INVALID;
  uint64_t n;
  int64_t lb;
  omprt_status s = loop_trip_count(d, &n, &lb);
  if (s) return s;
  DeviceGuard guard(c->device);
  return from_cuda(launch_static_table(n, lb, d->incr, (uint64_t)chunk, (unsigned)teams,
                                       (unsigned)threads, table, (cudaStream_t)stream));
}

omprt_status omprt_loop_trip_count(const omprt_loop_desc* d, uint64_t* n) {
  if (!d || !n) return OMPRT_ERR_INVALID;
  int64_t lb;
  return loop_trip_count(d, n, &lb);
}

omprt_status omprt_sync_status(omprt_ctx* c, void* stream, uint32_t* bits) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  DeviceGuard guard(c->device);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return OMPRT_ERR_CUDA;
  uint32_t h = 0;
  if (cudaMemcpy(&h, c->status_dev, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return OMPRT_ERR_CUDA;
  if (bits) *bits = h;
  if (h) {
    if (cudaMemset(c->status_dev, 0, 4) != cudaSuccess) return OMPRT_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return OMPRT_ERR_CUDA;
    return OMPRT_ERR_DEVICE;
  }
  return OMPRT_OK;
}

omprt_status omprt_test_atomics(omprt_ctx* c, int32_t teams, int32_t threads, int32_t reps,
                                uint32_t e, uint32_t* words, uint32_t* returned, void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (teams < 1 || threads < 1 || threads > 1024 || reps < 1 || !words) return OMPRT_ERR_INVALID;
  DeviceGuard guard(c->device);
  return from_cuda(launch_test_atomics((unsigned)teams, (unsigned)threads, reps, e, words,
                                       returned, c->status_dev, (cudaStream_t)stream));
}

omprt_status omprt_test_barrier(omprt_ctx* c, int32_t teams, int32_t threads, int32_t sub,
                                int32_t rounds, uint32_t* errors, void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (teams < 1 || threads < 32 || threads > 1024 || threads % 32 || rounds < 1 || !errors)
    return OMPRT_ERR_INVALID;
  if (sub) {
    // named barriers 1..15: at most 15 sub-teams, each whole warps
    if (sub < 32 || sub % 32 || threads % sub || threads / sub > 15) return OMPRT_ERR_INVALID;
  }
  DeviceGuard guard(c->device);
  return from_cuda(launch_test_barrier((unsigned)teams, (unsigned)threads, (unsigned)sub, rounds,
                                       errors, (cudaStream_t)stream));
}

omprt_status omprt_test_wait(omprt_ctx* c, int32_t teams, const uint32_t* flag, uint32_t expect,
                             int64_t timeout_us, int32_t* out, void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (teams < 1 || teams > 4096 || !flag || !out || timeout_us < 1 || timeout_us > 2000000)
    return OMPRT_ERR_INVALID;
  DeviceGuard guard(c->device);
  return from_cuda(launch_test_wait((unsigned)teams, flag, expect, (uint64_t)timeout_us * 1000,
                                    out, c->status_dev, (cudaStream_t)stream));
}

omprt_status omprt_test_stack(omprt_ctx* c, int32_t teams, int64_t S, int64_t Q,
                              const int64_t* ops, int64_t nops, int64_t* out, int64_t* status_out,
                              void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (teams < 1 || teams > OMPRT_MAX_RED_TEAMS || S < 0 || S > kMaxStackBytes ||
      S > c->max_smem_optin || Q < 0 || Q > OMPRT_POOL_BYTES_PER_TEAM || nops < 0 ||
      nops > 4096 || (nops && (!ops || !out)) || !status_out)
    return OMPRT_ERR_INVALID;
  DeviceGuard guard(c->device);
  return from_cuda(launch_test_stack((unsigned)teams, (uint32_t)S, (uint32_t)Q,
                                     Q ? c->pool_dev : nullptr, ops, nops, out, status_out,
                                     c->status_dev, (cudaStream_t)stream));
}

}  // extern "C"
