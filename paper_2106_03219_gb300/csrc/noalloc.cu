// A reduction entry point that allocates nothing: its cross-team scratch is a
// fixed array compiled into the library instead of memory from a context.
//
// Some callers cannot call cudaMalloc: code in a host callback or an
// allocator hook, code holding a lock that an allocation could need, or code
// running in a process whose device memory is owned and budgeted by someone
// else.  omprt_reduce_noalloc serves them.  It runs the same reduction kernel
// as omprt_reduce; only the place the kernel keeps its per-team partials and
// its ticket differs.
#include <cstring>
#include <mutex>

#include "api_internal.h"

using namespace rt;

namespace {

// Scratch: a 256-byte header (ticket, status word) and 16 bytes of partial
// per team.  Every GPU that loads the library holds this array until exit.
constexpr size_t kHeaderBytes = 256;
constexpr uint32_t kNoallocStackBytes = 4096;  // team stack (dynamic shared memory)
constexpr size_t kScratchBytes = kHeaderBytes + 16ull * OMPRT_NOALLOC_MAX_TEAMS;
// The only device-side error this path could raise is a team stack too small
// for the reduction's temporary (32 per-warp partials of at most 16 bytes,
// taken by the epilogue with team_alloc; the stack's bookkeeping lives in
// static shared memory).  With this capacity that allocation always
// succeeds, and the AUTO value loop has no waits, so the status word below
// is never set.
static_assert(kNoallocStackBytes >= 32 * 16, "noalloc team stack holds the reduction temporary");

static __device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

// Device address of the array, per device (host code must not use the
// symbol itself: on the host it names a stand-in, not device memory).
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {};

omprt_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return OMPRT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return OMPRT_ERR_CUDA;
    }
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return OMPRT_OK;
}

}  // namespace

extern "C" omprt_status omprt_reduce_noalloc(int32_t op, int32_t dtype, int32_t precision,
                                             const void* data, int64_t n, void* result,
                                             int32_t teams, int32_t threads, void* stream) {
  if (n < 0 || !result || (n && !data)) return OMPRT_ERR_INVALID;
  if (teams == 0) teams = OMPRT_NOALLOC_MAX_TEAMS;
  if (threads == 0) threads = 512;
  if (teams < 1 || teams > OMPRT_NOALLOC_MAX_TEAMS) return OMPRT_ERR_INVALID;
  if (threads < 32 || threads > 1024 || threads % 32) return OMPRT_ERR_INVALID;
  int acc;
  const bool integer = dtype == OMPRT_I32 || dtype == OMPRT_I64;
  if (!integer && dtype != OMPRT_F32 && dtype != OMPRT_BF16) return OMPRT_ERR_UNSUPPORTED;
  switch (op) {
    case OMPRT_OP_SUM:
      if (integer)
        acc = kAccSumI64;
      else if (precision == OMPRT_PREC_COMP_F64 || precision == OMPRT_PREC_COMP_F32)
        acc = kAccCompF32;
      else if (precision == OMPRT_PREC_NAIVE_F32)
        acc = kAccNaiveF32;
      else
        return OMPRT_ERR_INVALID;
      break;
    case OMPRT_OP_MAX: acc = integer ? kAccMaxI64 : kAccMaxF32; break;
    case OMPRT_OP_MIN: acc = integer ? kAccMinI64 : kAccMinF32; break;
    default: return OMPRT_ERR_INVALID;
  }
  unsigned char* scratch;
  omprt_status s = scratch_for_current_device(&scratch);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // A completed launch leaves its ticket at 0 (atomicInc(ticket, G - 1) wraps
  // on the last team); this clear, in stream order, only repairs a ticket (and
  // status word) left behind by a launch that did not run to the end.
  if (cudaMemsetAsync(scratch, 0, 8, st) != cudaSuccess) {
    cudaGetLastError();
    return OMPRT_ERR_CUDA;
  }
  RegionArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = (uint64_t)n;
  a.x = data;
  a.prec = (uint32_t)precision;
  a.stack_bytes = kNoallocStackBytes;
  a.pool = nullptr;
  a.pool_teams = 0;
  a.ticket = (uint32_t*)scratch;
  a.status = (uint32_t*)(scratch + 4);
  a.partials = scratch + kHeaderBytes;
  a.result = result;
  cudaError_t e;
  if (integer)
    e = launch_region_int(OMPRT_BODY_NONE, dtype, acc, kAuto, (unsigned)teams, (unsigned)threads,
                          kNoallocStackBytes, st, a);
  else
    e = launch_region_f32(OMPRT_BODY_NONE, dtype, acc, kAuto, (unsigned)teams,
                          (unsigned)threads, kNoallocStackBytes, st, a);
  if (e == cudaSuccess) return OMPRT_OK;
  cudaGetLastError();
  return e == cudaErrorNotSupported ? OMPRT_ERR_UNSUPPORTED : OMPRT_ERR_CUDA;
}
