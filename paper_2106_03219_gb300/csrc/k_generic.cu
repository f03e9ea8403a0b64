// Generic-mode (non-SPMD) target regions.
//
// The region form is a loop nest whose outer level is sequential per team:
//   #pragma omp target teams distribute        // segments over teams
//   for (s = 0; s < nseg; ++s) {              // run by the team's main thread
//     double v = 0, w = 0;                     // shared with the parallel regions
//     #pragma omp parallel for reduction(+: v) // region 1, run by the whole team
//     for (i = seg[s]; i < seg[s + 1]; ++i) v += x[i] * y[i];
//     float a = (float)v * alpha;              // main thread: uses region 1's result
//     #pragma omp parallel for reduction(+: w) // region 2
//     for (i = seg[s]; i < seg[s + 1]; ++i) { y[i] = a * x[i] + y[i]; w += y[i]; }
//     result[s] = {v, a, w};                   // main thread again
//   }
// (program OMPRT_GENERIC_DOT_AXPY; program OMPRT_GENERIC_REDUCE runs region 1
// alone, its body the descriptor's dot or axpy.)
//
// The runtime side (as in the paper's runtime, Sec. 2.1): thread 0 is the
// main thread and runs the sequential code; the other threads are workers
// waiting in a state machine.  To start a parallel region the main thread
// publishes a work descriptor in team-shared memory (the id of the outlined
// region, its loop bounds and its arguments, among them pointers to the
// variables it shares with the sequential code) and releases the workers;
// every thread reads the descriptor and dispatches on the region id, the
// main thread taking part as thread 0 of the parallel team; a join barrier
// ends the region and the main thread resumes.  The shared variables are
// "globalised" onto the team's shared-memory stack with alloc_shared
// (Sec. 2.1, Listing 1), capacity S from omprt_alloc_shared, overflowing to
// the team's slice of the context's pool; a request that neither holds sets
// OMPRT_DEV_STACK_NOMEM and the team stops.  Every hand-over and every join
// is a team barrier reached by all threads from the same loop, so no thread
// spins; the main thread's code between two regions is one step of its
// program (a small state machine over (segment, phase)).
#include "api_internal.h"

namespace rt {

// Outlined parallel regions a work descriptor can name.
enum : int32_t { kRegionExit = 0, kRegionDot = 1, kRegionAxpy = 2 };

// The hand-over: what the main thread publishes for its workers.
struct WorkDesc {
  int32_t fn;       // outlined region id
  float alpha;      // axpy scale, a value of the sequential code
  uint64_t lo, hi;  // the region's worksharing loop
  double* red;      // globalised reduction variable (on the team stack)
};

struct GenericArgs {
  const int64_t* seg;  // nseg + 1 offsets into x / y
  uint64_t nseg;
  uint64_t n;          // length of x / y (offsets are checked against it)
  int32_t program;     // OMPRT_GENERIC_*
  int32_t body;        // OMPRT_GENERIC_REDUCE: OMPRT_BODY_DOT or OMPRT_BODY_AXPY
  const float* x;
  float* y;
  float alpha;
  uint32_t stack_bytes;   // S of the team stack
  uint32_t pool_bytes;    // fallback pool bytes per team
  uint32_t pool_teams;    // teams with a pool slice
  unsigned char* pool;
  double* result;      // per segment: 1 (REDUCE) or 3 (DOT_AXPY) doubles
  uint32_t* status;
};

// parallel for over [lo, hi) under the default schedule, which OpenMP leaves
// to the implementation: static with a chunk of one 32-byte vector, round
// robin (a warp then covers 1 KB of contiguous memory per access; one
// contiguous piece per thread measured 0.77 of the copy rate for a dot over
// 2^14-element segments).  The iterations before the first 32-byte boundary
// and after the last run as scalars, round robin too.  Returns the thread's
// compensated partial of the reduction.
template <class Body>
__device__ __forceinline__ float2 generic_for(const Body& body, uint64_t lo, uint64_t hi) {
  const uint32_t t = threadIdx.x, T = blockDim.x;
  AccCompF32 acc;
  constexpr uint64_t V = Body::VEC;
  uint64_t vlo = lo, vhi = lo;
  if (body.vec_ok() && hi - lo >= V) {
    vlo = (lo + V - 1) / V * V;
    vhi = hi / V * V;
    if (vhi < vlo) vhi = vlo;
  }
  run_strided(body, lo, vlo - lo, t, T, acc);  // head
  {
    typename Body::Frag f[2];
    uint64_t v = vlo + (uint64_t)t * V;
    for (; v + (uint64_t)T * V < vhi; v += 2ull * T * V) {  // two vectors in flight
      body.load(v, f[0]);
      body.load(v + (uint64_t)T * V, f[1]);
      body.finish(v, f[0], acc);
      body.finish(v + (uint64_t)T * V, f[1], acc);
    }
    if (v < vhi) {
      body.load(v, f[0]);
      body.finish(v, f[0], acc);
    }
  }
  run_strided(body, vhi, hi - vhi, t, T, acc);  // tail
  return acc.part();
}

__global__ void __launch_bounds__(1024) generic_kernel(const GenericArgs A) {
  enter_region_grid();
  __shared__ WorkDesc s_work;  // the team-shared hand-over word
  const uint32_t t = threadIdx.x, g = blockIdx.x, G = gridDim.x;
  if (t == 0)
    stack_init(A.stack_bytes, g < A.pool_teams ? A.pool + (uint64_t)g * A.pool_bytes : nullptr,
               A.pool_bytes);
  // the runtime's team reduction scratch, the bottom block of the team stack
  float2* scratch = (float2*)team_alloc(32 * sizeof(float2), A.status);
  uint64_t s0, scnt;  // teams distribute: a balanced block of segments per team
  split_even(A.nseg, G, g, s0, scnt);
  // the main thread's program counter: segment k, phase within it, and the
  // globalised variables of the current segment
  uint64_t k = 0;
  int phase = 0;
  double *v = nullptr, *w = nullptr;
  float a = 0.f;
  bool stop = scratch == nullptr;  // uniform: team_alloc broadcasts its result
  for (;;) {
    if (t == 0) {  // sequential code up to the next parallel region (or the end)
      WorkDesc d;
      d.fn = kRegionExit;
      d.alpha = 0.f;
      d.lo = d.hi = 0;
      d.red = nullptr;
      while (!stop && d.fn == kRegionExit) {
        if (phase == 0) {  // a new segment: globalise its shared variables
          if (k == scnt) break;
          const int64_t lo = A.seg[s0 + k], hi = A.seg[s0 + k + 1];
          if (lo < 0 || lo > hi || (uint64_t)hi > A.n) {
            set_status(A.status, OMPRT_DEV_BAD_ARG);
            stop = true;
            break;
          }
          v = (double*)alloc_shared(sizeof(double), A.status);
          w = A.program == OMPRT_GENERIC_DOT_AXPY
                  ? (double*)alloc_shared(sizeof(double), A.status)
                  : nullptr;
          if (!v || (A.program == OMPRT_GENERIC_DOT_AXPY && !w)) {  // NOMEM bit already set
            if (w) free_shared(w, sizeof(double), A.status);
            if (v) free_shared(v, sizeof(double), A.status);
            stop = true;
            break;
          }
          *v = 0.0;
          if (w) *w = 0.0;
          d.fn = (A.program == OMPRT_GENERIC_REDUCE && A.body == OMPRT_BODY_AXPY) ? kRegionAxpy
                                                                                  : kRegionDot;
          d.alpha = A.alpha;
          d.lo = (uint64_t)lo;
          d.hi = (uint64_t)hi;
          d.red = v;
          phase = 1;
        } else if (phase == 1 && A.program == OMPRT_GENERIC_DOT_AXPY) {
          // between the regions: the sequential code reads region 1's result
          a = __fmul_rn((float)*v, A.alpha);
          d.fn = kRegionAxpy;
          d.alpha = a;
          d.lo = (uint64_t)A.seg[s0 + k];
          d.hi = (uint64_t)A.seg[s0 + k + 1];
          d.red = w;
          phase = 2;
        } else {  // after the segment's last region: results, release, next
          if (A.program == OMPRT_GENERIC_DOT_AXPY) {
            A.result[3 * (s0 + k)] = *v;
            A.result[3 * (s0 + k) + 1] = (double)a;
            A.result[3 * (s0 + k) + 2] = *w;
            free_shared(w, sizeof(double), A.status);
          } else {
            A.result[s0 + k] = *v;
          }
          free_shared(v, sizeof(double), A.status);
          ++k;
          phase = 0;
        }
      }
      s_work = d;
    }
    team_barrier();  // hand-over: workers leave the wait state
    const WorkDesc d = s_work;
    if (d.fn == kRegionExit) break;
    float2 part;
    RegionArgs ra;
    ra.x = A.x;
    ra.y = A.y;
    ra.alpha_f = d.alpha;
    if (d.fn == kRegionDot)  // dispatch on the outlined region's id
      part = generic_for(BodyDotF32(ra), d.lo, d.hi);
    else
      part = generic_for(BodyAxpyF32(ra), d.lo, d.hi);
    const float2 tv = team_reduce<AccCompF32>(part, scratch);
    if (t == 0) *d.red = __dadd_rn(*d.red, __dadd_rn((double)tv.x, (double)tv.y));
    team_barrier();  // join
  }
  if (scratch) team_free(scratch, 32 * sizeof(float2), A.status);
}

}  // namespace rt

using namespace rt;

extern "C" omprt_status omprt_launch_generic(omprt_ctx* c, const int64_t* seg_dev, int64_t nseg,
                                             const omprt_loop_desc* d, int32_t program,
                                             double* result_dev, int32_t teams, int32_t threads,
                                             void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!d || nseg < 0 || (nseg && (!seg_dev || !result_dev))) return OMPRT_ERR_INVALID;
  if (program != OMPRT_GENERIC_REDUCE && program != OMPRT_GENERIC_DOT_AXPY)
    return OMPRT_ERR_INVALID;
  if (d->data_type != OMPRT_F32 || d->reserved || d->seq) return OMPRT_ERR_UNSUPPORTED;
  if (program == OMPRT_GENERIC_REDUCE && d->body != OMPRT_BODY_DOT && d->body != OMPRT_BODY_AXPY)
    return OMPRT_ERR_UNSUPPORTED;
  uint64_t n;
  int64_t lb;
  omprt_status st = loop_trip_count(d, &n, &lb);
  if (st) return st;
  if (n && (!d->x || !d->y)) return OMPRT_ERR_INVALID;
  if (threads == 0) threads = 256;
  if (threads < 32 || threads > 1024 || threads % 32) return OMPRT_ERR_INVALID;
  if (teams == 0) teams = c->sm_count;
  if (teams < 1) return OMPRT_ERR_INVALID;
  if (nseg == 0) return OMPRT_OK;
  DeviceGuard guard(c->device);
  OverlapScope overlap(c->launch_overlap, (size_t)c->smem_per_sm);
  GenericArgs a;
  a.seg = seg_dev;
  a.nseg = (uint64_t)nseg;
  a.n = n;
  a.program = program;
  a.body = d->body;
  a.x = (const float*)d->x;
  a.y = (float*)d->y;
  a.alpha = (float)d->alpha;
  a.stack_bytes = c->stack_bytes;
  a.pool_bytes = OMPRT_POOL_BYTES_PER_TEAM;
  a.pool_teams = OMPRT_MAX_RED_TEAMS;
  a.pool = c->pool_dev;
  a.result = result_dev;
  a.status = c->status_dev;
  static const size_t static_bytes = static_smem_of(generic_kernel);
  if (smem_optin(generic_kernel, a.stack_bytes, static_bytes) != cudaSuccess) {
    cudaGetLastError();
    return OMPRT_ERR_CUDA;
  }
  return launch_kernel(generic_kernel, dim3(teams), dim3(threads), a.stack_bytes,
                       (cudaStream_t)stream, a) == cudaSuccess
             ? OMPRT_OK
             : OMPRT_ERR_CUDA;
}
