// Generic-mode (non-SPMD) target regions.
//
// The region form is a loop nest whose outer level is sequential per team:
//   #pragma omp target teams distribute        // segments over teams
//   for (s = 0; s < nseg; ++s) {              // run by the team's main thread
//     double v = 0;                            // shared with the parallel region
//     #pragma omp parallel for reduction(+: v) // run by all threads of the team
//     for (i = seg[s]; i < seg[s + 1]; ++i) v += body(i);
//     result[s] = v;                           // main thread again
//   }
// The runtime side of this (as in the paper's runtime, Sec. 2.1): thread 0 is
// the main thread and runs the sequential code; the other threads wait in a
// state machine for a parallel region to be handed to them; the variable the
// sequential code shares with the parallel region is "globalised" onto the
// team's shared-memory stack with alloc_shared (Sec. 2.1, Listing 1).  Here
// the state machine is one loop that main and workers walk together: every
// hand-over and every join is a team barrier, so no thread spins.
#include "api_internal.h"

namespace rt {

struct GenericArgs {
  const int64_t* seg;  // nseg + 1 offsets into x / y
  uint64_t nseg;
  uint64_t n;          // length of x / y (offsets are checked against it)
  int32_t body;        // OMPRT_BODY_DOT or OMPRT_BODY_AXPY
  int32_t pad;
  const float* x;
  float* y;
  float alpha;
  uint32_t stack_bytes;
  double* result;      // per segment
  uint32_t* status;
};

template <class Body>
__global__ void __launch_bounds__(1024) generic_kernel(const GenericArgs A) {
  // team-shared state machine word: the work the main thread hands over
  __shared__ uint64_t w_lo, w_hi;
  __shared__ double* w_var;
  __shared__ int w_exit;
  const uint32_t t = threadIdx.x, T = blockDim.x, g = blockIdx.x, G = gridDim.x;
  RegionArgs ra;
  ra.x = A.x;
  ra.y = A.y;
  ra.alpha_f = A.alpha;
  const Body body(ra);
  if (t == 0) stack_init(A.stack_bytes, nullptr, 0);
  // team reduction scratch, the bottom block of the team stack
  float2* scratch = (float2*)team_alloc(32 * sizeof(float2), A.status);
  uint64_t s0, scnt;  // teams distribute: a balanced block of segments per team
  split_even(A.nseg, G, g, s0, scnt);
  for (uint64_t k = 0;; ++k) {
    if (t == 0) {  // sequential part: set up the next parallel region or finish
      w_exit = 1;
      if (k < scnt && scratch) {
        const int64_t lo = A.seg[s0 + k], hi = A.seg[s0 + k + 1];
        double* v = (double*)alloc_shared(sizeof(double), A.status);  // globalised variable
        if (v && lo >= 0 && lo <= hi && (uint64_t)hi <= A.n) {
          *v = 0.0;
          w_lo = (uint64_t)lo;
          w_hi = (uint64_t)hi;
          w_var = v;
          w_exit = 0;
        } else {
          if (v) free_shared(v, sizeof(double), A.status);
          set_status(A.status, v ? OMPRT_DEV_BAD_ARG : OMPRT_DEV_STACK_NOMEM);
        }
      }
    }
    team_barrier();  // hand-over: workers leave the wait state
    if (w_exit) break;
    // the parallel region: parallel for over [lo, hi) under the default
    // schedule, which OpenMP leaves to the implementation: static with a
    // chunk of one 32-byte vector, round robin (a warp then covers 1 KB of
    // contiguous memory per access; one contiguous piece per thread measured
    // 0.77 of the copy rate for a dot over 2^14-element segments).  The
    // iterations before the first 32-byte boundary and after the last run as
    // scalars, round robin too.
    const uint64_t lo = w_lo, hi = w_hi;
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
    const float2 v = team_reduce<AccCompF32>(acc.part(), scratch);
    if (t == 0) *w_var = __dadd_rn(*w_var, __dadd_rn((double)v.x, (double)v.y));
    team_barrier();  // join
    if (t == 0) {    // sequential part after the region
      A.result[s0 + k] = *w_var;
      free_shared(w_var, sizeof(double), A.status);
    }
  }
  team_free(scratch, 32 * sizeof(float2), A.status);
}

}  // namespace rt

using namespace rt;

extern "C" omprt_status omprt_launch_generic(omprt_ctx* c, const int64_t* seg_dev, int64_t nseg,
                                             const omprt_loop_desc* d, double* result_dev,
                                             int32_t teams, int32_t threads, void* stream) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!d || nseg < 0 || (nseg && (!seg_dev || !result_dev))) return OMPRT_ERR_INVALID;
  if (d->data_type != OMPRT_F32 || d->reserved) return OMPRT_ERR_UNSUPPORTED;
  if (d->body != OMPRT_BODY_DOT && d->body != OMPRT_BODY_AXPY) return OMPRT_ERR_UNSUPPORTED;
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
  GenericArgs a;
  a.seg = seg_dev;
  a.nseg = (uint64_t)nseg;
  a.n = n;
  a.body = d->body;
  a.pad = 0;
  a.x = (const float*)d->x;
  a.y = (float*)d->y;
  a.alpha = (float)d->alpha;
  a.stack_bytes = 1024;  // reduction scratch + the globalised variables
  a.result = result_dev;
  a.status = c->status_dev;
  cudaStream_t s = (cudaStream_t)stream;
  if (d->body == OMPRT_BODY_DOT)
    generic_kernel<BodyDotF32><<<teams, threads, a.stack_bytes, s>>>(a);
  else
    generic_kernel<BodyAxpyF32><<<teams, threads, a.stack_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? OMPRT_OK : OMPRT_ERR_CUDA;
}
