// Batched persistent executor: many small target regions in one kernel.
//
// The host flattens the regions into work items (region r, chunk j) of
// `chunk` iterations.  Each CTA (one team) claims items with an atomic add on
// a queue head and runs the item's iterations with its threads (32-byte
// vectors, grid-stride inside the item).  A region with a reduction leaves one
// fp64 partial per item; the CTA that finishes the region's last item (ticket
// by atomic add) combines the partials in item order and writes the result.
// The queue head, the exit count and the tickets are reset by their last
// users, so the launch can be replayed from a CUDA graph with no memset.
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.h"

namespace rt {

struct BatchRegion {
  int32_t body;       // OMPRT_BODY_AXPY / _DOT / _STENCIL1D3
  int32_t has_red;
  uint64_t n;
  const void* x;
  void* y;
  void* out;
  float alpha, c0, c1;
  uint32_t nitems;
  uint64_t first_item;
  double* result;
};

struct BatchArgs {
  const BatchRegion* regions;
  const uint32_t* item_region;  // region of each item
  uint64_t nitems;
  uint64_t chunk;
  double* partials;             // one per item
  uint32_t* tickets;            // one per region, left at 0
  unsigned long long* head;     // queue head, left at 0
  uint32_t* exits;              // CTAs that left, left at 0
  uint32_t* status;
};

// Iterations [lo, hi) of one region run by the whole CTA.
template <class Body, class Acc>
__device__ __forceinline__ void run_item(const Body& b, uint64_t lo, uint64_t hi, Acc& acc) {
  constexpr uint64_t V = Body::VEC;
  const uint32_t t = threadIdx.x, T = blockDim.x;
  uint64_t tail = lo;
  if (b.vec_ok() && lo % V == 0) {
    const uint64_t nv = (hi - lo) / V;
    typename Body::Frag f0, f1;
    uint64_t v = t;
    if constexpr (InFlight<Body>::value >= 2) {
      for (; v + T < nv; v += 2 * T) {
        b.load(lo + v * V, f0);
        b.load(lo + (v + T) * V, f1);
        b.finish(lo + v * V, f0, acc);
        b.finish(lo + (v + T) * V, f1, acc);
      }
    }
    for (; v < nv; v += T) {
      b.load(lo + v * V, f0);
      b.finish(lo + v * V, f0, acc);
    }
    tail = lo + nv * V;
  }
  if (tail + t < hi) run_scalar(b, tail + t, T, (hi - tail - t + T - 1) / T, acc);
}

__device__ __forceinline__ RegionArgs region_args(const BatchRegion& R) {
  RegionArgs a;
  a.n = R.n;
  a.x = R.x;
  a.y = R.y;
  a.out = R.out;
  a.alpha_f = R.alpha;
  a.c0 = R.c0;
  a.c1 = R.c1;
  return a;
}

__global__ void __launch_bounds__(1024) batch_kernel(const BatchArgs A) {
  enter_region_grid();
  __shared__ unsigned long long s_item;
  __shared__ int s_last;
  __shared__ double s_scr[32];
  __shared__ float2 s_scr2[32];
  const uint32_t t = threadIdx.x;
  for (;;) {
    if (t == 0) s_item = atomicAdd(A.head, 1ull);
    team_barrier();
    const unsigned long long item = s_item;
    if (item >= A.nitems) break;
    const uint32_t r = __ldg(A.item_region + item);
    const BatchRegion& R = A.regions[r];
    const uint64_t j = item - R.first_item;
    const uint64_t lo = j * A.chunk;
    const uint64_t hi = R.n - lo > A.chunk ? lo + A.chunk : R.n;
    const RegionArgs ra = region_args(R);
    if (!R.has_red) {
      AccNone none;
      if (R.body == OMPRT_BODY_AXPY)
        run_item(BodyAxpyF32(ra), lo, hi, none);
      else if (R.body == OMPRT_BODY_STENCIL1D3)
        run_item(BodyStencil1D(ra), lo, hi, none);
    } else {
      AccCompF32 acc;
      if (R.body == OMPRT_BODY_DOT)
        run_item(BodyDotF32(ra), lo, hi, acc);
      else if (R.body == OMPRT_BODY_AXPY)
        run_item(BodyAxpyF32(ra), lo, hi, acc);
      else
        run_item(BodyStencil1D(ra), lo, hi, acc);
      const float2 v = team_reduce<AccCompF32>(acc.part(), s_scr2);
      if (t == 0) {
        A.partials[item] = __dadd_rn((double)v.x, (double)v.y);
        flush();
        const uint32_t done = atomic_add(A.tickets + r, 1u);
        s_last = done == R.nitems - 1;
      }
      team_barrier();
      if (s_last) {
        // this CTA finished the region: combine its item partials in order
        flush();
        double s = 0.0;
        for (uint64_t k = t; k < R.nitems; k += blockDim.x)
          s = __dadd_rn(s, __ldcg(A.partials + R.first_item + k));
        s = team_reduce<CombF64>(s, s_scr);
        if (t == 0) {
          *R.result = s;
          A.tickets[r] = 0;  // ready for the next launch
        }
      }
    }
    team_barrier();  // s_item / s_last are reused by the next claim
  }
  if (t == 0) {
    const uint32_t left = atomic_add(A.exits, 1u);
    if (left == gridDim.x - 1) {  // every other CTA has made its final claim
      *A.head = 0;
      *A.exits = 0;
    }
  }
}

}  // namespace rt

using namespace rt;

struct omprt_batch {
  omprt_ctx* ctx = nullptr;
  int64_t nitems = 0;
  int32_t nregions = 0;
  uint64_t chunk = 0;
  BatchRegion* regions_dev = nullptr;
  uint32_t* item_region_dev = nullptr;
  double* partials_dev = nullptr;
  uint32_t* tickets_dev = nullptr;
  unsigned long long* head_dev = nullptr;  // head and exit count share one allocation
};

static void batch_free(omprt_batch* b) {
  cudaFree(b->regions_dev);
  cudaFree(b->item_region_dev);
  cudaFree(b->partials_dev);
  cudaFree(b->tickets_dev);
  cudaFree(b->head_dev);
  delete b;
}

extern "C" {

omprt_status omprt_batch_create(omprt_ctx* c, const omprt_loop_desc* descs,
                                const omprt_reduce_desc* reds, int32_t nregions,
                                int64_t chunk_elems, omprt_batch** out) {
  if (!c) return OMPRT_ERR_NOT_INIT;
  if (!descs || !out || nregions < 1) return OMPRT_ERR_INVALID;
  if (chunk_elems == 0) chunk_elems = 8192;
  if (chunk_elems < 256 || chunk_elems % 256) return OMPRT_ERR_INVALID;
  std::vector<BatchRegion> regs(nregions);
  std::vector<uint32_t> item_region;
  uint64_t items = 0;
  for (int32_t r = 0; r < nregions; ++r) {
    const omprt_loop_desc& d = descs[r];
    uint64_t n;
    int64_t lb;
    omprt_status s = loop_trip_count(&d, &n, &lb);
    if (s) return s;
    if (d.lb != 0 || d.incr != 1 || d.data_type != OMPRT_F32 || d.reserved || d.seq)
      return OMPRT_ERR_INVALID;
    const bool red = reds && reds[r].result_dev;
    if (red && (reds[r].op != OMPRT_OP_SUM || reds[r].precision != OMPRT_PREC_COMP_F64))
      return OMPRT_ERR_UNSUPPORTED;
    switch (d.body) {
      case OMPRT_BODY_AXPY:
        if (n && (!d.x || !d.y)) return OMPRT_ERR_INVALID;
        break;
      case OMPRT_BODY_DOT:
        if (!red || (n && (!d.x || !d.y))) return OMPRT_ERR_INVALID;
        break;
      case OMPRT_BODY_STENCIL1D3:
        if (n && (!d.x || !d.out || d.x == d.out)) return OMPRT_ERR_INVALID;
        break;
      default:
        return OMPRT_ERR_UNSUPPORTED;
    }
    BatchRegion& R = regs[r];
    std::memset(&R, 0, sizeof(R));
    R.body = d.body;
    R.has_red = red ? 1 : 0;
    R.n = n;
    R.x = d.x;
    R.y = d.y;
    R.out = d.out;
    R.alpha = (float)d.alpha;
    R.c0 = (float)d.c0;
    R.c1 = (float)d.c1;
    // an empty region still gets one (empty) item so its reduction completes
    const uint64_t ni = n ? (n - 1) / (uint64_t)chunk_elems + 1 : 1;
    if (ni > 0xffffffffull || items + ni > (1ull << 32)) return OMPRT_ERR_UNSUPPORTED;
    R.nitems = (uint32_t)ni;
    R.first_item = items;
    R.result = red ? (double*)reds[r].result_dev : nullptr;
    items += ni;
    item_region.insert(item_region.end(), ni, (uint32_t)r);
  }
  DeviceGuard guard(c->device);
  omprt_batch* b = new (std::nothrow) omprt_batch();
  if (!b) return OMPRT_ERR_NOMEM;
  b->ctx = c;
  b->nitems = (int64_t)items;
  b->nregions = nregions;
  b->chunk = (uint64_t)chunk_elems;
  bool ok = cudaMalloc(&b->regions_dev, sizeof(BatchRegion) * nregions) == cudaSuccess &&
            cudaMalloc(&b->item_region_dev, sizeof(uint32_t) * items) == cudaSuccess &&
            cudaMalloc(&b->partials_dev, sizeof(double) * items) == cudaSuccess &&
            cudaMalloc(&b->tickets_dev, sizeof(uint32_t) * nregions) == cudaSuccess &&
            cudaMalloc(&b->head_dev, 256) == cudaSuccess;
  ok = ok &&
       cudaMemcpy(b->regions_dev, regs.data(), sizeof(BatchRegion) * nregions,
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->item_region_dev, item_region.data(), sizeof(uint32_t) * items,
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(b->tickets_dev, 0, sizeof(uint32_t) * nregions) == cudaSuccess &&
       cudaMemset(b->head_dev, 0, 256) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    batch_free(b);
    return OMPRT_ERR_NOMEM;
  }
  *out = b;
  return OMPRT_OK;
}

omprt_status omprt_launch_batch(omprt_batch* b, int32_t num_ctas, int32_t threads, void* stream) {
  if (!b || !b->ctx) return OMPRT_ERR_NOT_INIT;
  if (threads == 0) threads = 256;
  if (threads < 64 || threads > 1024 || threads % 32 || num_ctas < 0) return OMPRT_ERR_INVALID;
  DeviceGuard guard(b->ctx->device);
  OverlapScope overlap(b->ctx->launch_overlap, (size_t)b->ctx->smem_per_sm);
  if (num_ctas == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, threads, 0) !=
        cudaSuccess)
      return OMPRT_ERR_CUDA;
    num_ctas = per_sm * b->ctx->sm_count;
  }
  if (num_ctas < 1) return OMPRT_ERR_INVALID;
  BatchArgs a;
  a.regions = b->regions_dev;
  a.item_region = b->item_region_dev;
  a.nitems = (uint64_t)b->nitems;
  a.chunk = b->chunk;
  a.partials = b->partials_dev;
  a.tickets = b->tickets_dev;
  a.head = b->head_dev;
  a.exits = (uint32_t*)(b->head_dev + 1);
  a.status = b->ctx->status_dev;
  const cudaError_t e =
      launch_kernel(batch_kernel, dim3(num_ctas), dim3(threads), 0, (cudaStream_t)stream, a);
  return e == cudaSuccess ? OMPRT_OK : OMPRT_ERR_CUDA;
}

omprt_status omprt_batch_destroy(omprt_batch* b) {
  if (!b) return OMPRT_ERR_NOT_INIT;
  DeviceGuard guard(b->ctx->device);
  batch_free(b);
  return OMPRT_OK;
}

int64_t omprt_batch_items(const omprt_batch* b) { return b ? b->nitems : 0; }

}  // extern "C"
