// The 2-D 5-point stencil under dynamic(c) when every team's block is whole
// grid rows (G divides ny) and every chunk starts on a 16-byte boundary (c
// and nx multiples of 4).
//
// A launch has P <= G resident CTAs; CTA k plays the consecutive teams
// [k G / P, (k + 1) G / P) (OpenMP does not make teams run at the same time),
// whose blocks are the grid rows [R0, R1).  The rows R0 - 1 .. R1 (those in
// the grid) stream through a ring of S row slots in shared memory: a producer
// warp copies stream row i into slot i mod S with one bulk copy as soon as
// every group of the CTA has released the row the slot held before.  The
// CTA's K T threads form K groups of T; group gr plays the CTA's teams
// gr, gr + K, ... one at a time, its thread tt as the team's thread tt.  A
// team waits for the rows its block and the block's neighbour rows lie in,
// runs, ends in the group's barrier, and the group's leader then releases
// the rows the group will not read again.
//
// Inside a team's block (R rows, B = R nx points) lane 0 of a warp claims the
// next 32 chunks with one atomic add on the team's counter (in shared memory;
// a team is run by one group), lane l runs chunk base + l; a thread's claims
// increase (C4, monotonic).  A chunk runs row by row (it crosses a row end
// only where c does not divide nx); its piece of a row runs in 16-byte units:
// the rows above / at / below are read with 128-bit shared-memory loads
// through three row pointers fixed for the piece, west / east are carried
// from unit to unit, and the four outputs leave in one 128-bit store.  The
// lanes of a warp hold chunks c floats apart, so each starts its walk at a
// rotated unit and wraps to the piece's first unit, which puts the eight
// lanes of a 128-bit access phase on distinct 16-byte bank groups (the
// stencil's iterations are independent: a thread's order inside a chunk is
// not observable).  Boundary rows and columns are copied; the arithmetic is
// the body's fma(c1, (N+S)+(E+W), c0*C).  Every ring index is a slot number
// below S times the slot pitch plus a column below nx.
#include "api_internal.h"

namespace rt {

constexpr uint32_t kRrMaxGroups = 15;  // named barriers 1 .. 15, one per group
constexpr uint32_t kRrMaxSlots = 64;
constexpr uint64_t kRrWaitNs = 1000000000ull;  // 1 s: a team takes microseconds

struct RowRingArgs {
  const float* in;
  float* out;
  uint32_t nx, ny;  // nx * ny < 2^32, nx a multiple of 4
  uint32_t G, R;    // teams; rows per team block (G R = ny)
  uint32_t T, K;    // threads of a team (a multiple of 32); groups per CTA
  uint32_t chunk;   // c: a multiple of 4, at most R nx
  uint32_t slots;   // S: rows the ring holds
  uint32_t pitch;   // floats per slot: nx rounded up to 32 (128-byte slots)
  float c0, c1;
  uint32_t* status;
};

__device__ __forceinline__ float rr_point(float c0, float c1, float nn, float ss, float e, float w,
                                          float c) {
  return __fmaf_rn(c1, __fadd_rn(__fadd_rn(nn, ss), __fadd_rn(e, w)), __fmul_rn(c0, c));
}

__device__ __forceinline__ float4 rr_lds(const float* p) { return *(const float4*)p; }

__device__ __forceinline__ void rr_stg(float* p, float4 v) {
  asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

// the four outputs of a unit in an interior row, from its row c, the rows
// above / below nn / ss and its west / east neighbours w / e
__device__ __forceinline__ float4 rr_unit(float c0, float c1, float4 nn, float4 ss, float4 c,
                                          float w, float e) {
  float4 o;
  o.x = rr_point(c0, c1, nn.x, ss.x, c.y, w, c.x);
  o.y = rr_point(c0, c1, nn.y, ss.y, c.z, c.x, c.y);
  o.z = rr_point(c0, c1, nn.z, ss.z, c.w, c.y, c.z);
  o.w = rr_point(c0, c1, nn.w, ss.w, e, c.z, c.w);
  return o;
}

// Units [u0, u1) (u0 < u1) of a piece of an interior row whose unit 0 is
// column col0: pn / pc / ps point at column col0 of the rows above / at /
// below in the ring, po at column col0 of the output row.  Column 0 can only
// be the first unit of a run (u0 = 0, col0 = 0) and column nx - 1 only the
// last (the piece's last unit), so only those two units test for them.
__device__ __forceinline__ void rr_run(float c0, float c1, uint32_t nx, const float* pn,
                                       const float* pc, const float* ps, float* po, uint32_t col0,
                                       uint32_t u0, uint32_t u1) {
  uint32_t u = u0;
  float4 c = rr_lds(pc + 4 * u);
  float w = 0.f;
  if (col0 + 4 * u == 0) {  // the row's first unit: column 0 is copied
    if (u + 1 == u1) {      // and the run's last
      const float e = 4 < nx ? pc[4] : 0.f;
      float4 o = rr_unit(c0, c1, rr_lds(pn), rr_lds(ps), c, 0.f, e);
      o.x = c.x;
      if (4 == nx) o.w = c.w;
      rr_stg(po, o);
      return;
    }
    const float4 cn = rr_lds(pc + 4);
    float4 o = rr_unit(c0, c1, rr_lds(pn), rr_lds(ps), c, 0.f, cn.x);
    o.x = c.x;
    rr_stg(po, o);
    w = c.w;
    c = cn;
    ++u;
  } else {
    w = (pc + 4 * u)[-1];  // column col0 + 4 u - 1 >= 0 of the same row
  }
#pragma unroll 2
  for (; u + 1 < u1; ++u) {
    const float4 cn = rr_lds(pc + 4 * u + 4);
    const float4 nn = rr_lds(pn + 4 * u), ss = rr_lds(ps + 4 * u);
    rr_stg(po + 4 * u, rr_unit(c0, c1, nn, ss, c, w, cn.x));
    w = c.w;
    c = cn;
  }
  // the run's last unit, u = u1 - 1
  const uint32_t col = col0 + 4 * u;
  const float e = col + 4 < nx ? pc[4 * u + 4] : 0.f;
  float4 o = rr_unit(c0, c1, rr_lds(pn + 4 * u), rr_lds(ps + 4 * u), c, w, e);
  if (col + 4 == nx) o.w = c.w;
  rr_stg(po + 4 * u, o);
}

__device__ __forceinline__ const float* rr_slot(const RowRingArgs& A, const float* ring,
                                                uint32_t rb, uint32_t r) {
  return ring + (size_t)((r - rb) % A.slots) * A.pitch;
}

// The nu units of row r from column col0 (a multiple of 4) on.
__device__ __forceinline__ void rr_piece(const RowRingArgs& A, const float* ring, uint32_t rb,
                                         uint32_t r, uint32_t col0, uint32_t nu, uint32_t lane) {
  const float* pc = rr_slot(A, ring, rb, r) + col0;
  float* po = A.out + (size_t)r * A.nx + col0;
  if (r == 0 || r + 1 == A.ny) {  // a boundary row is copied
    for (uint32_t u = 0; u < nu; ++u) rr_stg(po + 4 * u, rr_lds(pc + 4 * u));
    return;
  }
  const float* pn = rr_slot(A, ring, rb, r - 1) + col0;
  const float* ps = rr_slot(A, ring, rb, r + 1) + col0;
  // lanes whose pieces sit nu units apart: 2^s = gcd(nu, 8) of every 8 lanes
  // of an access phase start in the same bank group, so they are spread over
  // 2^s starting units (off < 2^s <= nu)
  const uint32_t s = nu & 7u ? (uint32_t)(__ffs((int)(nu & 7u)) - 1) : 3u;
  const uint32_t off = ((lane & 7u) >> (3u - s)) & ((1u << s) - 1u);
  rr_run(A.c0, A.c1, A.nx, pn, pc, ps, po, col0, off, nu);
  if (off) rr_run(A.c0, A.c1, A.nx, pn, pc, ps, po, col0, 0, off);
}

// Points [lo, hi) of the block starting at row row0 (lo, hi multiples of 4),
// row by row.
__device__ __forceinline__ void rr_chunk(const RowRingArgs& A, const float* ring, uint32_t rb,
                                         uint32_t row0, uint32_t lo, uint32_t hi, uint32_t lane) {
  const uint32_t nx = A.nx;
  const uint32_t dr = lo / nx;
  uint32_t r = row0 + dr, col = lo - dr * nx;
  while (lo < hi) {
    const uint32_t len = hi - lo < nx - col ? hi - lo : nx - col;
    rr_piece(A, ring, rb, r, col, len >> 2, lane);
    lo += len;
    ++r;
    col = 0;
  }
}

__global__ void __launch_bounds__(1024) stencil2d_rowring_kernel(const RowRingArgs A) {
  enter_region_grid();
  __shared__ __align__(8) uint64_t full[kRrMaxSlots], empty[kRrMaxSlots];
  __shared__ uint32_t ctr[kRrMaxGroups][2];  // dynamic: each group's claim counters
  __shared__ int s_bad;
  // the ring on a 128-byte boundary, addressed from the shared array itself so
  // that every access compiles to a shared-memory load
  float* const ring = (float*)(rt_dyn_smem + ((128u - (smem_addr(rt_dyn_smem) & 127u)) & 127u));
  const uint32_t t = threadIdx.x, lane = t & 31u;
  const uint32_t T = A.T, K = A.K, gr = t / T, tt = t - gr * T;
  const uint32_t P = gridDim.x, k = blockIdx.x;
  const uint32_t g0 = (uint32_t)((uint64_t)k * A.G / P);
  const uint32_t g1 = (uint32_t)((uint64_t)(k + 1) * A.G / P);
  if (g0 >= g1) return;  // uniform; never with P <= G
  const uint32_t nx = A.nx, ny = A.ny, R = A.R, S = A.slots;
  // this CTA's stream: its blocks' rows and one row on each side
  const uint32_t rb = g0 * R > 0 ? g0 * R - 1 : 0u;
  const uint32_t re = g1 * R < ny ? g1 * R + 1 : ny;
  const uint32_t nrows = re - rb;
  const uint32_t full0 = smem_addr(&full[0]), empty0 = smem_addr(&empty[0]);
  if (t == 0) {
    for (uint32_t i = 0; i < S; ++i) {
      mbar_init(full0 + 8 * i);            // one arrival (with the bytes) per fill
      mbar_init_count(empty0 + 8 * i, K);  // one arrival per group per release
    }
    s_bad = 0;
  }
  if (t < 2 * kRrMaxGroups) ctr[t >> 1][t & 1] = 0;
  __syncthreads();
  // the stream rows [row_lo(g), row_hi(g)) team g's block and neighbours lie in
  auto row_lo = [&](uint32_t g) { return (g * R > 0 ? g * R - 1 : 0u) - rb; };
  auto row_hi = [&](uint32_t g) { return ((g + 1) * R < ny ? (g + 1) * R + 1 : ny) - rb; };
  if (t >= K * T) {  // the producer warp
    if (lane == 0) {
      // fill slot i % S with stream row i once every group has released row i - S
      uint32_t i = 0;
      for (; i < nrows && !*(volatile int*)&s_bad; ++i) {
        if (i >= S &&
            !mbar_wait(empty0 + 8 * (i % S), ((i / S) - 1) & 1u, kRrWaitNs, A.status)) {
          s_bad = 1;
          break;
        }
        mbar_expect_tx(full0 + 8 * (i % S), nx * 4u);
        bulk_g2s(ring + (size_t)(i % S) * A.pitch, A.in + (size_t)(rb + i) * nx, nx * 4u,
                 full0 + 8 * (i % S));
      }
      // no copy may still be landing when the CTA leaves: wait for the last
      // fill of every slot
      for (uint32_t j = i > S ? i - S : 0; j < i; ++j)
        mbar_wait(full0 + 8 * (j % S), (j / S) & 1u, kRrWaitNs, nullptr);
    }
  } else {
    uint32_t waited = 0;    // every thread: rows [0, waited) seen filled
    uint32_t released = 0;  // the group's leader: rows [0, released) released
    uint32_t j = 0;         // the group's team count (dynamic counter parity)
    // the group's barrier; every member gets the same answer to "has any
    // member seen the give-up flag", so the group stops as one
    auto group_sync_stop = [&]() {
      const bool v = *(volatile int*)&s_bad != 0;
      if (T == 32) {
        __syncwarp();
        return __any_sync(0xffffffffu, v) != 0;
      }
      return named_barrier_or(1 + gr, T, v);
    };
    // the leader releases rows [released, upto): each after it is seen
    // filled, so an arrival always counts for the row in the slot
    auto release = [&](uint32_t upto) {
      if (tt == 0) {
        for (; released < upto; ++released) {
          if (!mbar_wait(full0 + 8 * (released % S), (released / S) & 1u, kRrWaitNs,
                         A.status)) {
            s_bad = 1;
            break;
          }
          mbar_arrive(empty0 + 8 * (released % S));
        }
      }
    };
    const uint32_t B = R * nx, c = A.chunk;
    for (uint32_t g = g0 + gr; g < g1; g += K, ++j) {  // group gr plays team g
      const uint32_t hi = row_hi(g);
      if (waited < row_lo(g)) waited = row_lo(g);  // rows below are never read here
      bool ok = !*(volatile int*)&s_bad;
      while (ok && waited < hi) {
        if (!mbar_wait(full0 + 8 * (waited % S), (waited / S) & 1u, kRrWaitNs, A.status)) {
          ok = false;
          s_bad = 1;
          break;
        }
        ++waited;
      }
      ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the dynamic claims are warp-wide
      if (ok) {
        const uint32_t row0 = g * R;
        {
          const uint32_t nch = (uint32_t)(((uint64_t)B + c - 1) / c);
          uint32_t* const cp = &ctr[gr][j & 1u];
          for (;;) {
            uint32_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(cp, 32u);
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (b0 >= nch) break;
            const uint32_t jj = b0 + lane;
            if (jj < nch) {
              const uint32_t lo = jj * c;
              const uint32_t hi2 = B - lo > c ? lo + c : B;
              rr_chunk(A, ring, rb, row0, lo, hi2, lane);
            }
          }
        }
      }
      // the team is done: its rows are read out, its counter idle
      const bool stop = group_sync_stop();
      // this counter serves the team after next; the rows below the next
      // team's go back to the producer
      if (tt == 0) ctr[gr][j & 1u] = 0;
      if (stop) break;
      release(g + K < g1 ? row_lo(g + K) : nrows);
    }
    if (!*(volatile int*)&s_bad) release(nrows);  // what this group will not read any more
  }
  __syncthreads();
}

// cudaErrorNotSupported (nothing launched) where this form does not apply:
// a schedule other than dynamic(c); c not a multiple of 4; nx not a
// multiple of 4; teams not dividing ny (team
// blocks of whole rows); n = 0 or n >= 2^32; teams of more than 512 threads
// or not whole warps; pointers not 16-byte aligned; or a ring of `budget`
// bytes that holds fewer than R + 3 rows (one team's rows, its neighbour
// rows and one fill in flight).
cudaError_t launch_stencil2d_rowring(const void* in, float* out, uint64_t nx, uint64_t ny,
                                     int sched, uint64_t chunk, float c0, float c1,
                                     unsigned teams, unsigned threads, uint32_t budget,
                                     int sm_count, int max_smem, uint32_t* status,
                                     cudaStream_t st) {
  const uint64_t n = nx * ny;
  if (sched != kDynamic || budget == 0 || nx < 4 || nx % 4 || ny < 1 ||
      n == 0 || n >= (1ull << 32) || teams < 1 || teams > ny || ny % teams || threads < 32 ||
      threads > 512 || threads % 32 || (((uintptr_t)in | (uintptr_t)out) & 15))
    return cudaErrorNotSupported;
  if (chunk < 4 || chunk % 4) return cudaErrorNotSupported;
  const uint64_t R = ny / teams, B = R * nx;
  RowRingArgs a;
  a.in = (const float*)in;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.G = teams;
  a.R = (uint32_t)R;
  a.T = threads;
  // a chunk of at least a whole block is one chunk per block (B is a
  // multiple of 4, so c stays one)
  a.chunk = (uint32_t)(chunk < B ? chunk : B);
  a.c0 = c0;
  a.c1 = c1;
  a.status = status;
  auto* kern = stencil2d_rowring_kernel;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  // the ring and the kernel's own shared variables within the opt-in limit
  const uint64_t room = (uint64_t)max_smem > fa.sharedSizeBytes
                            ? (uint64_t)max_smem - fa.sharedSizeBytes
                            : 0;
  const uint64_t pitch = (nx + 31) / 32 * 32;
  const uint64_t cap = budget < room ? budget : room;
  uint64_t S = (cap > 256 ? cap - 256 : 0) / (4 * pitch);
  if (S > kRrMaxSlots) S = kRrMaxSlots;
  if (S < R + 3) return cudaErrorNotSupported;
  // K groups at work on K consecutive teams need K R + 2 rows at once; K is
  // the largest that leaves a quarter of the ring (at least two rows) for the
  // fills in flight, and fits 1024 threads with the producer warp
  const uint64_t spare = S / 4 > 2 ? S / 4 : 2;
  const uint64_t kmax =
      (1024 - 32) / threads < kRrMaxGroups ? (1024 - 32) / threads : kRrMaxGroups;
  uint64_t K = 1;
  while (K < kmax && (K + 1) * R + 2 + spare <= S) ++K;
  a.slots = (uint32_t)S;
  a.pitch = (uint32_t)pitch;
  const size_t smem = (size_t)(S * pitch * 4 + 128);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)(K * threads + 32), smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  // resident CTAs, and no more groups than a CTA has teams
  uint64_t P = (uint64_t)per_sm * (uint64_t)sm_count;
  if (P > teams) P = teams;
  const uint64_t per_cta = teams / P;  // every CTA has at least this many teams
  if (K > per_cta) K = per_cta;
  a.K = (uint32_t)K;
  return launch_kernel(kern, dim3((unsigned)P), dim3((unsigned)(K * threads + 32)), smem, st, a);
}

}  // namespace rt
