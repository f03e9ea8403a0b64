// Static schedules of the 2-D stencil whose owner map repeats row by row,
// run as vertical strips.
//
// When every team's block is whole rows and the schedule's period divides
// the row length, a thread owns the same columns in every row of the grid:
//   static(1), T | nx:           columns tt + k T       (k < M = nx / T)
//   static(c), c in {4, 8}, cT | nx: columns c (tt + k T) + [0, c)
//   static (no chunk), one row per team, p = nx / T in {1, 4, 8}:
//                                columns p tt + [0, p)
// (W = 1, c or p columns per strip, M strips per thread; chunk numbering
// restarts at each block, which starts a row.)  In every row the thread's
// iterations are its strips' points from left to right, and its next
// iterations are the same columns one row down, so the thread walks its
// strips down the rows (the CTAs of even index in exactly the order OpenMP
// gives it, those of odd index bottom up, see below), with the rows above,
// at and below in registers: each step loads one new row of
// its strips (the row after next, one step ahead) and takes the column west /
// east of each strip from the neighbouring lane by shuffle (the lane beyond a
// warp's edge loads it).  A warp's loads and stores cover contiguous memory.
// A launch has P <= G resident CTAs; CTA k plays the consecutive teams
// [k G / P, (k + 1) G / P), that is a contiguous band of rows, with its thread
// tt as thread tt of each of those teams (OpenMP does not make teams run at
// the same time).  The arithmetic is the body's: fma(c1, (N+S)+(E+W), c0*C),
// boundary points copied.
#include "api_internal.h"

namespace rt {

struct StripArgs {
  const float* in;
  float* out;
  uint32_t nx, ny;
  uint32_t G;              // teams
  uint32_t rows_per_team;  // every block is this many whole rows
  float c0, c1;
};

__device__ __forceinline__ float strip_point(const StripArgs& A, float nn, float ss, float e,
                                             float w, float c) {
  return __fmaf_rn(A.c1, __fadd_rn(__fadd_rn(nn, ss), __fadd_rn(e, w)), __fmul_rn(A.c0, c));
}

// W consecutive floats at p (W = 1, 4 or 8; p aligned to W floats)
template <int W>
__device__ __forceinline__ void strip_load(const float* p, float (&v)[W]) {
  if constexpr (W == 8) {
    uint32_t r[8];
    ld8_nc(p, r);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = as_f(r[k]);
  } else if constexpr (W == 4) {
    const float4 q = __ldg((const float4*)p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    v[0] = __ldg(p);
  }
}
template <int W>
__device__ __forceinline__ void strip_store(float* p, const float (&v)[W]) {
  if constexpr (W == 8) {
    uint32_t r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = as_u(v[k]);
    st8(p, r);
  } else if constexpr (W == 4) {
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
  } else {
    *p = v[0];
  }
}

// D: rows loaded ahead of the one being computed (the loads of rows r + 2 ..
// r + 1 + D are in flight while row r computes).
template <int W, int M, int D>
__global__ void __launch_bounds__(1024) stencil2d_strips_kernel(const StripArgs A) {
  enter_region_grid();
  const uint32_t t = threadIdx.x, T = blockDim.x, lane = t & 31u;
  const uint32_t P = gridDim.x, k = blockIdx.x;
  const uint32_t nx = A.nx, ny = A.ny;
  const uint32_t R0 = (uint32_t)((uint64_t)k * A.G / P) * A.rows_per_team;
  const uint32_t R1 = (uint32_t)((uint64_t)(k + 1) * A.G / P) * A.rows_per_team;
  if (R0 >= R1) return;
  uint32_t col[M];  // first column of each strip
#pragma unroll
  for (int m = 0; m < M; ++m) col[m] = (uint32_t)W * (t + (uint32_t)m * T);
  // Odd CTAs walk their band bottom up.  A row on the boundary of two bands
  // is read by both CTAs; with the walks in opposite directions both reads
  // come at the start of the two walks or both at the end, so the second
  // finds the row still in L2 (top-down walks read it a whole band apart,
  // after the L2 has turned over: 2 rows a band from DRAM again, 14% of the
  // input at 4096^2).  A thread's iterations are independent, so the order
  // of its rows is not observable.  (n < 2^32 and nx >= 32 keep rows in int.)
  const int dir = (k & 1u) ? -1 : 1;
  const int first = dir > 0 ? (int)R0 : (int)R1 - 1;
  // a row the band reads: inside the grid and at most one row beyond the band
  auto readable = [&](int r) {
    return r >= 0 && r < (int)ny && r >= (int)R0 - 1 && r <= (int)R1;
  };
  // v[0] the row behind (above when walking down), v[1] the row being
  // computed, v[2 ..] the rows ahead
  float v[D + 2][M][W];
  auto load_row = [&](int r, float (&x)[M][W]) {
#pragma unroll
    for (int m = 0; m < M; ++m) strip_load<W>(A.in + (size_t)r * nx + col[m], x[m]);
  };
  if (readable(first - dir)) load_row(first - dir, v[0]);
  load_row(first, v[1]);
#pragma unroll
  for (int d = 2; d < D + 2; ++d)  // the D rows ahead of the first, those the band reads
    if (readable(first + (d - 1) * dir)) load_row(first + (d - 1) * dir, v[d]);
  for (uint32_t i = 0; i < R1 - R0; ++i) {
    const uint32_t r = (uint32_t)(first + (int)i * dir);
    float nxt[M][W];
    // the row 1 + D ahead, needed D steps from now
    const int ahead = (int)r + (1 + D) * dir;
    const bool more = readable(ahead);
    if (more) load_row(ahead, nxt);
    const bool inner = r >= 1 && r + 1 < ny;
    const size_t row = (size_t)r * nx;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      // west / east of the strip: the neighbouring lanes' edge values; the
      // lanes at a warp's edge read theirs (columns 0 and nx - 1 are copied)
      float w = __shfl_up_sync(0xffffffffu, v[1][m][W - 1], 1);
      float e = __shfl_down_sync(0xffffffffu, v[1][m][0], 1);
      if (inner && lane == 0 && col[m] > 0) w = __ldg(A.in + row + col[m] - 1);
      if (inner && lane == 31 && col[m] + W < nx) e = __ldg(A.in + row + col[m] + W);
      float o[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const uint32_t cc = col[m] + q;
        const float ww = q > 0 ? v[1][m][q - 1] : w;
        const float ee = q + 1 < W ? v[1][m][q + 1] : e;
        // behind + ahead is N + S in either direction (the sum commutes)
        o[q] = (inner && cc > 0 && cc + 1 < nx)
                   ? strip_point(A, v[0][m][q], v[2][m][q], ee, ww, v[1][m][q])
                   : v[1][m][q];
      }
      strip_store<W>(A.out + row + col[m], o);
    }
#pragma unroll
    for (int d = 0; d < D + 1; ++d)
#pragma unroll
      for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < W; ++q) v[d][m][q] = v[d + 1][m][q];
    if (more) {
#pragma unroll
      for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < W; ++q) v[D + 1][m][q] = nxt[m][q];
    }
  }
}

// cudaErrorNotSupported (nothing launched) unless the owner map is one of the
// row-periodic forms above: n < 2^32, G dividing ny (whole-row blocks),
// thread counts with the period dividing nx, W M <= 8 floats a row, and the
// pointers aligned to the strip's vector.
cudaError_t launch_stencil2d_strips(const void* in, float* out, uint64_t nx, uint64_t ny, int sched,
                                    uint64_t chunk, float c0, float c1, unsigned teams,
                                    unsigned threads, int sm_count, cudaStream_t st) {
  const uint64_t n = nx * ny;
  if (n == 0 || n >= (1ull << 32) || teams < 1 || teams > ny || ny % teams || threads < 32 ||
      threads % 32 || nx % threads)
    return cudaErrorNotSupported;
  const uint64_t rpt = ny / teams;
  uint32_t W = 0, M = 0;
  if (sched == kChunked && chunk == 1) {
    W = 1;
    M = (uint32_t)(nx / threads);
  } else if (sched == kChunked && (chunk == 4 || chunk == 8)) {
    if (nx % (chunk * threads)) return cudaErrorNotSupported;
    W = (uint32_t)chunk;
    M = (uint32_t)(nx / (chunk * threads));
  } else if (sched == kStatic && rpt == 1) {
    W = (uint32_t)(nx / threads);
    M = 1;
  } else {
    return cudaErrorNotSupported;
  }
  if ((uintptr_t)in % (4 * W) || (uintptr_t)out % (4 * W)) return cudaErrorNotSupported;
  StripArgs a;
  a.in = (const float*)in;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.G = teams;
  a.rows_per_team = (uint32_t)rpt;
  a.c0 = c0;
  a.c1 = c1;
  // two rows ahead where a thread's row is at most four floats, else one
  void (*kern)(StripArgs) = nullptr;
  if (W == 1 && M == 1) kern = stencil2d_strips_kernel<1, 1, 2>;
  if (W == 1 && M == 2) kern = stencil2d_strips_kernel<1, 2, 2>;
  if (W == 1 && M == 4) kern = stencil2d_strips_kernel<1, 4, 2>;
  if (W == 1 && M == 8) kern = stencil2d_strips_kernel<1, 8, 1>;
  if (W == 4 && M == 1) kern = stencil2d_strips_kernel<4, 1, 2>;
  if (W == 4 && M == 2) kern = stencil2d_strips_kernel<4, 2, 1>;
  if (W == 8 && M == 1) kern = stencil2d_strips_kernel<8, 1, 1>;
  if (!kern) return cudaErrorNotSupported;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  uint64_t P = (uint64_t)per_sm * (uint64_t)sm_count;
  if (P > teams) P = teams;
  return launch_kernel(kern, dim3((unsigned)P), dim3(threads), 0, st, a);
}

}  // namespace rt
