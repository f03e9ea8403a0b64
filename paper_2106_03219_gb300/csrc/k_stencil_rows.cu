// static(c) schedules of the 2-D 5-point stencil, with the team's rows staged
// through a ring in shared memory.
//
// Under static(c) a team's block (level 1) and every thread's chunks of it
// (level 2: the chunks j with j mod T == t) are fixed, and the team can walk
// its block row by row.  It does so in passes of K grid rows.  The rows a
// pass reads (one above to one below its K rows) sit in a ring of 2K + 2 row
// slots: the two halo rows of a pass are the last two rows of the previous
// one, so each grid row is copied in once per team (one bulk copy of nx
// floats), and the K rows of the next pass are copied in while the current
// pass computes.  In every pass each thread runs exactly its chunks' part of
// the pass, in 16-byte units where its piece allows (a unit never straddles
// rows: nx is a multiple of 4): three 128-bit reads of the ring (the rows
// above, at and below), two scalar reads for the columns west and east of the
// unit, one 128-bit store of the four outputs; the few iterations before a
// piece's first 16-byte boundary and after its last run one at a time.  The
// lanes walk their units from rotated starting points so that the eight lanes
// of a 128-bit access phase hit distinct bank groups.  The arithmetic is the
// body's: fma(c1, (N+S)+(E+W), c0*C), boundary points copied.
//
// Measured on GB300 (4096^2 and 8192^2 grids, best teams x threads of each
// form) against the plain static(c) kernel, whose lanes read their chunks
// straight from global memory: c = 4 +28% / +35%, c = 32 +38% / +30%,
// c = 64 +39% / +35%, c = 128 +23% / +8%.  The plain form keeps c < 4 (no
// 16-byte units), c = 8 and 16 (a warp's 32 chunks span at most 2 KB and
// its 256-bit loads coalesce: the ring lost 14-26% at c = 8) and c > 128 (a
// long chunk walked by one lane per pass: the ring lost at c = 512).
#include "api_internal.h"

namespace rt {

constexpr uint64_t kRowsWaitNs = 1000000000ull;  // 1 s: a pass takes microseconds

struct RowsArgs {
  const float* in;
  float* out;
  uint32_t nx, ny;
  uint64_t n;
  uint64_t chunk;
  uint64_t nx_magic;     // ceil(2^64 / nx): row of i < 2^32 is umulhi(i, magic)
  uint32_t K;            // grid rows per pass
  uint32_t slot_floats;  // floats per ring slot (nx rounded up to 32)
  float c0, c1;
  uint32_t* status;
};

__device__ __forceinline__ float rows_point(const RowsArgs& A, float nn, float ss, float e,
                                            float w, float c) {
  return __fmaf_rn(A.c1, __fadd_rn(__fadd_rn(nn, ss), __fadd_rn(e, w)), __fmul_rn(A.c0, c));
}

// One output point i (global index, row r, column col) from the ring; rows
// r - 1 .. r + 1 are in slots sm, sc, sp.
__device__ __forceinline__ void rows_one(const RowsArgs& A, const float* ring, uint64_t i,
                                         uint32_t r, uint32_t col, uint32_t sm, uint32_t sc,
                                         uint32_t sp) {
  const float* crow = ring + (size_t)sc * A.slot_floats;
  const float c = crow[col];
  float v = c;
  if (r > 0 && r + 1 < A.ny && col > 0 && col + 1 < A.nx) {
    const float nn = ring[(size_t)sm * A.slot_floats + col];
    const float ss = ring[(size_t)sp * A.slot_floats + col];
    v = rows_point(A, nn, ss, crow[col + 1], crow[col - 1], c);
  }
  A.out[i] = v;
}

// Four outputs gi .. gi+3 (gi % 4 == 0: one row r, columns col .. col+3).
__device__ __forceinline__ void rows_unit(const RowsArgs& A, const float* ring, uint64_t gi,
                                          uint32_t r, uint32_t col, uint32_t sm, uint32_t sc,
                                          uint32_t sp) {
  const float* crow = ring + (size_t)sc * A.slot_floats;
  const float4 cc = *(const float4*)(crow + col);
  float4 o = cc;  // boundary rows are copied
  if (r > 0 && r + 1 < A.ny) {
    const float4 nn = *(const float4*)(ring + (size_t)sm * A.slot_floats + col);
    const float4 ss = *(const float4*)(ring + (size_t)sp * A.slot_floats + col);
    // of the four columns only col (== 0) and col + 3 (== nx - 1) can be boundary
    if (col > 0) o.x = rows_point(A, nn.x, ss.x, cc.y, crow[col - 1], cc.x);
    o.y = rows_point(A, nn.y, ss.y, cc.z, cc.x, cc.y);
    o.z = rows_point(A, nn.z, ss.z, cc.w, cc.y, cc.z);
    if (col + 4 < A.nx) o.w = rows_point(A, nn.w, ss.w, crow[col + 4], cc.z, cc.w);
  }
  asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(A.out + gi), "f"(o.x), "f"(o.y),
               "f"(o.z), "f"(o.w)
               : "memory");
}

__global__ void __launch_bounds__(1024) stencil2d_rows_kernel(const RowsArgs A) {
  enter_region_grid();
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_bad;
  float* const ring = (float*)rt_dyn_smem;  // 2K + 2 slots of slot_floats
  const uint32_t t = threadIdx.x, T = blockDim.x, g = blockIdx.x, lane = t & 31;
  const uint32_t K = A.K, S = 2 * K + 2, nx = A.nx;
  uint64_t bs, bn;
  split_even(A.n, gridDim.x, g, bs, bn);
  if (bn == 0) return;  // uniform over the team
  const uint32_t bar0 = smem_addr(&bars[0]);
  if (t == 0) {
    mbar_init(bar0);
    mbar_init(bar0 + 8);
    s_bad = 0;
  }
  __syncthreads();
  const uint32_t r_lo = (uint32_t)(bs / nx), r_hi = (uint32_t)((bs + bn - 1) / nx);  // inclusive
  const uint32_t npass = (r_hi - r_lo) / K + 1;
  // rows [a, b] (clipped to the grid) into their slots, completing on bar k
  auto load_rows = [&](int64_t a, int64_t b, uint32_t k) {
    if (a < 0) a = 0;
    if (b > (int64_t)A.ny - 1) b = (int64_t)A.ny - 1;
    const uint32_t bytes = nx * 4;
    mbar_expect_tx(bar0 + 8 * k, b >= a ? (uint32_t)(b - a + 1) * bytes : 0u);
    for (int64_t r = a; r <= b; ++r)
      bulk_g2s(ring + (size_t)((uint64_t)r % S) * A.slot_floats, A.in + (uint64_t)r * nx, bytes,
               bar0 + 8 * k);
  };
  if (t == 0) load_rows((int64_t)r_lo - 1, (int64_t)r_lo + K, 0);  // pass 0 reads these
  uint32_t phase = 0;
  for (uint32_t q = 0; q < npass; ++q) {
    const uint32_t k = q & 1u, rq = r_lo + q * K;
    // pass q + 1's new rows go to slots that no row of pass q occupies
    if (t == 0 && q + 1 < npass) load_rows((int64_t)rq + K + 1, (int64_t)rq + 2 * K, k ^ 1u);
    if (!mbar_wait(bar0 + 8 * k, (phase >> k) & 1u, kRowsWaitNs, A.status)) s_bad = 1;
    phase ^= 1u << k;
    __syncthreads();
    if (s_bad) {  // give up; let the copies in flight land first
      if (t == 0 && q + 1 < npass)
        mbar_wait(bar0 + 8 * (k ^ 1u), (phase >> (k ^ 1u)) & 1u, kRowsWaitNs, nullptr);
      break;
    }
    // team-relative output range of the pass
    const uint64_t P0 = (uint64_t)rq * nx > bs ? (uint64_t)rq * nx - bs : 0;
    const uint64_t P1e = (uint64_t)(rq + K) * nx - bs;
    const uint64_t P1 = P1e < bn ? P1e : bn;
    // one output, global index i
    auto one = [&](uint64_t i) {
      const uint32_t r = (uint32_t)__umul64hi(i, A.nx_magic);
      const uint32_t col = (uint32_t)(i - (uint64_t)r * nx);
      const uint32_t sc = r % S;
      rows_one(A, ring, i, r, col, sc == 0 ? S - 1 : sc - 1, sc, sc + 1 == S ? 0 : sc + 1);
    };
    // team-relative [lo, hi): scalar head, 16-byte units walked from a
    // rotated start, scalar tail.  The lanes' pieces are L units apart:
    // lane l starts L >= 8: l (1 - L) mod 8 units in, L < 8: floor(l L / 8)
    // units in; either way the 8 lanes of an access phase read distinct
    // bank groups.
    auto run_piece = [&](uint64_t lo, uint64_t hi) {
      uint64_t i = bs + lo;
      const uint64_t e = bs + hi;
      for (; i < e && (i & 3); ++i) one(i);
      const uint64_t ue = e & ~3ull;
      if (ue > i) {
        const uint32_t nu = (uint32_t)((ue - i) / 4);
        const uint32_t off = nu >= 8 ? ((lane * (1u - (nu & 7u))) & 7u) % nu
                                     : ((lane * nu) >> 3) % nu;
        for (uint32_t q0 = 0; q0 < nu; ++q0) {
          uint32_t u = q0 + off;
          if (u >= nu) u -= nu;
          const uint64_t gi = i + 4ull * u;
          const uint32_t r = (uint32_t)__umul64hi(gi, A.nx_magic);
          const uint32_t col = (uint32_t)(gi - (uint64_t)r * nx);
          const uint32_t sc = r % S;
          rows_unit(A, ring, gi, r, col, sc == 0 ? S - 1 : sc - 1, sc, sc + 1 == S ? 0 : sc + 1);
        }
        i = ue;
      }
      for (; i < e; ++i) one(i);
    };
    // this thread's chunks j = t, t + T, ... that meet [P0, P1)
    const uint64_t c = A.chunk;
    uint64_t j = t;
    const uint64_t jfirst = P0 / c;
    if (jfirst > j) j += (jfirst - j + T - 1) / T * T;
    for (; j * c < P1; j += T) {
      const uint64_t lo = j * c > P0 ? j * c : P0;
      const uint64_t hi = (j + 1) * c < P1 ? (j + 1) * c : P1;
      run_piece(lo, hi);
    }
    __syncthreads();  // the pass's rows are read out before later copies reuse their slots
  }
}

// cudaErrorNotSupported (nothing launched) where the ring is not the faster
// form (chunk outside [4, 8) and [32, 128]) or does not apply: nx % 4 != 0 or
// pointers not 16-byte aligned (bulk copies), n >= 2^32 (32-bit row
// arithmetic), or a ring of 2 rows per pass that does not fit the shared
// memory.
cudaError_t launch_stencil2d_rows(const void* in, float* out, uint64_t nx, uint64_t ny,
                                  uint64_t chunk, float c0, float c1, unsigned teams,
                                  unsigned threads, int max_smem, uint32_t* status,
                                  cudaStream_t st) {
  const uint64_t n = nx * ny;
  const bool faster = (chunk >= 4 && chunk < 8) || (chunk >= 32 && chunk <= 128);
  if (!faster || nx < 4 || nx % 4 || ny < 1 || n >= (1ull << 32) ||
      (((uintptr_t)in | (uintptr_t)out) & 15))
    return cudaErrorNotSupported;
  RowsArgs a;
  a.in = (const float*)in;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.n = n;
  a.chunk = chunk;
  a.nx_magic = (~0ull) / nx + 1;
  a.slot_floats = (uint32_t)((nx + 31) / 32 * 32);
  a.c0 = c0;
  a.c1 = c1;
  a.status = status;
  // K = 2 rows per pass: the ring holds 6 rows
  const uint64_t slot_bytes = (uint64_t)a.slot_floats * 4;
  a.K = 2;
  const uint64_t smem = (2ull * a.K + 2) * slot_bytes;
  if (smem + 2048 > (uint64_t)max_smem) return cudaErrorNotSupported;
  static const size_t static_bytes = static_smem_of(stencil2d_rows_kernel);
  const cudaError_t e = smem_optin(stencil2d_rows_kernel, smem, static_bytes);
  if (e != cudaSuccess) return e;
  return launch_kernel(stencil2d_rows_kernel, dim3(teams), dim3(threads), smem, st, a);
}

}  // namespace rt
