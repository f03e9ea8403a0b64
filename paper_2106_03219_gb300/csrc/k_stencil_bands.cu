// static(1) for the 2-D 5-point stencil when the team size T divides nx and
// every team's block is whole rows: each warp takes its strips a band of
// rows at a time from tensor copies.
//
// Under static(1) with T | nx and team blocks of whole rows, thread tt owns
// columns tt + k T (k < M = nx / T) in every row and runs them row by row, k
// ascending (C2 with c = 1; chunk numbering restarts at each block, which
// starts a row).  The 32 lanes of warp w hold the 32 consecutive columns
// 32 w + k T + [0, 32) of strip k.  A band is Rb consecutive rows of a CTA's
// range: for each strip k the warp copies the box of columns
// 32 w + k T + [-4, 36) over the band's rows and one row above and below
// (the copy's first column on a 16-byte boundary; columns outside the grid
// read as zero and only feed the copied boundary columns).  Lane l reads
// word 4 + l of a box row and its west / east neighbours at words 3 + l and
// 5 + l: the warp's 32 consecutive words, no bank conflicts.  Each warp
// pipelines its own bands through NB buffers (NB - 1 bands in flight).  A
// launch has P <= G resident CTAs of T threads; CTA k plays the consecutive
// teams [k G / P, (k + 1) G / P), the rows [R0, R1), its thread tt as thread
// tt of each team (OpenMP does not make teams run at the same time).  Every
// thread runs its own points band by band, each band's rows in order (the
// bands in order in CTAs of even index, from the last in those of odd
// index: below).  Boundary rows and columns copy their
// input; the arithmetic is the body's fma(c1, (N+S)+(E+W), c0*C).
#include "tensor_map.h"

namespace rt {

constexpr uint32_t kBandLine = 40;  // floats a box row: 32 columns and 4 on each side
constexpr uint32_t kBandMaxNB = 4;
constexpr uint64_t kBandWaitNs = 1000000000ull;  // 1 s: a band takes microseconds

struct BandArgs {
  float* out;
  uint32_t nx, ny;          // nx * ny < 2^32
  uint32_t G, rows_per_team;
  uint32_t M;               // strips a thread (nx / T)
  uint32_t Rb;              // rows a band
  uint32_t strip_bytes;     // one strip's box in shared memory (a multiple of 128)
  uint32_t box_bytes;       // the bytes one strip's copy brings: 160 (Rb + 2)
  uint32_t NB;              // buffers a warp
  float c0, c1;
  uint32_t* status;
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float lds32_at(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

// M strips a thread (a constant, so a thread's per-strip state is registers):
// the rows above and at the current one ride in registers down the band,
// each point reads the row below and its west / east words.
template <int M>
__global__ void __launch_bounds__(1024) stencil2d_bands_kernel(
    const __grid_constant__ CUtensorMap map, const BandArgs A) {
  enter_region_grid();
  __shared__ __align__(8) uint64_t bars[32][kBandMaxNB];
  const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5, T = blockDim.x;
  const uint32_t NB = A.NB, Rb = A.Rb;
  // buffers on a 128-byte boundary (a tensor copy's destination)
  const uint32_t bufs = (smem_addr(rt_dyn_smem) + 127u) & ~127u;
  const uint32_t sb = A.strip_bytes;
  const uint32_t wbytes = M * sb;  // one band of this warp
  const uint32_t buf0 = bufs + w * NB * wbytes;
  const uint32_t bar0 = smem_addr(&bars[w][0]);
  if (lane == 0)
    for (uint32_t i = 0; i < NB; ++i) mbar_init(bar0 + 8 * i);
  __syncthreads();
  const uint32_t P = gridDim.x, k = blockIdx.x;
  const uint32_t R0 = (uint32_t)((uint64_t)k * A.G / P) * A.rows_per_team;
  const uint32_t R1 = (uint32_t)((uint64_t)(k + 1) * A.G / P) * A.rows_per_team;
  if (R0 >= R1) return;  // uniform; never with P <= G
  const uint32_t nx = A.nx, ny = A.ny;
  const uint32_t nb = (R1 - R0 + Rb - 1) / Rb;
  // Odd CTAs take their bands from the last to the first: the rows on the
  // boundary of two CTAs' ranges are then read by both at about the same
  // time (at the start of both, or at the end of both), so the second read
  // hits in L2.  A thread's points are independent, so the order of its
  // rows is not observable.
  const bool rev = (k & 1u) != 0;
  auto band_row = [&](uint32_t b) { return R0 + (rev ? nb - 1u - b : b) * Rb; };
  auto issue = [&](uint32_t b, uint32_t slot) {
    const uint32_t bar = bar0 + 8 * slot;
    mbar_expect_tx(bar, M * A.box_bytes);
    const uint32_t dst = buf0 + slot * wbytes;
    const int y = (int)band_row(b) - 1;
#pragma unroll
    for (int m = 0; m < M; ++m)
      tma_load_2d(dst + m * sb, &map, (int)(32u * w + m * T) - 4, y, bar);
  };
  // per strip: is this lane's column interior (not 0, not nx - 1)
  bool in_col[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const uint32_t col = 32u * w + lane + m * T;
    in_col[m] = col > 0 && col + 1 < nx;
  }
  if (lane == 0)
    for (uint32_t b = 0; b + 1 < NB && b < nb; ++b) issue(b, b);
  uint32_t phase = 0;  // bit i: parity of buffer i's next completion
  constexpr uint32_t kRow = 4u * kBandLine;  // bytes a box row
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t slot = b % NB;
    // the band NB - 1 ahead goes to the buffer read out in the previous trip
    if (lane == 0 && b + NB - 1 < nb) issue(b + NB - 1, (b + NB - 1) % NB);
    bool ok = mbar_wait(bar0 + 8 * slot, (phase >> slot) & 1u, kBandWaitNs, A.status);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {  // give up; let the copies in flight land first
      if (lane == 0)
        for (uint32_t i = 0; i < NB && b + i < nb; ++i) {  // bands b .. b + NB - 1
          const uint32_t s2 = (b + i) % NB;
          mbar_wait(bar0 + 8 * s2, (phase >> s2) & 1u, kBandWaitNs, nullptr);
        }
      break;
    }
    phase ^= 1u << slot;
    const uint32_t rb0 = band_row(b), rb1 = rb0 + Rb < R1 ? rb0 + Rb : R1;
    // word 4 + l of box row 0 of strip 0; strip m is m sb further
    const uint32_t lw = buf0 + slot * wbytes + 4u * (4u + lane);
    float up[M], cu[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      up[m] = lds32_at(lw + m * sb);
      cu[m] = lds32_at(lw + m * sb + kRow);
    }
    uint32_t a = lw + kRow;  // box row of grid row r, strip 0
    float* orow = A.out + (size_t)rb0 * nx + 32u * w + lane;
    for (uint32_t r = rb0; r < rb1; ++r, a += kRow, orow += nx) {
      const bool inner = r >= 1 && r + 1 < ny;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const uint32_t am = a + m * sb;
        const float dn = lds32_at(am + kRow);
        float o = cu[m];
        if (inner && in_col[m]) {
          const float we = lds32_at(am - 4u), ea = lds32_at(am + 4u);
          o = __fmaf_rn(A.c1, __fadd_rn(__fadd_rn(up[m], dn), __fadd_rn(ea, we)),
                        __fmul_rn(A.c0, cu[m]));
        }
        orow[m * T] = o;
        up[m] = cu[m];
        cu[m] = dn;
      }
    }
    __syncwarp();  // buffer `slot` is read out before a later trip refills it
  }
}

// cudaErrorNotSupported (nothing launched) unless: n < 2^32, nx a multiple
// of 4 and of the team size with nx / T in {1, 2, 4, 8, 16}, teams dividing
// ny, whole warps, the input
// 16-byte aligned (a tensor copy's source), buffers in 2 .. 4 (0: 2), room in
// shared memory for at least one row a band, and a tensor-map encoder.
cudaError_t launch_stencil2d_bands(const void* in, float* out, uint64_t nx, uint64_t ny, float c0,
                                   float c1, unsigned teams, unsigned threads, uint32_t buffers,
                                   int sm_count, int max_smem, uint32_t* status,
                                   cudaStream_t st) {
  const uint64_t n = nx * ny;
  const uint32_t NB = buffers ? buffers : 2;
  if (n == 0 || n >= (1ull << 32) || nx < kBandLine || nx % 4 || teams < 1 || teams > ny ||
      ny % teams || threads < 32 || threads % 32 || threads > 1024 || nx % threads || NB < 2 ||
      NB > kBandMaxNB || ((uintptr_t)in & 15))
    return cudaErrorNotSupported;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  BandArgs a;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.G = teams;
  a.rows_per_team = (uint32_t)(ny / teams);
  a.M = (uint32_t)(nx / threads);
  a.NB = NB;
  a.c0 = c0;
  a.c1 = c1;
  a.status = status;
  void (*kern)(const CUtensorMap, const BandArgs) = nullptr;
  if (a.M == 1) kern = stencil2d_bands_kernel<1>;
  if (a.M == 2) kern = stencil2d_bands_kernel<2>;
  if (a.M == 4) kern = stencil2d_bands_kernel<4>;
  if (a.M == 8) kern = stencil2d_bands_kernel<8>;
  if (a.M == 16) kern = stencil2d_bands_kernel<16>;
  if (!kern) return cudaErrorNotSupported;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const uint64_t room = (uint64_t)max_smem > fa.sharedSizeBytes + 128
                            ? (uint64_t)max_smem - fa.sharedSizeBytes - 128
                            : 0;
  // the longest band whose buffers fit: every warp of the CTA holds NB bands
  // of its M strips, each strip's box rounded up to 128 bytes
  const uint64_t per_rowset = (uint64_t)(threads / 32) * NB * a.M;  // strip boxes a CTA holds
  auto strip_bytes = [](uint64_t rb) { return (4 * kBandLine * (rb + 2) + 127) / 128 * 128; };
  uint64_t Rb = 0;
  while (Rb + 1 <= 254 && per_rowset * strip_bytes(Rb + 1) <= room) ++Rb;
  if (Rb < 1) return cudaErrorNotSupported;
  a.Rb = (uint32_t)Rb;
  a.strip_bytes = (uint32_t)strip_bytes(Rb);
  a.box_bytes = 4 * kBandLine * (a.Rb + 2);
  CUtensorMap map;
  const cuuint64_t dims[2] = {nx, ny};
  const cuuint64_t strides[1] = {nx * 4};
  const cuuint32_t box[2] = {kBandLine, a.Rb + 2};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(in), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  const size_t smem = (size_t)(per_rowset * a.strip_bytes + 128);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  uint64_t P = (uint64_t)per_sm * (uint64_t)sm_count;
  if (P > teams) P = teams;
  return launch_kernel(kern, dim3((unsigned)P), dim3(threads), smem, st, map, a);
}

}  // namespace rt
