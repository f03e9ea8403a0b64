// schedule(auto) for the 2-D 5-point stencil on TMA tensor tiles.
//
// Under auto the assignment of iterations to threads is the runtime's
// (OpenMP leaves it to the implementation), so the loop is cut into 2-D tiles
// of 128 columns x 64 rows instead of 1-D pieces (on an 8192^2 grid: 0.96 of
// the copy rate with 64 rows, 0.94 with 32; the L2 promotion of the copies
// made no difference).  A persistent team walks
// tiles (team g takes g, g + G, ...) and double-buffers them: the tensor copy
// of the next tile's input box is in flight while the current one is computed.
// The box is the tile plus one row above and below and four columns on each
// side (the copy's first column must sit on a 16-byte boundary), 136 x 66
// floats; parts outside the grid read as zero and only feed boundary points,
// which copy their input, or points outside the grid, which are not stored.
// Each thread walks a 4-column strip down its rows with the rows above, at and
// below in registers (one 128-bit shared-memory read per output row); the
// columns west and east of the strip come from the neighbouring lanes by
// shuffle.  Stores are 128-bit and coalesced (a warp writes 512 contiguous
// bytes per row).  The arithmetic is the body's: fma(c1, (N+S)+(E+W), c0*C).
#include "tensor_map.h"

namespace rt {

#ifndef OMPRT_TILE_Y
#define OMPRT_TILE_Y 64
#endif
// L2 promotion of the tensor copies: 0 none, 1 128 bytes, 2 256 bytes
#ifndef OMPRT_TILE_L2
#define OMPRT_TILE_L2 2
#endif
constexpr uint32_t kTileX = 128, kTileY = OMPRT_TILE_Y;   // outputs per tile
constexpr uint32_t kBoxX = kTileX + 8, kBoxY = kTileY + 2;  // input box
constexpr uint32_t kBoxFloats = kBoxX * kBoxY;
// a tensor copy's shared-memory destination must be 128-byte aligned: the
// two boxes sit kBoxStride floats apart (the box rounded up to 128 bytes)
constexpr uint32_t kBoxStride = (kBoxFloats * 4 + 127) / 128 * 32;
static_assert(kBoxStride * 4 % 128 == 0 && kBoxStride >= kBoxFloats, "box stride");
constexpr uint32_t kTileSmem = 2 * kBoxStride * 4 + 128;  // two boxes, 128-byte aligned base
constexpr uint64_t kTileWaitNs = 1000000000ull;

struct TileArgs {
  float* out;
  uint32_t nx, ny;
  uint32_t ntx, ntiles;
  float c0, c1;
  uint32_t* status;
};

__device__ __forceinline__ void tma_load_box(float* dst, const CUtensorMap* map, int x, int y,
                                             uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float stencil_point(float c0, float c1, float nn, float ss, float e,
                                               float w, float c) {
  return __fmaf_rn(c1, __fadd_rn(__fadd_rn(nn, ss), __fadd_rn(e, w)), __fmul_rn(c0, c));
}

// W warps per team; warp w computes rows w*R .. w*R + R - 1 of a tile.
template <int W>
__global__ void __launch_bounds__(256) stencil2d_tiles_kernel(const __grid_constant__ CUtensorMap map,
                                                              const TileArgs A) {
  enter_region_grid();
  constexpr uint32_t R = kTileY / W;
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_bad;
  // box k at box0 + k * kBoxStride, on a 128-byte boundary; addressed from the
  // shared array itself so that every access compiles to a shared-memory load
  float* const box0 =
      (float*)(rt_dyn_smem + ((128u - (smem_addr(rt_dyn_smem) & 127u)) & 127u));
  const uint32_t t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t bar0 = smem_addr(&bars[0]);
  if (t == 0) {
    mbar_init(bar0);
    mbar_init(bar0 + 8);
    // never issue a tensor copy to a destination off a 128-byte boundary
    s_bad = ((smem_addr(box0) | smem_addr(box0 + kBoxStride)) & 127) != 0;
    if (s_bad) set_status(A.status, OMPRT_DEV_BAD_ARG);
  }
  __syncthreads();
  if (s_bad) return;
  const uint32_t G = gridDim.x;
  auto issue = [&](uint32_t tile, uint32_t k) {
    const int x = (int)((tile % A.ntx) * kTileX) - 4, y = (int)((tile / A.ntx) * kTileY) - 1;
    mbar_expect_tx(bar0 + 8 * k, kBoxFloats * 4);
    tma_load_box(box0 + k * kBoxStride, &map, x, y, bar0 + 8 * k);
  };
  uint32_t tile = blockIdx.x;
  if (t == 0 && tile < A.ntiles) issue(tile, 0);
  uint32_t phase = 0;  // bit k: parity of box k's next phase
  for (uint32_t k = 0; tile < A.ntiles; k ^= 1, tile += G) {
    const uint32_t nxt = tile + G;
    // box k ^ 1 was last read in the previous trip, which ended in a barrier
    if (t == 0 && nxt < A.ntiles) issue(nxt, k ^ 1);
    if (!mbar_wait(bar0 + 8 * k, (phase >> k) & 1u, kTileWaitNs, A.status)) s_bad = 1;
    phase ^= 1u << k;
    __syncthreads();
    if (s_bad) {  // give up; let the copies in flight land first
      if (t == 0) {
        mbar_wait(bar0 + 8 * k, ((phase >> k) & 1u) ^ 1u, kTileWaitNs, nullptr);
        if (nxt < A.ntiles) mbar_wait(bar0 + 8 * (k ^ 1), (phase >> (k ^ 1)) & 1u, kTileWaitNs, nullptr);
      }
      break;
    }
    const uint32_t x = (tile % A.ntx) * kTileX + 4 * lane;  // first of this lane's 4 columns
    const uint32_t ybase = (tile / A.ntx) * kTileY + w * R;
    // box row b holds grid row (tile row start) - 1 + b; this lane's strip
    // starts at box column 4 + 4 * lane
    const float* col = box0 + k * kBoxStride + 4 + 4 * lane;
    float4 nn = *(const float4*)(col + (w * R) * kBoxX);
    float4 cc = *(const float4*)(col + (w * R + 1) * kBoxX);
#pragma unroll 4
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t brow = w * R + r + 1;  // box row of the output row
      const float4 ss = *(const float4*)(col + (brow + 1) * kBoxX);
      float wl = __shfl_up_sync(0xffffffffu, cc.w, 1);
      float er = __shfl_down_sync(0xffffffffu, cc.x, 1);
      if (lane == 0) wl = col[brow * kBoxX - 1];
      if (lane == 31) er = col[brow * kBoxX + 4];
      const uint32_t y = ybase + r;
      if (y < A.ny && x < A.nx) {  // nx % 4 == 0: the 4 columns are all in or all out
        float4 o = cc;             // boundary rows and columns copy their input
        if (y >= 1 && y + 1 < A.ny) {
          if (x > 0) o.x = stencil_point(A.c0, A.c1, nn.x, ss.x, cc.y, wl, cc.x);
          o.y = stencil_point(A.c0, A.c1, nn.y, ss.y, cc.z, cc.x, cc.y);
          o.z = stencil_point(A.c0, A.c1, nn.z, ss.z, cc.w, cc.y, cc.z);
          if (x + 4 < A.nx) o.w = stencil_point(A.c0, A.c1, nn.w, ss.w, er, cc.z, cc.w);
        }
        float* p = A.out + (uint64_t)y * A.nx + x;
        asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(o.x), "f"(o.y),
                     "f"(o.z), "f"(o.w)
                     : "memory");
      }
      nn = cc;
      cc = ss;
    }
    __syncthreads();  // box k is read out before a later trip refills it
  }
}

// The driver's entry point is process-wide: looked up once, by the first
// caller (a function-local static is initialised exactly once, thread-safely).
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    cudaGetLastError();
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

// Returns cudaErrorNotSupported, launching nothing, when the tiled form does
// not apply: nx not a multiple of 4 (a 128-bit strip would straddle rows),
// pointers not 16-byte aligned, dimensions beyond the tensor copy's 32-bit
// coordinates, or no tensor-map encoder.
cudaError_t launch_stencil2d_tiles(const void* in, float* out, uint64_t nx, uint64_t ny, float c0,
                                   float c1, unsigned teams, unsigned threads, uint32_t* status,
                                   cudaStream_t st) {
  if (nx < 4 || nx % 4 || ny < 1 || nx >= (1ull << 31) - kTileX || ny >= (1ull << 31) - kTileY ||
      (((uintptr_t)in | (uintptr_t)out) & 15) || threads < 32)
    return cudaErrorNotSupported;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[2] = {nx, ny};
  const cuuint64_t strides[1] = {nx * 4};
  const cuuint32_t box[2] = {kBoxX, kBoxY};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(in), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          OMPRT_TILE_L2 == 2   ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
          : OMPRT_TILE_L2 == 1 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                               : CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  TileArgs a;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.ntx = (uint32_t)((nx + kTileX - 1) / kTileX);
  const uint64_t ntiles = (uint64_t)a.ntx * ((ny + kTileY - 1) / kTileY);
  if (ntiles >= (1ull << 31)) return cudaErrorNotSupported;
  a.ntiles = (uint32_t)ntiles;
  a.c0 = c0;
  a.c1 = c1;
  a.status = status;
  const unsigned grid = teams < a.ntiles ? teams : a.ntiles;
  // warps per team: the largest of 1, 2, 4, 8 within the thread limit
  const unsigned warps = threads >= 256 ? 8 : threads >= 128 ? 4 : threads >= 64 ? 2 : 1;
  auto* kern = warps == 8   ? stencil2d_tiles_kernel<8>
               : warps == 4 ? stencil2d_tiles_kernel<4>
               : warps == 2 ? stencil2d_tiles_kernel<2>
                            : stencil2d_tiles_kernel<1>;
  // the opt-in is a property of the kernel on the current device, so it is
  // set at every launch (as for the region kernels), not cached per process
  {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    if (e != cudaSuccess) return e;
  }
  return launch_kernel(kern, dim3(grid), dim3(32 * warps), kTileSmem, st, map, a);
}

}  // namespace rt
