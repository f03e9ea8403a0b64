// The 2-D 5-point stencil under static(c) and dynamic(c) with teams of one
// warp, when c is a multiple of 32, m = nx / c divides 32 with m < 32, and
// every team's block is the 32 / m rows that hold 32 chunks (the host uses
// it there: 4096^2 dynamic(256), 2048 teams of 32: 0.68 of the copy rate
// against 0.65 in the per-warp slabs; with one-row blocks, m >= 32, the
// slabs were faster, static(64) 0.73 against 0.64 in this form).
//
// A team of 32 threads holds its block's 32 chunks, one a lane: static(c)
// gives thread tt chunk tt (C2); under dynamic(c) the team's one warp claims
// the 32 chunks with one atomic add on the team's counter (C4), which hands
// lane l chunk l.  The grid is read as a 3-D tensor (x: the c floats of a
// chunk, y: the m chunks of a row, z: rows).  A launch has P <= G resident
// CTAs; CTA k plays the consecutive teams [k G / P, (k + 1) G / P) with K
// warps, warp gr playing teams gr, gr + K, ... (counted from the first team
// in CTAs of even index, by rounds from the last in those of odd index;
// OpenMP does not make teams run at the same time).  In round i the K warps play K consecutive teams,
// whose blocks stack up without gaps, so slab s of them (x in [32 s,
// 32 s + 32)), for all K teams, with one row above and below, is one box:
// 32 K + 2 m lines of 128 bytes, copied with the 128-byte swizzle.  A
// producer warp streams the boxes of the steps (i, s) through NB buffers
// (full / empty mbarriers, one arrival a warp a step), so the halo rows are
// read once a step instead of once a team.  Warp gr's lane l finds its rows
// in lines 32 gr + l (above), 32 gr + m + l and 32 gr + 2 m + l (below):
// eight consecutive lines an access phase, distinct bank groups.  Each lane
// runs its chunk slab by slab and each slab unit by unit, in order; its west
// neighbour at the chunk's first column and its east neighbour at a slab's
// last column are read from global memory two steps ahead.  Outputs leave
// two units (32 bytes) a store.  Boundary rows and columns copy their input;
// the arithmetic is the body's fma(c1, (N+S)+(E+W), c0*C).
#include "tensor_map.h"

namespace rt {

// compute warps: with the producer warp 512 threads, so a thread may hold
// 128 registers (the held first sector of a chunk would spill at 64)
constexpr uint32_t kColMaxWarps = 15;
constexpr uint32_t kColMaxNB = 4;
constexpr uint32_t kColMaxTeams = 1024;  // a CTA's teams (dynamic counters)
constexpr uint64_t kColWaitNs = 1000000000ull;  // 1 s: a step takes microseconds

struct ColArgs {
  const float* in;
  float* out;
  uint32_t nx, ny;     // nx * ny < 2^32
  uint32_t G, R;       // teams; rows a team block (32 / m)
  uint32_t c, m;       // chunk; chunks a row (m < 32, m | 32)
  uint32_t ns;         // slabs a chunk (c / 32)
  uint32_t K, NB;      // compute warps; buffers
  uint32_t box_bytes;  // 128 (32 K + 2 m)
  uint32_t slab;       // bytes a buffer (a multiple of 1024)
  float c0, c1;
  uint32_t* status;
};

template <int SCHED>
__global__ void __launch_bounds__((kColMaxWarps + 1) * 32, 1) stencil2d_colring_kernel(
    const __grid_constant__ CUtensorMap map, const ColArgs A) {
  enter_region_grid();
  __shared__ __align__(8) uint64_t full[kColMaxNB], empty[kColMaxNB];
  __shared__ uint32_t ctr[SCHED == kDynamic ? kColMaxTeams : 1];  // the teams' claim counters
  __shared__ int s_bad;
  const uint32_t bufs = (smem_addr(rt_dyn_smem) + 1023u) & ~1023u;  // the swizzle's period
  const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
  const uint32_t K = A.K, NB = A.NB;
  const uint32_t P = gridDim.x, k = blockIdx.x;
  const uint32_t g0 = (uint32_t)((uint64_t)k * A.G / P);
  const uint32_t g1 = (uint32_t)((uint64_t)(k + 1) * A.G / P);
  const uint32_t full0 = smem_addr(&full[0]), empty0 = smem_addr(&empty[0]);
  if (t == 0) {
    for (uint32_t i = 0; i < NB; ++i) {
      mbar_init(full0 + 8 * i);            // one arrival (with the bytes) a fill
      mbar_init_count(empty0 + 8 * i, K);  // one arrival a compute warp a step
    }
    s_bad = 0;
  }
  if (SCHED == kDynamic)
    for (uint32_t i = t; i < g1 - g0; i += blockDim.x) ctr[i] = 0;
  __syncthreads();
  if (g0 >= g1) return;  // uniform; never with P <= G
  const uint32_t ns = A.ns, m = A.m;
  const uint32_t nr = (g1 - g0 + K - 1) / K, nsteps = nr * ns;
  // Odd CTAs play their rounds from the last to the first: the rows on the
  // boundary of two CTAs' ranges are then read by both at about the same
  // time (at the start of both, or at the end of both), so the second read
  // hits in L2.  Teams do not run in any order OpenMP fixes, and a team's
  // chunks are its own.
  const bool rev = (k & 1u) != 0;
  auto round_of = [&](uint32_t q) { return rev ? nr - 1u - q / ns : q / ns; };
  // step q = i ns + s: round i, slab s
  if (w == K) {  // the producer warp
    if (lane == 0) {
      uint32_t q = 0;
      for (; q < nsteps && !*(volatile int*)&s_bad; ++q) {
        const uint32_t slot = q % NB;
        if (q >= NB &&
            !mbar_wait(empty0 + 8 * slot, ((q / NB) - 1) & 1u, kColWaitNs, A.status)) {
          s_bad = 1;
          break;
        }
        const uint32_t i = round_of(q), s = q % ns;
        const uint32_t z = (g0 + i * K) * A.R;  // the first team's first row
        mbar_expect_tx(full0 + 8 * slot, A.box_bytes);
        tma_load_3d(bufs + slot * A.slab, &map, (int)(32u * s), 0, (int)z - 1, full0 + 8 * slot);
      }
      // no copy may still be landing when the CTA leaves
      for (uint32_t j = q > NB ? q - NB : 0; j < q; ++j)
        mbar_wait(full0 + 8 * (j % NB), (j / NB) & 1u, kColWaitNs, nullptr);
    }
    return;
  }
  // a compute warp: warp w plays the teams g0 + i K + w
  const uint32_t rr = lane / m, ch = lane - rr * m;  // row within the block, chunk
  const uint32_t lN = 32u * w + lane, lC = lN + m, lS = lN + 2 * m;
  auto line_addr = [&](uint32_t bb, uint32_t L) { return (bb + 128u * L) | ((L & 7u) << 4); };
  // this lane's row and the slab's first column at step q
  auto place = [&](uint32_t q, uint32_t& g, uint32_t& row, uint32_t& colS) {
    const uint32_t i = round_of(q), s = q % ns;
    g = g0 + i * K + w;
    row = g * A.R + rr;
    colS = ch * A.c + 32u * s;
  };
  // The east word of a slab that is not its chunk's last is word 0 of the
  // chunk's next slab, read from global memory two steps ahead (about when
  // that slab's box arrives).  The words across a chunk boundary come from
  // the neighbouring lanes instead (lane l + 1 holds the next chunk of the
  // row): read from global memory they would be fetched ns - 1 steps away
  // from their boxes, after the L2 has turned over, 2 x 64 bytes a chunk
  // again from DRAM.
  auto halo = [&](uint32_t q, float& er) {
    uint32_t g, row, colS;
    place(q, g, row, colS);
    if (g < g1 && q % ns + 1 < ns) er = __ldg(A.in + (size_t)row * A.nx + colS + 32);
  };
  float er = 0.f, er1 = 0.f;  // the east words of this step and the next
  halo(0, er);
  if (nsteps > 1) halo(1, er1);
  float wl = 0.f;      // the west word of the current unit
  float e_last = 0.f;  // word 0 of the row's next chunk, for the chunk's last slab
  // A chunk's first 32-byte sector waits for its first point's west word,
  // lane l - 1's last word, at the chunk's last slab: that point's inputs
  // and the sector's other seven outputs are held until then.
  float d_n = 0.f, d_s = 0.f, d_e = 0.f, d_c = 0.f;
  float d_o[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  bool d_copy = true;
  float* d_po = nullptr;
  for (uint32_t q = 0; q < nsteps; ++q) {
    const uint32_t slot = q % NB, s = q % ns;
    float er_n = 0.f;
    if (q + 2 < nsteps) halo(q + 2, er_n);
    uint32_t g, row, colS;
    place(q, g, row, colS);
    bool mine = g < g1;
    if (SCHED == kDynamic && mine && s == 0) {
      // the claim of the team's 32 chunks, at its first slab
      uint32_t b0 = 0;
      if (lane == 0) b0 = atomicAdd(&ctr[g - g0], 32u);
      b0 = __shfl_sync(0xffffffffu, b0, 0);
      if (b0 != 0) {  // cannot happen: the team's one warp claims once
        if (lane == 0) set_status(A.status, OMPRT_DEV_BAD_ARG);
        mine = false;
      }
    }
    bool ok = mbar_wait(full0 + 8 * slot, (q / NB) & 1u, kColWaitNs, A.status);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      s_bad = 1;
      break;
    }
    const uint32_t bb = bufs + slot * A.slab;
    const uint32_t qN = line_addr(bb, lN), qC = line_addr(bb, lC), qS = line_addr(bb, lS);
    float4 c = lds128_at(qC);
    // at a chunk's first slab: lane l + 1's first word is the east word of
    // this lane's last slab (for the row's last chunk it is not used: the
    // chunk ends at column nx - 1, copied)
    if (s == 0) e_last = __shfl_down_sync(0xffffffffu, c.x, 1);
    const float er_s = s + 1 < ns ? er : e_last;
    if (mine) {
      const bool edge_row = row == 0 || row + 1 == A.ny;
      float* const po = A.out + (size_t)row * A.nx + colS;
      float4 op;  // the even unit of a pair, stored with the odd one
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) {
        const float4 cn = u < 7 ? lds128_at(qC ^ (16u * (u + 1))) : c;
        const float4 nn = lds128_at(qN ^ (16u * u)), ss = lds128_at(qS ^ (16u * u));
        const float e = u < 7 ? cn.x : er_s;
        float4 o;
        // (at a chunk's first slab o.x is not used: that point is computed
        // at the chunk's last slab, from the inputs kept here)
        o.x = slab_point(A.c0, A.c1, nn.x, ss.x, c.y, wl, c.x);
        o.y = slab_point(A.c0, A.c1, nn.y, ss.y, c.z, c.x, c.y);
        o.z = slab_point(A.c0, A.c1, nn.z, ss.z, c.w, c.y, c.z);
        o.w = slab_point(A.c0, A.c1, nn.w, ss.w, e, c.z, c.w);
        if (u == 0 && colS == 0) o.x = c.x;          // column 0
        if (u == 7 && colS + 32 == A.nx) o.w = c.w;  // column nx - 1
        if (edge_row) o = c;                         // rows 0 and ny - 1
        if (s == 0 && u == 0) {
          d_n = nn.x;
          d_s = ss.x;
          d_e = c.y;
          d_c = c.x;
          d_copy = edge_row || colS == 0;
        }
        if (u & 1) {
          if (s == 0 && u == 1) {  // the chunk's first sector: held
            d_o[0] = op.y;
            d_o[1] = op.z;
            d_o[2] = op.w;
            d_o[3] = o.x;
            d_o[4] = o.y;
            d_o[5] = o.z;
            d_o[6] = o.w;
            d_po = po;
          } else {
            const uint32_t r8[8] = {as_u(op.x), as_u(op.y), as_u(op.z), as_u(op.w),
                                    as_u(o.x),  as_u(o.y),  as_u(o.z),  as_u(o.w)};
            st8(po + 4 * (u - 1), r8);
          }
        } else {
          op = o;
        }
        wl = c.w;  // the next unit's west (the next slab's, within the chunk)
        c = cn;
      }
    }
    if (s + 1 == ns) {
      // wl is now this chunk's last word: lane l - 1's is the west word of
      // this lane's first point (a lane holding a row's first chunk starts
      // at column 0, copied)
      const float wprev = __shfl_up_sync(0xffffffffu, wl, 1);
      if (mine && d_po) {
        const float o0 = d_copy ? d_c : slab_point(A.c0, A.c1, d_n, d_s, d_e, wprev, d_c);
        const uint32_t r8[8] = {as_u(o0),     as_u(d_o[0]), as_u(d_o[1]), as_u(d_o[2]),
                                as_u(d_o[3]), as_u(d_o[4]), as_u(d_o[5]), as_u(d_o[6])};
        st8(d_po, r8);
      }
      d_po = nullptr;
    }
    __syncwarp();  // every lane has read the buffer before the warp releases it
    if (lane == 0) mbar_arrive(empty0 + 8 * slot);
    er = er1;
    er1 = er_n;
  }
}

// cudaErrorNotSupported (nothing launched) where this form does not apply:
// a schedule other than static(c) / dynamic(c); teams of other than 32
// threads; c not a multiple of 32 or not dividing nx; m = nx / c not a
// divisor of 32 below 32; team blocks other than 32 / m rows; n >= 2^32;
// pointers not 16-byte aligned; more than 1024 teams a CTA (dynamic); or no
// tensor-map encoder.  buffers: 2 .. 4, 0 for the default (3).
cudaError_t launch_stencil2d_colring(const void* in, float* out, uint64_t nx, uint64_t ny,
                                     int sched, uint64_t chunk, float c0, float c1,
                                     unsigned teams, unsigned threads, uint32_t buffers,
                                     int sm_count, int max_smem, uint32_t* status,
                                     cudaStream_t st) {
  const uint64_t n = nx * ny;
  const uint32_t NB = buffers ? buffers : 3;
  if ((sched != kChunked && sched != kDynamic) || threads != 32 || nx < 32 || ny < 1 ||
      n >= (1ull << 32) || chunk < 32 || chunk % 32 || nx % chunk || teams < 1 || teams > ny ||
      ny % teams || NB < 2 || NB > kColMaxNB || (((uintptr_t)in | (uintptr_t)out) & 15))
    return cudaErrorNotSupported;
  const uint64_t m = nx / chunk;
  if (m >= 32 || 32 % m != 0) return cudaErrorNotSupported;
  const uint64_t R = 32 / m;
  if (ny / teams != R) return cudaErrorNotSupported;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  auto* kern = sched == kChunked ? stencil2d_colring_kernel<kChunked>
                                 : stencil2d_colring_kernel<kDynamic>;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const uint64_t room = (uint64_t)max_smem > fa.sharedSizeBytes + 1024
                            ? (uint64_t)max_smem - fa.sharedSizeBytes - 1024
                            : 0;
  // K warps: NB boxes of 128 (32 K + 2 m) bytes (each rounded up to 1 KB)
  // within the shared memory, at most kColMaxWarps warps, at most 256 box rows
  auto slab_of = [&](uint64_t kk) { return (128 * (32 * kk + 2 * m) + 1023) / 1024 * 1024; };
  uint64_t K = 0;
  while (K + 1 <= kColMaxWarps && (K + 1) * R + 2 <= 256 && NB * slab_of(K + 1) <= room) ++K;
  if (K < 1) return cudaErrorNotSupported;
  // one CTA an SM, no more warps than a CTA's teams
  uint64_t P = (uint64_t)sm_count;
  if (P > teams) P = teams;
  const uint64_t per_cta_max = (teams + P - 1) / P;
  if (K > per_cta_max) K = per_cta_max;
  if (sched == kDynamic && per_cta_max > kColMaxTeams) return cudaErrorNotSupported;
  ColArgs a;
  a.in = (const float*)in;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.G = teams;
  a.R = (uint32_t)R;
  a.c = (uint32_t)chunk;
  a.m = (uint32_t)m;
  a.ns = (uint32_t)(chunk / 32);
  a.K = (uint32_t)K;
  a.NB = NB;
  a.box_bytes = (uint32_t)(128 * (32 * K + 2 * m));
  a.slab = (uint32_t)slab_of(K);
  a.c0 = c0;
  a.c1 = c1;
  a.status = status;
  CUtensorMap map;
  const cuuint64_t dims[3] = {chunk, m, ny};
  const cuuint64_t strides[2] = {chunk * 4, nx * 4};
  const cuuint32_t box[3] = {32, (cuuint32_t)m, (cuuint32_t)(K * R + 2)};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(in), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  const size_t smem = (size_t)NB * a.slab + 1024;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)(32 * K + 32), smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  return launch_kernel(kern, dim3((unsigned)P), dim3((unsigned)(32 * K + 32)), smem, st, map, a);
}

}  // namespace rt
