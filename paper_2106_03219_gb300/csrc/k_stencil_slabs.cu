// The 2-D 5-point stencil under static(c) and dynamic(c) when c is a
// multiple of the slab line X (16 or 32 floats) that divides nx, every team's
// block is whole rows (G divides ny), and m = nx / c (chunks per row) is a
// multiple or a divisor of 32.  The chunks a warp holds at one time arrive,
// X floats of each at a time, as one tensor copy.
//
// The grid is read as a 3-D tensor: x the c floats of a chunk, y the m
// chunks of a row, z the rows.  A warp holds 32 consecutive chunks of a team
// block starting at a multiple of 32: with m >= 32 they are chunks y0 .. y0 +
// 31 of one row, with m < 32 they are 32 / m whole rows.  Slab s of them is
// the box x in [X s, X s + X) over those chunks and their rows plus one row
// above and one below: nr = 32 / mb + 2 rows of mb = min(m, 32) chunks, mb nr
// lines of 4 X bytes, copied with the swizzle of the line's width (128-byte
// lines: 16-byte unit k of line L sits at unit k ^ (L mod 8); 64-byte lines:
// at k ^ ((L / 2) mod 4)).  Lane l's chunk has its row in line l + mb, the row
// above in line l and the row below in line l + 2 mb, so when every lane
// reads unit k of its own chunk the eight lanes of an access phase read
// eight consecutive lines: distinct bank groups.
//
// Every warp runs its own pipeline: NB slab buffers with an mbarrier each,
// lane 0 keeping NB - 1 copies of the warp's next slabs in flight while the
// lanes compute the current one.  A launch has P <= G resident CTAs; CTA k
// plays the consecutive teams [k G / P, (k + 1) G / P) (OpenMP does not make
// teams run at the same time).  Its W warps form K = W / (T / 32) groups;
// group gr plays the CTA's teams gr, gr + K, ... in turn (counted from the
// first team in CTAs of even index, from the last in those of odd index),
// its warp i as threads 32 i .. 32 i + 31 of the team.
//   static(c):  warp i's lanes run chunks j0 + l of the block for j0 = 32 i,
//               32 i + T, ... (thread tt runs chunks tt, tt + T, ...: C2);
//   dynamic(c): lane 0 claims 32 chunks with one atomic add on the team's
//               counter (one per team of the CTA, in shared memory), lane l
//               runs chunk base + l; a thread's claims increase (C4).
// A lane runs its chunk slab by slab and each slab unit by unit, in order.
// Its west neighbour at a chunk's first column and its east neighbour at a
// slab's last column are read from global memory one slab ahead; the others
// are carried from unit to unit.  Boundary rows and columns copy their
// input; the arithmetic is the body's fma(c1, (N+S)+(E+W), c0*C).  Outputs
// leave two units (32 bytes) a store.
#include "tensor_map.h"

namespace rt {

constexpr uint32_t kSlabMaxWarps = 16;
constexpr uint32_t kSlabMaxTeams = 1024;  // per CTA: the dynamic counters
constexpr uint64_t kSlabWaitNs = 1000000000ull;  // 1 s: a slab takes microseconds
// defaults: 32-float lines, and about 24 KB of slab buffers a warp (4096^2:
// 12 KB boxes best with 2 buffers, static(64) 0.73 against 0.72 with 3;
// 8 KB boxes with 3, dynamic(256) 0.64 against 0.54 with 2)
constexpr uint32_t kSlabDefaultFloats = 32, kSlabWarpBytes = 24 * 1024;

struct SlabArgs {
  const float* in;
  float* out;
  uint32_t nx, ny;    // nx * ny < 2^32
  uint32_t G, R;      // teams; rows per team block (G R = ny)
  uint32_t T, K;      // threads of a team; groups per CTA
  uint32_t c, m;      // chunk; chunks per row (m c = nx)
  uint32_t mb, nr;    // chunks and rows of a box
  uint32_t ns;        // slabs per chunk (c / X)
  uint32_t nch;       // chunks per block (R m)
  uint32_t slab;      // bytes per slab buffer (a multiple of 1024)
  uint32_t box_bytes;  // 4 X mb nr
  float c0, c1;
  uint32_t* status;
};

// A warp's place in its sequence of slabs: team g, first chunk j0 of its 32,
// slab s.  Warp-uniform.
struct SlabItem {
  uint32_t g, j0, s;
};

// X floats a slab line (32: 128-byte lines, 128-byte swizzle; 16: 64-byte
// lines, 64-byte swizzle), NB slab buffers a warp (NB - 1 copies in flight
// while one slab is computed).
template <int SCHED, int X, int NB>
__global__ void __launch_bounds__(kSlabMaxWarps * 32, 1) stencil2d_slabs_kernel(
    const __grid_constant__ CUtensorMap map, const SlabArgs A) {
  enter_region_grid();
  constexpr uint32_t U = X / 4;  // 16-byte units of a line
  __shared__ __align__(8) uint64_t bars[kSlabMaxWarps][NB];
  __shared__ uint32_t ctr[SCHED == kDynamic ? kSlabMaxTeams : 1];  // the teams' claim counters
  // slab buffers on a 1024-byte boundary (the swizzle's period), addressed as
  // 32-bit shared-memory addresses
  const uint32_t base0 = smem_addr(rt_dyn_smem);
  const uint32_t bufs = (base0 + 1023u) & ~1023u;
  const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
  const uint32_t wpt = A.T >> 5;  // warps per team
  const uint32_t gr = w / wpt, wi = w - gr * wpt;
  const uint32_t P = gridDim.x, k = blockIdx.x;
  const uint32_t g0 = (uint32_t)((uint64_t)k * A.G / P);
  const uint32_t g1 = (uint32_t)((uint64_t)(k + 1) * A.G / P);
  // Odd CTAs play their teams from the last to the first: the rows on the
  // boundary of two CTAs' bands are then read by both at about the same
  // time (at the start of both, or at the end of both), so the second read
  // hits in L2.  Teams do not run in any order OpenMP fixes, and each team
  // still claims its own chunks in increasing order.
  const bool rev = (k & 1u) != 0;
  auto team_of = [&](uint32_t g) { return rev ? g0 + g1 - 1u - g : g; };  // onto [g0, g1)
  if (SCHED == kDynamic)
    for (uint32_t i = t; i < g1 - g0; i += blockDim.x) ctr[i] = 0;
  const uint32_t bar0 = smem_addr(&bars[w][0]);
  if (lane == 0)
    for (int i = 0; i < NB; ++i) mbar_init(bar0 + 8 * i);
  __syncthreads();
  if (g0 >= g1) return;  // uniform; never with P <= G
  const uint32_t buf0 = bufs + w * (uint32_t)NB * A.slab;
  const uint32_t nch = A.nch, ns = A.ns, m = A.m, mb = A.mb;

  auto claim = [&](uint32_t g) {
    uint32_t b0 = 0;
    if (lane == 0) b0 = atomicAdd(&ctr[g - g0], 32u);
    return __shfl_sync(0xffffffffu, b0, 0);
  };
  // the first chunk group of team g at or after the warp's start; false if none
  auto first_of_team = [&](SlabItem& it) {
    for (; it.g < g1; it.g += A.K) {
      if constexpr (SCHED == kDynamic) {
        it.j0 = claim(it.g);
      } else {
        it.j0 = 32u * wi;
      }
      if (it.j0 < nch) {
        it.s = 0;
        return true;
      }
    }
    return false;
  };
  auto advance = [&](SlabItem& it) {
    if (++it.s < ns) return true;
    it.s = 0;
    if constexpr (SCHED == kDynamic) {
      it.j0 = claim(it.g);
    } else {
      it.j0 += A.T;
    }
    if (it.j0 < nch) return true;
    it.g += A.K;
    return first_of_team(it);
  };
  // the box of an item: x = X s, y = the first chunk's place in its row,
  // z = the row above the first chunk's row
  auto issue = [&](const SlabItem& it, uint32_t b) {
    const uint32_t row0 = team_of(it.g) * A.R + it.j0 / m;
    const uint32_t y = m >= 32 ? it.j0 % m : 0u;
    mbar_expect_tx(bar0 + 8 * b, A.box_bytes);
    tma_load_3d(buf0 + b * A.slab, &map, (int)((uint32_t)X * it.s), (int)y, (int)row0 - 1,
                bar0 + 8 * b);
  };
  // this lane's chunk in an item: its row, the slab's first column, and
  // whether the chunk is one of the block's
  const uint32_t rr = lane / mb, ch = lane - rr * mb;  // row within the group, chunk
  auto place = [&](const SlabItem& it, uint32_t& row, uint32_t& colS) {
    row = team_of(it.g) * A.R + it.j0 / m + rr;
    colS = ((m >= 32 ? it.j0 % m : 0u) + ch) * A.c + (uint32_t)X * it.s;
    return it.j0 + lane < nch;
  };
  // the west neighbour of a chunk's first slab and the east neighbour of
  // every slab, read from global memory one item ahead of their use
  auto halo = [&](const SlabItem& it, float& wl, float& er) {
    uint32_t row, colS;
    if (place(it, row, colS)) {
      const size_t ro = (size_t)row * A.nx;
      if (it.s == 0 && colS > 0) wl = __ldg(A.in + ro + colS - 1);
      if (colS + X < A.nx) er = __ldg(A.in + ro + colS + X);
    }
  };
  // box lines of this lane's rows above / at / below, with their swizzle
  // (the 16-byte unit index XORed with line bits above the line: 128-byte
  // swizzle bits 7..9, 64-byte swizzle bits 7..8)
  auto line_addr = [&](uint32_t bb, uint32_t L) {
    return X == 32 ? (bb + 128u * L) | ((L & 7u) << 4) : (bb + 64u * L) | (((L >> 1) & 3u) << 4);
  };
  const uint32_t lN = lane, lC = lane + mb, lS = lane + 2 * mb;

  SlabItem q[NB];  // q[0] the item being computed, q[1 ..] the ones in flight
  bool qv[NB];
  q[0] = SlabItem{g0 + gr, 0, 0};
  qv[0] = first_of_team(q[0]);
#pragma unroll
  for (int i = 1; i < NB; ++i) {
    q[i] = q[i - 1];
    qv[i] = qv[i - 1] && advance(q[i]);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i + 1 < NB; ++i)
      if (qv[i]) issue(q[i], (uint32_t)i);
  }
  float wl = 0.f, er = 0.f;  // the current item's west / east
  halo(q[0], wl, er);
  uint32_t b = 0, phase = 0;  // phase bit i: parity of buffer i's next completion
  while (qv[0]) {
    // the buffer of q[NB - 1] held the previous trip's item, read out before
    // that trip's __syncwarp
    const uint32_t blast = (b + NB - 1) % NB;
    if (qv[NB - 1] && lane == 0) issue(q[NB - 1], blast);
    float wl_n = 0.f, er_n = 0.f;
    if (qv[1]) halo(q[1], wl_n, er_n);
    bool ok = mbar_wait(bar0 + 8 * b, (phase >> b) & 1u, kSlabWaitNs, A.status);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {  // give up; let the copies in flight land first
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const uint32_t bi = (b + i) % NB;
          if (qv[i]) mbar_wait(bar0 + 8 * bi, (phase >> bi) & 1u, kSlabWaitNs, nullptr);
        }
      }
      break;
    }
    phase ^= 1u << b;
    uint32_t row, colS;
    const bool mine = place(q[0], row, colS);
    const uint32_t bb = buf0 + b * A.slab;
    const uint32_t qN = line_addr(bb, lN), qC = line_addr(bb, lC), qS = line_addr(bb, lS);
    const bool edge_row = row == 0 || row + 1 == A.ny;
    float* const po = A.out + (size_t)row * A.nx + colS;
    float4 c = lds128_at(qC);
    float4 op;  // the even unit of a pair, stored with the odd one
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const float4 cn = u + 1 < U ? lds128_at(qC ^ (16u * (u + 1))) : c;
      const float4 nn = lds128_at(qN ^ (16u * u)), ss = lds128_at(qS ^ (16u * u));
      const float e = u + 1 < U ? cn.x : er;
      float4 o;
      o.x = slab_point(A.c0, A.c1, nn.x, ss.x, c.y, wl, c.x);
      o.y = slab_point(A.c0, A.c1, nn.y, ss.y, c.z, c.x, c.y);
      o.z = slab_point(A.c0, A.c1, nn.z, ss.z, c.w, c.y, c.z);
      o.w = slab_point(A.c0, A.c1, nn.w, ss.w, e, c.z, c.w);
      if (u == 0 && colS == 0) o.x = c.x;          // column 0
      if (u + 1 == U && colS + X == A.nx) o.w = c.w;  // column nx - 1
      if (edge_row) o = c;                         // rows 0 and ny - 1
      // two units a store: whole 32-byte sectors (colS is a multiple of 16
      // floats, so unit pairs sit on 32-byte boundaries)
      if (u & 1) {
        if (mine) {
          const uint32_t r8[8] = {as_u(op.x), as_u(op.y), as_u(op.z), as_u(op.w),
                                  as_u(o.x),  as_u(o.y),  as_u(o.z),  as_u(o.w)};
          st8(po + 4 * (u - 1), r8);
        }
      } else {
        op = o;
      }
      wl = c.w;
      c = cn;
    }
    __syncwarp();  // buffer b is read out before a later trip refills it
    // the next slab of the same chunk takes its west from this one's last unit
    if (qv[1] && q[1].s == 0) wl = wl_n;
    er = er_n;
    const SlabItem last = q[NB - 1];
    const bool lastv = qv[NB - 1];
#pragma unroll
    for (int i = 0; i + 1 < NB; ++i) {
      q[i] = q[i + 1];
      qv[i] = qv[i + 1];
    }
    q[NB - 1] = last;
    qv[NB - 1] = lastv && advance(q[NB - 1]);
    b = b + 1 == NB ? 0 : b + 1;
  }
}

using SlabKernel = void (*)(const CUtensorMap, const SlabArgs);

template <int SCHED>
static SlabKernel slab_kernel(uint32_t X, uint32_t NB) {
  if (X == 32) {
    if (NB == 2) return stencil2d_slabs_kernel<SCHED, 32, 2>;
    if (NB == 3) return stencil2d_slabs_kernel<SCHED, 32, 3>;
    if (NB == 4) return stencil2d_slabs_kernel<SCHED, 32, 4>;
  } else if (X == 16) {
    if (NB == 2) return stencil2d_slabs_kernel<SCHED, 16, 2>;
    if (NB == 3) return stencil2d_slabs_kernel<SCHED, 16, 3>;
    if (NB == 4) return stencil2d_slabs_kernel<SCHED, 16, 4>;
  }
  return nullptr;
}

// cudaErrorNotSupported (nothing launched) where this form does not apply:
// a schedule other than static(c) / dynamic(c); c not a multiple of the slab
// line (16 or 32 floats) or not dividing nx; m = nx / c neither a multiple
// nor a divisor of 32; teams not dividing ny; n >= 2^32; teams of more than
// 512 threads or not whole warps; pointers not 16-byte aligned; more than
// 1024 teams a CTA (dynamic); or no tensor-map encoder.  slab_floats (16 or
// 32) and buffers (2 .. 4) pick the slab shape; 0 takes the default.
cudaError_t launch_stencil2d_slabs(const void* in, float* out, uint64_t nx, uint64_t ny, int sched,
                                   uint64_t chunk, float c0, float c1, unsigned teams,
                                   unsigned threads, uint32_t slab_floats, uint32_t buffers,
                                   int sm_count, int max_smem, uint32_t* status,
                                   cudaStream_t st) {
  const uint64_t n = nx * ny;
  const uint32_t X = slab_floats ? slab_floats : (chunk % 32 ? 16u : kSlabDefaultFloats);
  if ((sched != kChunked && sched != kDynamic) || (X != 16 && X != 32) ||
      nx < X || ny < 1 || n >= (1ull << 32) || chunk < X || chunk % X || nx % chunk ||
      teams < 1 || teams > ny || ny % teams || threads < 32 || threads % 32 ||
      threads > kSlabMaxWarps * 32 || (((uintptr_t)in | (uintptr_t)out) & 15))
    return cudaErrorNotSupported;
  const uint64_t m = nx / chunk;
  if (m % 32 != 0 && 32 % m != 0) return cudaErrorNotSupported;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  SlabArgs a;
  a.in = (const float*)in;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.G = teams;
  a.R = (uint32_t)(ny / teams);
  a.T = threads;
  a.c = (uint32_t)chunk;
  a.m = (uint32_t)m;
  a.mb = (uint32_t)(m < 32 ? m : 32);
  a.nr = 32u / a.mb + 2u;
  a.ns = (uint32_t)(chunk / X);
  a.nch = a.R * a.m;
  a.box_bytes = 4u * X * a.mb * a.nr;
  a.slab = (a.box_bytes + 1023u) & ~1023u;
  uint32_t NB = buffers ? buffers : kSlabWarpBytes / a.slab;
  if (NB < 2) NB = 2;
  if (NB > 4) NB = 4;
  a.c0 = c0;
  a.c1 = c1;
  a.status = status;
  CUtensorMap map;
  const cuuint64_t dims[3] = {chunk, m, ny};
  const cuuint64_t strides[2] = {chunk * 4, nx * 4};
  const cuuint32_t box[3] = {X, a.mb, a.nr};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(in), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          X == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  const SlabKernel kern =
      sched == kChunked ? slab_kernel<kChunked>(X, NB) : slab_kernel<kDynamic>(X, NB);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  // warps: whole teams, NB slab buffers each, within the shared memory left
  // beside the kernel's own variables (1024 bytes for the alignment)
  const uint64_t room = (uint64_t)max_smem > fa.sharedSizeBytes + 1024
                            ? (uint64_t)max_smem - fa.sharedSizeBytes - 1024
                            : 0;
  const uint64_t wpt = threads / 32;
  uint64_t W = room / ((uint64_t)NB * a.slab);
  if (W > kSlabMaxWarps) W = kSlabMaxWarps;
  uint64_t K = W / wpt;
  if (K < 1) return cudaErrorNotSupported;
  const size_t smem = (size_t)(K * wpt * NB * a.slab + 1024);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)(K * threads), smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  uint64_t P = (uint64_t)per_sm * (uint64_t)sm_count;
  if (P > teams) P = teams;
  // groups beyond a CTA's teams idle: with K groups a CTA of ceil(G / P)
  // teams takes ceil(ceil(G / P) / K) rounds, so K is not cut down to the
  // smaller CTAs' count (that would give the larger ones a second round)
  const uint64_t per_cta_max = (teams + P - 1) / P;
  if (K > per_cta_max) K = per_cta_max;
  if (sched == kDynamic && per_cta_max > kSlabMaxTeams) return cudaErrorNotSupported;
  a.K = (uint32_t)K;
  return launch_kernel(kern, dim3((unsigned)P), dim3((unsigned)(K * threads)), smem, st, map, a);
}

}  // namespace rt
