// The 2-D 5-point stencil under the schedules that fix which thread runs an
// iteration: static, static(c) and dynamic(c).  The input streams through a
// ring in shared memory, filled by bulk copies well ahead of the compute;
// every OpenMP thread runs exactly the iterations the schedule gives it,
// reading its operands from the ring and storing its outputs itself.
//
// Teams, groups and passes.  Level 1 is the usual balanced split of the
// n = nx * ny logical iterations over G teams (team g's block starts at
// q g + min(g, r), n = q G + r).  A launch has P <= G resident CTAs; CTA k
// plays the logical teams [k G / P, (k + 1) G / P) (OpenMP does not make
// teams run at the same time), so a CTA's teams are one contiguous range of
// the grid, and the CTA reads that range plus one grid row on each side as
// one stream.  A CTA of K * T threads holds K groups of T (T the team size,
// a multiple of 32): group gr plays one team at a time and its thread tt is
// that team's thread tt, so small teams still fill the SM.  The CTA takes its
// teams in passes of up to `pass_teams` teams (group gr runs the pass's teams
// gr, gr + K, ...).  The stream is cut into segments of L floats and the ring
// holds S of them (segment i in slot i mod S, completion counted on slot i's
// mbarrier): a pass waits for the segments its points and their neighbours
// lie in, computes, and ends in one barrier, after which thread 0 refills
// every slot that no later pass needs.  Each input element is copied into
// shared memory once per CTA, and the segments beyond the current pass are in
// flight while it computes.
//
// Ownership inside a team:
//   static:    thread t runs its balanced contiguous piece of the block (C1);
//   static(c): thread t runs chunks t, t + T, ... of the block (C2); c = 1 is
//              the stride-T sequence of single points;
//   dynamic(c): lane 0 of a warp claims the next 32 chunks of the team with
//              one atomic add on the team's counter (team-shared, in shared
//              memory: a team is run by one group in one pass), lane l runs
//              chunk base + l in full; a thread's claims increase.
// A piece runs in 16-byte units (four outputs in one row: nx is a multiple
// of 4) from its first 16-byte boundary to its last, one point at a time
// outside them.  A unit reads the rows above, at and below with 128-bit
// shared-memory loads; its west / east neighbours are carried over from the
// units before and after it.  Lanes walk their units from a rotated start
// (then wrap around), chosen so that the eight lanes of a 128-bit access
// phase read distinct 16-byte bank groups when the lanes' pieces sit a whole
// number of units apart; while no lane of the warp can have wrapped, the walk
// runs a loop without the wrap tests.  Outputs are stored straight from
// registers with 128-bit stores.  The arithmetic is the body's:
// fma(c1, (N+S)+(E+W), c0*C), boundary points copied.  Every ring index is
// taken modulo the ring's size, so no shared-memory access can leave the
// ring.
#include "api_internal.h"

namespace rt {

constexpr uint32_t kOwnerMaxGroups = 15;  // named barriers 1 .. 15, one per group
constexpr uint32_t kOwnerMaxSlots = 64;
constexpr uint64_t kOwnerWaitNs = 1000000000ull;  // 1 s: a pass takes microseconds

struct OwnerArgs {
  const float* in;
  float* out;
  uint32_t nx, ny, n;     // n = nx * ny < 2^32, nx a multiple of 4
  uint32_t G;             // logical teams
  uint32_t q, r;          // n = q G + r
  uint32_t T;             // threads of a logical team (a multiple of 32)
  uint32_t groups;        // K: teams a CTA runs at once (blockDim.x = K T)
  uint32_t chunk;         // static(c) / dynamic(c): c (at most q + 1); static: 0
  uint32_t seg;           // L: floats per ring segment (a multiple of 32)
  uint32_t slots;         // S: segments the ring holds, 2 .. kOwnerMaxSlots
  uint32_t pass_teams;    // unused (1)
  uint64_t nx_magic;      // ceil(2^64 / nx): the row of i < 2^32 is umulhi(i, magic)
  float c0, c1;
  uint32_t* status;
};

__device__ __forceinline__ float owner_point(const OwnerArgs& A, float nn, float ss, float e,
                                             float w, float c) {
  return __fmaf_rn(A.c1, __fadd_rn(__fadd_rn(nn, ss), __fadd_rn(e, w)), __fmul_rn(A.c0, c));
}

__device__ __forceinline__ uint32_t owner_col(const OwnerArgs& A, uint32_t p) {
  return p - (uint32_t)__umul64hi((uint64_t)p, A.nx_magic) * A.nx;
}

// Team g's block [bs, bs + bn) (C1 with P = G).
__device__ __forceinline__ void owner_block(const OwnerArgs& A, uint32_t g, uint32_t& bs,
                                            uint32_t& bn) {
  const bool lo = g < A.r;
  bn = A.q + (lo ? 1u : 0u);
  bs = A.q * g + (lo ? g : A.r);
}

__device__ __forceinline__ float4 lds128(const float* p) { return *(const float4*)p; }

__device__ __forceinline__ void stg128(float* p, float4 v) {
  asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

// The ring: stream element p (base <= p) sits at w[(p - base) mod cap].
struct Win {
  const float* w;
  uint32_t base, cap;
};

__device__ __forceinline__ uint32_t ring_of(const Win& W, uint32_t p) { return (p - W.base) % W.cap; }
// j + d and j - d modulo cap, for j < cap and d <= cap
__device__ __forceinline__ uint32_t ring_add(const Win& W, uint32_t j, uint32_t d) {
  const uint32_t k = j + d;
  return k >= W.cap ? k - W.cap : k;
}
__device__ __forceinline__ uint32_t ring_sub(const Win& W, uint32_t j, uint32_t d) {
  return j >= d ? j - d : j + W.cap - d;
}

// One output point p (global index, ring index j, column col).
__device__ __forceinline__ float owner_value(const OwnerArgs& A, const Win& W, uint32_t p,
                                             uint32_t j, uint32_t col) {
  const float c = W.w[j];
  float v = c;
  if (p >= A.nx && p < A.n - A.nx && col != 0 && col + 1 != A.nx)
    v = owner_point(A, W.w[ring_sub(W, j, A.nx)], W.w[ring_add(W, j, A.nx)],
                    W.w[ring_add(W, j, 1)], W.w[ring_sub(W, j, 1)], c);
  return v;
}

__device__ __forceinline__ void owner_one(const OwnerArgs& A, const Win& W, uint32_t p) {
  A.out[p] = owner_value(A, W, p, ring_of(W, p), owner_col(A, p));
}

// Points base, base + step, ... (cnt of them, step <= 1024 <= ring size),
// four at a time with all shared-memory reads of a group issued before its
// stores.
__device__ __forceinline__ void owner_strided(const OwnerArgs& A, const Win& W, uint32_t base,
                                              uint32_t step, uint32_t cnt) {
  if (cnt == 0) return;
  uint32_t k = 0, j = ring_of(W, base);  // ring index of point base + k * step
  for (; k + 4 <= cnt; k += 4) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t p = base + (k + u) * step;
      v[u] = owner_value(A, W, p, j, owner_col(A, p));
      j = ring_add(W, j, step);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) A.out[base + (k + u) * step] = v[u];
  }
  for (; k < cnt; ++k) {
    const uint32_t p = base + k * step;
    A.out[p] = owner_value(A, W, p, j, owner_col(A, p));
    j = ring_add(W, j, step);
  }
}

// The four outputs of the unit at p (ring index j, first column col) from
// its row c, west / east neighbours Wl / E.
__device__ __forceinline__ float4 owner_unit(const OwnerArgs& A, const Win& W, uint32_t p,
                                             uint32_t j, uint32_t col, float4 c, float Wl,
                                             float E) {
  float4 o = c;  // boundary rows are copied
  if (p >= A.nx && p < A.n - A.nx) {
    const float4 nn = lds128(W.w + ring_sub(W, j, A.nx));
    const float4 ss = lds128(W.w + ring_add(W, j, A.nx));
    // of the four columns only the first (0) and the last (nx - 1) can be boundary
    if (col != 0) o.x = owner_point(A, nn.x, ss.x, c.y, Wl, c.x);
    o.y = owner_point(A, nn.y, ss.y, c.z, c.x, c.y);
    o.z = owner_point(A, nn.z, ss.z, c.w, c.y, c.z);
    if (col + 4 != A.nx) o.w = owner_point(A, nn.w, ss.w, E, c.z, c.w);
  }
  return o;
}

// Units of four outputs p0, p0 + 4, ... (nu of them, p0 a multiple of 4),
// walked from unit `off` (< 8, < nu) to the last, then from unit 0.  The
// first nu - 8 steps cannot reach the last unit in any lane (off < 8), so
// they run without the wrap test.
__device__ __forceinline__ void owner_units(const OwnerArgs& A, const Win& W, uint32_t p0,
                                            uint32_t nu, uint32_t off) {
  const float* const w = W.w;
  // ring indices are multiples of 4 here: the ring is whole units
  const uint32_t jA = ring_of(W, p0);
  const uint32_t colA = owner_col(A, p0);
  uint32_t j = ring_add(W, jA, 4 * off), p = p0 + 4 * off;
  uint32_t col = colA + 4 * off;
  while (col >= A.nx) col -= A.nx;  // 4 off < 32: a few rows at most when nx is small
  float Wl = w[ring_sub(W, j, 1)];  // not yet loaded only for p == 0, a boundary point
  float4 c = lds128(w + j);
  uint32_t it = 0;
  const uint32_t straight = nu > 8 ? nu - 8 : 0;
#pragma unroll 2
  for (; it < straight; ++it) {
    const uint32_t jn = ring_add(W, j, 4);
    const float4 cn = lds128(w + jn);
    stg128(A.out + p, owner_unit(A, W, p, j, col, c, Wl, cn.x));
    Wl = c.w;
    c = cn;
    j = jn;
    p += 4;
    col += 4;
    if (col == A.nx) col = 0;
  }
  uint32_t m = off + it;  // this lane's unit index (< nu: no lane has wrapped yet)
  for (; it < nu; ++it) {
    const bool wrap = m + 1 == nu;
    const uint32_t jn = wrap ? jA : ring_add(W, j, 4);
    const float4 cn = lds128(w + jn);
    float E = cn.x, Wn = c.w;
    if (wrap) {  // the unit after the piece's last: read on its own
      E = w[ring_add(W, j, 4)];
      Wn = w[ring_sub(W, jA, 1)];
    }
    stg128(A.out + p, owner_unit(A, W, p, j, col, c, Wl, E));
    Wl = Wn;
    c = cn;
    if (wrap) {
      m = 0;
      j = jA;
      p = p0;
      col = colA;
    } else {
      ++m;
      j = jn;
      p += 4;
      col += 4;
      if (col == A.nx) col = 0;
    }
  }
}

// The calling thread's piece [a, e) of a team block: single points up to
// the first 16-byte boundary, units, single points after the last one.
__device__ __forceinline__ void owner_piece(const OwnerArgs& A, const Win& W, uint32_t a,
                                            uint32_t e, uint32_t lane) {
  uint32_t p = a;
  const uint32_t h = e < ((a + 3) & ~3u) ? e : ((a + 3) & ~3u);
  for (; p < h; ++p) owner_one(A, W, p);
  const uint32_t ue = e & ~3u;
  if (ue > p) {
    const uint32_t nu = (ue - p) >> 2;
    // lanes whose pieces sit nu units apart: 2^s = gcd(nu, 8) of every 8
    // lanes of an access phase start in the same bank group, so they are
    // spread over 2^s starting units
    const uint32_t s = nu & 7u ? (uint32_t)(__ffs((int)(nu & 7u)) - 1) : 3u;
    const uint32_t off = ((lane & 7u) >> (3u - s)) & ((1u << s) - 1u);
    owner_units(A, W, p, nu, off);
    p = ue;
  }
  for (; p < e; ++p) owner_one(A, W, p);
}

template <int SCHED>
__global__ void __launch_bounds__(1024) stencil2d_owner_kernel(const OwnerArgs A) {
  enter_region_grid();
  __shared__ __align__(8) uint64_t full[kOwnerMaxSlots], empty[kOwnerMaxSlots];
  __shared__ uint32_t ctr[kOwnerMaxGroups][2];  // dynamic: each group's claim counters
  __shared__ int s_bad;
  // the ring on a 128-byte boundary, addressed from the shared array itself so
  // that every access compiles to a shared-memory load
  float* const ring = (float*)(rt_dyn_smem + ((128u - (smem_addr(rt_dyn_smem) & 127u)) & 127u));
  const uint32_t t = threadIdx.x, lane = t & 31u;
  const uint32_t Tl = A.T, K = A.groups, gr = t / Tl, tt = t - gr * Tl;
  const uint32_t P = gridDim.x, k = blockIdx.x;
  const uint32_t g0 = (uint32_t)((uint64_t)k * A.G / P);
  const uint32_t g1 = (uint32_t)((uint64_t)(k + 1) * A.G / P);
  if (g0 >= g1) return;  // uniform; never with P <= G
  const uint32_t L = A.seg, S = A.slots;
  // this CTA's input stream: its teams' range plus one row on each side, in
  // whole 16-byte units
  uint32_t E0, E1, tmp;
  owner_block(A, g0, E0, tmp);
  owner_block(A, g1, E1, tmp);  // g1 <= G: the block of team G starts at n
  const uint32_t base = (E0 > A.nx ? E0 - A.nx : 0u) & ~3u;
  const uint32_t send = ((E1 < A.n - A.nx ? E1 + A.nx : A.n) + 3u) & ~3u;  // n % 4 == 0
  const uint32_t nseg = (send - base + L - 1) / L;
  const uint32_t full0 = smem_addr(&full[0]), empty0 = smem_addr(&empty[0]);
  if (t == 0) {
    for (uint32_t i = 0; i < S; ++i) {
      mbar_init(full0 + 8 * i);               // one arrival (with the bytes) per fill
      mbar_init_count(empty0 + 8 * i, K);     // one arrival per group per release
    }
    s_bad = 0;
  }
  if (SCHED == kDynamic && t < 2 * kOwnerMaxGroups) ctr[t >> 1][t & 1] = 0;
  __syncthreads();
  // the first / one past the last segment team g's points and neighbours lie in
  auto seg_lo = [&](uint32_t g) {
    uint32_t bs, bn;
    owner_block(A, g, bs, bn);
    return (((bs > A.nx ? bs - A.nx : 0u) & ~3u) - base) / L;
  };
  auto seg_hi = [&](uint32_t g) {
    uint32_t bs, bn;
    owner_block(A, g, bs, bn);
    const uint32_t e = bs + bn < A.n - A.nx ? bs + bn + A.nx : A.n;
    return (e - base + L - 1) / L;
  };
  const uint32_t W_threads = K * Tl;  // the producer is the warp after the groups
  if (t >= W_threads) {
    if (lane == 0) {
      // fill slot i % S with segment i once every group has released segment i - S
      uint32_t i = 0;
      for (; i < nseg && !*(volatile int*)&s_bad; ++i) {
        if (i >= S &&
            !mbar_wait(empty0 + 8 * (i % S), ((i / S) - 1) & 1u, kOwnerWaitNs, A.status)) {
          s_bad = 1;
          break;
        }
        const uint32_t lo = base + i * L;
        const uint32_t len = send - lo < L ? send - lo : L;
        mbar_expect_tx(full0 + 8 * (i % S), len * 4u);
        bulk_g2s(ring + (size_t)(i % S) * L, A.in + lo, len * 4u, full0 + 8 * (i % S));
      }
      // no copy may still be landing when the CTA leaves: wait for the last
      // fill of every slot
      for (uint32_t j = i > S ? i - S : 0; j < i; ++j)
        mbar_wait(full0 + 8 * (j % S), (j / S) & 1u, kOwnerWaitNs, nullptr);
    }
  } else {
    const Win W{ring, base, S * L};
    uint32_t waited = 0;    // every thread: segments [0, waited) seen filled
    uint32_t released = 0;  // the group's leader: segments [0, released) released
    uint32_t j = 0;         // the group's team count (dynamic counter parity)
    // the group's barrier; every member gets the same answer to "has any
    // member seen the give-up flag", so the group stops as one
    auto group_sync_stop = [&]() {
      const bool v = *(volatile int*)&s_bad != 0;
      if (Tl == 32) {
        __syncwarp();
        return __any_sync(0xffffffffu, v) != 0;
      }
      return named_barrier_or(1 + gr, Tl, v);
    };
    // the leader releases segments [released, upto): each after it is seen
    // filled, so an arrival always counts for the segment in the slot
    auto release = [&](uint32_t upto) {
      if (tt == 0) {
        for (; released < upto; ++released) {
          if (!mbar_wait(full0 + 8 * (released % S), (released / S) & 1u, kOwnerWaitNs,
                         A.status)) {
            s_bad = 1;
            break;
          }
          mbar_arrive(empty0 + 8 * (released % S));
        }
      }
    };
    for (uint32_t g = g0 + gr; g < g1; g += K, ++j) {  // group gr plays team g
      const uint32_t hi_seg = seg_hi(g);
      if (waited < seg_lo(g)) waited = seg_lo(g);  // segments below are never read here
      bool ok = !*(volatile int*)&s_bad;
      while (ok && waited < hi_seg) {
        if (!mbar_wait(full0 + 8 * (waited % S), (waited / S) & 1u, kOwnerWaitNs, A.status)) {
          ok = false;
          s_bad = 1;
          break;
        }
        ++waited;
      }
      ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the dynamic claims are warp-wide
      if (ok) {
        uint32_t bs, bn;
        owner_block(A, g, bs, bn);
        if constexpr (SCHED == kStatic) {
          const uint32_t qq = bn / Tl, rr = bn - qq * Tl;
          const uint32_t cnt = qq + (tt < rr ? 1u : 0u);
          const uint32_t s = qq * tt + (tt < rr ? tt : rr);
          owner_piece(A, W, bs + s, bs + s + cnt, lane);
        } else if constexpr (SCHED == kChunked) {
          const uint32_t c = A.chunk;
          if (c == 1) {
            if (tt < bn) owner_strided(A, W, bs + tt, Tl, (bn - tt + Tl - 1) / Tl);
          } else {
            for (uint64_t lo = (uint64_t)tt * c; lo < bn; lo += (uint64_t)Tl * c) {
              const uint64_t hi = lo + c < bn ? lo + c : bn;
              owner_piece(A, W, bs + (uint32_t)lo, bs + (uint32_t)hi, lane);
            }
          }
        } else {  // kDynamic
          const uint32_t c = A.chunk;
          const uint32_t nch = (uint32_t)(((uint64_t)bn + c - 1) / c);
          uint32_t* const cp = &ctr[gr][j & 1u];
          for (;;) {
            uint32_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(cp, 32u);
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (b0 >= nch) break;
            const uint32_t jj = b0 + lane;
            if (jj < nch) {
              const uint64_t lo = (uint64_t)jj * c;
              const uint64_t hi = lo + c < bn ? lo + c : bn;
              owner_piece(A, W, bs + (uint32_t)lo, bs + (uint32_t)hi, lane);
            }
          }
        }
      }
      // the team is done: its segments are read out, its counter idle
      const bool stop = group_sync_stop();
      // this counter serves the team after next; the segments below the next
      // team's go back to the producer
      if (SCHED == kDynamic && tt == 0) ctr[gr][j & 1u] = 0;
      if (stop) break;
      release(g + K < g1 ? seg_lo(g + K) : nseg);
    }
    if (!*(volatile int*)&s_bad) release(nseg);  // what this group will not read any more
  }
  __syncthreads();
}

// cudaErrorNotSupported (nothing launched) where this form does not apply:
// a schedule other than static / static(c) / dynamic(c), nx not a multiple of
// 4 (a unit would straddle rows), pointers not 16-byte aligned (bulk copies,
// 128-bit stores), n = 0 or n >= 2^32 (32-bit indices), teams of 1024 threads
// (the producer warp needs room), or a ring of `budget` bytes that cannot
// hold one team's segments with room to spare.
cudaError_t launch_stencil2d_owner(const void* in, float* out, uint64_t nx, uint64_t ny, int sched,
                                   uint64_t chunk, float c0, float c1, unsigned teams,
                                   unsigned threads, uint32_t budget, int sm_count, int max_smem,
                                   uint32_t* status, cudaStream_t st) {
  const uint64_t n = nx * ny;
  if ((sched != kStatic && sched != kChunked && sched != kDynamic) || budget == 0 || nx < 4 ||
      nx % 4 || ny < 1 || n == 0 || n >= (1ull << 32) || teams < 1 || threads < 32 ||
      threads > 512 || threads % 32 || (((uintptr_t)in | (uintptr_t)out) & 15))
    return cudaErrorNotSupported;
  if (sched != kStatic && chunk < 1) return cudaErrorNotSupported;
  OwnerArgs a;
  a.in = (const float*)in;
  a.out = out;
  a.nx = (uint32_t)nx;
  a.ny = (uint32_t)ny;
  a.n = (uint32_t)n;
  a.G = teams < n ? teams : (uint32_t)n;  // teams past n have empty blocks: nothing to run
  a.q = a.n / a.G;
  a.r = a.n - a.q * a.G;
  a.T = threads;
  const uint64_t maxb = (uint64_t)a.q + (a.r ? 1 : 0);
  // a chunk of at least a whole block is one chunk per block, as c itself
  a.chunk = sched == kStatic ? 0u : (uint32_t)(chunk < maxb ? chunk : maxb);
  a.nx_magic = (~0ull) / nx + 1;
  a.c0 = c0;
  a.c1 = c1;
  a.status = status;
  a.pass_teams = 1;
  // segments of about a row (4 KB .. 16 KB), the ring as many as the budget
  // holds.  K groups at work on K consecutive teams need about
  // (K maxb + 2 nx + 8) / L + 2 segments at once (span); K is the largest
  // that leaves a quarter of the ring (at least two segments) for the fills
  // in flight, and fits 1024 threads with the producer warp.
  const uint64_t cap = (budget < (uint64_t)max_smem ? budget : (uint64_t)max_smem);
  const uint64_t L = nx < 1024 ? 1024 : nx > 4096 ? 4096 : (nx + 31) / 32 * 32;
  uint64_t S = (cap > 256 ? cap - 256 : 0) / (4 * L);
  if (S > kOwnerMaxSlots) S = kOwnerMaxSlots;
  auto span = [&](uint64_t kk) { return (kk * maxb + 2 * nx + 8 + L - 1) / L + 1; };
  const uint64_t spare = S / 4 > 2 ? S / 4 : 2;
  if (S < 3 || span(1) + 2 > S) return cudaErrorNotSupported;
  uint64_t K = 1;
  const uint64_t kmax = (1024 - 32) / threads < kOwnerMaxGroups ? (1024 - 32) / threads
                                                                 : kOwnerMaxGroups;
  while (K < kmax && span(K + 1) + spare <= S) ++K;
  a.seg = (uint32_t)L;
  a.slots = (uint32_t)S;
  const size_t smem = (size_t)(S * L * 4 + 128);
  auto* kern = sched == kStatic    ? stencil2d_owner_kernel<kStatic>
               : sched == kChunked ? stencil2d_owner_kernel<kChunked>
                                   : stencil2d_owner_kernel<kDynamic>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)(K * threads + 32), smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  // resident CTAs, and no more groups than a CTA has teams
  uint64_t P = (uint64_t)per_sm * (uint64_t)sm_count;
  if (P > a.G) P = a.G;
  const uint64_t per_cta = a.G / P;  // every CTA has at least this many teams
  if (K > per_cta) K = per_cta;
  a.groups = (uint32_t)K;
  return launch_kernel(kern, dim3((unsigned)P), dim3((unsigned)(K * threads + 32)), smem, st, a);
}

}  // namespace rt
