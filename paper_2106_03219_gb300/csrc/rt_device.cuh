// Device runtime core for sm_103a: thread hierarchy, atomics, barriers, the
// static iteration split, the team shared-memory stack, accumulators and the
// team / cross-team reduction.  Header-only, instantiated into each executor
// kernel (the role the paper gives to linking the runtime as bitcode into every
// kernel so it is specialised with it, Sec. 2.3).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "omprt.h"

namespace rt {

// ---------------------------------------------------------------------------
// Thread hierarchy: one OpenMP team is one thread block (Sec. 3.1, "Global
// Shared Variables"); ids come from the hardware registers (Sec. 3.2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t team_id() { return blockIdx.x; }
__device__ __forceinline__ uint32_t num_teams() { return gridDim.x; }
__device__ __forceinline__ uint32_t thread_id() { return threadIdx.x; }
__device__ __forceinline__ uint32_t team_size() { return blockDim.x; }
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t warp_id() { return threadIdx.x >> 5; }

// ---------------------------------------------------------------------------
// Back-to-back regions on one stream (programmatic dependent launch, sm_90
// and later).  The host launches every executor grid with programmatic
// stream serialisation, so a grid may be scheduled while the grid before it
// drains.  Each executor kernel therefore starts with `wait_for_prior_grid`,
// before its first global load or store: it returns once the grid before it
// has completed and that grid's writes are visible (at once when the grid was
// launched without the attribute).  `allow_next_grid` then lets the next
// grid start as soon as every block of this one is running; its blocks sit in
// their own wait until this grid ends, so they only take over what this
// grid's finished blocks leave free.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void wait_for_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_next_grid() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void enter_region_grid() {
  wait_for_prior_grid();
  allow_next_grid();
}

// ---------------------------------------------------------------------------
// The five runtime atomics (Sec. 3.1, Listing 3 and the inc definition after
// it), sequentially consistent on 32-bit words at device scope: a full fence
// on both sides of the hardware read-modify-write.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t atomic_add(uint32_t* x, uint32_t e) {
  __threadfence();
  uint32_t v = atomicAdd(x, e);
  __threadfence();
  return v;
}
// { v = x; x = x >= e ? 0 : x + 1; } -- exactly the hardware atom.inc rule.
__device__ __forceinline__ uint32_t atomic_inc(uint32_t* x, uint32_t e) {
  __threadfence();
  uint32_t v = atomicInc(x, e);
  __threadfence();
  return v;
}
// { v = x; if (x < e) x = e; }
__device__ __forceinline__ uint32_t atomic_max(uint32_t* x, uint32_t e) {
  __threadfence();
  uint32_t v = atomicMax(x, e);
  __threadfence();
  return v;
}
__device__ __forceinline__ uint32_t atomic_exchange(uint32_t* x, uint32_t e) {
  __threadfence();
  uint32_t v = atomicExch(x, e);
  __threadfence();
  return v;
}
// { v = x; if (x == e) x = d; }
__device__ __forceinline__ uint32_t atomic_cas(uint32_t* x, uint32_t e, uint32_t d) {
  __threadfence();
  uint32_t v = atomicCAS(x, e, d);
  __threadfence();
  return v;
}
// __kmpc_flush (Sec. 3.1, Listing 2): a device-scope fence.
__device__ __forceinline__ void flush() { __threadfence(); }

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bits) {
  atomicOr(status, bits);
}

// Wait until *flag == expect, for at most max_ns nanoseconds of the GPU's
// global timer.  On expiry the timeout bit is set and false returned; the
// caller then stops waiting (no device wait of the runtime is unbounded).
__device__ inline bool bounded_wait_eq(const volatile uint32_t* flag, uint32_t expect,
                                       uint64_t max_ns, uint32_t* status) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (*flag == expect) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > max_ns) {
      set_status(status, OMPRT_DEV_TIMEOUT);
      return false;
    }
    __nanosleep(256);
  }
}

// ---------------------------------------------------------------------------
// Synchronisation (Sec. 3.2): the whole team, or a named sub-team barrier
// over `count` threads (a multiple of 32) on hardware barrier `id` (1..15).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void team_barrier() { __syncthreads(); }
__device__ __forceinline__ void named_barrier(uint32_t id, uint32_t count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// The same barrier, returning to every participant whether any of them
// passed v = true (one uniform answer for the sub-team).
__device__ __forceinline__ bool named_barrier_or(uint32_t id, uint32_t count, bool v) {
  uint32_t r;
  asm volatile(
      "{ .reg .pred p, q; setp.ne.u32 q, %1, 0; bar.red.or.pred p, %2, %3, q; selp.u32 %0, 1, 0, "
      "p; }"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// ---------------------------------------------------------------------------
// Static split without chunk: entity k of P gets q + (k < r) iterations
// starting at k*q + min(k, r), q = n / P, r = n % P (balanced blocks in
// entity order).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_even(uint64_t n, uint32_t P, uint32_t k, uint64_t& start,
                                           uint64_t& count) {
  const uint64_t q = n / P;
  const uint32_t r = (uint32_t)(n - q * P);
  count = q + (k < r ? 1u : 0u);
  start = q * k + (k < r ? k : r);
}

// ---------------------------------------------------------------------------
// Team shared-memory stack (__kmpc_alloc_shared, Sec. 2.1, Listing 1).
// LIFO in the team's dynamic shared memory (S bytes), overflow to this team's
// slice of a global pool (also LIFO), then NULL plus a status bit.  Requests
// are rounded up to 16 bytes (0 counts as 1).  The state is a team-shared
// variable that starts uninitialised and is set explicitly at kernel entry
// (Sec. 3.1, "loader_uninitialized").  Calls are made by one thread of the
// team (the runtime serialises through thread 0).
// ---------------------------------------------------------------------------
struct TeamStack {
  uint32_t top_s, cap_s, top_q, cap_q;
  unsigned char* pool;
};

extern __shared__ __align__(16) unsigned char rt_dyn_smem[];
static __shared__ TeamStack rt_stack;
static __shared__ void* rt_bcast_ptr;
static __shared__ int rt_bcast_flag;

__device__ __forceinline__ void stack_init(uint32_t cap_s, unsigned char* pool, uint32_t cap_q) {
  rt_stack.top_s = 0;
  rt_stack.cap_s = cap_s;
  rt_stack.top_q = 0;
  rt_stack.cap_q = pool ? cap_q : 0;
  rt_stack.pool = pool;
}

__device__ __forceinline__ uint64_t stack_round(uint64_t bytes) {
  return ((bytes ? bytes : 1) + 15) & ~uint64_t(15);
}

__device__ inline void* alloc_shared(uint64_t bytes, uint32_t* status) {
  const uint64_t r = stack_round(bytes);
  TeamStack& s = rt_stack;
  if (r <= (uint64_t)(s.cap_s - s.top_s)) {
    void* p = rt_dyn_smem + s.top_s;
    s.top_s += (uint32_t)r;
    return p;
  }
  if (r <= (uint64_t)(s.cap_q - s.top_q)) {
    void* p = s.pool + s.top_q;
    s.top_q += (uint32_t)r;
    return p;
  }
  set_status(status, OMPRT_DEV_STACK_NOMEM);
  return nullptr;
}

// Region of a pointer returned by alloc_shared: 0 shared, 1 pool, 2 neither.
__device__ __forceinline__ int stack_region(const void* p) {
  const unsigned char* c = (const unsigned char*)p;
  if (c >= rt_dyn_smem && c < rt_dyn_smem + rt_stack.cap_s) return 0;
  if (rt_stack.pool && c >= rt_stack.pool && c < rt_stack.pool + rt_stack.cap_q) return 1;
  return 2;
}

// Returns the status bits raised (0 or OMPRT_DEV_STACK_ORDER).
__device__ inline uint32_t free_shared(void* p, uint64_t bytes, uint32_t* status) {
  if (p == nullptr) return 0;
  const uint64_t r = stack_round(bytes);
  TeamStack& s = rt_stack;
  const unsigned char* c = (const unsigned char*)p;
  const int reg = stack_region(p);
  if (reg == 0 && c + r == rt_dyn_smem + s.top_s) {
    s.top_s -= (uint32_t)r;
    return 0;
  }
  if (reg == 1 && c + r == s.pool + s.top_q) {
    s.top_q -= (uint32_t)r;
    return 0;
  }
  set_status(status, OMPRT_DEV_STACK_ORDER);
  return OMPRT_DEV_STACK_ORDER;
}

// Team-wide temporary: thread 0 allocates, every thread gets the pointer.
// Must be reached by the whole team.
__device__ inline void* team_alloc(uint64_t bytes, uint32_t* status) {
  if (threadIdx.x == 0) rt_bcast_ptr = alloc_shared(bytes, status);
  team_barrier();
  void* p = rt_bcast_ptr;
  team_barrier();
  return p;
}
__device__ inline void team_free(void* p, uint64_t bytes, uint32_t* status) {
  team_barrier();
  if (threadIdx.x == 0) free_shared(p, bytes, status);
}

#ifndef OMPRT_LD_HINT
#define OMPRT_LD_HINT ""
#endif

// ---------------------------------------------------------------------------
// Global-memory access helpers (inline PTX; 256-bit vectors need sm_100+).
// OMPRT_LD_HINT may add a PTX L2 prefetch-size qualifier (".L2::128B",
// ".L2::256B") to the streaming loads.  Measured on GB300 it does not speed up
// any schedule, and with thousands of per-thread streams the 256-byte
// prefetch nearly doubled the DRAM bytes read (blocks evicted before use), so
// the default is no hint.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ld_nc(const float* p) {
  float v;
  asm("ld.global.nc" OMPRT_LD_HINT ".f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_f(const float* p) {
  float v;
  asm("ld.global" OMPRT_LD_HINT ".f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_nc(const int32_t* p) {
  int32_t v;
  asm("ld.global.nc" OMPRT_LD_HINT ".s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_i(const int32_t* p) {
  int32_t v;
  asm("ld.global" OMPRT_LD_HINT ".s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int64_t ld_nc(const int64_t* p) {
  int64_t v;
  asm("ld.global.nc" OMPRT_LD_HINT ".s64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint16_t ld_nc(const uint16_t* p) {
  uint16_t v;
  asm("ld.global.nc" OMPRT_LD_HINT ".u16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}

// 32 bytes = 8 x 32-bit.  Wide form: one 256-bit access (sm_100+), not kept
// in L1.  Narrow form: two 128-bit accesses through L1.  Measured on GB300,
// the narrow form is 1.5x faster for dynamic(256) axpy, where every lane
// streams its own 1 KB chunk, and the wide form is faster for the static
// schedules (1.9x for static(64)) and for the stencils; the region kernel
// uses the narrow form only for dynamic schedules of pointwise bodies.
template <bool kNarrow = false>
__device__ __forceinline__ void ld8_nc(const void* p, uint32_t (&r)[8]) {
  if constexpr (kNarrow) {
    asm("ld.global.nc.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(p));
    asm("ld.global.nc.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) : "l"((const char*)p + 16));
  } else {
    asm("ld.global.nc.L1::no_allocate" OMPRT_LD_HINT ".v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "l"(p));
  }
}
template <bool kNarrow = false>
__device__ __forceinline__ void ld8(const void* p, uint32_t (&r)[8]) {
  if constexpr (kNarrow) {
    asm("ld.global.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(p));
    asm("ld.global.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) : "l"((const char*)p + 16));
  } else {
    asm("ld.global.L1::no_allocate" OMPRT_LD_HINT ".v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "l"(p));
  }
}
template <bool kNarrow = false>
__device__ __forceinline__ void st8(void* p, const uint32_t (&r)[8]) {
  if constexpr (kNarrow) {
    asm volatile("st.global.v4.b32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3]) : "memory");
    asm volatile("st.global.v4.b32 [%0], {%1,%2,%3,%4};" ::"l"((char*)p + 16), "r"(r[4]),
                 "r"(r[5]), "r"(r[6]), "r"(r[7]) : "memory");
  } else {
    asm volatile("st.global.L1::no_allocate.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                 "r"(r[7])
                 : "memory");
  }
}
// 32 bytes = 4 x 64-bit
__device__ __forceinline__ void ld4x64_nc(const void* p, uint64_t (&r)[4]) {
  asm("ld.global.nc.L1::no_allocate" OMPRT_LD_HINT ".v4.b64 {%0,%1,%2,%3}, [%4];"
      : "=l"(r[0]), "=l"(r[1]), "=l"(r[2]), "=l"(r[3])
      : "l"(p));
}

// ---------------------------------------------------------------------------
// Bulk copies between global and shared memory (the TMA engine's untiled
// form) with an mbarrier that counts the bytes in.  Both addresses and the
// size must be multiples of 16 bytes; callers check that before issuing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// an mbarrier whose phases complete after `count` arrivals
__device__ __forceinline__ void mbar_init_count(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one plain arrival (release semantics: the caller's earlier shared-memory
// reads are ordered before a waiter's later writes)
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// the one arrival of a phase, announcing `bytes` to come from bulk copies
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// store, committed as its own bulk group of the issuing thread
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// this thread's bulk stores have finished reading shared memory / are done
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// order this thread's shared-memory writes before later bulk copies read them
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Wait for phase `phase` of the mbarrier to complete, for at most max_ns of
// the global timer; on expiry set the timeout bit (if status) and return false.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t phase, uint64_t max_ns, uint32_t* status) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, "
        "1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(20000u)  // suspend up to 20 us per try instead of spinning
        : "memory");
    if (done) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > max_ns) {
      if (status) set_status(status, OMPRT_DEV_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ float as_f(uint32_t u) { return __uint_as_float(u); }
__device__ __forceinline__ uint32_t as_u(float f) { return __float_as_uint(f); }

// ---------------------------------------------------------------------------
// Accumulators (thread-local partial of a reduction clause).
// Each provides: Part (the value carried through the team tree), part(),
// merge(Part, Part), identity(), shfl_xor(Part, mask).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  // Knuth's TwoSum: s + e == a + b exactly, for any magnitudes.
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

struct AccNone {
  static constexpr bool kActive = false;
  template <class V>
  __device__ __forceinline__ void add(V) {}
};

// Integer sums, exact modulo 2^64.
struct AccSumI64 {
  static constexpr bool kActive = true;
  using Part = unsigned long long;
  Part s = 0;
  __device__ __forceinline__ void add(int32_t v) { s += (Part)(int64_t)v; }
  __device__ __forceinline__ void add(int64_t v) { s += (Part)v; }
  __device__ __forceinline__ Part part() const { return s; }
  __device__ static __forceinline__ Part identity() { return 0; }
  __device__ static __forceinline__ Part merge(Part a, Part b) { return a + b; }
  __device__ static __forceinline__ Part shfl(Part a, int m) {
    return __shfl_xor_sync(0xffffffffu, a, m);
  }
};

template <bool kMax>
struct AccExtI64 {
  static constexpr bool kActive = true;
  using Part = long long;
  Part m = kMax ? (Part)INT64_MIN : (Part)INT64_MAX;
  __device__ __forceinline__ void add(int32_t v) { add((int64_t)v); }
  __device__ __forceinline__ void add(int64_t v) { m = kMax ? (v > m ? v : m) : (v < m ? v : m); }
  __device__ __forceinline__ Part part() const { return m; }
  __device__ static __forceinline__ Part identity() {
    return kMax ? (Part)INT64_MIN : (Part)INT64_MAX;
  }
  __device__ static __forceinline__ Part merge(Part a, Part b) {
    return kMax ? (a > b ? a : b) : (a < b ? a : b);
  }
  __device__ static __forceinline__ Part shfl(Part a, int mm) {
    return __shfl_xor_sync(0xffffffffu, a, mm);
  }
};

// Two fp32 lanes in one 64-bit register, for the packed fp32x2 arithmetic of
// sm_100+ (each lane rounded to nearest like the scalar instruction).
__device__ __forceinline__ uint64_t pack2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(uint64_t r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ uint64_t add2_rn(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// Compensated fp32 sum: running (s, c) with s + c the sum so far; every add
// is an exact TwoSum whose rounding error is collected in c.  Two such sums
// run interleaved, one per lane of a packed fp32x2 register: add2 feeds a
// pair of values to both with one packed TwoSum (half the instructions of two
// scalar ones); add feeds the first.  part() joins them with one more TwoSum.
struct AccCompF32 {
  static constexpr bool kActive = true;
  static constexpr bool kPacked = true;
  using Part = float2;  // (s, c)
  uint64_t s2 = 0, c2 = 0;  // lanes (s0, s1) and (c0, c1); all-zero bits are (0.f, 0.f)
  __device__ __forceinline__ void add(float v) {
    float2 s = unpack2(s2), c = unpack2(c2);
    float t, e;
    two_sum(s.x, v, t, e);
    s2 = pack2(t, s.y);
    c2 = pack2(__fadd_rn(c.x, e), c.y);
  }
  __device__ __forceinline__ void add2(float a, float b) {
    const uint64_t v = pack2(a, b);
    const uint64_t t = add2_rn(s2, v);  // TwoSum, lane by lane
    const uint64_t bp = sub2(t, s2);
    const uint64_t ap = sub2(t, bp);
    const uint64_t e = add2_rn(sub2(s2, ap), sub2(v, bp));
    s2 = t;
    c2 = add2_rn(c2, e);
  }
  __device__ __forceinline__ Part part() const {
    const float2 s = unpack2(s2), c = unpack2(c2);
    float t, e;
    two_sum(s.x, s.y, t, e);
    return make_float2(t, __fadd_rn(__fadd_rn(c.x, c.y), e));
  }
  __device__ static __forceinline__ Part identity() { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ Part merge(Part a, Part b) {
    float t, e;
    two_sum(a.x, b.x, t, e);
    return make_float2(t, __fadd_rn(__fadd_rn(a.y, b.y), e));
  }
  __device__ static __forceinline__ Part shfl(Part a, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
  }
};

// Feed a, b (in this order) to an accumulator: packed where it has a pair
// form, else two adds.
template <class Acc>
__device__ __forceinline__ void acc_add2(Acc& acc, float a, float b) {
  if constexpr (std::is_same<Acc, AccCompF32>::value) {
    acc.add2(a, b);
  } else {
    acc.add(a);
    acc.add(b);
  }
}

struct AccNaiveF32 {
  static constexpr bool kActive = true;
  using Part = float;
  float s = 0.f;
  __device__ __forceinline__ void add(float v) { s = __fadd_rn(s, v); }
  __device__ __forceinline__ Part part() const { return s; }
  __device__ static __forceinline__ Part identity() { return 0.f; }
  __device__ static __forceinline__ Part merge(Part a, Part b) { return __fadd_rn(a, b); }
  __device__ static __forceinline__ Part shfl(Part a, int m) {
    return __shfl_xor_sync(0xffffffffu, a, m);
  }
};

// max / min over fp32; a NaN operand is skipped (fmaxf / fminf rule).
template <bool kMax>
struct AccExtF32 {
  static constexpr bool kActive = true;
  using Part = float;
  float m = kMax ? -__builtin_huge_valf() : __builtin_huge_valf();
  __device__ __forceinline__ void add(float v) { m = kMax ? fmaxf(m, v) : fminf(m, v); }
  __device__ __forceinline__ Part part() const { return m; }
  __device__ static __forceinline__ Part identity() {
    return kMax ? -__builtin_huge_valf() : __builtin_huge_valf();
  }
  __device__ static __forceinline__ Part merge(Part a, Part b) {
    return kMax ? fmaxf(a, b) : fminf(a, b);
  }
  __device__ static __forceinline__ Part shfl(Part a, int mm) {
    return __shfl_xor_sync(0xffffffffu, a, mm);
  }
};

// fp64 sum used only for the cross-team combine (the one step kept in fp64).
struct CombF64 {
  using Part = double;
  __device__ static __forceinline__ Part identity() { return 0.0; }
  __device__ static __forceinline__ Part merge(Part a, Part b) { return __dadd_rn(a, b); }
  __device__ static __forceinline__ Part shfl(Part a, int m) {
    return __shfl_xor_sync(0xffffffffu, a, m);
  }
};

// ---------------------------------------------------------------------------
// Team reduction: butterfly over the warp (shuffle xor), then the per-warp
// values through shared scratch (>= 32 Parts) and one more warp butterfly.
// The tree shape depends only on the team size, so the result is the same on
// every run.  Returns the team value in every thread of warp 0.
// ---------------------------------------------------------------------------
template <class M>
__device__ __forceinline__ typename M::Part warp_reduce(typename M::Part v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = M::merge(v, M::shfl(v, m));
  return v;
}

template <class M>
__device__ inline typename M::Part team_reduce(typename M::Part v, typename M::Part* scratch) {
  v = warp_reduce<M>(v);
  const uint32_t nw = blockDim.x >> 5;
  if (lane_id() == 0) scratch[warp_id()] = v;
  team_barrier();
  if (warp_id() == 0) {
    v = lane_id() < nw ? scratch[lane_id()] : M::identity();
    v = warp_reduce<M>(v);
  }
  team_barrier();
  return v;
}

}  // namespace rt
