// Loop executors: the kernel one "target teams distribute parallel for"
// region runs.  Level 1 gives team g a contiguous balanced block; level 2
// divides the block among the team's threads by the schedule; the body runs
// per logical iteration; an optional reduction is finished in the same launch
// (partial per team, flush, atomic-inc ticket, the last team combines).
#pragma once

#include <type_traits>

#include "rt_device.cuh"

namespace rt {

enum : int { kStatic = 0, kChunked = 1, kDynamic = 2, kAuto = 3 };

// Everything a region kernel needs, passed by value (one parameter block).
struct RegionArgs {
  uint64_t n;       // trip count
  uint64_t chunk;   // level-2 chunk (kChunked / kDynamic)
  const void* x;
  void* y;
  void* out;
  float alpha_f;
  int32_t alpha_i;
  float c0, c1;     // stencil weights
  uint64_t nx, ny;  // 2-D grid
  uint64_t nx_magic;  // ceil(2^64 / nx) for the 32-bit-index division path
  uint32_t small_index;  // n < 2^32: row = umulhi(i, nx_magic)
  uint32_t prec;         // omprt_precision
  uint32_t stack_bytes;  // S of the team stack (dynamic shared memory)
  uint32_t pool_bytes;   // fallback pool bytes per team
  unsigned char* pool;   // team g's slice at pool + g * pool_bytes (g < pool_teams)
  uint32_t pool_teams;
  uint32_t pad;
  unsigned char* partials;        // 16 bytes per team
  uint32_t* ticket;               // cross-team ticket (wraps to 0 by itself)
  unsigned long long* dyn_next;   // per-team dynamic dispatch counters (left 0)
  void* result;                   // 8 bytes, device
  uint32_t* status;               // sticky device status word
};

// ---------------------------------------------------------------------------
// Loop bodies.  one(i, acc) runs logical iteration i; when kVec, load(i, f) /
// finish(i, f, acc) run iterations i .. i+VEC-1 (i a multiple of VEC) in two
// phases so several vectors can be in flight.
// ---------------------------------------------------------------------------
struct NoFrag {};

struct BodyMapRecord {
  static constexpr bool kVec = false;
  static constexpr int VEC = 1;
  using Frag = NoFrag;
  int32_t* owner;
  int32_t* count;
  int32_t* last;
  int32_t id;
  __device__ explicit BodyMapRecord(const RegionArgs& a)
      : owner((int32_t*)a.out), count((int32_t*)a.y), last((int32_t*)a.x), id(0) {}
  __device__ bool vec_ok() const { return false; }
  struct S1 {};
  __device__ __forceinline__ void load1(uint64_t, S1&) const {}
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t i, const S1&, Acc&) const {
    owner[i] = id;
    if (count) atomicAdd(count + i, 1);
  }
  __device__ void load(uint64_t, Frag&) const {}
  template <class Acc>
  __device__ void finish(uint64_t, Frag&, Acc&) const {}
};

struct BodyAxpyF32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  struct Frag { uint32_t x[8], y[8]; };
  const float* x;
  float* y;
  float a;
  __device__ explicit BodyAxpyF32(const RegionArgs& r)
      : x((const float*)r.x), y((float*)r.y), a(r.alpha_f) {}
  __device__ bool vec_ok() const { return (((uintptr_t)x | (uintptr_t)y) & 31) == 0; }
  struct S1 { float x, y; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const {
    s.x = ld_nc(x + i);
    s.y = ld_f(y + i);
  }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t i, const S1& s, Acc& acc) const {
    const float v = __fmaf_rn(a, s.x, s.y);
    y[i] = v;
    acc.add(v);
  }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc(x + i, f.x);
    ld8(y + i, f.y);
  }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t i, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) f.y[k] = as_u(__fmaf_rn(a, as_f(f.x[k]), as_f(f.y[k])));
    st8(y + i, f.y);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add(as_f(f.y[k]));
  }
};

struct BodyAxpyI32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  struct Frag { uint32_t x[8], y[8]; };
  const int32_t* x;
  int32_t* y;
  uint32_t a;
  __device__ explicit BodyAxpyI32(const RegionArgs& r)
      : x((const int32_t*)r.x), y((int32_t*)r.y), a((uint32_t)r.alpha_i) {}
  __device__ bool vec_ok() const { return (((uintptr_t)x | (uintptr_t)y) & 31) == 0; }
  struct S1 { int32_t x, y; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const {
    s.x = ld_nc(x + i);
    s.y = ld_i(y + i);
  }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t i, const S1& s, Acc& acc) const {
    const int32_t v = (int32_t)(a * (uint32_t)s.x + (uint32_t)s.y);
    y[i] = v;
    acc.add(v);
  }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc(x + i, f.x);
    ld8(y + i, f.y);
  }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t i, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) f.y[k] = a * f.x[k] + f.y[k];
    st8(y + i, f.y);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add((int32_t)f.y[k]);
  }
};

struct BodyDotF32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  struct Frag { uint32_t x[8], y[8]; };
  const float* x;
  const float* y;
  __device__ explicit BodyDotF32(const RegionArgs& r)
      : x((const float*)r.x), y((const float*)r.y) {}
  __device__ bool vec_ok() const { return (((uintptr_t)x | (uintptr_t)y) & 31) == 0; }
  struct S1 { float x, y; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const {
    s.x = ld_nc(x + i);
    s.y = ld_nc(y + i);
  }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const {
    acc.add(__fmul_rn(s.x, s.y));
  }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc(x + i, f.x);
    ld8_nc(y + i, f.y);
  }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add(__fmul_rn(as_f(f.x[k]), as_f(f.y[k])));
  }
};

// Value body: element i of x is the reduction operand.
struct BodyLoadF32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  struct Frag { uint32_t x[8]; };
  const float* x;
  __device__ explicit BodyLoadF32(const RegionArgs& r) : x((const float*)r.x) {}
  __device__ bool vec_ok() const { return ((uintptr_t)x & 31) == 0; }
  struct S1 { float x; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const { s.x = ld_nc(x + i); }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const { acc.add(s.x); }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld8_nc(x + i, f.x); }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add(as_f(f.x[k]));
  }
};

// bf16 is the upper half of an fp32 pattern: widening is exact.
struct BodyLoadBF16 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 16;
  struct Frag { uint32_t x[8]; };
  const uint16_t* x;
  __device__ explicit BodyLoadBF16(const RegionArgs& r) : x((const uint16_t*)r.x) {}
  __device__ bool vec_ok() const { return ((uintptr_t)x & 31) == 0; }
  struct S1 { uint16_t x; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const { s.x = ld_nc(x + i); }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const {
    acc.add(as_f((uint32_t)s.x << 16));
  }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld8_nc(x + i, f.x); }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      acc.add(as_f(f.x[k] << 16));           // element 2k (low half)
      acc.add(as_f(f.x[k] & 0xffff0000u));   // element 2k+1 (high half)
    }
  }
};

struct BodyLoadI32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  struct Frag { uint32_t x[8]; };
  const int32_t* x;
  __device__ explicit BodyLoadI32(const RegionArgs& r) : x((const int32_t*)r.x) {}
  __device__ bool vec_ok() const { return ((uintptr_t)x & 31) == 0; }
  struct S1 { int32_t x; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const { s.x = ld_nc(x + i); }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const { acc.add(s.x); }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld8_nc(x + i, f.x); }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add((int32_t)f.x[k]);
  }
};

struct BodyLoadI64 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 4;
  struct Frag { uint64_t x[4]; };
  const int64_t* x;
  __device__ explicit BodyLoadI64(const RegionArgs& r) : x((const int64_t*)r.x) {}
  __device__ bool vec_ok() const { return ((uintptr_t)x & 31) == 0; }
  struct S1 { int64_t x; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const { s.x = ld_nc(x + i); }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const { acc.add(s.x); }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld4x64_nc(x + i, f.x); }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.add((int64_t)f.x[k]);
  }
};

// 1-D 3-point stencil, out of place; end points copied.
struct BodyStencil1D {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  struct Frag { uint32_t c[8]; float w, e; bool interior; };
  const float* in;
  float* out;
  uint64_t n;
  float c0, c1;
  __device__ explicit BodyStencil1D(const RegionArgs& r)
      : in((const float*)r.x), out((float*)r.out), n(r.n), c0(r.c0), c1(r.c1) {}
  __device__ bool vec_ok() const { return (((uintptr_t)in | (uintptr_t)out) & 31) == 0; }
  __device__ __forceinline__ float point(float w, float c, float e) const {
    return __fmaf_rn(c1, __fadd_rn(w, e), __fmul_rn(c0, c));
  }
  struct S1 { float w, c, e; bool edge; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const {
    s.c = __ldg(in + i);
    s.edge = i == 0 || i + 1 == n;
    if (!s.edge) {
      s.w = __ldg(in + i - 1);
      s.e = __ldg(in + i + 1);
    }
  }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t i, const S1& s, Acc& acc) const {
    const float v = s.edge ? s.c : point(s.w, s.c, s.e);
    out[i] = v;
    acc.add(v);
  }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc(in + i, f.c);
    f.interior = i >= 1 && i + 8 < n;
    if (f.interior) {
      f.w = __ldg(in + i - 1);
      f.e = __ldg(in + i + 8);
    }
  }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t i, Frag& f, Acc& acc) const {
    if (!f.interior) {
#pragma unroll 1
      for (int k = 0; k < 8; ++k) run_one(*this, i + k, acc);
      return;
    }
    uint32_t o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = k > 0 ? as_f(f.c[k - 1]) : f.w;
      const float e = k < 7 ? as_f(f.c[k + 1]) : f.e;
      o[k] = as_u(point(w, as_f(f.c[k]), e));
    }
    st8(out + i, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add(as_f(o[k]));
  }
};

// 2-D 5-point stencil on ny x nx row-major, out of place; boundary copied.
struct BodyStencil2D {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  static constexpr int kInFlight = 1;  // 5 operands per vector: one in flight fits 64 registers
  struct Frag { uint32_t c[8], nn[8], ss[8]; float w, e; bool interior; };
  const float* in;
  float* out;
  uint64_t nx, ny, magic;
  uint32_t small;
  float c0, c1;
  __device__ explicit BodyStencil2D(const RegionArgs& r)
      : in((const float*)r.x), out((float*)r.out), nx(r.nx), ny(r.ny), magic(r.nx_magic),
        small(r.small_index), c0(r.c0), c1(r.c1) {}
  __device__ bool vec_ok() const {
    return ((((uintptr_t)in | (uintptr_t)out) & 31) == 0) && (nx % 8 == 0);
  }
  __device__ __forceinline__ uint64_t row_of(uint64_t i) const {
    // exact for i, nx < 2^32 with magic = ceil(2^64 / nx)
    if (nx == 1) return i;
    return small ? __umul64hi(i, magic) : i / nx;
  }
  __device__ __forceinline__ float point(float nn, float ss, float e, float w, float c) const {
    return __fmaf_rn(c1, __fadd_rn(__fadd_rn(nn, ss), __fadd_rn(e, w)), __fmul_rn(c0, c));
  }
  struct S1 { float nn, ss, e, w, c; bool edge; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const {
    const uint64_t r = row_of(i), c = i - r * nx;
    s.c = __ldg(in + i);
    s.edge = r == 0 || c == 0 || r + 1 == ny || c + 1 == nx;
    if (!s.edge) {
      s.nn = __ldg(in + i - nx);
      s.ss = __ldg(in + i + nx);
      s.e = __ldg(in + i + 1);
      s.w = __ldg(in + i - 1);
    }
  }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t i, const S1& s, Acc& acc) const {
    const float v = s.edge ? s.c : point(s.nn, s.ss, s.e, s.w, s.c);
    out[i] = v;
    acc.add(v);
  }
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    const uint64_t r = row_of(i), c = i - r * nx;
    ld8_nc(in + i, f.c);
    f.interior = r >= 1 && r + 1 < ny && c >= 1 && c + 9 <= nx;
    if (f.interior) {
      ld8_nc(in + i - nx, f.nn);
      ld8_nc(in + i + nx, f.ss);
      f.w = __ldg(in + i - 1);
      f.e = __ldg(in + i + 8);
    }
  }
  template <class Acc>
  __device__ __forceinline__ void finish(uint64_t i, Frag& f, Acc& acc) const {
    if (!f.interior) {
#pragma unroll 1
      for (int k = 0; k < 8; ++k) run_one(*this, i + k, acc);
      return;
    }
    uint32_t o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = k > 0 ? as_f(f.c[k - 1]) : f.w;
      const float e = k < 7 ? as_f(f.c[k + 1]) : f.e;
      o[k] = as_u(point(as_f(f.nn[k]), as_f(f.ss[k]), e, w, as_f(f.c[k])));
    }
    st8(out + i, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add(as_f(o[k]));
  }
};

// ---------------------------------------------------------------------------
// Schedule runners.
// ---------------------------------------------------------------------------

// One iteration through the two-phase scalar interface.
template <class Body, class Acc>
__device__ __forceinline__ void run_one(const Body& b, uint64_t i, Acc& acc) {
  typename Body::S1 s;
  b.load1(i, s);
  b.finish1(i, s, acc);
}

// Scalar iterations base, base + step, ... (cnt of them) in groups of kU:
// all loads of a group are issued before any of its stores.
constexpr int kU = 4;
template <class Body, class Acc>
__device__ __forceinline__ void run_scalar(const Body& b, uint64_t base, uint64_t step,
                                           uint64_t cnt, Acc& acc) {
  uint64_t k = 0;
  for (; k + kU <= cnt; k += kU) {
    typename Body::S1 s[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) b.load1(base + (k + u) * step, s[u]);
#pragma unroll
    for (int u = 0; u < kU; ++u) b.finish1(base + (k + u) * step, s[u], acc);
  }
  for (; k < cnt; ++k) run_one(b, base + k * step, acc);
}

template <class Body, class = void>
struct InFlight { static constexpr int value = 2; };
template <class Body>
struct InFlight<Body, std::void_t<decltype(Body::kInFlight)>> {
  static constexpr int value = Body::kInFlight;
};

// A contiguous range [a, e) owned by the calling thread: scalar head up to
// vector alignment, two vectors in flight, one more vector, scalar tail.
template <class Body, class Acc>
__device__ __forceinline__ void run_range(const Body& b, uint64_t a, uint64_t e, Acc& acc) {
  if constexpr (Body::kVec) {
    constexpr uint64_t V = Body::VEC;
    if (e - a >= V && b.vec_ok()) {
      const uint64_t head = (V - a % V) % V;
      run_scalar(b, a, 1, head, acc);
      a += head;
      typename Body::Frag f0, f1;
      if constexpr (InFlight<Body>::value >= 2) {
        for (; a + 2 * V <= e; a += 2 * V) {
          b.load(a, f0);
          b.load(a + V, f1);
          b.finish(a, f0, acc);
          b.finish(a + V, f1, acc);
        }
      }
      for (; a + V <= e; a += V) {
        b.load(a, f0);
        b.finish(a, f0, acc);
      }
    }
  }
  run_scalar(b, a, 1, e - a, acc);
}

// schedule(static, 1) inside a block: iterations base + t, base + t + T, ...
template <class Body, class Acc>
__device__ __forceinline__ void run_strided(const Body& b, uint64_t base, uint64_t cnt, uint32_t t,
                                            uint32_t T, Acc& acc) {
  if (t < cnt) run_scalar(b, base + t, T, (cnt - t + T - 1) / T, acc);
}

// schedule(auto): 32-byte vectors grid-stride over the whole loop.
template <class Body, class Acc>
__device__ __forceinline__ void run_auto(const Body& b, uint64_t n, Acc& acc) {
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  uint64_t tail_start = 0;
  if constexpr (Body::kVec) {
    constexpr uint64_t V = Body::VEC;
    if (b.vec_ok()) {
      const uint64_t nv = n / V;
      uint64_t v = gtid;
      typename Body::Frag f0, f1;
      if constexpr (InFlight<Body>::value >= 2) {
        for (; v + nthr < nv; v += 2 * nthr) {
          b.load(v * V, f0);
          b.load((v + nthr) * V, f1);
          b.finish(v * V, f0, acc);
          b.finish((v + nthr) * V, f1, acc);
        }
      }
      for (; v < nv; v += nthr) {
        b.load(v * V, f0);
        b.finish(v * V, f0, acc);
      }
      tail_start = nv * V;
    }
  }
  if (tail_start + gtid < n)
    run_scalar(b, tail_start + gtid, nthr, (n - tail_start - gtid + nthr - 1) / nthr, acc);
}

// ---------------------------------------------------------------------------
// Cross-team reduction epilogue.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_part(unsigned char* p, unsigned long long v) {
  *(unsigned long long*)p = v;
}
__device__ __forceinline__ void store_part(unsigned char* p, long long v) { *(long long*)p = v; }
__device__ __forceinline__ void store_part(unsigned char* p, float v) { *(float*)p = v; }
__device__ __forceinline__ void store_part(unsigned char* p, float2 v) { *(float2*)p = v; }
__device__ __forceinline__ void store_part(unsigned char* p, double v) { *(double*)p = v; }

template <class P>
__device__ __forceinline__ P load_part(const unsigned char* p) {
  return __ldcg((const P*)p);
}

__device__ __forceinline__ void write_result(void* r, unsigned long long v) {
  *(long long*)r = (long long)v;
}
__device__ __forceinline__ void write_result(void* r, long long v) { *(long long*)r = v; }
__device__ __forceinline__ void write_result(void* r, float v) { *(double*)r = (double)v; }
__device__ __forceinline__ void write_result(void* r, float2 v) {
  *(double*)r = (double)__fadd_rn(v.x, v.y);
}
__device__ __forceinline__ void write_result(void* r, double v) { *(double*)r = v; }

// Combine partials[0..G) in the last team: thread t folds partials t, t+T, ...
// in team order, then the fixed-shape team tree.
template <class M, class P>
__device__ inline void combine_partials(const RegionArgs& a, void* scratch) {
  P v = M::identity();
  for (uint32_t k = threadIdx.x; k < gridDim.x; k += blockDim.x)
    v = M::merge(v, load_part<P>(a.partials + 16ull * k));
  v = team_reduce<M>(v, (P*)scratch);
  if (threadIdx.x == 0) write_result(a.result, v);
}

template <class Acc>
__device__ inline void reduce_epilogue(const Acc& acc, const RegionArgs& a) {
  using P = typename Acc::Part;
  void* scratch = team_alloc(32 * 16, a.status);  // runtime temporary on the team stack
  if (scratch == nullptr) return;                  // flagged OMPRT_DEV_STACK_NOMEM
  const P v = team_reduce<Acc>(acc.part(), (P*)scratch);
  constexpr bool kComp = std::is_same<P, float2>::value;
  if (threadIdx.x == 0) {
    unsigned char* slot = a.partials + 16ull * blockIdx.x;
    if constexpr (kComp) {
      // compensated pair: fp64 partial (exact: |c| <= ulp(s)/2) or the pair
      if (a.prec == OMPRT_PREC_COMP_F64)
        store_part(slot, __dadd_rn((double)v.x, (double)v.y));
      else
        store_part(slot, v);
    } else {
      store_part(slot, v);
    }
    flush();  // the partial is visible device-wide before the ticket
    const uint32_t tk = atomic_inc(a.ticket, gridDim.x - 1);
    rt_bcast_flag = (tk == gridDim.x - 1);
  }
  team_barrier();
  if (rt_bcast_flag) {
    flush();
    if constexpr (kComp) {
      if (a.prec == OMPRT_PREC_COMP_F64)
        combine_partials<CombF64, double>(a, scratch);
      else
        combine_partials<Acc, P>(a, scratch);
    } else {
      combine_partials<Acc, P>(a, scratch);
    }
  }
  team_free(scratch, 32 * 16, a.status);
}

// ---------------------------------------------------------------------------
// The region kernel.
// ---------------------------------------------------------------------------
template <class Body, int SCHED, class Acc>
__global__ void __launch_bounds__(1024) region_kernel(const RegionArgs a) {
  const uint32_t g = blockIdx.x, G = gridDim.x, t = threadIdx.x, T = blockDim.x;
  Body body(a);
  Acc acc;
  if constexpr (Acc::kActive) {
    if (t == 0)
      stack_init(a.stack_bytes, g < a.pool_teams ? a.pool + (uint64_t)g * a.pool_bytes : nullptr,
                 a.pool_bytes);
    // made visible by the barrier inside team_alloc
  }
  bool last = false;  // this thread runs the loop's final iteration
  if constexpr (std::is_same<Body, BodyMapRecord>::value) body.id = (int32_t)(g * T + t);
  if constexpr (SCHED == kAuto) {
    run_auto(body, a.n, acc);
    if constexpr (std::is_same<Body, BodyMapRecord>::value) {
      const uint64_t gtid = (uint64_t)g * T + t, nthr = (uint64_t)G * T;
      last = a.n > 0 && (a.n - 1) % nthr == gtid;
    }
  } else {
    uint64_t bs, bn;  // level 1: the team's block
    split_even(a.n, G, g, bs, bn);
    const bool team_last = bn > 0 && bs + bn == a.n;
    if constexpr (SCHED == kStatic) {
      uint64_t s, cnt;
      split_even(bn, T, t, s, cnt);
      run_range(body, bs + s, bs + s + cnt, acc);
      last = team_last && cnt > 0 && s + cnt == bn;
    } else if constexpr (SCHED == kChunked) {
      const uint64_t c = a.chunk;
      const uint64_t nch = bn ? (bn - 1) / c + 1 : 0;
      if (c == 1) {
        run_strided(body, bs, bn, t, T, acc);
      } else {
        for (uint64_t j = t; j < nch; j += T) {
          const uint64_t lo = j * c;
          run_range(body, bs + lo, bs + (bn - lo > c ? lo + c : bn), acc);
        }
      }
      last = team_last && nch > 0 && (nch - 1) % T == t;
    } else {  // kDynamic: chunks of c claimed from this team's counter
      const uint64_t c = a.chunk;
      const uint64_t nch = bn ? (bn - 1) / c + 1 : 0;
      unsigned long long* ctr = a.dyn_next + g;
      const uint32_t lane = lane_id();
      for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(ctr, 32ull);  // one claim of 32 chunks per warp
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nch) break;
        const uint64_t j = base + lane;
        if (j < nch) {
          const uint64_t lo = j * c;
          run_range(body, bs + lo, bs + (bn - lo > c ? lo + c : bn), acc);
          if (j == nch - 1) last = team_last;
        }
      }
      team_barrier();
      if (t == 0) *ctr = 0;  // leave the counter at zero for the next launch
    }
  }
  if constexpr (std::is_same<Body, BodyMapRecord>::value) {
    if (body.last) body.last[(uint64_t)g * T + t] = last ? 1 : 0;
  }
  if constexpr (Acc::kActive) reduce_epilogue(acc, a);
}

}  // namespace rt
