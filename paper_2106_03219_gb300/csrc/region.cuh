// Loop executors: the kernel one "target teams distribute parallel for"
// region runs.  Level 1 gives team g a contiguous balanced block; level 2
// divides the block among the team's threads by the schedule; the body runs
// per logical iteration; an optional reduction is finished in the same launch
// (partial per team, flush, atomic-inc ticket, the last team combines).
#pragma once

#include <type_traits>

#include "rt_device.cuh"

namespace rt {

enum : int { kStatic = 0, kChunked = 1, kDynamic = 2, kAuto = 3, kDist = 4, kGuided = 5,
             kNonmono = 6 };

// Vectors each thread keeps in flight in the axpy body, and the largest team
// the region kernels are compiled for (the register budget follows from it).
#ifndef OMPRT_AXPY_INFLIGHT
#define OMPRT_AXPY_INFLIGHT 2
#endif
#ifndef OMPRT_MAX_THREADS
#define OMPRT_MAX_THREADS 1024
#endif
// Vectors each thread keeps in flight in the value bodies of reductions
// (int32: at most 2; with 3 its extremum instances under auto spill).
// Measured at n = 2^28 (L2 flushed), 3 against 2: fp32 max and min +6%,
// bf16 sum +3%, fp32 and int64 sums unchanged.
#ifndef OMPRT_LOAD_INFLIGHT
#define OMPRT_LOAD_INFLIGHT 3
#endif

// Everything a region kernel needs, passed by value (one parameter block).
struct RegionArgs {
  uint64_t n;       // trip count
  uint64_t chunk;   // level-2 chunk (kChunked / kDynamic / kDist; kGuided: minimum)
  uint64_t dist_chunk;  // kDist: level-1 distribute chunk d
  const void* x;
  void* y;
  void* out;
  int32_t* seq;     // map record: per-iteration ordinal within its thread (may be null)
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
  uint32_t stage_chunks;  // staged schedules: chunks per pass (0: the plain form)
  uint32_t stage_off;     // byte offset of the staging buffers in dynamic shared memory
  uint32_t stage_warp_bytes;  // staging buffer bytes per warp
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
  int32_t* seq;
  int32_t id;
  mutable int32_t ord;  // iterations this thread has run so far
  __device__ explicit BodyMapRecord(const RegionArgs& a)
      : owner((int32_t*)a.out), count((int32_t*)a.y), last((int32_t*)a.x), seq(a.seq), id(0),
        ord(0) {}
  __device__ bool vec_ok() const { return false; }
  struct S1 {};
  __device__ __forceinline__ void load1(uint64_t, S1&) const {}
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t i, const S1&, Acc&) const {
    owner[i] = id;
    if (count) atomicAdd(count + i, 1);
    if (seq) seq[i] = ord++;
  }
  template <bool kN = false>
  __device__ void load(uint64_t, Frag&) const {}
  template <class Acc, bool kN = false>
  __device__ void finish(uint64_t, Frag&, Acc&) const {}
};

struct BodyAxpyF32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  static constexpr int kInFlight = OMPRT_AXPY_INFLIGHT;
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
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc<kN>(x + i, f.x);
    ld8<kN>(y + i, f.y);
  }
  template <class Acc, bool kN = false>
  __device__ __forceinline__ void finish(uint64_t i, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) f.y[k] = as_u(__fmaf_rn(a, as_f(f.x[k]), as_f(f.y[k])));
    st8<kN>(y + i, f.y);
#pragma unroll
    for (int k = 0; k < 8; k += 2) acc_add2(acc, as_f(f.y[k]), as_f(f.y[k + 1]));
  }
  // staged dynamic path: x and y through shared memory, y written back
  static constexpr int kStageArrays = 2;
  static constexpr bool kStageWrites = true;
  static constexpr uint32_t kElemBytes = 4;
  __device__ const void* stage_src(int k) const { return k ? (const void*)y : (const void*)x; }
  __device__ void* stage_dst() const { return y; }
  template <class Acc>
  __device__ __forceinline__ void stage_unit(uint4 (&u)[2], Acc& acc) const {
    u[1].x = as_u(__fmaf_rn(a, as_f(u[0].x), as_f(u[1].x)));
    u[1].y = as_u(__fmaf_rn(a, as_f(u[0].y), as_f(u[1].y)));
    u[1].z = as_u(__fmaf_rn(a, as_f(u[0].z), as_f(u[1].z)));
    u[1].w = as_u(__fmaf_rn(a, as_f(u[0].w), as_f(u[1].w)));
    acc_add2(acc, as_f(u[1].x), as_f(u[1].y));
    acc_add2(acc, as_f(u[1].z), as_f(u[1].w));
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
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc<kN>(x + i, f.x);
    ld8<kN>(y + i, f.y);
  }
  template <class Acc, bool kN = false>
  __device__ __forceinline__ void finish(uint64_t i, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) f.y[k] = a * f.x[k] + f.y[k];
    st8<kN>(y + i, f.y);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add((int32_t)f.y[k]);
  }
  static constexpr int kStageArrays = 2;
  static constexpr bool kStageWrites = true;
  static constexpr uint32_t kElemBytes = 4;
  __device__ const void* stage_src(int k) const { return k ? (const void*)y : (const void*)x; }
  __device__ void* stage_dst() const { return y; }
  template <class Acc>
  __device__ __forceinline__ void stage_unit(uint4 (&u)[2], Acc& acc) const {
    u[1].x = a * u[0].x + u[1].x;
    u[1].y = a * u[0].y + u[1].y;
    u[1].z = a * u[0].z + u[1].z;
    u[1].w = a * u[0].w + u[1].w;
    acc.add((int32_t)u[1].x);
    acc.add((int32_t)u[1].y);
    acc.add((int32_t)u[1].z);
    acc.add((int32_t)u[1].w);
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
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc<kN>(x + i, f.x);
    ld8_nc<kN>(y + i, f.y);
  }
  template <class Acc, bool kN = false>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; k += 2)
      acc_add2(acc, __fmul_rn(as_f(f.x[k]), as_f(f.y[k])),
               __fmul_rn(as_f(f.x[k + 1]), as_f(f.y[k + 1])));
  }
  static constexpr int kStageArrays = 2;
  static constexpr bool kStageWrites = false;
  static constexpr uint32_t kElemBytes = 4;
  __device__ const void* stage_src(int k) const { return k ? (const void*)y : (const void*)x; }
  __device__ void* stage_dst() const { return nullptr; }
  template <class Acc>
  __device__ __forceinline__ void stage_unit(uint4 (&u)[2], Acc& acc) const {
    acc_add2(acc, __fmul_rn(as_f(u[0].x), as_f(u[1].x)), __fmul_rn(as_f(u[0].y), as_f(u[1].y)));
    acc_add2(acc, __fmul_rn(as_f(u[0].z), as_f(u[1].z)), __fmul_rn(as_f(u[0].w), as_f(u[1].w)));
  }
};

// Value body: element i of x is the reduction operand.
struct BodyLoadF32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  static constexpr int kInFlight = OMPRT_LOAD_INFLIGHT;
  struct Frag { uint32_t x[8]; };
  const float* x;
  __device__ explicit BodyLoadF32(const RegionArgs& r) : x((const float*)r.x) {}
  __device__ bool vec_ok() const { return ((uintptr_t)x & 31) == 0; }
  struct S1 { float x; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const { s.x = ld_nc(x + i); }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const { acc.add(s.x); }
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld8_nc<kN>(x + i, f.x); }
  template <class Acc, bool kN = false>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; k += 2) acc_add2(acc, as_f(f.x[k]), as_f(f.x[k + 1]));
  }
  static constexpr int kStageArrays = 1;
  static constexpr bool kStageWrites = false;
  static constexpr uint32_t kElemBytes = 4;
  __device__ const void* stage_src(int) const { return x; }
  __device__ void* stage_dst() const { return nullptr; }
  template <class Acc>
  __device__ __forceinline__ void stage_unit(uint4 (&u)[1], Acc& acc) const {
    acc_add2(acc, as_f(u[0].x), as_f(u[0].y));
    acc_add2(acc, as_f(u[0].z), as_f(u[0].w));
  }
};

// bf16 is the upper half of an fp32 pattern: widening is exact.
struct BodyLoadBF16 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 16;
  // one vector more in flight than the other value bodies: a 32-byte vector
  // holds 16 elements, twice the compensated adds per byte of fp32 (n = 2^28:
  // 6.25 TB/s with four against 5.76 with three; five or six: no change)
  static constexpr int kInFlight = OMPRT_LOAD_INFLIGHT + 1;
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
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld8_nc<kN>(x + i, f.x); }
  template <class Acc, bool kN = false>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k)  // elements 2k (low half) and 2k+1 (high half)
      acc_add2(acc, as_f(f.x[k] << 16), as_f(f.x[k] & 0xffff0000u));
  }
  static constexpr int kStageArrays = 1;
  static constexpr bool kStageWrites = false;
  static constexpr uint32_t kElemBytes = 2;
  __device__ const void* stage_src(int) const { return x; }
  __device__ void* stage_dst() const { return nullptr; }
  template <class Acc>
  __device__ __forceinline__ void stage_unit(uint4 (&u)[1], Acc& acc) const {
    const uint32_t w[4] = {u[0].x, u[0].y, u[0].z, u[0].w};
#pragma unroll
    for (int k = 0; k < 4; ++k) acc_add2(acc, as_f(w[k] << 16), as_f(w[k] & 0xffff0000u));
  }
};

struct BodyLoadI32 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 8;
  static constexpr int kInFlight = OMPRT_LOAD_INFLIGHT < 2 ? OMPRT_LOAD_INFLIGHT : 2;
  struct Frag { uint32_t x[8]; };
  const int32_t* x;
  __device__ explicit BodyLoadI32(const RegionArgs& r) : x((const int32_t*)r.x) {}
  __device__ bool vec_ok() const { return ((uintptr_t)x & 31) == 0; }
  struct S1 { int32_t x; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const { s.x = ld_nc(x + i); }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const { acc.add(s.x); }
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld8_nc<kN>(x + i, f.x); }
  template <class Acc, bool kN = false>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add((int32_t)f.x[k]);
  }
  static constexpr int kStageArrays = 1;
  static constexpr bool kStageWrites = false;
  static constexpr uint32_t kElemBytes = 4;
  __device__ const void* stage_src(int) const { return x; }
  __device__ void* stage_dst() const { return nullptr; }
  template <class Acc>
  __device__ __forceinline__ void stage_unit(uint4 (&u)[1], Acc& acc) const {
    acc.add((int32_t)u[0].x);
    acc.add((int32_t)u[0].y);
    acc.add((int32_t)u[0].z);
    acc.add((int32_t)u[0].w);
  }
};

struct BodyLoadI64 {
  static constexpr bool kVec = true;
  static constexpr int VEC = 4;
  static constexpr int kInFlight = OMPRT_LOAD_INFLIGHT;
  struct Frag { uint64_t x[4]; };
  const int64_t* x;
  __device__ explicit BodyLoadI64(const RegionArgs& r) : x((const int64_t*)r.x) {}
  __device__ bool vec_ok() const { return ((uintptr_t)x & 31) == 0; }
  struct S1 { int64_t x; };
  __device__ __forceinline__ void load1(uint64_t i, S1& s) const { s.x = ld_nc(x + i); }
  template <class Acc>
  __device__ __forceinline__ void finish1(uint64_t, const S1& s, Acc& acc) const { acc.add(s.x); }
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const { ld4x64_nc(x + i, f.x); }
  template <class Acc, bool kN = false>
  __device__ __forceinline__ void finish(uint64_t, Frag& f, Acc& acc) const {
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.add((int64_t)f.x[k]);
  }
  static constexpr int kStageArrays = 1;
  static constexpr bool kStageWrites = false;
  static constexpr uint32_t kElemBytes = 8;
  __device__ const void* stage_src(int) const { return x; }
  __device__ void* stage_dst() const { return nullptr; }
  template <class Acc>
  __device__ __forceinline__ void stage_unit(uint4 (&u)[1], Acc& acc) const {
    acc.add((int64_t)(((uint64_t)u[0].y << 32) | u[0].x));
    acc.add((int64_t)(((uint64_t)u[0].w << 32) | u[0].z));
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
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    ld8_nc<kN>(in + i, f.c);
    f.interior = i >= 1 && i + 8 < n;
    if (f.interior) {
      f.w = __ldg(in + i - 1);
      f.e = __ldg(in + i + 8);
    }
  }
  template <class Acc, bool kN = false>
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
    st8<kN>(out + i, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add(as_f(o[k]));
  }
  // staged form: one input window (the pass and one element on each side,
  // widened to 16-byte units) and an output buffer; needs n % 4 == 0
  static constexpr int kStageArrays = 1;
  static constexpr bool kStageWrites = true;
  static constexpr bool kStageHalo = true;
  static constexpr uint32_t kElemBytes = 4;
  __device__ const void* stage_src(int) const { return in; }
  __device__ void* stage_dst() const { return out; }
  __device__ uint64_t stage_halo() const { return 1; }
  __device__ uint64_t stage_n() const { return n; }
  // outputs gi .. gi+3 (gi % 4 == 0) from window w, w[j] = in[gi]
  template <class Acc>
  __device__ __forceinline__ float4 stage_unit_halo(const float* w, uint32_t j, uint64_t gi,
                                                    Acc& acc) const {
    const float4 cc = *(const float4*)(w + j);
    float4 o;
    if (gi >= 1 && gi + 4 < n) {  // all four interior
      const float wl = w[j - 1], er = w[j + 4];
      o.x = point(wl, cc.x, cc.y);
      o.y = point(cc.x, cc.y, cc.z);
      o.z = point(cc.y, cc.z, cc.w);
      o.w = point(cc.z, cc.w, er);
    } else {  // an end point among them: copied; its neighbours are not read
      o.x = gi == 0 || gi + 1 == n ? cc.x : point(w[j - 1], cc.x, cc.y);
      o.y = gi + 2 == n ? cc.y : point(cc.x, cc.y, cc.z);
      o.z = gi + 3 == n ? cc.z : point(cc.y, cc.z, cc.w);
      o.w = gi + 4 == n ? cc.w : point(cc.z, cc.w, w[j + 4]);
    }
    acc.add(o.x);
    acc.add(o.y);
    acc.add(o.z);
    acc.add(o.w);
    return o;
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
  template <bool kN = false>
  __device__ __forceinline__ void load(uint64_t i, Frag& f) const {
    const uint64_t r = row_of(i), c = i - r * nx;
    ld8_nc<kN>(in + i, f.c);
    f.interior = r >= 1 && r + 1 < ny && c >= 1 && c + 9 <= nx;
    if (f.interior) {
      ld8_nc<kN>(in + i - nx, f.nn);
      ld8_nc<kN>(in + i + nx, f.ss);
      f.w = __ldg(in + i - 1);
      f.e = __ldg(in + i + 8);
    }
  }
  template <class Acc, bool kN = false>
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
    st8<kN>(out + i, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc.add(as_f(o[k]));
  }
  // staged form: one input window (the pass and one row on each side,
  // widened to 16-byte units) and an output buffer; needs nx % 4 == 0, so a
  // 16-byte unit never straddles two rows
  static constexpr int kStageArrays = 1;
  static constexpr bool kStageWrites = true;
  static constexpr bool kStageHalo = true;
  static constexpr uint32_t kElemBytes = 4;
  __device__ const void* stage_src(int) const { return in; }
  __device__ void* stage_dst() const { return out; }
  __device__ uint64_t stage_halo() const { return nx; }
  __device__ uint64_t stage_n() const { return nx * ny; }
  // outputs gi .. gi+3 (gi % 4 == 0, so in one row, first column c % 4 == 0)
  // from window w, w[j] = in[gi].  Of the four, only column 0 (first) and
  // column nx - 1 (last) can be boundary columns.
  template <class Acc>
  __device__ __forceinline__ float4 stage_unit_halo(const float* w, uint32_t j, uint64_t gi,
                                                    Acc& acc) const {
    const float4 cc = *(const float4*)(w + j);
    const uint64_t r = row_of(gi), c = gi - r * nx;
    float4 o = cc;  // boundary rows are copied
    if (r >= 1 && r + 1 < ny) {
      const float4 nn = *(const float4*)(w + j - nx);
      const float4 ss = *(const float4*)(w + j + nx);
      o.x = c > 0 ? point(nn.x, ss.x, cc.y, w[j - 1], cc.x) : cc.x;
      o.y = point(nn.y, ss.y, cc.z, cc.x, cc.y);
      o.z = point(nn.z, ss.z, cc.w, cc.y, cc.z);
      o.w = c + 4 < nx ? point(nn.w, ss.w, w[j + 4], cc.z, cc.w) : cc.w;
    }
    acc.add(o.x);
    acc.add(o.y);
    acc.add(o.z);
    acc.add(o.w);
    return o;
  }
};

// ---------------------------------------------------------------------------
// Schedule runners.
// ---------------------------------------------------------------------------

template <class Body, class = void>
struct InFlight { static constexpr int value = 2; };
template <class Body>
struct InFlight<Body, std::void_t<decltype(Body::kInFlight)>> {
  static constexpr int value = Body::kInFlight;
};

// One iteration through the two-phase scalar interface.
template <class Body, class Acc>
__device__ __forceinline__ void run_one(const Body& b, uint64_t i, Acc& acc) {
  typename Body::S1 s;
  b.load1(i, s);
  b.finish1(i, s, acc);
}

// Scalar iterations base, base + step, ... (cnt of them) in groups of kU:
// all loads of a group are issued before any of its stores.  Bodies with
// many operands per iteration (the 2-D stencil) use groups of 2.
#ifndef OMPRT_WIDE_SCALAR_GROUP
#define OMPRT_WIDE_SCALAR_GROUP 2
#endif
#ifndef OMPRT_SCALAR_GROUP
#define OMPRT_SCALAR_GROUP 4
#endif
// static(1): each thread's iterations are a stride-T scalar sequence, the
// whole loop for that thread, so deeper groups pay (axpy at n = 2^26: 1.00 of
// the copy rate with 8, 0.92 with 4, 0.985 with 16; the 4096^2 2-D stencil:
// 0.38 with 4, 0.33 with 2, 0.31 with 8); elsewhere the scalar path is a head
// or tail and deeper groups only cost registers (spills in dist).
#ifndef OMPRT_STRIDED_GROUP
#define OMPRT_STRIDED_GROUP 8
#endif
#ifndef OMPRT_WIDE_STRIDED_GROUP
#define OMPRT_WIDE_STRIDED_GROUP 4
#endif
template <class Body>
struct ScalarGroup {
  static constexpr int value = InFlight<Body>::value >= 2 ? OMPRT_SCALAR_GROUP : OMPRT_WIDE_SCALAR_GROUP;
};
template <class Body>
struct StridedGroup {
  static constexpr int value = InFlight<Body>::value >= 2 ? OMPRT_STRIDED_GROUP : OMPRT_WIDE_STRIDED_GROUP;
};

template <class Body, class Acc, int kU = ScalarGroup<Body>::value>
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


// A contiguous range [a, e) owned by the calling thread: scalar head up to
// vector alignment, two vectors in flight, one more vector, scalar tail.
template <class Body, class Acc, bool kN = false>
__device__ __forceinline__ void run_range(const Body& b, uint64_t a, uint64_t e, Acc& acc) {
  if constexpr (Body::kVec) {
    constexpr uint64_t V = Body::VEC;
    if (e - a >= V && b.vec_ok()) {
      const uint64_t head = (V - a % V) % V;
      run_scalar(b, a, 1, head, acc);
      a += head;
      constexpr int N = InFlight<Body>::value;
      typename Body::Frag f[N];
      if constexpr (N >= 2) {
        for (; a + N * V <= e; a += N * V) {
#pragma unroll
          for (int k = 0; k < N; ++k) b.template load<kN>(a + k * V, f[k]);
#pragma unroll
          for (int k = 0; k < N; ++k) b.template finish<Acc, kN>(a + k * V, f[k], acc);
        }
      }
      for (; a + V <= e; a += V) {
        b.template load<kN>(a, f[0]);
        b.template finish<Acc, kN>(a, f[0], acc);
      }
    }
  }
  run_scalar(b, a, 1, e - a, acc);
}

// schedule(static, 1) inside a block: iterations base + t, base + t + T, ...
template <class Body, class Acc>
__device__ __forceinline__ void run_strided(const Body& b, uint64_t base, uint64_t cnt, uint32_t t,
                                            uint32_t T, Acc& acc) {
  if (t < cnt)
    run_scalar<Body, Acc, StridedGroup<Body>::value>(b, base + t, T, (cnt - t + T - 1) / T, acc);
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
      constexpr int N = InFlight<Body>::value;
      typename Body::Frag f[N];
      if constexpr (N >= 2) {
        for (; v + (N - 1) * nthr < nv; v += N * nthr) {
#pragma unroll
          for (int k = 0; k < N; ++k) b.load((v + k * nthr) * V, f[k]);
#pragma unroll
          for (int k = 0; k < N; ++k) b.finish((v + k * nthr) * V, f[k], acc);
        }
      }
      for (; v < nv; v += nthr) {
        b.load(v * V, f[0]);
        b.finish(v * V, f[0], acc);
      }
      tail_start = nv * V;
    }
  }
  if (tail_start + gtid < n)
    run_scalar(b, tail_start + gtid, nthr, (n - tail_start - gtid + nthr - 1) / nthr, acc);
}

// schedule(auto) for the 2-D stencil: the mapping is free, so each thread
// takes an 8-column strip of kStripRows rows (items numbered strip-fastest,
// so neighbouring threads take neighbouring strips) and walks down it with the
// rows above, at and below in registers: one new 32-byte row vector per output
// row, with the next row's load issued before the current row is computed.
// East / west neighbours across the strip edge are scalar loads that hit the
// sector a neighbouring thread just loaded.
constexpr uint32_t kStripRows = 8;

template <class Acc>
__device__ __forceinline__ void run_stencil2d_strips(const BodyStencil2D& b, Acc& acc) {
  const uint64_t nx = b.nx, ny = b.ny;
  const uint64_t strips = nx / 8, nrb = (ny + kStripRows - 1) / kStripRows;
  const uint64_t items = strips * nrb;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t it = gtid; it < items; it += nthr) {
    const uint64_t s = it % strips, rb = it / strips;
    const uint64_t col0 = 8 * s;
    const uint64_t r0 = rb * kStripRows, r1 = r0 + kStripRows < ny ? r0 + kStripRows : ny;
    uint32_t up[8], cur[8], dn[8];
    if (r0 >= 1) ld8_nc(b.in + (r0 - 1) * nx + col0, up);
    ld8_nc(b.in + r0 * nx + col0, cur);
    if (r0 + 1 < ny) ld8_nc(b.in + (r0 + 1) * nx + col0, dn);
    for (uint64_t r = r0; r < r1; ++r) {
      const uint64_t row = r * nx + col0;
      const bool inner = r != 0 && r + 1 != ny;
      float w = 0.f, e = 0.f;
      if (inner) {
        if (s > 0) w = __ldg(b.in + row - 1);
        if (s + 1 < strips) e = __ldg(b.in + row + 8);
      }
      uint32_t dn2[8];
      const bool more = r + 1 < r1 && r + 2 < ny;  // this strip needs row r + 2
      if (more) ld8_nc(b.in + (r + 2) * nx + col0, dn2);
      uint32_t o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint64_t col = col0 + k;
        if (!inner || col == 0 || col + 1 == nx) {
          o[k] = cur[k];
        } else {
          const float W = k > 0 ? as_f(cur[k - 1]) : w;
          const float E = k < 7 ? as_f(cur[k + 1]) : e;
          o[k] = as_u(b.point(as_f(up[k]), as_f(dn[k]), E, W, as_f(cur[k])));
        }
      }
      st8(b.out + row, o);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc.add(as_f(o[k]));
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        up[k] = cur[k];
        cur[k] = dn[k];
        if (more) dn[k] = dn2[k];
      }
    }
  }
}

// dist_schedule(static, d) with schedule(static, c): team g runs distribute
// chunks g, g + G, ...; inside each the threads split it by C1 (c = 0) or C2.
// Returns true when the calling thread runs the loop's final iteration.
template <class Body, class Acc>
__device__ __forceinline__ bool run_dist(const Body& b, uint64_t n, uint64_t d, uint64_t c,
                                         uint32_t g, uint32_t G, uint32_t t, uint32_t T,
                                         Acc& acc) {
  const uint64_t nd = n ? (n - 1) / d + 1 : 0;
  bool last = false;
  uint64_t j = g;
  if constexpr (Body::kVec) {
    constexpr uint64_t V = Body::VEC;
    // Fast path: d == c * T and c a multiple of the vector width, so every
    // full distribute chunk gives each thread c / V whole aligned vectors.
    if (InFlight<Body>::value >= 2 && c && c % V == 0 && d == c * T && b.vec_ok()) {
      const uint64_t per = c / V;                   // vectors per thread per chunk
      const uint64_t nfull = n / d;                 // full distribute chunks
      const uint64_t mine = g < nfull ? (nfull - 1 - g) / G + 1 : 0;
      const uint64_t total = mine * per;            // this thread's vectors
      const uint64_t base = (uint64_t)t * c;
      auto at = [=](uint64_t q) {                   // q-th vector of this thread
        return (g + (q / per) * G) * d + base + (q % per) * V;
      };
      constexpr int N = InFlight<Body>::value;
      typename Body::Frag f[N];
      uint64_t q = 0;
      if constexpr (N >= 2) {
        for (; q + N <= total; q += N) {
#pragma unroll
          for (int k = 0; k < N; ++k) b.load(at(q + k), f[k]);
#pragma unroll
          for (int k = 0; k < N; ++k) b.finish(at(q + k), f[k], acc);
        }
      }
      for (; q < total; ++q) {
        const uint64_t i0 = at(q);
        b.load(i0, f[0]);
        b.finish(i0, f[0], acc);
      }
      // what is left for this team is at most the partial last chunk
      j = (nd > nfull && nfull % G == g) ? nfull : nd;
      // a full last chunk ends in thread T-1's piece
      if (nd == nfull && nd && (nd - 1) % G == g && t == T - 1) last = true;
    }
  }
  // dist_schedule(static, T) with schedule(static, 1), the usual GPU
  // composite mapping: over the full distribute chunks thread t of team g
  // runs iterations g*T + t + q*G*T, one stride-G*T sequence, which the
  // scalar path runs in deep groups (one iteration per chunk at a time would
  // keep a single load in flight)
  if (j == g && c == 1 && d == T) {
    const uint64_t nfull = n / d;
    const uint64_t mine = g < nfull ? (nfull - 1 - g) / G + 1 : 0;
    run_scalar<Body, Acc, StridedGroup<Body>::value>(b, (uint64_t)g * T + t, (uint64_t)G * T, mine,
                                                     acc);
    j = (nd > nfull && nfull % G == g) ? nfull : nd;
    if (nd == nfull && nd && (nd - 1) % G == g && t == T - 1) last = true;
  }
  for (; j < nd; j += G) {
    const uint64_t bs = j * d;
    const uint64_t bn = n - bs > d ? d : n - bs;
    if (c == 0) {
      uint64_t s, cnt;
      split_even(bn, T, t, s, cnt);
      run_range(b, bs + s, bs + s + cnt, acc);
      if (j == nd - 1 && cnt > 0 && s + cnt == bn) last = true;
    } else if (c == 1) {
      run_strided(b, bs, bn, t, T, acc);
      if (j == nd - 1 && (bn - 1) % T == t) last = true;
    } else {
      const uint64_t nch = (bn - 1) / c + 1;
      for (uint64_t k = t; k < nch; k += T) {
        const uint64_t lo = k * c;
        run_range(b, bs + lo, bs + (bn - lo > c ? lo + c : bn), acc);
      }
      if (j == nd - 1 && (nch - 1) % T == t) last = true;
    }
  }
  return last;
}

// schedule(guided, c) inside the team block [bs, bs + bn): each request takes
// max(c, ceil(r / 2T)) of the r iterations not yet handed out (never more
// than r).  Lane 0 of a warp claims the next (up to) 32 such chunks with one
// compare-and-swap on the team's counter, writing their starts to the warp's
// row in shared memory as it computes them; every lane then runs the chunk
// its row entries bound.  The sizes depend only on r, so the partition is the
// same on every run.
__device__ __forceinline__ uint64_t guided_size(uint64_t r, uint64_t c, uint64_t twoT) {
  const uint64_t want = (r + twoT - 1) / twoT;
  const uint64_t s = want > c ? want : c;
  return s < r ? s : r;
}
// the same with 2T = 2^sh (a shift instead of a 64-bit division)
__device__ __forceinline__ uint64_t guided_size_sh(uint64_t r, uint64_t c, uint32_t sh) {
  const uint64_t want = (r + (1ull << sh) - 1) >> sh;
  const uint64_t s = want > c ? want : c;
  return s < r ? s : r;
}

constexpr uint32_t kGuidedMaxTries = 1u << 20;
// per warp: the 32 chunk starts of its current guided claim and the claim's end
static __shared__ unsigned long long rt_guided_row[OMPRT_MAX_THREADS / 32][33];

// Lane 0 claims the team's next (up to) 32 guided chunks, writing their starts
// and the claim's end to the warp's row.  Returns false (uniform over the
// warp) when the block is used up or the bounded retries ran out.  Kept out
// of line: inlined, its 32-step size loop shaped the register allocation of
// the streaming loop around it, and guided axpy at n = 2^26 ran at 0.29 /
// 0.64 / 0.37 of the copy rate for c = 1 / 64 / 256 against 0.48 / 0.84 /
// 0.84 out of line.
static __device__ __noinline__ bool guided_claim(unsigned long long* row, uint64_t bn, uint64_t c,
                                             unsigned long long* ctr, uint32_t* status) {
  const uint64_t twoT = 2ull * blockDim.x;
  const bool pow2 = (twoT & (twoT - 1)) == 0;
  const uint32_t sh = (uint32_t)__ffsll((long long)twoT) - 1;
  int done = 0;
  if (lane_id() == 0) {
    uint32_t tries = 0;
    for (;;) {
      const unsigned long long cur = atomicAdd(ctr, 0ull);
      if (cur >= bn) {
        done = 1;
        break;
      }
      uint64_t pos = cur;
      for (int k = 0; k < 32; ++k) {
        row[k] = pos;
        if (pos < bn) pos += pow2 ? guided_size_sh(bn - pos, c, sh) : guided_size(bn - pos, c, twoT);
      }
      row[32] = pos;
      if (atomicCAS(ctr, cur, (unsigned long long)pos) == cur) break;
      if (++tries >= kGuidedMaxTries) {  // bounded: give up, report, leave the loop
        set_status(status, OMPRT_DEV_TIMEOUT);
        done = 1;
        break;
      }
    }
  }
  done = __shfl_sync(0xffffffffu, done, 0);
  __syncwarp();  // the row lane 0 wrote is visible to the warp
  return !done;
}

template <class Body, class Acc>
__device__ __forceinline__ bool run_guided(const Body& b, uint64_t bs, uint64_t bn, uint64_t c,
                                           unsigned long long* ctr, uint32_t* status,
                                           Acc& acc) {
  const uint32_t lane = lane_id();
  unsigned long long* const row = rt_guided_row[warp_id()];
  bool last = false;
  while (guided_claim(row, bn, c, ctr, status)) {
    const uint64_t pos = row[lane], end = row[lane + 1];
    if (pos < end) {
      run_range(b, bs + pos, bs + end, acc);
      if (end == bn) last = true;
    }
    __syncwarp();  // the row is read before lane 0 writes the next claim's
  }
  return last;
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
// dynamic(c), static(c) and static for streaming bodies, staged through
// shared memory.
//
// The dispatch is the plain one: each warp takes 32 consecutive chunks (from
// the team's counter under dynamic, by the fixed round robin under static)
// and lane l owns chunk base + l, whose iterations it runs in full.  Only the
// data movement differs.  The 32 chunks are one contiguous
// range, so it is moved by bulk copies (one per array and pass of P chunks,
// P = a.stage_chunks) into the warp's buffer; each owner lane then runs its
// chunk's 16-byte units out of shared memory, starting at a lane-dependent
// unit so that the eight lanes of a 128-bit access phase hit distinct banks;
// a written array goes back by one bulk store per pass.  DRAM then sees whole
// contiguous ranges instead of 32 interleaved per-lane streams, which is what
// holds the plain form of this schedule far below the copy rate (measured
// 0.64 of peak for dynamic(256) axpy against 0.98 staged).  One buffer per
// warp: with shared memory fixed, more warps each waiting on a whole pass keep
// more bytes in flight than double-buffered warps do (measured 5.9 against
// 6.5 TB/s).  A trailing part of a pass that is not a whole 16-byte unit runs
// from global memory.
// ---------------------------------------------------------------------------
template <class Body, class = void>
struct Stageable : std::false_type {};
template <class Body>
struct Stageable<Body, std::void_t<decltype(Body::kStageArrays)>> : std::true_type {};
// bodies that read neighbours (the stencils): the pass's input window
// reaches stage_halo() elements beyond it on both sides
template <class Body, class = void>
struct StageHalo : std::false_type {};
template <class Body>
struct StageHalo<Body, std::void_t<decltype(Body::kStageHalo)>> : std::true_type {};

static __shared__ __align__(8) uint64_t rt_stage_bar[OMPRT_MAX_THREADS / 32];
constexpr uint64_t kStageWaitNs = 1000000000ull;  // 1 s: a pass takes microseconds

// True when team block [bs, ...) can be staged: every chunk starts on a
// 16-byte boundary of every staged array.
template <class Body>
__device__ __forceinline__ bool stage_ok(const Body& b, uint64_t bs) {
  uintptr_t m = (uintptr_t)(bs * Body::kElemBytes);
#pragma unroll
  for (int k = 0; k < Body::kStageArrays; ++k) m |= (uintptr_t)b.stage_src(k);
  if constexpr (Body::kStageWrites) m |= (uintptr_t)b.stage_dst();
  return (m & 15) == 0;
}

// Claim sources: the first chunk of the warp's next 32 (warp-uniform).
// dynamic: one atomicAdd(32) on the team's counter per warp.
struct ClaimDynamic {
  unsigned long long* ctr;
  __device__ __forceinline__ unsigned long long next() {
    unsigned long long base = 0;
    if (lane_id() == 0) base = atomicAdd(ctr, 32ull);
    return __shfl_sync(0xffffffffu, base, 0);
  }
};
// static(c): thread t owns chunks t, t + T, t + 2T, ..., so warp w's k-th
// set is chunks k*T + 32w + lane; static without chunk is the same with one
// chunk of bn / T per thread (used when T divides the block).
struct ClaimStatic {
  unsigned long long k;
  uint32_t T, w32;
  __device__ __forceinline__ unsigned long long next() { return (k++) * T + w32; }
};

// nonmonotonic dynamic: the team's groups of 32 chunks are split evenly
// among its warps (next[v] / end[v], in shared memory); a warp claims from its
// own range first, then from the other warps' ranges in turn.  A group is
// claimed by one atomicAdd on a range's counter; the plain read before it only
// skips ranges already used up (the add decides).  Returns the group's first
// chunk, or nch when no group is left.
struct ClaimNonmono {
  unsigned long long* gnext;      // [W] next group of each warp's range
  const unsigned long long* gend; // [W] end of each warp's range
  uint32_t W, w;
  unsigned long long nch;
  __device__ __forceinline__ unsigned long long next() {
    unsigned long long base = nch;
    if (lane_id() == 0) {
      for (uint32_t k = 0; k < W; ++k) {
        const uint32_t v = w + k < W ? w + k : w + k - W;
        if (*(volatile unsigned long long*)(gnext + v) >= gend[v]) continue;
        const unsigned long long grp = atomicAdd(gnext + v, 1ull);
        if (grp < gend[v]) {
          base = grp * 32ull;
          break;
        }
      }
    }
    return __shfl_sync(0xffffffffu, base, 0);
  }
};

template <class Body, class Acc, class Claim>
__device__ void run_staged(const Body& b, const RegionArgs& a, uint64_t bs, uint64_t bn,
                           uint64_t c, Claim claim, Acc& acc) {
  constexpr int A = Body::kStageArrays;
  constexpr uint32_t EB = Body::kElemBytes;
  constexpr uint32_t EPU = 16 / EB;  // elements per 16-byte unit
  const uint32_t P = a.stage_chunks;
  const uint32_t cb = (uint32_t)(c * EB);  // bytes per chunk, a multiple of 16 (host check)
  const uint32_t uc = cb / 16;             // units per chunk
  const uint64_t nch = bn ? (bn - 1) / c + 1 : 0;
  const uint32_t lane = lane_id(), w = warp_id();
  constexpr bool kHalo = StageHalo<Body>::value;
  // streaming bodies: array k at buf + k * array_bytes.  Halo bodies: the
  // input window at buf, the output buffer at the end of the warp's bytes.
  const size_t array_bytes = (size_t)P * cb;
  unsigned char* const buf = rt_dyn_smem + a.stage_off + (size_t)w * a.stage_warp_bytes;
  unsigned char* const outb = buf + a.stage_warp_bytes - array_bytes;
  const uint32_t bar = smem_addr(&rt_stage_bar[w]);
  if (lane == 0) mbar_init(bar);
  __syncwarp();
  uint32_t phase = 0;
  bool bad = false;
  while (!bad) {
    const unsigned long long base = claim.next();
    if (base >= nch) break;
    const uint32_t nclaim = (uint32_t)(nch - base < 32 ? nch - base : 32);
    for (uint32_t p0 = 0; p0 < nclaim; p0 += P) {
      const uint32_t np = nclaim - p0 < P ? nclaim - p0 : P;
      const uint64_t S = (base + p0) * c;  // the pass covers team-relative [S, E)
      const uint64_t E = (base + p0 + np) * c < bn ? (base + p0 + np) * c : bn;
      const uint32_t units = (uint32_t)((E - S) / EPU);
      const uint32_t bytes = units * 16;
      uint64_t wS = 0;  // halo bodies: the window is in[wS, wE)
      if (bytes) {
        bool ok = true;
        if constexpr (kHalo) {
          const uint64_t h = b.stage_halo(), nn = b.stage_n();  // nn % 4 == 0 (host check)
          wS = (bs + S > h ? bs + S - h : 0) & ~3ull;
          const uint64_t wE = ((bs + E + h < nn ? bs + E + h : nn) + 3) & ~3ull;
          if (lane == 0) {
            bulk_wait_read();  // the last store has read the output buffer
            const uint32_t wbytes = (uint32_t)((wE - wS) * 4);
            mbar_expect_tx(bar, wbytes);
            bulk_g2s(buf, (const float*)b.stage_src(0) + wS, wbytes, bar);
          }
        } else if (lane == 0) {
          if constexpr (Body::kStageWrites) bulk_wait_read();  // last store has read the buffer
          mbar_expect_tx(bar, A * bytes);
#pragma unroll
          for (int k = 0; k < A; ++k)
            bulk_g2s(buf + k * array_bytes, (const char*)b.stage_src(k) + (bs + S) * EB, bytes,
                     bar);
        }
        if (lane == 0) {
          // lane 0 waits (suspended, not spinning); the others block in the
          // warp barrier, which also orders their reads after lane 0's wait
          ok = mbar_wait(bar, phase, kStageWaitNs, a.status);
          if (!ok) mbar_wait(bar, phase, kStageWaitNs, nullptr);  // let copies in flight land
        }
        phase ^= 1;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        if (!ok) {  // give up on this team's remaining work
          bad = true;
          break;
        }
      }
      if (lane >= p0 && lane < p0 + np) {
        const uint64_t lo = (uint64_t)(lane - p0) * c;  // this lane's chunk, relative to S
        const uint64_t hi = lo + c < E - S ? lo + c : E - S;
        const uint64_t vend = (uint64_t)units * EPU;
        const uint32_t nu = vend > lo ? (uint32_t)(((hi < vend ? hi : vend) - lo) / EPU) : 0;
        if (nu) {
          const uint32_t u0 = (uint32_t)(lo / EPU);
          const uint32_t off = ((lane * (1u - uc)) & 7u) % nu;
          for (uint32_t q0 = 0; q0 < nu; ++q0) {
            uint32_t q = q0 + off;
            if (q >= nu) q -= nu;
            if constexpr (kHalo) {
              const uint64_t gi = bs + S + (uint64_t)(u0 + q) * 4;
              ((float4*)outb)[u0 + q] =
                  b.stage_unit_halo((const float*)buf, (uint32_t)(gi - wS), gi, acc);
            } else {
              uint4 u[A];
#pragma unroll
              for (int k = 0; k < A; ++k) u[k] = ((const uint4*)(buf + k * array_bytes))[u0 + q];
              b.stage_unit(u, acc);
              if constexpr (Body::kStageWrites)
                ((uint4*)(buf + (A - 1) * array_bytes))[u0 + q] = u[A - 1];
            }
          }
        }
        const uint64_t t0 = lo > vend ? lo : vend;
        if (hi > t0) run_scalar(b, bs + S + t0, 1, hi - t0, acc);
      }
      fence_proxy_async();
      __syncwarp();
      if constexpr (Body::kStageWrites) {
        if (lane == 0 && bytes)
          bulk_s2g((char*)b.stage_dst() + (bs + S) * EB, kHalo ? outb : buf + (A - 1) * array_bytes,
                   bytes);
      }
    }
  }
  if (lane == 0) bulk_wait_all();
  __syncwarp();
}

// ---------------------------------------------------------------------------
// The region kernel.
// ---------------------------------------------------------------------------
template <class Body, int SCHED, class Acc>
__global__ void __launch_bounds__(OMPRT_MAX_THREADS) region_kernel(const RegionArgs a) {
  enter_region_grid();
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
    if constexpr (std::is_same<Body, BodyStencil2D>::value) {
      if (body.vec_ok())
        run_stencil2d_strips(body, acc);
      else
        run_auto(body, a.n, acc);
    } else {
      run_auto(body, a.n, acc);
    }
    if constexpr (std::is_same<Body, BodyMapRecord>::value) {
      const uint64_t gtid = (uint64_t)g * T + t, nthr = (uint64_t)G * T;
      last = a.n > 0 && (a.n - 1) % nthr == gtid;
    }
  } else if constexpr (SCHED == kDist) {
    last = run_dist(body, a.n, a.dist_chunk, a.chunk, g, G, t, T, acc);
  } else {
    uint64_t bs, bn;  // level 1: the team's block
    split_even(a.n, G, g, bs, bn);
    const bool team_last = bn > 0 && bs + bn == a.n;
    if constexpr (SCHED == kStatic) {
      bool staged = false;
      if constexpr (Stageable<Body>::value) {
        // one chunk of bn / T per thread: the host stages only when every
        // team's block is T chunks of a.chunk (the size its buffers are for)
        staged = a.stage_chunks != 0 && a.chunk != 0 && bn == a.chunk * T && stage_ok(body, bs);
        if (staged) run_staged(body, a, bs, bn, a.chunk, ClaimStatic{0ull, T, warp_id() * 32u}, acc);
      }
      if (!staged) {
        uint64_t s, cnt;
        split_even(bn, T, t, s, cnt);
        run_range(body, bs + s, bs + s + cnt, acc);
        last = team_last && cnt > 0 && s + cnt == bn;
      }
    } else if constexpr (SCHED == kChunked) {
      const uint64_t c = a.chunk;
      const uint64_t nch = bn ? (bn - 1) / c + 1 : 0;
      bool staged = false;
      if constexpr (Stageable<Body>::value) {
        staged = a.stage_chunks != 0 && stage_ok(body, bs);
        if (staged) run_staged(body, a, bs, bn, c, ClaimStatic{0ull, T, warp_id() * 32u}, acc);
      }
      if (staged) {
      } else if (c == 1) {
        run_strided(body, bs, bn, t, T, acc);
      } else {
        for (uint64_t j = t; j < nch; j += T) {
          const uint64_t lo = j * c;
          run_range(body, bs + lo, bs + (bn - lo > c ? lo + c : bn), acc);
        }
      }
      last = team_last && nch > 0 && (nch - 1) % T == t;
    } else if constexpr (SCHED == kGuided) {
      unsigned long long* ctr = a.dyn_next + g;
      last = run_guided(body, bs, bn, a.chunk ? a.chunk : 1, ctr, a.status, acc) && team_last;
      team_barrier();
      if (t == 0) *ctr = 0;  // leave the counter at zero for the next launch
    } else if constexpr (SCHED == kNonmono) {
      // nonmonotonic dynamic: per-warp ranges of chunk groups in shared memory
      __shared__ unsigned long long nm_next[OMPRT_MAX_THREADS / 32], nm_end[OMPRT_MAX_THREADS / 32];
      const uint64_t c = a.chunk;
      const uint64_t nch = bn ? (bn - 1) / c + 1 : 0;
      const uint32_t lane = lane_id(), w = warp_id(), W = T / 32;
      if (lane == 0) {
        uint64_t s0, cnt;
        split_even((nch + 31) / 32, W, w, s0, cnt);
        nm_next[w] = s0;
        nm_end[w] = s0 + cnt;
      }
      team_barrier();  // every range is set before any warp steals
      ClaimNonmono cl{nm_next, nm_end, W, w, nch};
      bool staged = false;
      if constexpr (Stageable<Body>::value) {
        staged = a.stage_chunks != 0 && stage_ok(body, bs);
        if (staged) run_staged(body, a, bs, bn, c, cl, acc);
      }
      constexpr bool kNarrow = !std::is_same<Body, BodyStencil1D>::value &&
                               !std::is_same<Body, BodyStencil2D>::value;
      while (!staged) {
        const unsigned long long base = cl.next();
        if (base >= nch) break;
        const uint64_t j = base + lane;
        if (j < nch) {
          const uint64_t lo = j * c;
          run_range<Body, Acc, kNarrow>(body, bs + lo, bs + (bn - lo > c ? lo + c : bn), acc);
          if (j == nch - 1) last = team_last;
        }
      }
    } else {  // kDynamic: chunks of c claimed from this team's counter
      // pointwise bodies stream each lane's chunk with 128-bit accesses
      constexpr bool kNarrow = !std::is_same<Body, BodyStencil1D>::value &&
                               !std::is_same<Body, BodyStencil2D>::value;
      const uint64_t c = a.chunk;
      const uint64_t nch = bn ? (bn - 1) / c + 1 : 0;
      unsigned long long* ctr = a.dyn_next + g;
      const uint32_t lane = lane_id();
      bool staged = false;
      if constexpr (Stageable<Body>::value) {
        staged = a.stage_chunks != 0 && stage_ok(body, bs);  // uniform over the team
        if (staged) run_staged(body, a, bs, bn, c, ClaimDynamic{ctr}, acc);
      }
      while (!staged) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(ctr, 32ull);  // one claim of 32 chunks per warp
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nch) break;
        const uint64_t j = base + lane;
        if (j < nch) {
          const uint64_t lo = j * c;
          run_range<Body, Acc, kNarrow>(body, bs + lo, bs + (bn - lo > c ? lo + c : bn), acc);
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
