// Template launch helpers shared by the executor translation units (internal).
#pragma once

#include "launch.h"

namespace rt {

template <class Body, class Acc, int SCHED>
inline cudaError_t launch_one(unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                              const RegionArgs& a) {
  auto k = region_kernel<Body, SCHED, Acc>;
  static const size_t static_bytes = static_smem_of(k);
  const cudaError_t e = smem_optin(k, smem, static_bytes);
  if (e != cudaSuccess) return e;
  return launch_kernel(k, grid, block, smem, st, a);
}

template <class Body, class Acc>
inline cudaError_t launch_sched(int sched, unsigned grid, unsigned block, size_t smem,
                                cudaStream_t st, const RegionArgs& a) {
  switch (sched) {
    case kStatic: return launch_one<Body, Acc, kStatic>(grid, block, smem, st, a);
    case kChunked: return launch_one<Body, Acc, kChunked>(grid, block, smem, st, a);
    case kDynamic: return launch_one<Body, Acc, kDynamic>(grid, block, smem, st, a);
    case kAuto: return launch_one<Body, Acc, kAuto>(grid, block, smem, st, a);
    case kDist: return launch_one<Body, Acc, kDist>(grid, block, smem, st, a);
    case kGuided: return launch_one<Body, Acc, kGuided>(grid, block, smem, st, a);
    case kNonmono: return launch_one<Body, Acc, kNonmono>(grid, block, smem, st, a);
  }
  return cudaErrorNotSupported;
}

// Bodies whose reduction operand is fp32.
template <class Body>
inline cudaError_t launch_float_accs(int acc, int sched, unsigned grid, unsigned block,
                                     size_t smem, cudaStream_t st, const RegionArgs& a,
                                     bool allow_none) {
  switch (acc) {
    case kAccNone:
      if (!allow_none) return cudaErrorNotSupported;
      return launch_sched<Body, AccNone>(sched, grid, block, smem, st, a);
    case kAccCompF32: return launch_sched<Body, AccCompF32>(sched, grid, block, smem, st, a);
    case kAccNaiveF32: return launch_sched<Body, AccNaiveF32>(sched, grid, block, smem, st, a);
    case kAccMaxF32: return launch_sched<Body, AccExtF32<true>>(sched, grid, block, smem, st, a);
    case kAccMinF32: return launch_sched<Body, AccExtF32<false>>(sched, grid, block, smem, st, a);
  }
  return cudaErrorNotSupported;
}

// Bodies whose reduction operand is an integer.
template <class Body>
inline cudaError_t launch_int_accs(int acc, int sched, unsigned grid, unsigned block, size_t smem,
                                   cudaStream_t st, const RegionArgs& a, bool allow_none) {
  switch (acc) {
    case kAccNone:
      if (!allow_none) return cudaErrorNotSupported;
      return launch_sched<Body, AccNone>(sched, grid, block, smem, st, a);
    case kAccSumI64: return launch_sched<Body, AccSumI64>(sched, grid, block, smem, st, a);
    case kAccMaxI64: return launch_sched<Body, AccExtI64<true>>(sched, grid, block, smem, st, a);
    case kAccMinI64: return launch_sched<Body, AccExtI64<false>>(sched, grid, block, smem, st, a);
  }
  return cudaErrorNotSupported;
}

}  // namespace rt
