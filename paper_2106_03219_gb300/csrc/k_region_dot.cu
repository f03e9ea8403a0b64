// Executor instances: dot product and fp32 / bf16 value reductions.
#include "launch_common.cuh"

namespace rt {

cudaError_t launch_dot_load(int body, int dtype, int acc, int sched, unsigned grid,
                            unsigned block, size_t smem, cudaStream_t st, const RegionArgs& a) {
  if (body == OMPRT_BODY_DOT)
    return launch_float_accs<BodyDotF32>(acc, sched, grid, block, smem, st, a, false);
  if (dtype == OMPRT_F32)
    return launch_float_accs<BodyLoadF32>(acc, sched, grid, block, smem, st, a, false);
  if (dtype == OMPRT_BF16)
    return launch_float_accs<BodyLoadBF16>(acc, sched, grid, block, smem, st, a, false);
  return cudaErrorNotSupported;
}

}  // namespace rt
