// Executor instances: fp32 and int32 axpy.
#include "launch_common.cuh"

namespace rt {

cudaError_t launch_axpy(int dtype, int acc, int sched, unsigned grid, unsigned block, size_t smem,
                        cudaStream_t st, const RegionArgs& a) {
  if (dtype == OMPRT_F32)
    return launch_float_accs<BodyAxpyF32>(acc, sched, grid, block, smem, st, a, true);
  if (dtype == OMPRT_I32)
    return launch_int_accs<BodyAxpyI32>(acc, sched, grid, block, smem, st, a, true);
  return cudaErrorNotSupported;
}

}  // namespace rt
