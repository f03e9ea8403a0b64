// Executor instances for fp32 / bf16 data: axpy, stencils, dot, value loads.
#include "launch_common.cuh"

namespace rt {

cudaError_t launch_region_f32(int body, int dtype, int acc, int sched, unsigned grid,
                              unsigned block, size_t smem, cudaStream_t st, const RegionArgs& a) {
  switch (body) {
    case OMPRT_BODY_AXPY:
      if (dtype != OMPRT_F32) break;
      return launch_float_accs<BodyAxpyF32>(acc, sched, grid, block, smem, st, a, true);
    case OMPRT_BODY_STENCIL1D3:
      if (dtype != OMPRT_F32) break;
      return launch_float_accs<BodyStencil1D>(acc, sched, grid, block, smem, st, a, true);
    case OMPRT_BODY_STENCIL2D5:
      if (dtype != OMPRT_F32) break;
      return launch_float_accs<BodyStencil2D>(acc, sched, grid, block, smem, st, a, true);
    case OMPRT_BODY_DOT:
      if (dtype != OMPRT_F32) break;
      return launch_float_accs<BodyDotF32>(acc, sched, grid, block, smem, st, a, false);
    case OMPRT_BODY_NONE:
      if (dtype == OMPRT_F32)
        return launch_float_accs<BodyLoadF32>(acc, sched, grid, block, smem, st, a, false);
      if (dtype == OMPRT_BF16)
        return launch_float_accs<BodyLoadBF16>(acc, sched, grid, block, smem, st, a, false);
      break;
  }
  return cudaErrorNotSupported;
}

}  // namespace rt
