// Executor instances: 1-D and 2-D stencils.
#include "launch_common.cuh"

namespace rt {

cudaError_t launch_stencil(int body, int acc, int sched, unsigned grid, unsigned block,
                           size_t smem, cudaStream_t st, const RegionArgs& a) {
  if (body == OMPRT_BODY_STENCIL1D3)
    return launch_float_accs<BodyStencil1D>(acc, sched, grid, block, smem, st, a, true);
  return launch_float_accs<BodyStencil2D>(acc, sched, grid, block, smem, st, a, true);
}

}  // namespace rt
