// Dispatch of fp32 / bf16 region launches to the per-body instance units.
#include "launch.h"

namespace rt {

cudaError_t launch_region_f32(int body, int dtype, int acc, int sched, unsigned grid,
                              unsigned block, size_t smem, cudaStream_t st, const RegionArgs& a) {
  switch (body) {
    case OMPRT_BODY_AXPY:
      if (dtype != OMPRT_F32) break;
      return launch_axpy(dtype, acc, sched, grid, block, smem, st, a);
    case OMPRT_BODY_STENCIL1D3:
    case OMPRT_BODY_STENCIL2D5:
      if (dtype != OMPRT_F32) break;
      return launch_stencil(body, acc, sched, grid, block, smem, st, a);
    case OMPRT_BODY_DOT:
      if (dtype != OMPRT_F32) break;
      return launch_dot_load(body, dtype, acc, sched, grid, block, smem, st, a);
    case OMPRT_BODY_NONE:
      if (dtype != OMPRT_F32 && dtype != OMPRT_BF16) break;
      return launch_dot_load(body, dtype, acc, sched, grid, block, smem, st, a);
  }
  return cudaErrorNotSupported;
}

}  // namespace rt
