// Executor instances for integer data: map-record, int32 axpy, value loads.
#include "launch_common.cuh"

namespace rt {

cudaError_t launch_region_int(int body, int dtype, int acc, int sched, unsigned grid,
                              unsigned block, size_t smem, cudaStream_t st, const RegionArgs& a) {
  switch (body) {
    case OMPRT_BODY_MAP_RECORD:
      if (acc != kAccNone) break;
      return launch_sched<BodyMapRecord, AccNone>(sched, grid, block, smem, st, a);
    case OMPRT_BODY_AXPY:
      if (dtype != OMPRT_I32) break;
      return launch_axpy(dtype, acc, sched, grid, block, smem, st, a);
    case OMPRT_BODY_NONE:
      if (dtype == OMPRT_I32)
        return launch_int_accs<BodyLoadI32>(acc, sched, grid, block, smem, st, a, false);
      if (dtype == OMPRT_I64)
        return launch_int_accs<BodyLoadI64>(acc, sched, grid, block, smem, st, a, false);
      break;
  }
  return cudaErrorNotSupported;
}

}  // namespace rt
