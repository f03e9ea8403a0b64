// Batched persistent executor (placeholder until the kernel lands).
#include "api_internal.h"

extern "C" {
omprt_status omprt_batch_create(omprt_ctx*, const omprt_loop_desc*, const omprt_reduce_desc*,
                                int32_t, int64_t, omprt_batch**) {
  return OMPRT_ERR_UNSUPPORTED;
}
omprt_status omprt_launch_batch(omprt_batch*, int32_t, int32_t, void*) {
  return OMPRT_ERR_UNSUPPORTED;
}
omprt_status omprt_batch_destroy(omprt_batch*) { return OMPRT_ERR_UNSUPPORTED; }
int64_t omprt_batch_items(const omprt_batch*) { return 0; }
}
