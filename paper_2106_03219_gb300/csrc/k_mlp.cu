// MLP cost-model kernels (placeholder until the kernels land).
#include "api_internal.h"

extern "C" {
omprt_status omprt_mlp_forward(omprt_ctx*, const float*, const float*, int32_t, float*, void*) {
  return OMPRT_ERR_UNSUPPORTED;
}
omprt_status omprt_mlp_loss_grad(omprt_ctx*, const float*, const float*, const float*, int32_t,
                                 float*, float*, void*) {
  return OMPRT_ERR_UNSUPPORTED;
}
omprt_status omprt_mlp_adam(omprt_ctx*, float*, const float*, float*, float*, int32_t, int32_t,
                            float, float, float, float, void*) {
  return OMPRT_ERR_UNSUPPORTED;
}
}
