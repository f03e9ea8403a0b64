// Tensor maps for the TMA engine's tiled copies.
#pragma once
#include <cuda.h>  // CUtensorMap and its enums (types only; no driver library is linked)

#include "api_internal.h"

namespace rt {

// cuTensorMapEncodeTiled, looked up once through the runtime's driver entry
// point query (the driver library is not linked); null where the driver has
// none.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled();

}  // namespace rt
