// CUDA driver entry points the runtime API does not expose, looked up once
// through cudaGetDriverEntryPointByVersion (no link against libcuda).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace ndhss {

// Unique id of the CUDA context current on this thread (cuCtxGetId: ids are
// never reused within a process, so a reset device gets a new one).
ndhss_status drv_current_ctx_id(unsigned long long* id);

// cuTensorMapEncodeTiled, for TMA tile copies (cp.async.bulk.tensor).
ndhss_status drv_encode_tiled(CUtensorMap* map, CUtensorMapDataType dtype, uint32_t rank, void* gaddr,
                              const cuuint64_t* dims, const cuuint64_t* strides_bytes, const cuuint32_t* box,
                              const cuuint32_t* estrides, CUtensorMapSwizzle swizzle, CUtensorMapL2promotion l2,
                              CUtensorMapFloatOOBfill oob);

}  // namespace ndhss
