// Driver entry points through the runtime's entry-point query (driver.h).
#include "driver.h"

#include <cudaTypedefs.h>

#include <mutex>

namespace ndhss {
namespace {

struct DriverFns {
    PFN_cuCtxGetCurrent_v4000 ctx_current = nullptr;
    PFN_cuCtxGetId_v12000 ctx_id = nullptr;
    PFN_cuTensorMapEncodeTiled_v12000 encode_tiled = nullptr;
    bool ok = false;
};

std::once_flag g_once;
DriverFns g_fns;

template <typename F>
bool lookup(const char* name, unsigned version, F* out) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        cudaGetLastError();
        return false;
    }
    *out = reinterpret_cast<F>(p);
    return true;
}

const DriverFns* fns() {
    std::call_once(g_once, [] {
        DriverFns f;
        f.ok = lookup("cuCtxGetCurrent", 4000, &f.ctx_current) && lookup("cuCtxGetId", 12000, &f.ctx_id) &&
               lookup("cuTensorMapEncodeTiled", 12000, &f.encode_tiled);
        g_fns = f;
    });
    return g_fns.ok ? &g_fns : nullptr;
}

}  // namespace

ndhss_status drv_current_ctx_id(unsigned long long* id) {
    const DriverFns* f = fns();
    if (!f) return set_error(NDHSS_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not found");
    CUcontext ctx = nullptr;
    if (f->ctx_current(&ctx) != CUDA_SUCCESS || !ctx)
        return set_error(NDHSS_ERR_CUDA, "no current CUDA context");
    if (f->ctx_id(ctx, id) != CUDA_SUCCESS) return set_error(NDHSS_ERR_CUDA, "cuCtxGetId failed");
    return NDHSS_OK;
}

ndhss_status drv_encode_tiled(CUtensorMap* map, CUtensorMapDataType dtype, uint32_t rank, void* gaddr,
                              const cuuint64_t* dims, const cuuint64_t* strides_bytes, const cuuint32_t* box,
                              const cuuint32_t* estrides, CUtensorMapSwizzle swizzle, CUtensorMapL2promotion l2,
                              CUtensorMapFloatOOBfill oob) {
    const DriverFns* f = fns();
    if (!f) return set_error(NDHSS_ERR_CUDA, "driver entry point cuTensorMapEncodeTiled not found");
    const CUresult r = f->encode_tiled(map, dtype, rank, gaddr, dims, strides_bytes, box, estrides,
                                       CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, l2, oob);
    if (r != CUDA_SUCCESS) return set_error(NDHSS_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return NDHSS_OK;
}

}  // namespace ndhss
