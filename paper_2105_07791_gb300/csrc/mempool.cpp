// Stream-ordered work space of the library: one memory pool per device whose
// release threshold is unbounded, so memory freed with cudaFreeAsync stays
// mapped for the next call instead of going back to the driver at every
// stream synchronisation (the default pool's threshold of 0 does that, and
// remapping ~100 MB of GMRES work space costs far more than the solve step
// it serves).  The pool is created on first use per device and lives until
// the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

namespace ndhss {

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[MAX_DEVICES] = {};
}  // namespace

cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            e = cudaMemPoolCreate(&np, &props);
            if (e != cudaSuccess) return e;
            uint64_t thr = UINT64_MAX;
            e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &thr);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(np);
                return e;
            }
            g_pool[dev] = np;
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

}  // namespace ndhss
