// Measurement aid with no counterpart in the paper: the sustained FMA
// throughput of the device's CUDA cores, the denominator of the rooflines of
// the kernels bound by plain arithmetic (the FP64 sparse product and
// Gram-Schmidt steps, the FP32 exchange steps on the CUDA cores).  Every
// thread runs eight independent FMA chains on register values; with eight
// 256-thread CTAs per SM the issue rate, not the chain latency, bounds the
// kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace ndhss {
namespace {

constexpr int PK_THREADS = 256, PK_CTAS_PER_SM = 8, PK_CHAINS = 8;

template <typename R>
__global__ void __launch_bounds__(PK_THREADS) fma_peak_kernel(const R* __restrict__ in, R* __restrict__ out, int iters) {
    R a[PK_CHAINS];
    const R b = in[0], c = in[1];
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) a[u] = in[2 + u] + (R)threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PK_CHAINS; ++u) a[u] = fma(a[u], b, c);
    }
    R s = 0;
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) s += a[u];
    // the inputs keep every chain bounded away from this value; the store
    // only keeps the chains alive
    if (s == (R)-1.0) out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
ndhss_status measure(int iters, cudaStream_t st, double* tflops) {
    int dev = 0, sms = 0;
    NDHSS_CUDA_TRY(cudaGetDevice(&dev));
    NDHSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)(sms * PK_CTAS_PER_SM);
    R h[2 + PK_CHAINS] = {(R)0.999, (R)1e-3};
    for (int u = 0; u < PK_CHAINS; ++u) h[2 + u] = (R)(0.1 * (u + 1));
    R *d_in = nullptr, *d_out = nullptr;
    NDHSS_CUDA_TRY(pool_malloc_async((void**)&d_in, sizeof(h), st));
    NDHSS_CUDA_TRY(pool_malloc_async((void**)&d_out, sizeof(R) * grid * PK_THREADS, st));
    NDHSS_CUDA_TRY(cudaMemcpyAsync(d_in, h, sizeof(h), cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    NDHSS_CUDA_TRY(cudaEventCreate(&e0));
    NDHSS_CUDA_TRY(cudaEventCreate(&e1));
    float best = 0.0f;
    ndhss_status rc = NDHSS_OK;
    for (int rep = 0; rep < 4 && rc == NDHSS_OK; ++rep) {
        cudaEventRecord(e0, st);
        fma_peak_kernel<R><<<grid, PK_THREADS, 0, st>>>(d_in, d_out, iters);
        note_launches(1);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_measure_fma_peak: kernel failed");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;      // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(d_in, st);
    cudaFreeAsync(d_out, st);
    if (rc != NDHSS_OK) return rc;
    const double fmas = (double)grid * PK_THREADS * PK_CHAINS * (double)iters;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return NDHSS_OK;
}

}  // namespace
}  // namespace ndhss

extern "C" ndhss_status ndhss_measure_fma_peak(int32_t which, void* stream, double* tflops) {
    return ::ndhss::guarded("ndhss_measure_fma_peak", [&]() -> ndhss_status {
        using namespace ndhss;
        clear_error();
        if (!tflops || (which != 0 && which != 1))
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_measure_fma_peak: which must be 0 (FP64) or 1 (FP32)");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        return which == 0 ? measure<double>(2048, st, tflops) : measure<float>(32768, st, tflops);
    });
}
