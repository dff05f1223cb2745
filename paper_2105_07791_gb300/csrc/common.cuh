// Scalar types and small device helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace ndhss {

// Stream-ordered allocation from the library's per-device pool (freed memory
// stays cached between calls); release with cudaFreeAsync.  mempool.cpp.
cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t st);

// Interleaved complex number (re = x, im = y), layout-compatible with
// std::complex / numpy complex64 and complex128.
template <typename R>
struct alignas(2 * sizeof(R)) Cx {
    R x, y;
};
using c64 = Cx<float>;
using c128 = Cx<double>;

template <typename T> struct Tr;
template <> struct Tr<double> { using real = double; static constexpr bool cplx = false; using val = double; };
template <> struct Tr<float> { using real = float; static constexpr bool cplx = false; using val = double; };
template <> struct Tr<c128> { using real = double; static constexpr bool cplx = true; using val = c128; };
template <> struct Tr<c64> { using real = float; static constexpr bool cplx = true; using val = c128; };

template <typename R> __host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return {-a.x, -a.y}; }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> __host__ __device__ __forceinline__ Cx<R>& operator+=(Cx<R>& a, Cx<R> b) { a.x += b.x; a.y += b.y; return a; }
template <typename R> __host__ __device__ __forceinline__ Cx<R>& operator-=(Cx<R>& a, Cx<R> b) { a.x -= b.x; a.y -= b.y; return a; }

template <typename T> __host__ __device__ __forceinline__ T zero() { return T{}; }
template <typename T> __host__ __device__ __forceinline__ T one();
template <> __host__ __device__ __forceinline__ double one<double>() { return 1.0; }
template <> __host__ __device__ __forceinline__ float one<float>() { return 1.0f; }
template <> __host__ __device__ __forceinline__ c128 one<c128>() { return {1.0, 0.0}; }
template <> __host__ __device__ __forceinline__ c64 one<c64>() { return {1.0f, 0.0f}; }

// c + a * b with fused multiply-adds
__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ c128 fmac(c128 a, c128 b, c128 c) {
    c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ c64 fmac(c64 a, c64 b, c64 c) {
    c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
    return c;
}

// |re| + |im| (the pivot magnitude of LAPACK's i?amax)
__host__ __device__ __forceinline__ double abs1(double a) { return fabs(a); }
__host__ __device__ __forceinline__ float abs1(float a) { return fabsf(a); }
__host__ __device__ __forceinline__ double abs1(c128 a) { return fabs(a.x) + fabs(a.y); }
__host__ __device__ __forceinline__ float abs1(c64 a) { return fabsf(a.x) + fabsf(a.y); }

__host__ __device__ __forceinline__ double conjv(double a) { return a; }
__host__ __device__ __forceinline__ float conjv(float a) { return a; }
__host__ __device__ __forceinline__ c128 conjv(c128 a) { return {a.x, -a.y}; }
__host__ __device__ __forceinline__ c64 conjv(c64 a) { return {a.x, -a.y}; }

// 1 / a; complex reciprocal by Smith's scaled formula (Smith, CACM 1962)
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }
template <typename R>
__device__ __forceinline__ Cx<R> recip(Cx<R> a) {
    if (fabs(a.x) >= fabs(a.y)) {
        R r = a.y / a.x, den = a.x + a.y * r;
        return {R(1) / den, -r / den};
    }
    R r = a.x / a.y, den = a.x * r + a.y;
    return {r / den, R(-1) / den};
}

__device__ __forceinline__ double scale(double a, double s) { return a * s; }
__device__ __forceinline__ float scale(float a, float s) { return a * s; }
template <typename R> __device__ __forceinline__ Cx<R> scale(Cx<R> a, R s) { return {a.x * s, a.y * s}; }

// |a|^2
__device__ __forceinline__ double norm2(double a) { return a * a; }
__device__ __forceinline__ double norm2(c128 a) { return a.x * a.x + a.y * a.y; }

// conversions between the float64 value type of A / GMRES and the factor type
template <typename T> __device__ __forceinline__ T from_val(double v);
template <> __device__ __forceinline__ double from_val<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_val<float>(double v) { return (float)v; }
template <typename T> __device__ __forceinline__ T from_val(c128 v);
template <> __device__ __forceinline__ c128 from_val<c128>(c128 v) { return v; }
template <> __device__ __forceinline__ c64 from_val<c64>(c128 v) { return {(float)v.x, (float)v.y}; }

__device__ __forceinline__ double to_val(double v) { return v; }
__device__ __forceinline__ double to_val(float v) { return (double)v; }
__device__ __forceinline__ c128 to_val(c128 v) { return v; }
__device__ __forceinline__ c128 to_val(c64 v) { return {(double)v.x, (double)v.y}; }

// Warp-wide maximum of a pivot candidate's key.  The bits of a non-negative
// float (double) order like its value; key 0 marks "no candidate" (a NaN, or
// a lane without one), so a NaN never wins, as with a strict comparison
// against a negative start value.  FP32 keys take one redux.sync; FP64 keys
// shuffles.
template <typename R> struct PivKey;
template <> struct PivKey<float> {
    using K = unsigned;
    static __device__ __forceinline__ K of(float v) { return v >= 0.0f ? __float_as_uint(v) + 1u : 0u; }
    static __device__ __forceinline__ K wmax(K k) { return __reduce_max_sync(0xffffffffu, k); }
    static __device__ __forceinline__ float val(K k) { return __uint_as_float(k - 1u); }
};
template <> struct PivKey<double> {
    using K = unsigned long long;
    static __device__ __forceinline__ K of(double v) {
        return v >= 0.0 ? (unsigned long long)__double_as_longlong(v) + 1ull : 0ull;
    }
    static __device__ __forceinline__ K wmax(K k) {
        for (int o = 16; o; o >>= 1) {
            const K x = __shfl_xor_sync(0xffffffffu, k, o);
            k = x > k ? x : k;
        }
        return k;
    }
    static __device__ __forceinline__ double val(K k) { return __longlong_as_double((long long)(k - 1ull)); }
};

// The warp's argmax over (value, index) pairs: the largest value, then the
// lowest index among equal values (the i?amax convention); invalid or NaN
// entries never win.  Returns the index (INT_MAX when no lane has a
// candidate) and its value in *best (-1 when none).
template <typename R>
__device__ __forceinline__ int warp_argmax(R val, int idx, bool valid, R* best) {
    using PK = PivKey<R>;
    using K = typename PK::K;
    const K key = valid ? PK::of(val) : K(0);
    const K kmax = PK::wmax(key);
    const unsigned imin = __reduce_min_sync(0xffffffffu, (kmax != K(0) && key == kmax) ? (unsigned)idx : 0xffffffffu);
    *best = kmax != K(0) ? PK::val(kmax) : R(-1);
    return kmax != K(0) ? (int)imin : 0x7fffffff;
}

// Device status word written by kernels that detect a numerical failure.
struct DevStatus {
    int32_t code;
    int32_t node;
};

#define NDHSS_CUDA_TRY(call)                                                                   \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return ::ndhss::set_error(NDHSS_ERR_CUDA, "%s failed: %s (%s:%d)", #call,          \
                                      cudaGetErrorString(e_), __FILE__, __LINE__);             \
    } while (0)


#define NDHSS_LAUNCH_CHECK(what)                                                               \
    do {                                                                                       \
        ::ndhss::note_launches(1);                                                             \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess)                                                                 \
            return ::ndhss::set_error(NDHSS_ERR_CUDA, "launch of %s failed: %s", what,         \
                                      cudaGetErrorString(e_));                                 \
    } while (0)

inline bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace ndhss
