// Sparse product and restarted, left-preconditioned GMRES (Eq. 1.2, Sec. 4)
// in float64 / complex128 on the device.
//
// A cycle ends when the least-squares residual drops to inner * tol * ||P^{-1} b||
// (inner = 0.1 by default: Sec. 4 stops one decade below the accuracy it
// reports), when it has fallen by cycle_rtol relative to the cycle's start
// (with a reduced-precision preconditioner the Krylov estimate cannot be
// trusted beyond what one apply resolves, so the float64 restart does the
// refinement), after `restart` steps, on breakdown or at maxit.  Once a cycle
// fails to halve the true residual, the next cycles end only when their
// estimate fell by the reduction the true residual still needs, relative to
// their own start.
//
// Per Arnoldi step j:  t = A v_j (CSR SpMV);  w = P^{-1} t (Algorithm 3.1);
// classical Gram-Schmidt twice: h = V^H w, w -= V h (x2); ||w||; a one-thread
// kernel stores the Hessenberg column, applies the previous complex Givens
// rotations G = [[c, s], [-conj(s), c]], forms the new one and updates the
// least-squares residual |g_{j+1}|; v_{j+1} = w / h_{j+1,j}.  The host reads
// that residual once per step to decide whether the cycle ends.  After each
// cycle x += V y with H y = g solved on the device, and the float64 true
// residual ||b - A x|| / ||b|| decides convergence (restarts refine).
//
// Reductions are deterministic: each block writes its partial sums and the
// last block to finish (ticket counter) adds them in block order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "factor.cuh"

namespace ndhss {
namespace {

constexpr int KMAX = 32;          // restart + 1 <= KMAX
constexpr int RT = 256;           // reduction block size
constexpr int RB = 2 * 152;       // reduction grid (two blocks per SM)

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ c128 ldcg(const c128* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ c128 warp_sum(c128 v) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double absv(double a) { return fabs(a); }
__device__ __forceinline__ double absv(c128 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ c128 cdiv(c128 a, c128 b) { return a * recip(b); }
__device__ __forceinline__ double cdiv(double a, double b) { return a / b; }

// ----------------------------------------------------------------- SpMV
// acc + a * b.  GB300's FP64 pipe is narrow, and most entries of the FEM
// matrices are real (the impedance term is on the boundary only): the FMAs
// with a zero imaginary part are skipped.  The test reads the bit pattern
// (a float64 compare would itself take an FP64-pipe slot; -0.0 just takes
// the full product).  The rounding of the remaining operations is that of
// the full product.
__device__ __forceinline__ double spmv_mac(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ c128 spmv_mac(c128 a, c128 b, c128 c) {
    c.x = fma(a.x, b.x, c.x);
    c.y = fma(a.x, b.y, c.y);
    if (__double_as_longlong(a.y) != 0) {
        c.x = fma(-a.y, b.y, c.x);
        c.y = fma(a.y, b.x, c.y);
    }
    return c;
}

// TPR threads per row; each issues all U of its column indices and values
// at once, then the U gathers of x, so a row costs three dependent memory
// round trips (row pointers, entries, x) instead of two per entry.
template <typename V, int TPR, int U>
__global__ void __launch_bounds__(256) spmv_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                   const V* __restrict__ vals, const V* __restrict__ x, V* __restrict__ y) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int lane = (int)(gt % TPR);
    if (row >= n) return;               // whole TPR groups leave together
    const int k0 = rowptr[row], k1 = rowptr[row + 1];
    V acc = zero<V>();
    for (int base = k0; base < k1; base += U * TPR) {
        int c[U];
        V a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = base + lane + u * TPR;
            c[u] = k < k1 ? col[k] : -1;
            a[u] = k < k1 ? vals[k] : zero<V>();
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c[u] >= 0) acc = spmv_mac(a[u], x[c[u]], acc);
    }
    if constexpr (sizeof(V) == 8) {
        for (int o = TPR / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
    } else {
        for (int o = TPR / 2; o; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o, TPR);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o, TPR);
        }
    }
    if (lane == 0) y[row] = acc;
}

template <typename V>
ndhss_status spmv_launch(int n, const int32_t* rowptr, const int32_t* col, const V* vals, const V* x, V* y,
                         cudaStream_t st) {
    const int64_t threads = (int64_t)n * 4;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    spmv_kernel<V, 4, 4><<<blocks, 256, 0, st>>>(n, rowptr, col, vals, x, y);
    NDHSS_LAUNCH_CHECK("spmv_kernel");
    return NDHSS_OK;
}

// ---------------------------------------------------------- reductions
// out[i] = sum_rows conj(Vb(row, i)) * w(row), i < k.  Grid (RB, k): block
// (b, i) sums its grid-stride rows of column i into partial[i * RB + b]; the
// last block to finish adds each column's partials with one warp in a fixed
// order.
template <typename V>
__global__ void __launch_bounds__(RT)
mdot_kernel(int n, const V* __restrict__ Vb, int64_t ldv, int k, const V* __restrict__ w, V* __restrict__ partial,
            V* __restrict__ out, unsigned* __restrict__ counter) {
    __shared__ V sred[RT / 32];
    __shared__ bool s_last;
    const int i = blockIdx.y;
    const V* v = Vb + (int64_t)i * ldv;
    V acc0 = zero<V>(), acc1 = zero<V>();
    const int64_t stride = (int64_t)gridDim.x * RT;
    int64_t row = (int64_t)blockIdx.x * RT + threadIdx.x;
    for (; row + stride < n; row += 2 * stride) {
        acc0 = fmac(conjv(v[row]), w[row], acc0);
        acc1 = fmac(conjv(v[row + stride]), w[row + stride], acc1);
    }
    if (row < n) acc0 = fmac(conjv(v[row]), w[row], acc0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const V ws = warp_sum(acc0 + acc1);
    if (lane == 0) sred[warp] = ws;
    __syncthreads();
    if (threadIdx.x == 0) {
        V sum = zero<V>();
        for (int q = 0; q < RT / 32; ++q) sum += sred[q];
        partial[(int64_t)i * gridDim.x + blockIdx.x] = sum;
    }
    __threadfence();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1);
    __syncthreads();
    if (s_last) {
        for (int c = warp; c < k; c += RT / 32) {
            V sum = zero<V>();
            for (unsigned b = lane; b < gridDim.x; b += 32) sum += ldcg(partial + (int64_t)c * gridDim.x + b);
            sum = warp_sum(sum);
            if (lane == 0) out[c] = sum;
        }
        if (threadIdx.x == 0) *counter = 0;
    }
}

// out = sum |w|^2
template <typename V>
__global__ void __launch_bounds__(RT)
nrm2_kernel(int n, const V* __restrict__ w, double* __restrict__ partial, double* __restrict__ out,
            unsigned* __restrict__ counter) {
    __shared__ double sred[RT / 32];
    __shared__ bool s_last;
    double acc = 0.0;
    for (int64_t row = (int64_t)blockIdx.x * RT + threadIdx.x; row < n; row += (int64_t)gridDim.x * RT) acc += norm2(w[row]);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < RT / 32; ++q) s += sred[q];
        partial[blockIdx.x] = s;
    }
    __threadfence();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
        double s = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) s += __ldcg(partial + b);
        s = warp_sum(s);
        if (threadIdx.x == 0) {
            *out = s;
            *counter = 0;
        }
    }
}

// w += sgn * Vb(:, 0:k) h
template <typename V>
__global__ void maxpy_kernel(int n, V* __restrict__ w, const V* __restrict__ Vb, int64_t ldv, int k,
                             const V* __restrict__ h, double sgn) {
    __shared__ V sh[KMAX];
    if (threadIdx.x < k) sh[threadIdx.x] = scale(h[threadIdx.x], sgn);
    __syncthreads();
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
        V acc = w[row];
        for (int i = 0; i < k; ++i) acc = fmac(Vb[row + i * ldv], sh[i], acc);
        w[row] = acc;
    }
}

template <typename V>
__global__ void scale_kernel(int n, const V* __restrict__ src, V* __restrict__ dst, const double* __restrict__ s) {
    const double f = *s;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = scale(src[i], f);
}

template <typename V>
__global__ void residual_kernel(int n, const V* __restrict__ b, const V* __restrict__ ax, V* __restrict__ r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - ax[i];
}

// v <- conj(v): the adjoint solve of a complex symmetric A, A^H x = b, is
// A conj(x) = conj(b).
__global__ void __launch_bounds__(256) conj_kernel(int64_t n, c128* __restrict__ v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i].y = -v[i].y;
}

static ndhss_status conj_inplace(c128* v, int64_t n, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    if (blocks < 1) return NDHSS_OK;
    conj_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, v);
    NDHSS_LAUNCH_CHECK("conj_kernel");
    return NDHSS_OK;
}

// scalars: [0] scale for the next basis vector, [1] |g_{j+1}|, [2] h_{j+1,j}, [3] beta
struct GmState {
    double scal[4];
};

// start of a cycle: beta = ||z||, g = beta e_1
template <typename V>
__global__ void cycle_init_kernel(const double* __restrict__ nrm2z, V* __restrict__ g, int restart, GmState* stt) {
    const double beta = sqrt(*nrm2z);
    for (int i = 0; i <= restart; ++i) g[i] = zero<V>();
    V b0 = zero<V>();
    if constexpr (sizeof(V) == 8) b0 = beta; else b0.x = beta;
    g[0] = b0;
    stt->scal[0] = beta > 0 ? 1.0 / beta : 0.0;
    stt->scal[3] = beta;
    stt->scal[1] = beta;
}

// Hessenberg column j, Givens rotations, residual estimate
template <typename V>
__global__ void arnoldi_step_kernel(int j, V* __restrict__ H, int ldh, const V* __restrict__ h1, const V* __restrict__ h2,
                                    const double* __restrict__ nrm2w, V* __restrict__ g, double* __restrict__ cs,
                                    V* __restrict__ sn, GmState* stt) {
    V* Hj = H + (int64_t)j * ldh;
    for (int i = 0; i <= j; ++i) Hj[i] = h1[i] + h2[i];
    const double hn = sqrt(*nrm2w);
    V hv = zero<V>();
    if constexpr (sizeof(V) == 8) hv = hn; else hv.x = hn;
    Hj[j + 1] = hv;
    for (int i = 0; i < j; ++i) {
        const V t0 = scale(Hj[i], cs[i]) + sn[i] * Hj[i + 1];
        const V t1 = scale(Hj[i + 1], cs[i]) - conjv(sn[i]) * Hj[i];
        Hj[i] = t0;
        Hj[i + 1] = t1;
    }
    const V a = Hj[j], b = Hj[j + 1];
    double c;
    V s;
    const double aa = absv(a), ab = absv(b);
    if (ab == 0.0) {
        c = 1.0;
        s = zero<V>();
    } else if (aa == 0.0) {
        c = 0.0;
        s = scale(conjv(b), 1.0 / ab);
    } else {
        const double t = hypot(aa, ab);
        c = aa / t;
        s = scale(a, 1.0 / aa) * scale(conjv(b), 1.0 / t);
    }
    cs[j] = c;
    sn[j] = s;
    Hj[j] = scale(a, c) + s * b;
    Hj[j + 1] = zero<V>();
    const V gj = g[j];
    g[j + 1] = -(conjv(s) * gj);
    g[j] = scale(gj, c);
    stt->scal[0] = hn > 0 ? 1.0 / hn : 0.0;
    stt->scal[1] = absv(g[j + 1]);
    stt->scal[2] = hn;
}

// y = H(0:k, 0:k)^{-1} g(0:k) (upper triangular)
template <typename V>
__global__ void hsolve_kernel(int k, const V* __restrict__ H, int ldh, const V* __restrict__ g, V* __restrict__ y) {
    for (int i = k - 1; i >= 0; --i) {
        V acc = g[i];
        for (int l = i + 1; l < k; ++l) acc = acc - H[(int64_t)l * ldh + i] * y[l];
        y[i] = cdiv(acc, H[(int64_t)i * ldh + i]);
    }
}

template <typename V>
ndhss_status gmres_one(const FactorData& F, const int32_t* rowptr, const int32_t* col, const V* vals,
                       const V* b, V* x, const ndhss_gmres_opts& o, ndhss_gmres_stats* stats, unsigned char* ws,
                       cudaStream_t st) {
    const int n = F.n;
    const int R = o.restart;
    const int64_t ldv = ((int64_t)n + 31) / 32 * 32;
    auto carve = [&](size_t bytes) {
        unsigned char* p = ws;
        ws += (bytes + 255) / 256 * 256;
        return p;
    };
    V* Vb = (V*)carve(sizeof(V) * ldv * (R + 1));
    V* w = (V*)carve(sizeof(V) * n);
    V* t = (V*)carve(sizeof(V) * n);
    V* r = (V*)carve(sizeof(V) * n);
    V* H = (V*)carve(sizeof(V) * (R + 1) * R);
    V* g = (V*)carve(sizeof(V) * (R + 1));
    double* cs = (double*)carve(sizeof(double) * R);
    V* sn = (V*)carve(sizeof(V) * R);
    V* h1 = (V*)carve(sizeof(V) * KMAX);
    V* h2 = (V*)carve(sizeof(V) * KMAX);
    V* yv = (V*)carve(sizeof(V) * KMAX);
    V* part = (V*)carve(sizeof(V) * RB * KMAX);
    double* dpart = (double*)carve(sizeof(double) * RB);
    double* nrm = (double*)carve(sizeof(double) * 4);
    unsigned* counter = (unsigned*)carve(sizeof(unsigned) * 4);
    GmState* stt = (GmState*)carve(sizeof(GmState));
    void* awork = carve(apply_work_bytes(F));
    NDHSS_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned) * 4, st));
    NDHSS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(V) * n, st));
    const int eb = std::min((n + 255) / 256, 4 * 152);
    ndhss_status rc;
    double hb[4];

    auto read_scalars = [&](const void* src, size_t bytes, void* dst) -> ndhss_status {
        NDHSS_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
        NDHSS_CUDA_TRY(cudaStreamSynchronize(st));
        return NDHSS_OK;
    };

    ndhss_gmres_stats S{};
    // optional CUDA-event timing of every apply and sparse product
    // events come from a per-thread pool that lives as long as the thread, so
    // timing adds two records per product and no event creation
    thread_local std::vector<cudaEvent_t> pool;
    size_t pool_next = 0;
    std::vector<cudaEvent_t> ev_apply, ev_spmv;
    auto event_pair = [&](std::vector<cudaEvent_t>& v) -> ndhss_status {
        for (int q = 0; q < 2; ++q) {
            if (pool_next == pool.size()) {
                cudaEvent_t e;
                NDHSS_CUDA_TRY(cudaEventCreate(&e));
                pool.push_back(e);
            }
            v.push_back(pool[pool_next++]);
        }
        return NDHSS_OK;
    };
    auto timed_apply = [&](const V* in, V* outv) -> ndhss_status {
        ndhss_status r2;
        if (o.timing) {
            if ((r2 = event_pair(ev_apply))) return r2;
            cudaEventRecord(ev_apply[ev_apply.size() - 2], st);
        }
        if ((r2 = apply_device(F, 1, in, n, outv, n, awork, st))) return r2;
        if (o.timing) cudaEventRecord(ev_apply.back(), st);
        S.napply++;
        return NDHSS_OK;
    };
    auto timed_spmv = [&](const V* in, V* outv) -> ndhss_status {
        ndhss_status r2;
        if (o.timing) {
            if ((r2 = event_pair(ev_spmv))) return r2;
            cudaEventRecord(ev_spmv[ev_spmv.size() - 2], st);
        }
        if ((r2 = spmv_launch<V>(n, rowptr, col, vals, in, outv, st))) return r2;
        if (o.timing) cudaEventRecord(ev_spmv.back(), st);
        S.nspmv++;
        return NDHSS_OK;
    };
    auto collect = [&]() {
        if (!o.timing) return;
        cudaStreamSynchronize(st);
        float ms;
        for (size_t i = 0; i + 1 < ev_apply.size(); i += 2)
            if (cudaEventElapsedTime(&ms, ev_apply[i], ev_apply[i + 1]) == cudaSuccess) S.apply_ms += ms;
        for (size_t i = 0; i + 1 < ev_spmv.size(); i += 2)
            if (cudaEventElapsedTime(&ms, ev_spmv[i], ev_spmv[i + 1]) == cudaSuccess) S.spmv_ms += ms;
        ev_apply.clear();
        ev_spmv.clear();
        pool_next = 0;
    };
    nrm2_kernel<V><<<RB, RT, 0, st>>>(n, b, dpart, nrm, counter);
    NDHSS_LAUNCH_CHECK("nrm2_kernel");
    if ((rc = read_scalars(nrm, sizeof(double), hb))) return rc;
    const double bnorm = sqrt(hb[0]);
    if (bnorm == 0.0) {
        S.converged = 1;
        if (stats) *stats = S;
        return NDHSS_OK;
    }
    double zbnorm = -1.0;
    int its = 0, cycles = 0;
    double last_res = 1.0;
    // After a cycle that did not halve the true residual (a preconditioner
    // whose ||P^{-1} r|| / ||P^{-1} b|| no longer tracks ||r|| / ||b||), a cycle
    // no longer ends on cycle_rtol or on the inner test against ||P^{-1} b||,
    // but once its residual estimate fell by the factor the true residual
    // still needs (0.1 tol / relres), relative to the cycle's start.
    double rtol_eff = o.cycle_rtol, prev_rel = INFINITY, cyc_target = 0.0;
    while (true) {
        if ((rc = timed_spmv(x, t))) return rc;
        residual_kernel<V><<<eb, 256, 0, st>>>(n, b, t, r);
        NDHSS_LAUNCH_CHECK("residual_kernel");
        nrm2_kernel<V><<<RB, RT, 0, st>>>(n, r, dpart, nrm, counter);
        NDHSS_LAUNCH_CHECK("nrm2_kernel");
        if ((rc = read_scalars(nrm, sizeof(double), hb))) return rc;
        const double rel = sqrt(hb[0]) / bnorm;
        S.true_relres = rel;
        if (rel <= o.tol) { S.converged = 1; break; }
        if (its >= o.maxit) break;
        if (rel > 0.5 * prev_rel) {
            rtol_eff = 0.0;
            cyc_target = 0.1 * o.tol / rel;
        } else if (cyc_target > 0.0) {
            cyc_target = 0.1 * o.tol / rel;
        }
        prev_rel = rel;
        ++cycles;
        if ((rc = timed_apply(r, w))) return rc;
        nrm2_kernel<V><<<RB, RT, 0, st>>>(n, w, dpart, nrm, counter);
        NDHSS_LAUNCH_CHECK("nrm2_kernel");
        cycle_init_kernel<V><<<1, 1, 0, st>>>(nrm, g, R, stt);
        NDHSS_LAUNCH_CHECK("cycle_init_kernel");
        scale_kernel<V><<<eb, 256, 0, st>>>(n, w, Vb, &stt->scal[0]);
        NDHSS_LAUNCH_CHECK("scale_kernel");
        if (zbnorm < 0) {
            if ((rc = read_scalars(stt, sizeof(GmState), hb))) return rc;
            zbnorm = hb[3];
            if (zbnorm == 0.0) return set_error(NDHSS_ERR_INTERNAL, "ndhss_gmres: P^{-1} b vanished");
        }
        int jend = 0;
        for (int j = 0; j < R; ++j) {
            V* vj = Vb + (int64_t)j * ldv;
            if ((rc = timed_spmv(vj, t))) return rc;
            if ((rc = timed_apply(t, w))) return rc;
            ++its;
            mdot_kernel<V><<<dim3(RB, j + 1), RT, 0, st>>>(n, Vb, ldv, j + 1, w, part, h1, counter);
            NDHSS_LAUNCH_CHECK("mdot_kernel");
            maxpy_kernel<V><<<eb, 256, 0, st>>>(n, w, Vb, ldv, j + 1, h1, -1.0);
            NDHSS_LAUNCH_CHECK("maxpy_kernel");
            mdot_kernel<V><<<dim3(RB, j + 1), RT, 0, st>>>(n, Vb, ldv, j + 1, w, part, h2, counter);
            NDHSS_LAUNCH_CHECK("mdot_kernel");
            maxpy_kernel<V><<<eb, 256, 0, st>>>(n, w, Vb, ldv, j + 1, h2, -1.0);
            NDHSS_LAUNCH_CHECK("maxpy_kernel");
            nrm2_kernel<V><<<RB, RT, 0, st>>>(n, w, dpart, nrm, counter);
            NDHSS_LAUNCH_CHECK("nrm2_kernel");
            arnoldi_step_kernel<V><<<1, 1, 0, st>>>(j, H, R + 1, h1, h2, nrm, g, cs, sn, stt);
            NDHSS_LAUNCH_CHECK("arnoldi_step_kernel");
            scale_kernel<V><<<eb, 256, 0, st>>>(n, w, Vb + (int64_t)(j + 1) * ldv, &stt->scal[0]);
            NDHSS_LAUNCH_CHECK("scale_kernel");
            if ((rc = read_scalars(stt, sizeof(GmState), hb))) return rc;
            jend = j + 1;
            last_res = hb[1] / zbnorm;
            const bool inner_done = cyc_target > 0.0 ? hb[1] <= cyc_target * hb[3] : last_res <= o.inner * o.tol;
            if (inner_done || hb[1] <= rtol_eff * hb[3] || hb[2] == 0.0 || its >= o.maxit) break;
        }
        hsolve_kernel<V><<<1, 1, 0, st>>>(jend, H, R + 1, g, yv);
        NDHSS_LAUNCH_CHECK("hsolve_kernel");
        maxpy_kernel<V><<<eb, 256, 0, st>>>(n, x, Vb, ldv, jend, yv, 1.0);
        NDHSS_LAUNCH_CHECK("maxpy_kernel");
    }
    collect();
    S.iters = its;
    S.cycles = cycles;
    S.precond_relres = last_res;
    if (stats) *stats = S;
    return NDHSS_OK;
}

size_t gmres_work_bytes(const FactorData& F, int R, size_t vsz) {
    const int64_t ldv = ((int64_t)F.n + 31) / 32 * 32;
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
    add(vsz * ldv * (R + 1));
    add(vsz * F.n); add(vsz * F.n); add(vsz * F.n);
    add(vsz * (R + 1) * R); add(vsz * (R + 1)); add(8 * R); add(vsz * R);
    add(vsz * KMAX); add(vsz * KMAX); add(vsz * KMAX);
    add(vsz * RB * KMAX); add(8 * RB); add(32); add(16); add(sizeof(GmState));
    add(apply_work_bytes(F));
    return b;
}

}  // namespace
}  // namespace ndhss

extern "C" {

ndhss_status ndhss_spmv(int32_t n, int32_t vtype, const int32_t* d_rowptr, const int32_t* d_col, const void* d_vals,
                        const void* d_x, void* d_y, void* stream) {
    return ::ndhss::guarded("ndhss_spmv", [&]() -> ndhss_status {
        using namespace ndhss;
        clear_error();
        if (n < 0 || !d_rowptr || !d_col || !d_vals || !d_x || !d_y) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_spmv: bad argument");
        if (n == 0) return NDHSS_OK;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (vtype == NDHSS_R64)
            return spmv_launch<double>(n, d_rowptr, d_col, (const double*)d_vals, (const double*)d_x, (double*)d_y, st);
        if (vtype == NDHSS_C128)
            return spmv_launch<c128>(n, d_rowptr, d_col, (const c128*)d_vals, (const c128*)d_x, (c128*)d_y, st);
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_spmv: bad vtype %d", vtype);
    });
}

ndhss_status ndhss_gmres(const ndhss_factorization* fh, const int32_t* d_rowptr, const int32_t* d_col, const void* d_vals,
                         int32_t nrhs, const void* b, int64_t ldb, void* x, int64_t ldx, const ndhss_gmres_opts* opts,
                         ndhss_gmres_stats* stats, void* stream) {
    return ::ndhss::guarded("ndhss_gmres", [&]() -> ndhss_status {
        using namespace ndhss;
        clear_error();
        if (!fh || !d_rowptr || !d_col || !d_vals || !b || !x || nrhs < 0)
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres: bad argument");
        const FactorData& F = fh->f;
        if (ldb < F.n || ldx < F.n) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres: leading dimension < n");
        ndhss_gmres_opts o{30, 300, 1e-8, 0, 0, 0.1, -1.0};
        if (opts) o = *opts;
        if (o.restart < 1 || o.restart > KMAX - 1 || o.maxit < 0 || !(o.tol >= 0) || !(o.inner > 0 && o.inner <= 1) ||
            o.conj_transpose < 0 || o.conj_transpose > 1)
            return set_error(NDHSS_ERR_INVALID_ARG,
                             "ndhss_gmres: need 1 <= restart <= %d, maxit >= 0, tol >= 0, 0 < inner <= 1, conj_transpose 0 or 1",
                             KMAX - 1);
        if (nrhs == 0) return NDHSS_OK;
        if (o.cycle_rtol < 0) o.cycle_rtol = (F.prec == NDHSS_FP64) ? 0.0 : 1e-3;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const size_t vsz = F.vtype == NDHSS_C128 ? 16 : 8;
        const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
        // A^H = A for real symmetric A: the flag changes nothing there
        const bool conj = o.conj_transpose != 0 && F.vtype == NDHSS_C128;
        const bool stage_b = !bdev || conj;          // conj(b) is formed in scratch, never in the caller's b
        const size_t vec = ((size_t)F.n * vsz + 255) / 256 * 256;
        const size_t wb = gmres_work_bytes(F, o.restart, vsz) + (stage_b ? vec : 0) + (xdev ? 0 : vec);
        void* work = nullptr;
        NDHSS_CUDA_TRY(pool_malloc_async(&work, wb, st));
        unsigned char* ws = static_cast<unsigned char*>(work);
        unsigned char* extra = ws + gmres_work_bytes(F, o.restart, vsz);
        void* db = stage_b ? extra : nullptr;
        void* dx = xdev ? nullptr : extra + (stage_b ? vec : 0);
        ndhss_status rc = NDHSS_OK;
        bool any_fail = false;
        for (int rhs = 0; rhs < nrhs && rc == NDHSS_OK; ++rhs) {
            const unsigned char* bsrc = (const unsigned char*)b + (size_t)rhs * ldb * vsz;
            unsigned char* xdst = (unsigned char*)x + (size_t)rhs * ldx * vsz;
            const void* bb = bsrc;
            void* xx = xdst;
            if (stage_b) {
                const cudaMemcpyKind kind = bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
                if (cudaMemcpyAsync(db, bsrc, (size_t)F.n * vsz, kind, st) != cudaSuccess) {
                    rc = set_error(NDHSS_ERR_CUDA, "ndhss_gmres: copy of b failed");
                    break;
                }
                bb = db;
                if (conj && (rc = conj_inplace(static_cast<c128*>(db), F.n, st)) != NDHSS_OK) break;
            }
            if (!xdev) xx = dx;
            ndhss_gmres_stats S{};
            if (F.vtype == NDHSS_R64)
                rc = gmres_one<double>(F, d_rowptr, d_col, (const double*)d_vals, (const double*)bb, (double*)xx, o, &S, ws, st);
            else
                rc = gmres_one<c128>(F, d_rowptr, d_col, (const c128*)d_vals, (const c128*)bb, (c128*)xx, o, &S, ws, st);
            if (rc == NDHSS_OK && conj) rc = conj_inplace(static_cast<c128*>(xx), F.n, st);
            if (rc == NDHSS_OK && !xdev) {
                if (cudaMemcpyAsync(xdst, dx, (size_t)F.n * vsz, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    rc = set_error(NDHSS_ERR_CUDA, "ndhss_gmres: device-to-host copy failed");
            }
            if (stats) stats[rhs] = S;
            if (!S.converged) any_fail = true;
        }
        cudaFreeAsync(work, st);
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == NDHSS_OK)
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_gmres: stream synchronisation failed");
        if (rc == NDHSS_OK) rc = apply_check_error(F, "ndhss_gmres");
        if (rc == NDHSS_OK && any_fail)
            rc = set_error(NDHSS_ERR_NOT_CONVERGED, "ndhss_gmres: tolerance not reached within maxit");
        return rc;
    });
}

}  // extern "C"
