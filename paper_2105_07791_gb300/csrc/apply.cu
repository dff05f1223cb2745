// y = P^{-1} x by Algorithm 3.1 on the device.
//
//   gather/cast   y = x(perm) converted to the factor precision
//   up-sweep      levels bottom-up:  y(B^s) += L^s y(I^s)          (L = -BL P)
//   diagonal      all nodes at once: z(I^s) = A_ii^{-1} y(I^s)     ("fully in parallel")
//   down-sweep    levels top-down:   z(I^s) += R^s z(B^s)
//   scatter/cast  out(perm) = z converted back to float64
//
// Work is split into tasks of APPLY_ROWS output rows of one node; the tasks
// of a level (or of the diagonal step) form one launch.  The whole factor is
// streamed once per apply: A_ii^{-1}, L and R of every node once each.
#include <mutex>

#include "factor.cuh"

namespace ndhss {
namespace {

constexpr int AT = 256;

__device__ __forceinline__ int nf(const int32_t* node, int s, int f) { return node[s * NODE_NF + f]; }

__device__ __forceinline__ double shfl_xor_t(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_xor_t(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <typename R>
__device__ __forceinline__ Cx<R> shfl_xor_t(Cx<R> v, int o) {
    return {__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}

template <typename T, typename V>
__global__ void gather_cast_kernel(int n, const int32_t* __restrict__ perm, const V* __restrict__ x, T* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = from_val<T>(x[perm[i]]);
}

template <typename T, typename V>
__global__ void scatter_cast_kernel(int n, const int32_t* __restrict__ perm, const T* __restrict__ z, V* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = to_val(z[i]);
}

// Rows [r0, r0 + 64) of (block A, column-major, leading dimension lda) times
// the vector xs (shared memory): 8 warps take every 8th column, each lane
// owns rows r0 + lane and r0 + lane + 32, and four columns are in flight per
// step, so a thread keeps eight independent loads outstanding and a warp
// reads each column segment as one contiguous 64-row access.  The eight warp
// partial sums are added in shared memory; lanes of warp 0 and 1 return the
// results for rows r0 + tid (tid < 64).
constexpr int AW = AT / 32;

template <typename T>
__device__ __forceinline__ T gemv_rows64(const T* __restrict__ A, int64_t lda, int rows, int cols, int r0,
                                         const T* __restrict__ xs, T (*red)[APPLY_ROWS]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ra = r0 + lane, rb = r0 + lane + 32;
    const bool va = ra < rows, vb = rb < rows;
    T acc0 = zero<T>(), acc1 = zero<T>();
    int c = warp;
    for (; c + 3 * AW < cols; c += 4 * AW) {
        T a[4], b[4], x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T* col = A + (int64_t)(c + u * AW) * lda;
            a[u] = va ? col[ra] : zero<T>();
            b[u] = vb ? col[rb] : zero<T>();
            x[u] = xs[c + u * AW];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc0 = fmac(a[u], x[u], acc0);
            acc1 = fmac(b[u], x[u], acc1);
        }
    }
    for (; c < cols; c += AW) {
        const T* col = A + (int64_t)c * lda;
        const T xv = xs[c];
        if (va) acc0 = fmac(col[ra], xv, acc0);
        if (vb) acc1 = fmac(col[rb], xv, acc1);
    }
    red[warp][lane] = acc0;
    red[warp][lane + 32] = acc1;
    __syncthreads();
    T sum = zero<T>();
    if (threadIdx.x < APPLY_ROWS)
        for (int w = 0; w < AW; ++w) sum += red[w][threadIdx.x];
    return sum;
}

// y(B^s) -= BL y(I^s)(sigma)   (= L^s y(I^s), Eq. 3.3a)
template <typename T>
__global__ void __launch_bounds__(AT)
upsweep_kernel(const int32_t* __restrict__ tasks, const int32_t* __restrict__ node, const int64_t* __restrict__ foff,
               const int32_t* __restrict__ blist, const int32_t* __restrict__ sigma, const T* __restrict__ front,
               T* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[AW][APPLY_ROWS];
    T* ys = reinterpret_cast<T*>(smem_raw);
    const int s = tasks[2 * blockIdx.x], j0 = tasks[2 * blockIdx.x + 1];
    const int m_i = nf(node, s, 5), m_b = nf(node, s, 7), i_off = nf(node, s, 4), b_off = nf(node, s, 6);
    const int64_t m = (int64_t)m_i + m_b;
    for (int c = threadIdx.x; c < m_i; c += AT) ys[c] = y[i_off + sigma[i_off + c]];
    __syncthreads();
    const T sum = gemv_rows64(front + foff[s] + m_i, m, m_b, m_i, j0, ys, red);
    const int j = j0 + threadIdx.x;
    if (threadIdx.x < APPLY_ROWS && j < m_b) {
        const int g = blist[b_off + j];
        y[g] = y[g] - sum;
    }
}

// z(I^s) = X y(I^s)(sigma)   (= A_ii^{-1} y(I^s))
template <typename T>
__global__ void __launch_bounds__(AT)
diag_kernel(const int32_t* __restrict__ tasks, const int32_t* __restrict__ node, const int64_t* __restrict__ foff,
            const int32_t* __restrict__ sigma, const T* __restrict__ front, const T* __restrict__ y, T* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[AW][APPLY_ROWS];
    T* ys = reinterpret_cast<T*>(smem_raw);
    const int s = tasks[2 * blockIdx.x], i0 = tasks[2 * blockIdx.x + 1];
    const int m_i = nf(node, s, 5), i_off = nf(node, s, 4);
    const int64_t m = (int64_t)m_i + nf(node, s, 7);
    for (int c = threadIdx.x; c < m_i; c += AT) ys[c] = y[i_off + sigma[i_off + c]];
    __syncthreads();
    const T sum = gemv_rows64(front + foff[s], m, m_i, m_i, i0, ys, red);
    const int i = i0 + threadIdx.x;
    if (threadIdx.x < APPLY_ROWS && i < m_i) z[i_off + i] = sum;
}

// z(I^s) += R z(B^s)   (Eq. 3.3b)
template <typename T>
__global__ void __launch_bounds__(AT)
downsweep_kernel(const int32_t* __restrict__ tasks, const int32_t* __restrict__ node, const int64_t* __restrict__ foff,
                 const int32_t* __restrict__ blist, const T* __restrict__ front, T* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[AW][APPLY_ROWS];
    T* zb = reinterpret_cast<T*>(smem_raw);
    const int s = tasks[2 * blockIdx.x], i0 = tasks[2 * blockIdx.x + 1];
    const int m_i = nf(node, s, 5), m_b = nf(node, s, 7), i_off = nf(node, s, 4), b_off = nf(node, s, 6);
    const int64_t m = (int64_t)m_i + m_b;
    for (int j = threadIdx.x; j < m_b; j += AT) zb[j] = z[blist[b_off + j]];
    __syncthreads();
    const T sum = gemv_rows64(front + foff[s] + (int64_t)m_i * m, m, m_i, m_b, i0, zb, red);
    const int i = i0 + threadIdx.x;
    if (threadIdx.x < APPLY_ROWS && i < m_i) z[i_off + i] = z[i_off + i] + sum;
}


// Low-rank levels (R ~ X R(J, :), stored as X (m_i x k) and RJt = R(J, :)^T
// (m_b x k), both column-major; L = R^T by symmetry).  Each level is two
// launches over all its nodes:
//   dot   tasks (node, 8 outputs): warp w forms t[a0 + w] as a coalesced,
//         4-way unrolled dot product of a stored column with the gathered
//         vector, written to scratch;
//   axpy  tasks (node, 256 rows): each thread adds sum_a M(row, a) t[a].
// up-sweep (mode 0):   t = X^T y(I^s);     y(B^s) += RJt t
// down-sweep (mode 1): t = RJt^T z(B^s);   z(I^s) += X t
template <typename T>
__global__ void __launch_bounds__(AT)
lr_dot_kernel(const int32_t* __restrict__ tasks, const int32_t* __restrict__ node, const uint64_t* __restrict__ lrp,
              const int32_t* __restrict__ lrk, const int64_t* __restrict__ toff, const int32_t* __restrict__ blist,
              const T* __restrict__ v, T* __restrict__ tsc, int mode) {
    const int s = tasks[2 * blockIdx.x], a0 = tasks[2 * blockIdx.x + 1];
    const int m_i = nf(node, s, 5), m_b = nf(node, s, 7), i_off = nf(node, s, 4), b_off = nf(node, s, 6);
    const int k = lrk[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a = a0 + warp;
    if (a >= k) return;
    const T* X = reinterpret_cast<const T*>(lrp[s]);
    const T* col = (mode == 0) ? X + (int64_t)a * m_i : X + (int64_t)m_i * k + (int64_t)a * m_b;
    const int len = (mode == 0) ? m_i : m_b;
    T acc0 = zero<T>(), acc1 = zero<T>(), acc2 = zero<T>(), acc3 = zero<T>();
    int i = lane;
    if (mode == 0) {
        const T* x = v + i_off;
        for (; i + 96 < len; i += 128) {
            acc0 = fmac(col[i], x[i], acc0);
            acc1 = fmac(col[i + 32], x[i + 32], acc1);
            acc2 = fmac(col[i + 64], x[i + 64], acc2);
            acc3 = fmac(col[i + 96], x[i + 96], acc3);
        }
        for (; i < len; i += 32) acc0 = fmac(col[i], x[i], acc0);
    } else {
        const int32_t* bl = blist + b_off;
        for (; i + 96 < len; i += 128) {
            acc0 = fmac(col[i], v[bl[i]], acc0);
            acc1 = fmac(col[i + 32], v[bl[i + 32]], acc1);
            acc2 = fmac(col[i + 64], v[bl[i + 64]], acc2);
            acc3 = fmac(col[i + 96], v[bl[i + 96]], acc3);
        }
        for (; i < len; i += 32) acc0 = fmac(col[i], v[bl[i]], acc0);
    }
    T acc = (acc0 + acc1) + (acc2 + acc3);
    for (int o = 16; o; o >>= 1) acc = acc + shfl_xor_t(acc, o);
    if (lane == 0) tsc[toff[s] + a] = acc;
}

template <typename T>
__global__ void __launch_bounds__(AT)
lr_axpy_kernel(const int32_t* __restrict__ tasks, const int32_t* __restrict__ node, const uint64_t* __restrict__ lrp,
               const int32_t* __restrict__ lrk, const int64_t* __restrict__ toff, const int32_t* __restrict__ blist,
               const T* __restrict__ tsc, T* __restrict__ v, int mode) {
    __shared__ T ts[512];
    const int s = tasks[2 * blockIdx.x], r0 = tasks[2 * blockIdx.x + 1];
    const int m_i = nf(node, s, 5), m_b = nf(node, s, 7), i_off = nf(node, s, 4), b_off = nf(node, s, 6);
    const int k = lrk[s];
    for (int a = threadIdx.x; a < k && a < 512; a += AT) ts[a] = tsc[toff[s] + a];
    __syncthreads();
    const T* X = reinterpret_cast<const T*>(lrp[s]);
    const T* M = (mode == 0) ? X + (int64_t)m_i * k : X;       // RJt (m_b x k) or X (m_i x k)
    const int len = (mode == 0) ? m_b : m_i;
    const int r = r0 + threadIdx.x;
    if (r >= len) return;
    T acc0 = zero<T>(), acc1 = zero<T>(), acc2 = zero<T>(), acc3 = zero<T>();
    int a = 0;
    for (; a + 3 < k; a += 4) {
        acc0 = fmac(M[(int64_t)a * len + r], ts[a], acc0);
        acc1 = fmac(M[(int64_t)(a + 1) * len + r], ts[a + 1], acc1);
        acc2 = fmac(M[(int64_t)(a + 2) * len + r], ts[a + 2], acc2);
        acc3 = fmac(M[(int64_t)(a + 3) * len + r], ts[a + 3], acc3);
    }
    for (; a < k; ++a) acc0 = fmac(M[(int64_t)a * len + r], ts[a], acc0);
    const T acc = (acc0 + acc1) + (acc2 + acc3);
    if (mode == 0) {
        const int g = blist[b_off + r];
        v[g] = v[g] + acc;
    } else {
        v[i_off + r] = v[i_off + r] + acc;
    }
}

template <typename T, typename V>
ndhss_status apply_run(const FactorData& F, int32_t nrhs, const V* x, int64_t ldx, V* y, int64_t ldy, T* w0, T* w1,
                       cudaStream_t st) {
    const T* front = static_cast<const T*>(F.d_front);
    const int nb = (F.n + 255) / 256;
    const size_t smem_i = (size_t)std::max(F.max_mi, 1) * sizeof(T);
    const size_t smem_b = (size_t)std::max(F.max_mb, 1) * sizeof(T);
    if (smem_i > 48 * 1024) {
        NDHSS_CUDA_TRY(cudaFuncSetAttribute(upsweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_i));
        NDHSS_CUDA_TRY(cudaFuncSetAttribute(diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_i));
    }
    if (smem_b > 48 * 1024)
        NDHSS_CUDA_TRY(cudaFuncSetAttribute(downsweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    T* tsc = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(w1) + ((size_t)F.n * sizeof(T) + 255) / 256 * 256);
    for (int r = 0; r < nrhs; ++r) {
        gather_cast_kernel<T, V><<<nb, 256, 0, st>>>(F.n, F.d_perm, x + r * ldx, w0);
        NDHSS_LAUNCH_CHECK("gather_cast_kernel");
        for (int l = F.depth; l >= 0; --l) {
            if (l < F.L_hss && !F.lr_cnt.empty()) {
                if (F.lr_dot_cnt[l]) {
                    lr_dot_kernel<T><<<(unsigned)F.lr_dot_cnt[l], AT, 0, st>>>(F.d_tasks + 2 * F.lr_dot_off[l], F.d_node,
                                                                             F.d_lr_ptr, F.d_lr_k, F.d_lr_toff, F.d_blist,
                                                                             w0, tsc, 0);
                    NDHSS_LAUNCH_CHECK("lr_dot_kernel");
                    lr_axpy_kernel<T><<<(unsigned)F.lr_bax_cnt[l], AT, 0, st>>>(F.d_tasks + 2 * F.lr_bax_off[l], F.d_node,
                                                                              F.d_lr_ptr, F.d_lr_k, F.d_lr_toff, F.d_blist,
                                                                              tsc, w0, 0);
                    NDHSS_LAUNCH_CHECK("lr_axpy_kernel");
                }
                continue;
            }
            if (F.up_cnt[l] == 0) continue;
            upsweep_kernel<T><<<(unsigned)F.up_cnt[l], AT, smem_i, st>>>(F.d_tasks + 2 * F.up_off[l], F.d_node, F.d_foff,
                                                                         F.d_blist, F.d_sigma, front, w0);
            NDHSS_LAUNCH_CHECK("upsweep_kernel");
        }
        if (F.diag_cnt > 0) {
            diag_kernel<T><<<(unsigned)F.diag_cnt, AT, smem_i, st>>>(F.d_tasks + 2 * F.diag_off, F.d_node, F.d_foff,
                                                                     F.d_sigma, front, w0, w1);
            NDHSS_LAUNCH_CHECK("diag_kernel");
        }
        for (int l = 0; l <= F.depth; ++l) {
            if (l < F.L_hss && !F.lr_cnt.empty()) {
                if (F.lr_dot_cnt[l]) {
                    lr_dot_kernel<T><<<(unsigned)F.lr_dot_cnt[l], AT, 0, st>>>(F.d_tasks + 2 * F.lr_dot_off[l], F.d_node,
                                                                             F.d_lr_ptr, F.d_lr_k, F.d_lr_toff, F.d_blist,
                                                                             w1, tsc, 1);
                    NDHSS_LAUNCH_CHECK("lr_dot_kernel");
                    lr_axpy_kernel<T><<<(unsigned)F.lr_iax_cnt[l], AT, 0, st>>>(F.d_tasks + 2 * F.lr_iax_off[l], F.d_node,
                                                                              F.d_lr_ptr, F.d_lr_k, F.d_lr_toff, F.d_blist,
                                                                              tsc, w1, 1);
                    NDHSS_LAUNCH_CHECK("lr_axpy_kernel");
                }
                continue;
            }
            if (F.dn_cnt[l] == 0) continue;
            downsweep_kernel<T><<<(unsigned)F.dn_cnt[l], AT, smem_b, st>>>(F.d_tasks + 2 * F.dn_off[l], F.d_node, F.d_foff,
                                                                           F.d_blist, front, w1);
            NDHSS_LAUNCH_CHECK("downsweep_kernel");
        }
        scatter_cast_kernel<T, V><<<nb, 256, 0, st>>>(F.n, F.d_perm, w1, y + r * ldy);
        NDHSS_LAUNCH_CHECK("scatter_cast_kernel");
    }
    return NDHSS_OK;
}

}  // namespace

// two permuted work vectors plus the low-rank scratch t (one slot per rank of every low-rank node)
size_t apply_work_bytes(const FactorData& F) {
    return 2 * (((size_t)F.n * F.esize + 255) / 256 * 256) + (size_t)std::max<int64_t>(F.lr_t_total, 1) * F.esize + 256;
}

ndhss_status apply_device(const FactorData& F, int32_t nrhs, const void* d_x, int64_t ldx, void* d_y, int64_t ldy,
                          void* d_work, cudaStream_t st) {
    const bool cplx = F.vtype == NDHSS_C128;
    unsigned char* w = static_cast<unsigned char*>(d_work);
    const size_t half = ((size_t)F.n * F.esize + 255) / 256 * 256;
    if (!cplx && F.prec == NDHSS_FP64)
        return apply_run<double, double>(F, nrhs, (const double*)d_x, ldx, (double*)d_y, ldy, (double*)w, (double*)(w + half), st);
    if (!cplx)
        return apply_run<float, double>(F, nrhs, (const double*)d_x, ldx, (double*)d_y, ldy, (float*)w, (float*)(w + half), st);
    if (F.prec == NDHSS_FP64)
        return apply_run<c128, c128>(F, nrhs, (const c128*)d_x, ldx, (c128*)d_y, ldy, (c128*)w, (c128*)(w + half), st);
    return apply_run<c64, c128>(F, nrhs, (const c128*)d_x, ldx, (c128*)d_y, ldy, (c64*)w, (c64*)(w + half), st);
}

}  // namespace ndhss

extern "C" ndhss_status ndhss_apply(const ndhss_factorization* fh, int32_t nrhs, const void* x, int64_t ldx, void* y,
                                    int64_t ldy, void* stream) {
    using namespace ndhss;
    clear_error();
    if (!fh || !x || !y || nrhs < 0) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply: bad argument");
    const FactorData& F = fh->f;
    if (ldx < F.n || ldy < F.n) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply: leading dimension < n");
    if (nrhs == 0) return NDHSS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t vsz = F.vtype == NDHSS_C128 ? 16 : 8;
    const bool xdev = is_device_ptr(x), ydev = is_device_ptr(y);
    const size_t wb = apply_work_bytes(F) + (xdev ? 0 : (size_t)F.n * nrhs * vsz + 256) + (ydev ? 0 : (size_t)F.n * nrhs * vsz + 256);
    void* work = nullptr;
    NDHSS_CUDA_TRY(cudaMallocAsync(&work, wb, st));
    unsigned char* p = static_cast<unsigned char*>(work) + (apply_work_bytes(F) + 255) / 256 * 256;
    const void* dx = x;
    void* dy = y;
    int64_t lx = ldx, ly = ldy;
    ndhss_status rc = NDHSS_OK;
    if (!xdev) {
        dx = p;
        lx = F.n;
        p += ((size_t)F.n * nrhs * vsz + 255) / 256 * 256;
        for (int r = 0; r < nrhs && rc == NDHSS_OK; ++r)
            if (cudaMemcpyAsync((unsigned char*)dx + (size_t)r * F.n * vsz, (const unsigned char*)x + (size_t)r * ldx * vsz,
                                (size_t)F.n * vsz, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = set_error(NDHSS_ERR_CUDA, "ndhss_apply: host-to-device copy failed");
    }
    if (!ydev) {
        dy = p;
        ly = F.n;
    }
    if (rc == NDHSS_OK) rc = apply_device(F, nrhs, dx, lx, dy, ly, work, st);
    if (rc == NDHSS_OK && !ydev) {
        for (int r = 0; r < nrhs && rc == NDHSS_OK; ++r)
            if (cudaMemcpyAsync((unsigned char*)y + (size_t)r * ldy * vsz, (const unsigned char*)dy + (size_t)r * F.n * vsz,
                                (size_t)F.n * vsz, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                rc = set_error(NDHSS_ERR_CUDA, "ndhss_apply: device-to-host copy failed");
    }
    cudaFreeAsync(work, st);
    if (!xdev || !ydev) {
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == NDHSS_OK)
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_apply: stream synchronisation failed");
    }
    return rc;
}

// --------------------------------------------------------------------------
// Allocation-free apply (no counterpart in the paper).
//
// Callers that must not allocate (graph recording without memory nodes, host
// callbacks, foreign allocators) get the same Alg. 3.1 result with the two
// work vectors in this fixed static array instead of stream-ordered
// allocations.  The array is part of the module image, so every device that
// loads the library holds it until exit.  Host code must not take its address
// directly (that would be a host-side shadow): the device address is looked
// up once per device with cudaGetSymbolAddress.  Every call overwrites the
// whole work area it uses before reading it (gather writes all of the first
// vector, the diagonal step all of the second), so nothing needs clearing;
// overlapping calls race on the array.
namespace ndhss {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;
__device__ __align__(256) unsigned char g_apply_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};

ndhss_status scratch_for_current_device(void** out) {
    int dev = -1;
    NDHSS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply_noalloc: device %d beyond the supported %d", dev,
                         NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
        if (e != cudaSuccess || !p)
            return set_error(NDHSS_ERR_CUDA, "ndhss_apply_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                             cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return NDHSS_OK;
}

}  // namespace
}  // namespace ndhss

extern "C" ndhss_status ndhss_apply_noalloc(const ndhss_factorization* fh, const void* d_x, void* d_y, void* stream) {
    using namespace ndhss;
    clear_error();
    if (!fh || !d_x || !d_y) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply_noalloc: NULL argument");
    const FactorData& F = fh->f;
    const size_t need = apply_work_bytes(F);
    if (need > NOALLOC_SCRATCH_BYTES)
        return set_error(NDHSS_ERR_INVALID_ARG,
                         "ndhss_apply_noalloc: n = %d needs %zu bytes of work space but the static scratch holds %zu; "
                         "use ndhss_apply", F.n, need, NOALLOC_SCRATCH_BYTES);
    if (!is_device_ptr(d_x) || !is_device_ptr(d_y))
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply_noalloc: x and y must be device pointers");
    void* scratch = nullptr;
    const ndhss_status rc = scratch_for_current_device(&scratch);
    if (rc != NDHSS_OK) return rc;
    return apply_device(F, 1, d_x, F.n, d_y, F.n, scratch, static_cast<cudaStream_t>(stream));
}
