// ULV factorization of HSS matrices (the interior blocks A_ii of the fronts
// strictly above the switching level), one CTA per HSS node, nodes of one
// HSS level of every front in one launch, deepest level first.
//
// A node's current block D (m x m) has row basis U and column basis V
// (m x k; the coupling to the rest of A_ii is U B V'^T through transposes,
// A_ii being complex symmetric).  With Householder QR, Q^H U = [R; 0]: the
// last ne = m - k rows of Q^H D do not couple to the rest.  The QR of their
// conjugate transpose gives W with (Q^H D)_b W = [L 0]: the first ne unknowns
// of W^H x are eliminated by a triangular solve.  What remains is the
// reduced block D^ = (Q^H D W)(0:k, ne:m) with bases U^ = R and V^ (from
// V^T W); siblings merge into the parent's block
//   [[D^_a, U^_a B12 V^_b^T], [U^_b B21 V^_a^T, D^_b]],
// bases blockdiag(U^_a, U^_b) E and blockdiag(V^_a, V^_b) E (E the nested
// transfer matrix of the compression); the root block is inverted (Gauss-
// Jordan, partial pivoting).  The apply needs matrix-vector products only:
//   Mup = [L^-1 Q^H_b; Q^H_t - C L^-1 Q^H_b; P1 L^-1 Q^H_b]   ((m + k) x m)
// maps a node's right-hand side to (eliminated unknowns y1, reduced
// right-hand side r^, coupling G of the eliminated unknowns to the outside),
// C = (Q^H D W)(0:k, 0:ne), P1 = (V^T W)(:, 0:ne); Mm corrects a merged
// right-hand side by the children's G; W maps [y1; x2] back on the way down.
// All matrices are column-major; the arithmetic is the factor's type.
#include "ulv.cuh"

namespace ndhss {
namespace {

constexpr int UT = 256;

__device__ __forceinline__ double re_(double a) { return a; }
__device__ __forceinline__ float re_(float a) { return a; }
template <typename R> __device__ __forceinline__ R re_(Cx<R> a) { return a.x; }
__device__ __forceinline__ double im_(double) { return 0.0; }
__device__ __forceinline__ float im_(float) { return 0.0f; }
template <typename R> __device__ __forceinline__ R im_(Cx<R> a) { return a.y; }
__device__ __forceinline__ float absq(float a) { return a * a; }
__device__ __forceinline__ double absq(double a) { return a * a; }
template <typename R> __device__ __forceinline__ R absq(Cx<R> a) { return a.x * a.x + a.y * a.y; }
template <typename T> __device__ __forceinline__ T mk(typename Tr<T>::real r);
template <> __device__ __forceinline__ double mk<double>(double r) { return r; }
template <> __device__ __forceinline__ float mk<float>(float r) { return r; }
template <> __device__ __forceinline__ c128 mk<c128>(double r) { return {r, 0.0}; }
template <> __device__ __forceinline__ c64 mk<c64>(float r) { return {r, 0.0f}; }
template <typename T> __device__ __forceinline__ T mul(T a, T b) { return fmac(a, b, zero<T>()); }

template <typename R>
__device__ R block_sum(R v, R* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    R s = 0;
    for (int i = 0; i < UT / 32; ++i) s += red[i];
    return s;
}

template <typename T>
__device__ void cta_set(T* A, int lda, int rows, int cols, bool identity) {
    for (int64_t q = threadIdx.x; q < (int64_t)rows * cols; q += UT) {
        const int i = (int)(q % rows), j = (int)(q / rows);
        A[(int64_t)j * lda + i] = (identity && i == j) ? one<T>() : zero<T>();
    }
}

template <typename T>
__device__ void cta_copy(T* B, int ldb, const T* A, int lda, int rows, int cols) {
    for (int64_t q = threadIdx.x; q < (int64_t)rows * cols; q += UT) {
        const int i = (int)(q % rows), j = (int)(q / rows);
        B[(int64_t)j * ldb + i] = A[(int64_t)j * lda + i];
    }
}

// op: 0 = A, 1 = A^T, 2 = A^H
template <typename T>
__device__ __forceinline__ T opget(const T* A, int lda, int op, int i, int l) {
    if (op == 0) return A[(int64_t)l * lda + i];
    const T v = A[(int64_t)i * lda + l];
    return op == 2 ? conjv(v) : v;
}

// C (M x N) = s * op(A) (M x K) op(B) (K x N) (+ C when acc)
template <typename T>
__device__ void cta_gemm(int M, int N, int K, const T* A, int lda, int opA, const T* B, int ldb, int opB, T* C, int ldc,
                         bool acc, bool neg) {
    for (int64_t q = threadIdx.x; q < (int64_t)M * N; q += UT) {
        const int i = (int)(q % M), j = (int)(q / M);
        T s = zero<T>();
        for (int l = 0; l < K; ++l) s = fmac(opget(A, lda, opA, i, l), opget(B, ldb, opB, l, j), s);
        if (neg) s = -s;
        T* c = C + (int64_t)j * ldc + i;
        *c = acc ? *c + s : s;
    }
}

// In-place Householder QR of A (m x n, ld lda), LAPACK conventions (zgeqr2):
// H_j = I - tau_j v_j v_j^H with v_j(j) = 1 stored below the diagonal, R on
// and above it; during the factorization H_j^H is applied to the trailing
// columns.
template <typename T>
__device__ void cta_qr(T* A, int lda, int m, int n, T* tau, typename Tr<T>::real* red, T* sh) {
    using R = typename Tr<T>::real;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kk = min(m, n);
    for (int j = 0; j < kk; ++j) {
        T* a = A + (int64_t)j * lda;
        R part = 0;
        for (int i = j + 1 + threadIdx.x; i < m; i += UT) part += absq(a[i]);
        const R xn2 = block_sum(part, red);
        if (threadIdx.x == 0) {
            const T alpha = a[j];
            T t = zero<T>(), sc = zero<T>();
            if (!(xn2 == R(0) && im_(alpha) == R(0))) {
                const R nrm = sqrt(absq(alpha) + xn2);
                const R beta = re_(alpha) >= R(0) ? -nrm : nrm;
                const T bt = mk<T>(beta);
                t = mul(bt - alpha, recip(bt));
                sc = recip(alpha - bt);
                a[j] = bt;
            }
            sh[0] = t;
            sh[1] = sc;
            tau[j] = t;
        }
        __syncthreads();
        const T t = sh[0], sc = sh[1];
        if (!(re_(t) == R(0) && im_(t) == R(0))) {
            for (int i = j + 1 + threadIdx.x; i < m; i += UT) a[i] = mul(a[i], sc);
            __syncthreads();
            const T tc = conjv(t);
            for (int c = j + 1 + warp; c < n; c += UT / 32) {
                T* b = A + (int64_t)c * lda;
                T w = zero<T>();
                for (int i = j + lane; i < m; i += 32) w = fmac(conjv(i == j ? one<T>() : a[i]), b[i], w);
                for (int o = 16; o; o >>= 1) {
                    if constexpr (Tr<T>::cplx) {
                        w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
                        w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
                    } else {
                        w += __shfl_xor_sync(0xffffffffu, w, o);
                    }
                }
                const T f = mul(tc, w);
                for (int i = j + lane; i < m; i += 32) b[i] = b[i] - mul(i == j ? one<T>() : a[i], f);
            }
        }
        __syncthreads();
    }
}

// X (m x ncol) <- H_{j0} ... applied from the left: forward order with
// conjugated tau gives Q^H X, backward order with tau gives Q X.
template <typename T>
__device__ void cta_apply_q(const T* V, int ldv, const T* tau, int m, int nr, T* X, int ldx, int ncol, bool qh) {
    using R = typename Tr<T>::real;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < nr; ++s) {
        const int j = qh ? s : nr - 1 - s;
        const T t = qh ? conjv(tau[j]) : tau[j];
        if (re_(t) == R(0) && im_(t) == R(0)) continue;
        const T* v = V + (int64_t)j * ldv;
        for (int c = warp; c < ncol; c += UT / 32) {
            T* b = X + (int64_t)c * ldx;
            T w = zero<T>();
            for (int i = j + lane; i < m; i += 32) w = fmac(conjv(i == j ? one<T>() : v[i]), b[i], w);
            for (int o = 16; o; o >>= 1) {
                if constexpr (Tr<T>::cplx) {
                    w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
                    w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
                } else {
                    w += __shfl_xor_sync(0xffffffffu, w, o);
                }
            }
            const T f = mul(t, w);
            for (int i = j + lane; i < m; i += 32) b[i] = b[i] - mul(i == j ? one<T>() : v[i], f);
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(UT) ulv_factor_kernel(const UlvJob<T>* __restrict__ jobs, const UlvJob<T>* __restrict__ all) {
    using R = typename Tr<T>::real;
    __shared__ R red[UT / 32];
    __shared__ T sh[4];
    __shared__ int s_piv;
    const UlvJob<T> J = jobs[blockIdx.x];
    const int m = J.m, k = J.k, ne = J.ne;
    // work layout (ulv_work_elems)
    T* wD = J.w;                          // m x m: D, then Q^H D
    T* wQ = wD + (int64_t)m * m;          // m x m: Q^H
    T* wDW = wQ + (int64_t)m * m;         // m x m: Q^H D W
    T* wU = wDW + (int64_t)m * m;         // m x k: U, then its QR
    T* wV = wU + (int64_t)m * k;          // m x k
    T* wT = wV + (int64_t)m * k;          // m x ne: (Q^H D)_b^H, then its QR
    T* wVW = wT + (int64_t)m * ne;        // k x m: V^T W
    T* wLi = wVW + (int64_t)k * m;        // ne x ne: L^-1
    T* wY = wLi + (int64_t)ne * ne;       // ne x m: L^-1 Q^H_b
    T* tau1 = wY + (int64_t)ne * m;       // m
    T* tau2 = tau1 + m;                   // m
    T* wA = wD + 3 * (int64_t)m * m;      // (re-used) scratch for merge products: starts at wU
    // ---- current block and bases
    if (J.leaf) {
        cta_copy(wD, m, J.D0, (int)J.ldd0, m, m);
        if (!J.root) {
            cta_copy(wU, m, J.X, (int)J.ldx, m, k);
            cta_copy(wV, m, J.X, (int)J.ldx, m, k);
        }
    } else {
        const UlvJob<T>& A = all[J.c1];
        const UlvJob<T>& B = all[J.c2];
        const int ta = A.kt, tb = B.kt, ka = J.ka, kb = J.kb;
        // Mm = [[0, U^_a B12], [U^_b B21, 0]]
        cta_set(J.Mm, m, m, ka + kb, false);
        __syncthreads();
        cta_gemm(ta, kb, ka, A.Uh, ta, 0, J.B12, ka, 0, J.Mm + (int64_t)ka * m, m, false, false);
        cta_gemm(tb, ka, kb, B.Uh, tb, 0, J.B21, kb, 0, J.Mm + ta, m, false, false);
        cta_copy(wD, m, A.Dh, ta, ta, ta);
        cta_copy(wD + (int64_t)ta * m + ta, m, B.Dh, tb, tb, tb);
        __syncthreads();
        // off-diagonal blocks of D: (U^_a B12) V^_b^T and (U^_b B21) V^_a^T
        cta_gemm(ta, tb, kb, J.Mm + (int64_t)ka * m, m, 0, B.Vh, tb, 1, wD + (int64_t)ta * m, m, false, false);
        cta_gemm(tb, ta, ka, J.Mm + ta, m, 0, A.Vh, ta, 1, wD + ta, m, false, false);
        if (!J.root) {
            // U = blockdiag(U^_a, U^_b) E, V likewise
            cta_copy(J.E, ka + kb, J.X, (int)J.ldx, ka + kb, k);
            cta_gemm(ta, k, ka, A.Uh, ta, 0, J.X, (int)J.ldx, 0, wU, m, false, false);
            cta_gemm(tb, k, kb, B.Uh, tb, 0, J.X + ka, (int)J.ldx, 0, wU + ta, m, false, false);
            cta_gemm(ta, k, ka, A.Vh, ta, 0, J.X, (int)J.ldx, 0, wV, m, false, false);
            cta_gemm(tb, k, kb, B.Vh, tb, 0, J.X + ka, (int)J.ldx, 0, wV + ta, m, false, false);
        }
    }
    __syncthreads();
    (void)wA;
    if (J.root) {
        // Dinv by Gauss-Jordan with partial pivoting (wD is destroyed)
        T* Di = J.Dinv;
        cta_set(Di, m, m, m, true);
        __syncthreads();
        for (int j = 0; j < m; ++j) {
            if (threadIdx.x == 0) {
                int p = j;
                R best = -1;
                for (int i = j; i < m; ++i) {
                    const R v = absq(wD[(int64_t)j * m + i]);
                    if (v > best) { best = v; p = i; }
                }
                s_piv = p;
                if (best <= R(0) && J.status) *J.status = 1;
            }
            __syncthreads();
            const int p = s_piv;
            if (p != j)
                for (int c = threadIdx.x; c < 2 * m; c += UT) {
                    T* M = c < m ? wD : Di;
                    const int cc = c < m ? c : c - m;
                    const T t = M[(int64_t)cc * m + j];
                    M[(int64_t)cc * m + j] = M[(int64_t)cc * m + p];
                    M[(int64_t)cc * m + p] = t;
                }
            __syncthreads();
            if (threadIdx.x == 0) sh[0] = recip(wD[(int64_t)j * m + j]);
            __syncthreads();
            const T ip = sh[0];
            for (int c = threadIdx.x; c < 2 * m; c += UT) {
                T* M = c < m ? wD : Di;
                const int cc = c < m ? c : c - m;
                M[(int64_t)cc * m + j] = mul(M[(int64_t)cc * m + j], ip);
            }
            __syncthreads();
            for (int64_t q = threadIdx.x; q < (int64_t)m * 2 * m; q += UT) {
                const int i = (int)(q % m), c = (int)(q / m);
                if (i == j) continue;
                T* M = c < m ? wD : Di;
                const int cc = c < m ? c : c - m;
                const T f = wD[(int64_t)j * m + i];
                if (cc == j && c < m) continue;     // column j of D is cleared after the sweep
                M[(int64_t)cc * m + i] = M[(int64_t)cc * m + i] - mul(f, M[(int64_t)cc * m + j]);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < m; i += UT)
                if (i != j) wD[(int64_t)j * m + i] = zero<T>();
            __syncthreads();
        }
        return;
    }
    if (ne == 0) {
        // nothing to eliminate: pass the block up unchanged
        cta_set(J.Mup, m + k, m + k, m, false);
        cta_set(J.W, m, m, m, true);
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += UT) J.Mup[(int64_t)i * (m + k) + i] = one<T>();
        cta_copy(J.Dh, m, wD, m, m, m);
        cta_copy(J.Uh, m, wU, m, m, k);
        cta_copy(J.Vh, m, wV, m, m, k);
        return;
    }
    // ---- Q^H U = [R; 0]
    cta_qr(wU, m, m, k, tau1, red, sh);
    cta_set(wQ, m, m, m, true);
    __syncthreads();
    cta_apply_q(wU, m, tau1, m, k, wQ, m, m, true);        // Q^H
    cta_apply_q(wU, m, tau1, m, k, wD, m, m, true);        // Q^H D
    // U^ = R (k x k)
    for (int64_t q = threadIdx.x; q < (int64_t)k * k; q += UT) {
        const int i = (int)(q % k), j = (int)(q / k);
        J.Uh[(int64_t)j * k + i] = i <= j ? wU[(int64_t)j * m + i] : zero<T>();
    }
    // ---- (Q^H D)_b^H = W [Rl; 0]  (m x ne), W explicit
    for (int64_t q = threadIdx.x; q < (int64_t)m * ne; q += UT) {
        const int i = (int)(q % m), j = (int)(q / m);
        wT[(int64_t)j * m + i] = conjv(wD[(int64_t)i * m + (k + j)]);
    }
    __syncthreads();
    cta_qr(wT, m, m, ne, tau2, red, sh);
    cta_set(J.W, m, m, m, true);
    __syncthreads();
    cta_apply_q(wT, m, tau2, m, ne, J.W, m, m, false);    // W = H_0 ... H_{ne-1}
    // ---- Q^H D W, V^T W
    cta_gemm(m, m, m, wD, m, 0, J.W, m, 0, wDW, m, false, false);
    cta_gemm(k, m, m, wV, m, 1, J.W, m, 0, wVW, k, false, false);
    // ---- L^-1, L = Rl^H (ne x ne lower triangular): column c by forward substitution
    for (int c = threadIdx.x; c < ne; c += UT) {
        for (int i = 0; i < ne; ++i) {
            if (i < c) { wLi[(int64_t)c * ne + i] = zero<T>(); continue; }
            T s = (i == c) ? one<T>() : zero<T>();
            for (int l = c; l < i; ++l) s = s - mul(conjv(wT[(int64_t)i * m + l]), wLi[(int64_t)c * ne + l]);
            wLi[(int64_t)c * ne + i] = mul(s, recip(conjv(wT[(int64_t)i * m + i])));
        }
    }
    __syncthreads();
    // D^, V^ for the parent
    cta_copy(J.Dh, k, wDW + (int64_t)ne * m, m, k, k);
    for (int64_t q = threadIdx.x; q < (int64_t)k * k; q += UT) {
        const int i = (int)(q % k), j = (int)(q / k);
        J.Vh[(int64_t)j * k + i] = wVW[(int64_t)(ne + i) * k + j];
    }
    // ---- Mup = [Y; Q^H_t - C Y; P1 Y] with Y = L^-1 Q^H_b
    cta_gemm(ne, m, ne, wLi, ne, 0, wQ + k, m, 0, wY, ne, false, false);
    __syncthreads();
    const int lm = m + k;
    cta_copy(J.Mup, lm, wY, ne, ne, m);
    cta_copy(J.Mup + ne, lm, wQ, m, k, m);
    __syncthreads();
    cta_gemm(k, m, ne, wDW, m, 0, wY, ne, 0, J.Mup + ne, lm, true, true);
    cta_gemm(k, m, ne, wVW, k, 0, wY, ne, 0, J.Mup + ne + k, lm, false, false);
}

}  // namespace

template <typename T>
ndhss_status ulv_launch_level(const UlvJob<T>* d_jobs, const UlvJob<T>* d_all, int count, cudaStream_t st) {
    if (count <= 0) return NDHSS_OK;
    ulv_factor_kernel<T><<<(unsigned)count, UT, 0, st>>>(d_jobs, d_all);
    NDHSS_LAUNCH_CHECK("ulv_factor_kernel");
    return NDHSS_OK;
}

template ndhss_status ulv_launch_level<double>(const UlvJob<double>*, const UlvJob<double>*, int, cudaStream_t);
template ndhss_status ulv_launch_level<float>(const UlvJob<float>*, const UlvJob<float>*, int, cudaStream_t);
template ndhss_status ulv_launch_level<c128>(const UlvJob<c128>*, const UlvJob<c128>*, int, cudaStream_t);
template ndhss_status ulv_launch_level<c64>(const UlvJob<c64>*, const UlvJob<c64>*, int, cudaStream_t);

}  // namespace ndhss
