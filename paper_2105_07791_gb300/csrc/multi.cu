// Many right-hand sides at once: Alg. 3.1 applied to 32 interleaved vectors
// (one pass over the factor serves all of them), and restarted GMRES run in
// lockstep for many independent problems x 32 right-hand sides (the batched
// workload: the problems of a forest factorization, ndhss_build_tree_batched).
//
// Block vectors are stored interleaved: element (row, c) at row * 32 + c, so a
// row of 32 right-hand sides is one 512-byte (complex128) or 256-byte
// (complex64) line and every gather by a row index stays coalesced.
//
// Multi apply (dense fronts).  With u = y in elimination order, per level,
// deepest first, every node s of the level computes from u(I^s) read through
// its interchanges sigma:
//     z(I^s) = X11 u(I^s o sigma)          (A_ii^{-1} P^T, the diagonal step)
//     u(B^s) -= X21 u(I^s o sigma)          (the up-sweep, -L P^T)
// then per level, root level first:  z(I^s) += X12 z(B^s)  (the down-sweep, R).
// B^s lies inside the box of s, so the B sets of one level are disjoint and
// the I rows of a level are never B rows of the same level: a level is one
// launch of independent 64-row x 32-column tiles with no atomics.
//
// Batched GMRES.  System q = (problem s, column c) owns rows [off_s, off_s+1)
// of column c.  Every reduction is segmented by problem: a CTA covers up to
// SEG_ROWS rows of one problem and writes its partial sums, a second kernel
// adds a problem's partials in block order (deterministic).  Hessenberg,
// Givens rotations and the least-squares residual are per system (one thread
// each), with the same arithmetic and stopping rules as ndhss_gmres; a system
// that stops or converges keeps its x while the others go on.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "factor.cuh"
#include "mapply_tune.h"

namespace ndhss {
namespace {

constexpr int MR = 32;            // interleaved right-hand sides
constexpr int MT_ROWS = 64;       // rows per apply tile
constexpr int MT_K = 16;          // K chunk of an apply tile
constexpr int MT_THREADS = 128;   // threads of a dense apply tile (4 x 4 products each)
constexpr int SEG_ROWS = 1024;    // rows per reduction block
constexpr int BK = 32;            // restart + 1 <= BK

__device__ __forceinline__ double babs(double a) { return fabs(a); }
__device__ __forceinline__ double babs(c128 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double bre(double a) { return a; }
__device__ __forceinline__ double bre(c128 a) { return a.x; }
template <typename V> __device__ __forceinline__ V breal(double v);
template <> __device__ __forceinline__ double breal<double>(double v) { return v; }
template <> __device__ __forceinline__ c128 breal<c128>(double v) { return {v, 0.0}; }

// ------------------------------------------------------------ multi apply
// N consecutive elements from 16-byte aligned shared memory in 16-byte loads
template <int N, typename T>
__device__ __forceinline__ void lds_vec(const T* p, T (&v)[N]) {
    static_assert((N * sizeof(T)) % 16 == 0 || N * sizeof(T) < 16, "whole 16-byte words");
    if constexpr ((N * sizeof(T)) % 16 == 0) {
        constexpr int W = (int)(N * sizeof(T) / 16);
        float4 w[W];
#pragma unroll
        for (int i = 0; i < W; ++i) w[i] = reinterpret_cast<const float4*>(p)[i];
        memcpy(v, w, sizeof(v));
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = p[i];
    }
}
template <typename T, typename V>
__global__ void mgather_kernel(int64_t n, int nrhs, const int32_t* __restrict__ perm, const V* __restrict__ X,
                               int64_t ldx, T* __restrict__ U) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * MR; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pos = q / MR;
        const int c = (int)(q % MR);
        U[q] = c < nrhs ? from_val<T>(X[(int64_t)perm[pos] * ldx + c]) : zero<T>();
    }
}

template <typename T, typename V>
__global__ void mscatter_kernel(int64_t n, int nrhs, const int32_t* __restrict__ perm, const T* __restrict__ Z,
                                V* __restrict__ Y, int64_t ldy) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * MR; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pos = q / MR;
        const int c = (int)(q % MR);
        if (c < nrhs) Y[(int64_t)perm[pos] * ldy + c] = to_val(Z[q]);
    }
}

// One ROWS-row x 32-column tile of node s (ROWS 32 or 64, 2 ROWS threads):
// UP = the first m_i columns of the front against u(I^s o sigma) (rows < m_i
// to z, rows >= m_i subtracted from u(B^s)); !UP = the R block against
// z(B^s), added to z(I^s).
template <typename T, bool UP, int ROWS>
__global__ void __launch_bounds__(2 * ROWS)
mapply_kernel(const int2* __restrict__ jobs, const int32_t* __restrict__ node, const int64_t* __restrict__ foff,
              const T* __restrict__ front, const int32_t* __restrict__ sigma, const int32_t* __restrict__ blist,
              T* __restrict__ U, T* __restrict__ Z, const int* __restrict__ pact, const int32_t* __restrict__ nprob,
              const uint64_t* __restrict__ lr_ptr) {
    constexpr int NTH = 2 * ROWS;
    __shared__ __align__(16) T As[MT_K][ROWS];
    __shared__ __align__(16) T Bs[MT_K][MR];
    const int2 J = jobs[blockIdx.x];
    const int s = J.x, r0 = J.y;
    if (pact && !pact[nprob[s]]) return;          // a problem whose systems all stopped
    const int32_t* nd = node + (size_t)s * 14;
    const int i_off = nd[4], m_i = nd[5], b_off = nd[6], m_b = nd[7];
    const int64_t m = (int64_t)m_i + m_b;
    const T* F = front + foff[s];
    // a low-rank node's B rows go through mlr_kernel (its up tiles cover I only)
    const bool lowrank = lr_ptr && lr_ptr[s];
    const int rows = (UP && !lowrank) ? (int)m : m_i;
    const int K = UP ? m_i : m_b;
    const T* A = UP ? F : F + (int64_t)m_i * m;
    const T* src = UP ? U : Z;
    // thread (ty, tx) owns rows 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3
    // of the tile (16 products per 64 bytes read from shared memory)
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
    // the next K chunk's A entries, its row indices and then its B rows are
    // loaded into registers while the current chunk is multiplied
    T ra[ROWS * MT_K / NTH], rb[MT_K * MR / NTH];
    auto load_a = [&](int k0) {
        const int kc = min(MT_K, K - k0);
#pragma unroll
        for (int u = 0; u < ROWS * MT_K / NTH; ++u) {
            const int q = tid + NTH * u, r = q % ROWS, kk = q / ROWS;
            ra[u] = (r0 + r < rows && kk < kc) ? A[(int64_t)(k0 + kk) * m + r0 + r] : zero<T>();
        }
    };
    auto src_row = [&](int k0, int kk) {
        return k0 + kk < K ? (UP ? i_off + sigma[i_off + k0 + kk] : blist[b_off + k0 + kk]) : -1;
    };
    auto load_b = [&](int k0) {
#pragma unroll
        for (int u = 0; u < MT_K * MR / NTH; ++u) {
            const int q = tid + NTH * u, kk = q / MR, c = q % MR;
            const int sr = src_row(k0, kk);
            rb[u] = sr >= 0 ? src[(int64_t)sr * MR + c] : zero<T>();
        }
    };
    if (K > 0) {
        load_a(0);
        load_b(0);
    }
    for (int k0 = 0; k0 < K; k0 += MT_K) {
#pragma unroll
        for (int u = 0; u < ROWS * MT_K / NTH; ++u) {
            const int q = tid + NTH * u;
            As[q / ROWS][q % ROWS] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < MT_K * MR / NTH; ++u) {
            const int q = tid + NTH * u;
            Bs[q / MR][q % MR] = rb[u];
        }
        __syncthreads();
        if (k0 + MT_K < K) {
            load_a(k0 + MT_K);
            load_b(k0 + MT_K);
        }
#pragma unroll
        for (int kk = 0; kk < MT_K; ++kk) {
            // the thread's four rows of A and four columns of B as 16-byte
            // shared loads
            T a[4], bv[4];
            lds_vec<4>(&As[kk][4 * ty], a);
            lds_vec<4>(&Bs[kk][4 * tx], bv);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmac(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + 4 * ty + i;
        if (r >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * tx + j;
            if (UP) {
                if (r < m_i) {
                    Z[(int64_t)(i_off + r) * MR + c] = acc[i][j];
                } else {
                    T* p = U + (int64_t)blist[b_off + r - m_i] * MR + c;
                    *p = *p - acc[i][j];
                }
            } else {
                T* p = Z + (int64_t)(i_off + r) * MR + c;
                *p = *p + acc[i][j];
            }
        }
    }
}

// Low-rank nodes (R ~ X R(J, :), stored as X (m_i x k) then RJt = R(J, :)^T
// (m_b x k), column-major; L = R^T): one 64-row x 32-column tile of
//   MODE 0: T = X^T u(I)          (rows: k, K: m_i)
//   MODE 1: u(B) += RJt T         (rows: m_b, K: k)
//   MODE 2: T = RJt^T z(B)        (rows: k, K: m_b)
//   MODE 3: z(I) += X T           (rows: m_i, K: k)
// the same products as the one-vector apply's low-rank dot and axpy tasks;
// T: k x 32 per node (row a at a * 32) in the job's slot.  Job: node, first
// row, T offset (lo, hi).
template <typename T, int MODE>
__global__ void __launch_bounds__(MT_THREADS)
mlr_kernel(const int4* __restrict__ jobs, const int32_t* __restrict__ node, const uint64_t* __restrict__ lr_ptr,
           const int32_t* __restrict__ lr_k, const int32_t* __restrict__ blist, T* __restrict__ U, T* __restrict__ Z,
           T* __restrict__ Tb, const int* __restrict__ pact, const int32_t* __restrict__ nprob) {
    __shared__ __align__(16) T As[MT_K][MT_ROWS];
    __shared__ __align__(16) T Bs[MT_K][MR];
    const int4 J = jobs[blockIdx.x];
    const int s = J.x, r0 = J.y;
    const int64_t toff = (int64_t)(((uint64_t)(uint32_t)J.w << 32) | (uint32_t)J.z);
    if (pact && !pact[nprob[s]]) return;
    const int32_t* nd = node + (size_t)s * 14;
    const int i_off = nd[4], m_i = nd[5], b_off = nd[6], m_b = nd[7];
    const int k = lr_k[s];
    const T* X = reinterpret_cast<const T*>(lr_ptr[s]);
    const T* RJt = X + (int64_t)m_i * k;
    T* Ts = Tb + toff;
    const int rows = (MODE == 0 || MODE == 2) ? k : (MODE == 1 ? m_b : m_i);
    const int K = MODE == 0 ? m_i : (MODE == 2 ? m_b : k);
    const T* src = (MODE == 0) ? U : (MODE == 2 ? Z : Ts);
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
    // transposed operands (MODE 0, 2) are loaded along K, the others along rows
    constexpr bool kfast = MODE == 0 || MODE == 2;
    auto a_pos = [&](int q, int& r, int& kk) {
        r = kfast ? q / MT_K : q % MT_ROWS;
        kk = kfast ? q % MT_K : q / MT_ROWS;
    };
    T ra[MT_ROWS * MT_K / MT_THREADS], rb[MT_K * MR / MT_THREADS];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < MT_ROWS * MT_K / MT_THREADS; ++u) {
            int r, kk;
            a_pos(tid + MT_THREADS * u, r, kk);
            T a = zero<T>();
            if (r0 + r < rows && k0 + kk < K) {
                const int rr = r0 + r, ki = k0 + kk;
                a = MODE == 0 ? X[(int64_t)rr * m_i + ki]
                  : MODE == 1 ? RJt[(int64_t)ki * m_b + rr]
                  : MODE == 2 ? RJt[(int64_t)rr * m_b + ki]
                              : X[(int64_t)ki * m_i + rr];
            }
            ra[u] = a;
        }
#pragma unroll
        for (int u = 0; u < MT_K * MR / MT_THREADS; ++u) {
            const int q = tid + MT_THREADS * u, kk = q / MR, c = q % MR, ki = k0 + kk;
            int sr = -1;
            if (ki < K) sr = MODE == 0 ? i_off + ki : (MODE == 2 ? blist[b_off + ki] : ki);
            rb[u] = sr >= 0 ? src[(int64_t)sr * MR + c] : zero<T>();
        }
    };
    if (K > 0) load(0);
    for (int k0 = 0; k0 < K; k0 += MT_K) {
#pragma unroll
        for (int u = 0; u < MT_ROWS * MT_K / MT_THREADS; ++u) {
            int r, kk;
            a_pos(tid + MT_THREADS * u, r, kk);
            As[kk][r] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < MT_K * MR / MT_THREADS; ++u) {
            const int q = tid + MT_THREADS * u;
            Bs[q / MR][q % MR] = rb[u];
        }
        __syncthreads();
        if (k0 + MT_K < K) load(k0 + MT_K);
#pragma unroll
        for (int kk = 0; kk < MT_K; ++kk) {
            T a[4], bv[4];
            lds_vec<4>(&As[kk][4 * ty], a);
            lds_vec<4>(&Bs[kk][4 * tx], bv);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmac(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + 4 * ty + i;
        if (r >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * tx + j;
            if (MODE == 0 || MODE == 2) {
                Ts[(int64_t)r * MR + c] = acc[i][j];
            } else if (MODE == 1) {
                T* p = U + (int64_t)blist[b_off + r] * MR + c;
                *p = *p + acc[i][j];
            } else {
                T* p = Z + (int64_t)(i_off + r) * MR + c;
                *p = *p + acc[i][j];
            }
        }
    }
}

template <typename T, typename V>
ndhss_status multi_apply_run(const FactorData& F, int nrhs, const V* X, int64_t ldx, V* Y, int64_t ldy, T* U, T* Z,
                             const int* pact, const int32_t* nprob, cudaStream_t st) {
    const int64_t n = F.n;
    const int eb = (int)std::min<int64_t>((n * MR + 255) / 256, 8 * 152);
    mgather_kernel<T, V><<<eb, 256, 0, st>>>(n, nrhs, F.d_perm, X, ldx, U);
    NDHSS_LAUNCH_CHECK("mgather_kernel");
    const T* front = static_cast<const T*>(F.d_front);
    T* Tb = Z + (int64_t)F.n * MR;                  // the low-rank nodes' k x 32 blocks
    const uint64_t* lrp = F.d_mlr ? F.d_lr_ptr : nullptr;
    auto lr_launch = [&](int mode, int l) -> ndhss_status {
        if (!F.d_mlr) return NDHSS_OK;
        const int64_t a = F.ml_off[mode][l], b = F.ml_off[mode][l + 1];
        if (b == a) return NDHSS_OK;
        const int4* jb = F.d_mlr + a;
        switch (mode) {
            case 0: mlr_kernel<T, 0><<<(unsigned)(b - a), MT_THREADS, 0, st>>>(jb, F.d_node, F.d_lr_ptr, F.d_lr_k, F.d_blist, U, Z, Tb, pact, nprob); break;
            case 1: mlr_kernel<T, 1><<<(unsigned)(b - a), MT_THREADS, 0, st>>>(jb, F.d_node, F.d_lr_ptr, F.d_lr_k, F.d_blist, U, Z, Tb, pact, nprob); break;
            case 2: mlr_kernel<T, 2><<<(unsigned)(b - a), MT_THREADS, 0, st>>>(jb, F.d_node, F.d_lr_ptr, F.d_lr_k, F.d_blist, U, Z, Tb, pact, nprob); break;
            default: mlr_kernel<T, 3><<<(unsigned)(b - a), MT_THREADS, 0, st>>>(jb, F.d_node, F.d_lr_ptr, F.d_lr_k, F.d_blist, U, Z, Tb, pact, nprob); break;
        }
        NDHSS_LAUNCH_CHECK("mlr_kernel");
        return NDHSS_OK;
    };
    // the dense tiles of level l in its two tile shapes (plan: variant-major per level)
    auto dense_launch = [&](bool up, int l) -> ndhss_status {
        const std::vector<int64_t>& off = up ? F.mj_up_off : F.mj_dn_off;
        for (int v = 0; v < 2; ++v) {
            const int64_t a = off[2 * l + v], b = off[2 * l + v + 1];
            if (b == a) continue;
            const int2* jb = F.d_mjobs + a;
            if (up && v == 0)
                mapply_kernel<T, true, 32><<<(unsigned)(b - a), 64, 0, st>>>(jb, F.d_node, F.d_foff, front, F.d_sigma, F.d_blist, U, Z, pact, nprob, lrp);
            else if (up)
                mapply_kernel<T, true, 64><<<(unsigned)(b - a), 128, 0, st>>>(jb, F.d_node, F.d_foff, front, F.d_sigma, F.d_blist, U, Z, pact, nprob, lrp);
            else if (v == 0)
                mapply_kernel<T, false, 32><<<(unsigned)(b - a), 64, 0, st>>>(jb, F.d_node, F.d_foff, front, F.d_sigma, F.d_blist, U, Z, pact, nprob, lrp);
            else
                mapply_kernel<T, false, 64><<<(unsigned)(b - a), 128, 0, st>>>(jb, F.d_node, F.d_foff, front, F.d_sigma, F.d_blist, U, Z, pact, nprob, lrp);
            NDHSS_LAUNCH_CHECK("mapply_kernel");
        }
        return NDHSS_OK;
    };
    for (int l = F.depth; l >= 0; --l) {
        {
            const ndhss_status rc = dense_launch(true, l);
            if (rc != NDHSS_OK) return rc;
        }
        ndhss_status rc = lr_launch(0, l);
        if (rc == NDHSS_OK) rc = lr_launch(1, l);
        if (rc != NDHSS_OK) return rc;
    }
    for (int l = 0; l <= F.depth; ++l) {
        {
            const ndhss_status rc = dense_launch(false, l);
            if (rc != NDHSS_OK) return rc;
        }
        ndhss_status rc = lr_launch(2, l);
        if (rc == NDHSS_OK) rc = lr_launch(3, l);
        if (rc != NDHSS_OK) return rc;
    }
    mscatter_kernel<T, V><<<eb, 256, 0, st>>>(n, nrhs, F.d_perm, Z, Y, ldy);
    NDHSS_LAUNCH_CHECK("mscatter_kernel");
    return NDHSS_OK;
}

// X, Y: n x ld interleaved float64 / complex128 (per the factor's vtype);
// work: 2 n x 32 front-type elements; pact / nprob (or null): a node's
// tiles are skipped when pact[nprob[node]] == 0 (rows of a problem the
// caller no longer reads)
ndhss_status multi_apply_device(const FactorData& F, int nrhs, const void* X, int64_t ldx, void* Y, int64_t ldy,
                                void* work, cudaStream_t st, const int* pact = nullptr,
                                const int32_t* nprob = nullptr) {
    const int64_t nm = (int64_t)F.n * MR;
    const bool cplx = F.vtype == NDHSS_C128;
    if (!cplx && F.prec == NDHSS_FP64)
        return multi_apply_run<double, double>(F, nrhs, (const double*)X, ldx, (double*)Y, ldy, (double*)work,
                                               (double*)work + nm, pact, nprob, st);
    if (!cplx)
        return multi_apply_run<float, double>(F, nrhs, (const double*)X, ldx, (double*)Y, ldy, (float*)work,
                                              (float*)work + nm, pact, nprob, st);
    if (F.prec == NDHSS_FP64)
        return multi_apply_run<c128, c128>(F, nrhs, (const c128*)X, ldx, (c128*)Y, ldy, (c128*)work, (c128*)work + nm,
                                           pact, nprob, st);
    return multi_apply_run<c64, c128>(F, nrhs, (const c128*)X, ldx, (c128*)Y, ldy, (c64*)work, (c64*)work + nm, pact,
                                      nprob, st);
}

size_t multi_work_bytes(const FactorData& F) { return ((size_t)2 * F.n * MR + (size_t)F.ml_t_total) * F.esize + 256; }

ndhss_status multi_supported(const FactorData& F, const char* who) {
    if (!F.d_mjobs) return set_error(NDHSS_ERR_INVALID_ARG, "%s: the factorization has no multi-apply plan", who);
    if (F.ulv) return set_error(NDHSS_ERR_INVALID_ARG, "%s: ULV factorizations are applied one column at a time (ndhss_apply)", who);
    return NDHSS_OK;
}

// ---------------------------------------------------------- batched GMRES
struct Seg {
    int32_t s, row0, row1, pad;
};

enum : int32_t { ST_ACTIVE = 0, ST_STOPPED = 1, ST_CONVERGED = 2, ST_FAILED = 3, ST_PAD = 4 };

struct BState {
    double bnorm, zb, beta, inv, est, relres;
    double prev_rel, crtol;      // true residual of the previous cycle; this system's cycle_rtol
    double ctgt;                 // > 0 after a stagnating cycle: the cycle-relative inner target
    int32_t status, jend, its, cycles;
};

// Y(:, c) = A X(:, c) for the 32 interleaved columns of one block of rows
// per CTA: one warp per row, lane = column; blocks of a problem with
// pact[s] == 0 are skipped (pact null: every block)
template <typename V>
__global__ void __launch_bounds__(256)
spmm_kernel(const Seg* __restrict__ segs, const int* __restrict__ pact, const int32_t* __restrict__ rowptr,
            const int32_t* __restrict__ col, const V* __restrict__ vals, const V* __restrict__ X, V* __restrict__ Y) {
    const Seg sg = segs[blockIdx.x];
    if (pact && !pact[sg.s]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int row = sg.row0 + warp; row < sg.row1; row += 8) {
        V acc = zero<V>();
        for (int k = rowptr[row]; k < rowptr[row + 1]; ++k) acc = fmac(vals[k], X[(int64_t)col[k] * MR + lane], acc);
        Y[(int64_t)row * MR + lane] = acc;
    }
}

// part[blk][i][c] = sum over the block's rows of conj(V_i(row, c)) w(row, c),
// i < nvec.  Lane = column, warp = a contiguous eighth of the block's rows,
// four basis vectors per pass and four rows per iteration, so every warp has
// 4 + 16 independent 512-byte loads in flight (the float64 accumulation
// chains are too slow to wait on one load at a time).
template <typename V>
__global__ void __launch_bounds__(256, 4)
bdot_kernel(const Seg* __restrict__ segs, const int* __restrict__ pact, const V* __restrict__ Vb, int64_t ldv, int nvec,
            const V* __restrict__ w, V* __restrict__ part) {
    constexpr int NB = 4, UR = 4;
    __shared__ V red[NB][8][MR];
    const Seg sg = segs[blockIdx.x];
    if (pact && !pact[sg.s]) return;
    const int c = threadIdx.x & 31, rg = threadIdx.x >> 5;
    const int len = sg.row1 - sg.row0, per = (len + 7) / 8;
    const int r0 = sg.row0 + rg * per, r1 = min(sg.row1, r0 + per);
    for (int i0 = 0; i0 < nvec; i0 += NB) {
        const int ni = min(NB, nvec - i0);
        V acc[NB];
#pragma unroll
        for (int ii = 0; ii < NB; ++ii) acc[ii] = zero<V>();
        int row = r0;
        for (; row + UR <= r1; row += UR) {
            V wv[UR];
#pragma unroll
            for (int u = 0; u < UR; ++u) wv[u] = w[(int64_t)(row + u) * MR + c];
#pragma unroll
            for (int ii = 0; ii < NB; ++ii) {
                if (ii < ni) {
                    const V* vp = Vb + (int64_t)(i0 + ii) * ldv + (int64_t)row * MR + c;
                    V vv[UR];
#pragma unroll
                    for (int u = 0; u < UR; ++u) vv[u] = vp[(int64_t)u * MR];
#pragma unroll
                    for (int u = 0; u < UR; ++u) acc[ii] = fmac(conjv(vv[u]), wv[u], acc[ii]);
                }
            }
        }
        for (; row < r1; ++row) {
            const V wv = w[(int64_t)row * MR + c];
#pragma unroll
            for (int ii = 0; ii < NB; ++ii)
                if (ii < ni) acc[ii] = fmac(conjv(Vb[(int64_t)(i0 + ii) * ldv + (int64_t)row * MR + c]), wv, acc[ii]);
        }
#pragma unroll
        for (int ii = 0; ii < NB; ++ii) red[ii][rg][c] = acc[ii];
        __syncthreads();
        for (int q = threadIdx.x; q < ni * MR; q += blockDim.x) {
            const int ii = q / MR, cc = q % MR;
            V sum = red[ii][0][cc];
            for (int g = 1; g < 8; ++g) sum = sum + red[ii][g][cc];
            part[((int64_t)blockIdx.x * BK + i0 + ii) * MR + cc] = sum;
        }
        __syncthreads();
    }
}

// out[i][s * 32 + c] = sum of problem s's blocks (block order)
template <typename V>
__global__ void breduce_kernel(int nsys, const int32_t* __restrict__ seg_off, int nvec, const V* __restrict__ part,
                               V* __restrict__ out) {
    const int Q = nsys * MR;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q * nvec; q += gridDim.x * blockDim.x) {
        const int i = q / Q, sc = q % Q, s = sc / MR, c = sc % MR;
        V sum = zero<V>();
        for (int b = seg_off[s]; b < seg_off[s + 1]; ++b) sum = sum + part[((int64_t)b * BK + i) * MR + c];
        out[(int64_t)i * Q + sc] = sum;
    }
}

// w(row, c) += sign * sum_{i < nvec} V_i(row, c) h[i][s * 32 + c]; blocks of a
// problem with pact[s] == 0 are skipped; with bs, column c uses only its own
// system's jend basis vectors (the others may hold stale rows)
template <typename V>
__global__ void __launch_bounds__(256)
baxpy_kernel(const Seg* __restrict__ segs, const int* __restrict__ pact, int nsys, const V* __restrict__ Vb,
             int64_t ldv, int nvec, const V* __restrict__ h, double sign, V* __restrict__ w,
             const BState* __restrict__ bs) {
    __shared__ V sh[BK][MR];
    const Seg sg = segs[blockIdx.x];
    if (pact && !pact[sg.s]) return;
    const int Q = nsys * MR;
    for (int q = threadIdx.x; q < nvec * MR; q += blockDim.x) sh[q / MR][q % MR] = h[(int64_t)(q / MR) * Q + sg.s * MR + q % MR];
    __syncthreads();
    const int c = threadIdx.x & 31, rg = threadIdx.x >> 5;
    int nv = nvec;
    if (bs) {
        const BState S = bs[sg.s * MR + c];
        nv = (S.status == ST_STOPPED || S.status == ST_ACTIVE) ? min(nvec, S.jend) : 0;
    }
    for (int row = sg.row0 + rg; row < sg.row1; row += 8) {
        V acc = zero<V>();
        for (int i = 0; i < nv; ++i) acc = fmac(Vb[(int64_t)i * ldv + (int64_t)row * MR + c], sh[i][c], acc);
        V* p = w + (int64_t)row * MR + c;
        *p = *p + scale(acc, sign);
    }
}

// dst(row, c) = src(row, c) * f[s * 32 + c]
template <typename V>
__global__ void bscale_kernel(const Seg* __restrict__ segs, const int* __restrict__ pact, const BState* __restrict__ bs,
                              const V* __restrict__ src, V* __restrict__ dst) {
    const Seg sg = segs[blockIdx.x];
    if (pact && !pact[sg.s]) return;
    const int c = threadIdx.x & 31, rg = threadIdx.x >> 5;
    const double f = bs[sg.s * MR + c].inv;
    for (int row = sg.row0 + rg; row < sg.row1; row += 8) {
        const int64_t e = (int64_t)row * MR + c;
        dst[e] = scale(src[e], f);
    }
}

template <typename V>
__global__ void bsub_kernel(int64_t cnt, const V* __restrict__ a, const V* __restrict__ b, V* __restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = a[q] - b[q];
}

template <typename V>
__global__ void binterleave_kernel(int64_t n, int nrhs, const V* __restrict__ b, int64_t ldb, V* __restrict__ Bi) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * MR; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q / MR;
        const int c = (int)(q % MR);
        Bi[q] = c < nrhs ? b[(int64_t)c * ldb + row] : zero<V>();
    }
}

template <typename V>
__global__ void bdeinterleave_kernel(int64_t n, int nrhs, const V* __restrict__ Xi, V* __restrict__ x, int64_t ldx) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * nrhs; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q % n;
        const int c = (int)(q / n);
        x[(int64_t)c * ldx + row] = Xi[row * MR + c];
    }
}

// ||b_q||, padding columns and zero right-hand sides settle at once
template <typename V>
__global__ void binit_kernel(int Q, int nrhs, const V* __restrict__ nb2, double cycle_rtol, BState* __restrict__ bs) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        BState S{};
        S.bnorm = sqrt(bre(nb2[q]));
        S.zb = -1.0;
        S.prev_rel = INFINITY;
        S.crtol = cycle_rtol;
        S.status = (q % MR) >= nrhs ? ST_PAD : (S.bnorm == 0.0 ? ST_CONVERGED : ST_ACTIVE);
        bs[q] = S;
    }
}

// cycle start: the true residual decides convergence; count the systems that go on
template <typename V>
__global__ void bcheck_kernel(int Q, const V* __restrict__ nr2, double tol, int maxit, BState* __restrict__ bs,
                              int* __restrict__ count) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        BState S = bs[q];
        if (S.status == ST_ACTIVE || S.status == ST_STOPPED) {
            S.relres = sqrt(bre(nr2[q])) / S.bnorm;
            if (S.relres <= tol) S.status = ST_CONVERGED;
            else if (S.its >= maxit) S.status = ST_FAILED;
            else {
                // a cycle that did not halve the true residual: from now on a cycle ends
                // when its estimate fell by what the true residual still needs
                if (S.relres > 0.5 * S.prev_rel) {
                    S.crtol = 0.0;
                    S.ctgt = 0.1 * tol / S.relres;
                } else if (S.ctgt > 0.0) {
                    S.ctgt = 0.1 * tol / S.relres;
                }
                S.prev_rel = S.relres;
                S.status = ST_ACTIVE;
                S.cycles++;
                atomicAdd(count, 1);
            }
            S.jend = 0;
        }
        bs[q] = S;
    }
}

// beta = ||P^{-1} r||, g = beta e_1, first cycle: ||P^{-1} b|| = beta
template <typename V>
__global__ void bcycle_kernel(int Q, int ldg, const V* __restrict__ nz2, V* __restrict__ g, BState* __restrict__ bs) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        BState S = bs[q];
        S.inv = 0.0;
        if (S.status == ST_ACTIVE) {
            S.beta = sqrt(bre(nz2[q]));
            if (S.zb < 0) S.zb = S.beta;
            if (!(S.beta > 0.0) || !(S.zb > 0.0)) {
                S.status = ST_FAILED;
            } else {
                S.inv = 1.0 / S.beta;
                S.est = S.beta;
                V* gq = g + (int64_t)q * ldg;
                gq[0] = breal<V>(S.beta);
                for (int i = 1; i < ldg; ++i) gq[i] = zero<V>();
            }
        }
        bs[q] = S;
    }
}

// Hessenberg column j of every active system, its Givens rotations and the
// least-squares residual (as arnoldi_step_kernel of the one-system solver)
template <typename V>
__global__ void barnoldi_kernel(int Q, int j, int R, const V* __restrict__ h1, const V* __restrict__ h2,
                                const V* __restrict__ nw2, V* __restrict__ H, V* __restrict__ g, double* __restrict__ cs,
                                V* __restrict__ sn, BState* __restrict__ bs, double inner_tol, int maxit,
                                int* __restrict__ count) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        BState S = bs[q];
        if (S.status != ST_ACTIVE) {
            S.inv = 0.0;
            bs[q] = S;
            continue;
        }
        V* Hj = H + ((int64_t)q * R + j) * (R + 1);
        V* gq = g + (int64_t)q * (R + 1);
        double* cq = cs + (int64_t)q * R;
        V* sq = sn + (int64_t)q * R;
        for (int i = 0; i <= j; ++i) Hj[i] = h1[(int64_t)i * Q + q] + h2[(int64_t)i * Q + q];
        const double hn = sqrt(bre(nw2[q]));
        Hj[j + 1] = breal<V>(hn);
        for (int i = 0; i < j; ++i) {
            const V t0 = scale(Hj[i], cq[i]) + sq[i] * Hj[i + 1];
            const V t1 = scale(Hj[i + 1], cq[i]) - conjv(sq[i]) * Hj[i];
            Hj[i] = t0;
            Hj[i + 1] = t1;
        }
        const V a = Hj[j], b = Hj[j + 1];
        double c;
        V s;
        const double aa = babs(a), ab = babs(b);
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
        cq[j] = c;
        sq[j] = s;
        Hj[j] = scale(a, c) + s * b;
        Hj[j + 1] = zero<V>();
        const V gj = gq[j];
        gq[j + 1] = -(conjv(s) * gj);
        gq[j] = scale(gj, c);
        S.est = babs(gq[j + 1]);
        S.its++;
        S.jend = j + 1;
        S.inv = hn > 0 ? 1.0 / hn : 0.0;
        const bool inner_done = S.ctgt > 0.0 ? S.est <= S.ctgt * S.beta : S.est / S.zb <= inner_tol;
        if (inner_done || S.est <= S.crtol * S.beta || hn == 0.0 || S.its >= maxit ||
            j + 1 >= R) {
            S.status = ST_STOPPED;
            S.inv = 0.0;
        } else {
            atomicAdd(count, 1);
        }
        bs[q] = S;
    }
}

// y = H(0:jend, 0:jend)^{-1} g(0:jend) per system, zero beyond jend
template <typename V>
__global__ void bhsolve_kernel(int Q, int R, const V* __restrict__ H, const V* __restrict__ g, const BState* __restrict__ bs,
                               V* __restrict__ y) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        const BState S = bs[q];
        const int k = (S.status == ST_STOPPED || S.status == ST_ACTIVE) ? S.jend : 0;
        const V* Hq = H + (int64_t)q * R * (R + 1);
        const V* gq = g + (int64_t)q * (R + 1);
        for (int i = BK - 1; i >= k; --i) y[(int64_t)i * Q + q] = zero<V>();
        for (int i = k - 1; i >= 0; --i) {
            V acc = gq[i];
            for (int l = i + 1; l < k; ++l) acc = acc - Hq[(int64_t)l * (R + 1) + i] * y[(int64_t)l * Q + q];
            y[(int64_t)i * Q + q] = acc * recip(Hq[(int64_t)i * (R + 1) + i]);
        }
    }
}

// pact[s] = 1 when a system of problem s is still iterating in this cycle
__global__ void bpact_kernel(int nsys, const BState* __restrict__ bs, int* __restrict__ pact) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
        int a = 0;
        for (int c = 0; c < MR; ++c) a |= bs[s * MR + c].status == ST_ACTIVE ? 1 : 0;
        pact[s] = a;
    }
}

template <typename V>
ndhss_status gmres_batched_run(const FactorData& F, const int32_t* rowptr, const int32_t* col, const V* vals,
                               int nsys, const int64_t* sys_off, int nrhs, const V* b, int64_t ldb, V* x, int64_t ldx,
                               const ndhss_gmres_opts& o, ndhss_gmres_stats* stats, cudaStream_t st) {
    const int64_t n = F.n;
    const int R = o.restart;
    const int Q = nsys * MR;
    const int64_t nm = n * MR;
    std::vector<Seg> segs;
    std::vector<int32_t> seg_off(nsys + 1, 0);
    for (int s = 0; s < nsys; ++s) {
        seg_off[s] = (int32_t)segs.size();
        for (int64_t r0 = sys_off[s]; r0 < sys_off[s + 1]; r0 += SEG_ROWS)
            segs.push_back({s, (int32_t)r0, (int32_t)std::min<int64_t>(r0 + SEG_ROWS, sys_off[s + 1]), 0});
    }
    seg_off[nsys] = (int32_t)segs.size();
    const int nseg = (int)segs.size();
    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o2 = off; off += (bytes + 255) / 256 * 256; return o2; };
    const size_t o_seg = take(sizeof(Seg) * std::max(nseg, 1)), o_soff = take(sizeof(int32_t) * (nsys + 1));
    const size_t o_B = take(sizeof(V) * nm), o_X = take(sizeof(V) * nm), o_w = take(sizeof(V) * nm),
                 o_t = take(sizeof(V) * nm), o_V = take(sizeof(V) * nm * (R + 1));
    const size_t o_part = take(sizeof(V) * (size_t)std::max(nseg, 1) * BK * MR);
    const size_t o_h1 = take(sizeof(V) * (size_t)BK * Q), o_h2 = take(sizeof(V) * (size_t)BK * Q),
                 o_y = take(sizeof(V) * (size_t)BK * Q), o_n2 = take(sizeof(V) * (size_t)Q);
    const size_t o_H = take(sizeof(V) * (size_t)Q * R * (R + 1)), o_g = take(sizeof(V) * (size_t)Q * (R + 1)),
                 o_cs = take(sizeof(double) * (size_t)Q * R), o_sn = take(sizeof(V) * (size_t)Q * R);
    const size_t o_bs = take(sizeof(BState) * Q), o_cnt = take(sizeof(int) * 4);
    const size_t o_pact = take(sizeof(int) * nsys), o_nprob = take(sizeof(int32_t) * std::max(F.nnodes, 1));
    const size_t o_mw = take(multi_work_bytes(F));
    void* work = nullptr;
    NDHSS_CUDA_TRY(pool_malloc_async(&work, off, st));
    unsigned char* W = static_cast<unsigned char*>(work);
    Seg* d_seg = (Seg*)(W + o_seg);
    int32_t* d_soff = (int32_t*)(W + o_soff);
    V *Bi = (V*)(W + o_B), *Xi = (V*)(W + o_X), *w = (V*)(W + o_w), *t = (V*)(W + o_t), *Vb = (V*)(W + o_V);
    V *part = (V*)(W + o_part), *h1 = (V*)(W + o_h1), *h2 = (V*)(W + o_h2), *yv = (V*)(W + o_y), *n2 = (V*)(W + o_n2);
    V *H = (V*)(W + o_H), *g = (V*)(W + o_g), *sn = (V*)(W + o_sn);
    double* cs = (double*)(W + o_cs);
    BState* bs = (BState*)(W + o_bs);
    int* cnt = (int*)(W + o_cnt);
    int* pact = (int*)(W + o_pact);
    int32_t* nprob = (int32_t*)(W + o_nprob);
    void* mw = W + o_mw;
    int napply = 0, nspmv = 0;
    std::vector<BState> hb(Q);
    // everything that uses the workspace; any early return comes back here and
    // the workspace goes back to the pool below
    auto body = [&]() -> ndhss_status {
    ndhss_status rc = NDHSS_OK;
    if (nseg > 0) NDHSS_CUDA_TRY(cudaMemcpyAsync(d_seg, segs.data(), sizeof(Seg) * nseg, cudaMemcpyHostToDevice, st));
    NDHSS_CUDA_TRY(cudaMemcpyAsync(d_soff, seg_off.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, st));
    // each node's problem: the one whose rows hold the node's I block
    std::vector<int32_t> hprob(std::max(F.nnodes, 1), 0);
    for (int v = 0; v < F.nnodes; ++v) {
        const int64_t io = F.info(v, 4);
        hprob[v] = (int32_t)(std::upper_bound(sys_off, sys_off + nsys + 1, io) - sys_off - 1);
        hprob[v] = std::min(std::max(hprob[v], 0), nsys - 1);
    }
    NDHSS_CUDA_TRY(cudaMemcpyAsync(nprob, hprob.data(), sizeof(int32_t) * hprob.size(), cudaMemcpyHostToDevice, st));
    NDHSS_CUDA_TRY(cudaStreamSynchronize(st));
    NDHSS_CUDA_TRY(cudaMemsetAsync(Xi, 0, sizeof(V) * nm, st));
    const int eb = (int)std::min<int64_t>((nm + 255) / 256, 8 * 152);
    const int qb = (Q + 255) / 256;
    binterleave_kernel<V><<<eb, 256, 0, st>>>(n, nrhs, b, ldb, Bi);
    NDHSS_LAUNCH_CHECK("binterleave_kernel");
    auto dots = [&](const V* basis, int nvec, const V* vec, V* out, const int* mask) {
        bdot_kernel<V><<<nseg, 256, 0, st>>>(d_seg, mask, basis, nm, nvec, vec, part);
        breduce_kernel<V><<<(Q * nvec + 255) / 256, 256, 0, st>>>(nsys, d_soff, nvec, part, out);
    };
    auto read_count = [&](int* h) -> ndhss_status {
        NDHSS_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        NDHSS_CUDA_TRY(cudaStreamSynchronize(st));
        return NDHSS_OK;
    };
    const int pb = (nsys + 255) / 256;
    dots(Bi, 1, Bi, n2, nullptr);
    binit_kernel<V><<<qb, 256, 0, st>>>(Q, nrhs, n2, o.cycle_rtol, bs);
    NDHSS_LAUNCH_CHECK("binit_kernel");
    while (true) {
        spmm_kernel<V><<<nseg, 256, 0, st>>>(d_seg, nullptr, rowptr, col, vals, Xi, t);
        ++nspmv;
        bsub_kernel<V><<<eb, 256, 0, st>>>(nm, Bi, t, w);
        dots(w, 1, w, n2, nullptr);
        NDHSS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int), st));
        bcheck_kernel<V><<<qb, 256, 0, st>>>(Q, n2, o.tol, o.maxit, bs, cnt);
        NDHSS_LAUNCH_CHECK("bcheck_kernel");
        int active = 0;
        if ((rc = read_count(&active))) return rc;
        if (active == 0) break;
        bpact_kernel<<<pb, 256, 0, st>>>(nsys, bs, pact);
        if ((rc = multi_apply_device(F, MR, w, MR, t, MR, mw, st, pact, nprob))) return rc;
        ++napply;
        dots(t, 1, t, n2, pact);
        bcycle_kernel<V><<<qb, 256, 0, st>>>(Q, R + 1, n2, g, bs);
        bscale_kernel<V><<<nseg, 256, 0, st>>>(d_seg, pact, bs, t, Vb);
        NDHSS_LAUNCH_CHECK("bscale_kernel");
        int jend = 0;
        for (int j = 0; j < R; ++j) {
            bpact_kernel<<<pb, 256, 0, st>>>(nsys, bs, pact);
            spmm_kernel<V><<<nseg, 256, 0, st>>>(d_seg, pact, rowptr, col, vals, Vb + (int64_t)j * nm, w);
            ++nspmv;
            if ((rc = multi_apply_device(F, MR, w, MR, t, MR, mw, st, pact, nprob))) return rc;
            ++napply;
            dots(Vb, j + 1, t, h1, pact);
            baxpy_kernel<V><<<nseg, 256, 0, st>>>(d_seg, pact, nsys, Vb, nm, j + 1, h1, -1.0, t, nullptr);
            dots(Vb, j + 1, t, h2, pact);
            baxpy_kernel<V><<<nseg, 256, 0, st>>>(d_seg, pact, nsys, Vb, nm, j + 1, h2, -1.0, t, nullptr);
            dots(t, 1, t, n2, pact);
            NDHSS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int), st));
            barnoldi_kernel<V><<<qb, 256, 0, st>>>(Q, j, R, h1, h2, n2, H, g, cs, sn, bs, o.inner * o.tol, o.maxit, cnt);
            bscale_kernel<V><<<nseg, 256, 0, st>>>(d_seg, pact, bs, t, Vb + (int64_t)(j + 1) * nm);
            NDHSS_LAUNCH_CHECK("barnoldi_kernel");
            jend = j + 1;
            if ((rc = read_count(&active))) return rc;
            if (active == 0) break;
        }
        bhsolve_kernel<V><<<qb, 256, 0, st>>>(Q, R, H, g, bs, yv);
        baxpy_kernel<V><<<nseg, 256, 0, st>>>(d_seg, nullptr, nsys, Vb, nm, jend, yv, 1.0, Xi, bs);
        NDHSS_LAUNCH_CHECK("baxpy_kernel");
    }
    bdeinterleave_kernel<V><<<eb, 256, 0, st>>>(n, nrhs, Xi, x, ldx);
    NDHSS_LAUNCH_CHECK("bdeinterleave_kernel");
    NDHSS_CUDA_TRY(cudaMemcpyAsync(hb.data(), bs, sizeof(BState) * Q, cudaMemcpyDeviceToHost, st));
    NDHSS_CUDA_TRY(cudaStreamSynchronize(st));
    return NDHSS_OK;
    };
    const ndhss_status rb = body();
    cudaFreeAsync(work, st);
    if (rb != NDHSS_OK) return rb;
    bool all = true;
    for (int s = 0; s < nsys; ++s)
        for (int c = 0; c < nrhs; ++c) {
            const BState& S = hb[s * MR + c];
            ndhss_gmres_stats Z{};
            Z.iters = S.its;
            Z.cycles = S.cycles;
            Z.converged = S.status == ST_CONVERGED ? 1 : 0;
            Z.true_relres = S.relres;
            Z.precond_relres = S.zb > 0 ? S.est / S.zb : 0.0;
            Z.napply = napply;
            Z.nspmv = nspmv;
            if (stats) stats[(int64_t)s * nrhs + c] = Z;
            all = all && Z.converged;
        }
    if (!all) return set_error(NDHSS_ERR_NOT_CONVERGED, "ndhss_gmres_batched: tolerance not reached within maxit");
    return NDHSS_OK;
}

}  // namespace

// The tile-rows table (32 or 64 per front-size bucket): the autotuned one,
// or NDHSS_MAPPLY_TILES ("r0,r1,r2,r3"), read at every plan
static void mapply_tile_table(int (&table)[MAPPLY_NBUCKET]) {
    for (int q = 0; q < MAPPLY_NBUCKET; ++q) table[q] = MAPPLY_TILE_ROWS[q];
    if (const char* e = std::getenv("NDHSS_MAPPLY_TILES")) {
        int q = 0;
        for (const char* c = e; *c && q < MAPPLY_NBUCKET; ++q) {
            const int v = std::atoi(c);
            if (v == 32 || v == 64) table[q] = v;
            while (*c && *c != ',') ++c;
            if (*c == ',') ++c;
        }
    }
}

// The multi-apply plan: per level and tile shape the (node, first row) of
// every tile of the up-sweep (all m rows of the first m_i columns; a
// low-rank node's m_i) and of the down-sweep (the m_i rows of R), one device
// array; offsets at [2 level + shape], shape 0: 32 rows, 1: 64 rows.
ndhss_status build_multi_plan(FactorData& F, cudaStream_t st) {
    std::vector<int32_t> jobs;
    int table[MAPPLY_NBUCKET];
    mapply_tile_table(table);
    auto mapply_tile_rows = [&](int rows) {
        int q = 0;
        while (q < MAPPLY_NBUCKET - 1 && rows >= MAPPLY_BUCKET_EDGES[q]) ++q;
        return table[q];
    };
    F.mj_up_off.assign(2 * (F.depth + 1) + 1, 0);
    F.mj_dn_off.assign(2 * (F.depth + 1) + 1, 0);
    auto lowrank = [&](int s) { return !F.lr_ptr.empty() && F.lr_ptr[s] != 0; };
    for (int l = 0; l <= F.depth; ++l)
        for (int v = 0; v < 2; ++v) {
            F.mj_up_off[2 * l + v] = (int64_t)jobs.size() / 2;
            for (int s : F.levels[l]) {
                const int mi = F.m_i(s), m = lowrank(s) ? mi : mi + F.m_b(s);
                if (mi == 0) continue;
                const int tr = mapply_tile_rows(m);
                if ((tr == 32) != (v == 0)) continue;
                for (int r0 = 0; r0 < m; r0 += tr) { jobs.push_back(s); jobs.push_back(r0); }
            }
        }
    F.mj_up_off[2 * (F.depth + 1)] = (int64_t)jobs.size() / 2;
    for (int l = 0; l <= F.depth; ++l)
        for (int v = 0; v < 2; ++v) {
            F.mj_dn_off[2 * l + v] = (int64_t)jobs.size() / 2;
            for (int s : F.levels[l]) {
                const int mi = F.m_i(s);
                if (mi == 0 || F.m_b(s) == 0 || lowrank(s)) continue;
                const int tr = mapply_tile_rows(mi);
                if ((tr == 32) != (v == 0)) continue;
                for (int r0 = 0; r0 < mi; r0 += tr) { jobs.push_back(s); jobs.push_back(r0); }
            }
        }
    F.mj_dn_off[2 * (F.depth + 1)] = (int64_t)jobs.size() / 2;
    // low-rank tiles: T = X^T u(I), u(B) += RJt T, T = RJt^T z(B), z(I) += X T
    std::vector<int32_t> lj;
    std::vector<int64_t> toff(std::max(F.nnodes, 1), 0);
    F.ml_t_total = 0;
    for (int s = 0; s < F.nnodes; ++s)
        if (lowrank(s) && F.lr_k[s] > 0) {
            toff[s] = F.ml_t_total;
            F.ml_t_total += (int64_t)F.lr_k[s] * MR;
        }
    for (int mode = 0; mode < 4; ++mode) {
        F.ml_off[mode].assign(F.depth + 2, 0);
        for (int l = 0; l <= F.depth; ++l) {
            F.ml_off[mode][l] = (int64_t)lj.size() / 4;
            for (int s : F.levels[l]) {
                if (!lowrank(s) || F.lr_k[s] == 0 || F.m_i(s) == 0 || F.m_b(s) == 0) continue;
                const int rows = (mode == 0 || mode == 2) ? F.lr_k[s] : (mode == 1 ? F.m_b(s) : F.m_i(s));
                for (int r0 = 0; r0 < rows; r0 += MT_ROWS) {
                    lj.push_back(s);
                    lj.push_back(r0);
                    lj.push_back((int32_t)(uint32_t)(uint64_t)toff[s]);
                    lj.push_back((int32_t)(uint32_t)((uint64_t)toff[s] >> 32));
                }
            }
        }
        F.ml_off[mode][F.depth + 1] = (int64_t)lj.size() / 4;
    }
    if (!lj.empty()) {
        void* q = nullptr;
        NDHSS_CUDA_TRY(pool_malloc_async(&q, lj.size() * sizeof(int32_t), st));
        NDHSS_CUDA_TRY(cudaMemcpyAsync(q, lj.data(), lj.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        F.d_mlr = static_cast<int4*>(q);
        F.dev_bytes += (int64_t)(lj.size() * sizeof(int32_t));
    }
    if (jobs.empty()) jobs.assign(2, 0);
    void* p = nullptr;
    NDHSS_CUDA_TRY(pool_malloc_async(&p, jobs.size() * sizeof(int32_t), st));
    NDHSS_CUDA_TRY(cudaMemcpyAsync(p, jobs.data(), jobs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NDHSS_CUDA_TRY(cudaStreamSynchronize(st));
    F.d_mjobs = static_cast<int2*>(p);
    F.dev_bytes += (int64_t)(jobs.size() * sizeof(int32_t));
    return NDHSS_OK;
}

}  // namespace ndhss

extern "C" {

ndhss_status ndhss_apply_multi(const ndhss_factorization* fh, int32_t nrhs, const void* d_x, int64_t ldx, void* d_y,
                               int64_t ldy, void* stream) {
    return ::ndhss::guarded("ndhss_apply_multi", [&]() -> ndhss_status {
        using namespace ndhss;
        clear_error();
        if (!fh || !d_x || !d_y || nrhs < 0 || nrhs > MR || ldx < nrhs || ldy < nrhs)
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply_multi: bad argument (need 0 <= nrhs <= 32 <= ld)");
        const FactorData& F = fh->f;
        if (nrhs == 0 || F.n == 0) return NDHSS_OK;
        if (!is_device_ptr(d_x) || !is_device_ptr(d_y))
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply_multi: x and y must be device pointers");
        ndhss_status rc = multi_supported(F, "ndhss_apply_multi");
        if (rc != NDHSS_OK) return rc;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        void* work = nullptr;
        NDHSS_CUDA_TRY(pool_malloc_async(&work, multi_work_bytes(F), st));
        rc = multi_apply_device(F, nrhs, d_x, ldx, d_y, ldy, work, st);
        cudaFreeAsync(work, st);
        if (rc == NDHSS_OK && cudaStreamSynchronize(st) != cudaSuccess)
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_apply_multi: %s", cudaGetErrorString(cudaGetLastError()));
        return rc;
    });
}

ndhss_status ndhss_gmres_batched(const ndhss_factorization* fh, const int32_t* d_rowptr, const int32_t* d_col,
                                 const void* d_vals, int32_t nsys, const int64_t* sys_off, int32_t nrhs, const void* d_b,
                                 int64_t ldb, void* d_x, int64_t ldx, const ndhss_gmres_opts* opts,
                                 ndhss_gmres_stats* stats, void* stream) {
    return ::ndhss::guarded("ndhss_gmres_batched", [&]() -> ndhss_status {
        using namespace ndhss;
        clear_error();
        if (!fh || !d_rowptr || !d_col || !d_vals || !sys_off || !d_b || !d_x || nsys < 1 || nrhs < 0 || nrhs > MR)
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres_batched: bad argument (need nsys >= 1, 0 <= nrhs <= 32)");
        const FactorData& F = fh->f;
        if (ldb < F.n || ldx < F.n) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres_batched: leading dimension < n");
        if (sys_off[0] != 0 || sys_off[nsys] != F.n)
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres_batched: sys_off must run from 0 to n");
        for (int s = 0; s < nsys; ++s)
            if (sys_off[s + 1] < sys_off[s]) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres_batched: sys_off decreases");
        if (!is_device_ptr(d_b) || !is_device_ptr(d_x))
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres_batched: b and x must be device pointers");
        ndhss_gmres_opts o{30, 300, 1e-8, 0, 0, 0.1, -1.0};
        if (opts) o = *opts;
        if (o.restart < 1 || o.restart > BK - 1 || o.maxit < 0 || !(o.tol >= 0) || !(o.inner > 0 && o.inner <= 1))
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres_batched: need 1 <= restart <= %d, maxit >= 0, tol >= 0, 0 < inner <= 1",
                             BK - 1);
        if (o.conj_transpose != 0)
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_gmres_batched: conj_transpose is not supported (use ndhss_gmres)");
        if (nrhs == 0) return NDHSS_OK;
        ndhss_status rc = multi_supported(F, "ndhss_gmres_batched");
        if (rc != NDHSS_OK) return rc;
        if (o.cycle_rtol < 0) o.cycle_rtol = (F.prec == NDHSS_FP64) ? 0.0 : 1e-3;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (F.vtype == NDHSS_R64)
            rc = gmres_batched_run<double>(F, d_rowptr, d_col, (const double*)d_vals, nsys, sys_off, nrhs, (const double*)d_b,
                                           ldb, (double*)d_x, ldx, o, stats, st);
        else
            rc = gmres_batched_run<c128>(F, d_rowptr, d_col, (const c128*)d_vals, nsys, sys_off, nrhs, (const c128*)d_b, ldb,
                                         (c128*)d_x, ldx, o, stats, st);
        if (rc == NDHSS_OK || rc == NDHSS_ERR_NOT_CONVERGED) {
            const ndhss_status r2 = apply_check_error(F, "ndhss_gmres_batched");
            if (r2 != NDHSS_OK) rc = r2;
        }
        return rc;
    });
}

}  // extern "C"
