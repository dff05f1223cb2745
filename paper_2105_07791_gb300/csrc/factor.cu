// Front factorization (Sec. 3.1, Eq. 3.2 - 3.5; Alg. 3.4 below the
// switching level), level by level from the leaves up.
//
// Every level is one batch: all its fronts are assembled by the extend-add
// of the children's Schur complements plus the sparse cross blocks of A
// (Eq. 3.4), then their first m_i unknowns are eliminated by a blocked,
// in-place Gauss-Jordan sweep with partial pivoting inside A_ii.  After the
// sweep a front holds A_ii^{-1} (column-permuted), R = -A_ii^{-1} A_ib,
// -L (column-permuted) and S = A_bb - A_bi A_ii^{-1} A_ib, which is what the
// apply (Alg. 3.1) and the parent's assembly read.
//
// One pivot block of width kb costs three launches per level:
//   panel_factor  one CTA per front: LU with partial pivoting of the
//                 candidate rows [k0, m_i) of the kb panel columns, held in
//                 shared memory; emits the row interchanges and
//                 Ainv = (A_PP)^{-1}                       (kb x kb)
//   panel_prep    applies the interchanges to every column, packs the
//                 column panel C (pivot rows replaced by identity rows) and
//                 Z = [Ainv | -Ainv * M(P, others)]
//   gemm_update   M = beta .* M + C * Z, beta = 0 on pivot rows / columns,
//                 i.e. the rank-kb Gauss-Jordan update of the whole front.
#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <deque>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>

#include "factor.cuh"

namespace ndhss {
namespace {

constexpr int KBMAX = 32;
constexpr int PANEL_THREADS = 512;
constexpr int PREP_WARPS = 8;
constexpr int GT = 64;          // gemm tile
constexpr int MAX_GRID_YZ = 65535;   // largest grid y or z dimension
constexpr int GK = 16;          // gemm k chunk
constexpr size_t PANEL_SMEM_MAX = 220 * 1024;      // panel values + one int per candidate row

__device__ __forceinline__ int nf(const int32_t* node, int s, int f) { return node[s * NODE_NF + f]; }

template <typename T> __device__ __forceinline__ T shfl_idx(T v, int src);
template <> __device__ __forceinline__ double shfl_idx<double>(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <> __device__ __forceinline__ float shfl_idx<float>(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <> __device__ __forceinline__ c128 shfl_idx<c128>(c128 v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}
template <> __device__ __forceinline__ c64 shfl_idx<c64>(c64 v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// ---------------------------------------------------------------- assembly
// F = blockdiag(S^mu, S^nu) scattered to the parent order of Eq. 3.4 (zero
// where the row and column come from different children).  fsrc[pos] =
// (child << 30) | row of that child's S.
template <typename T>
__global__ void assemble_kernel(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                                const int64_t* __restrict__ foff, const int32_t* __restrict__ fsrc,
                                const int64_t* __restrict__ poff, T* __restrict__ front) {
    const int s = lev[blockIdx.y];
    const int64_t m = nf(node, s, 5) + nf(node, s, 7);
    T* F = front + foff[s];
    const int c0 = nf(node, s, 2);
    if (c0 < 0) {
        for (int64_t c = blockIdx.x; c < m; c += gridDim.x)
            for (int64_t r = threadIdx.x; r < m; r += blockDim.x) F[c * m + r] = zero<T>();
        return;
    }
    const int ch[2] = {c0, nf(node, s, 3)};
    const T* CF[2];
    int64_t cm[2], cmi[2];
    for (int w = 0; w < 2; ++w) {
        cmi[w] = nf(node, ch[w], 5);
        cm[w] = cmi[w] + nf(node, ch[w], 7);
        CF[w] = front + foff[ch[w]];
    }
    const int32_t* src = fsrc + poff[s];
    for (int64_t c = blockIdx.x; c < m; c += gridDim.x) {
        const int sc = src[c];
        const int wc = sc >> 30;
        const int64_t lc = sc & 0x3fffffff;
        const T* colS = CF[wc] + (cmi[wc] + lc) * cm[wc] + cmi[wc];
        for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
            const int sr = src[r];
            T v = zero<T>();
            if ((sr >> 30) == wc) v = colS[sr & 0x3fffffff];
            F[c * m + r] = v;
        }
    }
}

// Sparse entries of A that enter this front (Eq. 3.2 for leaves, the A~
// blocks of Eq. 3.4 otherwise); each front position receives at most one.
template <typename T, typename V>
__global__ void scatter_entries_kernel(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                                       const int64_t* __restrict__ foff, const int32_t* __restrict__ e_off,
                                       const int32_t* __restrict__ e_row, const int32_t* __restrict__ e_col,
                                       const int32_t* __restrict__ e_idx, const V* __restrict__ vals,
                                       T* __restrict__ front) {
    const int s = lev[blockIdx.x];
    const int64_t m = nf(node, s, 5) + nf(node, s, 7);
    T* F = front + foff[s];
    for (int e = e_off[s] + threadIdx.x; e < e_off[s + 1]; e += blockDim.x)
        F[(int64_t)e_col[e] * m + e_row[e]] += from_val<T>(vals[e_idx[e]]);
}

// -0 in every component: the exact additive identity (x + -0 = x, also for x = +0)
template <typename T> __device__ __forceinline__ T neg_zero();
template <> __device__ __forceinline__ float neg_zero<float>() { return -0.0f; }
template <> __device__ __forceinline__ double neg_zero<double>() { return -0.0; }
template <> __device__ __forceinline__ c64 neg_zero<c64>() { return {-0.0f, -0.0f}; }

// r = v when i == j, by a predicated move: a plain select on a runtime
// column index lets the compiler turn the row's registers into a
// local-memory array with an indexed load
__device__ __forceinline__ void take_if(int j, int i, float v, float& r) {
    asm("{\n\t.reg .pred q;\n\tsetp.eq.s32 q, %1, %2;\n\t@q mov.f32 %0, %3;\n\t}" : "+f"(r) : "r"(i), "r"(j), "f"(v));
}
__device__ __forceinline__ void take_if(int j, int i, double v, double& r) {
    asm("{\n\t.reg .pred q;\n\tsetp.eq.s32 q, %1, %2;\n\t@q mov.f64 %0, %3;\n\t}" : "+d"(r) : "r"(i), "r"(j), "d"(v));
}
__device__ __forceinline__ void take_if(int j, int i, c64 v, c64& r) {
    asm("{\n\t.reg .pred q;\n\tsetp.eq.s32 q, %2, %3;\n\t@q mov.f32 %0, %4;\n\t@q mov.f32 %1, %5;\n\t}"
        : "+f"(r.x), "+f"(r.y) : "r"(i), "r"(j), "f"(v.x), "f"(v.y));
}

// ---------------------------------------------------------------- panel
// One CTA per front.  The candidate rows [k0, m_i) of the kb panel columns
// are swept in shared memory with the in-place Gauss-Jordan exchange step
// and partial pivoting; below each pivot this is exactly the LU elimination,
// so the interchanges are those of row-pivoted LU, and afterwards the top
// kb x kb block holds (A_PP)^{-1} of the interchanged pivot block.  The pivot
// search of the next column rides on the update of the current one, so a
// pivot costs two barriers.  Outputs per front: the interchanges (ipiv), the
// net row map they induce (<= 2 kb rows) and Ainv.
template <typename T, int KB>
__global__ void __launch_bounds__(PANEL_THREADS)
panel_factor_kernel(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                    const int64_t* __restrict__ foff, const T* __restrict__ front, int32_t* __restrict__ ipiv,
                    T* __restrict__ ainv_buf, int32_t* __restrict__ swapmap, int k0, int kb, DevStatus* status) {
    using real = typename Tr<T>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_piv[KBMAX];
    __shared__ real s_val[32];
    __shared__ int s_idx[32];
    __shared__ T s_prow[KBMAX];
    __shared__ int s_na;
    for (int j = threadIdx.x; j < KBMAX; j += blockDim.x) s_prow[j] = zero<T>();
    const int s = lev[blockIdx.x];
    const int m_i = nf(node, s, 5);
    if (k0 >= m_i) return;
    const int64_t m = m_i + nf(node, s, 7);
    const int kbp = min(kb, m_i - k0);
    const int mc = m_i - k0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    T* P = reinterpret_cast<T*>(smem_raw);                       // mc x kbp, ld mc
    int* idx = reinterpret_cast<int*>(P + (size_t)mc * kbp);     // row arrangement, mc
    const T* F = front + foff[s];
    {
        // eight loads in flight per thread (a panel of the root front is ~200 KB:
        // one load-store pair at a time waits out the memory latency ~50 times)
        constexpr int LB = 8;
        const int tot = mc * kbp;
        for (int q0 = tid; q0 < tot; q0 += LB * blockDim.x) {
            T tmp[LB];
#pragma unroll
            for (int u = 0; u < LB; ++u) {
                const int q = q0 + u * blockDim.x;
                if (q < tot) tmp[u] = F[(int64_t)(k0 + q / mc) * m + k0 + q % mc];
            }
#pragma unroll
            for (int u = 0; u < LB; ++u) {
                const int q = q0 + u * blockDim.x;
                if (q < tot) P[q] = tmp[u];
            }
        }
    }
    for (int r = tid; r < mc; r += blockDim.x) idx[r] = r;
    if (tid == 0) s_na = 0;
    __syncthreads();
    // pivot search of column 0
    {
        real best = real(-1);
        int bi = INT_MAX;
        for (int r = tid; r < mc; r += blockDim.x) {
            const real v = abs1(P[r]);
            if (v > best) { best = v; bi = r; }
        }
        for (int off = 16; off; off >>= 1) {
            const real ov = __shfl_down_sync(0xffffffffu, best, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
    }
    __syncthreads();
    for (int c = 0; c < kbp; ++c) {
        if (warp == 0) {
            // finish the search, interchange rows c and p, form the new pivot row
            real best = lane < nwarps ? s_val[lane] : real(-1);
            int bi = lane < nwarps ? s_idx[lane] : INT_MAX;
            for (int off = 16; off; off >>= 1) {
                const real ov = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            int p = __shfl_sync(0xffffffffu, bi, 0);
            if (p == INT_MAX) p = c;                              // all-NaN column: keep the diagonal
            T piv = P[c * mc + p];
            if (!(abs1(piv) > real(0))) {                         // exact zero (or NaN) pivot
                piv = one<T>();
                if (lane == 0 && atomicCAS(&status->code, 0, (int)NDHSS_ERR_SINGULAR) == 0) status->node = s;
            }
            const T pinv = recip(piv);
            __syncwarp();
            if (lane < kbp) {
                const T a = P[lane * mc + c];
                const T b = P[lane * mc + p];
                P[lane * mc + c] = b;
                if (p != c) P[lane * mc + p] = a;
                s_prow[lane] = (lane == c) ? pinv : -(b * pinv);
            }
            if (lane == 0) {
                s_piv[c] = p;
                const int t = idx[c];
                idx[c] = idx[p];
                idx[p] = t;
            }
        }
        __syncthreads();
        // exchange step on every candidate row (one panel row in registers per
        // step, all loads issued before the independent updates); search of
        // column c + 1 on the fly
        real best = real(-1);
        int bi = INT_MAX;
        const bool next = c + 1 < kbp;
        const T* pr = s_prow;            // pivot row, read as a shared-memory broadcast
        for (int r = tid; r < mc; r += blockDim.x) {
            if (r == c) {
#pragma unroll
                for (int j = 0; j < KB; ++j)
                    if (j < kbp) P[j * mc + r] = pr[j];
                continue;
            }
            T v[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) v[j] = (j < kbp) ? P[j * mc + r] : zero<T>();
            const T a = P[c * mc + r];
            real nv = real(-1);
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                v[j] = (j == c) ? a * pr[j] : fmac(a, pr[j], v[j]);
                if (j == c + 1) nv = abs1(v[j]);
            }
#pragma unroll
            for (int j = 0; j < KB; ++j)
                if (j < kbp) P[j * mc + r] = v[j];
            if (next && r > c && nv > best) { best = nv; bi = r; }
        }
        if (next) {
            for (int off = 16; off; off >>= 1) {
                const real ov = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
        }
        __syncthreads();
    }
    const int i_off = nf(node, s, 4);
    if (tid < kbp) ipiv[i_off + k0 + tid] = k0 + s_piv[tid];
    T* Ai = ainv_buf + (size_t)blockIdx.x * KBMAX * KBMAX;
    for (int q = tid; q < kbp * kbp; q += blockDim.x) {
        const int i = q % kbp, j = q / kbp;
        Ai[j * KBMAX + i] = P[j * mc + i];
    }
    // net row map of the interchanges: row k0 + r receives the old row k0 + idx[r]
    int32_t* sm = swapmap + (size_t)blockIdx.x * (4 * KBMAX + 1);
    for (int r = tid; r < mc; r += blockDim.x) {
        if (idx[r] != r) {
            const int a = atomicAdd(&s_na, 1);
            sm[1 + a] = k0 + r;
            sm[1 + 2 * KBMAX + a] = k0 + idx[r];
        }
    }
    __syncthreads();
    if (tid == 0) sm[0] = s_na;
}

// The warp's best pivot candidate (largest key, then lowest position): its
// key and position to key / pos (lane 0), its row to cand (the winning lane).
template <typename T, int KB>
__device__ __forceinline__ void panel_publish(const T (&v)[KB], typename Tr<T>::real val, bool cand, int pos, T* cand_row,
                                              typename PivKey<typename Tr<T>::real>::K* key_out, int* pos_out, int lane) {
    using PK = PivKey<typename Tr<T>::real>;
    using K = typename PK::K;
    const K key = cand ? PK::of(val) : K(0);
    const K kmax = PK::wmax(key);
    const unsigned pmin = __reduce_min_sync(0xffffffffu, (kmax != K(0) && key == kmax) ? (unsigned)pos : 0xffffffffu);
    if (kmax != K(0) && (unsigned)pos == pmin) {
#pragma unroll
        for (int j = 0; j < KB; ++j) cand_row[j] = v[j];
    }
    if (lane == 0) {
        *key_out = kmax;
        *pos_out = (int)pmin;
    }
}

// The panel of panel_factor_kernel with every candidate row in the
// registers of one thread (fronts with at most MAXT candidate rows, elements
// of at most 8 bytes).  Rows are never moved: each thread tracks the
// position its row would hold after the interchanges, so pivots, ties
// (lowest position first) and the exchange arithmetic are those of the
// shared-memory kernel: real outputs are bit for bit the same, complex ones
// up to how the compiler contracts the complex products.  A pivot costs one barrier:
// at the end of a step every warp publishes its best candidate for the next
// column together with that row's values (double-buffered by step parity);
// after the barrier every warp picks the winner and forms the pivot row
// itself (lane j: entry j), then each thread updates its own row.
template <typename T, int KB, int MAXT>
__global__ void __launch_bounds__(MAXT)
panel_reg_kernel(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                 const int64_t* __restrict__ foff, const T* __restrict__ front, int32_t* __restrict__ ipiv,
                 T* __restrict__ ainv_buf, int32_t* __restrict__ swapmap, int k0, int kb, DevStatus* status) {
    using real = typename Tr<T>::real;
    using PK = PivKey<real>;
    using K = typename PK::K;
    constexpr int NW = MAXT / 32;
    static_assert(KB <= 32 && NW <= 32, "one lane per pivot-row entry and per warp");
    __shared__ T s_cand[2][NW][KB];          // each warp's best candidate row
    __shared__ K s_key[2][NW];
    __shared__ int s_pos[2][NW];
    __shared__ T s_pr[NW][KB];               // the pivot row, formed by each warp for itself
    __shared__ int s_na;
    const int s = lev[blockIdx.x];
    const int m_i = nf(node, s, 5);
    if (k0 >= m_i) return;
    const int64_t m = m_i + nf(node, s, 7);
    const int kbp = min(kb, m_i - k0);
    const int mc = m_i - k0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const bool has = tid < mc;
    const T* F = front + foff[s];
    T v[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) v[j] = (has && j < kbp) ? F[(int64_t)(k0 + j) * m + k0 + tid] : zero<T>();
    int pos = tid;                           // this row's position after the interchanges so far
    if (tid == 0) s_na = 0;
    panel_publish<T, KB>(v, abs1(v[0]), has, pos, s_cand[0][warp], &s_key[0][warp], &s_pos[0][warp], lane);
    __syncthreads();
    int32_t* ip = ipiv + nf(node, s, 4) + k0;
    T a = v[0];                              // this row's entry in the pivot column
    for (int c = 0; c < kbp; ++c) {
        const int par = c & 1;
        const K kw = lane < nwarps ? s_key[par][lane] : K(0);
        const K kmax = PK::wmax(kw);
        const unsigned pw = __reduce_min_sync(
            0xffffffffu, (lane < nwarps && kmax != K(0) && kw == kmax) ? ((unsigned)s_pos[par][lane] << 5) | (unsigned)lane
                                                                        : 0xffffffffu);
        // all candidates NaN: keep the diagonal (its pivot is then flagged below)
        const int p = kmax != K(0) ? (int)(pw >> 5) : c;
        const int w = kmax != K(0) ? (int)(pw & 31u) : -1;
        if (lane < KB) {
            T piv = w >= 0 ? s_cand[par][w][c] : zero<T>();
            if (!(abs1(piv) > real(0))) {                         // exact zero (or NaN) pivot
                piv = one<T>();
                if (tid == 0 && atomicCAS(&status->code, 0, (int)NDHSS_ERR_SINGULAR) == 0) status->node = s;
            }
            const T pinv = recip(piv);
            const T b = w >= 0 ? s_cand[par][w][lane] : zero<T>();
            s_pr[warp][lane] = lane >= kbp ? zero<T>() : (lane == c) ? pinv : -(b * pinv);
        }
        if (tid == 0) ip[c] = k0 + p;
        __syncwarp();
        const bool is_piv = has && pos == p;
        // one FMA form for every entry: the pivot column's entry becomes
        // a * pr(c) and the pivot row becomes pr; both are fmac with the
        // addend -0 (x + -0 = x exactly), the pivot row with multiplier one
        const T am = is_piv ? one<T>() : a;
        T an = a;                            // this row's updated entry in the next column
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            const T prj = s_pr[warp][j];
            const T vin = (is_piv || j == c) ? neg_zero<T>() : v[j];
            v[j] = fmac(am, prj, vin);
            take_if(j, c + 1, v[j], an);
        }
        a = an;
        if (pos == c) pos = p;
        else if (pos == p) pos = c;
        if (c + 1 < kbp)
            panel_publish<T, KB>(v, abs1(a), has && pos > c, pos, s_cand[par ^ 1][warp], &s_key[par ^ 1][warp],
                                 &s_pos[par ^ 1][warp], lane);
        __syncthreads();
    }
    // rows at positions < kbp hold (A_PP)^{-1} of the interchanged pivot block
    T* Ai = ainv_buf + (size_t)blockIdx.x * KBMAX * KBMAX;
    if (has && pos < kbp) {
#pragma unroll
        for (int j = 0; j < KB; ++j)
            if (j < kbp) Ai[j * KBMAX + pos] = v[j];
    }
    // net row map of the interchanges: position k0 + pos receives the old row k0 + tid
    int32_t* sm = swapmap + (size_t)blockIdx.x * (4 * KBMAX + 1);
    if (has && pos != tid) {
        const int a = atomicAdd(&s_na, 1);
        sm[1 + a] = k0 + pos;
        sm[1 + 2 * KBMAX + a] = k0 + tid;
    }
    __syncthreads();
    if (tid == 0) sm[0] = s_na;
}

template <typename T>
__global__ void __launch_bounds__(PREP_WARPS * 32)
panel_prep_kernel(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                  const int64_t* __restrict__ foff, T* __restrict__ front, const int32_t* __restrict__ swapmap,
                  const T* __restrict__ ainv_buf, T* __restrict__ cbuf, T* __restrict__ zbuf,
                  const int64_t* __restrict__ woff, int k0, int kb, int slab0, int slabw) {
    __shared__ T s_ai[KBMAX * KBMAX];
    __shared__ int s_rows[2 * KBMAX], s_org[2 * KBMAX];
    const int li = blockIdx.y;
    const int s = lev[li];
    const int m_i = nf(node, s, 5);
    if (k0 >= m_i) return;
    const int64_t m = m_i + nf(node, s, 7);
    // columns that take part in this pivot block's exchange: the whole front,
    // or (two-level blocking) the slab [slab0, slab0 + slabw) of the outer
    // block; the interchanges go to every column
    const int64_t zlo = slabw ? slab0 : 0, zhi = slabw ? min((int64_t)slab0 + slabw, (int64_t)m_i) : m;
    const int kbp = min(kb, m_i - k0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T* Ai = ainv_buf + (size_t)li * KBMAX * KBMAX;
    for (int q = tid; q < KBMAX * KBMAX; q += blockDim.x) s_ai[q] = Ai[q];
    const int32_t* sm = swapmap + (size_t)li * (4 * KBMAX + 1);
    const int na = sm[0];
    for (int a = tid; a < na; a += blockDim.x) {
        s_rows[a] = sm[1 + a];
        s_org[a] = sm[1 + 2 * KBMAX + a];
    }
    __syncthreads();
    T* F = front + foff[s];
    T* C = cbuf + woff[li] * KBMAX;     // m x kbp, ld m
    T* Z = zbuf + woff[li] * KBMAX;     // kbp x m, ld KBMAX
    for (int64_t j = (int64_t)blockIdx.x * PREP_WARPS + warp; j < m; j += (int64_t)gridDim.x * PREP_WARPS) {
        T* Fj = F + j * m;
        T v0 = zero<T>(), v1 = zero<T>();
        if (lane < na) v0 = Fj[s_org[lane]];
        if (lane + 32 < na) v1 = Fj[s_org[lane + 32]];
        __syncwarp();
        if (lane < na) Fj[s_rows[lane]] = v0;
        if (lane + 32 < na) Fj[s_rows[lane + 32]] = v1;
        __syncwarp();
        if (j < zlo || j >= zhi) continue;
        if (j >= k0 && j < k0 + kbp) {
            const int cidx = (int)(j - k0);
            // the whole pivot column: eight rows per lane loaded before they are
            // stored (one load-store pair at a time waits out the latency m / 32 times)
            for (int64_t i0 = lane; i0 < m; i0 += 32 * 8) {
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t i = i0 + 32 * u;
                    v[u] = i < m ? Fj[i] : zero<T>();
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t i = i0 + 32 * u;
                    if (i >= m) continue;
                    if (i >= k0 && i < k0 + kbp) v[u] = (i - k0 == cidx) ? one<T>() : zero<T>();
                    C[(int64_t)cidx * m + i] = v[u];
                }
            }
            if (lane < kbp) Z[j * KBMAX + lane] = s_ai[cidx * KBMAX + lane];
        } else {
            const T w = lane < kbp ? Fj[k0 + lane] : zero<T>();
            T acc = zero<T>();
            for (int l = 0; l < kbp; ++l) acc = fmac(s_ai[l * KBMAX + (lane < kbp ? lane : 0)], shfl_idx(w, l), acc);
            if (lane < kbp) Z[j * KBMAX + lane] = -acc;
        }
    }
}

// M = beta .* M + C * Z over one 64 x 64 tile (beta = 0 on pivot rows or columns).
template <typename T>
__global__ void __launch_bounds__(256)
gemm_update_kernel(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                   const int64_t* __restrict__ foff, T* __restrict__ front, const T* __restrict__ cbuf,
                   const T* __restrict__ zbuf, const int64_t* __restrict__ woff, int k0, int kb, int slab0, int slabw) {
    __shared__ T sC[GK][GT];
    __shared__ T sZ[GK][GT];
    const int li = blockIdx.z;
    const int s = lev[li];
    const int m_i = nf(node, s, 5);
    if (k0 >= m_i) return;
    const int64_t m = m_i + nf(node, s, 7);
    // columns [zlo, zhi): the whole front, or the slab of the outer block
    const int64_t zlo = slabw ? slab0 : 0, zhi = slabw ? min((int64_t)slab0 + slabw, (int64_t)m_i) : m;
    const int64_t i0 = (int64_t)blockIdx.x * GT, j0 = zlo + (int64_t)blockIdx.y * GT;
    if (i0 >= m || j0 >= zhi) return;
    const int kbp = min(kb, m_i - k0);
    const T* C = cbuf + woff[li] * KBMAX;
    const T* Z = zbuf + woff[li] * KBMAX;
    T* F = front + foff[s];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = zero<T>();
    for (int kc = 0; kc < kbp; kc += GK) {
        for (int idx = tid; idx < GK * GT; idx += 256) {
            const int ii = idx % GT, l = idx / GT;
            const int64_t i = i0 + ii;
            sC[l][ii] = (kc + l < kbp && i < m) ? C[(int64_t)(kc + l) * m + i] : zero<T>();
        }
        for (int idx = tid; idx < GK * GT; idx += 256) {
            const int l = idx % GK, jj = idx / GK;
            const int64_t j = j0 + jj;
            sZ[l][jj] = (kc + l < kbp && j < zhi) ? Z[j * KBMAX + kc + l] : zero<T>();
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < GK; ++l) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sC[l][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = sZ[l][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmac(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int64_t j = j0 + ty + 16 * b;
        if (j >= zhi) continue;
        const bool pj = (j >= k0 && j < k0 + kbp);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t i = i0 + tx + 16 * a;
            if (i >= m) continue;
            const bool pi = (i >= k0 && i < k0 + kbp);
            T* dst = F + j * m + i;
            *dst = (pi || pj) ? acc[a][b] : (*dst + acc[a][b]);
        }
    }
}

// sigma(j) = original row of A_ii now at row j, from the interchange record
__global__ void finalize_sigma_kernel(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                                      const int32_t* __restrict__ ipiv, int32_t* __restrict__ sigma) {
    extern __shared__ int s_a[];
    const int s = lev[blockIdx.x];
    const int m_i = nf(node, s, 5), i_off = nf(node, s, 4);
    int* a = s_a;
    int* pv = s_a + m_i;
    for (int j = threadIdx.x; j < m_i; j += blockDim.x) { a[j] = j; pv[j] = ipiv[i_off + j]; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < m_i; ++k) {
            const int p = pv[k];
            const int t = a[k]; a[k] = a[p]; a[p] = t;
        }
    __syncthreads();
    for (int j = threadIdx.x; j < m_i; j += blockDim.x) sigma[i_off + j] = a[j];
}

// One panel launch: the register-resident kernel when asked and the element
// fits (8 bytes at most), else the shared-memory kernel.  More than
// PANEL_THREADS rows take the 2 * PANEL_THREADS instance (64 registers a
// thread: KB <= 16).
template <typename T, int KB>
void launch_panel(bool reg, int grid, int threads, size_t smem, cudaStream_t st, const int32_t* lev,
                  const int32_t* node, const int64_t* foff, const T* front, int32_t* ipiv, T* ainv, int32_t* swapmap,
                  int k0, int kb, DevStatus* status) {
    if constexpr (sizeof(T) <= 8) {
        if (reg && threads <= PANEL_THREADS) {
            panel_reg_kernel<T, KB, PANEL_THREADS><<<grid, threads, 0, st>>>(lev, node, foff, front, ipiv, ainv, swapmap,
                                                                             k0, kb, status);
            return;
        }
        if constexpr (KB <= 16) {
            if (reg) {
                panel_reg_kernel<T, KB, 2 * PANEL_THREADS><<<grid, threads, 0, st>>>(lev, node, foff, front, ipiv, ainv,
                                                                                     swapmap, k0, kb, status);
                return;
            }
        }
    }
    panel_factor_kernel<T, KB><<<grid, threads, smem, st>>>(lev, node, foff, front, ipiv, ainv, swapmap, k0, kb, status);
}

int choose_kb(int64_t mc, size_t esize, int panel_opt) {
    int kb = KBMAX;
    while (kb > 1 && (size_t)mc * (kb * esize + sizeof(int)) > PANEL_SMEM_MAX) kb >>= 1;
    if (panel_opt > 0)
        while (kb > panel_opt) kb >>= 1;     // powers of two only (the panel kernel is templated on it)
    return kb;
}

template <typename T>
ndhss_status set_smem_attrs() {
    void (*kernels[])(const int32_t*, const int32_t*, const int64_t*, const T*, int32_t*, T*, int32_t*, int, int,
                      DevStatus*) = {panel_factor_kernel<T, 1>, panel_factor_kernel<T, 2>, panel_factor_kernel<T, 4>,
                                     panel_factor_kernel<T, 8>, panel_factor_kernel<T, 16>, panel_factor_kernel<T, 32>};
    for (auto k : kernels)
        NDHSS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM_MAX));
    return NDHSS_OK;
}

// Device copy of a host table, stream-ordered on st from the library pool
// (the pageable source may be released once this returns).
template <typename U>
ndhss_status upload(U** dst, const U* src, size_t count, int64_t* acc, cudaStream_t st) {
    *dst = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(U);
    if (pool_malloc_async((void**)dst, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return set_error(NDHSS_ERR_OOM, "device allocation of %zu bytes failed", bytes);
    }
    *acc += (int64_t)bytes;
    if (count) NDHSS_CUDA_TRY(cudaMemcpyAsync(*dst, src, count * sizeof(U), cudaMemcpyHostToDevice, st));
    return NDHSS_OK;
}

// Optional per-launch CUDA-event timing, summed per kernel class.
struct LaunchTimer {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    cudaEvent_t pending = nullptr;
    void begin() {
        if (!on) return;
        cudaEventCreate(&pending);
        cudaEventRecord(pending, st);
    }
    void end(int cls) {
        if (!on) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        ev.push_back({cls, {pending, e}});
    }
    void collect(FactorData& F) {
        for (auto& x : ev) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, x.second.first, x.second.second) == cudaSuccess) F.class_ms[x.first] += ms;
            F.class_launches[x.first]++;
            cudaEventDestroy(x.second.first);
            cudaEventDestroy(x.second.second);
        }
        ev.clear();
    }
};

// A_ii of a ULV front in its HSS order, copied out of the assembled front
// before the elimination overwrites it: aii(j, j') = A_ii(ord[j], ord[j']).
struct AiiJob {
    int64_t aii_off, foff, ord_off;
    int32_t m, mi;
};

template <typename T>
__global__ void gather_aii_kernel(const AiiJob* __restrict__ jobs, const int32_t* __restrict__ ord,
                                  const T* __restrict__ front, T* __restrict__ aii) {
    const AiiJob J = jobs[blockIdx.y];
    const int32_t* o = ord + J.ord_off;
    const int64_t tot = (int64_t)J.mi * J.mi;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q % J.mi), jj = (int)(q / J.mi);
        aii[J.aii_off + q] = front[J.foff + (int64_t)o[jj] * J.m + o[j]];
    }
}

// Compresses the low-rank R of finished fronts on a stream and host thread
// of its own while the main stream goes on factoring (R is read only by the
// apply; the compression's adaptive rounds synchronise only the worker's
// stream).  Each hand-over carries an event recorded on the main stream
// once its fronts are final; finish() waits for every hand-over, merges the
// storage and counters, and makes the main stream wait for the worker's.
class LowRankWorker {
public:
    LowRankWorker(FactorData& F, const ndhss_factor_opts& o) : F_(F), o_(o) {}
    LowRankWorker(const LowRankWorker&) = delete;
    LowRankWorker& operator=(const LowRankWorker&) = delete;
    ~LowRankWorker() {
        stop();
        // storage of a factorization that failed before finish(): freed after
        // the worker's stream has drained
        for (void* b : acc_.lr_bufs) cudaFreeAsync(b, st_);
        for (cudaStream_t& x : acc_.side_streams)
            if (x) cudaStreamDestroy(x);
        if (st_) cudaStreamDestroy(st_);
    }
    ndhss_status start() {
        NDHSS_CUDA_TRY(cudaGetDevice(&dev_));
        NDHSS_CUDA_TRY(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
        for (cudaStream_t& x : acc_.side_streams) NDHSS_CUDA_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        th_ = std::thread([this] { run(); });
        return NDHSS_OK;
    }
    // the fronts' R blocks are final once the main stream reaches this point
    ndhss_status submit(std::vector<int32_t>&& fronts, cudaStream_t main) {
        cudaEvent_t ev = nullptr;
        NDHSS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        const cudaError_t e = cudaEventRecord(ev, main);
        if (e != cudaSuccess) {
            cudaEventDestroy(ev);
            return set_error(NDHSS_ERR_CUDA, "ndhss_factor: low-rank hand-over: %s", cudaGetErrorString(e));
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            q_.push_back({std::move(fronts), ev});
        }
        cv_.notify_one();
        return NDHSS_OK;
    }
    ndhss_status finish(cudaStream_t main) {
        stop();
        if (status_ != NDHSS_OK) return set_error(status_, "%s", msg_.c_str());
        F_.dev_bytes += acc_.dev_bytes;
        F_.lr_bufs.insert(F_.lr_bufs.end(), acc_.lr_bufs.begin(), acc_.lr_bufs.end());
        acc_.lr_bufs.clear();
        F_.hss_rounds_max = std::max(F_.hss_rounds_max, acc_.hss_rounds_max);
        F_.kmax = std::max(F_.kmax, kmax_);
        cudaEvent_t ev = nullptr;
        NDHSS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, st_);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess) return set_error(NDHSS_ERR_CUDA, "ndhss_factor: low-rank join: %s", cudaGetErrorString(e));
        return NDHSS_OK;
    }

private:
    struct Job {
        std::vector<int32_t> fronts;
        cudaEvent_t ev;
    };
    void stop() {
        if (!th_.joinable()) return;
        {
            std::lock_guard<std::mutex> lk(mu_);
            done_ = true;
        }
        cv_.notify_one();
        th_.join();
    }
    void run() {
        cudaSetDevice(dev_);
        for (;;) {
            Job j;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return done_ || !q_.empty(); });
                if (q_.empty()) return;
                j = std::move(q_.front());
                q_.pop_front();
            }
            if (status_ == NDHSS_OK) {
                ndhss_status rc = NDHSS_OK;
                try {
                    const cudaError_t e = cudaStreamWaitEvent(st_, j.ev, 0);
                    rc = e == cudaSuccess ? hss_lowrank_fronts(F_, j.fronts, acc_, &kmax_, o_, st_)
                                          : set_error(NDHSS_ERR_CUDA, "ndhss_factor: %s", cudaGetErrorString(e));
                } catch (const std::bad_alloc&) {
                    rc = set_error(NDHSS_ERR_OOM, "ndhss_factor: host allocation failed in the low-rank worker");
                } catch (...) {
                    rc = set_error(NDHSS_ERR_INTERNAL, "ndhss_factor: exception in the low-rank worker");
                }
                if (rc != NDHSS_OK) {
                    status_ = rc;
                    msg_ = ndhss_last_error();
                }
            }
            cudaEventDestroy(j.ev);
        }
    }
    FactorData& F_;
    const ndhss_factor_opts& o_;
    FactorData acc_;
    int kmax_ = 0;
    int dev_ = 0;
    cudaStream_t st_ = nullptr;
    std::thread th_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<Job> q_;
    bool done_ = false;
    ndhss_status status_ = NDHSS_OK;     // written by the worker only, read after the join
    std::string msg_;
};

template <typename T, typename V>
ndhss_status factor_run(FactorData& F, const Tree& t, const V* d_vals, const int32_t* d_eoff,
                        const int32_t* d_erow, const int32_t* d_ecol, const int32_t* d_eidx,
                        const int32_t* d_fsrc, const int64_t* d_poff, const int32_t* d_lev,
                        const std::vector<int64_t>& lev_off, const int64_t* d_woff, T* d_cbuf, T* d_zbuf,
                        T* d_ainv, int32_t* d_swapmap, DevStatus* d_status, const ndhss_factor_opts& o,
                        LaunchTimer& tm, cudaStream_t st) {
    const int panel_opt = o.panel;
    // the low-rank R of the levels below the switching level compresses on a
    // second stream while the main stream factors the root level
    LowRankWorker lrw(F, o);
    const bool lr_async = F.L_hss > 1;
    if (lr_async) {
        const ndhss_status rcw = lrw.start();
        if (rcw != NDHSS_OK) return rcw;
    }
    // NDHSS_PANEL=smem keeps every panel in shared memory (panel_factor_kernel;
    // a cross-check of the register-resident panel: the same real outputs, the
    // complex ones up to FMA contraction)
    const char* pe = std::getenv("NDHSS_PANEL");
    const bool reg_panel_ok = sizeof(T) <= 8 && !(pe && std::strcmp(pe, "smem") == 0);
    ndhss_status rc = set_smem_attrs<T>();
    if (rc != NDHSS_OK) return rc;
    T* front = static_cast<T*>(F.d_front);
    const double flops_per_mac = Tr<T>::cplx ? 8.0 : 2.0;
    for (int l = F.depth; l >= 0; --l) {
        const auto& nodes = F.levels[l];
        const int L = (int)nodes.size();
        if (L == 0) continue;
        const int32_t* lev = d_lev + lev_off[l];
        const int64_t* woff = d_woff + lev_off[l];
        int64_t mmax = 0, mimax = 0;
        for (int s : nodes) {
            mmax = std::max<int64_t>(mmax, F.m_i(s) + F.m_b(s));
            mimax = std::max<int64_t>(mimax, F.m_i(s));
        }
        if (mmax == 0) continue;
        const int agx = (int)std::min<int64_t>(mmax, 256);
        tm.begin();
        for (int c0 = 0; c0 < L; c0 += MAX_GRID_YZ) {
            assemble_kernel<T><<<dim3(agx, std::min(MAX_GRID_YZ, L - c0)), 256, 0, st>>>(lev + c0, F.d_node, F.d_foff,
                                                                                       d_fsrc, d_poff, front);
            NDHSS_LAUNCH_CHECK("assemble_kernel");
        }
        tm.end(0);
        tm.begin();
        scatter_entries_kernel<T, V><<<L, 256, 0, st>>>(lev, F.d_node, F.d_foff, d_eoff, d_erow, d_ecol, d_eidx,
                                                        d_vals, front);
        NDHSS_LAUNCH_CHECK("scatter_entries_kernel");
        tm.end(1);
        F.launches += 2;
        // ULV fronts of this level: their A_ii in HSS order, before the sweep below
        std::vector<int64_t> aii_off;
        void* d_aii = nullptr;
        if (F.ulv && l < F.L_hss) {
            aii_off.assign(t.nnodes, -1);
            std::vector<AiiJob> jobs;
            int64_t tot = 0;
            for (int s : nodes)
                if (F.ulv_ord_off[s] >= 0) {
                    aii_off[s] = tot;
                    jobs.push_back({tot, F.foff[s], F.ulv_ord_off[s], F.m_i(s) + F.m_b(s), F.m_i(s)});
                    tot += (int64_t)F.m_i(s) * F.m_i(s);
                }
            if (!jobs.empty()) {
                AiiJob* d_jobs = nullptr;
                if (pool_malloc_async(&d_aii, (size_t)tot * sizeof(T), st) != cudaSuccess ||
                    pool_malloc_async((void**)&d_jobs, jobs.size() * sizeof(AiiJob), st) != cudaSuccess) {
                    cudaGetLastError();
                    return set_error(NDHSS_ERR_OOM, "ndhss_factor: A_ii copies of level %d", l);
                }
                NDHSS_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(AiiJob), cudaMemcpyHostToDevice, st));
                gather_aii_kernel<T><<<dim3(64, (unsigned)jobs.size()), 256, 0, st>>>(d_jobs, F.d_ulv_ord, front,
                                                                                       static_cast<T*>(d_aii));
                NDHSS_LAUNCH_CHECK("gather_aii_kernel");
                cudaFreeAsync(d_jobs, st);
            }
        }
        // Two-level blocking on the tensor cores (tcgemm.cu) for levels with
        // large fronts: the pivots go in outer blocks of TC_KB2 columns; inside
        // one, the rank-kb steps exchange only the block's own columns (its
        // slab), then one GEMM with K = TC_KB2 applies the block's exchange to
        // every other column of the front.  The arithmetic is the sweep's own
        // (a block of exchanges composed), so S stays the elimination's Schur
        // complement.  Small fronts keep the rank-kb steps over the whole front.
        const bool tcl = tc_front_path(F, mimax);
        const int kb2 = tcl ? TC_KB2 : 0;
        const int gt = (int)((mmax + GT - 1) / GT);
        const int gty = tcl ? (TC_KB2 + GT - 1) / GT : gt;
        const int pgx = (int)std::min<int64_t>((mmax + PREP_WARPS - 1) / PREP_WARPS, 1024);
        for (int64_t k0 = 0; k0 < mimax;) {
            const int64_t s0 = tcl ? k0 / TC_KB2 * TC_KB2 : 0;     // the outer block's first pivot
            int kb = choose_kb(mimax - k0, sizeof(T), panel_opt);
            while (tcl && k0 + kb > s0 + TC_KB2) kb >>= 1;
            // every candidate row in one thread's registers when the rows fit one
            // CTA (up to 2 * PANEL_THREADS rows, at most 16 columns beyond PANEL_THREADS)
            const bool reg_panel = reg_panel_ok && mimax - k0 <= 2 * PANEL_THREADS;
            if (reg_panel && mimax - k0 > PANEL_THREADS) kb = std::min(kb, 16);
            const size_t smem = (size_t)(mimax - k0) * kb * sizeof(T) + (size_t)(mimax - k0) * sizeof(int);
            if (smem > PANEL_SMEM_MAX)
                return set_error(NDHSS_ERR_INVALID_ARG, "front with %lld interior unknowns exceeds the panel kernel's shared memory",
                                 (long long)(mimax - k0));
            // one thread per candidate row up to 512: small fronts get small CTAs, so a level of
            // thousands of leaves runs in one wave instead of repeating its pivot chain per wave
            const int pthreads = (int)std::min<int64_t>(reg_panel ? 2 * PANEL_THREADS : PANEL_THREADS,
                                                        std::max<int64_t>(64, (mimax - k0 + 31) / 32 * 32));
            // a level of more than 65535 fronts (the grid's y / z limit) goes in
            // chunks; the three kernels of a chunk share its per-front scratch
            for (int c0 = 0; c0 < L; c0 += MAX_GRID_YZ) {
                const int Lc = std::min(MAX_GRID_YZ, L - c0);
                const int32_t* levc = lev + c0;
                const int64_t* woffc = woff + c0;
                tm.begin();
                switch (kb) {
#define NDHSS_PANEL(KBV)                                                                                          \
    case KBV:                                                                                                   \
        launch_panel<T, KBV>(reg_panel, Lc, pthreads, smem, st, levc, F.d_node, F.d_foff, front, F.d_ipiv, d_ainv, \
                             d_swapmap, (int)k0, kb, d_status);                                                 \
        break;
                    NDHSS_PANEL(1) NDHSS_PANEL(2) NDHSS_PANEL(4) NDHSS_PANEL(8) NDHSS_PANEL(16) NDHSS_PANEL(32)
#undef NDHSS_PANEL
                    default: return set_error(NDHSS_ERR_INTERNAL, "panel width %d is not a power of two <= 32", kb);
                }
                NDHSS_LAUNCH_CHECK("panel_factor_kernel");
                tm.end(2);
                tm.begin();
                panel_prep_kernel<T><<<dim3(pgx, Lc), PREP_WARPS * 32, 0, st>>>(levc, F.d_node, F.d_foff, front,
                                                                               d_swapmap, d_ainv, d_cbuf, d_zbuf, woffc,
                                                                               (int)k0, kb, (int)s0, kb2);
                NDHSS_LAUNCH_CHECK("panel_prep_kernel");
                tm.end(3);
                tm.begin();
                gemm_update_kernel<T><<<dim3(gt, gty, Lc), 256, 0, st>>>(levc, F.d_node, F.d_foff, front, d_cbuf,
                                                                       d_zbuf, woffc, (int)k0, kb, (int)s0, kb2);
                NDHSS_LAUNCH_CHECK("gemm_update_kernel");
                tm.end(4);
            }
            F.launches += 3;
            for (int s2 : nodes) {
                const int64_t mi = F.m_i(s2), m2 = mi + F.m_b(s2);
                const int64_t cols = tcl ? std::min<int64_t>(TC_KB2, mi - s0) : m2;
                if (mi > k0) F.update_flops += flops_per_mac * (double)m2 * (double)cols * (double)std::min<int64_t>(kb, mi - k0);
            }
            k0 += kb;
            if (tcl && (k0 == s0 + TC_KB2 || k0 >= mimax)) {
                // the outer block's exchange on the columns outside its slab
                tm.begin();
                const ndhss_status rc2 = tc_block_exchange(F, nodes, (int)s0, d_status, st);
                if (rc2 != NDHSS_OK) {
                    if (d_aii) cudaFreeAsync(d_aii, st);
                    return rc2;
                }
                tm.end(7);
            }
        }
        if (mimax > 0) {
            tm.begin();
            finalize_sigma_kernel<<<L, 256, (size_t)mimax * 2 * sizeof(int), st>>>(lev, F.d_node, F.d_ipiv, F.d_sigma);
            NDHSS_LAUNCH_CHECK("finalize_sigma_kernel");
            tm.end(5);
            F.launches += 1;
        }
        if (F.L_hss >= 0 && l <= F.L_hss) {
            // Alg. 3.4 at and above the switching level: compress S (and R above it)
            tm.begin();
            ndhss_status rc2 = hss_compress_level(F, t, l, o, st);
            if (rc2 == NDHSS_OK && d_aii) rc2 = hss_ulv_level(F, t, l, d_aii, aii_off, o, st);
            if (d_aii) cudaFreeAsync(d_aii, st);
            // all levels' R in one batch (as few adaptive rounds as at the end),
            // handed over before the root level, whose elimination runs one CTA
            // at a time and leaves the SMs to the worker (handing over level
            // by level slowed the main stream's latency-bound kernels more than
            // it saved)
            if (rc2 == NDHSS_OK && lr_async && l == 1 && !F.lr_pending.empty()) {
                std::vector<int32_t> fronts;
                fronts.swap(F.lr_pending);
                rc2 = lrw.submit(std::move(fronts), st);
            }
            if (rc2 != NDHSS_OK) return rc2;
            tm.end(6);
        } else if (d_aii) {
            cudaFreeAsync(d_aii, st);
        }
    }
    if (lr_async) {
        tm.begin();
        const ndhss_status rc2 = lrw.finish(st);
        if (rc2 != NDHSS_OK) return rc2;
        tm.end(6);
    }
    if (!F.lr_pending.empty()) {
        tm.begin();
        ndhss_status rc2 = hss_lowrank_pending(F, o, st);
        if (rc2 != NDHSS_OK) return rc2;
        tm.end(6);
    }
    return NDHSS_OK;
}

}  // namespace

// --------------------------------------------------------------------------
// public entry points
// --------------------------------------------------------------------------

static ndhss_status factor_impl(const ndhss_tree* th, int32_t vtype, const int32_t* d_rowptr, const int32_t* d_col,
                                const void* d_vals, const ndhss_factor_opts* opts, void* stream, ndhss_factorization** out) {
    (void)d_rowptr;
    (void)d_col;
    const auto t_entry = std::chrono::steady_clock::now();
    if (!th || !d_vals || !out) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor: NULL argument");
    if (vtype != NDHSS_R64 && vtype != NDHSS_C128) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor: bad vtype %d", vtype);
    const Tree& t = th->t;
    ndhss_factor_opts o{};
    o.prec = NDHSS_FP64;
    o.hss_levels = -1;
    if (opts) o = *opts;
    if (o.prec != NDHSS_FP64 && o.prec != NDHSS_FP32 && o.prec != NDHSS_FP32_TF32 && o.prec != NDHSS_FP32_BF16)
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor: bad precision %d", o.prec);
    if (o.hss_levels >= 0 && (!(o.eps_hss > 0) || o.beta < 1 || o.k0 < 1 || o.r < 1 || o.rank_cap < 1))
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor: compression needs eps_hss > 0 and beta, k0, r, rank_cap >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool cplx = vtype == NDHSS_C128;
    const bool fp64 = o.prec == NDHSS_FP64;
    const size_t esize = cplx ? (fp64 ? 16 : 8) : (fp64 ? 8 : 4);

    auto* h = new ndhss_factorization();
    FactorData& F = h->f;
    F.vtype = vtype;
    F.prec = o.prec;
    F.n = t.n;
    F.nnodes = t.nnodes;
    F.depth = t.depth;
    F.esize = esize;
    F.node_info = t.node_info;
    F.blist_h = t.blist;
    F.L_hss = (o.hss_levels >= 0) ? t.depth - o.hss_levels : -1;
    F.levels.assign(t.depth + 1, {});
    for (int s = 0; s < t.nnodes; ++s) F.levels[t.level(s)].push_back(s);
    // ULV tier: the HSS order of every A_ii strictly above the switching level,
    // by the coordinate along the node's cut (ties: position in I^s)
    F.ulv = o.ulv != 0 && F.L_hss > 0;
    F.ulv_root_of.assign(t.nnodes, -1);
    F.ulv_ord_off.assign(t.nnodes, -1);
    if (F.ulv) {
        for (int s = 0; s < t.nnodes; ++s) {
            const int mi = t.m_i(s);
            if (t.level(s) >= F.L_hss || mi == 0) continue;
            const int axis = t.info(s, 12);
            std::vector<int32_t> ord(mi);
            std::vector<int64_t> along(mi, 0);
            for (int c = 0; c < mi; ++c) {
                ord[c] = c;
                const int d = t.perm[t.i_off(s) + c];
                if (axis == 0 || axis == 1) along[c] = t.coords[2 * (size_t)d + (1 - axis)];
            }
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return along[a] < along[b]; });
            F.ulv_ord_off[s] = (int64_t)F.ulv_ord.size();
            F.ulv_ord.insert(F.ulv_ord.end(), ord.begin(), ord.end());
        }
    }
    F.foff.resize(t.nnodes);
    int64_t acc = 0, posacc = 0;
    std::vector<int64_t> poff(t.nnodes);
    for (int s = 0; s < t.nnodes; ++s) {
        const int64_t m = (int64_t)t.m_i(s) + t.m_b(s);
        F.foff[s] = acc;
        acc += m * m;
        poff[s] = posacc;
        posacc += m;
        F.max_mi = std::max(F.max_mi, t.m_i(s));
        F.max_mb = std::max(F.max_mb, t.m_b(s));
    }
    F.front_elems = acc;
    // inverse extend-add map per front position
    std::vector<int32_t> fsrc(std::max<int64_t>(posacc, 1), 0);
    for (int s = 0; s < t.nnodes; ++s) {
        for (int w = 0; w < 2; ++w) {
            const int k = t.child(s, w);
            if (k < 0) continue;
            for (int r = 0; r < t.m_b(k); ++r) fsrc[poff[s] + t.emap[t.b_off(k) + r]] = (w << 30) | r;
        }
    }
    // level lists and per-level workspace offsets
    std::vector<int32_t> lev_flat;
    std::vector<int64_t> lev_off(t.depth + 2, 0), woff_flat;
    int64_t wmax = 0, lmax = 0;
    for (int l = 0; l <= t.depth; ++l) {
        lev_off[l] = (int64_t)lev_flat.size();
        int64_t w = 0;
        for (int s : F.levels[l]) {
            lev_flat.push_back(s);
            woff_flat.push_back(w);
            w += (int64_t)t.m_i(s) + t.m_b(s);
        }
        wmax = std::max(wmax, w);
        lmax = std::max<int64_t>(lmax, (int64_t)F.levels[l].size());
    }
    lev_off[t.depth + 1] = (int64_t)lev_flat.size();
    int64_t apply_elems = 0;
    for (int s = 0; s < t.nnodes; ++s)
        apply_elems += (int64_t)t.m_i(s) * t.m_i(s) + 2 * (int64_t)t.m_i(s) * t.m_b(s);
    F.apply_bytes = apply_elems * (int64_t)esize;

    ndhss_status rc = NDHSS_OK;
    int32_t *d_eoff = nullptr, *d_erow = nullptr, *d_ecol = nullptr, *d_eidx = nullptr, *d_fsrc = nullptr, *d_lev = nullptr;
    int64_t *d_poff = nullptr, *d_woff = nullptr;
    void *d_cbuf = nullptr, *d_zbuf = nullptr, *d_ainv = nullptr;
    int32_t* d_swapmap = nullptr;
    DevStatus* d_status = nullptr;
    int64_t tmp_bytes = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto t_done = std::chrono::steady_clock::now();
    auto cleanup = [&]() {
        for (void* q : {(void*)d_eoff, (void*)d_erow, (void*)d_ecol, (void*)d_eidx, (void*)d_fsrc, (void*)d_lev,
                        (void*)d_poff, (void*)d_woff, d_cbuf, d_zbuf, d_ainv, (void*)d_swapmap, (void*)d_status})
            if (q) cudaFreeAsync(q, st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
#define UP(dst, vec) do { rc = upload(&dst, (vec).data(), (vec).size(), &F.dev_bytes, st); if (rc) { cleanup(); ndhss_factor_destroy(h); return rc; } } while (0)
#define UPT(dst, vec) do { rc = upload(&dst, (vec).data(), (vec).size(), &tmp_bytes, st); if (rc) { cleanup(); ndhss_factor_destroy(h); return rc; } } while (0)
    UP(F.d_node, t.node_info);
    UP(F.d_foff, F.foff);
    UP(F.d_blist, t.blist);
    UP(F.d_perm, t.perm);
    if (F.ulv) UP(F.d_ulv_ord, F.ulv_ord);
    UPT(d_eoff, t.e_off);
    UPT(d_erow, t.e_row);
    UPT(d_ecol, t.e_col);
    UPT(d_eidx, t.e_idx);
    UPT(d_fsrc, fsrc);
    UPT(d_poff, poff);
    UPT(d_lev, lev_flat);
    UPT(d_woff, woff_flat);
#undef UP
#undef UPT
    auto dalloc = [&](void** p, size_t bytes, int64_t* accb) -> bool {
        if (pool_malloc_async(p, std::max<size_t>(bytes, 16), st) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        *accb += (int64_t)bytes;
        return true;
    };
    if (!dalloc((void**)&F.d_sigma, (size_t)t.n * 4, &F.dev_bytes) ||
        !dalloc((void**)&F.d_ipiv, (size_t)t.n * 4, &F.dev_bytes) ||
        !dalloc(&F.d_front, (size_t)F.front_elems * esize, &F.dev_bytes) ||
        !dalloc(&d_cbuf, (size_t)wmax * KBMAX * esize, &tmp_bytes) ||
        !dalloc(&d_zbuf, (size_t)wmax * KBMAX * esize, &tmp_bytes) ||
        !dalloc(&d_ainv, (size_t)lmax * KBMAX * KBMAX * esize, &tmp_bytes) ||
        !dalloc((void**)&d_swapmap, (size_t)lmax * (4 * KBMAX + 1) * sizeof(int32_t), &tmp_bytes) ||
        !dalloc((void**)&d_status, sizeof(DevStatus), &tmp_bytes)) {
        cleanup();
        ndhss_factor_destroy(h);
        return set_error(NDHSS_ERR_OOM, "ndhss_factor: device allocation failed (front arena %lld elements)",
                         (long long)F.front_elems);
    }
    NDHSS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(DevStatus), st));
    NDHSS_CUDA_TRY(cudaEventCreate(&e0));
    NDHSS_CUDA_TRY(cudaEventCreate(&e1));
    LaunchTimer tm;
    tm.on = o.timing != 0;
    tm.st = st;
    NDHSS_CUDA_TRY(cudaEventRecord(e0, st));
    F.host_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_entry).count();
    if (!cplx && fp64)
        rc = factor_run<double, double>(F, t, (const double*)d_vals, d_eoff, d_erow, d_ecol, d_eidx, d_fsrc, d_poff, d_lev,
                                        lev_off, d_woff, (double*)d_cbuf, (double*)d_zbuf, (double*)d_ainv, d_swapmap, d_status,
                                        o, tm, st);
    else if (!cplx)
        rc = factor_run<float, double>(F, t, (const double*)d_vals, d_eoff, d_erow, d_ecol, d_eidx, d_fsrc, d_poff, d_lev,
                                       lev_off, d_woff, (float*)d_cbuf, (float*)d_zbuf, (float*)d_ainv, d_swapmap, d_status,
                                       o, tm, st);
    else if (fp64)
        rc = factor_run<c128, c128>(F, t, (const c128*)d_vals, d_eoff, d_erow, d_ecol, d_eidx, d_fsrc, d_poff, d_lev,
                                    lev_off, d_woff, (c128*)d_cbuf, (c128*)d_zbuf, (c128*)d_ainv, d_swapmap, d_status, o, tm, st);
    else
        rc = factor_run<c64, c128>(F, t, (const c128*)d_vals, d_eoff, d_erow, d_ecol, d_eidx, d_fsrc, d_poff, d_lev,
                                   lev_off, d_woff, (c64*)d_cbuf, (c64*)d_zbuf, (c64*)d_ainv, d_swapmap, d_status, o, tm, st);
    if (rc == NDHSS_OK) {
        cudaEventRecord(e1, st);
        DevStatus hs{};
        cudaError_t e = cudaMemcpyAsync(&hs, d_status, sizeof(hs), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        t_done = std::chrono::steady_clock::now();
        if (e != cudaSuccess) {
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_factor: %s", cudaGetErrorString(e));
        } else if (hs.code == (int)NDHSS_ERR_TIMEOUT) {
            rc = set_error(NDHSS_ERR_TIMEOUT, "ndhss_factor: a tensor-core update of level %d did not complete", hs.node);
        } else if (hs.code != 0) {
            rc = set_error((ndhss_status)hs.code, "ndhss_factor: zero pivot in A_ii of node %d (level %d)", hs.node,
                           t.level(hs.node));
        } else {
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            F.factor_ms = ms;
            tm.collect(F);
        }
    }
    if (rc == NDHSS_OK && !F.lr_ptr.empty()) {
        int64_t elems = 0;
        for (int s = 0; s < t.nnodes; ++s) {
            const int64_t mi = t.m_i(s), mb = t.m_b(s);
            elems += mi * mi + (F.lr_ptr[s] ? 2 * (mi + mb) * (int64_t)F.lr_k[s] : 2 * mi * mb);
        }
        F.apply_bytes = elems * (int64_t)esize;
        if (F.ulv) {
            for (int s = 0; s < t.nnodes; ++s)
                if (F.ulv_root_of[s] >= 0) F.apply_bytes -= (int64_t)t.m_i(s) * t.m_i(s) * (int64_t)esize;
            F.apply_bytes += F.ulv_bytes;
        }
        std::vector<int32_t> lst;
        F.lr_off_l.assign(t.depth + 1, 0);
        F.lr_cnt.assign(t.depth + 1, 0);
        for (int l = 0; l <= t.depth; ++l) {
            F.lr_off_l[l] = (int64_t)lst.size();
            for (int s : F.levels[l])
                if (F.lr_ptr[s] && F.lr_k[s] > 0) lst.push_back(s);
            F.lr_cnt[l] = (int64_t)lst.size() - F.lr_off_l[l];
        }
        // each low-rank node's slot for the apply's per-chunk partial products
        std::vector<int64_t>& toff = F.lr_toff;
        toff.assign(t.nnodes, 0);
        F.lr_t_total = 0;
        for (int s = 0; s < t.nnodes; ++s)
            if (F.lr_ptr[s] && F.lr_k[s] > 0) {
                const int64_t nch = (std::max(t.m_i(s), t.m_b(s)) + LR_CHUNK - 1) / LR_CHUNK;
                toff[s] = F.lr_t_total;
                F.lr_t_total += nch * F.lr_k[s];
            }
        if (upload(&F.d_lr_ptr, F.lr_ptr.data(), F.lr_ptr.size(), &F.dev_bytes, st) != NDHSS_OK ||
            upload(&F.d_lr_k, F.lr_k.data(), F.lr_k.size(), &F.dev_bytes, st) != NDHSS_OK ||
            upload(&F.d_lr_list, lst.data(), lst.size(), &F.dev_bytes, st) != NDHSS_OK)
            rc = set_error(NDHSS_ERR_OOM, "ndhss_factor: low-rank tables");
    }
    cleanup();
    if (rc == NDHSS_OK) rc = build_apply_schedule(F, st);
    if (rc == NDHSS_OK) rc = build_multi_plan(F, st);
    if (rc != NDHSS_OK) {
        cudaStreamSynchronize(st);
        ndhss_factor_destroy(h);
        return rc;
    }
    F.host_tail_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_done).count();
    *out = h;
    return NDHSS_OK;
}

template <typename T, typename V>
static void convert_block(const T* src, V* dst, int64_t rows, int64_t cols, int64_t ldsrc, int64_t lddst,
                          const int32_t* colperm, double sign);

template <>
void convert_block<double, double>(const double* src, double* dst, int64_t rows, int64_t cols, int64_t ls, int64_t ld,
                                   const int32_t* cp, double sign) {
    for (int64_t j = 0; j < cols; ++j)
        for (int64_t i = 0; i < rows; ++i) dst[(cp ? cp[j] : j) * ld + i] = sign * src[j * ls + i];
}
template <>
void convert_block<float, double>(const float* src, double* dst, int64_t rows, int64_t cols, int64_t ls, int64_t ld,
                                  const int32_t* cp, double sign) {
    for (int64_t j = 0; j < cols; ++j)
        for (int64_t i = 0; i < rows; ++i) dst[(cp ? cp[j] : j) * ld + i] = sign * (double)src[j * ls + i];
}
template <>
void convert_block<c128, c128>(const c128* src, c128* dst, int64_t rows, int64_t cols, int64_t ls, int64_t ld,
                               const int32_t* cp, double sign) {
    for (int64_t j = 0; j < cols; ++j)
        for (int64_t i = 0; i < rows; ++i) {
            const c128 v = src[j * ls + i];
            dst[(cp ? cp[j] : j) * ld + i] = {sign * v.x, sign * v.y};
        }
}
template <>
void convert_block<c64, c128>(const c64* src, c128* dst, int64_t rows, int64_t cols, int64_t ls, int64_t ld,
                              const int32_t* cp, double sign) {
    for (int64_t j = 0; j < cols; ++j)
        for (int64_t i = 0; i < rows; ++i) {
            const c64 v = src[j * ls + i];
            dst[(cp ? cp[j] : j) * ld + i] = {sign * (double)v.x, sign * (double)v.y};
        }
}

static ndhss_status get_block_impl(const ndhss_factorization* fh, int32_t node, int32_t which, void* host_out, int64_t ld) {
    if (!fh || !host_out) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor_get_block: NULL argument");
    const FactorData& F = fh->f;
    if (node < 0 || node >= F.nnodes || which < 0 || which > 3)
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor_get_block: bad node %d or block %d", node, which);
    const int64_t mi = F.m_i(node), mb = F.m_b(node), m = mi + mb;
    const int64_t rows = (which == 0 || which == 1) ? mi : mb;
    const int64_t cols = (which == 0 || which == 2) ? mi : mb;
    if (ld < std::max<int64_t>(rows, 1)) return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor_get_block: ld too small");
    if (rows == 0 || cols == 0) return NDHSS_OK;
    if ((which == 1 || which == 2) && !F.lr_ptr.empty() && F.lr_ptr[node]) {
        // low-rank R = X R(J, :): X (m_i x k) then R(J, :)^T (m_b x k); L = R^T
        const int64_t k = F.lr_k[node];
        std::vector<unsigned char> lb((size_t)(mi * k + k * mb) * F.esize);
        NDHSS_CUDA_TRY(cudaDeviceSynchronize());
        if (!lb.empty())
            NDHSS_CUDA_TRY(cudaMemcpy(lb.data(), reinterpret_cast<const void*>(F.lr_ptr[node]), lb.size(), cudaMemcpyDeviceToHost));
        const bool cplx = F.vtype == NDHSS_C128;
        for (int64_t j = 0; j < mb; ++j)
            for (int64_t i = 0; i < mi; ++i) {
                double re = 0, im = 0;
                for (int64_t a = 0; a < k; ++a) {
                    double xr, xi, rr, ri;
                    const size_t xo = (size_t)(a * mi + i), ro = (size_t)(mi * k + a * mb + j);
                    if (!cplx && F.prec == NDHSS_FP64) { xr = ((double*)lb.data())[xo]; rr = ((double*)lb.data())[ro]; xi = ri = 0; }
                    else if (!cplx) { xr = ((float*)lb.data())[xo]; rr = ((float*)lb.data())[ro]; xi = ri = 0; }
                    else if (F.prec == NDHSS_FP64) {
                        const c128 x = ((c128*)lb.data())[xo], r = ((c128*)lb.data())[ro];
                        xr = x.x; xi = x.y; rr = r.x; ri = r.y;
                    } else {
                        const c64 x = ((c64*)lb.data())[xo], r = ((c64*)lb.data())[ro];
                        xr = x.x; xi = x.y; rr = r.x; ri = r.y;
                    }
                    re += xr * rr - xi * ri;
                    im += xr * ri + xi * rr;
                }
                const int64_t di = (which == 1) ? i : j, dj = (which == 1) ? j : i;
                if (cplx) ((c128*)host_out)[dj * ld + di] = {re, im};
                else ((double*)host_out)[dj * ld + di] = re;
            }
        return NDHSS_OK;
    }
    std::vector<unsigned char> buf((size_t)(m * m) * F.esize);
    NDHSS_CUDA_TRY(cudaDeviceSynchronize());
    NDHSS_CUDA_TRY(cudaMemcpy(buf.data(), (const unsigned char*)F.d_front + (size_t)F.foff[node] * F.esize, buf.size(),
                              cudaMemcpyDeviceToHost));
    std::vector<int32_t> sig;
    if (which == 0 || which == 2) {
        sig.resize(mi);
        NDHSS_CUDA_TRY(cudaMemcpy(sig.data(), F.d_sigma + F.info(node, 4), mi * 4, cudaMemcpyDeviceToHost));
    }
    const int64_t r0 = (which == 0 || which == 1) ? 0 : mi;
    const int64_t c0 = (which == 0 || which == 2) ? 0 : mi;
    const int32_t* cp = sig.empty() ? nullptr : sig.data();
    const double sign = (which == 2) ? -1.0 : 1.0;
    const bool cplx = F.vtype == NDHSS_C128;
    const size_t off = (size_t)(c0 * m + r0);
    if (!cplx && F.prec == NDHSS_FP64)
        convert_block<double, double>((const double*)buf.data() + off, (double*)host_out, rows, cols, m, ld, cp, sign);
    else if (!cplx)
        convert_block<float, double>((const float*)buf.data() + off, (double*)host_out, rows, cols, m, ld, cp, sign);
    else if (F.prec == NDHSS_FP64)
        convert_block<c128, c128>((const c128*)buf.data() + off, (c128*)host_out, rows, cols, m, ld, cp, sign);
    else
        convert_block<c64, c128>((const c64*)buf.data() + off, (c128*)host_out, rows, cols, m, ld, cp, sign);
    return NDHSS_OK;
}

}  // namespace ndhss

extern "C" {

ndhss_status ndhss_factor(const ndhss_tree* t, int32_t vtype, const int32_t* d_rowptr, const int32_t* d_col,
                          const void* d_vals, const ndhss_factor_opts* opts, void* stream, ndhss_factorization** out) {
    return ::ndhss::guarded("ndhss_factor", [&]() -> ndhss_status {
        ndhss::clear_error();
        return ndhss::factor_impl(t, vtype, d_rowptr, d_col, d_vals, opts, stream, out);
    });
}

ndhss_status ndhss_factor_get_block(const ndhss_factorization* f, int32_t node, int32_t which, void* host_out, int64_t ld) {
    return ::ndhss::guarded("ndhss_factor_get_block", [&]() -> ndhss_status {
        ndhss::clear_error();
        return ndhss::get_block_impl(f, node, which, host_out, ld);
    });
}

ndhss_status ndhss_factor_stats_get(const ndhss_factorization* fh, ndhss_factor_stats* st) {
    ndhss::clear_error();
    if (!fh || !st) return ndhss::set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor_stats_get: NULL argument");
    const auto& F = fh->f;
    st->n = F.n;
    st->nnodes = F.nnodes;
    st->depth = F.depth;
    st->front_elems = F.front_elems;
    st->apply_bytes = F.apply_bytes;
    st->factor_bytes = F.dev_bytes;
    st->factor_ms = F.factor_ms;
    st->kmax = F.kmax;
    st->prec = F.prec;
    st->launches = F.launches;
    for (int k = 0; k < 8; ++k) {
        st->class_ms[k] = F.class_ms[k];
        st->class_launches[k] = F.class_launches[k];
    }
    st->update_flops = F.update_flops;
    st->tc_flops = F.tc_flops;
    st->host_setup_ms = F.host_setup_ms;
    st->host_tail_ms = F.host_tail_ms;
    return NDHSS_OK;
}

void ndhss_factor_destroy(ndhss_factorization* fh) {
    if (!fh) return;
    auto& F = fh->f;
    // everything below came from the library's stream-ordered pool; work on
    // any stream may still read it, so wait for the device first
    cudaDeviceSynchronize();
    for (void* p : {(void*)F.d_node, (void*)F.d_foff, (void*)F.d_blist, (void*)F.d_perm, (void*)F.d_sigma,
                    (void*)F.d_ipiv, F.d_front, (void*)F.d_lr_ptr, (void*)F.d_lr_k, (void*)F.d_lr_list, (void*)F.d_sched,
                    (void*)F.d_need, (void*)F.d_wdesc, (void*)F.d_apply_err, (void*)F.d_mjobs, (void*)F.d_mlr, (void*)F.d_sublist,
                    (void*)F.d_sched_dep})
        if (p) cudaFreeAsync(p, 0);
    for (void* b : F.lr_bufs)
        if (b) cudaFreeAsync(b, 0);
    for (void* b : F.ulv_bufs)
        if (b) cudaFreeAsync(b, 0);
    if (F.d_ulv_ord) cudaFreeAsync(F.d_ulv_ord, 0);
    if (F.d_ulvdev) cudaFreeAsync(F.d_ulvdev, 0);
    cudaStreamSynchronize(0);
    delete fh;
}

}  // extern "C"
