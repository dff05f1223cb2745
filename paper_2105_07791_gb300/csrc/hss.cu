// Randomized HSS compression of Schur complements (Alg. A.1) and low-rank
// Gauss transforms (Sec. 3.4) for the fronts of one tree level, in the
// dense-then-compress form of Alg. 3.4: the fronts are already eliminated
// densely; S^sigma is compressed with the parent-conforming cluster tree of
// Fig. 4 and replaced by its HSS reconstruction (so the parent assembles the
// compressed Schur complement), and strictly above the switching level
// R^sigma is replaced by a row interpolative decomposition R ~ X R(J, :) used
// by the apply (with L = R^T, A symmetric).
//
// All fronts of the level are compressed together, round by round: every
// front still active in a round has the same number p of samples; the
// estimator (Eq. 2.7) on r fresh samples retires the fronts that meet eps and
// the others continue with p + r samples (all previous samples reused).
//
// Gaussian samples are Philox4x32-10 (Salmon et al., SC'11) + Box-Muller with
// the same (seed, stream, element) mapping as the oracle, so both draw the
// same matrices.  Per HSS node one CTA forms the local sample block, computes
// its row interpolative decomposition by Householder QR with column pivoting
// (Businger-Golub) of S_loc^T, and passes Omega_i = U_i^T Omega_loc and
// S_i = S_loc(J_i, :) upward.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>
#include <memory>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "factor.cuh"
#include "ulv.cuh"

namespace ndhss {
namespace {

constexpr int HT = 256;
constexpr int OVERSAMPLE_MIN = 10;   // the rank may use at most (samples - 10) columns
constexpr int MAX_SAMPLES = 256;     // samples per block (the row ID keeps a column in 8 registers x 32 lanes)

// 10^3 unit roundoffs of the working precision, relative to a block's norm
template <typename T> constexpr double stagnation_floor() {
    return sizeof(typename Tr<T>::real) == 4 ? 1e3 * 5.9604644775390625e-8 : 1e3 * 1.1102230246251565e-16;
}

// ----------------------------------------------------------------- Philox
__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                             uint32_t k1) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

// Four standard normals of counter block `blk` of stream `stream`.
__device__ void philox_normals(uint64_t seed, uint64_t stream, uint64_t blk, double out[4]) {
    uint32_t c0 = (uint32_t)blk, c1 = (uint32_t)stream, c2 = (uint32_t)(stream >> 32), c3 = 0;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        philox_round(c0, c1, c2, c3, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    const double u0 = ((double)c0 + 0.5) / 4294967296.0, u1 = ((double)c1 + 0.5) / 4294967296.0;
    const double u2 = ((double)c2 + 0.5) / 4294967296.0, u3 = ((double)c3 + 0.5) / 4294967296.0;
    const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    const double pi2 = 6.283185307179586476925286766559;
    out[0] = r0 * cos(pi2 * u1);
    out[1] = r0 * sin(pi2 * u1);
    out[2] = r1 * cos(pi2 * u3);
    out[3] = r1 * sin(pi2 * u3);
}

__device__ __forceinline__ double shfl_xor_h(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_xor_h(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <typename R>
__device__ __forceinline__ Cx<R> shfl_xor_h(Cx<R> v, int o) {
    return {__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}

__host__ __device__ __forceinline__ int rows_cap_even(int r) { return (r + 1) & ~1; }

template <typename T> __device__ __forceinline__ T real_to(double v);
template <> __device__ __forceinline__ double real_to<double>(double v) { return v; }
template <> __device__ __forceinline__ float real_to<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ c128 real_to<c128>(double v) { return {v, 0.0}; }
template <> __device__ __forceinline__ c64 real_to<c64>(double v) { return {(float)v, 0.0f}; }

__device__ __forceinline__ double nrm2v(double a) { return a * a; }
__device__ __forceinline__ double nrm2v(float a) { return (double)a * a; }
__device__ __forceinline__ double nrm2v(c128 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double nrm2v(c64 a) { return (double)a.x * a.x + (double)a.y * a.y; }
// |a|^2 in the element's own real type (GB300's FP64 pipe is narrow: FP32 paths stay FP32)
__device__ __forceinline__ double nrm2r(double a) { return a * a; }
__device__ __forceinline__ float nrm2r(float a) { return a * a; }
__device__ __forceinline__ double nrm2r(c128 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float nrm2r(c64 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double absv(double a) { return fabs(a); }
__device__ __forceinline__ double absv(float a) { return fabs((double)a); }
__device__ __forceinline__ double absv(c128 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double absv(c64 a) { return hypot((double)a.x, (double)a.y); }

// One Gaussian block: dst(i, col0 + j) for i < rows, j < cols (element e = i + j*rows of the stream).
struct GaussJob {
    void* dst;
    int64_t ld;
    int rows, cols, col0;
    uint64_t stream;
};

// Four standard normals in single precision (same Philox words, float Box-Muller).
__device__ void philox_normals_f(uint64_t seed, uint64_t stream, uint64_t blk, double out[4]) {
    uint32_t c0 = (uint32_t)blk, c1 = (uint32_t)stream, c2 = (uint32_t)(stream >> 32), c3 = 0;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        philox_round(c0, c1, c2, c3, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    const float s = 2.3283064365386963e-10f;            // 2^-32
    const float u0 = ((float)c0 + 0.5f) * s, u1 = ((float)c1 + 0.5f) * s;
    const float u2 = ((float)c2 + 0.5f) * s, u3 = ((float)c3 + 0.5f) * s;
    const float r0 = sqrtf(-2.0f * logf(fmaxf(u0, 1e-38f))), r1 = sqrtf(-2.0f * logf(fmaxf(u2, 1e-38f)));
    float s1, cs1, s3, cs3;
    sincospif(2.0f * u1, &s1, &cs1);
    sincospif(2.0f * u3, &s3, &cs3);
    out[0] = r0 * cs1;
    out[1] = r0 * s1;
    out[2] = r1 * cs3;
    out[3] = r1 * s3;
}

template <typename T>
__global__ void gauss_kernel(const GaussJob* __restrict__ jobs, uint64_t seed) {
    const GaussJob jb = jobs[blockIdx.y];
    T* dst = static_cast<T*>(jb.dst);
    const int64_t n = (int64_t)jb.rows * jb.cols;
    for (int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; blk * 4 < n; blk += (int64_t)gridDim.x * blockDim.x) {
        double z[4];
        if (sizeof(typename Tr<T>::real) == 4) philox_normals_f(seed, jb.stream, (uint64_t)blk, z);
        else philox_normals(seed, jb.stream, (uint64_t)blk, z);
        for (int q = 0; q < 4; ++q) {
            const int64_t e = blk * 4 + q;
            if (e < n) {
                const int64_t i = e % jb.rows, j = e / jb.rows;
                dst[(jb.col0 + j) * jb.ld + i] = real_to<T>(z[q]);
            }
        }
    }
}

// c + a * b for a complex a and a real b (the products of a complex block
// with a real Gaussian sample matrix): the values of fmac with b's imaginary
// part zero, in two FMAs instead of four
template <typename R>
__device__ __forceinline__ Cx<R> fmar(Cx<R> a, R b, Cx<R> c) {
    c.x = fma(a.x, b, c.x);
    c.y = fma(a.y, b, c.y);
    return c;
}

// ------------------------------------------------------- batched GEMM
// C = (beta ? C : 0) + alpha * A * B, column-major, A M x K, B K x N.
struct GemmJob {
    const void* A;
    const void* B;
    void* C;
    int64_t lda, ldb, ldc;
    int M, N, K, beta;
    double alpha;
    int transA = 0, transB = 0;   // operand stored transposed (plain transpose, no conjugation)
    int realB = 0;                // complex T: B holds real values (zero imaginary parts); 2 FMAs per product
};

// 64 x 64 tiles of every job; blockIdx.z = job * ksplit + split.  The K
// chunks are staged in shared memory, the next chunk's loads in registers
// while the current chunk is multiplied.  ksplit > 1: the CTA of split q
// takes K chunks q, q + ksplit, ... and writes its raw partial tile to
// part[(z * tiles + tile) * 4096]; bgemm_reduce_kernel adds the partials in
// split order (deterministic) and applies alpha / beta.
template <typename T, bool RB>
__global__ void __launch_bounds__(256) bgemm_kernel(const GemmJob* __restrict__ jobs, int ksplit, T* __restrict__ part) {
    constexpr int TT = 64, TK = 16;
    __shared__ T sA[TK][TT];
    __shared__ T sB[TK][TT];
    const int job = blockIdx.z / ksplit, split = blockIdx.z % ksplit;
    const GemmJob jb = jobs[job];
    const int64_t i0 = (int64_t)blockIdx.x * TT, j0 = (int64_t)blockIdx.y * TT;
    if (i0 >= jb.M || j0 >= jb.N) return;
    const T* A = static_cast<const T*>(jb.A);
    const T* B = static_cast<const T*>(jb.B);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = zero<T>();
    // element u of this thread's share of the A and B chunks at K offset kc
    auto a_idx = [&](int u, int& ii, int& l) {
        const int q = tid + 256 * u;
        if (!jb.transA) { ii = q % TT; l = q / TT; } else { l = q % TK; ii = q / TK; }
    };
    auto b_idx = [&](int u, int& jj, int& l) {
        const int q = tid + 256 * u;
        if (!jb.transB) { l = q % TK; jj = q / TK; } else { jj = q % TT; l = q / TT; }
    };
    T ra[4], rb[4];
    auto load = [&](int kc) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int ii, l, jj, lb;
            a_idx(u, ii, l);
            b_idx(u, jj, lb);
            const bool va = kc + l < jb.K && i0 + ii < jb.M, vb = kc + lb < jb.K && j0 + jj < jb.N;
            ra[u] = va ? (!jb.transA ? A[(int64_t)(kc + l) * jb.lda + i0 + ii] : A[(i0 + ii) * jb.lda + kc + l]) : zero<T>();
            rb[u] = vb ? (!jb.transB ? B[(j0 + jj) * jb.ldb + kc + lb] : B[(int64_t)(kc + lb) * jb.ldb + j0 + jj]) : zero<T>();
        }
    };
    const int step = TK * ksplit;
    int kc = split * TK;
    if (kc < jb.K) load(kc);
    for (; kc < jb.K; kc += step) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int ii, l, jj, lb;
            a_idx(u, ii, l);
            b_idx(u, jj, lb);
            sA[l][ii] = ra[u];
            sB[lb][jj] = rb[u];
        }
        __syncthreads();
        if (kc + step < jb.K) load(kc + step);
#pragma unroll
        for (int l = 0; l < TK; ++l) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sA[l][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = sB[l][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if constexpr (RB && Tr<T>::cplx) acc[a][b] = fmar(av[a], bv[b].x, acc[a][b]);
                    else acc[a][b] = fmac(av[a], bv[b], acc[a][b]);
                }
        }
        __syncthreads();
    }
    if (ksplit > 1) {
        T* P = part + ((int64_t)blockIdx.z * gridDim.x * gridDim.y + (int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (TT * TT);
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) P[(ty + 16 * b) * TT + tx + 16 * a] = acc[a][b];
        return;
    }
    using real = typename Tr<T>::real;
    T* Cm = static_cast<T*>(jb.C);
    for (int b = 0; b < 4; ++b) {
        const int64_t j = j0 + ty + 16 * b;
        if (j >= jb.N) continue;
        for (int a = 0; a < 4; ++a) {
            const int64_t i = i0 + tx + 16 * a;
            if (i >= jb.M) continue;
            T* dst = Cm + j * jb.ldc + i;
            const T v = scale(acc[a][b], (real)jb.alpha);
            *dst = jb.beta ? (*dst + v) : v;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) bgemm_reduce_kernel(const GemmJob* __restrict__ jobs, int ksplit,
                                                           const T* __restrict__ part) {
    constexpr int TT = 64;
    const GemmJob jb = jobs[blockIdx.z];
    const int64_t i0 = (int64_t)blockIdx.x * TT, j0 = (int64_t)blockIdx.y * TT;
    if (i0 >= jb.M || j0 >= jb.N) return;
    using real = typename Tr<T>::real;
    T* Cm = static_cast<T*>(jb.C);
    const int64_t tiles = (int64_t)gridDim.x * gridDim.y, tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    for (int e = threadIdx.x; e < TT * TT; e += 256) {
        const int il = e % TT, jl = e / TT;
        const int64_t i = i0 + il, j = j0 + jl;
        if (i >= jb.M || j >= jb.N) continue;
        T acc = zero<T>();
        for (int q = 0; q < ksplit; ++q) acc = acc + part[(((int64_t)blockIdx.z * ksplit + q) * tiles + tile) * (TT * TT) + e];
        T* dst = Cm + j * jb.ldc + i;
        const T v = scale(acc, (real)jb.alpha);
        *dst = jb.beta ? (*dst + v) : v;
    }
}

// ------------------------------------------------------ HSS node tables
struct HFront {
    void* S;          // the dense block being compressed (n x n, ld lds), or R (rows x cols)
    int64_t lds;
    int n;            // S: order; R: rows (m_i)
    int ncol;         // R: columns (m_b); S: n
    void* Om;         // samples (n x p) / R: (ncol x p)
    void* Y;          // S Om (n x p) / R Om (n x p)
    void* Ot;         // fresh samples (n x r) / R: (ncol x r)
    void* Yt;         // S Ot / R Ot (n x r)
    void* Zt;         // HSS(S) Ot / X R(J,:) Ot (n x r)
    void* T1;         // R: R(J,:) Ot (kcap x r)
    void* RJ;         // R: R(J,:) (kcap x ncol)
    int root;         // index of the root HSS node
};

struct HNode {
    int front, lo, hi, level, c1, c2;
    int rows_cap, kcap, p;
    int64_t o_w, o_sl, o_x, o_om, o_si, o_xh, o_yh;   // element offsets in the workspace
    int64_t o_skel, o_iloc, o_piv;                      // int offsets
};

// ---------------------------------------------- per-node small products
// One 64 x 64 tile (rows i0.., columns j0..) of C = A B, K in chunks of 16
// staged in shared memory; the next chunk's loads are in registers while the
// current chunk is multiplied, so a tile waits for memory about once, not
// once per product term.  A(i, l) and B(l, j) come from the caller's
// accessors (gathers allowed); A_KMAJ: consecutive threads load consecutive l
// of A (A stored along K), else consecutive i; B is always loaded along K.
// out(i, j, c) receives every valid entry of the tile.  All 256 threads call it.
constexpr int NT_TILE = 64, NT_K = 16;

__host__ __device__ __forceinline__ int tiles64(int n) { return (n + NT_TILE - 1) / NT_TILE; }

template <typename T, bool A_KMAJ, typename FA, typename FB, typename FO>
__device__ __forceinline__ void tile_gemm64(int M, int N, int K, int i0, int j0, FA fa, FB fb, FO out) {
    __shared__ T sA[NT_K][NT_TILE];
    __shared__ T sB[NT_K][NT_TILE];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = zero<T>();
    T ra[4], rb[4];
    auto load = [&](int kc) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = tid + 256 * u;
            const int ia = A_KMAJ ? q / NT_K : q % NT_TILE, la = A_KMAJ ? q % NT_K : q / NT_TILE;
            ra[u] = (kc + la < K && i0 + ia < M) ? fa(i0 + ia, kc + la) : zero<T>();
            const int jb = q / NT_K, lb = q % NT_K;
            rb[u] = (kc + lb < K && j0 + jb < N) ? fb(kc + lb, j0 + jb) : zero<T>();
        }
    };
    load(0);
    for (int kc = 0; kc < K; kc += NT_K) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = tid + 256 * u;
            const int ia = A_KMAJ ? q / NT_K : q % NT_TILE, la = A_KMAJ ? q % NT_K : q / NT_TILE;
            sA[la][ia] = ra[u];
            sB[q % NT_K][q / NT_K] = rb[u];
        }
        __syncthreads();
        if (kc + NT_K < K) load(kc + NT_K);
#pragma unroll
        for (int l = 0; l < NT_K; ++l) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sA[l][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = sB[l][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmac(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = j0 + ty + 16 * b;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + tx + 16 * a;
            if (i < M && j < N) out(i, j, acc[a][b]);
        }
    }
}

// S_loc^T into W (p x rows, ld p) and S_loc into SL (rows x p, ld rows_cap); iloc = global rows.
// Leaf: S_loc = Y(I, :) - S(I, I) Om(I, :).  Inner node: the children's
// skeleton rows, S_loc = [S_c1(J1, :) - S(J1, J2) Om_c2; S_c2(J2, :) - S(J2, J1) Om_c1].
// Grid: (nodes, tiles): a leaf's tiles cover rows x p; an inner node's two
// parts (rows of c1, rows of c2) ceil(kcap / 64) row tiles each.
template <typename T>
__global__ void __launch_bounds__(HT)
form_sloc_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes, const HFront* __restrict__ fronts,
                 T* __restrict__ ws, int* __restrict__ iws, int* __restrict__ kk, int* __restrict__ rows_out) {
    const HNode nd = nodes[list[blockIdx.x]];
    const HFront fr = fronts[nd.front];
    const T* S = static_cast<const T*>(fr.S);
    const T* Om = static_cast<const T*>(fr.Om);
    const T* Y = static_cast<const T*>(fr.Y);
    const int64_t n = fr.n, lds = fr.lds;
    const int p = nd.p;
    T* W = ws + nd.o_w;
    T* SL = ws + nd.o_sl;
    int* iloc = iws + nd.o_iloc;
    const int tn = tiles64(p);
    const int t = blockIdx.y;
    if (nd.c1 < 0) {
        const int rows = nd.hi - nd.lo;
        const int i0 = (t / tn) * NT_TILE, j0 = (t % tn) * NT_TILE;
        if (t == 0) {
            for (int r = threadIdx.x; r < rows; r += HT) iloc[r] = nd.lo + r;
            if (threadIdx.x == 0) rows_out[list[blockIdx.x]] = rows;
        }
        if (i0 >= rows) return;
        tile_gemm64<T, false>(
            rows, p, rows, i0, j0, [&](int r, int c) { return -S[(int64_t)(nd.lo + c) * lds + nd.lo + r]; },
            [&](int c, int j) { return Om[(int64_t)j * n + nd.lo + c]; },
            [&](int r, int j, T acc) {
                acc = acc + Y[(int64_t)j * n + nd.lo + r];
                W[(int64_t)r * p + j] = acc;
                SL[(int64_t)j * nd.rows_cap + r] = acc;
            });
    } else {
        const HNode a = nodes[nd.c1], b = nodes[nd.c2];
        const int k1 = kk[nd.c1], k2 = kk[nd.c2];
        const int* sk1 = iws + a.o_skel;
        const int* sk2 = iws + b.o_skel;
        if (t == 0) {
            for (int r = threadIdx.x; r < k1 + k2; r += HT) iloc[r] = (r < k1) ? sk1[r] : sk2[r - k1];
            if (threadIdx.x == 0) rows_out[list[blockIdx.x]] = k1 + k2;
        }
        const int tm = tiles64(nd.kcap);
        const int part = t / (tm * tn), tt = t % (tm * tn);
        const int i0 = (tt / tn) * NT_TILE, j0 = (tt % tn) * NT_TILE;
        // part 0: rows of c1 (coupled to c2's skeleton), part 1: rows of c2
        const int M = part == 0 ? k1 : k2, K = part == 0 ? k2 : k1, roff = part == 0 ? 0 : k1;
        if (part > 1 || i0 >= M) return;
        const int* own = part == 0 ? sk1 : sk2;
        const int* oth = part == 0 ? sk2 : sk1;
        const T* Sown = ws + (part == 0 ? a.o_si : b.o_si);
        const T* Ooth = ws + (part == 0 ? b.o_om : a.o_om);
        const int kcown = part == 0 ? a.kcap : b.kcap, kcoth = part == 0 ? b.kcap : a.kcap;
        tile_gemm64<T, false>(
            M, p, K, i0, j0, [&](int r, int c) { return -S[(int64_t)oth[c] * lds + own[r]]; },
            [&](int c, int j) { return Ooth[(int64_t)j * kcoth + c]; },
            [&](int r, int j, T acc) {
                acc = acc + Sown[(int64_t)j * kcown + r];
                W[(int64_t)(roff + r) * p + j] = acc;
                SL[(int64_t)j * nd.rows_cap + roff + r] = acc;
            });
    }
}

// Row interpolative decomposition of S_loc from a Householder QR with column
// pivoting (largest remaining norm, first index on ties) of W = S_loc^T.
// Rank = number of steps with pivot norm > eps * (first pivot norm), at most
// kmax.  Output: kk[node] = k, piv (local rows, first k = skeleton J),
// X (rows x k, ld rows_cap) with X(J, :) = I.
template <typename T>
__global__ void __launch_bounds__(512)
row_id_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes, T* __restrict__ ws,
              int* __restrict__ iws, int* __restrict__ kk, const int* __restrict__ rows_in, double eps, int rank_cap,
              int w_in_smem) {
    using real = typename Tr<T>::real;
    constexpr int CH = 8;                // column entries per lane held in registers (p <= 256)
    extern __shared__ __align__(16) unsigned char smem[];
    const int id = list[blockIdx.x];
    const HNode nd = nodes[id];
    const int rows = rows_in[id], p = nd.p;
    int* piv = iws + nd.o_piv;
    const int rr = (rows_cap_even(nd.rows_cap));
    double* nrm = reinterpret_cast<double*>(smem);          // remaining squared column norms
    T* vsh = reinterpret_cast<T*>(nrm + rr);                 // reflector (p), 16-byte aligned
    T* W = ws + nd.o_w;                                      // p x rows, column c = row c of S_loc
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5, NT = blockDim.x;
    int ldw = p;                          // column stride of W
    if (w_in_smem) {
        // staged copy with an odd column stride: thread-per-column loops stay free of bank conflicts
        T* Ws = vsh + ((p + 1) & ~1);
        const int lds = p | 1;
        for (int64_t q = tid; q < (int64_t)p * rows; q += NT) Ws[(q / p) * lds + q % p] = W[q];
        W = Ws;
        ldw = lds;
        __syncthreads();
    }
    __shared__ double s_val[32];
    __shared__ int s_idx[32];
    __shared__ double s_r11, s_bestv, s_vn2;
    __shared__ int s_best;
    __shared__ T s_beta;
    for (int c = warp; c < rows; c += NW) {
        const T* col = W + (int64_t)c * ldw;
        real sacc = real(0);
        for (int j = lane; j < p; j += 32) sacc += nrm2r(col[j]);
        for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        if (lane == 0) nrm[c] = (double)sacc;
    }
    for (int c = tid; c < rows; c += NT) piv[c] = c;
    const int kmax = min(min(nd.kcap, rank_cap), min(p, rows));
    int t = 0;
    __syncthreads();
    for (; t < min(p, rows); ++t) {
        double best = -1.0;
        int bi = INT_MAX;
        for (int c = t + tid; c < rows; c += NT) {
            const double v = nrm[c];
            if (v > best) { best = v; bi = c; }
        }
        for (int o = 16; o; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            double bv = lane < NW ? s_val[lane] : -1.0;
            int bb = lane < NW ? s_idx[lane] : INT_MAX;
            for (int o = 16; o; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, bv, o);
                const int oi = __shfl_down_sync(0xffffffffu, bb, o);
                if (ov > bv || (ov == bv && oi < bb)) { bv = ov; bb = oi; }
            }
            if (lane == 0) {
                s_best = bb;
                s_bestv = sqrt(fmax(bv, 0.0));
                if (t == 0) s_r11 = s_bestv;
            }
        }
        __syncthreads();
        const int cb = s_best;
        if (t >= kmax || cb == INT_MAX || !(s_bestv > eps * s_r11)) break;
        if (cb != t) {
            for (int j = tid; j < p; j += NT) {
                const T a = W[(int64_t)t * ldw + j];
                W[(int64_t)t * ldw + j] = W[(int64_t)cb * ldw + j];
                W[(int64_t)cb * ldw + j] = a;
            }
            if (tid == 0) {
                const int a = piv[t];
                piv[t] = piv[cb];
                piv[cb] = a;
                const double n1 = nrm[t];
                nrm[t] = nrm[cb];
                nrm[cb] = n1;
            }
        }
        __syncthreads();
        // reflector v = x - beta e1 of x = W(t:p, t), beta = -phase(x0) ||x||
        T* xcol = W + (int64_t)t * ldw;
        for (int j = t + tid; j < p; j += NT) vsh[j] = xcol[j];
        __syncthreads();
        if (tid == 0) {
            const double xn = s_bestv;
            const T a0 = vsh[t];
            const double aa = absv(a0);
            T ph = one<T>();
            if (aa > 0) ph = scale(a0, (real)(1.0 / aa));
            const T beta = scale(ph, (real)(-xn));
            const T v0 = a0 - beta;
            s_vn2 = xn * xn - aa * aa + nrm2v(v0);
            vsh[t] = v0;
            s_beta = beta;
        }
        __syncthreads();
        const double vn2 = s_vn2;
        if (vn2 > 0) {
            const real f = (real)(2.0 / vn2);
            T vl[CH];
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                const int j = t + lane + 32 * q;
                vl[q] = (j < p) ? vsh[j] : zero<T>();
            }
            for (int c = t + 1 + warp; c < rows; c += NW) {
                T* col = W + (int64_t)c * ldw;
                T cv[CH];
                T w = zero<T>();
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    const int j = t + lane + 32 * q;
                    cv[q] = (j < p) ? col[j] : zero<T>();
                }
#pragma unroll
                for (int q = 0; q < CH; ++q) w = fmac(conjv(vl[q]), cv[q], w);
                for (int o = 16; o; o >>= 1) w = w + shfl_xor_h(w, o);
                const T g = scale(w, f);
                real sacc = real(0);
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    const int j = t + lane + 32 * q;
                    if (j < p) {
                        const T u = cv[q] - vl[q] * g;
                        col[j] = u;
                        if (j > t) sacc += nrm2r(u);
                    }
                }
                for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                if (lane == 0) nrm[c] = (double)sacc;
            }
        }
        __syncthreads();
        if (tid == 0) xcol[t] = s_beta;
        __syncthreads();
    }
    const int k = t;
    // T = R11^{-1} R12 in place of R12 (one column per thread)
    for (int c = k + tid; c < rows; c += NT) {
        T* col = W + (int64_t)c * ldw;
        for (int i = k - 1; i >= 0; --i) {
            T acc = col[i];
            for (int l = i + 1; l < k; ++l) acc = fmac(-W[(int64_t)l * ldw + i], col[l], acc);
            col[i] = acc * recip(W[(int64_t)i * ldw + i]);
        }
    }
    __syncthreads();
    T* X = ws + nd.o_x;
    for (int q = tid; q < rows * k; q += NT) {
        const int i = q % rows, a = q / rows;
        T v;
        if (i < k) v = (i == a) ? one<T>() : zero<T>();
        else v = W[(int64_t)i * ldw + a];
        X[(int64_t)a * nd.rows_cap + piv[i]] = v;
    }
    if (tid == 0) kk[id] = k;
}

// The same row ID with the columns of W = S_loc^T split over the C CTAs of a
// thread-block cluster (C = 1: one CTA), every CTA holding its share in shared
// memory.  A pivot step is one cluster barrier (the CTAs' per-warp candidates
// of the next pivot become visible and every warp reduces them through
// distributed shared memory), the copy of the pivot column from its owner, one
// CTA barrier and the reflection of the remaining local columns, which also
// yields their new norms and the next candidates.  A column is reflected by a
// segment of LPC lanes (LPC = 8, 16 or 32 as p <= 64, 128, 256; 8 entries per
// lane), so a warp works on 32 / LPC columns at once.  Columns never move: a
// pivot is flagged, the pivot order kept, and R11 = R(0:k, 0:k) gathered at
// the end.  Ties of the pivot norm go to the lowest row index.
constexpr int RID_THREADS = 256;
constexpr int RID_NW = RID_THREADS / 32;
constexpr int RID_KMAX = 256;                 // ranks stay below the 256-sample limit
constexpr int RID_MAX_CLUSTER = 8;
constexpr size_t RID_SMEM = 200 * 1024;       // dynamic shared memory of one CTA's share
constexpr int RID_SPLIT_COLS = 128;

__host__ __device__ __forceinline__ int rid_lpc(int p) { return p <= 64 ? 8 : p <= 128 ? 16 : 32; }

template <typename T>
__device__ __forceinline__ T seg_sum(T v, int lpc) {
    for (int o = lpc >> 1; o; o >>= 1) v = v + shfl_xor_h(v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(RID_THREADS, sizeof(T) > 8 ? 2 : 4)
row_id_cluster_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes, T* __restrict__ ws,
                      int* __restrict__ iws, int* __restrict__ kk, const int* __restrict__ rows_in, double eps,
                      int rank_cap) {
    using real = typename Tr<T>::real;
    namespace cg = cooperative_groups;
    constexpr int CH = 8;                        // column entries per lane in registers
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rk = (int)cl.block_rank();
    const int id = list[blockIdx.x / C];
    const HNode nd = nodes[id];
    const int rows = rows_in[id], p = nd.p;
    const int chunk = (rows + C - 1) / C;
    const int c_lo = min(rows, rk * chunk);
    const int nloc = min(rows, c_lo + chunk) - c_lo;
    const int lds = p | 1;                       // odd column stride: per-column loops free of bank conflicts
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lpc = rid_lpc(p), spw = 32 / lpc;  // lanes per column, columns per warp
    const int seg = lane / lpc, sl = lane % lpc;
    extern __shared__ __align__(16) unsigned char smem[];
    T* Ws = reinterpret_cast<T*>(smem);          // nloc columns of W, ld lds
    unsigned char* used = reinterpret_cast<unsigned char*>(Ws + (size_t)lds * chunk + p + 1);
    __shared__ real s_cv[2][RID_NW];
    __shared__ int s_ci[2][RID_NW];
    __shared__ T s_beta[RID_KMAX];
    __shared__ int s_order[RID_KMAX];
    const T* Wg = ws + nd.o_w;
    for (int q = tid; q < p * nloc; q += RID_THREADS) {
        const int c = q / p, j = q % p;
        Ws[(size_t)c * lds + j] = Wg[(int64_t)(c_lo + c) * p + j];
    }
    for (int c = tid; c < nloc; c += RID_THREADS) used[c] = 0;
    __syncthreads();
    // the warp's best candidate (squared norm, row) over its segments, to s_cv/s_ci[par]
    auto publish = [&](real best, int nb, int par) {
        real wv;
        const int wi = warp_argmax(best, nb, nb != INT_MAX, &wv);
        if (lane == 0) { s_cv[par][warp] = wv; s_ci[par][warp] = wi; }
    };
    {
        real best = real(-1);
        int nb = INT_MAX;
        for (int c0 = warp * spw; c0 < nloc; c0 += RID_NW * spw) {
            const int c = c0 + seg;
            const bool act = c < nloc;
            const T* col = Ws + (size_t)(act ? c : 0) * lds;
            real sacc = real(0);
            for (int j = sl; j < p; j += lpc) sacc += act ? nrm2r(col[j]) : real(0);
            sacc = seg_sum(sacc, lpc);
            if (act && sacc > best) { best = sacc; nb = c_lo + c; }
        }
        publish(best, nb, 0);
    }
    const int kmax = min(min(min(nd.kcap, rank_cap), min(p, rows)), RID_KMAX);
    // pivot scalars in the working precision, computed by every thread (no
    // broadcast barrier; double would run on the narrow FP64 pipe)
    real r11 = real(0);
    const real reps = (real)eps;
    int t = 0;
    for (;; ++t) {
        if (C > 1) cl.sync(); else __syncthreads();
        const int par = t & 1;
        real bv = real(-1);
        int bi = INT_MAX;
        for (int q = lane; q < C * RID_NW; q += 32) {
            const int r = q / RID_NW, w = q % RID_NW;
            real v;
            int i;
            if (C > 1) {
                v = *cl.map_shared_rank(&s_cv[par][w], r);
                i = *cl.map_shared_rank(&s_ci[par][w], r);
            } else {
                v = s_cv[par][w];
                i = s_ci[par][w];
            }
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
        {
            real gv;
            bi = warp_argmax(bv, bi, bi != INT_MAX, &gv);
            bv = gv;
        }
        const real xn = sqrt(bv > real(0) ? bv : real(0));
        if (t == 0) r11 = xn;
        if (t >= kmax || bi == INT_MAX || !(xn > reps * r11)) break;
        const int cb = bi, owner = cb / chunk;
        // the pivot column, read in place by every thread (local or through
        // distributed shared memory): no step writes it from here on
        const T* src = (owner == rk) ? Ws + (size_t)(cb - c_lo) * lds
                                     : cl.map_shared_rank(Ws, owner) + (size_t)(cb - owner * chunk) * lds;
        if (tid == 0) {
            s_order[t] = cb;
            if (owner == rk) used[cb - c_lo] = 1;    // read from the next step on (after its barrier)
        }
        // reflector v = x - beta e_t of the pivot column x, beta = -phase(x_t) ||x||
        const T a0 = src[t];
        const real aa2 = nrm2r(a0), aa = sqrt(aa2);
        T ph = one<T>();
        if (aa > real(0)) ph = scale(a0, real(1) / aa);
        const T beta = scale(ph, -xn);
        const T v0 = a0 - beta;
        const real vn2 = xn * xn - aa2 + nrm2r(v0);
        if (tid == 0) s_beta[t] = beta;
        const real f = real(2) / vn2;
        T vl[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int j = t + sl + lpc * q;
            vl[q] = (j < p) ? (j == t ? v0 : src[j]) : zero<T>();
        }
        real best = real(-1);
        int nb = INT_MAX;
        for (int c0 = warp * spw; c0 < nloc; c0 += RID_NW * spw) {
            const int c = c0 + seg;
            const bool act = c < nloc && !used[c] && c_lo + c != cb;
            T* col = Ws + (size_t)(act ? c : 0) * lds;
            T cv[CH];
            T w = zero<T>();
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                const int j = t + sl + lpc * q;
                cv[q] = (act && j < p) ? col[j] : zero<T>();
            }
#pragma unroll
            for (int q = 0; q < CH; ++q) w = fmac(conjv(vl[q]), cv[q], w);
            w = seg_sum(w, lpc);
            const T g = scale(w, f);
            real sacc = real(0);
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                const int j = t + sl + lpc * q;
                if (act && j < p) {
                    const T u = cv[q] - vl[q] * g;
                    col[j] = u;
                    if (j > t) sacc += nrm2r(u);
                }
            }
            sacc = seg_sum(sacc, lpc);
            if (act && sacc > best) { best = sacc; nb = c_lo + c; }
        }
        publish(best, nb, par ^ 1);
    }
    const int k = t;
    // R11 stays in the pivot columns, in the shared memory of their owners
    // (the pivot columns are not written below): one pointer per column,
    // local or through distributed shared memory
    __shared__ const T* s_pcol[RID_KMAX];
    for (int a = tid; a < k; a += RID_THREADS) {
        const int cb = s_order[a], owner = cb / chunk;
        s_pcol[a] = (owner == rk) ? Ws + (size_t)(cb - c_lo) * lds
                                  : cl.map_shared_rank(Ws, owner) + (size_t)(cb - owner * chunk) * lds;
    }
    if (C > 1) cl.sync(); else __syncthreads();
    // T = R11^{-1} R12 in place of R12 (one column per thread)
    for (int c = tid; c < nloc; c += RID_THREADS) {
        if (used[c]) continue;
        T* col = Ws + (size_t)c * lds;
        for (int i = k - 1; i >= 0; --i) {
            T acc = col[i];
            for (int l = i + 1; l < k; ++l) acc = fmac(-s_pcol[l][i], col[l], acc);
            col[i] = acc * recip(s_beta[i]);
        }
    }
    // no CTA leaves while another may still read its pivot columns
    if (C > 1) cl.sync(); else __syncthreads();
    T* X = ws + nd.o_x;
    int* piv = iws + nd.o_piv;
    for (int q = tid; q < nloc * k; q += RID_THREADS) {
        const int c = q % nloc, a = q / nloc;
        T v;
        if (used[c]) v = (s_order[a] == c_lo + c) ? one<T>() : zero<T>();
        else v = Ws[(size_t)c * lds + a];
        X[(int64_t)a * nd.rows_cap + c_lo + c] = v;
    }
    // piv: skeleton in pivot order, then the other rows in increasing order
    if (rk == 0)
        for (int a = tid; a < k; a += RID_THREADS) piv[a] = s_order[a];
    for (int c = tid; c < nloc; c += RID_THREADS) {
        if (used[c]) continue;
        int below = 0;
        for (int a = 0; a < k; ++a) below += (s_order[a] < c_lo + c) ? 1 : 0;
        piv[k + c_lo + c - below] = c_lo + c;
    }
    if (rk == 0 && tid == 0) kk[id] = k;
}

// Omega_i = X^T Omega_loc, S_i = S_loc(J, :), skeleton = iloc(J).
template <typename T>
__global__ void __launch_bounds__(HT)
finish_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes, const HFront* __restrict__ fronts,
              T* __restrict__ ws, int* __restrict__ iws, const int* __restrict__ kk, const int* __restrict__ rows_in) {
    const int id = list[blockIdx.x];
    const HNode nd = nodes[id];
    const HFront fr = fronts[nd.front];
    const int rows = rows_in[id], k = kk[id], p = nd.p;
    const T* X = ws + nd.o_x;
    const T* SL = ws + nd.o_sl;
    const int* piv = iws + nd.o_piv;
    const int* iloc = iws + nd.o_iloc;
    T* OM = ws + nd.o_om;
    T* SI = ws + nd.o_si;
    int* skel = iws + nd.o_skel;
    const T* Om = static_cast<const T*>(fr.Om);
    int k1 = 0;
    const T *O1 = nullptr, *O2 = nullptr;
    int ld1 = 0, ld2 = 0;
    if (nd.c1 >= 0) {
        k1 = kk[nd.c1];
        O1 = ws + nodes[nd.c1].o_om;
        O2 = ws + nodes[nd.c2].o_om;
        ld1 = nodes[nd.c1].kcap;
        ld2 = nodes[nd.c2].kcap;
    }
    const int tn = tiles64(p), t = blockIdx.y;
    if (t == 0)
        for (int a = threadIdx.x; a < k; a += HT) skel[a] = iloc[piv[a]];
    const int i0 = (t / tn) * NT_TILE, j0 = (t % tn) * NT_TILE;
    if (i0 >= k) return;
    // Om_i = X^T Om_loc (k x p), S_i = S_loc(J, :)
    tile_gemm64<T, true>(
        k, p, rows, i0, j0, [&](int a, int r) { return X[(int64_t)a * nd.rows_cap + r]; },
        [&](int r, int j) {
            if (nd.c1 < 0) return Om[(int64_t)j * fr.n + nd.lo + r];
            return (r < k1) ? O1[(int64_t)j * ld1 + r] : O2[(int64_t)j * ld2 + (r - k1)];
        },
        [&](int a, int j, T acc) {
            OM[(int64_t)j * nd.kcap + a] = acc;
            SI[(int64_t)j * nd.kcap + a] = SL[(int64_t)j * nd.rows_cap + piv[a]];
        });
}

// ---------------------------------------------- HSS matvec (nc columns)
// up: xh_i = X_i^T (x(lo:hi) or [xh_c1; xh_c2]); grid (nodes, k x nc tiles)
template <typename T>
__global__ void __launch_bounds__(HT)
hss_up_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes, const T* __restrict__ ws, T* __restrict__ hb,
              const int* __restrict__ kk, const int* __restrict__ rows_in, const T* const* __restrict__ xin,
              const int64_t* __restrict__ ldx, const int* __restrict__ ncs, int64_t xh_ld) {
    const int id = list[blockIdx.x];
    const HNode nd = nodes[id];
    const int rows = rows_in[id], k = kk[id], nc = ncs[nd.front];
    const T* X = ws + nd.o_x;
    T* xh = hb + nd.o_xh;
    const T* x = xin[nd.front];
    const int64_t lx = ldx[nd.front];
    int k1 = 0;
    const T *h1 = nullptr, *h2 = nullptr;
    if (nd.c1 >= 0) {
        k1 = kk[nd.c1];
        h1 = hb + nodes[nd.c1].o_xh;
        h2 = hb + nodes[nd.c2].o_xh;
    }
    const int tn = tiles64(nc), t = blockIdx.y;
    const int i0 = (t / tn) * NT_TILE, j0 = (t % tn) * NT_TILE;
    if (i0 >= k) return;
    tile_gemm64<T, true>(
        k, nc, rows, i0, j0, [&](int a, int r) { return X[(int64_t)a * nd.rows_cap + r]; },
        [&](int r, int j) {
            if (nd.c1 < 0) return x[(int64_t)j * lx + nd.lo + r];
            return (r < k1) ? h1[(int64_t)j * xh_ld + r] : h2[(int64_t)j * xh_ld + (r - k1)];
        },
        [&](int a, int j, T acc) { xh[(int64_t)j * xh_ld + a] = acc; });
}

// down at inner node i: yh_c1 = S(sk1, sk2) xh_c2 + (X_i yh_i)(0:k1), yh_c2 = S(sk2, sk1) xh_c1 + (X_i yh_i)(k1:);
// grid (nodes, 2 parts x row tiles x nc tiles), K = [X_i's columns | the sibling's skeleton]
template <typename T>
__global__ void __launch_bounds__(HT)
hss_down_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes, const HFront* __restrict__ fronts,
                const T* __restrict__ ws, T* __restrict__ hb, const int* __restrict__ iws, const int* __restrict__ kk,
                const int* __restrict__ ncs, int64_t xh_ld) {
    const int id = list[blockIdx.x];
    const HNode nd = nodes[id];
    const HFront fr = fronts[nd.front];
    const int nc = ncs[nd.front];
    const T* S = static_cast<const T*>(fr.S);
    const int64_t lds = fr.lds;
    const HNode a = nodes[nd.c1], b = nodes[nd.c2];
    const int k1 = kk[nd.c1], k2 = kk[nd.c2];
    const bool root = (id == fr.root);
    const int k = root ? 0 : kk[id];
    const T* X = ws + nd.o_x;
    const T* yh = hb + nd.o_yh;
    const int tn = tiles64(nc), tm = tiles64(nd.kcap), t = blockIdx.y;
    const int part = t / (tm * tn), tt = t % (tm * tn);
    const int i0 = (tt / tn) * NT_TILE, j0 = (tt % tn) * NT_TILE;
    const int M = part == 0 ? k1 : k2, Ko = part == 0 ? k2 : k1, roff = part == 0 ? 0 : k1;
    if (part > 1 || i0 >= M) return;
    const int* own = iws + (part == 0 ? a.o_skel : b.o_skel);
    const int* oth = iws + (part == 0 ? b.o_skel : a.o_skel);
    const T* xo = hb + (part == 0 ? b.o_xh : a.o_xh);
    T* yo = hb + (part == 0 ? a.o_yh : b.o_yh);
    tile_gemm64<T, false>(
        M, nc, k + Ko, i0, j0,
        [&](int r, int l) {
            return l < k ? X[(int64_t)l * nd.rows_cap + roff + r] : S[(int64_t)oth[l - k] * lds + own[r]];
        },
        [&](int l, int j) { return l < k ? yh[(int64_t)j * xh_ld + l] : xo[(int64_t)j * xh_ld + (l - k)]; },
        [&](int r, int j, T acc) { yo[(int64_t)j * xh_ld + r] = acc; });
}

// leaves: y(lo:hi) = D x(lo:hi) + X yh; grid (nodes, rows x nc tiles), K = [D's columns | X's columns]
template <typename T>
__global__ void __launch_bounds__(HT)
hss_leaf_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes, const HFront* __restrict__ fronts,
                const T* __restrict__ ws, const T* __restrict__ hb, const int* __restrict__ kk,
                const T* const* __restrict__ xin, const int64_t* __restrict__ ldx, T* const* __restrict__ yout,
                const int64_t* __restrict__ ldy, const int* __restrict__ ncs, int64_t xh_ld) {
    const int id = list[blockIdx.x];
    const HNode nd = nodes[id];
    const HFront fr = fronts[nd.front];
    const int nc = ncs[nd.front];
    const T* S = static_cast<const T*>(fr.S);
    const int64_t lds = fr.lds;
    const int rows = nd.hi - nd.lo;
    const bool root = (id == fr.root);
    const int k = root ? 0 : kk[id];
    const T* X = ws + nd.o_x;
    const T* yh = hb + nd.o_yh;
    const T* x = xin[nd.front];
    T* y = yout[nd.front];
    const int64_t lx = ldx[nd.front], ly = ldy[nd.front];
    const int tn = tiles64(nc), t = blockIdx.y;
    const int i0 = (t / tn) * NT_TILE, j0 = (t % tn) * NT_TILE;
    if (i0 >= rows) return;
    tile_gemm64<T, false>(
        rows, nc, rows + k, i0, j0,
        [&](int r, int l) {
            return l < rows ? S[(int64_t)(nd.lo + l) * lds + nd.lo + r] : X[(int64_t)(l - rows) * nd.rows_cap + r];
        },
        [&](int l, int j) { return l < rows ? x[(int64_t)j * lx + nd.lo + l] : yh[(int64_t)j * xh_ld + (l - rows)]; },
        [&](int r, int j, T acc) { y[(int64_t)j * ly + nd.lo + r] = acc; });
}

// coupling blocks of inner node i: B12 = S(skel_c1, skel_c2) (k1 x k2), B21 = S(skel_c2, skel_c1)
template <typename T>
__global__ void gather_b_kernel(const int* __restrict__ list, const HNode* __restrict__ nodes,
                                const HFront* __restrict__ fronts, const int* __restrict__ iws, const int* __restrict__ kk,
                                T* const* __restrict__ b12, T* const* __restrict__ b21) {
    const HNode nd = nodes[list[blockIdx.x]];
    const HFront fr = fronts[nd.front];
    const T* S = static_cast<const T*>(fr.S);
    const int k1 = kk[nd.c1], k2 = kk[nd.c2];
    const int* sk1 = iws + nodes[nd.c1].o_skel;
    const int* sk2 = iws + nodes[nd.c2].o_skel;
    T* a = b12[blockIdx.x];
    T* b = b21[blockIdx.x];
    for (int q = threadIdx.x; q < k1 * k2; q += blockDim.x) {
        const int i = q % k1, j = q / k1;
        a[q] = S[(int64_t)sk2[j] * fr.lds + sk1[i]];
    }
    for (int q = threadIdx.x; q < k1 * k2; q += blockDim.x) {
        const int i = q % k2, j = q / k2;
        b[q] = S[(int64_t)sk1[j] * fr.lds + sk2[i]];
    }
}

// estimator norms per front: err^2 = ||Yt - Zt||^2, ref^2 = ||Yt||^2
template <typename T>
__global__ void est_norm_kernel(const HFront* __restrict__ fronts, int r, double* __restrict__ out) {
    const HFront fr = fronts[blockIdx.x];
    const T* Yt = static_cast<const T*>(fr.Yt);
    const T* Zt = static_cast<const T*>(fr.Zt);
    const int64_t n = (int64_t)fr.n * r;
    double e = 0.0, f = 0.0;
    // eight elements of each operand in flight per thread
    for (int64_t q0 = threadIdx.x; q0 < n; q0 += 8 * (int64_t)blockDim.x) {
        T y[8], z[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t q = q0 + (int64_t)u * blockDim.x;
            y[u] = q < n ? Yt[q] : zero<T>();
            z[u] = q < n ? Zt[q] : zero<T>();
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            e += nrm2v(y[u] - z[u]);
            f += nrm2v(y[u]);
        }
    }
    __shared__ double se[HT], sf[HT];
    se[threadIdx.x] = e;
    sf[threadIdx.x] = f;
    __syncthreads();
    for (int s = HT / 2; s; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sf[threadIdx.x] += sf[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = sqrt(se[0]);
        out[2 * blockIdx.x + 1] = sqrt(sf[0]);
    }
}

// identity columns (n x n, ld n) per front
template <typename T>
__global__ void eye_kernel(T* const* __restrict__ dst, const int* __restrict__ ns) {
    T* d = dst[blockIdx.y];
    const int64_t n = ns[blockIdx.y];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * n; q += (int64_t)gridDim.x * blockDim.x)
        d[q] = (q % n == q / n) ? one<T>() : zero<T>();
}

// copy an n x n block (ld n) into S (ld lds)
template <typename T>
__global__ void copy_back_kernel(const T* const* __restrict__ src, const HFront* __restrict__ fronts, const int* __restrict__ which) {
    const HFront fr = fronts[which[blockIdx.y]];
    const T* s = src[blockIdx.y];
    T* S = static_cast<T*>(fr.S);
    const int64_t n = fr.n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * n; q += (int64_t)gridDim.x * blockDim.x)
        S[(q / n) * fr.lds + q % n] = s[q];
}

// R(J, :) rows gathered (k x ncol, ld kcap), and the transposed samples W = Y^T (p x n, ld p)
template <typename T>
__global__ void gather_rows_kernel(const HFront* __restrict__ fronts, const HNode* __restrict__ nodes, const T* __restrict__ ws,
                                   const int* __restrict__ iws, const int* __restrict__ kk) {
    const HFront fr = fronts[blockIdx.y];
    const HNode nd = nodes[fr.root];
    const int k = kk[fr.root];
    const int* piv = iws + nd.o_piv;
    const T* R = static_cast<const T*>(fr.S);
    T* RJ = static_cast<T*>(fr.RJ);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)k * fr.ncol;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(q % k);
        const int64_t j = q / k;
        RJ[j * nd.kcap + a] = R[j * fr.lds + piv[a]];
    }
}

template <typename T>
__global__ void transpose_samples_kernel(const HFront* __restrict__ fronts, const HNode* __restrict__ nodes, T* __restrict__ ws,
                                         int* __restrict__ iws, int* __restrict__ rows_out) {
    const HFront fr = fronts[blockIdx.y];
    const HNode nd = nodes[fr.root];
    const T* Y = static_cast<const T*>(fr.Y);
    T* W = ws + nd.o_w;
    const int p = nd.p;
    const int64_t n = fr.n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * p; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % n, j = q / n;
        W[i * p + j] = Y[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rows_out[fr.root] = fr.n;
}

// host-side cluster tree identical to the oracle's (breadth-first, Fig. 4 top split, halving to <= beta)
struct HCl {
    int lo, hi, level, parent, c1, c2;
};
std::vector<HCl> cluster_tree(int n, int top, int beta) {
    std::vector<HCl> t;
    t.push_back({0, n, 0, -1, -1, -1});
    for (size_t q = 0; q < t.size(); ++q) {
        HCl c = t[q];
        if (c.hi - c.lo <= beta) continue;
        const int mid = (q == 0 && top > 0 && top < n) ? top : c.lo + (c.hi - c.lo) / 2;
        const int a = (int)t.size();
        t.push_back({c.lo, mid, c.level + 1, (int)q, -1, -1});
        t.push_back({mid, c.hi, c.level + 1, (int)q, -1, -1});
        t[q].c1 = a;
        t[q].c2 = a + 1;
    }
    return t;
}

// Stream-ordered scratch (pool allocator): no device-wide synchronisation on
// allocation or release, uploads from pageable host memory are staged by the
// runtime before cudaMemcpyAsync returns.
template <typename U>
struct DeviceVec {
    U* p = nullptr;
    size_t n = 0;
    cudaStream_t st = nullptr;
    explicit DeviceVec(cudaStream_t s = nullptr) : st(s) {}
    ~DeviceVec() { if (p) cudaFreeAsync(p, st); }
    cudaError_t alloc(size_t count) {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        n = count;
        return pool_malloc_async((void**)&p, std::max<size_t>(n, 1) * sizeof(U), st);
    }
    cudaError_t upload(const std::vector<U>& v, cudaStream_t s) {
        st = s;
        cudaError_t e = alloc(v.size());
        if (e == cudaSuccess && !v.empty()) e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice, st);
        return e;
    }
};

// Independent launches of one step on side streams: forked from the
// caller's stream st by an event, each joined back to st by its own event,
// so everything after the join stays ordered on st.  Without side launches
// (n == 0) every stream() is st itself.  The side streams are the caller's
// own when it passes four (a second host thread of the factorization), else
// a pool created once per device and kept (shared by all such callers:
// sharing only orders their launches more strictly).
struct SideFork {
    static constexpr int NS = 4;
    cudaStream_t st;
    int n;
    cudaError_t status = cudaSuccess;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> done;
    cudaStream_t side[NS] = {};
    SideFork(cudaStream_t s, int count, const cudaStream_t* own = nullptr) : st(s), n(std::min(count, NS)) {
        if (n <= 1) { n = 0; return; }
        if (own && own[0]) {
            for (int i = 0; i < NS; ++i) side[i] = own[i];
            if ((status = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming)) != cudaSuccess) { n = 0; return; }
            status = cudaEventRecord(fork_ev, st);
            done.assign(n, nullptr);
            return;
        }
        static std::mutex mu;
        static cudaStream_t pool[64][NS];
        static bool made[64] = {};
        int dev = 0;
        if ((status = cudaGetDevice(&dev)) != cudaSuccess) { n = 0; return; }
        {
            std::lock_guard<std::mutex> lk(mu);
            if (!made[dev & 63]) {
                for (int i = 0; i < NS && status == cudaSuccess; ++i)
                    status = cudaStreamCreateWithFlags(&pool[dev & 63][i], cudaStreamNonBlocking);
                if (status != cudaSuccess) { n = 0; return; }
                made[dev & 63] = true;
            }
            for (int i = 0; i < NS; ++i) side[i] = pool[dev & 63][i];
        }
        if ((status = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming)) != cudaSuccess) { n = 0; return; }
        status = cudaEventRecord(fork_ev, st);
        done.assign(n, nullptr);
    }
    // launch i goes to stream(i); call start(i) after its inputs are enqueued on st
    cudaStream_t stream(int i) const { return n ? side[i % NS] : st; }
    cudaError_t start(int i) {
        if (!n) return cudaSuccess;
        // the fork event was recorded before this launch's inputs: re-record it
        cudaError_t e = cudaEventRecord(fork_ev, st);
        return e == cudaSuccess ? cudaStreamWaitEvent(stream(i), fork_ev, 0) : e;
    }
    cudaError_t finish(int i) {
        if (!n) return cudaSuccess;
        cudaError_t e = cudaSuccess;
        if (!done[i % n]) e = cudaEventCreateWithFlags(&done[i % n], cudaEventDisableTiming);
        return e == cudaSuccess ? cudaEventRecord(done[i % n], stream(i)) : e;
    }
    cudaError_t join() {
        for (cudaEvent_t ev : done) {
            if (!ev) continue;
            cudaError_t e = cudaStreamWaitEvent(st, ev, 0);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    ~SideFork() {
        if (fork_ev) cudaEventDestroy(fork_ev);
        for (cudaEvent_t ev : done)
            if (ev) cudaEventDestroy(ev);
    }
};

#define HSS_TRY(expr)                                                                                      \
    do {                                                                                                   \
        cudaError_t e_ = (expr);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return set_error(NDHSS_ERR_CUDA, "hss: %s failed: %s", #expr, cudaGetErrorString(e_));           \
    } while (0)

// The batched GEMM of a job list: one launch of 64 x 64 tiles, or, when the
// tiles of all jobs leave the GPU mostly idle and K is long, K split over
// ksplit CTAs per tile plus an ordered reduction of their partials.
template <typename T, bool RB>
ndhss_status run_bgemm_group(const std::vector<GemmJob>& jobs, cudaStream_t st) {
    if (jobs.empty()) return NDHSS_OK;
    int maxM = 1, maxN = 1, maxK = 1;
    for (const GemmJob& g : jobs) {
        maxM = std::max(maxM, g.M);
        maxN = std::max(maxN, g.N);
        maxK = std::max(maxK, g.K);
    }
    const int tm = (maxM + 63) / 64, tn = (maxN + 63) / 64;
    int dev = 0, sms = 1;
    HSS_TRY(cudaGetDevice(&dev));
    HSS_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t base = (int64_t)tm * tn * (int64_t)jobs.size();
    int ks = 1;
    if (base < 2 * sms && maxK >= 256)
        ks = (int)std::min<int64_t>({(2 * sms + base - 1) / base, maxK / 128, 16});
    ks = std::max(ks, 1);
    DeviceVec<GemmJob> dj(st);
    HSS_TRY(dj.upload(jobs, st));
    const size_t per = (size_t)std::max(1, 65535 / ks);     // jobs per launch (grid z limit)
    DeviceVec<T> part(st);
    if (ks > 1) HSS_TRY(part.alloc((size_t)std::min(per, jobs.size()) * ks * tm * tn * 4096));
    for (size_t j0 = 0; j0 < jobs.size(); j0 += per) {
        const unsigned nj = (unsigned)std::min(per, jobs.size() - j0);
        bgemm_kernel<T, RB><<<dim3(tm, tn, nj * ks), 256, 0, st>>>(dj.p + j0, ks, part.p);
        NDHSS_LAUNCH_CHECK("bgemm_kernel");
        if (ks > 1) {
            bgemm_reduce_kernel<T><<<dim3(tm, tn, nj), 256, 0, st>>>(dj.p + j0, ks, part.p);
            NDHSS_LAUNCH_CHECK("bgemm_reduce_kernel");
        }
    }
    return NDHSS_OK;
}

// Jobs with a real B (complex T) take the two-FMA products; the rest the
// full complex ones.
template <typename T>
ndhss_status run_bgemm(const std::vector<GemmJob>& jobs, cudaStream_t st) {
    std::vector<GemmJob> gr, gc;
    for (const GemmJob& g : jobs) ((Tr<T>::cplx && g.realB) ? gr : gc).push_back(g);
    ndhss_status rc = run_bgemm_group<T, true>(gr, st);
    if (rc == NDHSS_OK) rc = run_bgemm_group<T, false>(gc, st);
    return rc;
}


// y = A_HSS x for the fronts listed in the node table: up-sweep deepest level
// first, coupling + down-sweep root first, then the leaf blocks.
template <typename T>
ndhss_status hss_matvec_run(const std::vector<HNode>& nodes, const std::vector<char>& keep, int maxlev,
                            const HNode* dnodes, const HFront* dfr, const T* ws, T* hb, const int* iws, const int* kk,
                            const int* rows, const T* const* dx, const int64_t* dlx, T* const* dy, const int64_t* dly,
                            const int* dncs, int nc_max, int64_t xh_ld, cudaStream_t st) {
    std::vector<int> flat;
    std::vector<size_t> up_off(maxlev + 2, 0), dn_off(maxlev + 2, 0);
    for (int l = 0; l <= maxlev; ++l) {            // up lists (non-root)
        up_off[l] = flat.size();
        for (size_t i = 0; i < nodes.size(); ++i)
            if (keep[nodes[i].front] && nodes[i].level == l && l > 0) flat.push_back((int)i);
    }
    up_off[maxlev + 1] = flat.size();
    for (int l = 0; l <= maxlev; ++l) {            // down lists (inner nodes)
        dn_off[l] = flat.size();
        for (size_t i = 0; i < nodes.size(); ++i)
            if (keep[nodes[i].front] && nodes[i].level == l && nodes[i].c1 >= 0) flat.push_back((int)i);
    }
    dn_off[maxlev + 1] = flat.size();
    const size_t leaf_off = flat.size();
    for (size_t i = 0; i < nodes.size(); ++i)
        if (keep[nodes[i].front] && nodes[i].c1 < 0) flat.push_back((int)i);
    const size_t leaf_cnt = flat.size() - leaf_off;
    DeviceVec<int> dflat(st);
    HSS_TRY(dflat.upload(flat, st));
    // tile grids: k x nc (up), 2 parts x kcap x nc (down), leaf rows x nc (leaves)
    int kcap = 1, leaf_rows = 1;
    for (size_t i = 0; i < nodes.size(); ++i) {
        if (!keep[nodes[i].front]) continue;
        kcap = std::max(kcap, nodes[i].kcap);
        if (nodes[i].c1 < 0) leaf_rows = std::max(leaf_rows, nodes[i].hi - nodes[i].lo);
    }
    const unsigned tnc = (unsigned)tiles64(nc_max);
    for (int l = maxlev; l >= 1; --l) {
        const unsigned cnt = (unsigned)(up_off[l + 1] - up_off[l]);
        if (!cnt) continue;
        hss_up_kernel<T><<<dim3(cnt, tiles64(kcap) * tnc), HT, 0, st>>>(dflat.p + up_off[l], dnodes, ws, hb, kk, rows, dx,
                                                                         dlx, dncs, xh_ld);
        NDHSS_LAUNCH_CHECK("hss_up_kernel");
    }
    for (int l = 0; l <= maxlev; ++l) {
        const unsigned cnt = (unsigned)(dn_off[l + 1] - dn_off[l]);
        if (!cnt) continue;
        hss_down_kernel<T><<<dim3(cnt, 2 * tiles64(kcap) * tnc), HT, 0, st>>>(dflat.p + dn_off[l], dnodes, dfr, ws, hb,
                                                                               iws, kk, dncs, xh_ld);
        NDHSS_LAUNCH_CHECK("hss_down_kernel");
    }
    if (leaf_cnt) {
        hss_leaf_kernel<T><<<dim3((unsigned)leaf_cnt, tiles64(leaf_rows) * tnc), HT, 0, st>>>(
            dflat.p + leaf_off, dnodes, dfr, ws, hb, kk, dx, dlx, dy, dly, dncs, xh_ld);
        NDHSS_LAUNCH_CHECK("hss_leaf_kernel");
    }
    return NDHSS_OK;
}

// One compression problem set (all S blocks, or all R blocks, of a level).
// One retired low-rank problem: X (n x k, ld ldx) and R(J, :) (k x nc, ld ldr)
// go to dst as X (ld n) followed by R(J, :)^T (nc x k, ld nc).
struct LrOut {
    const void* X;
    const void* RJ;
    void* dst;
    int64_t ldx, ldr;
    int n, nc, k, pad;
};

template <typename T>
__global__ void __launch_bounds__(256) lr_out_kernel(const LrOut* __restrict__ jobs) {
    const LrOut j = jobs[blockIdx.x];
    const T* X = static_cast<const T*>(j.X);
    const T* RJ = static_cast<const T*>(j.RJ);
    T* d = static_cast<T*>(j.dst);
    const int64_t nx = (int64_t)j.n * j.k, nr = (int64_t)j.nc * j.k;
    for (int64_t q = threadIdx.x; q < nx; q += blockDim.x) d[q] = X[(q / j.n) * j.ldx + q % j.n];
    for (int64_t q = threadIdx.x; q < nr; q += blockDim.x) d[nx + q] = RJ[(q % j.nc) * j.ldr + q / j.nc];
}

struct Problem {
    int node;          // tree node
    int n, ncol;       // rows and columns of the block
    int64_t lds;
    void* ptr;         // block in the front arena
    int top;           // Fig. 4 top split (S), unused for R
    uint64_t stream;   // 2*node (S) or 2*node+1 (R), as the oracle
};

// ULV factorization of HSS fronts whose generators sit in device memory:
// per HSS node its leaf block (in the front's block), basis / transfer matrix
// X (ld x_ld), coupling blocks B12 / B21 (inner nodes), rank; jobs run one
// HSS level per launch, deepest first.  Appends the solve records to F.
struct UlvIn {
    int s;              // tree node of the front
    int lo, hi, level, c1, c2, root;   // c1 / c2: indices into the same input list
    int k;              // basis width (root: unused)
    const void* D0;     // leaf block, ld ldd0
    int64_t ldd0;
    const void* X;      // leaf basis / inner transfer matrix, ld ldx
    int64_t ldx;
    const void* B12;
    const void* B21;
};

template <typename T>
ndhss_status ulv_factor_nodes(const std::vector<UlvIn>& in, FactorData& F, cudaStream_t st) {
    const int nn = (int)in.size();
    if (!nn) return NDHSS_OK;
    std::vector<int> m(nn), ne(nn), kt(nn), kw(nn);
    int maxlev = 0;
    for (auto& u : in) maxlev = std::max(maxlev, u.level);
    std::vector<int> order;
    for (int l = maxlev; l >= 0; --l)
        for (int q = 0; q < nn; ++q)
            if (in[q].level == l) order.push_back(q);
    std::vector<int> job_of(nn);
    for (int j = 0; j < nn; ++j) job_of[order[j]] = j;
    int64_t pers = 0, pass = 0;
    std::vector<int64_t> o_mup(nn), o_w(nn), o_mm(nn), o_e(nn), o_di(nn), o_dh(nn);
    for (int q : order) {
        const UlvIn& u = in[q];
        m[q] = (u.c1 < 0) ? u.hi - u.lo : kt[u.c1] + kt[u.c2];
        kw[q] = u.root ? 0 : u.k;
        ne[q] = u.root ? 0 : std::max(0, m[q] - kw[q]);
        kt[q] = m[q] - ne[q];
        const int ka = u.c1 < 0 ? 0 : kw[u.c1], kb = u.c1 < 0 ? 0 : kw[u.c2];
        auto take = [&](int64_t c) { const int64_t o = pers; pers += (c + 31) / 32 * 32; return o; };
        o_mup[q] = u.root ? -1 : take((int64_t)(m[q] + kw[q]) * m[q]);
        o_w[q] = u.root ? -1 : take((int64_t)m[q] * m[q]);
        o_mm[q] = u.c1 < 0 ? -1 : take((int64_t)m[q] * std::max(ka + kb, 1));
        o_e[q] = (u.c1 < 0 || u.root) ? -1 : take((int64_t)std::max(ka + kb, 1) * std::max(kw[q], 1));
        o_di[q] = u.root ? take((int64_t)m[q] * m[q]) : -1;
        o_dh[q] = pass;
        pass += ((int64_t)kt[q] * kt[q] + 2 * (int64_t)kt[q] * std::max(kw[q], 1) + 31) / 32 * 32;
    }
    void* buf = nullptr;
    if (pool_malloc_async(&buf, std::max<int64_t>(pers, 1) * sizeof(T), st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(NDHSS_ERR_OOM, "ulv: solve data (%lld elements)", (long long)pers);
    }
    F.ulv_bufs.push_back(buf);
    F.dev_bytes += pers * (int64_t)sizeof(T);
    T* P = static_cast<T*>(buf);
    // work space: the largest level
    std::vector<int64_t> lvl_work(maxlev + 1, 0), o_wk(nn);
    for (int q = 0; q < nn; ++q) {
        o_wk[q] = lvl_work[in[q].level];
        lvl_work[in[q].level] += (ulv_work_elems(m[q], kw[q], ne[q]) + 31) / 32 * 32;
    }
    int64_t wmax = 1;
    for (int64_t w : lvl_work) wmax = std::max(wmax, w);
    DeviceVec<T> work(st), passbuf(st);
    DeviceVec<int> status(st);
    HSS_TRY(work.alloc(wmax));
    HSS_TRY(passbuf.alloc(std::max<int64_t>(pass, 1)));
    HSS_TRY(status.alloc(1));
    HSS_TRY(cudaMemsetAsync(status.p, 0, sizeof(int), st));
    std::vector<UlvJob<T>> jobs(nn);
    const int rec0 = (int)F.ulv_recs.size();
    F.ulv_recs.resize(rec0 + nn);
    for (int j = 0; j < nn; ++j) {
        const int q = order[j];
        const UlvIn& u = in[q];
        UlvJob<T> J{};
        J.m = m[q];
        J.k = kw[q];
        J.ne = ne[q];
        J.kt = kt[q];
        J.leaf = u.c1 < 0;
        J.root = u.root;
        J.ka = u.c1 < 0 ? 0 : kw[u.c1];
        J.kb = u.c1 < 0 ? 0 : kw[u.c2];
        J.c1 = u.c1 < 0 ? -1 : job_of[u.c1];
        J.c2 = u.c1 < 0 ? -1 : job_of[u.c2];
        J.D0 = static_cast<const T*>(u.D0);
        J.ldd0 = u.ldd0;
        J.X = static_cast<const T*>(u.X);
        J.ldx = u.ldx;
        J.B12 = static_cast<const T*>(u.B12);
        J.B21 = static_cast<const T*>(u.B21);
        J.Mup = o_mup[q] >= 0 ? P + o_mup[q] : nullptr;
        J.W = o_w[q] >= 0 ? P + o_w[q] : nullptr;
        J.Mm = o_mm[q] >= 0 ? P + o_mm[q] : nullptr;
        J.E = o_e[q] >= 0 ? P + o_e[q] : nullptr;
        J.Dinv = o_di[q] >= 0 ? P + o_di[q] : nullptr;
        T* ph = passbuf.p + o_dh[q];
        J.Dh = ph;
        J.Uh = ph + (int64_t)kt[q] * kt[q];
        J.Vh = J.Uh + (int64_t)kt[q] * std::max(kw[q], 1);
        J.w = work.p + o_wk[q];
        J.status = status.p;
        jobs[j] = J;
        FactorData::UlvRec& r = F.ulv_recs[rec0 + j];
        r.s = u.s;
        r.lo = J.leaf ? u.lo : -1;
        r.hi = J.leaf ? u.hi : -1;
        r.m = J.m;
        r.k = J.k;
        r.ne = J.ne;
        r.kt = J.kt;
        r.ka = J.ka;
        r.kb = J.kb;
        r.c1 = J.c1 < 0 ? -1 : rec0 + J.c1;
        r.c2 = J.c2 < 0 ? -1 : rec0 + J.c2;
        r.parent = -1;
        r.level = u.level;
        r.leaf = J.leaf;
        r.root = J.root;
        r.Mup = reinterpret_cast<uint64_t>(J.Mup);
        r.W = reinterpret_cast<uint64_t>(J.W);
        r.Mm = reinterpret_cast<uint64_t>(J.Mm);
        r.E = reinterpret_cast<uint64_t>(J.E);
        r.Dinv = reinterpret_cast<uint64_t>(J.Dinv);
        if (J.root) F.ulv_root_of[u.s] = rec0 + j;
    }
    for (int j = 0; j < nn; ++j) {
        const FactorData::UlvRec& r = F.ulv_recs[rec0 + j];
        if (r.c1 >= 0) F.ulv_recs[r.c1].parent = F.ulv_recs[r.c2].parent = rec0 + j;
    }
    F.ulv_bytes += pers * (int64_t)sizeof(T);
    DeviceVec<UlvJob<T>> djobs(st);
    HSS_TRY(djobs.upload(jobs, st));
    int j0 = 0;
    for (int l = maxlev; l >= 0; --l) {
        int cnt = 0;
        while (j0 + cnt < nn && in[order[j0 + cnt]].level == l) ++cnt;
        ndhss_status rc = ulv_launch_level<T>(djobs.p + j0, djobs.p, cnt, st);
        if (rc != NDHSS_OK) return rc;
        j0 += cnt;
    }
    int hs = 0;
    HSS_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HSS_TRY(cudaStreamSynchronize(st));
    if (hs) return set_error(NDHSS_ERR_SINGULAR, "ulv: singular root block of an HSS(A_ii) at level %d", in[0].level);
    return NDHSS_OK;
}

// Runs the adaptive rounds of Alg. A.1 (lowrank == false) or of the low-rank
// range finder (lowrank == true) on all problems; on success S blocks are
// overwritten by their HSS reconstruction and for R blocks (X, R(J,:)) are
// written to `lr_out` (per problem: X m_i x k then RJ k x m_b), ranks to kout.
template <typename T>
ndhss_status compress_problems(std::vector<Problem>& probs, bool lowrank, const ndhss_factor_opts& o,
                               std::vector<int>& kout, std::vector<uint64_t>* lr_dev, FactorData& F,
                               cudaStream_t st, bool ulv = false) {
    const int r = std::max(o.r, 1), k0 = std::max(o.k0, 1), beta = std::max(o.beta, 1);
    const int rank_cap = std::max(o.rank_cap, 1);
    const double eps = o.eps_hss;
    kout.assign(probs.size(), 0);
    if (lr_dev) lr_dev->assign(probs.size(), 0);
    std::vector<int> active(probs.size());
    for (size_t i = 0; i < probs.size(); ++i) active[i] = (int)i;
    std::vector<double> prev_err(probs.size(), INFINITY);
    int p = k0 + r;
    int round = 0;
    while (!active.empty()) {
        const int kcap = std::max(1, std::min(rank_cap, p - OVERSAMPLE_MIN));
        std::vector<HFront> fr;
        std::vector<HNode> nodes;
        std::vector<std::vector<HCl>> trees;
        int64_t ews = 0, iwsz = 0;
        auto take = [&](int64_t cnt) { int64_t o2 = ews; ews += (cnt + 31) / 32 * 32; return o2; };
        auto itake = [&](int64_t cnt) { int64_t o2 = iwsz; iwsz += (cnt + 31) / 32 * 32; return o2; };
        int maxlev = 0;
        int64_t max_rows = 1;
        for (int a : active) {
            const Problem& pb = probs[a];
            HFront f{};
            f.S = pb.ptr;
            f.lds = pb.lds;
            f.n = pb.n;
            f.ncol = pb.ncol;
            auto tr = lowrank ? std::vector<HCl>{{0, pb.n, 0, -1, -1, -1}} : cluster_tree(pb.n, pb.top, beta);
            const int base = (int)nodes.size();
            f.root = base;
            for (auto& c : tr) {
                HNode nd{};
                nd.front = (int)fr.size();
                nd.lo = c.lo;
                nd.hi = c.hi;
                nd.level = c.level;
                nd.c1 = c.c1 >= 0 ? base + c.c1 : -1;
                nd.c2 = c.c2 >= 0 ? base + c.c2 : -1;
                nd.p = p;
                nd.kcap = kcap;
                nd.rows_cap = (c.c1 < 0) ? (c.hi - c.lo) : 2 * kcap;
                max_rows = std::max<int64_t>(max_rows, nd.rows_cap);
                nd.o_w = take((int64_t)p * nd.rows_cap);
                nd.o_sl = take((int64_t)p * nd.rows_cap);
                nd.o_x = take((int64_t)nd.rows_cap * kcap);
                nd.o_om = take((int64_t)kcap * p);
                nd.o_si = take((int64_t)kcap * p);
                nd.o_skel = itake(kcap);
                nd.o_iloc = itake(nd.rows_cap);
                nd.o_piv = itake(nd.rows_cap);
                maxlev = std::max(maxlev, c.level);
                nodes.push_back(nd);
            }
            trees.push_back(tr);
            fr.push_back(f);
        }
        // per-front sample buffers
        const int nf = (int)fr.size();
        std::vector<int64_t> o_om(nf), o_y(nf), o_ot(nf), o_yt(nf), o_zt(nf), o_t1(nf), o_rj(nf);
        for (int i = 0; i < nf; ++i) {
            const int64_t n = fr[i].n, nc = fr[i].ncol;
            // [Omega | Omega~] and [Y | Y~] side by side (same leading dimension):
            // one product per block gives both
            const int64_t ro = lowrank ? nc : n;
            o_om[i] = take(ro * (p + r));
            o_ot[i] = o_om[i] + ro * p;
            o_y[i] = take(n * (p + r));
            o_yt[i] = o_y[i] + n * p;
            o_zt[i] = take(n * r);
            o_t1[i] = take((int64_t)kcap * r);
            o_rj[i] = take((int64_t)kcap * nc);
        }
        // matvec scratch (estimator: r columns)
        for (auto& nd : nodes) {
            nd.o_xh = take((int64_t)kcap * r);
            nd.o_yh = take((int64_t)kcap * r);
        }
        DeviceVec<T> ws(st);
        DeviceVec<int> iws(st), kk(st), rows(st);
        HSS_TRY(ws.alloc(ews));
        HSS_TRY(iws.alloc(iwsz));
        HSS_TRY(kk.alloc(nodes.size()));
        HSS_TRY(rows.alloc(nodes.size()));
        HSS_TRY(cudaMemsetAsync(kk.p, 0, nodes.size() * sizeof(int), st));
        for (int i = 0; i < nf; ++i) {
            fr[i].Om = ws.p + o_om[i];
            fr[i].Y = ws.p + o_y[i];
            fr[i].Ot = ws.p + o_ot[i];
            fr[i].Yt = ws.p + o_yt[i];
            fr[i].Zt = ws.p + o_zt[i];
            fr[i].T1 = ws.p + o_t1[i];
            fr[i].RJ = ws.p + o_rj[i];
        }
        DeviceVec<HFront> dfr(st);
        DeviceVec<HNode> dnodes(st);
        HSS_TRY(dfr.upload(fr, st));
        HSS_TRY(dnodes.upload(nodes, st));
        // Gaussian samples, block by block exactly as the oracle draws them
        std::vector<GaussJob> gj;
        for (int i = 0; i < nf; ++i) {
            const Problem& pb = probs[active[i]];
            const int rows_o = lowrank ? pb.ncol : pb.n;
            const uint64_t sb = pb.stream * 64 + (lowrank ? 32 : 0);
            gj.push_back({fr[i].Om, rows_o, rows_o, k0 + r, 0, sb});
            for (int q = 0; q < round; ++q) gj.push_back({fr[i].Om, rows_o, rows_o, r, k0 + r + q * r, sb + 1 + q});
            gj.push_back({fr[i].Ot, rows_o, rows_o, r, 0, sb + 1 + round});
        }
        DeviceVec<GaussJob> dgj(st);
        HSS_TRY(dgj.upload(gj, st));
        gauss_kernel<T><<<dim3(64, (unsigned)gj.size()), 256, 0, st>>>(dgj.p, o.seed);
        NDHSS_LAUNCH_CHECK("gauss_kernel");
        // Y = block * Omega, Yt = block * Omega~
        std::vector<GemmJob> gm;
        int maxM = 1, maxN = 1;
        for (int i = 0; i < nf; ++i) {
            const Problem& pb = probs[active[i]];
            const int K = lowrank ? pb.ncol : pb.n;
            GemmJob g{pb.ptr, fr[i].Om, fr[i].Y, pb.lds, K, pb.n, pb.n, p + r, K, 0, 1.0};
            g.realB = 1;
            gm.push_back(g);
            maxM = std::max(maxM, pb.n);
            maxN = std::max(maxN, p);
        }
        {
            const ndhss_status rc = run_bgemm<T>(gm, st);
            if (rc != NDHSS_OK) return rc;
        }
        // node lists per HSS level
        std::vector<std::vector<int>> bylev(maxlev + 1);
        for (size_t i = 0; i < nodes.size(); ++i) bylev[nodes[i].level].push_back((int)i);
        std::vector<int> flat;
        std::vector<size_t> loff(maxlev + 2, 0);
        for (int l = 0; l <= maxlev; ++l) {
            loff[l] = flat.size();
            flat.insert(flat.end(), bylev[l].begin(), bylev[l].end());
        }
        loff[maxlev + 1] = flat.size();
        DeviceVec<int> dflat(st);
        HSS_TRY(dflat.upload(flat, st));
        // the sample block of a node sits in shared memory when it fits (p <= 256 always)
        if (p > 256) return set_error(NDHSS_ERR_RANK_CAP, "hss: more than 256 samples per block (rank_cap too large)");
        const size_t smem_base = (size_t)(rows_cap_even((int)max_rows)) * sizeof(double) + (size_t)(p + 2) * sizeof(T) + 64;
        const size_t smem_w = smem_base + (size_t)(p | 1) * max_rows * sizeof(T);
        const int w_in_smem = smem_w <= 200 * 1024 ? 1 : 0;
        (void)w_in_smem;
        HSS_TRY(cudaFuncSetAttribute(row_id_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem_base, 48 * 1024)));
        HSS_TRY(cudaFuncSetAttribute(row_id_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RID_SMEM));
        // row IDs of the nodes flat[b, e): the cluster kernel with the smallest
        // cluster whose share of W fits in shared memory, one launch per cluster
        // size; a node too large for RID_MAX_CLUSTER CTAs keeps W in global memory
        auto rid_bytes = [&](int rows_cap, int C) {
            const size_t chunk = (size_t)(rows_cap + C - 1) / C;
            return ((size_t)(p | 1) * chunk + (size_t)p + 1) * sizeof(T) + chunk + 16;
        };
        int num_sms = 0, dev = 0;
        HSS_TRY(cudaGetDevice(&dev));
        HSS_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        auto launch_row_id = [&](size_t b, size_t e) -> ndhss_status {
            std::vector<int> grp[5], big;
            // a node whose share would exceed RID_SPLIT_COLS columns per CTA is
            // split further (its pivot steps run shorter) when all such nodes
            // together take at most two CTAs per SM: the launch lasts as long
            // as its longest pivot chain
            auto g_fit = [&](int rc) {
                int g = 0;
                while ((1 << g) <= RID_MAX_CLUSTER && rid_bytes(rc, 1 << g) > RID_SMEM) ++g;
                return g;
            };
            auto g_split = [&](int rc, int g) {
                while ((1 << g) < RID_MAX_CLUSTER && (rc + (1 << g) - 1) / (1 << g) > RID_SPLIT_COLS) ++g;
                return g;
            };
            int64_t split_ctas = 0;
            for (size_t q = b; q < e; ++q) {
                const int rc = nodes[flat[q]].rows_cap, g0 = g_fit(rc);
                if (g0 > 0 || g_split(rc, g0) > g0) split_ctas += (int64_t)1 << g_split(rc, g0);
            }
            const bool split = split_ctas <= 2 * (int64_t)num_sms;
            for (size_t q = b; q < e; ++q) {
                const int rc = nodes[flat[q]].rows_cap;
                int g = g_fit(rc);
                if (split && (1 << g) <= RID_MAX_CLUSTER) g = g_split(rc, g);
                ((1 << g) <= RID_MAX_CLUSTER ? grp[g] : big).push_back(flat[q]);
            }
            // a cluster shape the device cannot co-schedule falls back to global memory
            for (int g = 1; (1 << g) <= RID_MAX_CLUSTER; ++g) {
                if (grp[g].empty()) continue;
                cudaLaunchConfig_t cfg{};
                cfg.gridDim = dim3((unsigned)(1 << g));
                cfg.blockDim = dim3(RID_THREADS);
                cfg.dynamicSmemBytes = RID_SMEM;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = (unsigned)(1 << g);
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int ncl = 0;
                if (cudaOccupancyMaxActiveClusters(&ncl, row_id_cluster_kernel<T>, &cfg) != cudaSuccess || ncl < 1) {
                    cudaGetLastError();
                    big.insert(big.end(), grp[g].begin(), grp[g].end());
                    grp[g].clear();
                }
            }
            // the launches of different cluster shapes are independent: with more
            // than one, each runs on a side stream forked from st and joined back
            int nlaunch = big.empty() ? 0 : 1;
            for (int g = 0; (1 << g) <= RID_MAX_CLUSTER; ++g) nlaunch += grp[g].empty() ? 0 : 1;
            SideFork fork(st, nlaunch > 1 ? nlaunch : 0, F.side_streams);
            HSS_TRY(fork.status);
            std::vector<std::unique_ptr<DeviceVec<int>>> lists;
            int li = 0;
            for (int g = 0; (1 << g) <= RID_MAX_CLUSTER; ++g) {
                if (grp[g].empty()) continue;
                const int C = 1 << g;
                cudaStream_t ls = fork.stream(li++);
                int rcmax = 1;
                for (int id : grp[g]) rcmax = std::max(rcmax, nodes[id].rows_cap);
                lists.emplace_back(new DeviceVec<int>(st));
                DeviceVec<int>& dl = *lists.back();
                HSS_TRY(dl.upload(grp[g], st));
                HSS_TRY(fork.start(li - 1));
                const size_t sm = rid_bytes(rcmax, C);
                if (C == 1) {
                    row_id_cluster_kernel<T><<<(unsigned)grp[g].size(), RID_THREADS, sm, ls>>>(dl.p, dnodes.p, ws.p, iws.p,
                                                                                              kk.p, rows.p, eps, rank_cap);
                } else {
                    cudaLaunchConfig_t cfg{};
                    cfg.gridDim = dim3((unsigned)(grp[g].size() * C));
                    cfg.blockDim = dim3(RID_THREADS);
                    cfg.dynamicSmemBytes = sm;
                    cfg.stream = ls;
                    cudaLaunchAttribute at[1];
                    at[0].id = cudaLaunchAttributeClusterDimension;
                    at[0].val.clusterDim.x = (unsigned)C;
                    at[0].val.clusterDim.y = 1;
                    at[0].val.clusterDim.z = 1;
                    cfg.attrs = at;
                    cfg.numAttrs = 1;
                    HSS_TRY(cudaLaunchKernelEx(&cfg, row_id_cluster_kernel<T>, (const int*)dl.p, (const HNode*)dnodes.p,
                                               ws.p, iws.p, kk.p, (const int*)rows.p, eps, rank_cap));
                }
                NDHSS_LAUNCH_CHECK("row_id_cluster_kernel");
                HSS_TRY(fork.finish(li - 1));
            }
            if (!big.empty()) {
                cudaStream_t ls = fork.stream(li++);
                lists.emplace_back(new DeviceVec<int>(st));
                DeviceVec<int>& dl = *lists.back();
                HSS_TRY(dl.upload(big, st));
                HSS_TRY(fork.start(li - 1));
                row_id_kernel<T><<<(unsigned)big.size(), 512, smem_base, ls>>>(dl.p, dnodes.p, ws.p, iws.p, kk.p, rows.p,
                                                                                eps, rank_cap, 0);
                NDHSS_LAUNCH_CHECK("row_id_kernel");
                HSS_TRY(fork.finish(li - 1));
            }
            // st waits for every side launch before the node lists are freed on it
            HSS_TRY(fork.join());
            return NDHSS_OK;
        };
        if (lowrank) {
            transpose_samples_kernel<T><<<dim3(64, nf), 256, 0, st>>>(dfr.p, dnodes.p, ws.p, iws.p, rows.p);
            NDHSS_LAUNCH_CHECK("transpose_samples_kernel");
            {
                const ndhss_status rc = launch_row_id(loff[0], loff[1]);
                if (rc != NDHSS_OK) return rc;
            }
            gather_rows_kernel<T><<<dim3(64, nf), 256, 0, st>>>(dfr.p, dnodes.p, ws.p, iws.p, kk.p);
            NDHSS_LAUNCH_CHECK("gather_rows_kernel");
            // Zt = X (R(J,:) Omega~) : needs the ranks on the host for the GEMM shapes
            std::vector<int> hk(nodes.size());
            HSS_TRY(cudaMemcpyAsync(hk.data(), kk.p, hk.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
            HSS_TRY(cudaStreamSynchronize(st));
            std::vector<GemmJob> g2, g3;
            for (int i = 0; i < nf; ++i) {
                const int k = hk[fr[i].root];
                const HNode& nd = nodes[fr[i].root];
                g2.push_back({fr[i].RJ, fr[i].Ot, fr[i].T1, kcap, fr[i].ncol, kcap, k, r, fr[i].ncol, 0, 1.0});
                g2.back().realB = 1;
                g3.push_back({ws.p + nd.o_x, fr[i].T1, fr[i].Zt, nd.rows_cap, kcap, fr[i].n, fr[i].n, r, k, 0, 1.0});
            }
            {
                ndhss_status rc = run_bgemm<T>(g2, st);
                if (rc == NDHSS_OK) rc = run_bgemm<T>(g3, st);
                if (rc != NDHSS_OK) return rc;
            }
        } else {
            for (int l = maxlev; l >= 1; --l) {
                const unsigned cnt = (unsigned)(loff[l + 1] - loff[l]);
                if (!cnt) continue;
                int leaf_rows = 1;
                for (size_t q = loff[l]; q < loff[l + 1]; ++q)
                    if (nodes[flat[q]].c1 < 0) leaf_rows = std::max(leaf_rows, nodes[flat[q]].hi - nodes[flat[q]].lo);
                const unsigned tf = (unsigned)(std::max(tiles64(leaf_rows), 2 * tiles64(kcap)) * tiles64(p));
                form_sloc_kernel<T><<<dim3(cnt, tf), HT, 0, st>>>(dflat.p + loff[l], dnodes.p, dfr.p, ws.p, iws.p, kk.p,
                                                                 rows.p);
                NDHSS_LAUNCH_CHECK("form_sloc_kernel");
                {
                    const ndhss_status rc = launch_row_id(loff[l], loff[l + 1]);
                    if (rc != NDHSS_OK) return rc;
                }
                finish_kernel<T><<<dim3(cnt, tiles64(kcap) * tiles64(p)), HT, 0, st>>>(dflat.p + loff[l], dnodes.p, dfr.p,
                                                                                      ws.p, iws.p, kk.p, rows.p);
                NDHSS_LAUNCH_CHECK("finish_kernel");
            }
            // estimator: Zt = HSS(S) Omega~
            std::vector<const T*> xin(nf);
            std::vector<T*> yout(nf);
            std::vector<int64_t> lx(nf), ly(nf);
            std::vector<int> ncs(nf, r);
            for (int i = 0; i < nf; ++i) {
                xin[i] = static_cast<const T*>(fr[i].Ot);
                yout[i] = static_cast<T*>(fr[i].Zt);
                lx[i] = ly[i] = fr[i].n;
            }
            DeviceVec<const T*> dx(st);
            DeviceVec<T*> dy(st);
            DeviceVec<int64_t> dlx(st), dly(st);
            DeviceVec<int> dncs(st);
            HSS_TRY(dx.upload(xin, st));
            HSS_TRY(dy.upload(yout, st));
            HSS_TRY(dlx.upload(lx, st));
            HSS_TRY(dly.upload(ly, st));
            HSS_TRY(dncs.upload(ncs, st));
            std::vector<char> all(nf, 1);
            ndhss_status rc = hss_matvec_run<T>(nodes, all, maxlev, dnodes.p, dfr.p, ws.p, ws.p, iws.p, kk.p, rows.p, dx.p,
                                               dlx.p, dy.p, dly.p, dncs.p, r, (int64_t)kcap, st);
            if (rc != NDHSS_OK) return rc;
        }
        DeviceVec<double> dn(st);
        HSS_TRY(dn.alloc(2 * nf));
        est_norm_kernel<T><<<nf, HT, 0, st>>>(dfr.p, r, dn.p);
        NDHSS_LAUNCH_CHECK("est_norm_kernel");
        std::vector<double> hn(2 * nf);
        std::vector<int> hk(nodes.size());
        HSS_TRY(cudaMemcpyAsync(hn.data(), dn.p, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        HSS_TRY(cudaMemcpyAsync(hk.data(), kk.p, hk.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
        HSS_TRY(cudaStreamSynchronize(st));
        std::vector<int> done, still;
        for (int i = 0; i < nf; ++i) {
            const Problem& pb = probs[active[i]];
            const int lim = lowrank ? std::min({pb.n, pb.ncol, rank_cap + OVERSAMPLE_MIN})
                                    : std::min(pb.n, rank_cap + OVERSAMPLE_MIN);
            // stop when eps is met, when the samples exhaust the block or reach
            // MAX_SAMPLES, or when a round did not halve an estimate that is already
            // within 10^3 unit roundoffs of the block's norm (the arithmetic's floor;
            // above it a slowly decaying spectrum keeps sampling)
            const double err = hn[2 * i], ref = hn[2 * i + 1];
            const bool stalled = err > 0.5 * prev_err[active[i]] && err <= stagnation_floor<T>() * ref;
            if (err <= eps * ref || p >= lim || p + r > MAX_SAMPLES || stalled) done.push_back(i);
            else still.push_back(active[i]);
            prev_err[active[i]] = err;
        }
        // finalize the retired problems
        if (!done.empty()) {
            if (lowrank) {
                // X (n x k, ld n) then R(J, :)^T (ncol x k, ld ncol) of every retired
                // problem, gathered on the device into one buffer per sampling round
                std::vector<LrOut> jobs;
                std::vector<int64_t> offs;
                int64_t tot = 0;
                for (int i : done) {
                    const int k = hk[fr[i].root];
                    const HNode& nd = nodes[fr[i].root];
                    kout[active[i]] = k;
                    offs.push_back(tot);
                    if (k > 0) {
                        jobs.push_back({ws.p + nd.o_x, fr[i].RJ, nullptr, nd.rows_cap, kcap, (int)fr[i].n,
                                        (int)fr[i].ncol, k, 0});
                        jobs.back().dst = reinterpret_cast<void*>(tot);
                    }
                    tot += ((int64_t)fr[i].n + fr[i].ncol) * k;
                }
                void* buf = nullptr;
                if (pool_malloc_async(&buf, (size_t)std::max<int64_t>(tot, 1) * sizeof(T), st) != cudaSuccess) {
                    cudaGetLastError();
                    return set_error(NDHSS_ERR_OOM, "hss: low-rank storage");
                }
                F.lr_bufs.push_back(buf);
                F.dev_bytes += tot * (int64_t)sizeof(T);
                for (size_t q = 0; q < done.size(); ++q)
                    (*lr_dev)[active[done[q]]] = reinterpret_cast<uint64_t>(static_cast<T*>(buf) + offs[q]);
                for (auto& j : jobs) j.dst = static_cast<T*>(buf) + reinterpret_cast<int64_t>(j.dst);
                if (!jobs.empty()) {
                    DeviceVec<LrOut> dj(st);
                    HSS_TRY(dj.upload(jobs, st));
                    lr_out_kernel<T><<<(unsigned)jobs.size(), 256, 0, st>>>(dj.p);
                    NDHSS_LAUNCH_CHECK("lr_out_kernel");
                }
            } else if (ulv) {
                // HSS generators of the retired blocks into a ULV factorization (the
                // blocks themselves stay as they are)
                std::vector<char> keep(nf, 0);
                for (int i : done) keep[i] = 1;
                std::vector<int> inner;
                std::vector<int64_t> ob;
                int64_t btot = 0;
                for (size_t q = 0; q < nodes.size(); ++q) {
                    const HNode& nd = nodes[q];
                    if (!keep[nd.front] || nd.c1 < 0) continue;
                    inner.push_back((int)q);
                    ob.push_back(btot);
                    btot += 2 * std::max<int64_t>((int64_t)hk[nd.c1] * hk[nd.c2], 1);
                }
                DeviceVec<T> bb(st);
                HSS_TRY(bb.alloc(std::max<int64_t>(btot, 1)));
                std::vector<T*> p12, p21;
                for (size_t q = 0; q < inner.size(); ++q) {
                    const HNode& nd = nodes[inner[q]];
                    p12.push_back(bb.p + ob[q]);
                    p21.push_back(bb.p + ob[q] + std::max<int64_t>((int64_t)hk[nd.c1] * hk[nd.c2], 1));
                }
                DeviceVec<int> dinner(st);
                DeviceVec<T*> dp12(st), dp21(st);
                HSS_TRY(dinner.upload(inner, st));
                HSS_TRY(dp12.upload(p12, st));
                HSS_TRY(dp21.upload(p21, st));
                if (!inner.empty()) {
                    gather_b_kernel<T><<<(unsigned)inner.size(), HT, 0, st>>>(dinner.p, dnodes.p, dfr.p, iws.p, kk.p, dp12.p,
                                                                             dp21.p);
                    NDHSS_LAUNCH_CHECK("gather_b_kernel");
                }
                std::vector<int> inner_of(nodes.size(), -1);
                for (size_t q = 0; q < inner.size(); ++q) inner_of[inner[q]] = (int)q;
                std::vector<UlvIn> uin;
                std::vector<int> idx_of(nodes.size(), -1);
                for (size_t q = 0; q < nodes.size(); ++q)
                    if (keep[nodes[q].front]) { idx_of[q] = (int)uin.size(); uin.push_back({}); }
                for (size_t q = 0; q < nodes.size(); ++q) {
                    if (idx_of[q] < 0) continue;
                    const HNode& nd = nodes[q];
                    const HFront& f = fr[nd.front];
                    UlvIn& u = uin[idx_of[q]];
                    u.s = probs[active[nd.front]].node;
                    u.lo = nd.lo;
                    u.hi = nd.hi;
                    u.level = nd.level;
                    u.c1 = nd.c1 < 0 ? -1 : idx_of[nd.c1];
                    u.c2 = nd.c2 < 0 ? -1 : idx_of[nd.c2];
                    u.root = (int)q == f.root;
                    u.k = hk[q];
                    u.D0 = static_cast<const T*>(f.S) + (int64_t)nd.lo * f.lds + nd.lo;
                    u.ldd0 = f.lds;
                    u.X = ws.p + nd.o_x;
                    u.ldx = nd.rows_cap;
                    u.B12 = inner_of[q] >= 0 ? p12[inner_of[q]] : nullptr;
                    u.B21 = inner_of[q] >= 0 ? p21[inner_of[q]] : nullptr;
                }
                ndhss_status rc = ulv_factor_nodes<T>(uin, F, st);
                if (rc != NDHSS_OK) return rc;
                for (int i : done) {
                    int km = 0;
                    for (size_t q = 0; q < nodes.size(); ++q)
                        if (nodes[q].front == i && (int)q != fr[i].root) km = std::max(km, hk[q]);
                    kout[active[i]] = km;
                }
            } else {
                // S_HSS written over S: leaf diagonal blocks stay; every off-diagonal block
                // S(I_c1, I_c2) = U~_c1 B12 U~_c2^T with the expanded nested bases
                // U~_leaf = X_leaf, U~_i = blockdiag(U~_c1, U~_c2) X_i (Eq. 2.3)
                std::vector<char> keep(nf, 0);
                for (int i : done) keep[i] = 1;
                std::vector<const T*> up(nodes.size(), nullptr);
                std::vector<int64_t> uld(nodes.size(), 1), uoff(nodes.size(), -1);
                int64_t utot = 0;
                for (size_t q = 0; q < nodes.size(); ++q) {
                    const HNode& nd = nodes[q];
                    if (!keep[nd.front] || (int)q == fr[nd.front].root) continue;
                    if (nd.c1 < 0) {
                        up[q] = ws.p + nd.o_x;
                        uld[q] = nd.rows_cap;
                    } else {
                        uoff[q] = utot;
                        uld[q] = nd.hi - nd.lo;
                        utot += (int64_t)(nd.hi - nd.lo) * std::max(hk[q], 1);
                    }
                }
                int64_t btot = 0;
                std::vector<int> inner;
                std::vector<int64_t> o12, o21, ot12, ot21;
                for (size_t q = 0; q < nodes.size(); ++q) {
                    const HNode& nd = nodes[q];
                    if (!keep[nd.front] || nd.c1 < 0) continue;
                    const int64_t k1 = hk[nd.c1], k2 = hk[nd.c2];
                    const int64_t s1 = nodes[nd.c1].hi - nodes[nd.c1].lo, s2 = nodes[nd.c2].hi - nodes[nd.c2].lo;
                    inner.push_back((int)q);
                    o12.push_back(btot); btot += std::max<int64_t>(k1 * k2, 1);
                    o21.push_back(btot); btot += std::max<int64_t>(k1 * k2, 1);
                    ot12.push_back(btot); btot += std::max<int64_t>(k1 * s2, 1);
                    ot21.push_back(btot); btot += std::max<int64_t>(k2 * s1, 1);
                }
                DeviceVec<T> ub(st), bb(st);
                HSS_TRY(ub.alloc(utot));
                HSS_TRY(bb.alloc(btot));
                for (size_t q = 0; q < nodes.size(); ++q)
                    if (uoff[q] >= 0) up[q] = ub.p + uoff[q];
                // expanded bases, deepest level first
                for (int l = maxlev; l >= 1; --l) {
                    std::vector<GemmJob> gj2;
                    for (size_t q = 0; q < nodes.size(); ++q) {
                        const HNode& nd = nodes[q];
                        if (nd.level != l || uoff[q] < 0) continue;
                        const int k = hk[q], k1 = hk[nd.c1], k2 = hk[nd.c2];
                        const int s1 = nodes[nd.c1].hi - nodes[nd.c1].lo, s2 = nodes[nd.c2].hi - nodes[nd.c2].lo;
                        const T* X = ws.p + nd.o_x;
                        T* U = const_cast<T*>(up[q]);
                        gj2.push_back({up[nd.c1], X, U, uld[nd.c1], nd.rows_cap, uld[q], s1, k, k1, 0, 1.0});
                        gj2.push_back({up[nd.c2], X + k1, U + s1, uld[nd.c2], nd.rows_cap, uld[q], s2, k, k2, 0, 1.0});
                    }
                    if (gj2.empty()) continue;
                    const ndhss_status rc = run_bgemm<T>(gj2, st);
                    if (rc != NDHSS_OK) return rc;
                }
                // coupling blocks (all gathered before any block of S is overwritten)
                std::vector<T*> p12, p21;
                for (size_t q = 0; q < inner.size(); ++q) {
                    p12.push_back(bb.p + o12[q]);
                    p21.push_back(bb.p + o21[q]);
                }
                DeviceVec<int> dinner(st);
                DeviceVec<T*> dp12(st), dp21(st);
                HSS_TRY(dinner.upload(inner, st));
                HSS_TRY(dp12.upload(p12, st));
                HSS_TRY(dp21.upload(p21, st));
                if (!inner.empty()) {
                    gather_b_kernel<T><<<(unsigned)inner.size(), HT, 0, st>>>(dinner.p, dnodes.p, dfr.p, iws.p, kk.p, dp12.p,
                                                                             dp21.p);
                    NDHSS_LAUNCH_CHECK("gather_b_kernel");
                }
                // T12 = B12 U~_c2^T, T21 = B21 U~_c1^T; then the blocks of S
                std::vector<GemmJob> g1, g2;
                int m1 = 1, n1 = 1, m2 = 1, n2 = 1;
                for (size_t q = 0; q < inner.size(); ++q) {
                    const HNode& nd = nodes[inner[q]];
                    const HFront& f = fr[nd.front];
                    const int k1 = hk[nd.c1], k2 = hk[nd.c2];
                    const HNode& a = nodes[nd.c1];
                    const HNode& b = nodes[nd.c2];
                    const int s1 = a.hi - a.lo, s2 = b.hi - b.lo;
                    T* t12 = bb.p + ot12[q];
                    T* t21 = bb.p + ot21[q];
                    GemmJob x{p12[q], up[nd.c2], t12, std::max(k1, 1), uld[nd.c2], std::max(k1, 1), k1, s2, k2, 0, 1.0};
                    x.transB = 1;
                    GemmJob y{p21[q], up[nd.c1], t21, std::max(k2, 1), uld[nd.c1], std::max(k2, 1), k2, s1, k1, 0, 1.0};
                    y.transB = 1;
                    g1.push_back(x);
                    g1.push_back(y);
                    T* Sb = static_cast<T*>(f.S);
                    g2.push_back({up[nd.c1], t12, Sb + (int64_t)b.lo * f.lds + a.lo, uld[nd.c1], std::max(k1, 1), f.lds, s1,
                                  s2, k1, 0, 1.0});
                    g2.push_back({up[nd.c2], t21, Sb + (int64_t)a.lo * f.lds + b.lo, uld[nd.c2], std::max(k2, 1), f.lds, s2,
                                  s1, k2, 0, 1.0});
                    m1 = std::max({m1, k1, k2});
                    n1 = std::max({n1, s1, s2});
                    m2 = std::max({m2, s1, s2});
                    n2 = std::max({n2, s1, s2});
                }
                if (!g1.empty()) {
                    ndhss_status rc = run_bgemm<T>(g1, st);
                    if (rc == NDHSS_OK) rc = run_bgemm<T>(g2, st);
                    if (rc != NDHSS_OK) return rc;
                }
                HSS_TRY(cudaStreamSynchronize(st));
                for (int i : done) {
                    int km = 0;
                    for (size_t q = 0; q < nodes.size(); ++q)
                        if (nodes[q].front == i && (int)q != fr[i].root) km = std::max(km, hk[q]);
                    kout[active[i]] = km;
                }
            }
        }
        F.hss_rounds_max = std::max(F.hss_rounds_max, round + 1);
        active = still;
        p += r;
        ++round;
    }
    return NDHSS_OK;
}

template <typename T>
ndhss_status compress_level_impl(FactorData& F, const Tree& t, int level, const ndhss_factor_opts& o, cudaStream_t st) {
    T* base = static_cast<T*>(F.d_front);
    const int beta = std::max(o.beta, 1);
    std::vector<Problem> sp;
    for (int s : F.levels[level]) {
        const int64_t mi = F.m_i(s), mb = F.m_b(s), m = mi + mb;
        T* Fs = base + F.foff[s];
        const int par = t.parent(s);
        if (mb > beta && par >= 0) {
            int top = 0;
            for (int q = 0; q < mb; ++q) top += (t.emap[t.b_off(s) + q] < t.m_i(par)) ? 1 : 0;
            sp.push_back({s, (int)mb, (int)mb, m, Fs + mi * m + mi, top, (uint64_t)2 * s});
        }
        // R^sigma is read only by the apply: queued here, compressed in one
        // batch of all levels beside the root level's elimination (or after
        // the level loop)
        if (level < F.L_hss && mb > 0 && mi > 0) F.lr_pending.push_back(s);
    }
    std::vector<int> ks;
    if (!sp.empty()) {
        ndhss_status rc = compress_problems<T>(sp, false, o, ks, nullptr, F, st);
        if (rc != NDHSS_OK) return rc;
        for (int k : ks) F.kmax = std::max(F.kmax, k);
    }
    return NDHSS_OK;
}

// Low-rank R^sigma ~ X R(J, :) of the given fronts (each keeps its own
// Philox stream 2 s + 1, so the result does not depend on the batching).
// F is only read here, apart from the fronts' own lr_ptr / lr_k elements;
// the storage and counters go to acc: the factorization runs this on a
// second host thread while the main stream eliminates the root level.
template <typename T>
ndhss_status lowrank_fronts_impl(FactorData& F, const std::vector<int32_t>& fronts, FactorData& acc, int* kmax,
                                 const ndhss_factor_opts& o, cudaStream_t st) {
    T* base = static_cast<T*>(F.d_front);
    std::vector<Problem> rp;
    for (int s : fronts) {
        const int64_t mi = F.m_i(s), mb = F.m_b(s), m = mi + mb;
        rp.push_back({s, (int)mi, (int)mb, m, base + F.foff[s] + mi * m, 0, (uint64_t)2 * s + 1});
    }
    if (rp.empty()) return NDHSS_OK;
    std::vector<int> kr;
    std::vector<uint64_t> ptr;
    ndhss_status rc = compress_problems<T>(rp, true, o, kr, &ptr, acc, st);
    if (rc != NDHSS_OK) return rc;
    for (size_t i = 0; i < rp.size(); ++i) {
        F.lr_ptr[rp[i].node] = ptr[i];
        F.lr_k[rp[i].node] = kr[i];
        *kmax = std::max(*kmax, kr[i]);
    }
    return NDHSS_OK;
}

// The fronts queued by compress_level_impl, all levels in one batch.
template <typename T>
ndhss_status lowrank_pending_impl(FactorData& F, const ndhss_factor_opts& o, cudaStream_t st) {
    std::vector<int32_t> pending;
    pending.swap(F.lr_pending);
    int kmax = F.kmax;
    const ndhss_status rc = lowrank_fronts_impl<T>(F, pending, F, &kmax, o, st);
    F.kmax = kmax;
    return rc;
}

}  // namespace

namespace {

template <typename T>
ndhss_status ulv_level_impl(FactorData& F, const Tree& t, int level, T* aii, const std::vector<int64_t>& aii_off,
                            const ndhss_factor_opts& o, cudaStream_t st) {
    const int beta = std::max(o.beta, 1);
    std::vector<Problem> probs;
    std::vector<UlvIn> small;
    for (int s : F.levels[level]) {
        if (aii_off[s] < 0) continue;
        const int mi = t.m_i(s);
        T* blk = aii + aii_off[s];
        if (mi <= beta) {
            // one HSS block: the ULV is the inverse of A_ii (as the oracle's single-node tree)
            UlvIn u{};
            u.s = s;
            u.lo = 0;
            u.hi = mi;
            u.level = 0;
            u.c1 = u.c2 = -1;
            u.root = 1;
            u.D0 = blk;
            u.ldd0 = mi;
            small.push_back(u);
        } else {
            probs.push_back({s, mi, mi, mi, blk, -1, (uint64_t)2 * t.nnodes + s});
        }
    }
    if (!small.empty()) {
        // independent single-node fronts: one launch, each its own root
        ndhss_status rc = ulv_factor_nodes<T>(small, F, st);
        if (rc != NDHSS_OK) return rc;
    }
    if (!probs.empty()) {
        std::vector<int> ks;
        ndhss_status rc = compress_problems<T>(probs, false, o, ks, nullptr, F, st, true);
        if (rc != NDHSS_OK) return rc;
        for (int k : ks) F.kmax = std::max(F.kmax, k);
    }
    return NDHSS_OK;
}

}  // namespace

ndhss_status hss_ulv_level(FactorData& F, const Tree& t, int level, void* aii, const std::vector<int64_t>& aii_off,
                           const ndhss_factor_opts& o, cudaStream_t st) {
    const bool cplx = F.vtype == NDHSS_C128;
    if (!cplx && F.prec == NDHSS_FP64) return ulv_level_impl<double>(F, t, level, (double*)aii, aii_off, o, st);
    if (!cplx) return ulv_level_impl<float>(F, t, level, (float*)aii, aii_off, o, st);
    if (F.prec == NDHSS_FP64) return ulv_level_impl<c128>(F, t, level, (c128*)aii, aii_off, o, st);
    return ulv_level_impl<c64>(F, t, level, (c64*)aii, aii_off, o, st);
}

ndhss_status hss_lowrank_pending(FactorData& F, const ndhss_factor_opts& o, cudaStream_t st) {
    const bool cplx = F.vtype == NDHSS_C128;
    if (!cplx && F.prec == NDHSS_FP64) return lowrank_pending_impl<double>(F, o, st);
    if (!cplx) return lowrank_pending_impl<float>(F, o, st);
    if (F.prec == NDHSS_FP64) return lowrank_pending_impl<c128>(F, o, st);
    return lowrank_pending_impl<c64>(F, o, st);
}

ndhss_status hss_lowrank_fronts(FactorData& F, const std::vector<int32_t>& fronts, FactorData& acc, int* kmax,
                                const ndhss_factor_opts& o, cudaStream_t st) {
    const bool cplx = F.vtype == NDHSS_C128;
    if (!cplx && F.prec == NDHSS_FP64) return lowrank_fronts_impl<double>(F, fronts, acc, kmax, o, st);
    if (!cplx) return lowrank_fronts_impl<float>(F, fronts, acc, kmax, o, st);
    if (F.prec == NDHSS_FP64) return lowrank_fronts_impl<c128>(F, fronts, acc, kmax, o, st);
    return lowrank_fronts_impl<c64>(F, fronts, acc, kmax, o, st);
}

ndhss_status hss_compress_level(FactorData& F, const Tree& t, int level, const ndhss_factor_opts& o, cudaStream_t st) {
    if (F.lr_ptr.size() != (size_t)F.nnodes) {
        F.lr_ptr.assign(F.nnodes, 0);
        F.lr_k.assign(F.nnodes, 0);
    }
    const bool cplx = F.vtype == NDHSS_C128;
    if (!cplx && F.prec == NDHSS_FP64) return compress_level_impl<double>(F, t, level, o, st);
    if (!cplx) return compress_level_impl<float>(F, t, level, o, st);
    if (F.prec == NDHSS_FP64) return compress_level_impl<c128>(F, t, level, o, st);
    return compress_level_impl<c64>(F, t, level, o, st);
}

}  // namespace ndhss
