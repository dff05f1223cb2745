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
// least-squares residual |g_{j+1}|; v_{j+1} = w / h_{j+1,j}.  The device
// decides whether the cycle ends (see "device-driven GMRES" below).  After
// each cycle x += V y with H y = g solved on the device, and the float64 true
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
constexpr int RB = 4 * 152;       // reduction grid (four 256-thread blocks per SM)
constexpr int GM_BARRIER = KMAX / 4 + 1;   // counter word of the Arnoldi kernel's grid barrier

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
// GB300's FP64 pipe retires 2 DFMA per clock per SM, and a predicated-off
// FP64 instruction still takes its slot, so the row product issues exactly
// the FMAs it needs: TPR threads per row load all their entries of the row
// at once (up to SP_U each; then the x gathers), the FMA loops run over a
// warp-uniform count (the longest row of the warp, dispatched to an
// exact-count instance), and the imaginary parts of the matrix entries
// (zero inside the domain: the impedance term sits on the boundary) are
// multiplied only when some lane of the warp holds one, after the products
// of the real parts of the same batch of entries.
constexpr int SP_TPR = 2, SP_U = 6;   // best measured on the 256 x 256 P2 Helmholtz matrix (cold L2: 31 us; 4 x 8: 54 us)
static_assert(SP_U <= 8, "spmv_row dispatches up to eight passes per batch");

__device__ __forceinline__ bool spmv_cplx(double) { return false; }
__device__ __forceinline__ bool spmv_cplx(c128 a) { return __double_as_longlong(a.y) != 0; }

template <int NP>
__device__ __forceinline__ void spmv_fmas(const double* a, const double* xv, double& acc, bool) {
#pragma unroll
    for (int u = 0; u < NP; ++u) acc = fma(a[u], xv[u], acc);
}
template <int NP>
__device__ __forceinline__ void spmv_fmas(const c128* a, const c128* xv, c128& acc, bool any_cplx) {
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        acc.x = fma(a[u].x, xv[u].x, acc.x);
        acc.y = fma(a[u].x, xv[u].y, acc.y);
    }
    if (any_cplx) {
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            acc.x = fma(-a[u].y, xv[u].y, acc.x);
            acc.y = fma(a[u].y, xv[u].x, acc.y);
        }
    }
}

// this thread's share of row `row` (lane = its index among the row's TPR
// threads; U <= 8 entries per batch); `valid` false for threads past the
// last row (they still take part in the warp's votes)
template <typename V, int TPR, int U>
__device__ __forceinline__ V spmv_row(bool valid, int64_t row, int lane, const int32_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ col, const V* __restrict__ vals,
                                      const V* __restrict__ x) {
    const int k0 = valid ? rowptr[row] : 0, k1 = valid ? rowptr[row + 1] : 0;
    int np = (k1 - k0 + TPR - 1) / TPR;          // passes this row needs
    for (int o = 16; o; o >>= 1) np = max(np, __shfl_xor_sync(0xffffffffu, np, o));
    V acc = zero<V>();
    for (int p0 = 0; p0 < np; p0 += U) {
        int c[U];
        V a[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + lane + (p0 + u) * TPR;
            const bool ok = p0 + u < np && k < k1;
            c[u] = ok ? col[k] : -1;
            a[u] = ok ? vals[k] : zero<V>();
        }
        bool cx = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xv[u] = c[u] >= 0 ? x[c[u]] : zero<V>();
            cx = cx || spmv_cplx(a[u]);
        }
        const bool any_cplx = __any_sync(0xffffffffu, cx);
        switch (min(U, np - p0)) {
#define NDHSS_SPF(NN) case NN: if constexpr (NN <= U) spmv_fmas<NN>(a, xv, acc, any_cplx); break;
            NDHSS_SPF(1) NDHSS_SPF(2) NDHSS_SPF(3) NDHSS_SPF(4) NDHSS_SPF(5) NDHSS_SPF(6) NDHSS_SPF(7) NDHSS_SPF(8)
#undef NDHSS_SPF
            default: break;
        }
    }
    if constexpr (sizeof(V) == 8) {
        for (int o = TPR / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
    } else {
        for (int o = TPR / 2; o; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o, TPR);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o, TPR);
        }
    }
    return acc;
}

template <typename V, int TPR, int U>
__global__ void __launch_bounds__(256) spmv_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                   const V* __restrict__ vals, const V* __restrict__ x, V* __restrict__ y) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int lane = (int)(gt % TPR);
    const V acc = spmv_row<V, TPR, U>(row < n, row, lane, rowptr, col, vals, x);
    if (row < n && lane == 0) y[row] = acc;
}

template <typename V>
ndhss_status spmv_launch(int n, const int32_t* rowptr, const int32_t* col, const V* vals, const V* x, V* y,
                         cudaStream_t st) {
    const int64_t threads = (int64_t)n * SP_TPR;
    spmv_kernel<V, SP_TPR, SP_U><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rowptr, col, vals, x, y);
    NDHSS_LAUNCH_CHECK("spmv_kernel");
    return NDHSS_OK;
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

// ------------------------------------------------ device-driven GMRES
// The host enqueues the same block of launches again and again; the device
// state decides what each block does, so no launch waits for a decision
// taken on the host:
//   begin     (RESTART with a finished cycle: x += V y; chooses the vectors
//             of the SpMV and the apply below)
//   SpMV      t = s A v  (RESTART: v = x, s = 1; STEP: v = raw basis vector
//             j, s its scale)
//   resid     RESTART: r = b - t, ||r||, the float64 true residual decides
//             convergence, maxit and the cycle tolerances
//   apply     RESTART: V_0 = P^{-1} r;  STEP: V_{j+1} = P^{-1} t
//   dot       RESTART: beta = ||V_0||, g = beta e_1;  STEP: h1 = V^H w
//   axdot     STEP: w -= V h1, h2 = V^H w   (classical Gram-Schmidt twice)
//   axnorm    STEP: w -= V h2, ||w||, the Hessenberg column and its Givens
//             rotation, |g_{j+1}| decides whether the cycle ends (then
//             y = H^{-1} g for the next block's begin); writes the block's
//             status word to pinned host memory
// Basis vectors stay unnormalised (raw w); each carries its scale 1/||w||,
// applied wherever it is read.  Kernels of a finished solve return at once.
// The host reads the status word of block b - 1 while block b runs, so the
// GPU never idles on a host round trip; at most one block of no-op
// launches follows convergence.
//
// Reductions are deterministic: each block writes its partial sums and the
// last block to finish (ticket counter) adds them in block order.
enum : int { GM_RESTART = 0, GM_STEP = 1 };
constexpr int GM_MAX_IT = 1000;               // maxit allowed by ndhss_gmres
constexpr int GM_MAX_BLOCKS = 2 * GM_MAX_IT + 8;   // a solve takes at most 2 maxit + 2 blocks

struct GmStatus {
    int32_t done, its, pad0, pad1;
};

template <typename V>
struct alignas(16) GmDev {
    int32_t mode, bmode, j, jend, its, cycles, done, have_cycle, skip, bnorm_set, maxit, R;
    int32_t spmv_zero, pad_[3];        // 1: this block's SpMV input is x = 0 (the first restart)
    double bnorm, zbnorm, beta, relres, last_res, prev_rel, cyc_target, rtol_eff, tol, inner;
    const V* spmv_in;
    V* spmv_out;
    double spmv_scale;
    ApplyInd ind;
    unsigned counter[KMAX / 4 + 2];      // reduction tickets (one per dot-product chunk)
    double scale[KMAX];
    V g[KMAX], H[KMAX * KMAX], sn[KMAX], h1[KMAX], h2[KMAX], y[KMAX];
    double cs[KMAX];
    uint8_t ran[GM_MAX_BLOCKS];          // per block: 1 the SpMV ran, 2 the apply ran
};

// The last block of a reduction takes its decisions on a shared-memory copy
// of the state (one parallel load; thread 0's scalar code would otherwise wait
// out a global-memory round trip per field) and writes it back.
template <typename V> __device__ __forceinline__ V from_real(double v);
template <> __device__ __forceinline__ double from_real<double>(double v) { return v; }
template <> __device__ __forceinline__ c128 from_real<c128>(double v) { return {v, 0.0}; }

// ticket of the last block of a reduction (resets the counter for the next
// one).  Only thread 0 wrote the block's partial, so only thread 0 fences
// before taking its ticket (a fence in every thread of every block costs
// more than the reduction).
__device__ __forceinline__ bool last_block(unsigned* counter, unsigned nblocks) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter, 1u) == nblocks - 1;
        if (s_last) *counter = 0;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// block sum of one value per thread, valid in thread 0
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
    __shared__ T sred[RT / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = zero<T>();
    if (threadIdx.x == 0)
        for (int q = 0; q < RT / 32; ++q) s += sred[q];
    __syncthreads();
    return s;
}

// sum of the grid's partials by the whole (last) block, four loads in flight
// per thread, each thread's share in a fixed order, then the block's fixed
// tree (deterministic); valid in thread 0
template <typename T>
__device__ T block_sum_partials(const T* partial, unsigned nb) {
    T s = zero<T>();
    unsigned q = threadIdx.x;
    for (; q + 3 * RT < nb; q += 4 * RT) {
        const T a0 = ldcg(partial + q), a1 = ldcg(partial + q + RT), a2 = ldcg(partial + q + 2 * RT),
                a3 = ldcg(partial + q + 3 * RT);
        s += a0;
        s += a1;
        s += a2;
        s += a3;
    }
    for (; q < nb; q += RT) s += ldcg(partial + q);
    return block_sum(s);
}

template <typename V>
__global__ void gm_init_kernel(GmDev<V>* S, int R, int maxit, double tol, double inner, double rtol) {
    S->mode = GM_RESTART;
    S->bmode = GM_RESTART;
    S->j = S->jend = S->its = S->cycles = S->done = S->have_cycle = S->skip = S->bnorm_set = 0;
    S->spmv_zero = 0;
    S->maxit = maxit;
    S->R = R;
    S->bnorm = 0.0;
    S->zbnorm = -1.0;
    S->beta = S->relres = 0.0;
    S->last_res = 1.0;
    S->prev_rel = INFINITY;
    S->cyc_target = 0.0;
    S->rtol_eff = rtol;
    S->tol = tol;
    S->inner = inner;
    for (int q = 0; q < KMAX / 4 + 2; ++q) S->counter[q] = 0;
    S->ind.skip = &S->skip;
    for (int b = 0; b < GM_MAX_BLOCKS; ++b) S->ran[b] = 0;
}

template <typename V>
__global__ void __launch_bounds__(256) gm_begin_kernel(GmDev<V>* S, V* __restrict__ x, const V* __restrict__ Vb, int64_t ldv,
                                                       V* t, V* r, int n, int blk) {
    if (S->done) return;
    const int mode = S->mode;
    if (mode == GM_RESTART && S->have_cycle) {
        // x += V y, V_i = scale_i raw_i (y solved when the cycle ended)
        __shared__ V cy[KMAX];
        const int k = S->jend;
        if (threadIdx.x < k) cy[threadIdx.x] = scale(S->y[threadIdx.x], S->scale[threadIdx.x]);
        __syncthreads();
        for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
            V acc = x[row];
            for (int i = 0; i < k; ++i) acc = fmac(Vb[row + i * ldv], cy[i], acc);
            x[row] = acc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->bmode = mode;
        S->spmv_out = t;
        if (mode == GM_RESTART) {
            // x = 0 before the first cycle (the solver zeroes it): A x = 0, no product
            S->spmv_zero = (!S->have_cycle && S->its == 0) ? 1 : 0;
            S->spmv_in = x;
            S->spmv_scale = 1.0;
            S->ind.x = r;
            S->ind.y = const_cast<V*>(Vb);
            S->ran[blk] = S->spmv_zero ? 0 : 1;
        } else {
            S->spmv_zero = 0;
            S->spmv_in = Vb + (int64_t)S->j * ldv;
            S->spmv_scale = S->scale[S->j];
            S->ind.x = t;
            S->ind.y = const_cast<V*>(Vb) + (int64_t)(S->j + 1) * ldv;
            S->ran[blk] = 3;
        }
    }
}

// t = s A v with v, t, s chosen by gm_begin (see spmv_kernel)
template <typename V>
__global__ void __launch_bounds__(256) gm_spmv_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                      const V* __restrict__ vals, const GmDev<V>* S) {
    if (S->done || S->spmv_zero) return;
    const V* __restrict__ x = S->spmv_in;
    V* __restrict__ y = S->spmv_out;
    const double sc = S->spmv_scale;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / SP_TPR;
    const int lane = (int)(gt % SP_TPR);
    const V acc = spmv_row<V, SP_TPR, SP_U>(row < n, row, lane, rowptr, col, vals, x);
    if (row < n && lane == 0) y[row] = scale(acc, sc);
}

template <typename V>
__device__ void gm_decide(GmDev<V>* S, double rr, int blk);

// RESTART: r = b - t and the true residual's decisions (gm_decide)
template <typename V>
__global__ void __launch_bounds__(RT, 4) gm_resid_kernel(GmDev<V>* S, const V* __restrict__ b, const V* __restrict__ t,
                                                         V* __restrict__ r, int n, double* __restrict__ partial, int blk) {
    if (S->done || S->bmode != GM_RESTART) return;
    const bool tz = S->spmv_zero != 0;                 // t = A 0 was not formed
    double acc = 0.0;
    for (int64_t row = (int64_t)blockIdx.x * RT + threadIdx.x; row < n; row += (int64_t)gridDim.x * RT) {
        const V v = tz ? b[row] : b[row] - t[row];
        r[row] = v;
        acc += norm2(v);
    }
    const double bs = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = bs;
    if (!last_block(S->counter, gridDim.x)) return;
    const double tot = block_sum_partials(partial, gridDim.x);
    // a handful of scalar fields: thread 0 works on the state in place
    if (threadIdx.x == 0) gm_decide(S, tot, blk);
}

// RESTART: the float64 true residual ||r||^2 = rr decides convergence,
// maxit and the cycle tolerances
template <typename V>
__device__ void gm_decide(GmDev<V>* S, double rr, int blk) {
    const double nr = sqrt(rr);
    if (!S->bnorm_set) {                  // x0 = 0: the first residual is b
        S->bnorm = nr;
        S->bnorm_set = 1;
    }
    S->have_cycle = 0;
    if (S->bnorm == 0.0) {
        S->relres = 0.0;
        S->done = 1;
    } else {
        const double rel = nr / S->bnorm;
        S->relres = rel;
        if (rel <= S->tol) {
            S->done = 1;
        } else if (S->its >= S->maxit) {
            S->done = 2;
        } else {
            // a cycle that did not halve the true residual: later cycles end once
            // their estimate fell by the reduction the true residual still needs
            if (rel > 0.5 * S->prev_rel) {
                S->rtol_eff = 0.0;
                S->cyc_target = 0.1 * S->tol / rel;
            } else if (S->cyc_target > 0.0) {
                S->cyc_target = 0.1 * S->tol / rel;
            }
            S->prev_rel = rel;
            S->cycles++;
            S->ran[blk] |= 2;
        }
    }
    S->skip = S->done != 0;
}

// acc + conj(v) w, with the conjugation in the FMAs' operand signs (GB300's
// FP64 pipe is narrow: a separate negation would cost an FP64 slot)
__device__ __forceinline__ double fmac_conj(double v, double w, double acc) { return fma(v, w, acc); }
__device__ __forceinline__ c128 fmac_conj(c128 v, c128 w, c128 acc) {
    acc.x = fma(v.x, w.x, acc.x);
    acc.x = fma(v.y, w.y, acc.x);
    acc.y = fma(v.x, w.y, acc.y);
    acc.y = fma(-v.y, w.x, acc.y);
    return acc;
}

// STEP, one chunk of C basis vectors i0 .. i0 + C - 1 (<= j): this block's
// partial dot products with w over its rows (every block takes the same rows
// in every pass), one partial per vector and block.  AXPY: w += sum_i
// raw_i cw[i] with all j + 1 vectors first (the first chunk of the second
// Gram-Schmidt pass).  Exact-count instantiations: a predicated-off FP64
// instruction still occupies the FP64 pipe.
template <typename V, int C, bool AXPY>
__device__ void gm_pass_chunk(V* __restrict__ Vb, int64_t ldv, int n, int j, int i0, const V* cw,
                              V* __restrict__ partial) {
    V* w = Vb + (int64_t)(j + 1) * ldv;
    V acc[C];
#pragma unroll
    for (int u = 0; u < C; ++u) acc[u] = zero<V>();
    for (int64_t row = (int64_t)blockIdx.x * RT + threadIdx.x; row < n; row += (int64_t)gridDim.x * RT) {
        V wv = w[row];
        if (AXPY) {
            for (int i = 0; i <= j; ++i) wv = fmac(Vb[row + i * ldv], cw[i], wv);
            w[row] = wv;
        }
        V v[C];
#pragma unroll
        for (int u = 0; u < C; ++u) v[u] = Vb[row + (i0 + u) * ldv];
#pragma unroll
        for (int u = 0; u < C; ++u) acc[u] = fmac_conj(v[u], wv, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < C; ++u) {
        const V bs = block_sum(acc[u]);
        if (threadIdx.x == 0) partial[(int64_t)(i0 + u) * gridDim.x + blockIdx.x] = bs;
    }
}

// basis vectors per chunk: eight real or four complex accumulators and
// loads in flight keep a thread within the 64 registers of four resident
// 256-thread blocks per SM
template <typename V> constexpr int cgs_width() { return sizeof(V) == 16 ? 4 : 8; }

// one Gram-Schmidt pass's partials: V^H w (AXPY: after w += V cw)
template <typename V, bool AXPY>
__device__ void gm_pass(V* Vb, int64_t ldv, int n, int j, const V* cw, V* partial) {
    constexpr int CW = cgs_width<V>();
    for (int i0 = 0; i0 <= j; i0 += CW) {
        const bool ax = AXPY && i0 == 0;
        switch (min(CW, j + 1 - i0)) {
#define NDHSS_CGS(CC)                                                                               \
    case CC:                                                                                        \
        if constexpr (CC <= CW) {                                                                   \
            if (ax) gm_pass_chunk<V, CC, true>(Vb, ldv, n, j, i0, cw, partial);                     \
            else gm_pass_chunk<V, CC, false>(Vb, ldv, n, j, i0, cw, partial);                       \
        }                                                                                           \
        break;
            NDHSS_CGS(1) NDHSS_CGS(2) NDHSS_CGS(3) NDHSS_CGS(4) NDHSS_CGS(5) NDHSS_CGS(6) NDHSS_CGS(7) NDHSS_CGS(8)
#undef NDHSS_CGS
            default: break;
        }
    }
}

// after a grid barrier: h[i] = scale_i * (sum over blocks of the partials of
// vector i), i <= j, into shared memory; warp w adds vectors w, w + 8, ...
// (lane-strided in block order, then the warp's fixed tree: every block gets
// the same values)
template <typename V>
__device__ void gm_sum_partials(const V* __restrict__ partial, int j, const double* scl, V* h) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i <= j; i += RT / 32) {
        V acc = zero<V>();
        for (unsigned q = lane; q < gridDim.x; q += 32) acc += ldcg(partial + (int64_t)i * gridDim.x + q);
        acc = warp_sum(acc);
        if (lane == 0) h[i] = scale(acc, scl[i]);
    }
    __syncthreads();
}

// STEP, last part: w -= V h2, ||w||; the last block forms the Hessenberg
// column j from h1 + h2 and ||w||, applies the previous Givens rotations,
// forms the new one, runs the cycle's stopping tests (and, when the cycle
// ends, solves H y = g), clears the barrier word and writes the status word.
// Only the fields it needs are staged in shared memory.
template <typename V>
__device__ void gm_axnorm_step(GmDev<V>* S, V* __restrict__ Vb, int64_t ldv, int n, double* __restrict__ dpartial,
                               GmStatus* hstat, const V* h1, const V* h2, const double* scl, int j) {
    __shared__ V ch[KMAX];
    if (threadIdx.x <= j) ch[threadIdx.x] = -scale(h2[threadIdx.x], scl[threadIdx.x]);
    __syncthreads();
    V* w = Vb + (int64_t)(j + 1) * ldv;
    double acc = 0.0;
    for (int64_t row = (int64_t)blockIdx.x * RT + threadIdx.x; row < n; row += (int64_t)gridDim.x * RT) {
        V wv = w[row];
        for (int i = 0; i <= j; ++i) wv = fmac(Vb[row + i * ldv], ch[i], wv);
        w[row] = wv;
        acc += norm2(wv);
    }
    const double bs = block_sum(acc);
    if (threadIdx.x == 0) dpartial[blockIdx.x] = bs;
    if (!last_block(S->counter, gridDim.x)) return;
    const double ss = block_sum_partials(dpartial, gridDim.x);
    __shared__ V sHj[KMAX + 1], ssn[KMAX], sy[KMAX], sg[KMAX + 1];
    __shared__ double scs[KMAX];
    __shared__ int s_end, s_k;
    for (int i = threadIdx.x; i < j; i += RT) {
        ssn[i] = S->sn[i];
        scs[i] = S->cs[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        S->counter[GM_BARRIER] = 0;
        const double hn = sqrt(ss);
        V* Hj = sHj;
        for (int i = 0; i <= j; ++i) Hj[i] = h1[i] + h2[i];
        Hj[j + 1] = from_real<V>(hn);
        for (int i = 0; i < j; ++i) {
            const V t0 = scale(Hj[i], scs[i]) + ssn[i] * Hj[i + 1];
            const V t1 = scale(Hj[i + 1], scs[i]) - conjv(ssn[i]) * Hj[i];
            Hj[i] = t0;
            Hj[i + 1] = t1;
        }
        const V a = Hj[j], bb = Hj[j + 1];
        double c;
        V sn;
        const double aa = absv(a), ab = absv(bb);
        if (ab == 0.0) {
            c = 1.0;
            sn = zero<V>();
        } else if (aa == 0.0) {
            c = 0.0;
            sn = scale(conjv(bb), 1.0 / ab);
        } else {
            const double tt = hypot(aa, ab);
            c = aa / tt;
            sn = scale(a, 1.0 / aa) * scale(conjv(bb), 1.0 / tt);
        }
        S->cs[j] = c;
        S->sn[j] = sn;
        Hj[j] = scale(a, c) + sn * bb;
        Hj[j + 1] = zero<V>();
        const V gj = S->g[j];
        const V gj1 = -(conjv(sn) * gj);
        S->g[j + 1] = gj1;
        S->g[j] = scale(gj, c);
        S->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
        const int its = S->its + 1;
        S->its = its;
        const double gres = absv(gj1), beta = S->beta, cyc_target = S->cyc_target;
        const double last_res = gres / S->zbnorm;
        S->last_res = last_res;
        const bool inner_done = cyc_target > 0.0 ? gres <= cyc_target * beta : last_res <= S->inner * S->tol;
        const bool end = inner_done || gres <= S->rtol_eff * beta || hn == 0.0 || its >= S->maxit || j + 1 >= S->R;
        s_end = end ? 1 : 0;
        s_k = j + 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += RT) S->H[(int64_t)j * KMAX + i] = sHj[i];
    if (s_end) {
        // the cycle ends: y = H(0:k, 0:k)^{-1} g(0:k) for the next block's x update
        const int k = s_k;
        __shared__ V sH[KMAX * KMAX];
        for (int q = threadIdx.x; q < k * k; q += RT) {
            const int col = q / k, row = q % k;
            sH[col * KMAX + row] = col == j ? sHj[row] : S->H[(int64_t)col * KMAX + row];
        }
        for (int i = threadIdx.x; i < k; i += RT) sg[i] = S->g[i];
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = k - 1; i >= 0; --i) {
                V yv = sg[i];
                for (int l = i + 1; l < k; ++l) yv = yv - sH[l * KMAX + i] * sy[l];
                sy[i] = cdiv(yv, sH[i * KMAX + i]);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += RT) S->y[i] = sy[i];
        if (threadIdx.x == 0) {
            S->jend = k;
            S->have_cycle = 1;
            S->mode = GM_RESTART;
        }
    } else if (threadIdx.x == 0) {
        S->j = j + 1;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        hstat->done = S->done;
        hstat->its = S->its;
        __threadfence_system();
    }
}

// Grid barrier of a cooperative launch (every block resident): thread 0
// publishes the block's writes and counts in, then waits, bounded, until
// `target` blocks have; false if the wait gave up.
__device__ bool gm_grid_sync(unsigned* ctr, unsigned target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        int ok = 1;
        uint64_t t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            __nanosleep(64);
            uint64_t t1;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
            if (t1 - t0 > 2000000000ull) {
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}


// One cooperative launch per GMRES block for what follows the apply.
// RESTART: beta = ||V_0||, g = beta e_1.  STEP: h1 = V^H w (grid barrier),
// w -= V h1 and h2 = V^H w (grid barrier), w -= V h2, ||w||, the Hessenberg
// column and the cycle's tests.  Every path leaves the status word for the
// host.  All blocks read the solver state's mode words before any block can
// change them (the last block of each reduction is the only writer).
template <typename V>
__global__ void __launch_bounds__(RT, 4) gm_arnoldi_kernel(GmDev<V>* S, V* __restrict__ Vb, int64_t ldv, int n,
                                                        V* __restrict__ partial, double* __restrict__ dpartial,
                                                        GmStatus* hstat) {
    const int done = S->done, bmode = S->bmode;
    if (done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            hstat->done = done;
            hstat->its = S->its;
            __threadfence_system();
        }
        return;
    }
    if (bmode == GM_RESTART) {
        double acc = 0.0;
        for (int64_t row = (int64_t)blockIdx.x * RT + threadIdx.x; row < n; row += (int64_t)gridDim.x * RT)
            acc += norm2(Vb[row]);
        const double bs = block_sum(acc);
        if (threadIdx.x == 0) dpartial[blockIdx.x] = bs;
        if (!last_block(S->counter, gridDim.x)) return;
        const double ss = block_sum_partials(dpartial, gridDim.x);
        const double beta = sqrt(ss);
        for (int i = threadIdx.x; i < KMAX; i += RT) S->g[i] = i == 0 ? from_real<V>(beta) : zero<V>();
        if (threadIdx.x == 0) {
            bool ok = true;
            if (S->zbnorm < 0.0) {
                S->zbnorm = beta;
                if (beta == 0.0) {                   // P^{-1} b vanished
                    S->done = 3;
                    S->skip = 1;
                    ok = false;
                }
            }
            if (ok) {
                S->beta = beta;
                S->scale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
                S->j = 0;
                S->mode = GM_STEP;
            }
            __threadfence();
            hstat->done = S->done;
            hstat->its = S->its;
            __threadfence_system();
        }
        return;
    }
    unsigned* bar = S->counter + GM_BARRIER;
    const int j = S->j;
    __shared__ double scl[KMAX];
    __shared__ V h1[KMAX], h2[KMAX], cw[KMAX];
    if (threadIdx.x <= j) scl[threadIdx.x] = S->scale[threadIdx.x];
    __syncthreads();
    // h1 = V^H w: partials, grid barrier, every block adds them
    gm_pass<V, false>(Vb, ldv, n, j, nullptr, partial);
    bool ok = gm_grid_sync(bar, gridDim.x);
    if (ok) {
        gm_sum_partials(partial, j, scl, h1);
        if (threadIdx.x <= j) cw[threadIdx.x] = -scale(h1[threadIdx.x], scl[threadIdx.x]);
        __syncthreads();
        // w -= V h1, h2 = V^H w (the second pass's partials in their own buffer:
        // other blocks may still be adding the first pass's)
        gm_pass<V, true>(Vb, ldv, n, j, cw, partial + (int64_t)RB * KMAX);
        ok = gm_grid_sync(bar, 2 * gridDim.x);
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            S->done = 4;
            hstat->done = 4;
            __threadfence_system();
        }
        return;
    }
    gm_sum_partials(partial + (int64_t)RB * KMAX, j, scl, h2);
    gm_axnorm_step<V>(S, Vb, ldv, n, dpartial, hstat, h1, h2, scl, j);
}

// Pinned status words of this thread's solves (two blocks in flight), mapped
// into the device address space; kept for the thread's lifetime.
GmStatus* pinned_status() {
    thread_local GmStatus* p = nullptr;
    if (!p) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, 2 * sizeof(GmStatus), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p = static_cast<GmStatus*>(h);
    }
    return p;
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
    V* t = (V*)carve(sizeof(V) * n);
    V* r = (V*)carve(sizeof(V) * n);
    V* part = (V*)carve(sizeof(V) * 2 * RB * KMAX);   // the two Gram-Schmidt passes' partials
    double* dpart = (double*)carve(sizeof(double) * RB);
    GmDev<V>* S = (GmDev<V>*)carve(sizeof(GmDev<V>));
    void* awork = carve(apply_work_bytes(F));
    GmStatus* hst = pinned_status();
    if (!hst) return set_error(NDHSS_ERR_OOM, "ndhss_gmres: pinned status words");
    hst[0] = hst[1] = GmStatus{0, 0, 0, 0};
    const int eb = std::min((n + 255) / 256, 4 * 152);
    const unsigned sblocks = (unsigned)(((int64_t)n * SP_TPR + 255) / 256);
    // the Arnoldi kernel's grid: every block resident at once (its grid barriers)
    int agrid = 0;
    {
        int dev = 0, sms = 0, per_sm = 0;
        NDHSS_CUDA_TRY(cudaGetDevice(&dev));
        NDHSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NDHSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gm_arnoldi_kernel<V>, RT, 0));
        agrid = std::min(RB, per_sm * sms);
        if (agrid < 1) return set_error(NDHSS_ERR_CUDA, "ndhss_gmres: the Arnoldi kernel cannot be resident");
    }
    gm_init_kernel<V><<<1, 1, 0, st>>>(S, R, o.maxit, o.tol, o.inner, o.cycle_rtol);
    NDHSS_LAUNCH_CHECK("gm_init_kernel");
    NDHSS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(V) * n, st));

    // optional CUDA-event timing of every apply and sparse product; events
    // come from a per-thread pool that lives as long as the thread
    thread_local std::vector<cudaEvent_t> pool;
    size_t pool_next = 0;
    auto ev = [&]() -> cudaEvent_t {
        if (pool_next == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[pool_next++];
    };
    std::vector<cudaEvent_t> evs;             // per block: SpMV start, end, apply start, end
    cudaEvent_t blk_done[2] = {nullptr, nullptr};
    if (cudaEventCreateWithFlags(&blk_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&blk_done[1], cudaEventDisableTiming) != cudaSuccess)
        return set_error(NDHSS_ERR_CUDA, "ndhss_gmres: event creation failed");
    ndhss_status rc = NDHSS_OK;
    const int max_blocks = std::min(GM_MAX_BLOCKS, 2 * o.maxit + 4);
    int nblk = 0;
    for (int blk = 0; blk < max_blocks && rc == NDHSS_OK; ++blk) {
        gm_begin_kernel<V><<<eb, 256, 0, st>>>(S, x, Vb, ldv, t, r, n, blk);
        note_launches(1);
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
        if (o.timing) { e0 = ev(); e1 = ev(); e2 = ev(); e3 = ev(); }
        if (e0) cudaEventRecord(e0, st);
        gm_spmv_kernel<V><<<sblocks, 256, 0, st>>>(n, rowptr, col, vals, S);
        note_launches(1);
        if (e1) cudaEventRecord(e1, st);
        gm_resid_kernel<V><<<RB, RT, 0, st>>>(S, b, t, r, n, dpart, blk);
        note_launches(1);
        if (e2) cudaEventRecord(e2, st);
        rc = apply_device(F, 1, nullptr, n, nullptr, n, awork, st, &S->ind);
        if (rc != NDHSS_OK) break;
        if (e3) cudaEventRecord(e3, st);
        {
            GmStatus* hs_blk = hst + (blk & 1);
            void* args[] = {(void*)&S, (void*)&Vb, (void*)&ldv, (void*)&n, (void*)&part, (void*)&dpart, (void*)&hs_blk};
            cudaError_t ce = cudaLaunchCooperativeKernel((const void*)gm_arnoldi_kernel<V>, dim3(agrid), dim3(RT), args, 0, st);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                rc = set_error(NDHSS_ERR_CUDA, "ndhss_gmres: cooperative launch failed: %s", cudaGetErrorString(ce));
                break;
            }
        }
        note_launches(1);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_gmres: launch failed: %s", cudaGetErrorString(le));
            break;
        }
        if (o.timing) evs.insert(evs.end(), {e0, e1, e2, e3});
        cudaEventRecord(blk_done[blk & 1], st);
        nblk = blk + 1;
        if (blk >= 1) {
            // the previous block's status while this one runs
            if (cudaEventSynchronize(blk_done[(blk - 1) & 1]) != cudaSuccess) {
                rc = set_error(NDHSS_ERR_CUDA, "ndhss_gmres: event synchronisation failed");
                break;
            }
            if (((volatile GmStatus*)hst)[(blk - 1) & 1].done) break;
        }
    }
    GmDev<V> hs;
    if (rc == NDHSS_OK) {
        if (cudaMemcpyAsync(&hs, S, sizeof(GmDev<V>), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_gmres: reading the solver state failed");
    }
    cudaEventDestroy(blk_done[0]);
    cudaEventDestroy(blk_done[1]);
    if (rc != NDHSS_OK) return rc;
    if (hs.done == 3) return set_error(NDHSS_ERR_INTERNAL, "ndhss_gmres: P^{-1} b vanished");
    if (hs.done == 4) return set_error(NDHSS_ERR_TIMEOUT, "ndhss_gmres: a grid barrier of the Arnoldi step gave up");
    ndhss_gmres_stats Sx{};
    Sx.converged = hs.done == 1;
    Sx.iters = hs.its;
    Sx.cycles = hs.cycles;
    Sx.true_relres = hs.relres;
    Sx.precond_relres = hs.last_res;
    for (int blk = 0; blk < nblk; ++blk) {
        Sx.nspmv += (hs.ran[blk] & 1) ? 1 : 0;
        Sx.napply += (hs.ran[blk] & 2) ? 1 : 0;
    }
    if (o.timing) {
        float ms;
        for (int blk = 0; blk < nblk && 4 * blk + 3 < (int)evs.size(); ++blk) {
            if ((hs.ran[blk] & 1) && cudaEventElapsedTime(&ms, evs[4 * blk], evs[4 * blk + 1]) == cudaSuccess)
                Sx.spmv_ms += ms;
            if ((hs.ran[blk] & 2) && cudaEventElapsedTime(&ms, evs[4 * blk + 2], evs[4 * blk + 3]) == cudaSuccess)
                Sx.apply_ms += ms;
        }
    }
    if (stats) *stats = Sx;
    return NDHSS_OK;
}

size_t gmres_work_bytes(const FactorData& F, int R, size_t vsz) {
    const int64_t ldv = ((int64_t)F.n + 31) / 32 * 32;
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
    add(vsz * ldv * (R + 1));
    add(vsz * F.n);
    add(vsz * F.n);
    add(vsz * 2 * RB * KMAX);
    add(8 * RB);
    add(std::max(sizeof(GmDev<double>), sizeof(GmDev<c128>)));
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
        if (o.restart < 1 || o.restart > KMAX - 1 || o.maxit < 0 || o.maxit > GM_MAX_IT || !(o.tol >= 0) ||
            !(o.inner > 0 && o.inner <= 1) ||
            o.conj_transpose < 0 || o.conj_transpose > 1)
            return set_error(NDHSS_ERR_INVALID_ARG,
                             "ndhss_gmres: need 1 <= restart <= %d, 0 <= maxit <= %d, tol >= 0, 0 < inner <= 1, "
                             "conj_transpose 0 or 1", KMAX - 1, GM_MAX_IT);
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
