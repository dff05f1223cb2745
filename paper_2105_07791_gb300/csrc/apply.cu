// y = P^{-1} x by Algorithm 3.1 on the device.
//
//   gather/cast   y = x(perm) converted to the factor precision
//   up-sweep      levels bottom-up:  y(B^s) += L^s y(I^s)          (L = -BL P)
//   diagonal      all nodes:         z(I^s) = A_ii^{-1} y(I^s)     (independent across nodes)
//   down-sweep    levels top-down:   z(I^s) += R^s z(B^s)
//   scatter/cast  out(perm) = z converted back to float64, by whichever task
//                 writes a row's final value
//
// The apply is a queue of row tasks, built once per factorization in
// topological order.  Dense nodes with m_i <= DIAG_COLS take one pass over
// the first m_i columns of the eliminated front, [A_ii^{-1} P^T ; -L P^T]:
// the diagonal solve and the up-sweep product share the input y(I^s) and
// the same dependencies, so one 64-row task gives z rows or y(B^s) updates.
// A_ii^{-1} of larger nodes is split into DIAG_COLS-column chunks whose
// partial products a second task sums (a 1539-column row is otherwise one
// long dependent chain on the critical path).  Low-rank nodes use dot tasks
// over LR_CHUNK-row chunks and 64-row axpy tasks.  Every task first issues
// the loads that do not depend on other tasks (its first group of matrix
// entries, the gather indices of its vector), then waits, then stages the
// vector and finishes: the wait overlaps the matrix traffic.
//
// The bottom levels [Ls, depth] (every node dense, small fronts) are not
// split into per-node tasks: each subtree rooted on level Ls is one up task
// and one down task.  The subtree's boxes hold its interior rows as one
// contiguous range of the new numbering and every row its nodes touch lies
// in that range or in B of the subtree root, so the task keeps that vector
// segment in shared memory and takes the subtree's levels in turn, separated
// by CTA barriers instead of cross-SM dependency hops: per level, every row
// of every node of the level is one dot product (threads over rows, several
// threads per row with a fixed-order reduction when rows are few).  The up
// task writes z(I) of its nodes and adds its contributions to y(B^root); the
// down task, once the root's parent is final, finishes z(I) of the subtree
// and writes the output rows.
//
// Two schedules run the same queue:
// * dataflow (default): ONE persistent launch.  A CTA takes the next ticket
//   with one atomic (prefetched while the previous task runs), waits until
//   the nodes its task depends on have signalled their counters, runs the
//   task and signals.  The boxes of one level own disjoint unknowns (B^s is
//   part of box s), so a node's up-sweep and diagonal step need only its two
//   children finished, and its down-sweep its parent's final rows.  A CTA
//   only ever waits for tickets handed out before its own, which running
//   CTAs hold, so the queue cannot deadlock for any grid size.  Every wait
//   is bounded: after APPLY_WAIT_NS the CTA raises the sticky error word of
//   the factorization and every CTA leaves (NDHSS_ERR_TIMEOUT at the next
//   synchronising call).
// * levels: the queue cut into its dependency groups (one tree level and
//   phase each), one launch per group; selected with
//   NDHSS_APPLY_SCHEDULE=levels and kept as the bit-exact cross-check.
#include <algorithm>
#include <atomic>
#include <thread>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "driver.h"
#include "factor.cuh"

namespace ndhss {
namespace {

constexpr int AT = 256;
constexpr int AW = AT / 32;
constexpr int GATHER_CHUNK = 8 * AT;     // rows per gather task
constexpr int DIAG_COLS = 256;    // column chunk of A_ii^{-1} per task (and fused-pass limit)
constexpr int SUM_ROWS = AT;      // rows per partial-sum task
constexpr int ROOT_DIAG_COLS = 128; // the same for the top level's nodes
constexpr uint64_t APPLY_WAIT_NS = 2000000000ull;   // 2 s

__device__ __forceinline__ int nf(const int32_t* node, int s, int f) { return node[s * NODE_NF + f]; }

__device__ __forceinline__ double shfl_xor_t(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_xor_t(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <typename R>
__device__ __forceinline__ Cx<R> shfl_xor_t(Cx<R> v, int o) {
    return {__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}

// Loads and stores of the work vectors go through L2 (ld/st.cg): other CTAs
// of the same launch write them, so no copy may come from a stale L1 line.
__device__ __forceinline__ double ldw(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldw(const float* p) { return __ldcg(p); }
__device__ __forceinline__ c128 ldw(const c128* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ c64 ldw(const c64* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ void stw(double* p, double v) { __stcg(p, v); }
__device__ __forceinline__ void stw(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void stw(c128* p, c128 v) { __stcg(reinterpret_cast<double2*>(p), make_double2(v.x, v.y)); }
__device__ __forceinline__ void stw(c64* p, c64 v) { __stcg(reinterpret_cast<float2*>(p), make_float2(v.x, v.y)); }

// Task kinds of the queue.
enum : int {
    TK_GATHER = 0,
    TK_UPDIAG,    // dense, m_i <= DIAG_COLS: 64 rows of [A_ii^{-1}; -L] (z rows / y(B) updates)
    TK_UP,        // dense, larger m_i: 64 rows of -L
    TK_UPDOT,     // low-rank: partial X(chunk, :)^T y(I)(chunk)
    TK_UPAXPY,    // low-rank: 64 rows of y(B) += RJt t
    TK_UPNOP,     // completes a node with no up-sweep work
    TK_DPART,     // 64 rows x DIAG_COLS columns of A_ii^{-1} y(I), partial
    TK_DSUM,      // 256 rows: z(I) = sum of the partials
    TK_DN,        // dense: 64 rows of z(I) += R z(B)
    TK_DNDOT,     // low-rank: partial RJt(chunk, :)^T z(B)(chunk)
    TK_DNAXPY,    // low-rank: 64 rows of z(I) += X t
    TK_FINNOP,    // completes a node without interior rows
    TK_UPW,       // up to 8 tiny dense nodes of a level, one per warp: [A_ii^{-1}; -L] y(I)
    TK_DNW,       // the same nodes coming down: z(I) += R z(B), final rows
    TK_HUP,       // ULV solve of HSS(A_ii), one HSS node going up (entry node = ULV record)
    TK_HROOT,     // the root block of a ULV front
    TK_HDN,       // one HSS node coming down (leaves write z(I) rows)
    TK_SUBUP,     // a bottom subtree going up (diagonal steps and y(B) updates of all its nodes)
    TK_SUBDN      // the same subtree coming down (z(I) += R z(B), output rows)
};
// Subtree tasks: limits of a subtree (nodes, levels, nodes per level) and
// of its shared-memory vector segment (interior rows + B of the root) and
// per-level staged inputs.
constexpr int SUB_NODES = 256, SUB_LV = 16, SUB_LVN = 64, SUB_V = 1536, SUB_XIN = 1024;
constexpr int SUB_MIN_ROOTS = 128;   // fewest subtrees worth the restructuring (GPU fill)
// Tiny dense nodes (the bottom levels) are handled a warp per node, eight per
// task: their blocks are a few KB, so one 64-row task per node would be all
// latency.  Limits of a warp node (rows of the fused pass, interior rows,
// boundary columns) and its per-warp shared-memory region.
constexpr int WN_M = 96, WN_MI = 64, WREG = 128;
// per-node counters (NCNT arrays of nnodes each) and what signals them
enum : int { CN_UP = 0, CN_DOT, CN_DIAG, CN_DDOT, CN_FIN, CN_DPART, NCNT };
constexpr int TK_SHIFT = 25;       // entry word 0 = kind << TK_SHIFT | node (5 bits of kind)
constexpr int TK_FINAL = 1 << 30;  // entry word 0 flag: the task writes final rows (scatter)
constexpr int CTL_WORDS = 4;       // ticket, gather count, abort, pad
// ints per queue entry: flags | kind | node, a, b, m_i, m_b, i_off, b_off, k,
// base (64-bit: front offset, or low-rank storage address), aux (64-bit:
// partial-product slot); everything a task reads before its first matrix load
constexpr int QW = 12;

// Read-only views of the factor for one apply (per-task sizes, offsets and
// pointers travel in the queue entries).
template <typename T>
struct ApplyCtx {
    const int32_t* node;
    const int32_t* blist;
    const int32_t* sigma;
    const int32_t* perm;
    const T* front;
    const int32_t* wdesc;     // warp nodes, 8 ints each: node, m_i, m_b, i_off, b_off, front offset (lo, hi), 0
    const struct UlvDev* ulv; // ULV records (HSS nodes of the ULV fronts)
    const int32_t* ulv_ord;   // HSS order of each ULV front's I^s
    const int64_t* foff;      // front offset of every node
    const int32_t* sublist;   // per subtree: nl, level offsets [nl + 1], nodes (deepest level first)
};

// One HSS node of a ULV front on the device: sizes, links, its front, the
// apply scratch slots of its vectors and the addresses of its solve data.
struct UlvDev {
    int32_t s, lo, hi, m, k, ne, kt, ka, kb, parent, c1, c2, leaf, root, i_off, pad;
    int64_t ord_off, o_y1, o_rh, o_g, o_x2;
    uint64_t Mup, W, Mm, E, Dinv;
};

// Registers a task fills before its wait: the first group of matrix entries
// and the gather / scatter index of its own output row.
template <typename T>
struct Pre {
    T v[8];
    int gi, pi;
};

// ---- L2 prefetch of read-only factor data ---------------------------------
// One prefetch request per 128-byte line of [p, p + bytes); each request
// names an address inside the range (the first byte, then line starts), so
// none leaves the buffer.  Requests q0, q0 + step, ... of the range's lines.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ int range_lines(const void* p, int64_t bytes) {
    if (bytes <= 0) return 0;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    return (int)(((a + bytes - 1) >> 7) - (a >> 7) + 1);
}
__device__ __forceinline__ void prefetch_line(const void* p, int l) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    prefetch_l2(l == 0 ? p : reinterpret_cast<const void*>(((a >> 7) + l) << 7));
}

// ---- 64-row GEMV ----------------------------------------------------------
// Rows [r0, r0 + 64) of (block A, column-major, leading dimension lda) times
// the vector xs (shared memory): 8 warps take every 8th column, each lane
// owns rows r0 + lane and r0 + lane + 32, and four columns are in flight per
// step, so a thread keeps eight independent loads outstanding and a warp
// reads each column segment as one contiguous 64-row access.  The first
// group of four columns is loaded by gemv_pre before the task's wait.  The
// eight warp partial sums are added in shared memory; lanes of warp 0 and 1
// return the results for rows r0 + tid (tid < 64).
template <typename T>
__device__ __forceinline__ void gemv_pre(const T* __restrict__ A, int64_t lda, int rows, int cols, int r0, T (&pre)[8]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ra = r0 + lane, rb = r0 + lane + 32;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = warp + u * AW;
        const T* col = A + (int64_t)c * lda;
        pre[u] = (c < cols && ra < rows) ? col[ra] : zero<T>();
        pre[4 + u] = (c < cols && rb < rows) ? col[rb] : zero<T>();
    }
    // the rest of the 64-row segment into L2 while the task waits
    const int nr = min(APPLY_ROWS, rows - r0);
    if (nr > 0 && cols > 4 * AW) {
        constexpr int LPC = (APPLY_ROWS * (int)sizeof(T) + 127) / 128 + 1;   // lines a segment can touch
        const int tot = (cols - 4 * AW) * LPC;
        for (int q = threadIdx.x; q < tot; q += AT) {
            const T* seg = A + (int64_t)(4 * AW + q / LPC) * lda + r0;
            const int l = q % LPC;
            if (l < range_lines(seg, (int64_t)nr * sizeof(T))) prefetch_line(seg, l);
        }
    }
}

template <typename T>
__device__ __forceinline__ T gemv_rows64(const T* __restrict__ A, int64_t lda, int rows, int cols, int r0,
                                         const T* __restrict__ xs, T (*red)[APPLY_ROWS], const T (&pre)[8]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ra = r0 + lane, rb = r0 + lane + 32;
    const bool va = ra < rows, vb = rb < rows;
    T acc0 = zero<T>(), acc1 = zero<T>();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = warp + u * AW;
        if (c < cols) {
            const T x = xs[c];
            acc0 = fmac(pre[u], x, acc0);
            acc1 = fmac(pre[4 + u], x, acc1);
        }
    }
    int c = warp + 4 * AW;
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
    if (c < cols) {                  // the ragged last columns: one round of predicated loads
        T a[3], b[3], x[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int cu = c + u * AW;
            const bool ok = cu < cols;
            const T* col = A + (int64_t)(ok ? cu : c) * lda;
            a[u] = (ok && va) ? col[ra] : zero<T>();
            b[u] = (ok && vb) ? col[rb] : zero<T>();
            x[u] = ok ? xs[cu] : zero<T>();
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            acc0 = fmac(a[u], x[u], acc0);
            acc1 = fmac(b[u], x[u], acc1);
        }
    }
    red[warp][lane] = acc0;
    red[warp][lane + 32] = acc1;
    __syncthreads();
    T sum = zero<T>();
    if (threadIdx.x < APPLY_ROWS)
        for (int w = 0; w < AW; ++w) sum += red[w][threadIdx.x];
    return sum;
}

// ---- one task: pre-phase (independent loads) and run-phase ----------------

struct Entry {
    int kind, s, a, b;
    bool fin;
    int m_i, m_b, i_off, b_off, k;
    int64_t base, aux;
};
__device__ __forceinline__ Entry decode(const int32_t* q, int64_t t) {
    const int4* p = reinterpret_cast<const int4*>(q + QW * t);
    const int4 v0 = p[0], v1 = p[1], v2 = p[2];
    Entry e;
    e.fin = (v0.x & TK_FINAL) != 0;
    e.kind = (v0.x >> TK_SHIFT) & 31;
    e.s = v0.x & ((1 << TK_SHIFT) - 1);
    e.a = v0.y;
    e.b = v0.z;
    e.m_i = v0.w;
    e.m_b = v1.x;
    e.i_off = v1.y;
    e.b_off = v1.z;
    e.k = v1.w;
    e.base = (int64_t)(((uint64_t)(uint32_t)v2.y << 32) | (uint32_t)v2.x);
    e.aux = (int64_t)(((uint64_t)(uint32_t)v2.w << 32) | (uint32_t)v2.z);
    return e;
}

// ---- warp-node tasks (TK_UPW / TK_DNW) -------------------------------------
// Warp w < e.a takes node e.base + w of the warp-node table; wd[w] receives
// its descriptor, idx + w * WREG its gather indices, vec + w * WREG its
// staged vector.
__device__ __forceinline__ void taskw_pre(const int32_t* __restrict__ wdesc, const int32_t* __restrict__ sigma,
                                          const int32_t* __restrict__ blist, const Entry& e, int* idx, int (*wd)[8]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w >= e.a) return;
    if (lane < 8) wd[w][lane] = wdesc[(e.base + w) * 8 + lane];
    __syncwarp();
    const int m_i = wd[w][1], m_b = wd[w][2], i_off = wd[w][3], b_off = wd[w][4];
    int* iw = idx + w * WREG;
    if (e.kind == TK_UPW)
        for (int c = lane; c < m_i; c += 32) iw[c] = sigma[i_off + c];
    else
        for (int j = lane; j < m_b; j += 32) iw[j] = blist[b_off + j];
}

template <typename T, typename V>
__device__ __forceinline__ void taskw_run(const ApplyCtx<T>& C, const Entry& e, const int* idx, T* vec,
                                          const int (*wd)[8], V* __restrict__ out, T* y, T* z) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w >= e.a) return;
    const int m_i = wd[w][1], m_b = wd[w][2], i_off = wd[w][3], b_off = wd[w][4];
    const int64_t foff = (int64_t)(((uint64_t)(uint32_t)wd[w][6] << 32) | (uint32_t)wd[w][5]);
    const int m = m_i + m_b;
    const T* F = C.front + foff;
    const int* iw = idx + w * WREG;
    T* vw = vec + w * WREG;
    constexpr int WU = sizeof(T) <= 8 ? 8 : 4;     // columns in flight per lane
    if (e.kind == TK_UPW) {
        // rows r of the first m_i columns, lanes over rows, WU columns in flight
        for (int c = lane; c < m_i; c += 32) vw[c] = ldw(y + i_off + iw[c]);
        __syncwarp();
        for (int r0 = 0; r0 < m; r0 += 32) {
            const int r = r0 + lane;
            const int g = (r >= m_i && r < m) ? C.blist[b_off + r - m_i] : -1;
            T acc = zero<T>();
            for (int c0 = 0; c0 < m_i; c0 += WU) {
                T a[WU];
#pragma unroll
                for (int u = 0; u < WU; ++u) a[u] = (r < m && c0 + u < m_i) ? F[(int64_t)(c0 + u) * m + r] : zero<T>();
#pragma unroll
                for (int u = 0; u < WU; ++u)
                    if (c0 + u < m_i) acc = fmac(a[u], vw[c0 + u], acc);
            }
            if (r < m_i) stw(z + i_off + r, acc);
            else if (r < m) stw(y + g, ldw(y + g) - acc);
        }
    } else {
        // interior rows of R (m_i x m_b at column m_i), lanes over rows
        for (int j = lane; j < m_b; j += 32) vw[j] = ldw(z + iw[j]);
        __syncwarp();
        const T* R = F + (int64_t)m_i * m;
        for (int r0 = 0; r0 < m_i; r0 += 32) {
            const int r = r0 + lane;
            const int pi = r < m_i ? C.perm[i_off + r] : 0;
            T acc = zero<T>();
            for (int c0 = 0; c0 < m_b; c0 += WU) {
                T a[WU];
#pragma unroll
                for (int u = 0; u < WU; ++u) a[u] = (r < m_i && c0 + u < m_b) ? R[(int64_t)(c0 + u) * m + r] : zero<T>();
#pragma unroll
                for (int u = 0; u < WU; ++u)
                    if (c0 + u < m_b) acc = fmac(a[u], vw[c0 + u], acc);
            }
            if (r < m_i) {
                const T v = ldw(z + i_off + r) + acc;
                stw(z + i_off + r, v);
                out[pi] = to_val(v);
            }
        }
    }
}

// ---- ULV solve tasks (TK_HUP / TK_HROOT / TK_HDN) --------------------------
// Every step is a matrix-vector product with precomputed ULV data (ulv.cu):
// up: r (the front's rows of y in HSS order at a leaf; the children's
// reduced right-hand sides corrected by their couplings G at an inner node)
// -> Mup r = (y1, r^, G); root: x = Dinv r; down: x~ = W [y1; x2], split
// among the children or (leaf) written to z(I^s) in the front's order.
template <typename T, typename Fn>
__device__ __forceinline__ void ulv_gemv(const T* A, int rows, int cols, const T* xs, T (*red)[APPLY_ROWS], Fn&& emit) {
    for (int r0 = 0; r0 < rows; r0 += APPLY_ROWS) {
        T pre[8];
        gemv_pre(A, rows, rows, cols, r0, pre);
        const T sum = gemv_rows64(A, rows, rows, cols, r0, xs, red, pre);
        if (threadIdx.x < APPLY_ROWS && r0 + (int)threadIdx.x < rows) emit(r0 + (int)threadIdx.x, sum);
        __syncthreads();
    }
}

template <typename T, typename V>
__device__ __forceinline__ void ulv_task(const ApplyCtx<T>& C, const Entry& e, const int* idx, T* vec,
                                         T (*red)[APPLY_ROWS], V* __restrict__ out, const T* y, T* z, T* us) {
    const UlvDev R = C.ulv[e.s];
    const int tid = threadIdx.x;
    const int m = R.m;
    if (e.kind == TK_HUP || e.kind == TK_HROOT) {
        T* g = vec + m;
        int ka = 0, kb = 0;
        if (R.leaf) {
            for (int j = tid; j < m; j += AT) vec[j] = ldw(y + R.i_off + idx[j]);
            __syncthreads();
        } else {
            const UlvDev A = C.ulv[R.c1], B = C.ulv[R.c2];
            ka = R.ka;
            kb = R.kb;
            for (int c = tid; c < ka + kb; c += AT) g[c] = c < ka ? ldw(us + A.o_g + c) : ldw(us + B.o_g + c - ka);
            __syncthreads();
            // r = [r^_a; r^_b] - Mm [G_a; G_b]
            const T* Mm = reinterpret_cast<const T*>(R.Mm);
            ulv_gemv(Mm, m, ka + kb, g, red, [&](int j, T v) {
                const T rh = j < A.kt ? ldw(us + A.o_rh + j) : ldw(us + B.o_rh + j - A.kt);
                vec[j] = rh - v;
            });
        }
        if (e.kind == TK_HROOT) {
            const T* Di = reinterpret_cast<const T*>(R.Dinv);
            if (R.leaf) {
                ulv_gemv(Di, m, m, vec, red, [&](int j, T v) {
                    const int row = R.i_off + idx[j];
                    stw(z + row, v);
                    if (e.fin) out[C.perm[row]] = to_val(v);
                });
            } else {
                const UlvDev A = C.ulv[R.c1], B = C.ulv[R.c2];
                ulv_gemv(Di, m, m, vec, red, [&](int j, T v) {
                    if (j < A.kt) stw(us + A.o_x2 + j, v);
                    else stw(us + B.o_x2 + j - A.kt, v);
                });
            }
        } else {
            const T* Mup = reinterpret_cast<const T*>(R.Mup);
            const int ne = R.ne, kt = R.kt, k = R.k;
            const T* E = reinterpret_cast<const T*>(R.E);
            ulv_gemv(Mup, m + k, m, vec, red, [&](int j, T v) {
                if (j < ne) {
                    stw(us + R.o_y1 + j, v);
                } else if (j < ne + kt) {
                    stw(us + R.o_rh + j - ne, v);
                } else {
                    const int a = j - ne - kt;
                    if (!R.leaf)       // G += E^T [G_a; G_b]
                        for (int c = 0; c < ka + kb; ++c) v = fmac(E[(int64_t)a * (ka + kb) + c], g[c], v);
                    stw(us + R.o_g + a, v);
                }
            });
        }
        return;
    }
    // TK_HDN: x~ = W [y1; x2]
    for (int j = tid; j < m; j += AT) vec[j] = j < R.ne ? ldw(us + R.o_y1 + j) : ldw(us + R.o_x2 + j - R.ne);
    __syncthreads();
    const T* W = reinterpret_cast<const T*>(R.W);
    if (R.leaf) {
        ulv_gemv(W, m, m, vec, red, [&](int j, T v) {
            const int row = R.i_off + idx[j];
            stw(z + row, v);
            if (e.fin) out[C.perm[row]] = to_val(v);
        });
    } else {
        const UlvDev A = C.ulv[R.c1], B = C.ulv[R.c2];
        ulv_gemv(W, m, m, vec, red, [&](int j, T v) {
            if (j < A.kt) stw(us + A.o_x2 + j, v);
            else stw(us + B.o_x2 + j - A.kt, v);
        });
    }
}

// ---- subtree tasks (TK_SUBUP / TK_SUBDN) ----------------------------------
// Entry: s = subtree root, a = first interior row lo, b = interior rows nI,
// m_b / b_off = the root's, aux = offset of the subtree's table, k = its
// length.  The table (built on the host, copied to shared memory at the
// start of the task, so no level waits on a dependent global load):
//   header  nl, nodes
//   level   nl records: count, first node, rows up, rows down, inputs up,
//           inputs down (deepest level first)
//   node    records: m_i, m_b, front offset (lo, hi), rows and inputs before
//           it in its level (up: rows, inputs; down: rows, inputs), interior
//           slot i_off - lo, B rows before it in its level
//   slots   the vector slot of every staged input, level by level: up, y(I)
//           in the order of A_ii^{-1}'s columns; down, z(B) (also the slot
//           each up-sweep B row adds into)
// vec holds [z or y rows lo .. lo + nI) | B^root slots | staged inputs | partials].
constexpr int SUB_HDR = 2, SUB_LREC = 6, SUB_NREC = 10;

struct Sched;
// bounded wait of one thread for every gather task (defined with the queue)
__device__ bool wait_gather(const Sched* S);

template <typename T, typename V>
__device__ void subtree_task(const ApplyCtx<T>& C, const Entry& e, int* idx, T* vec, const V* __restrict__ x,
                             V* __restrict__ out, T* y, T* z, const Sched* Sp) {
    const bool up = e.kind == TK_SUBUP;
    const int tid = threadIdx.x;
    const int lo = e.a, nI = e.b, mbr = e.m_b;
    const int tlen = e.k;
    // the set-up loads go out in batches of four, so a thread waits for
    // memory once per batch
    {
        const int32_t* __restrict__ g = C.sublist + e.aux;
        for (int i0 = 0; i0 < tlen; i0 += 4 * AT) {
            int v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + tid + u * AT;
                v[u] = i < tlen ? g[i] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + tid + u * AT < tlen) idx[i0 + tid + u * AT] = v[u];
        }
    }
    for (int i0 = 0; i0 < nI; i0 += 4 * AT) {
        int pi[4];
        T v[4];
        if (up) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + tid + u * AT;
                pi[u] = i < nI ? C.perm[lo + i] : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = pi[u] >= 0 ? from_val<T>(x[pi[u]]) : zero<T>();
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + tid + u * AT;
                v[u] = i < nI ? ldw(z + lo + i) : zero<T>();
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + tid + u * AT < nI) vec[i0 + tid + u * AT] = v[u];
    }
    for (int j = tid; j < mbr; j += AT) vec[nI + j] = up ? zero<T>() : ldw(z + C.blist[e.b_off + j]);
    __syncthreads();
    const int nl = idx[0], nn = idx[1];
    const int* lrec = idx + SUB_HDR;
    const int* nrec = lrec + SUB_LREC * nl;
    const int* src_up = nrec + SUB_NREC * nn;
    int n_src_up = 0, n_src_dn = 0;
    for (int h = 0; h < nl; ++h) {
        n_src_up += lrec[SUB_LREC * h + 4];
        n_src_dn += lrec[SUB_LREC * h + 5];
    }
    const int* src_dn = src_up + n_src_up;
    const int* dst_up = src_dn;           // an up-sweep B row adds into the slot its down input reads
    // the matrix data of level hh (in sweep order) into L2: up, [A_ii^{-1}; -L]
    // of each node (m x m_i, contiguous); down, the m_i rows of each column of R
    auto prefetch_level = [&](int hh) {
        if (hh >= nl) return;
        const int* L = lrec + SUB_LREC * (up ? hh : nl - 1 - hh);
        for (int j = 0; j < L[0]; ++j) {
            const int* nd = nrec + SUB_NREC * (L[1] + j);
            const int mi = nd[0], mb = nd[1];
            const int64_t m = (int64_t)mi + mb;
            const T* F = C.front + (int64_t)(((uint64_t)(uint32_t)nd[3] << 32) | (uint32_t)nd[2]);
            if (up) {
                const int nlines = range_lines(F, m * mi * (int64_t)sizeof(T));
                for (int l = tid; l < nlines; l += AT) prefetch_line(F, l);
            } else if (mi > 0) {
                const int lpc = (int)((mi * (int64_t)sizeof(T) + 127) / 128) + 1;
                for (int q = tid; q < mb * lpc; q += AT) {
                    const T* seg = F + (int64_t)(mi + q / lpc) * m;
                    if (q % lpc < range_lines(seg, mi * (int64_t)sizeof(T))) prefetch_line(seg, q % lpc);
                }
            }
        }
    };
    prefetch_level(0);
    T* xin = vec + nI + mbr;
    T* part = xin + SUB_XIN;
    // first staged input / first up output of each level
    int sx_up = 0, sx_dn = 0, so_up = 0;
    if (!up)
        for (int h = 0; h < nl; ++h) sx_dn += lrec[SUB_LREC * h + 5];
    for (int hh = 0; hh < nl; ++hh) {
        prefetch_level(hh + 1);
        const int h = up ? hh : nl - 1 - hh;              // the table lists the deepest level first
        const int* L = lrec + SUB_LREC * h;
        const int cnt = L[0], n0 = L[1];
        const int R = up ? L[2] : L[3];
        const int nx = up ? L[4] : L[5];
        if (!up) sx_dn -= nx;
        const int* srcs = up ? src_up + sx_up : src_dn + sx_dn;
        const int* N = nrec + SUB_NREC * n0;
        // staged inputs (the previous level's results are in vec: barrier above)
        for (int q = tid; q < nx; q += AT) xin[q] = vec[srcs[q]];
        __syncthreads();
        const int qp = R >= AT ? 1 : AT / R;               // threads per row
        for (int ee = tid; ee < R * qp; ee += AT) {
            const int row = ee % R, p = ee / R;
            int j = 0;
            while (j + 1 < cnt && row >= N[SUB_NREC * (j + 1) + (up ? 4 : 6)]) ++j;
            const int* nd = N + SUB_NREC * j;
            const int mi = nd[0], mb = nd[1];
            const int r = row - nd[up ? 4 : 6];
            const int64_t m = (int64_t)mi + mb;
            const int64_t foff = (int64_t)(((uint64_t)(uint32_t)nd[3] << 32) | (uint32_t)nd[2]);
            // up: row r of [A_ii^{-1} P^T ; -L P^T] (m rows, m_i columns);
            // down: row r of R (m_i rows, m_b columns, at column m_i)
            const T* A = C.front + foff + (up ? 0 : (int64_t)mi * m) + r;
            const int cols = up ? mi : mb;
            const T* xs = xin + nd[up ? 5 : 7];
            // rounds of eight loads, the ragged last one predicated: it costs one
            // memory wait, not one per column
            T acc = zero<T>();
            int c = p;
            for (; c + 7 * qp < cols; c += 8 * qp) {
                T a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = A[(int64_t)(c + u * qp) * m];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc = fmac(a[u], xs[c + u * qp], acc);
            }
            if (c < cols) {
                T a[7];
#pragma unroll
                for (int u = 0; u < 7; ++u) a[u] = c + u * qp < cols ? A[(int64_t)(c + u * qp) * m] : zero<T>();
#pragma unroll
                for (int u = 0; u < 7; ++u) acc = fmac(a[u], c + u * qp < cols ? xs[c + u * qp] : zero<T>(), acc);
            }
            if (qp > 1) {
                part[ee] = acc;
            } else if (up) {
                if (r < mi) stw(z + lo + nd[8] + r, acc);
                else vec[dst_up[so_up + nd[9] + r - mi]] -= acc;
            } else {
                vec[nd[8] + r] += acc;
            }
        }
        if (qp > 1) {
            __syncthreads();
            for (int row = tid; row < R; row += AT) {
                T acc = part[row];
                for (int p = 1; p < qp; ++p) acc += part[p * R + row];
                int j = 0;
                while (j + 1 < cnt && row >= N[SUB_NREC * (j + 1) + (up ? 4 : 6)]) ++j;
                const int* nd = N + SUB_NREC * j;
                const int r = row - nd[up ? 4 : 6];
                if (up) {
                    if (r < nd[0]) stw(z + lo + nd[8] + r, acc);
                    else vec[dst_up[so_up + nd[9] + r - nd[0]]] -= acc;
                } else {
                    vec[nd[8] + r] += acc;
                }
            }
        }
        if (up) {
            sx_up += nx;
            for (int j = 0; j < cnt; ++j) so_up += N[SUB_NREC * j + 1];
        }
        __syncthreads();
    }
    if (up) {
        // the subtree's part of y(B^root), once the gather has written those
        // rows (the task reads x itself, so only this step waits for it;
        // one launch per level has run the gather before)
        if (Sp) {
            __shared__ int s_gok;
            if (tid == 0) s_gok = wait_gather(Sp) ? 1 : 0;
            __syncthreads();
            if (!s_gok) return;
        }
        for (int j = tid; j < mbr; j += AT) {
            const int g = C.blist[e.b_off + j];
            stw(y + g, ldw(y + g) + vec[nI + j]);
        }
    } else {
        for (int i0 = 0; i0 < nI; i0 += 4 * AT) {
            int pi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + tid + u * AT;
                pi[u] = i < nI ? C.perm[lo + i] : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (pi[u] >= 0) out[pi[u]] = to_val(vec[i0 + tid + u * AT]);
        }
    }
}

// Loads every task can issue before its dependencies are met: matrix
// entries (read-only during the apply) and index lists.  idx: shared int
// array of at least max(m_i, m_b, LR_CHUNK) entries.
template <typename T>
__device__ __forceinline__ void task_pre(const ApplyCtx<T>& C, const Entry& e, Pre<T>& P, int* idx, int (*wd)[8]) {
    const int tid = threadIdx.x;
    P.gi = -1;
    P.pi = -1;
    if (e.kind == TK_GATHER) return;
    if (e.kind == TK_UPW || e.kind == TK_DNW) {
        taskw_pre(C.wdesc, C.sigma, C.blist, e, idx, wd);
        return;
    }
    if (e.kind == TK_SUBUP || e.kind == TK_SUBDN) return;
    if (e.kind == TK_HUP || e.kind == TK_HROOT || e.kind == TK_HDN) {
        if (e.b_off & 1) {                       // leaf: the rows of I^s it owns, in HSS order
            const UlvDev& R = C.ulv[e.s];
            for (int j = tid; j < R.m; j += AT) idx[j] = C.ulv_ord[R.ord_off + R.lo + j];
        }
        return;
    }
    const int m_i = e.m_i, m_b = e.m_b, i_off = e.i_off, b_off = e.b_off;
    const int64_t m = (int64_t)m_i + m_b;
    const T* F = C.front + e.base;
    switch (e.kind) {
    case TK_UPDIAG: {
        gemv_pre(F, m, (int)m, m_i, e.a, P.v);
        for (int c = tid; c < m_i; c += AT) idx[c] = C.sigma[i_off + c];
        const int r = e.a + tid;
        if (tid < APPLY_ROWS && r < m) {
            if (r >= m_i) P.gi = C.blist[b_off + r - m_i];
            else if (e.fin) P.pi = C.perm[i_off + r];
        }
        break;
    }
    case TK_UP: {
        gemv_pre(F + m_i, m, m_b, m_i, e.a, P.v);
        for (int c = tid; c < m_i; c += AT) idx[c] = C.sigma[i_off + c];
        if (tid < APPLY_ROWS && e.a + tid < m_b) P.gi = C.blist[b_off + e.a + tid];
        break;
    }
    case TK_DPART: {
        const int nc = min(e.k, m_i - e.b);
        gemv_pre(F + (int64_t)e.b * m, m, m_i, nc, e.a, P.v);
        for (int c = tid; c < nc; c += AT) idx[c] = C.sigma[i_off + e.b + c];
        break;
    }
    case TK_DSUM:
        if (e.fin && e.a + tid < m_i) P.pi = C.perm[i_off + e.a + tid];
        break;
    case TK_DN: {
        gemv_pre(F + (int64_t)m_i * m, m, m_i, m_b, e.a, P.v);
        for (int j = tid; j < m_b; j += AT) idx[j] = C.blist[b_off + j];
        if (tid < APPLY_ROWS && e.a + tid < m_i) P.pi = C.perm[i_off + e.a + tid];
        break;
    }
    case TK_UPDOT: case TK_DNDOT: {
        const int k = e.k;
        const bool up = e.kind == TK_UPDOT;
        const int len = up ? m_i : m_b;
        const int rn = min(LR_CHUNK, len - e.a);
        const T* X = reinterpret_cast<const T*>(e.base);
        const T* M = (up ? X : X + (int64_t)m_i * k) + e.a;
        const int lane = tid & 31, warp = tid >> 5;
        const int a = e.b + warp;           // first column of this warp in the task's column group
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = lane + 32 * u;
            P.v[u] = (a < k && i < rn) ? M[(int64_t)a * len + i] : zero<T>();
        }
        if (sizeof(T) <= 8) {                 // the column the warp loads after the wait, into L2
            const int a1 = a + AW;
            if (a1 < k) {
                const T* seg = M + (int64_t)a1 * len;
                const int nl = range_lines(seg, (int64_t)rn * sizeof(T));
                for (int l = lane; l < nl; l += 32) prefetch_line(seg, l);
            }
        }
        if (!up)
            for (int i = tid; i < rn; i += AT) idx[i] = C.blist[b_off + e.a + i];
        break;
    }
    case TK_UPAXPY: {
        const int k = e.k;
        const T* X = reinterpret_cast<const T*>(e.base);
        gemv_pre(X + (int64_t)m_i * k, m_b, m_b, k, e.a, P.v);
        if (tid < APPLY_ROWS && e.a + tid < m_b) P.gi = C.blist[b_off + e.a + tid];
        break;
    }
    case TK_DNAXPY: {
        const int k = e.k;
        const T* X = reinterpret_cast<const T*>(e.base);
        gemv_pre(X, m_i, m_i, k, e.a, P.v);
        if (tid < APPLY_ROWS && e.a + tid < m_i) P.pi = C.perm[i_off + e.a + tid];
        break;
    }
    default: break;
    }
}

// The rest of the task, once the tasks it depends on have finished.  vec:
// shared T array of at least max(m_i, m_b, LR_CHUNK) entries.  Starts with a
// barrier (idx was written in the pre-phase) and ends with its last shared
// memory use before the caller's next barrier.
template <typename T, typename V>
__device__ __forceinline__ void task_run(const ApplyCtx<T>& C, const Entry& e, const Pre<T>& P, const int* idx, T* vec,
                                         T (*red)[APPLY_ROWS], const int (*wd)[8], int n, const V* __restrict__ x,
                                         V* __restrict__ out, T* y, T* z, T* tup, T* tdn, T* dpart, T* us,
                                         const Sched* Sp) {
    const int tid = threadIdx.x;
    if (e.kind == TK_GATHER) {
        // index loads, then gathers, four at a time (register budget)
        for (int h = 0; h < e.b / AT; h += 4) {             // e.b rows, a multiple of 4 AT
            int pi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = e.a + tid + (h + u) * AT;
                pi[u] = i < n ? C.perm[i] : -1;
            }
            V xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = pi[u] >= 0 ? x[pi[u]] : V{};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (pi[u] >= 0) stw(y + e.a + tid + (h + u) * AT, from_val<T>(xv[u]));
        }
        return;
    }
    __syncthreads();
    if (e.kind == TK_UPW || e.kind == TK_DNW) {
        taskw_run<T, V>(C, e, idx, vec, wd, out, y, z);
        return;
    }
    if (e.kind == TK_HUP || e.kind == TK_HROOT || e.kind == TK_HDN) {
        ulv_task<T, V>(C, e, idx, vec, red, out, y, z, us);
        return;
    }
    if (e.kind == TK_SUBUP || e.kind == TK_SUBDN) {
        subtree_task<T, V>(C, e, const_cast<int*>(idx), vec, x, out, y, z, Sp);
        return;
    }
    const int m_i = e.m_i, m_b = e.m_b, i_off = e.i_off;
    const int64_t m = (int64_t)m_i + m_b;
    const T* F = C.front + e.base;
    switch (e.kind) {
    case TK_UPDIAG: {
        for (int c = tid; c < m_i; c += AT) vec[c] = ldw(y + i_off + idx[c]);
        __syncthreads();
        const T sum = gemv_rows64(F, m, (int)m, m_i, e.a, vec, red, P.v);
        const int r = e.a + tid;
        if (tid < APPLY_ROWS && r < m) {
            if (r < m_i) {
                stw(z + i_off + r, sum);
                if (e.fin) out[P.pi] = to_val(sum);
            } else {
                stw(y + P.gi, ldw(y + P.gi) - sum);
            }
        }
        break;
    }
    case TK_UP: {
        for (int c = tid; c < m_i; c += AT) vec[c] = ldw(y + i_off + idx[c]);
        __syncthreads();
        const T sum = gemv_rows64(F + m_i, m, m_b, m_i, e.a, vec, red, P.v);
        if (P.gi >= 0) stw(y + P.gi, ldw(y + P.gi) - sum);
        break;
    }
    case TK_DPART: {
        const int nc = min(e.k, m_i - e.b);
        for (int c = tid; c < nc; c += AT) vec[c] = ldw(y + i_off + idx[c]);
        __syncthreads();
        const T sum = gemv_rows64(F + (int64_t)e.b * m, m, m_i, nc, e.a, vec, red, P.v);
        const int r = e.a + tid;
        if (tid < APPLY_ROWS && r < m_i) stw(dpart + e.aux + (int64_t)(e.b / e.k) * m_i + r, sum);
        break;
    }
    case TK_DSUM: {
        const int r = e.a + tid;
        if (r < m_i) {
            // the column-chunk partials (chunk width e.k), eight loads in flight
            const int nch = (m_i + e.k - 1) / e.k;
            const T* p = dpart + e.aux + r;
            T acc = zero<T>();
            for (int c0 = 0; c0 < nch; c0 += 8) {
                T pv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) pv[u] = c0 + u < nch ? ldw(p + (int64_t)(c0 + u) * m_i) : zero<T>();
#pragma unroll
                for (int u = 0; u < 8; ++u) acc = acc + pv[u];
            }
            stw(z + i_off + r, acc);
            if (e.fin) out[P.pi] = to_val(acc);
        }
        break;
    }
    case TK_DN: {
        for (int j = tid; j < m_b; j += AT) vec[j] = ldw(z + idx[j]);
        __syncthreads();
        const T sum = gemv_rows64(F + (int64_t)m_i * m, m, m_i, m_b, e.a, vec, red, P.v);
        const int r = e.a + tid;
        if (tid < APPLY_ROWS && r < m_i) {
            const T v = ldw(z + i_off + r) + sum;
            stw(z + i_off + r, v);
            out[P.pi] = to_val(v);
        }
        break;
    }
    case TK_UPDOT: case TK_DNDOT: {
        // Low-rank (R ~ X R(J, :), stored as X (m_i x k) then RJt = R(J, :)^T
        // (m_b x k), column-major; L = R^T): t_c = M(chunk, :)^T v(chunk) with
        // M = X going up (v = y(I)), M = RJt coming down (v = z(B)); warp w
        // takes columns w, w + 8, ...; each lane 8 rows of each column.
        const bool up = e.kind == TK_UPDOT;
        const int k = e.k;
        const int len = up ? m_i : m_b;
        const int rn = min(LR_CHUNK, len - e.a);
        const int lane = tid & 31, warp = tid >> 5;
        const T* X = reinterpret_cast<const T*>(e.base);
        const T* M = (up ? X : X + (int64_t)m_i * k) + e.a;
        T* dst = (up ? tup : tdn) + e.aux + (int64_t)(e.a / LR_CHUNK) * k;
        // the task's column group: columns b + warp + v * AW, v < CPS (two per
        // warp for 8-byte types, one for 16-byte types); v = 0 was loaded in
        // the pre-phase, v >= 1 goes out together with the input rows
        constexpr int CPS = sizeof(T) <= 8 ? 2 : 1;
        T p[CPS][8];
#pragma unroll
        for (int v = 0; v < CPS; ++v)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = lane + 32 * u, av = e.b + warp + v * AW;
                p[v][u] = (v == 0) ? P.v[u] : ((av < k && i < rn) ? M[(int64_t)av * len + i] : zero<T>());
            }
        for (int i = tid; i < rn; i += AT) vec[i] = up ? ldw(y + i_off + e.a + i) : ldw(z + idx[i]);
        __syncthreads();
        T sp[CPS];
#pragma unroll
        for (int v = 0; v < CPS; ++v) sp[v] = zero<T>();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = lane + 32 * u;
            const T xv = (i < rn) ? vec[i] : zero<T>();
#pragma unroll
            for (int v = 0; v < CPS; ++v) sp[v] = fmac(p[v][u], xv, sp[v]);
        }
#pragma unroll
        for (int v = 0; v < CPS; ++v) {
            for (int o = 16; o; o >>= 1) sp[v] = sp[v] + shfl_xor_t(sp[v], o);
            const int av = e.b + warp + v * AW;
            if (lane == 0 && av < k) stw(dst + av, sp[v]);
        }
        break;
    }
    case TK_UPAXPY: case TK_DNAXPY: {
        // t = sum of the dot tasks' chunk partials, then 64 rows of M t with
        // M = RJt going up (rows of B), X coming down (rows of I)
        const bool up = e.kind == TK_UPAXPY;
        const int k = e.k;
        const int len_in = up ? m_i : m_b, len = up ? m_b : m_i;
        const int nch = (len_in + LR_CHUNK - 1) / LR_CHUNK;
        const T* tp = (up ? tup : tdn) + e.aux;
        const int r = e.a + tid;
        // the row this thread updates is final once the task's dependencies
        // are (siblings' B sets are disjoint): its load goes out with the
        // chunk partials of t, eight chunks at a time
        T old = zero<T>();
        if (tid < APPLY_ROWS && r < len) old = up ? ldw(y + P.gi) : ldw(z + i_off + r);
        for (int a = tid; a < k; a += AT) {
            T acc = zero<T>();
            for (int c0 = 0; c0 < nch; c0 += 8) {
                T pv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) pv[u] = c0 + u < nch ? ldw(tp + (int64_t)(c0 + u) * k + a) : zero<T>();
#pragma unroll
                for (int u = 0; u < 8; ++u) acc = acc + pv[u];
            }
            vec[a] = acc;
        }
        __syncthreads();
        const T* X = reinterpret_cast<const T*>(e.base);
        const T sum = gemv_rows64(up ? X + (int64_t)m_i * k : X, len, len, k, e.a, vec, red, P.v);
        if (tid < APPLY_ROWS && r < len) {
            if (up) {
                stw(y + P.gi, old + sum);
            } else {
                const T v = old + sum;
                stw(z + i_off + r, v);
                out[P.pi] = to_val(v);
            }
        }
        break;
    }
    default: break;
    }
}

// ---- dataflow schedule: one persistent launch -----------------------------

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct Sched {
    const int32_t* q;          // [QW * nq] entries
    const int4* dep;           // [2 * nq] dependency records (sched_deps_kernel)
    int32_t nq, ngather, nn, nrec;
    const int32_t* need;       // [NCNT * nn + 2 * nrec]
    int32_t* ctl;              // [CTL_WORDS + NCNT * nn + 2 * nrec], zeroed before the launch
    int32_t* err;              // sticky error word of the factorization
};
// counters of the ULV records (up / down), after the per-node counters
__device__ __forceinline__ int hu_index(const Sched& S, int rec) { return NCNT * S.nn + rec; }
__device__ __forceinline__ int hd_index(const Sched& S, int rec) { return NCNT * S.nn + S.nrec + rec; }

// Bounded wait until *ctr >= need; false once the wait gave up or another
// CTA reported a failure.
__device__ bool wait_geq(const Sched& S, const int32_t* ctr, int need, uint64_t& t0) {
    if (need <= 0 || ld_acquire(ctr) >= need) return true;
    // short sleeps while the wait is young (a dependency in the low-rank
    // chain is usually a few microseconds away), the abort flag and the clock
    // every 16th poll
    for (unsigned it = 0;; ++it) {
        if (ld_acquire(ctr) >= need) return true;
        if ((it & 15) == 15) {
            if (ld_relaxed(S.ctl + 2)) return false;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > APPLY_WAIT_NS) {
                atomicExch(S.ctl + 2, 1);
                atomicExch(S.err, 1);
                return false;
            }
        }
        __nanosleep(it < 64 ? 20 : 200);
    }
}

// Up to three (counter, requirement) pairs a task waits for.
struct Deps {
    const int32_t* c[3];
    int need[3];
    int n;
};

__device__ __forceinline__ Deps task_deps(const Sched& S, const int32_t* node, const Entry& e) {
    Deps d;
    d.n = 0;
    const int32_t* cnt = S.ctl + CTL_WORDS;
    const int nn = S.nn, s = e.s;
    auto add = [&](int c, int which) {
        d.c[d.n] = cnt + which * nn + c;
        d.need[d.n] = S.need[which * nn + c];
        ++d.n;
    };
    switch (e.kind) {
    case TK_UPDIAG: case TK_UP: case TK_UPDOT: case TK_UPNOP: case TK_DPART: {
        d.c[0] = S.ctl + 1;
        d.need[0] = S.ngather;
        d.n = 1;
        const int c0 = nf(node, s, 2), c1 = nf(node, s, 3);
        if (c0 >= 0) add(c0, CN_UP);
        if (c1 >= 0) add(c1, CN_UP);
        break;
    }
    case TK_UPAXPY: add(s, CN_DOT); break;
    case TK_DSUM: add(s, CN_DPART); break;
    case TK_DN: case TK_DNDOT: case TK_FINNOP: {
        const int p = nf(node, s, 1);
        if (p >= 0) add(p, CN_FIN);
        if (e.kind == TK_DN) add(s, CN_DIAG);
        break;
    }
    case TK_DNAXPY: add(s, CN_DDOT); add(s, CN_DIAG); break;
    case TK_HUP: case TK_HROOT:
        if (e.b_off & 1) {                          // leaf: the front's y(I^s) is final
            d.c[0] = S.ctl + 1;
            d.need[0] = S.ngather;
            d.n = 1;
            const int c0 = nf(node, e.a, 2), c1 = nf(node, e.a, 3);
            if (c0 >= 0) add(c0, CN_UP);
            if (c1 >= 0) add(c1, CN_UP);
        } else {                                    // inner: both HSS children went up
            d.c[0] = cnt + hu_index(S, e.m_i);
            d.need[0] = S.need[hu_index(S, e.m_i)];
            d.c[1] = cnt + hu_index(S, e.m_b);
            d.need[1] = S.need[hu_index(S, e.m_b)];
            d.n = 2;
        }
        break;
    case TK_HDN:
        d.c[0] = cnt + hd_index(S, e.i_off);
        d.need[0] = S.need[hd_index(S, e.i_off)];
        d.n = 1;
        break;
    case TK_SUBUP:                                  // waits for the gather only before adding to y(B^root)
        break;
    case TK_SUBDN: {                                // the root's parent final, the subtree's up done
        const int p = nf(node, s, 1);
        if (p >= 0) add(p, CN_FIN);
        add(s, CN_UP);
        break;
    }
    default: break;
    }
    return d;
}

// The dependency record of every queue entry, written once per schedule
// (and again when a requirement changes): counter words relative to ctl and
// their count, then the requirements.  A task's wait then reads its counters
// in one round of loads instead of walking the node table first.
__global__ void sched_deps_kernel(Sched S, const int32_t* __restrict__ node, int4* __restrict__ dep) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.nq) return;
    const Entry e = decode(S.q, t);
    Deps d;
    d.n = 0;
    if (e.kind != TK_UPW && e.kind != TK_DNW) d = task_deps(S, node, e);
    int c[3] = {0, 0, 0}, need[3] = {0, 0, 0};
    for (int i = 0; i < d.n; ++i) {
        c[i] = (int)(d.c[i] - S.ctl);
        need[i] = d.need[i];
    }
    dep[2 * t] = make_int4(c[0], c[1], c[2], d.n);
    dep[2 * t + 1] = make_int4(need[0], need[1], need[2], 0);
}

// All requirements read at once with acquire loads, together with the abort
// flags (the common case: already met), otherwise bounded spins with acquire
// loads.  The waiting thread's acquire and the CTA barrier after it order the
// task's reads after the producers' release fences.
__device__ bool wait_deps(const Sched& S, int4 d0, int4 d1) {
    const int n = d0.w;
    const int c[3] = {d0.x, d0.y, d0.z}, need[3] = {d1.x, d1.y, d1.z};
    int v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = (i < n) ? ld_acquire(S.ctl + c[i]) : 0;
    if (ld_relaxed(S.ctl + 2) || ld_relaxed(S.err)) return false;
    bool met = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) met = met && (i >= n || v[i] >= need[i]);
    if (!met) {
        uint64_t t0 = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i < n && !wait_geq(S, S.ctl + c[i], need[i], t0)) return false;
    }
    return true;
}

__device__ bool wait_gather(const Sched* S) {
    uint64_t t0 = 0;
    return wait_geq(*S, S->ctl + 1, S->ngather, t0);
}

// Dependencies of a warp-node task, checked by warp 0: lane j < e.a waits for
// node j's children (TK_UPW; lane 0 also for the gather) or for its parent's
// final rows and its own diagonal rows (TK_DNW).  True on every lane when all
// are met.
__device__ bool wait_deps_w(const Sched& S, const int32_t* node, const int32_t* wdesc, const Entry& e) {
    const int lane = threadIdx.x & 31;
    bool ok = !(ld_relaxed(S.ctl + 2) || ld_relaxed(S.err));
    const int32_t* cnt = S.ctl + CTL_WORDS;
    const int nn = S.nn;
    uint64_t t0 = 0;
    if (ok && e.kind == TK_UPW && lane == 0) ok = wait_geq(S, S.ctl + 1, S.ngather, t0);
    if (ok && lane < e.a) {
        const int s = wdesc[(e.base + lane) * 8];
        if (e.kind == TK_UPW) {
            const int c0 = nf(node, s, 2), c1 = nf(node, s, 3);
            if (c0 >= 0) ok = ok && wait_geq(S, cnt + CN_UP * nn + c0, S.need[CN_UP * nn + c0], t0);
            if (c1 >= 0) ok = ok && wait_geq(S, cnt + CN_UP * nn + c1, S.need[CN_UP * nn + c1], t0);
        } else {
            const int p = nf(node, s, 1);
            if (p >= 0) ok = ok && wait_geq(S, cnt + CN_FIN * nn + p, S.need[CN_FIN * nn + p], t0);
            ok = ok && wait_geq(S, cnt + CN_DIAG * nn + s, S.need[CN_DIAG * nn + s], t0);
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    __threadfence();
    return ok;
}

// counters a finished task signals (bit per CN_*), -1 bit 31 for the gather count
__device__ __forceinline__ unsigned task_signals(const Entry& e) {
    switch (e.kind) {
    case TK_GATHER: return 1u << 31;
    case TK_UPDIAG: return (1u << CN_UP) | (1u << CN_DIAG) | (e.fin ? (1u << CN_FIN) : 0u);
    case TK_UP: case TK_UPAXPY: case TK_UPNOP: return 1u << CN_UP;
    case TK_UPDOT: return 1u << CN_DOT;
    case TK_DPART: return 1u << CN_DPART;
    case TK_DSUM: return (1u << CN_DIAG) | (e.fin ? (1u << CN_FIN) : 0u);
    case TK_DN: case TK_DNAXPY: case TK_FINNOP: return 1u << CN_FIN;
    case TK_DNDOT: return 1u << CN_DDOT;
    case TK_SUBUP: return 1u << CN_UP;
    case TK_SUBDN: return 1u << CN_FIN;
    default: return 0u;
    }
}

// resident CTAs per SM the register budget is sized for (latency hiding)
template <typename T> constexpr int apply_min_blocks() { return sizeof(T) <= 8 ? 4 : 3; }

template <typename T, typename V>
__global__ void __launch_bounds__(AT, apply_min_blocks<T>()) apply_dataflow_kernel(ApplyCtx<T> C, Sched S, int n, const V* __restrict__ x,
                                                            V* __restrict__ out, T* y, T* z, T* tup, T* tdn, T* dpart,
                                                            T* us, int vlen, const ApplyInd* ind) {
    if (ind) {
        // vectors chosen on the device by the caller's previous kernel
        if (*(volatile const int32_t*)ind->skip) return;
        x = static_cast<const V*>(ind->x);
        out = static_cast<V*>(ind->y);
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[AW][APPLY_ROWS];
    __shared__ int s_task, s_ok;
    __shared__ int wd[AW][8];
    T* vec = reinterpret_cast<T*>(smem_raw);
    int* idx = reinterpret_cast<int*>(vec + vlen);
    int32_t* cnt = S.ctl + CTL_WORDS;
    // thread 0 holds the next ticket while the CTA works on the current task:
    // the ticket's atomic overlaps the work (deadlock-free: a held ticket is
    // only waited on by higher tickets, and its holder starts it as soon as
    // its current task ends); subtree tasks take theirs at the end
    int next = (threadIdx.x == 0) ? atomicAdd(S.ctl, 1) : 0;
    for (;;) {
        if (threadIdx.x == 0) s_task = next;
        __syncthreads();
        const int t = s_task;
        if (t >= S.nq) break;
        int4 d0 = make_int4(0, 0, 0, 0), d1 = d0;
        if (threadIdx.x == 0) {
            d0 = __ldg(S.dep + 2 * (int64_t)t);
            d1 = __ldg(S.dep + 2 * (int64_t)t + 1);
        }
        const Entry e = decode(S.q, t);
        Pre<T> P;
        task_pre(C, e, P, idx, wd);
        const bool warp_nodes = e.kind == TK_UPW || e.kind == TK_DNW;
        // a subtree task runs for tens of microseconds: the CTA takes its next
        // ticket when it ends, so no ready task waits behind it
        const bool long_task = e.kind == TK_SUBUP || e.kind == TK_SUBDN;
        if (warp_nodes ? threadIdx.x < 32 : threadIdx.x == 0) {
            const bool ok = warp_nodes ? wait_deps_w(S, C.node, C.wdesc, e) : wait_deps(S, d0, d1);
            if (threadIdx.x == 0) {
                s_ok = ok ? 1 : 0;
                if (ok && !long_task) next = atomicAdd(S.ctl, 1);
            }
        }
        __syncthreads();
        if (!s_ok) break;
        task_run<T, V>(C, e, P, idx, vec, red, wd, n, x, out, y, z, tup, tdn, dpart, us, &S);
        // publish: the barrier orders every thread's stores before the
        // signalling threads' gpu-scope fences, which order them before the
        // signals
        __syncthreads();
        if (long_task && threadIdx.x == 0) next = atomicAdd(S.ctl, 1);
        if (warp_nodes) {
            const int lane = threadIdx.x;
            if (lane < e.a) {
                const int sj = wd[lane][0];
                __threadfence();
                if (e.kind == TK_UPW) {
                    atomicAdd(cnt + CN_UP * S.nn + sj, 1);
                    atomicAdd(cnt + CN_DIAG * S.nn + sj, 1);
                } else {
                    atomicAdd(cnt + CN_FIN * S.nn + sj, 1);
                }
            }
        } else if (threadIdx.x == 0 && (e.kind == TK_HUP || e.kind == TK_HROOT || e.kind == TK_HDN)) {
            __threadfence();
            atomicAdd(cnt + (e.kind == TK_HUP ? hu_index(S, e.s) : hd_index(S, e.s)), 1);
            if (e.kind != TK_HUP && (e.b_off & 1)) {        // a leaf wrote its rows of z(I^s)
                atomicAdd(cnt + CN_DIAG * S.nn + e.a, 1);
                if (e.fin) atomicAdd(cnt + CN_FIN * S.nn + e.a, 1);
            }
        } else if (threadIdx.x == 0) {
            __threadfence();
            const unsigned sig = task_signals(e);
            if (sig >> 31) atomicAdd(S.ctl + 1, 1);
#pragma unroll
            for (int w = 0; w < NCNT; ++w)
                if ((sig >> w) & 1u) atomicAdd(cnt + w * S.nn + e.s, 1);
        }
    }
}

// ---- level schedule: one launch per dependency group of the queue ---------

template <typename T, typename V>
__global__ void __launch_bounds__(AT, apply_min_blocks<T>()) apply_group_kernel(ApplyCtx<T> C, const int32_t* __restrict__ q, int n,
                                                         const V* __restrict__ x, V* __restrict__ out, T* y, T* z, T* tup,
                                                         T* tdn, T* dpart, T* us, int vlen, const ApplyInd* ind) {
    if (ind) {
        if (*(volatile const int32_t*)ind->skip) return;
        x = static_cast<const V*>(ind->x);
        out = static_cast<V*>(ind->y);
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[AW][APPLY_ROWS];
    __shared__ int wd[AW][8];
    T* vec = reinterpret_cast<T*>(smem_raw);
    int* idx = reinterpret_cast<int*>(vec + vlen);
    const Entry e = decode(q, blockIdx.x);
    Pre<T> P;
    task_pre(C, e, P, idx, wd);
    task_run<T, V>(C, e, P, idx, vec, red, wd, n, x, out, y, z, tup, tdn, dpart, us, nullptr);
}

bool levels_schedule_requested() {
    const char* e = std::getenv("NDHSS_APPLY_SCHEDULE");
    return e && std::strcmp(e, "levels") == 0;
}

template <typename T>
ApplyCtx<T> make_ctx(const FactorData& F) {
    return ApplyCtx<T>{F.d_node, F.d_blist, F.d_sigma, F.d_perm, static_cast<const T*>(F.d_front), F.d_wdesc,
                       reinterpret_cast<const UlvDev*>(F.d_ulvdev), F.d_ulv_ord, F.d_foff, F.d_sublist};
}

// work space: y, z (n each), low-rank partials for each sweep, diagonal
// partials, control words
struct WorkLayout {
    size_t y, z, tup, tdn, dpart, us, ctl, total;
};
WorkLayout work_layout(const FactorData& F) {
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    WorkLayout L{};
    const size_t vec = r256((size_t)F.n * F.esize);
    const size_t tb = r256((size_t)std::max<int64_t>(F.lr_t_total, 1) * F.esize);
    L.y = 0;
    L.z = vec;
    L.tup = 2 * vec;
    L.tdn = L.tup + tb;
    L.dpart = L.tdn + tb;
    L.us = L.dpart + r256((size_t)std::max<int64_t>(F.dpart_total, 1) * F.esize);
    L.ctl = L.us + r256((size_t)std::max<int64_t>(F.ulv_scratch, 1) * F.esize);
    L.total = L.ctl + r256(sizeof(int32_t) * (CTL_WORDS + (size_t)NCNT * std::max(F.nnodes, 1) +
                                              2 * (size_t)F.ulv_recs.size()));
    return L;
}

size_t smem_bytes(const FactorData& F, size_t esize) {
    return (size_t)F.sched_vlen * (esize + sizeof(int));
}

template <typename T, typename V>
ndhss_status apply_run(const FactorData& F, int32_t nrhs, const V* x, int64_t ldx, V* y, int64_t ldy, unsigned char* w,
                       cudaStream_t st, const ApplyInd* ind) {
    if (!F.d_sched) return set_error(NDHSS_ERR_INTERNAL, "apply: factorization has no task queue");
    const WorkLayout WL = work_layout(F);
    const ApplyCtx<T> C = make_ctx<T>(F);
    T* wy = reinterpret_cast<T*>(w + WL.y);
    T* wz = reinterpret_cast<T*>(w + WL.z);
    T* tup = reinterpret_cast<T*>(w + WL.tup);
    T* tdn = reinterpret_cast<T*>(w + WL.tdn);
    T* dpart = reinterpret_cast<T*>(w + WL.dpart);
    T* us = reinterpret_cast<T*>(w + WL.us);
    const size_t smem = smem_bytes(F, sizeof(T));
    const int vlen = F.sched_vlen;
    if (levels_schedule_requested()) {
        for (int r = 0; r < nrhs; ++r)
            for (size_t g = 0; g + 1 < F.sched_groups.size(); ++g) {
                const int64_t g0 = F.sched_groups[g], g1 = F.sched_groups[g + 1];
                if (g1 == g0) continue;
                apply_group_kernel<T, V><<<(unsigned)(g1 - g0), AT, smem, st>>>(
                    C, F.d_sched + QW * g0, F.n, x + r * ldx, y + r * ldy, wy, wz, tup, tdn, dpart, us, vlen, ind);
                NDHSS_LAUNCH_CHECK("apply_group_kernel");
            }
        return NDHSS_OK;
    }
    Sched S{F.d_sched, reinterpret_cast<const int4*>(F.d_sched_dep), (int32_t)F.sched_n, F.sched_ngather, F.nnodes,
            (int32_t)F.ulv_recs.size(), F.d_need, reinterpret_cast<int32_t*>(w + WL.ctl), F.d_apply_err};
    const size_t ctl_bytes = sizeof(int32_t) * (CTL_WORDS + (size_t)NCNT * F.nnodes + 2 * F.ulv_recs.size());
    for (int r = 0; r < nrhs; ++r) {
        NDHSS_CUDA_TRY(cudaMemsetAsync(S.ctl, 0, ctl_bytes, st));
        apply_dataflow_kernel<T, V><<<(unsigned)F.sched_grid, AT, smem, st>>>(C, S, F.n, x + r * ldx, y + r * ldy, wy, wz,
                                                                              tup, tdn, dpart, us, vlen, ind);
        NDHSS_LAUNCH_CHECK("apply_dataflow_kernel");
    }
    return NDHSS_OK;
}

// Grid of the persistent launch: every SM filled to its occupancy limit.
template <typename T, typename V>
ndhss_status launch_shape(FactorData& F) {
    // the opt-in limit also admits dynamic memory that, with the kernels'
    // static shared memory, passes the default 48 KB
    const size_t smem = smem_bytes(F, sizeof(T));
    NDHSS_CUDA_TRY(cudaFuncSetAttribute(apply_dataflow_kernel<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    NDHSS_CUDA_TRY(cudaFuncSetAttribute(apply_group_kernel<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    NDHSS_CUDA_TRY(cudaGetDevice(&dev));
    NDHSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NDHSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_dataflow_kernel<T, V>, AT, smem));
    if (per_sm < 1) return set_error(NDHSS_ERR_INVALID_ARG, "apply: %zu bytes of shared memory per CTA do not fit an SM", smem);
    F.sched_grid = sms * per_sm;
    return NDHSS_OK;
}

}  // namespace

// Host-built task queue of the apply (see the top of this file).
ndhss_status fill_sched_deps(const FactorData& F, cudaStream_t st) {
    const Sched S{F.d_sched, nullptr, (int32_t)F.sched_n, F.sched_ngather, F.nnodes, (int32_t)F.ulv_recs.size(),
                  F.d_need, nullptr, nullptr};
    const unsigned blocks = (unsigned)((F.sched_n + 255) / 256);
    sched_deps_kernel<<<blocks, 256, 0, st>>>(S, F.d_node, reinterpret_cast<int4*>(F.d_sched_dep));
    NDHSS_LAUNCH_CHECK("sched_deps_kernel");
    return NDHSS_OK;
}

ndhss_status build_apply_schedule(FactorData& F, cudaStream_t st) {
    const int nn = F.nnodes;
    if ((int64_t)nn >= (int64_t(1) << TK_SHIFT)) return set_error(NDHSS_ERR_INVALID_ARG, "apply: too many tree nodes");
    const int nrec = (int)F.ulv_recs.size();
    std::vector<int32_t> q, need((size_t)NCNT * std::max(nn, 1) + 2 * (size_t)nrec, 0);
    std::vector<int64_t> groups{0};
    std::vector<int64_t> dpoff(std::max(nn, 1), 0);
    std::vector<int32_t> dcols(std::max(nn, 1), DIAG_COLS);   // column chunk of each node's diagonal tasks
    auto push = [&](int kind, int s, int a, int b, bool fin) {
        const bool lr = kind == TK_UPDOT || kind == TK_UPAXPY || kind == TK_DNDOT || kind == TK_DNAXPY;
        const int64_t base = kind == TK_GATHER ? 0 : lr ? (int64_t)F.lr_ptr[s] : F.foff[s];
        const int64_t aux = lr ? F.lr_toff[s] : (kind == TK_DPART || kind == TK_DSUM) ? dpoff[s] : 0;
        const bool g = kind == TK_GATHER;
        const int32_t w[QW] = {(fin ? TK_FINAL : 0) | (kind << TK_SHIFT) | s, a, b,
                               g ? 0 : F.m_i(s), g ? 0 : F.m_b(s), g ? 0 : F.info(s, 4), g ? 0 : F.info(s, 6),
                               lr ? F.lr_k[s] : (kind == TK_DPART || kind == TK_DSUM) ? dcols[s] : 0,
                               (int32_t)(uint32_t)(uint64_t)base, (int32_t)(uint32_t)((uint64_t)base >> 32),
                               (int32_t)(uint32_t)(uint64_t)aux, (int32_t)(uint32_t)((uint64_t)aux >> 32)};
        q.insert(q.end(), w, w + QW);
    };
    auto cut = [&]() {
        if ((int64_t)q.size() / QW != groups.back()) groups.push_back((int64_t)q.size() / QW);
    };
    auto ceil_div = [](int a, int b) { return (a + b - 1) / b; };
    // node mode: 0 dense, 1 low-rank with rank k > 0, 2 low-rank with k = 0
    auto mode = [&](int s) {
        if (F.lr_ptr.empty() || !F.lr_ptr[s]) return 0;
        return F.lr_k[s] > 0 ? 1 : 2;
    };
    auto fused = [&](int s) { return F.m_i(s) > 0 && mode(s) == 0 && F.m_i(s) <= DIAG_COLS; };
    // the tasks that write z(I^s) last: the diagonal step when nothing is added later
    auto diag_final = [&](int s) { return F.m_b(s) == 0 || mode(s) == 2; };
    F.dpart_total = 0;
    // low-rank dot tasks: one LR_CHUNK-row chunk times one column group
    const int dgw = (AT / 32) * (F.esize <= 8 ? 2 : 1);
    // warp-node levels: the bottom range of levels whose nodes are all dense
    // and tiny; a task takes up to AW consecutive nodes of one level
    auto tiny = [&](int s) {
        return mode(s) == 0 && F.m_i(s) <= WN_MI && F.m_i(s) + F.m_b(s) <= WN_M && F.m_b(s) <= WREG;
    };
    // bottom subtrees: the shallowest level Ls from which every node down to
    // the leaves is dense with small fronts and every subtree fits one task
    // (NDHSS_APPLY_SUBTREES=0 keeps per-node tasks everywhere)
    auto ulv_node = [&](int s) { return !F.ulv_root_of.empty() && F.ulv_root_of[s] >= 0; };
    std::vector<int32_t> sublist;
    std::vector<int> sub_off(nn, -1), sub_lo(nn, 0), sub_ni(nn, 0), sub_len(nn, 0);   // per subtree root
    int Ls = F.depth + 1;
    {
        const char* ev = std::getenv("NDHSS_APPLY_SUBTREES");
        const bool enabled = !(ev && std::strcmp(ev, "0") == 0);
        std::vector<int> first(nn), cntn(nn, 1), nlev(nn, 1);
        std::vector<int64_t> ni(nn), mxin(nn, 0);
        for (int s = 0; s < nn; ++s) {           // post-order: children before parents
            const int c0 = F.info(s, 2), c1 = F.info(s, 3);
            first[s] = c0 >= 0 ? first[c0] : s;
            ni[s] = F.m_i(s) + (c0 >= 0 ? ni[c0] : 0) + (c1 >= 0 ? ni[c1] : 0);
            cntn[s] = 1 + (c0 >= 0 ? cntn[c0] : 0) + (c1 >= 0 ? cntn[c1] : 0);
            nlev[s] = 1 + std::max(c0 >= 0 ? nlev[c0] : 0, c1 >= 0 ? nlev[c1] : 0);
        }
        auto node_ok = [&](int s) {
            return mode(s) == 0 && !ulv_node(s) && F.m_i(s) <= 2 * WN_MI && F.m_b(s) <= 4 * WREG;
        };
        // a subtree fits: nodes, levels, nodes and staged inputs per level, vector segment
        auto root_ok = [&](int r) {
            if (cntn[r] > SUB_NODES || nlev[r] > SUB_LV || ni[r] + F.m_b(r) > SUB_V) return false;
            std::vector<int> per(nlev[r], 0), xu(nlev[r], 0), xd(nlev[r], 0);
            const int l0 = F.info(r, 0);
            for (int s = first[r]; s <= r; ++s) {
                const int h = F.info(s, 0) - l0;
                per[h]++;
                xu[h] += F.m_i(s);
                xd[h] += F.m_b(s);
            }
            for (int h = 0; h < nlev[r]; ++h)
                if (per[h] > SUB_LVN || xu[h] > SUB_XIN || xd[h] > SUB_XIN) return false;
            return true;
        };
        if (enabled && F.nnodes > 0) {
            std::vector<char> deep_ok(F.depth + 2, 1);   // every node on levels >= l qualifies
            for (int l = F.depth; l >= 0; --l) {
                bool ok = deep_ok[l + 1];
                for (int s : F.levels[l]) ok = ok && node_ok(s);
                deep_ok[l] = ok;
            }
            for (int l = F.depth; l >= 0; --l) {
                if (!deep_ok[l]) break;
                bool ok = true;
                for (int s : F.levels[l]) ok = ok && root_ok(s);
                if (!ok) break;
                Ls = l;
            }
            // enough subtrees to fill the GPU (deeper levels have more of them)
            while (Ls <= F.depth && (int)F.levels[Ls].size() < SUB_MIN_ROOTS) ++Ls;
        }
        if (Ls <= F.depth) {
            // the pivot order of every interior block (final: the factorization
            // has synchronised) resolves the staged inputs of the up sweep here
            std::vector<int32_t> sig_h(std::max(F.n, 1));
            cudaError_t ce = cudaMemcpyAsync(sig_h.data(), F.d_sigma, sizeof(int32_t) * (size_t)F.n,
                                             cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            if (ce != cudaSuccess) return set_error(NDHSS_ERR_CUDA, "apply: %s", cudaGetErrorString(ce));
            // the tables of all subtrees, built in parallel: sizes and offsets
            // first, then every subtree fills its own range
            const std::vector<int>& roots = F.levels[Ls];
            const int nsub = (int)roots.size();
            std::vector<int64_t> soff(nsub + 1, 0);
            for (int i = 0; i < nsub; ++i) {
                const int r = roots[i];
                int64_t mbs = 0;
                for (int q = first[r]; q <= r; ++q) mbs += F.m_b(q);
                soff[i + 1] = soff[i] + SUB_HDR + (int64_t)SUB_LREC * nlev[r] + (int64_t)SUB_NREC * cntn[r] + ni[r] + mbs;
            }
            if (soff[nsub] >= (int64_t)INT32_MAX) return set_error(NDHSS_ERR_INVALID_ARG, "apply: subtree tables too long");
            sublist.assign((size_t)soff[nsub], 0);
            std::atomic<int> bad{-1};
            auto fill = [&](int i) {
                const int r = roots[i];
                const int lo = F.info(first[r], 4);
                const int nI = (int)ni[r];
                int32_t* out = sublist.data() + soff[i];
                // the task's table (see subtree_task): levels deepest first,
                // ascending ids within a level
                const int nl = nlev[r], l0 = F.info(r, 0);
                std::vector<std::vector<int>> bylev(nl);
                for (int q = first[r]; q <= r; ++q) bylev[nl - 1 - (F.info(q, 0) - l0)].push_back(q);
                // the vector slot of every B^root row (sorted by row for the lookups)
                std::vector<std::pair<int, int>> broot((size_t)F.m_b(r));
                for (int j = 0; j < F.m_b(r); ++j) broot[j] = {F.blist_h[F.info(r, 6) + j], nI + j};
                std::sort(broot.begin(), broot.end());
                auto bslot_of = [&](int q, int j) {
                    const int g = F.blist_h[F.info(q, 6) + j];
                    if (g >= lo && g < lo + nI) return g - lo;
                    auto it = std::lower_bound(broot.begin(), broot.end(), std::make_pair(g, INT32_MIN));
                    return (it != broot.end() && it->first == g) ? it->second : -1;
                };
                int32_t* lrec = out + SUB_HDR;
                int32_t* nrec = lrec + SUB_LREC * nl;
                int32_t* src_up = nrec + SUB_NREC * cntn[r];
                int32_t* src_dn = src_up + nI;
                int nidx = 0;
                for (int h = 0; h < nl; ++h) {
                    int ru = 0, rd = 0, xu = 0, xd = 0, bo = 0;
                    for (int q : bylev[h]) {
                        const uint64_t fo = (uint64_t)F.foff[q];
                        const int32_t nd[SUB_NREC] = {F.m_i(q), F.m_b(q), (int32_t)(uint32_t)fo, (int32_t)(uint32_t)(fo >> 32),
                                                      ru, xu, rd, xd, F.info(q, 4) - lo, bo};
                        std::copy(nd, nd + SUB_NREC, nrec);
                        nrec += SUB_NREC;
                        // column c of A_ii^{-1} multiplies interior row sigma(c)
                        for (int c = 0; c < F.m_i(q); ++c) *src_up++ = F.info(q, 4) - lo + sig_h[F.info(q, 4) + c];
                        for (int j = 0; j < F.m_b(q); ++j) {
                            const int sl = bslot_of(q, j);
                            if (sl < 0) bad.store(q);
                            *src_dn++ = sl;
                        }
                        ru += F.m_i(q) + F.m_b(q);
                        rd += F.m_i(q);
                        xu += F.m_i(q);
                        xd += F.m_b(q);
                        bo += F.m_b(q);
                    }
                    const int32_t lr[SUB_LREC] = {(int32_t)bylev[h].size(), nidx, ru, rd, xu, xd};
                    std::copy(lr, lr + SUB_LREC, lrec + SUB_LREC * h);
                    nidx += (int)bylev[h].size();
                }
                out[0] = nl;
                out[1] = nidx;
            };
            const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            if (nth == 1 || nsub < 64) {
                for (int i = 0; i < nsub; ++i) fill(i);
            } else {
                std::vector<std::thread> pool;
                for (int w = 0; w < nth; ++w)
                    pool.emplace_back([&, w]() {
                        for (int i = w; i < nsub; i += nth) fill(i);
                    });
                for (auto& th : pool) th.join();
            }
            if (bad.load() >= 0)
                return set_error(NDHSS_ERR_INTERNAL, "apply: a B row of node %d lies outside its subtree", bad.load());
            for (int i = 0; i < nsub; ++i) {
                const int r = roots[i];
                sub_lo[r] = F.info(first[r], 4);
                sub_ni[r] = (int)ni[r];
                sub_off[r] = (int)soff[i];
                sub_len[r] = (int)(soff[i + 1] - soff[i]);
                F.sched_vlen = std::max(F.sched_vlen, sub_len[r]);
                F.sched_vlen = std::max(F.sched_vlen, (int)(ni[r] + F.m_b(r) + SUB_XIN + AT));
            }
        }
    }
    F.sched_sub_level = Ls;
    int L_w = F.depth + 1;
    for (int l = std::min(F.depth, Ls - 1); l >= 0 && Ls > F.depth; --l) {
        bool all = true;
        for (int s : F.levels[l]) all = all && tiny(s);
        if (!all) break;
        L_w = l;
    }
    std::vector<int32_t> wdesc;
    std::vector<int64_t> wlev(F.depth + 2, 0);      // first warp-node index of each level
    for (int l = L_w; l <= F.depth; ++l) {
        wlev[l] = (int64_t)wdesc.size() / 8;
        for (int s : F.levels[l]) {
            const uint64_t fo = (uint64_t)F.foff[s];
            const int32_t d[8] = {s, F.m_i(s), F.m_b(s), F.info(s, 4), F.info(s, 6),
                                  (int32_t)(uint32_t)fo, (int32_t)(uint32_t)(fo >> 32), 0};
            wdesc.insert(wdesc.end(), d, d + 8);
            need[CN_UP * nn + s] = 1;
            need[CN_DIAG * nn + s] = 1;
            need[CN_FIN * nn + s] = 1;
        }
    }
    auto push_w = [&](int kind, int l) {
        const int cnt = (int)F.levels[l].size();
        for (int j = 0; j < cnt; j += AW) {
            const int64_t base = wlev[l] + j;
            const int32_t w[QW] = {(kind << TK_SHIFT) | F.levels[l][j], std::min(AW, cnt - j), l, 0, 0, 0, 0, 0,
                                   (int32_t)(uint32_t)(uint64_t)base, (int32_t)(uint32_t)((uint64_t)base >> 32), 0, 0};
            q.insert(q.end(), w, w + QW);
        }
    };
    auto ulv_front = [&](int s) { return !F.ulv_root_of.empty() && F.ulv_root_of[s] >= 0; };
    const int ng = ceil_div(F.n, GATHER_CHUNK);
    for (int i = 0; i < ng; ++i) push(TK_GATHER, 0, i * GATHER_CHUNK, GATHER_CHUNK, false);
    cut();
    auto push_sub = [&](int kind, int r) {
        const int32_t w[QW] = {(kind << TK_SHIFT) | r, sub_lo[r], sub_ni[r], F.m_i(r), F.m_b(r),
                               F.info(r, 4), F.info(r, 6), sub_len[r], 0, 0, sub_off[r], 0};
        q.insert(q.end(), w, w + QW);
    };
    if (Ls <= F.depth) {
        for (int r : F.levels[Ls]) {
            push_sub(TK_SUBUP, r);
            need[CN_UP * nn + r] = 1;
        }
        cut();
    }
    for (int l = F.depth; l >= L_w; --l) {
        push_w(TK_UPW, l);
        cut();
    }
    // The diagonal step of the nodes not fused into their up-sweep tasks:
    // column-chunk partial products, then their sums.  Same dependencies as
    // the node's up-sweep, so they are queued with it: ready together, and the
    // tickets of the up-sweep chain above do not hold them back.
    const int l_top = std::min({F.depth, L_w - 1, Ls - 1});
    auto push_dpart = [&](int l) {
        for (int s : F.levels[l]) {
            const int mi = F.m_i(s);
            if (mi == 0 || fused(s) || ulv_front(s)) continue;
            // the top level's diagonal step lies on the critical path (the down
            // sweep starts from it): narrower chunks, more tasks in parallel
            dcols[s] = l == 0 ? ROOT_DIAG_COLS : DIAG_COLS;
            const int nch = ceil_div(mi, dcols[s]);
            dpoff[s] = F.dpart_total;
            F.dpart_total += (int64_t)nch * mi;
            for (int c0 = 0; c0 < mi; c0 += dcols[s])
                for (int r0 = 0; r0 < mi; r0 += APPLY_ROWS) push(TK_DPART, s, r0, c0, false);
            need[CN_DPART * nn + s] = nch * ceil_div(mi, APPLY_ROWS);
        }
    };
    auto push_dsum = [&](int l) {
        for (int s : F.levels[l]) {
            const int mi = F.m_i(s);
            if (mi == 0 || fused(s) || ulv_front(s)) continue;
            for (int r0 = 0; r0 < mi; r0 += SUM_ROWS) push(TK_DSUM, s, r0, 0, diag_final(s));
            need[CN_DIAG * nn + s] = ceil_div(mi, SUM_ROWS);
            if (diag_final(s)) need[CN_FIN * nn + s] = need[CN_DIAG * nn + s];
        }
    };
    for (int l = l_top; l >= 0; --l) {
        // fused / dense / low-rank-dot tasks of the level, then what completes each node
        for (int s : F.levels[l]) {
            const int mi = F.m_i(s), mb = F.m_b(s);
            if (fused(s)) {
                const int rows = mi + mb, cnt = ceil_div(rows, APPLY_ROWS);
                for (int r0 = 0; r0 < rows; r0 += APPLY_ROWS) push(TK_UPDIAG, s, r0, 0, diag_final(s));
                need[CN_UP * nn + s] = cnt;
                need[CN_DIAG * nn + s] = cnt;
                if (diag_final(s)) need[CN_FIN * nn + s] = cnt;
            } else if (mi > 0 && mb > 0 && mode(s) == 0) {
                for (int j0 = 0; j0 < mb; j0 += APPLY_ROWS) push(TK_UP, s, j0, 0, false);
                need[CN_UP * nn + s] = ceil_div(mb, APPLY_ROWS);
            } else if (mi > 0 && mb > 0 && mode(s) == 1) {
                for (int r0 = 0; r0 < mi; r0 += LR_CHUNK)
                    for (int a0 = 0; a0 < F.lr_k[s]; a0 += dgw) push(TK_UPDOT, s, r0, a0, false);
                need[CN_DOT * nn + s] = ceil_div(mi, LR_CHUNK) * ceil_div(F.lr_k[s], dgw);
            }
        }
        push_dpart(l);
        cut();
        for (int s : F.levels[l]) {
            if (fused(s) || (F.m_i(s) > 0 && F.m_b(s) > 0 && mode(s) == 0)) continue;
            if (F.m_i(s) > 0 && F.m_b(s) > 0 && mode(s) == 1) {
                for (int r0 = 0; r0 < F.m_b(s); r0 += APPLY_ROWS) push(TK_UPAXPY, s, r0, 0, false);
                need[CN_UP * nn + s] = ceil_div(F.m_b(s), APPLY_ROWS);
            } else if (F.info(s, 1) >= 0) {
                push(TK_UPNOP, s, 0, 0, false);
                need[CN_UP * nn + s] = 1;
            }
        }
        push_dsum(l);
        cut();
    }
    // ULV solves of the HSS fronts: every front's HSS nodes going up (deepest
    // HSS level first), the roots, then down; the leaves (or a root that is
    // a leaf) write z(I^s)
    std::vector<UlvDev> udev(std::max(nrec, 1));
    F.ulv_scratch = 0;
    int ulv_maxlev = 0;
    for (int i = 0; i < nrec; ++i) {
        const FactorData::UlvRec& r = F.ulv_recs[i];
        UlvDev& d = udev[i];
        d.s = r.s; d.lo = r.lo; d.hi = r.hi; d.m = r.m; d.k = r.k; d.ne = r.ne; d.kt = r.kt; d.ka = r.ka; d.kb = r.kb;
        d.parent = r.parent; d.c1 = r.c1; d.c2 = r.c2; d.leaf = r.leaf; d.root = r.root; d.i_off = F.info(r.s, 4);
        d.pad = 0;
        d.ord_off = F.ulv_ord_off[r.s];
        auto slot = [&](int64_t c) { const int64_t o = F.ulv_scratch; F.ulv_scratch += std::max<int64_t>(c, 1); return o; };
        d.o_y1 = slot(r.ne);
        d.o_rh = slot(r.kt);
        d.o_g = slot(r.k);
        d.o_x2 = slot(r.kt);
        d.Mup = r.Mup; d.W = r.W; d.Mm = r.Mm; d.E = r.E; d.Dinv = r.Dinv;
        ulv_maxlev = std::max(ulv_maxlev, r.level);
        F.sched_vlen = std::max(F.sched_vlen, r.m + r.ka + r.kb);
        need[NCNT * nn + i] = 1;
        need[NCNT * nn + nrec + i] = 1;
        if (r.leaf) {
            need[CN_DIAG * nn + r.s] += 1;
            if (diag_final(r.s)) need[CN_FIN * nn + r.s] += 1;
        }
    }
    auto push_u = [&](int kind, int i) {
        const FactorData::UlvRec& r = F.ulv_recs[i];
        const bool writes = r.leaf && kind != TK_HUP;
        const int32_t w[QW] = {((writes && diag_final(r.s)) ? TK_FINAL : 0) | (kind << TK_SHIFT) | i, r.s, r.level,
                               r.c1, r.c2, r.parent, (r.leaf ? 1 : 0) | (r.root ? 2 : 0), 0, 0, 0, 0, 0};
        q.insert(q.end(), w, w + QW);
    };
    for (int lv = ulv_maxlev; lv >= 1; --lv) {
        for (int i = 0; i < nrec; ++i)
            if (F.ulv_recs[i].level == lv && !F.ulv_recs[i].root) push_u(TK_HUP, i);
        cut();
    }
    for (int i = 0; i < nrec; ++i)
        if (F.ulv_recs[i].root) push_u(TK_HROOT, i);
    cut();
    for (int lv = 1; lv <= ulv_maxlev; ++lv) {
        for (int i = 0; i < nrec; ++i)
            if (F.ulv_recs[i].level == lv) push_u(TK_HDN, i);
        cut();
    }
    for (int l = 0; l < std::min(L_w, Ls); ++l) {
        for (int s : F.levels[l]) {
            if (F.m_i(s) == 0 || diag_final(s) || mode(s) != 1) continue;
            for (int r0 = 0; r0 < F.m_b(s); r0 += LR_CHUNK)
                for (int a0 = 0; a0 < F.lr_k[s]; a0 += dgw) push(TK_DNDOT, s, r0, a0, false);
            need[CN_DDOT * nn + s] = ceil_div(F.m_b(s), LR_CHUNK) * ceil_div(F.lr_k[s], dgw);
        }
        cut();
        for (int s : F.levels[l]) {
            if (F.m_i(s) == 0) {
                push(TK_FINNOP, s, 0, 0, false);
                need[CN_FIN * nn + s] = 1;
                continue;
            }
            if (diag_final(s)) continue;
            if (mode(s) == 0) {
                for (int i0 = 0; i0 < F.m_i(s); i0 += APPLY_ROWS) push(TK_DN, s, i0, 0, true);
            } else {
                for (int r0 = 0; r0 < F.m_i(s); r0 += APPLY_ROWS) push(TK_DNAXPY, s, r0, 0, true);
            }
            need[CN_FIN * nn + s] = ceil_div(F.m_i(s), APPLY_ROWS);
        }
        cut();
    }
    for (int l = L_w; l <= F.depth; ++l) {
        push_w(TK_DNW, l);
        cut();
    }
    if (Ls <= F.depth) {
        for (int r : F.levels[Ls]) push_sub(TK_SUBDN, r);
        cut();
    }
    F.sched_n = (int64_t)q.size() / QW;
    F.sched_ngather = ng;
    F.sched_groups = groups;
    F.sched_vlen = std::max(F.sched_vlen, std::max(std::max(F.max_mi, F.max_mb), LR_CHUNK));
    if (L_w <= F.depth) F.sched_vlen = std::max(F.sched_vlen, AW * WREG);
    F.sched_warp_level = L_w;
    if (F.sched_n >= (int64_t)INT32_MAX / QW) return set_error(NDHSS_ERR_INVALID_ARG, "apply: task queue too long");
    ndhss_status rc = NDHSS_OK;
    auto up = [&](auto** dst, const auto& v) {
        if (rc != NDHSS_OK) return;
        const size_t bytes = v.size() * sizeof(v[0]);
        if (pool_malloc_async((void**)dst, std::max<size_t>(bytes, 8), st) != cudaSuccess ||
            cudaMemcpyAsync(*dst, v.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(NDHSS_ERR_OOM, "apply: schedule tables");
            return;
        }
        F.dev_bytes += (int64_t)bytes;
    };
    up(&F.d_sched, q);
    up(&F.d_need, need);
    up(&F.d_wdesc, wdesc);
    up(&F.d_sublist, sublist);
    if (nrec) {
        if (pool_malloc_async(&F.d_ulvdev, udev.size() * sizeof(UlvDev), st) != cudaSuccess ||
            cudaMemcpyAsync(F.d_ulvdev, udev.data(), udev.size() * sizeof(UlvDev), cudaMemcpyHostToDevice, st) !=
                cudaSuccess) {
            cudaGetLastError();
            rc = set_error(NDHSS_ERR_OOM, "apply: ULV records");
        }
    }
    if (rc == NDHSS_OK && (pool_malloc_async((void**)&F.d_apply_err, sizeof(int32_t), st) != cudaSuccess ||
                           cudaMemsetAsync(F.d_apply_err, 0, sizeof(int32_t), st) != cudaSuccess)) {
        cudaGetLastError();
        rc = set_error(NDHSS_ERR_OOM, "apply: error word");
    }
    if (rc == NDHSS_OK && F.sched_n > 0) {
        if (pool_malloc_async((void**)&F.d_sched_dep, sizeof(int4) * 2 * (size_t)F.sched_n, st) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(NDHSS_ERR_OOM, "apply: dependency records");
        } else {
            F.dev_bytes += (int64_t)(sizeof(int4) * 2 * F.sched_n);
            rc = fill_sched_deps(F, st);
        }
    }
    if (rc != NDHSS_OK) return rc;
    const bool cplx = F.vtype == NDHSS_C128;
    if (!cplx && F.prec == NDHSS_FP64) return launch_shape<double, double>(F);
    if (!cplx) return launch_shape<float, double>(F);
    if (F.prec == NDHSS_FP64) return launch_shape<c128, c128>(F);
    return launch_shape<c64, c128>(F);
}

// Sticky failure of an earlier asynchronous apply (a bounded wait gave up).
ndhss_status apply_check_error(const FactorData& F, const char* who) {
    if (!F.d_apply_err) return NDHSS_OK;
    int32_t e = 0;
    NDHSS_CUDA_TRY(cudaMemcpy(&e, F.d_apply_err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) return set_error(NDHSS_ERR_TIMEOUT, "%s: a wait of the persistent apply kernel gave up after %.1f s",
                            who, APPLY_WAIT_NS * 1e-9);
    return NDHSS_OK;
}

size_t apply_work_bytes(const FactorData& F) { return work_layout(F).total; }

ndhss_status apply_device(const FactorData& F, int32_t nrhs, const void* d_x, int64_t ldx, void* d_y, int64_t ldy,
                          void* d_work, cudaStream_t st, const ApplyInd* ind) {
    const bool cplx = F.vtype == NDHSS_C128;
    unsigned char* w = static_cast<unsigned char*>(d_work);
    if (!cplx && F.prec == NDHSS_FP64)
        return apply_run<double, double>(F, nrhs, (const double*)d_x, ldx, (double*)d_y, ldy, w, st, ind);
    if (!cplx)
        return apply_run<float, double>(F, nrhs, (const double*)d_x, ldx, (double*)d_y, ldy, w, st, ind);
    if (F.prec == NDHSS_FP64)
        return apply_run<c128, c128>(F, nrhs, (const c128*)d_x, ldx, (c128*)d_y, ldy, w, st, ind);
    return apply_run<c64, c128>(F, nrhs, (const c128*)d_x, ldx, (c128*)d_y, ldy, w, st, ind);
}

}  // namespace ndhss

extern "C" ndhss_status ndhss_apply(const ndhss_factorization* fh, int32_t nrhs, const void* x, int64_t ldx, void* y,
                                    int64_t ldy, void* stream) {
    return ::ndhss::guarded("ndhss_apply", [&]() -> ndhss_status {
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
        NDHSS_CUDA_TRY(pool_malloc_async(&work, wb, st));
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
            if (rc == NDHSS_OK) rc = apply_check_error(F, "ndhss_apply");
        }
        return rc;
    });
}

// --------------------------------------------------------------------------
// Allocation-free apply (no counterpart in the paper).
//
// Some callers cannot allocate device memory at the moment they need P^{-1}:
// a solver loop in a process whose device memory is reserved up front by
// another allocator (a framework's caching allocator, a fixed budget), or
// code under a no-allocation-after-setup rule, where an allocation can fail
// or stall.  They get the same Alg. 3.1 result with the work area in this
// fixed static array instead of stream-ordered allocations.  The array is
// part of the module image, so every device that loads the library holds it
// until exit.  Host code must not take its address directly (that would be a
// host-side shadow): the device address is looked up once per device with
// cudaGetSymbolAddress, and again if the device's context was replaced (a
// device reset reloads the module, possibly at another address).  Every call
// writes the work area before reading it (the gather all of the first
// vector, the diagonal step all of the second, the low-rank tasks their
// partial-product slots, an asynchronous memset the queue's control words),
// so nothing needs clearing between calls; overlapping calls race on the
// array.
namespace ndhss {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;
__device__ __align__(256) unsigned char g_apply_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_scratch_mu;
struct ScratchAddr {
    unsigned long long ctx_id = 0;       // context the address was looked up in
    void* addr = nullptr;
};
ScratchAddr g_scratch_addr[NOALLOC_MAX_DEVICES];

ndhss_status scratch_for_current_device(void** out) {
    int dev = -1;
    NDHSS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_apply_noalloc: device %d beyond the supported %d", dev,
                         NOALLOC_MAX_DEVICES);
    // cudaGetSymbolAddress also makes the device's primary context current
    // if no context was, so the id is read after it on a first lookup
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchAddr& a = g_scratch_addr[dev];
    unsigned long long id = 0;
    if (a.addr) {
        const ndhss_status rc = drv_current_ctx_id(&id);
        if (rc != NDHSS_OK) return rc;
        if (id == a.ctx_id) {
            *out = a.addr;
            return NDHSS_OK;
        }
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
    if (e != cudaSuccess || !p)
        return set_error(NDHSS_ERR_CUDA, "ndhss_apply_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                         cudaGetErrorString(e));
    const ndhss_status rc = drv_current_ctx_id(&id);
    if (rc != NDHSS_OK) return rc;
    a.addr = p;
    a.ctx_id = id;
    *out = p;
    return NDHSS_OK;
}

}  // namespace
}  // namespace ndhss

extern "C" ndhss_status ndhss_apply_noalloc(const ndhss_factorization* fh, const void* d_x, void* d_y, void* stream) {
    return ::ndhss::guarded("ndhss_apply_noalloc", [&]() -> ndhss_status {
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
    });
}

// Failure-detection hook: one requirement that no task will ever satisfy.
extern "C" ndhss_status ndhss_testing_stall_apply(ndhss_factorization* fh) {
    return ::ndhss::guarded("ndhss_testing_stall_apply", [&]() -> ndhss_status {
        using namespace ndhss;
        clear_error();
        if (!fh || !fh->f.d_need || fh->f.levels.empty() || fh->f.levels[0].empty())
            return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_testing_stall_apply: no dataflow queue");
        FactorData& F = fh->f;
        const int root = F.levels[0][0];
        int32_t* p = F.d_need + (size_t)CN_FIN * F.nnodes + root;
        int32_t v = 0;
        NDHSS_CUDA_TRY(cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost));
        ++v;
        NDHSS_CUDA_TRY(cudaMemcpy(p, &v, sizeof(v), cudaMemcpyHostToDevice));
        const ndhss_status rc = fill_sched_deps(F, 0);
        if (rc != NDHSS_OK) return rc;
        NDHSS_CUDA_TRY(cudaDeviceSynchronize());
        return NDHSS_OK;
    });
}
