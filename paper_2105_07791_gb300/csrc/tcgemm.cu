// The rank-128 block exchanges of the Gauss-Jordan sweep of the dense
// fronts on the tensor cores: tcgen05 MMAs with operands staged by TMA
// (cp.async.bulk.tensor) and the accumulator in tensor memory (Sec. 3.1,
// Eq. 3.3 - 3.5).
//
// The sweep of factor.cu eliminates the interior unknowns of a front M in
// outer blocks of TC_KB2 = 128 pivots.  Inside a block, rank-kb exchange
// steps touch only the block's own columns Q (its slab, all rows), and the
// row interchanges go to every column.  After that the slab holds the
// exchanged values  M'(P, Q) = M(P, Q)^{-1},  M'(o, Q) = M(o, Q) M(P, Q)^{-1}
// (P the block's pivot rows, o every other row), and the block exchange of
// every column j outside the slab is
//
//      M'(:, j) = beta .* M(:, j) + M'(:, Q) (-M(P, j)),   beta = 0 on rows P,
//
// one GEMM with K = |Q| over the whole front per outer block: the same
// exchanges as the rank-kb sweep, composed (S = A_bb - A_bi A_ii^{-1} A_ib
// stays the elimination's Schur complement).  Complex products are real
// GEMMs: the A operand row i becomes the real rows 2i = [Re, -Im] and
// 2i + 1 = [Im, Re] over the K pairs (2q, 2q + 1), the B operand keeps
// (Re, Im) interleaved along K, so one real accumulator holds Re in even rows
// and Im in odd rows.
//
// Precision.  Every operand is split into parts that the tensor core takes
// exactly (rounded to nearest), v = hi + lo with hi = rn(v), lo = rn(v - hi),
// and a product is formed as hi*hi + (hi*lo + lo*hi) in FP32 (the split of
// Ootomo & Yokota 2022 for TF32; Henry, Tang & Heinecke 2019 for BF16): with
// TF32 parts (10 + 1 mantissa bits each) ~22 bits, the accuracy of an FP32
// product (NDHSS_FP32).  NDHSS_FP32_BF16 splits into three BF16 parts
// (hi, mid, lo; 8 bits each) and forms the six products whose part indices
// sum to at most 2, again ~22-24 bits; NDHSS_FP32_TF32 takes one rounded
// TF32 part (11 bits).  As Ootomo & Yokota
// recommend, the correction terms accumulate in their own tensor-memory
// accumulator; every TC_CHUNK K-stages the MMA issuer switches to a second
// accumulator pair while eight warps add the finished pair into FP32
// registers (round to nearest), so no sum runs long inside the tensor core.
//
// Data flow per outer block: a pack kernel writes both operands K-major into
// one packed array (K padded with zeros to Kp); one 2D tensor map with
// 128-byte swizzle covers it; the GEMM kernel runs one 128 x 128 output tile
// per CTA: a producer thread issues the TMA loads of a 3- or 5-stage ring,
// one thread issues the MMAs (four K-steps of 32 bytes per 128-byte swizzle
// row, up to three products each) and commits each stage back to the
// producer, and the accumulating warps store the tile.  Every wait on an
// mbarrier is bounded (2 s of %globaltimer); a wait that gives up sets a
// TIMEOUT status and the CTA leaves after its copies and MMAs have landed.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "driver.h"
#include "factor.cuh"
#include "tcgen05.cuh"

namespace ndhss {
namespace {

constexpr int TC_TILE = 128;                  // output tile rows (real) and columns
constexpr int TC_THREADS = 320;                // warps 0-7 accumulate and store, 8 loads, 9 issues MMAs
constexpr int TC_PRODUCER = 256, TC_ISSUER = 288;
constexpr int TC_HALF = TC_TILE / 2;           // columns per accumulating warp (warps w and w + 4 share lanes)
constexpr int TC_CHUNK = 2;                    // K stages per tensor-memory accumulation chunk
constexpr uint32_t TC_TILE_BYTES = 128u * 128u;   // 128 rows x one 128-byte swizzle row
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

// One front's part of an outer block: the slab's width w (pivots
// [k0, k0 + w)), the first packed row row0 of its operands (A: cx m rows per
// part, then B: m - w rows per part).
struct TcFront {
    int64_t foff, row0;
    int32_t m, w;
};

// The block exchange of one front: C = A B (real rows of A = M, rows of B =
// N = columns outside the slab, real K), column c of the product is front
// column c (c < k0) or c + w, rows [k0, k0 + w) of the front are overwritten,
// the others accumulated.
struct TcJob {
    int32_t a_row, a_pstride, b_row, b_pstride;
    int32_t M, N, K, k0;
    int64_t out;                 // front element offset of the front's (0, 0)
    int32_t ldo, w, pad0, pad1;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity; false when TC_WAIT_NS passed.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = tc::smem_u32(bar);
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0) {
            const unsigned long long t = globaltimer();
            if (it == 0) t0 = t;
            else if (t - t0 > TC_WAIT_NS) return false;
        }
    }
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tc::smem_u32(bar))
        : "memory");
}

// K-major operand tile with 128-byte swizzle: 8-row groups 1024 bytes apart
// (stride byte offset), the leading byte offset unused, layout type 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = __uint_as_float(r[u]);
}

// the parts of a value in the packed element type (rounded to nearest)
template <int ESZ> struct Part;
template <> struct Part<4> {
    using E = uint32_t;
    static __device__ __forceinline__ E hi(float v, float& rest) {
        const uint32_t h = tc::to_tf32_rn(v);
        rest = v - __uint_as_float(h);
        return h;
    }
    static __device__ __forceinline__ E last(float v) { return tc::to_tf32_rn(v); }
};
template <> struct Part<2> {
    using E = __nv_bfloat16;
    static __device__ __forceinline__ E hi(float v, float& rest) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        rest = v - __bfloat162float(h);
        return h;
    }
    static __device__ __forceinline__ E last(float v) { return __float2bfloat16_rn(v); }
};

// write the NS parts of v at rows row, row + pstride, ... (column k)
template <int ESZ, int NS>
__device__ __forceinline__ void put_parts(typename Part<ESZ>::E* packed, int64_t Kp, int64_t row, int64_t pstride,
                                          int64_t k, float v) {
    float rest = v;
#pragma unroll
    for (int p = 0; p + 1 < NS; ++p) {
        float r;
        packed[(row + p * pstride) * Kp + k] = Part<ESZ>::hi(rest, r);
        rest = r;
    }
    packed[(row + (NS - 1) * pstride) * Kp + k] = Part<ESZ>::last(rest);
}

// ---------------------------------------------------------------- pack
// One CTA per (32 logical rows x 32 complex K columns) tile of one operand of
// one front (blockIdx.y = front).  Row tiles: first the A operand (the
// slab, rows i < m: M'(i, k0 + q)), then the B operand (row r = output
// column r (< k0) or r + w: -M(k0 + q, column)).  K columns beyond the
// slab's width are written as zeros up to Kp.
template <typename T, int ESZ, int NS>
__global__ void __launch_bounds__(256)
tc_pack_kernel(const TcFront* __restrict__ fronts, const T* __restrict__ front, int k0, void* __restrict__ packed_v,
               int64_t Kp) {
    constexpr bool CPLX = Tr<T>::cplx;
    constexpr int CX = CPLX ? 2 : 1;
    using E = typename Part<ESZ>::E;
    __shared__ T ts[32][33];
    const TcFront P = fronts[blockIdx.y];
    const int m = P.m, w = P.w, nb = m - w;
    const int LT = (int)(Kp / CX / 32);
    const int rt_a = (m + 31) / 32, rt_b = (nb + 31) / 32;
    if ((int)blockIdx.x >= (rt_a + rt_b) * LT) return;
    const int lt = blockIdx.x % LT;
    int rt = blockIdx.x / LT;
    const bool is_a = rt < rt_a;
    if (!is_a) rt -= rt_a;
    const int rows = is_a ? m : nb;
    const int r0 = rt * 32, l0 = lt * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const T* F = front + P.foff;
    // the slab is contiguous along its rows, -M(P, j) along K
    if (is_a) {
        for (int ll = ty; ll < 32; ll += 8) {
            const int r = r0 + tx, l = l0 + ll;
            ts[tx][ll] = (r < rows && l < w) ? F[(int64_t)(k0 + l) * m + r] : zero<T>();
        }
    } else {
        for (int rr = ty; rr < 32; rr += 8) {
            const int r = r0 + rr, l = l0 + tx;
            const int64_t j = r < k0 ? r : r + w;
            ts[rr][tx] = (r < rows && l < w) ? -F[j * m + k0 + l] : zero<T>();
        }
    }
    __syncthreads();
    E* packed = static_cast<E*>(packed_v);
    const int64_t a_rows = (int64_t)CX * m;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr;
        if (r >= rows) continue;
        const int64_t l = l0 + tx;
        const T v = ts[rr][tx];
        if (is_a) {
            if constexpr (CPLX) {
                put_parts<ESZ, NS>(packed, Kp, P.row0 + 2 * r, a_rows, 2 * l, v.x);
                put_parts<ESZ, NS>(packed, Kp, P.row0 + 2 * r, a_rows, 2 * l + 1, -v.y);
                put_parts<ESZ, NS>(packed, Kp, P.row0 + 2 * r + 1, a_rows, 2 * l, v.y);
                put_parts<ESZ, NS>(packed, Kp, P.row0 + 2 * r + 1, a_rows, 2 * l + 1, v.x);
            } else {
                put_parts<ESZ, NS>(packed, Kp, P.row0 + r, a_rows, l, v);
            }
        } else {
            const int64_t brow = P.row0 + NS * a_rows + r;
            if constexpr (CPLX) {
                put_parts<ESZ, NS>(packed, Kp, brow, nb, 2 * l, v.x);
                put_parts<ESZ, NS>(packed, Kp, brow, nb, 2 * l + 1, v.y);
            } else {
                put_parts<ESZ, NS>(packed, Kp, brow, nb, l, v);
            }
        }
    }
}

// ---------------------------------------------------------------- GEMM
template <int NS> struct Stages { static constexpr int value = NS == 3 ? 2 : (NS == 2 ? 3 : 5); };

// The products of a K-step (part of A, part of B): all pairs whose part
// indices sum to at most NS - 1, largest first; (0, 0) goes to the main
// accumulator, the rest to the correction accumulator.
template <int NS> struct Products { static constexpr int n = NS * (NS + 1) / 2; };
__host__ __device__ constexpr int prod_a(int q) { return q < 3 ? (q == 2 ? 1 : 0) : (q == 3 ? 0 : (q == 4 ? 1 : 2)); }
__host__ __device__ constexpr int prod_b(int q) { return q < 3 ? (q == 1 ? 1 : 0) : (q == 3 ? 2 : (q == 4 ? 1 : 0)); }

template <typename T, int ESZ, int NS>
constexpr size_t tc_gemm_smem() {
    return (size_t)Stages<NS>::value * 2 * NS * TC_TILE_BYTES + 1024;
}

template <typename T, int ESZ, int NS>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmap, const TcJob* __restrict__ jobs, const int2* __restrict__ tiles,
               T* __restrict__ front, DevStatus* status) {
    constexpr bool CPLX = Tr<T>::cplx;
    constexpr int STAGES = Stages<NS>::value;
    constexpr int NP = Products<NS>::n;               // products per K-step
    constexpr int BK = 128 / ESZ;                     // K elements per stage
    constexpr uint32_t STAGE_BYTES = 2u * NS * TC_TILE_BYTES;
    // an accumulator pair: columns 0..127 hi * hi, 128..255 the correction
    // terms (NS > 1); two pairs alternate chunk by chunk
    constexpr uint32_t PAIR_COLS = NS > 1 ? 2 * TC_TILE : TC_TILE;
    constexpr uint32_t TMEM_COLS = 2 * PAIR_COLS;
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t accfull_bar[2];
    __shared__ __align__(8) uint64_t accfree_bar[2];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ int s_abort;

    const int2 tl = tiles[blockIdx.x];
    const TcJob J = jobs[tl.x];
    const int tiles_m = (J.M + TC_TILE - 1) / TC_TILE;
    const int m0 = (tl.y % tiles_m) * TC_TILE, n0 = (tl.y / tiles_m) * TC_TILE;
    const int nk = (J.K + BK - 1) / BK;
    const int nchunk = (nk + TC_CHUNK - 1) / TC_CHUNK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (tc::smem_u32(dsm) + 1023u) & ~1023u;
    auto tileA = [&](int s, int p) { return base + (uint32_t)s * STAGE_BYTES + (uint32_t)p * TC_TILE_BYTES; };
    auto tileB = [&](int s, int p) { return base + (uint32_t)s * STAGE_BYTES + (uint32_t)(NS + p) * TC_TILE_BYTES; };

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full_bar[s], 1);
            tc::mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&accfull_bar[b], 1);
            tc::mbar_init(&accfree_bar[b], 8);         // one arrival per accumulating warp
        }
        tc::mbar_init(&done_bar, 1);
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_holder, TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_holder;

    int issued = 0;                                   // producer: stages loaded
    if (tid == TC_PRODUCER) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !bar_wait(&empty_bar[s], ((kb / STAGES) & 1) ^ 1)) {
                atomicExch(&s_abort, 1);
                break;
            }
            if (*(volatile int*)&s_abort) break;
            bar_expect_tx(&full_bar[s], STAGE_BYTES);
            for (int p = 0; p < NS; ++p) {
                tma_load_2d(tileA(s, p), &tmap, kb * BK, J.a_row + p * J.a_pstride + m0, &full_bar[s]);
                tma_load_2d(tileB(s, p), &tmap, kb * BK, J.b_row + p * J.b_pstride + n0, &full_bar[s]);
            }
            issued = kb + 1;
        }
    } else if (tid == TC_ISSUER) {
        const uint32_t idesc = ESZ == 4 ? tc::idesc_tf32(TC_TILE, TC_TILE) : tc::idesc_bf16(TC_TILE, TC_TILE);
        bool ok = true;
        for (int c = 0; c < nchunk && ok; ++c) {
            const int b = c & 1;
            if (c >= 2 && !bar_wait(&accfree_bar[b], ((c >> 1) & 1) ^ 1)) {
                ok = false;
                break;
            }
            tc::fence_after();
            const uint32_t acc0 = tmem + (uint32_t)b * PAIR_COLS;
            const int kb1 = min(nk, (c + 1) * TC_CHUNK);
            for (int kb = c * TC_CHUNK; kb < kb1; ++kb) {
                const int s = kb % STAGES;
                if (!bar_wait(&full_bar[s], (kb / STAGES) & 1)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const uint64_t ad = sw128_desc(tileA(s, prod_a(q)) + 32u * kk);
                        const uint64_t bd = sw128_desc(tileB(s, prod_b(q)) + 32u * kk);
                        const uint32_t d = q == 0 ? acc0 : acc0 + (uint32_t)TC_TILE;
                        const uint32_t acc = (kb != c * TC_CHUNK || kk != 0 || q >= 2) ? 1u : 0u;
                        if constexpr (ESZ == 4) tc::mma_tf32(d, ad, bd, idesc, acc);
                        else tc::mma_f16(d, ad, bd, idesc, acc);
                    }
                }
                tc::commit(&empty_bar[s]);
            }
            if (ok) tc::commit(&accfull_bar[b]);
        }
        if (!ok) atomicExch(&s_abort, 1);
        tc::commit(&done_bar);                        // fires once every MMA issued above has retired
        bar_wait(&done_bar, 0);
    } else if (warp < 8) {
        // accumulating warps: each finished chunk pair of this thread's TMEM
        // lane (real row m0 + rr of the product) is added into FP32 registers
        // (round to nearest), then handed back to the MMA issuer; warp w takes
        // the lanes 32 (w % 4) .. + 31 and the columns 64 (w / 4) .. + 63
        const int rr = (warp & 3) * 32 + lane;
        const int cb = (warp >> 2) * TC_HALF;
        float sum[TC_HALF];
#pragma unroll
        for (int u = 0; u < TC_HALF; ++u) sum[u] = 0.0f;
        const uint32_t lane_off = ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb;
        bool ok = true;
        for (int c = 0; c < nchunk; ++c) {
            const int b = c & 1;
            if (!bar_wait(&accfull_bar[b], (c >> 1) & 1)) {
                ok = false;
                break;
            }
            tc::fence_after();
            const uint32_t acc0 = tmem + lane_off + (uint32_t)b * PAIR_COLS;
#pragma unroll
            for (int c0 = 0; c0 < TC_HALF; c0 += 16) {
                float v[16];
                tmem_ld16(acc0 + (uint32_t)c0, v);
                if constexpr (NS > 1) {
                    float w[16];
                    tmem_ld16(acc0 + (uint32_t)(TC_TILE + c0), w);
#pragma unroll
                    for (int u = 0; u < 16; ++u) v[u] += w[u];
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) sum[c0 + u] += v[u];
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&accfree_bar[b])) : "memory");
        }
        if (!ok || *(volatile int*)&s_abort) {
            if (lane == 0 && atomicCAS(&status->code, 0, (int)NDHSS_ERR_TIMEOUT) == 0) status->node = -1;
        } else {
            // epilogue from the registers: rows of the block's pivots take the
            // product, the others add it
            const int64_t grow = m0 + rr;
            const bool rowok = grow < J.M;
            T* out = front + J.out;
            if constexpr (CPLX) {
                // even lanes hold Re, odd lanes Im of complex row grow / 2; even
                // lanes write the even columns, odd lanes the odd ones
                const int64_t crow = grow >> 1;
                const bool piv = crow >= J.k0 && crow < J.k0 + J.w;
                const int odd = lane & 1;
                // eight columns at a time: their old values are loaded before any
                // is stored (one load-store pair at a time serialises the latency)
#pragma unroll
                for (int g = 0; g < TC_HALF / 2; g += 8) {
                    T val[8], old[8];
                    T* ptr[8];
#pragma unroll
                    for (int h = 0; h < 8; ++h) {
                        const int u = 2 * (g + h);
                        const float send = odd ? sum[u] : sum[u + 1];
                        const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                        val[h].x = odd ? recv : sum[u];
                        val[h].y = odd ? sum[u + 1] : recv;
                        const int64_t col = n0 + cb + u + odd;
                        const int64_t j = col < J.k0 ? col : col + J.w;
                        ptr[h] = (rowok && col < J.N) ? out + j * J.ldo + crow : nullptr;
                        old[h] = (ptr[h] && !piv) ? *ptr[h] : zero<T>();
                    }
#pragma unroll
                    for (int h = 0; h < 8; ++h)
                        if (ptr[h]) *ptr[h] = old[h] + val[h];
                }
            } else {
                const bool piv = grow >= J.k0 && grow < J.k0 + J.w;
#pragma unroll
                for (int g = 0; g < TC_HALF; g += 8) {
                    float old[8];
                    float* ptr[8];
#pragma unroll
                    for (int h = 0; h < 8; ++h) {
                        const int64_t col = n0 + cb + g + h;
                        const int64_t j = col < J.k0 ? col : col + J.w;
                        ptr[h] = (rowok && col < J.N) ? out + j * J.ldo + grow : nullptr;
                        old[h] = (ptr[h] && !piv) ? *ptr[h] : 0.0f;
                    }
#pragma unroll
                    for (int h = 0; h < 8; ++h)
                        if (ptr[h]) *ptr[h] = old[h] + sum[g + h];
                }
            }
        }
    }
    // leave only once every copy issued by this CTA has landed
    if (tid == TC_PRODUCER) {
        for (int kb = max(0, issued - STAGES); kb < issued; ++kb)
            if (!bar_wait(&full_bar[kb % STAGES], (kb / STAGES) & 1)) break;
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

template <typename T, int ESZ, int NS>
ndhss_status tc_block_run(FactorData& F, const std::vector<int>& nodes, int k0, DevStatus* d_status, cudaStream_t st) {
    constexpr int CX = Tr<T>::cplx ? 2 : 1;
    constexpr int BK = 128 / ESZ;
    const int64_t Kp = ((int64_t)CX * TC_KB2 + 63) / 64 * 64;
    std::vector<TcFront> fr;
    std::vector<TcJob> jobs;
    std::vector<int2> tiles;
    int64_t rows = 0;
    int rt_max = 0;
    for (int s : nodes) {
        const int mi = F.m_i(s), m = mi + F.m_b(s);
        if (mi <= k0) continue;
        const int w = std::min(TC_KB2, mi - k0);
        if (m - w == 0) continue;                      // the slab is the whole front
        const TcFront f{F.foff[s], rows, m, w};
        const int64_t a_rows = (int64_t)CX * m;
        const TcJob j{(int32_t)rows, (int32_t)a_rows, (int32_t)(rows + NS * a_rows), m - w,
                      (int32_t)a_rows, m - w, CX * w, k0, F.foff[s], m, w, 0, 0};
        rows += NS * (a_rows + (m - w));
        const int id = (int)jobs.size();
        jobs.push_back(j);
        fr.push_back(f);
        const int nt = ((j.M + TC_TILE - 1) / TC_TILE) * ((j.N + TC_TILE - 1) / TC_TILE);
        for (int q = 0; q < nt; ++q) tiles.push_back(make_int2(id, q));
        rt_max = std::max(rt_max, (m + 31) / 32 + (m - w + 31) / 32);
    }
    if (fr.empty()) return NDHSS_OK;
    if (rows >= ((int64_t)1 << 31) - TC_TILE)
        return set_error(NDHSS_ERR_INVALID_ARG, "ndhss_factor: %lld packed operand rows exceed the tensor map's range",
                         (long long)rows);
    // one pool allocation: packed operands, then the tables
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t packed_bytes = r256((size_t)rows * Kp * ESZ);
    const size_t fr_bytes = r256(fr.size() * sizeof(TcFront)), job_bytes = r256(jobs.size() * sizeof(TcJob));
    const size_t t_bytes = r256(tiles.size() * sizeof(int2));
    unsigned char* buf = nullptr;
    if (pool_malloc_async((void**)&buf, packed_bytes + fr_bytes + job_bytes + t_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(NDHSS_ERR_OOM, "ndhss_factor: %zu bytes of packed tensor-core operands", packed_bytes);
    }
    TcFront* d_fr = reinterpret_cast<TcFront*>(buf + packed_bytes);
    TcJob* d_jobs = reinterpret_cast<TcJob*>(buf + packed_bytes + fr_bytes);
    int2* d_t = reinterpret_cast<int2*>(buf + packed_bytes + fr_bytes + job_bytes);
    ndhss_status rc = NDHSS_OK;
    auto cp = [&](void* dst, const void* src, size_t b) {
        if (rc == NDHSS_OK && cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = set_error(NDHSS_ERR_CUDA, "ndhss_factor: upload of the tensor-core tables failed");
    };
    cp(d_fr, fr.data(), fr.size() * sizeof(TcFront));
    cp(d_jobs, jobs.data(), jobs.size() * sizeof(TcJob));
    cp(d_t, tiles.data(), tiles.size() * sizeof(int2));
    CUtensorMap tmap;
    if (rc == NDHSS_OK) {
        const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
        const cuuint64_t strides[1] = {(cuuint64_t)Kp * ESZ};
        const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)TC_TILE};
        const cuuint32_t estr[2] = {1, 1};
        rc = drv_encode_tiled(&tmap, ESZ == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                              buf, dims, strides, box, estr, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (rc == NDHSS_OK) {
        const int LT = (int)(Kp / CX / 32);
        tc_pack_kernel<T, ESZ, NS><<<dim3((unsigned)(rt_max * LT), (unsigned)fr.size()), 256, 0, st>>>(
            d_fr, static_cast<const T*>(F.d_front), k0, buf, Kp);
        cudaError_t e = cudaGetLastError();
        note_launches(1);
        if (e != cudaSuccess) rc = set_error(NDHSS_ERR_CUDA, "launch of tc_pack_kernel failed: %s", cudaGetErrorString(e));
    }
    if (rc == NDHSS_OK) {
        tc_gemm_kernel<T, ESZ, NS><<<(unsigned)tiles.size(), TC_THREADS, tc_gemm_smem<T, ESZ, NS>(), st>>>(
            tmap, d_jobs, d_t, static_cast<T*>(F.d_front), d_status);
        cudaError_t e = cudaGetLastError();
        note_launches(1);
        if (e != cudaSuccess) rc = set_error(NDHSS_ERR_CUDA, "launch of tc_gemm_kernel failed: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(buf, st);
    if (rc == NDHSS_OK) {
        F.launches += 2;
        for (const auto& f : fr) F.tc_flops += (Tr<T>::cplx ? 8.0 : 2.0) * (double)f.m * (double)(f.m - f.w) * f.w;
    }
    return rc;
}

template <typename T, int ESZ, int NS>
ndhss_status tc_attrs() {
    NDHSS_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<T, ESZ, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tc_gemm_smem<T, ESZ, NS>()));
    return NDHSS_OK;
}

template <typename T>
ndhss_status tc_block_t(FactorData& F, const std::vector<int>& nodes, int k0, DevStatus* d_status, cudaStream_t st) {
    ndhss_status rc;
    switch (F.prec) {
        case NDHSS_FP32_TF32:
            if ((rc = tc_attrs<T, 4, 1>()) != NDHSS_OK) return rc;
            return tc_block_run<T, 4, 1>(F, nodes, k0, d_status, st);
        case NDHSS_FP32_BF16:
            if ((rc = tc_attrs<T, 2, 3>()) != NDHSS_OK) return rc;
            return tc_block_run<T, 2, 3>(F, nodes, k0, d_status, st);
        default:
            if ((rc = tc_attrs<T, 4, 2>()) != NDHSS_OK) return rc;
            return tc_block_run<T, 4, 2>(F, nodes, k0, d_status, st);
    }
}

}  // namespace

bool tc_front_path(const FactorData& F, int64_t mi_max) {
    // NDHSS_TC_MIN_MI: smallest largest-interior-block of a level that takes
    // the two-level sweep (default 96; smaller fronts leave the blocks and
    // 128 x 128 tiles mostly empty); NDHSS_FRONT_UPDATE=simt keeps every
    // level on the rank-kb sweep over whole fronts (CUDA cores; a cross-check)
    if (F.prec == NDHSS_FP64) return false;
    const char* u = std::getenv("NDHSS_FRONT_UPDATE");
    if (u && std::strcmp(u, "simt") == 0) return false;
    const char* e = std::getenv("NDHSS_TC_MIN_MI");
    const int min_mi = e ? std::atoi(e) : 96;
    return min_mi > 0 && mi_max >= min_mi;
}

ndhss_status tc_block_exchange(FactorData& F, const std::vector<int>& nodes, int k0, DevStatus* d_status,
                               cudaStream_t st) {
    if (F.vtype == NDHSS_C128) return tc_block_t<c64>(F, nodes, k0, d_status, st);
    return tc_block_t<float>(F, nodes, k0, d_status, st);
}

}  // namespace ndhss
