// Blackwell (sm_100 family) tensor-core primitives as inline PTX: tcgen05 MMA
// with operands in shared memory and the accumulator in tensor memory (TMEM).
//
// Operand layout (K-major, no swizzle): an R x K tile of 32-bit elements is
// stored as "core matrices" of 8 rows x 16 bytes (128 contiguous bytes, row r
// at r * 16); core (r / 8, k / 4) sits at ((r / 8) * (K / 4) + k / 4) * 128.
// The shared-memory descriptor then has leading byte offset 128 (the next
// core along K) and stride byte offset (K / 4) * 128 (the next 8 rows); one
// kind::tf32 MMA consumes K = 8, i.e. the start address advances by 256
// bytes per step.  The accumulator of an M = 128 MMA (cta_group::1) holds row
// i in TMEM lane i, column j in TMEM column base + j (32-bit each).
#pragma once

#include <cstdint>

namespace ndhss {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a K-major tile of K 32-bit columns
__device__ __forceinline__ uint32_t core_off(int r, int k, int K) {
    return ((uint32_t)(r >> 3) * (uint32_t)(K >> 2) + (uint32_t)(k >> 2)) * 128u + (uint32_t)(r & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;             // descriptor version of the tcgen05 family
    return d;                           // base offset 0, no swizzle
}

// instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// FP32 -> TF32 bit pattern, rounded to nearest (ties away from zero)
__device__ __forceinline__ uint32_t to_tf32_rn(float v) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
    return u;
}

// instruction descriptor, kind::f16 with BF16 A and B (both operands of one
// MMA share the type), FP32 accumulator, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (r, k) in a K-major tile of K 16-bit columns: core
// matrices of 8 rows x 8 elements (16 bytes), LBO 128 (along K), SBO (K / 8) * 128
__device__ __forceinline__ uint32_t core_off16(int r, int k, int K) {
    return ((uint32_t)(r >> 3) * (uint32_t)(K >> 3) + (uint32_t)(k >> 3)) * 128u + (uint32_t)(r & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// one kind::f16 MMA (K = 16 for 16-bit operands: the start addresses advance 256 bytes per step)
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

// whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// generic-proxy shared-memory writes become visible to the MMA (async proxy)
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Bounded wait for the given phase parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int max_iter) {
    uint32_t done = 0;
    for (int it = 0; it < max_iter && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity));
    }
    return done != 0;
}

// eight consecutive 32-bit columns of this thread's TMEM lane (warp w reads
// lanes 32 w .. 32 w + 31: taddr carries the lane offset in bits 16..31)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __uint_as_float(r[u]);
}

}  // namespace tc
}  // namespace ndhss
