// qsim_tcgen05.cuh -- small building blocks for tcgen05 (5th-generation tensor core) MMAs with
// fp16 operands in shared memory and FP32 accumulators in tensor memory, used by the
// learner's tensor-core forward pass.
//
// Operand layout: the canonical no-swizzle K-major layout -- 8-row x 16-byte core matrices
// (8 halves along K), K-adjacent core matrices 128 B apart (leading byte offset), 8-row
// groups kc * 128 B apart (stride byte offset), kc = K / 8.
// FP32 accuracy from fp16 tensor cores: every operand x is held as x_hi = fp16(x) and
// x_lo = fp16(x - x_hi), and A W ~ A_hi W_hi + A_hi W_lo + A_lo W_hi, accumulated in FP32
// (the dropped A_lo W_lo and the rounding of the lo halves are ~2^-22 relative).
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

namespace qsim {
namespace tc {

// element (r, k) of a canonical K-major 16-bit operand with kc core-matrix columns
__device__ __forceinline__ int cano16(int r, int k, int kc) {
    return ((r >> 3) * kc + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle, K-major: LBO = 128 B, SBO = kc * 128 B
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, int kc) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(((uint32_t)kc * 128u) >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D f32, A and B f16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_f16(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits (bounded) for the phase of `bar` with the given parity; false when it gave up.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes; the wait sits in the
// same asm statement so that no use of the registers is scheduled before it.
__device__ __forceinline__ void ld16(uint32_t ta, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta) : "memory");
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

// Split a pair into packed hi and lo halves.
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 f = __half22float2(h);
    hi = h2u(h);
    lo = h2u(__floats2half2_rn(x0 - f.x, x1 - f.y));
}

}  // namespace tc
}  // namespace qsim
