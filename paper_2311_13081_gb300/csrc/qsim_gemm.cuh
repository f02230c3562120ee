// qsim_gemm.cuh -- CTA-wide SIMT FP32 GEMM on strided global operands (learner and
// adjoint weight-gradient reductions).
#pragma once
#include <cstdint>

namespace qsim {

constexpr int LT = 256;                 // threads per CTA
constexpr int GM = 64, GN = 64, GK = 32, GLD = 68;
constexpr int GEMM_SMEM = 2 * GK * GLD; // floats

// L2-only load (operands may have been written by another SM of the cluster).  The asm is
// volatile so that it executes only where control flow reaches it: a conditional
// `cond ? load : 0` must never be turned into an unconditional load.
__device__ __forceinline__ float ldcg(const float* p) {
    float r;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(r) : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t ldcg(const uint32_t* p) {
    uint32_t r;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

struct Mat {
    const float* p;
    int64_t s0, s1;  // element (i, j) = p[i * s0 + j * s1]
};

__device__ __forceinline__ int psize(int in, int h, int out) { return h * in + h + h * h + h + out * h + out; }

// ------------------------------------------------------------------ CTA-wide SIMT GEMM
// C(m, n) = sum_k A(m, k) B(k, n) for m < M, n < N; epi(m, n, value) consumes each output.
// Operands are read with L2-only loads (they may have been written by other SMs of the
// cluster), staged in shared memory 64 x 32 / 32 x 64 per step, 4 x 4 outputs per thread.
template <class Epi>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, Mat A, Mat B, float* sm, Epi epi) {
    float* As = sm;
    float* Bs = sm + GK * GLD;
    const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
    for (int m0 = 0; m0 < M; m0 += GM) {
        for (int n0 = 0; n0 < N; n0 += GN) {
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
            for (int k0 = 0; k0 < K; k0 += GK) {
                for (int i = tid; i < GM * GK; i += LT) {
                    int mm, kk;
                    if (A.s1 == 1) { kk = i % GK; mm = i / GK; } else { mm = i % GM; kk = i / GM; }
                    const int m = m0 + mm, k = k0 + kk;
                    float v = 0.0f;
                    if (m < M && k < K) v = ldcg(A.p + m * A.s0 + k * A.s1);
                    As[kk * GLD + mm] = v;
                }
                for (int i = tid; i < GK * GN; i += LT) {
                    int kk, nn;
                    if (B.s1 == 1) { nn = i % GN; kk = i / GN; } else { kk = i % GK; nn = i / GK; }
                    const int k = k0 + kk, n = n0 + nn;
                    float v = 0.0f;
                    if (k < K && n < N) v = ldcg(B.p + k * B.s0 + n * B.s1);
                    Bs[kk * GLD + nn] = v;
                }
                __syncthreads();
                const int kc = min(GK, K - k0);
                for (int kk = 0; kk < kc; ++kk) {
                    const float4 a = *reinterpret_cast<const float4*>(As + kk * GLD + tm * 4);
                    const float4 b = *reinterpret_cast<const float4*>(Bs + kk * GLD + tn * 4);
                    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = m0 + tm * 4 + i, n = n0 + tn * 4 + j;
                    if (m < M && n < N) epi(m, n, acc[i][j]);
                }
        }
    }
    __syncthreads();
}

}  // namespace qsim
