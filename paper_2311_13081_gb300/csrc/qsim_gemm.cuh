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
// C(m, n) = sum_k A(m, k) B(k, n) (+ bias[n]) for m < M, n < N; epi(m, n, value) consumes
// each output.  Operands are read with L2-only loads (they may have been written by other
// SMs of the cluster) and staged in shared memory 64 x 32 / 32 x 64 per k-chunk, 4 x 4
// outputs per thread.  Every load address is clamped into the operand, so all 16 loads of
// a chunk are unconditional and in flight together; the next chunk is fetched into
// registers while the current one is multiplied.
template <class Epi>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, Mat A, Mat B, float* sm, Epi epi,
                                         const float* bias = nullptr) {
    if (M <= 0 || N <= 0) return;
    float* As = sm;
    float* Bs = sm + GK * GLD;
    const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
    const bool a_k_inner = A.s1 == 1, b_n_inner = B.s1 == 1;
    constexpr int PER = GM * GK / LT;  // 8 elements of each operand per thread
    for (int m0 = 0; m0 < M; m0 += GM) {
        for (int n0 = 0; n0 < N; n0 += GN) {
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
            float av[PER], bv[PER];
            auto fetch = [&](int k0) {
#pragma unroll
                for (int r = 0; r < PER; ++r) {
                    const int i = tid + r * LT;
                    const int mm = a_k_inner ? (i >> 5) : (i & (GM - 1));
                    const int kk = a_k_inner ? (i & (GK - 1)) : (i >> 6);
                    const int m = m0 + mm, k = k0 + kk;
                    const bool ok = (m < M) && (k < K);
                    av[r] = ldcg(A.p + (int64_t)min(m, M - 1) * A.s0 + (int64_t)min(k, K - 1) * A.s1);
                    if (!ok) av[r] = 0.0f;
                }
#pragma unroll
                for (int r = 0; r < PER; ++r) {
                    const int i = tid + r * LT;
                    const int nn = b_n_inner ? (i & (GN - 1)) : (i >> 5);
                    const int kk = b_n_inner ? (i >> 6) : (i & (GK - 1));
                    const int k = k0 + kk, n = n0 + nn;
                    const bool ok = (k < K) && (n < N);
                    bv[r] = ldcg(B.p + (int64_t)min(k, K - 1) * B.s0 + (int64_t)min(n, N - 1) * B.s1);
                    if (!ok) bv[r] = 0.0f;
                }
            };
            if (K > 0) fetch(0);
            for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
                for (int r = 0; r < PER; ++r) {
                    const int i = tid + r * LT;
                    const int mm = a_k_inner ? (i >> 5) : (i & (GM - 1));
                    const int kk = a_k_inner ? (i & (GK - 1)) : (i >> 6);
                    As[kk * GLD + mm] = av[r];
                }
#pragma unroll
                for (int r = 0; r < PER; ++r) {
                    const int i = tid + r * LT;
                    const int nn = b_n_inner ? (i & (GN - 1)) : (i >> 5);
                    const int kk = b_n_inner ? (i >> 6) : (i & (GK - 1));
                    Bs[kk * GLD + nn] = bv[r];
                }
                __syncthreads();
                if (k0 + GK < K) fetch(k0 + GK);
                const int kc = min(GK, K - k0);
                for (int kk = 0; kk < kc; ++kk) {
                    const float4 a = *reinterpret_cast<const float4*>(As + kk * GLD + tm * 4);
                    const float4 b = *reinterpret_cast<const float4*>(Bs + kk * GLD + tn * 4);
                    const float ar[4] = {a.x, a.y, a.z, a.w}, br[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
                }
                __syncthreads();
            }
            float bb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (bias) {
#pragma unroll
                for (int j = 0; j < 4; ++j) bb[j] = ldcg(bias + min(n0 + tn * 4 + j, N - 1));
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = m0 + tm * 4 + i, n = n0 + tn * 4 + j;
                    if (m < M && n < N) epi(m, n, acc[i][j] + bb[j]);
                }
        }
    }
    __syncthreads();
}

}  // namespace qsim
