// qsim_smlp.cuh -- shared-memory-resident MLP engine of the learner (hidden width <= 128).
//
// One network pass of a CTA: the network's weights are staged into shared memory once (a
// straight row-major copy), then the CTA's samples are processed in chunks of rows whose
// activations stay in shared memory between layers; weight gradients accumulate across
// chunks and are written out once.  Compared with the global-scratch path this replaces
// ~30 L2 round trips per update with one weight stage per pass.  Two shapes: hidden <= 64
// (64-row chunks, gradient accumulators in shared memory) and hidden <= 128 (64-row
// chunks, gradients accumulated directly in the CTA's own gradient output, which stays in
// L2: there is no room for both next to the 128-wide weights; the backward's deltas
// overwrite the hidden activations they are masked with, dZ2 over H2 and dZ1 over H1).
//
// Layouts (floats): everything row-major with padded row strides chosen == 4 (mod 32) so
// that the GEMMs' 128-bit shared loads are conflict-free: input chunk Xs[r][k], hidden
// activations and deltas [r][j], W1s[j][k], W2s[i][j], W3s[o][j].
#pragma once
#include "qsim_gemm.cuh"

namespace qsim {
namespace smlp {

constexpr int HP = 64;    // hidden bound of the 64-wide shape
constexpr int INP = 104;  // row stride of the input chunk (critic input <= 100), multiple of 8
constexpr int AS = 68;    // row stride of hidden activations (== 4 mod 32: conflict-free)
constexpr int LD1 = 100;  // row stride of W1 [j][k] (>= input width, == 4 mod 32)
constexpr int LD2 = 68;   // row stride of W2 [j][k]
constexpr int MC = 64;    // rows per chunk
// the 128-wide shape
constexpr int HP2 = 128, AS2 = 132, LD22 = 132, MC2 = 64;

struct Buf {
    float *Xs, *H1s, *H2s, *dZ2s, *dZ1s, *dZ3s;
    float *W1s, *b1, *W2s, *b2, *W3s, *b3;
    float *gW1, *gb1, *gW2, *gb2, *gW3, *gb3;
    int hp, as, ld2, mc;  // hidden bound, activation and W2 row strides, rows per chunk
    int g1, g2, g3;       // row strides of the gradient accumulators gW1, gW2, gW3
    bool gsm;             // accumulators in shared memory (else the gradient output itself)
};

__host__ __device__ constexpr int floats() {
    return MC * INP + 4 * MC * AS + MC * 4 +                // activations
           HP * LD1 + HP + HP * LD2 + HP + 4 * HP + 4 +    // weights
           HP * INP + HP + HP * HP + HP + 4 * HP + 4 + 64; // gradient accumulators (+ slack)
}

__host__ __device__ constexpr int floats2() {
    return MC2 * INP + 2 * MC2 * AS2 + MC2 * 4 +                  // activations (deltas in place)
           HP2 * LD1 + HP2 + HP2 * LD22 + HP2 + 4 * HP2 + 4 + 64;  // weights (+ slack)
}

__device__ __forceinline__ Buf carve(float* sm) {
    Buf b;
    float* p = sm;
    b.Xs = p; p += MC * INP;
    b.H1s = p; p += MC * AS;
    b.H2s = p; p += MC * AS;
    b.dZ2s = p; p += MC * AS;
    b.dZ1s = p; p += MC * AS;
    b.dZ3s = p; p += MC * 4;
    b.W1s = p; p += HP * LD1;
    b.b1 = p; p += HP;
    b.W2s = p; p += HP * LD2;
    b.b2 = p; p += HP;
    b.W3s = p; p += 4 * HP;
    b.b3 = p; p += 4;
    b.gW1 = p; p += HP * INP;
    b.gb1 = p; p += HP;
    b.gW2 = p; p += HP * HP;
    b.gb2 = p; p += HP;
    b.gW3 = p; p += 4 * HP;
    b.gb3 = p;
    b.hp = HP; b.as = AS; b.ld2 = LD2; b.mc = MC;
    b.g1 = INP; b.g2 = HP; b.g3 = HP;
    b.gsm = true;
    return b;
}

// The 128-wide shape; the gradient accumulators are bound per network by bind_grads.
__device__ __forceinline__ Buf carve2(float* sm) {
    Buf b;
    float* p = sm;
    b.Xs = p; p += MC2 * INP;
    b.H1s = p; p += MC2 * AS2;
    b.H2s = p; p += MC2 * AS2;
    b.dZ2s = b.H2s;  // each delta replaces the activation that masks it (see backward)
    b.dZ1s = b.H1s;
    b.dZ3s = p; p += MC2 * 4;
    b.W1s = p; p += HP2 * LD1;
    b.b1 = p; p += HP2;
    b.W2s = p; p += HP2 * LD22;
    b.b2 = p; p += HP2;
    b.W3s = p; p += 4 * HP2;
    b.b3 = p;
    b.gW1 = b.gb1 = b.gW2 = b.gb2 = b.gW3 = b.gb3 = nullptr;
    b.hp = HP2; b.as = AS2; b.ld2 = LD22; b.mc = MC2;
    b.g1 = b.g2 = b.g3 = 0;
    b.gsm = false;
    return b;
}

// Point the accumulators of a 128-wide engine at the gradient output G (W1[H][in] b1
// W2[H][H] b2 W3[out][H] b3, global, owned by this CTA); the shared-memory shape keeps its own.
__device__ __forceinline__ void bind_grads(Buf& b, float* G, int in, int H, int out) {
    if (b.gsm) return;
    b.gW1 = G; b.g1 = in;
    b.gb1 = G + H * in;
    b.gW2 = b.gb1 + H; b.g2 = H;
    b.gb2 = b.gW2 + H * H;
    b.gW3 = b.gb2 + H; b.g3 = H;
    b.gb3 = b.gW3 + out * H;
}

// C(m, n) = sum_k A(m, k) B(k, n) with A row-major [m][k] (lda, K a multiple of 4, padded
// with zeros) and B [k][n] (ldb); 4 x 4 outputs per thread, float4 loads along k for A and
// along n for B.  Operands may extend past M / N inside their buffers; outputs beyond M, N
// are discarded.
template <int RM, class Epi>
__device__ __forceinline__ void gemm_mk_t(int M, int N, int K4, const float* A, int lda,
                                        const float* B, int ldb, Epi epi) {
    const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
    for (int m0 = 0; m0 < M; m0 += 16 * RM)
        for (int n0 = 0; n0 < N; n0 += 64) {
            const int mb = m0 + tm * RM, nb = n0 + tn * 4;
            if (mb >= M || nb >= N) continue;
            float acc[RM][4];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
            for (int k = 0; k < K4; k += 4) {
                float a[RM][4], b[4][4];
#pragma unroll
                for (int i = 0; i < RM; ++i) {
                    const float4 v = *reinterpret_cast<const float4*>(A + (mb + i) * lda + k);
                    a[i][0] = v.x; a[i][1] = v.y; a[i][2] = v.z; a[i][3] = v.w;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4 v = *reinterpret_cast<const float4*>(B + (k + kk) * ldb + nb);
                    b[kk][0] = v.x; b[kk][1] = v.y; b[kk][2] = v.z; b[kk][3] = v.w;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                    for (int i = 0; i < RM; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i][kk], b[kk][j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (mb + i < M && nb + j < N) epi(mb + i, nb + j, acc[i][j]);
        }
    __syncthreads();
}
// gemm_mk with 4 rows per thread, or 2 when M <= 32 so that all warps take part.
template <class Epi>
__device__ __forceinline__ void gemm_mk(int M, int N, int K4, const float* A, int lda,
                                        const float* B, int ldb, Epi epi) {
    if (M <= 32) gemm_mk_t<2>(M, N, K4, A, lda, B, ldb, epi);
    else gemm_mk_t<4>(M, N, K4, A, lda, B, ldb, epi);
}

// C(m, n) = sum_k A(m, k) B(n, k): A row-major [m][k], B row-major [n][k] (the weights as
// stored), both read with float4 along k.  Lane (tm, tn) takes rows 4 tm + i and the
// interleaved columns tn + 16 j, so that with ldb == 4 (mod 32) the 16 column rows a warp
// reads per instruction fall into distinct bank quads.
template <int RM, class Epi>
__device__ __forceinline__ void gemm_nt_t(int M, int N, int K4, const float* A, int lda,
                                        const float* B, int ldb, Epi epi) {
    const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
    for (int m0 = 0; m0 < M; m0 += 16 * RM)
        for (int n0 = 0; n0 < N; n0 += 64) {
            const int mb = m0 + tm * RM, nb = n0 + tn;
            if (mb >= M || nb >= N) continue;
            float acc[RM][4];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
            for (int k = 0; k < K4; k += 4) {
                float a[RM][4], b[4][4];
#pragma unroll
                for (int i = 0; i < RM; ++i) {
                    const float4 v = *reinterpret_cast<const float4*>(A + (mb + i) * lda + k);
                    a[i][0] = v.x; a[i][1] = v.y; a[i][2] = v.z; a[i][3] = v.w;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 v = *reinterpret_cast<const float4*>(B + (nb + 16 * j) * ldb + k);
                    b[j][0] = v.x; b[j][1] = v.y; b[j][2] = v.z; b[j][3] = v.w;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                    for (int i = 0; i < RM; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i][kk], b[j][kk], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (mb + i < M && nb + 16 * j < N) epi(mb + i, nb + 16 * j, acc[i][j]);
        }
    __syncthreads();
}
// gemm_nt with 4 rows per thread, or 2 when M <= 32 so that all warps take part.
template <class Epi>
__device__ __forceinline__ void gemm_nt(int M, int N, int K4, const float* A, int lda,
                                        const float* B, int ldb, Epi epi) {
    if (M <= 32) gemm_nt_t<2>(M, N, K4, A, lda, B, ldb, epi);
    else gemm_nt_t<4>(M, N, K4, A, lda, B, ldb, epi);
}

// Dot products y[r][o] = b3[o] + sum_j W3[o][j] H[r][j] for rows r < mc: one warp per
// (row, output), lanes over j, shuffle reduction (conflict-free row reads).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Weight-gradient accumulation G(m, n) (+)= sum_k A(m, k) B(k, n) with A stored [k][m]
// (lda) and B [k][n] (ldb): dW = dZ^T X, reduced over the chunk's rows.  G (row stride ldg)
// is overwritten when `first`, else added to; its previous values are read before the
// reduction starts, 4 x NC independent loads per tile whose latency the k loop hides (G
// may be the L2-resident gradient output itself).  Lane (tm, tn) owns rows 4 tm .. 4 tm + 3
// and columns NC tn .. NC tn + NC - 1 of a 64 x 16 NC block; NC = 6 covers the input widths
// 65..96 in one block (B read as float2: 8-byte aligned, conflict-free).
template <int NC>
__device__ __forceinline__ void gemm_km_acc_t(int M, int N, int K, const float* A, int lda,
                                              const float* B, int ldb, float* G, int ldg, bool first) {
    const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
    for (int m0 = 0; m0 < M; m0 += 64)
        for (int n0 = 0; n0 < N; n0 += 16 * NC) {
            const int mb = m0 + tm * 4, nb = n0 + tn * NC;
            if (mb >= M || nb >= N) continue;
            float acc[4][NC];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < NC; ++j)
                    acc[i][j] = (!first && mb + i < M && nb + j < N) ? G[(mb + i) * ldg + nb + j] : 0.0f;
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(A + k * lda + mb);
                float bv[NC];
                if constexpr (NC == 4) {
                    const float4 b = *reinterpret_cast<const float4*>(B + k * ldb + nb);
                    bv[0] = b.x; bv[1] = b.y; bv[2] = b.z; bv[3] = b.w;
                } else {
#pragma unroll
                    for (int j = 0; j < NC; j += 2) {
                        const float2 b = *reinterpret_cast<const float2*>(B + k * ldb + nb + j);
                        bv[j] = b.x; bv[j + 1] = b.y;
                    }
                }
                const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < NC; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < NC; ++j)
                    if (mb + i < M && nb + j < N) G[(mb + i) * ldg + nb + j] = acc[i][j];
        }
    __syncthreads();
}
__device__ __forceinline__ void gemm_km_acc(int M, int N, int K, const float* A, int lda,
                                            const float* B, int ldb, float* G, int ldg, bool first) {
    if (N > 64 && N <= 96) gemm_km_acc_t<6>(M, N, K, A, lda, B, ldb, G, ldg, first);
    else gemm_km_acc_t<4>(M, N, K, A, lda, B, ldb, G, ldg, first);
}

__device__ __forceinline__ int k4(int in) { return (in + 3) & ~3; }

__device__ __forceinline__ float4 ldcg4(const float* p) {
    float4 r;
    asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}

// Copies n elements: dst(i) = src(i) for i < n (src index map `sidx`, dst map `didx`,
// elements past `valid` written as zero), 8 L2 loads in flight per thread before the
// shared-memory stores that consume them.
template <class SIdx, class DIdx, class Valid>
__device__ __forceinline__ void batched_copy(int n, const float* src, float* dst, SIdx sidx,
                                             DIdx didx, Valid valid) {
    constexpr int U = 8;
    for (int base = threadIdx.x; base < n; base += LT * U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * LT;
            const bool ok = i < n && valid(i);
            v[u] = ldcg(src + (ok ? sidx(i) : 0));
            if (!ok) v[u] = 0.0f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * LT;
            if (i < n) dst[didx(i)] = v[u];
        }
    }
}

// Reads the contiguous global range src[0, n) with L2-only loads and hands every element
// to place(i, value) (a shared-memory store).  The 16-byte-aligned body is read as float4,
// U of them per thread in flight at once; the unaligned head and tail (< 4 elements each)
// element by element.  Nothing outside src[0, n) is read.
template <class Place>
__device__ __forceinline__ void load_scatter(const float* src, int n, Place place) {
    constexpr int U = 12;
    const int lead = (int)((4u - ((uint32_t)(uintptr_t)src >> 2)) & 3u);  // elements to 16-byte alignment
    const int ia = min(lead, n);
    const int nv = (n - ia) >> 2;
    const int ib = ia + 4 * nv;
    if (threadIdx.x < ia) place(threadIdx.x, ldcg(src + threadIdx.x));
    if (threadIdx.x < n - ib) place(ib + threadIdx.x, ldcg(src + ib + threadIdx.x));
    const float* body = src + ia;
    for (int v0 = threadIdx.x; v0 < nv; v0 += LT * U) {
        float4 x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * LT;
            x[u] = v < nv ? ldcg4(body + 4 * v) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * LT;
            if (v < nv) {
                const int i = ia + 4 * v;
                place(i, x[u].x);
                place(i + 1, x[u].y);
                place(i + 2, x[u].z);
                place(i + 3, x[u].w);
            }
        }
    }
}

// Stage a network W1[H][in] b1 W2[H][H] b2 W3[out][H] b3 (global, contiguous, possibly just
// updated by another SM: L2 loads) into shared memory, W1 rows zero-padded to a multiple
// of 4 columns.
__device__ __forceinline__ void stage(const float* W, int in, int H, int out, const Buf& b) {
    const int K4 = k4(in);
    const int e1 = H * in, e2 = e1 + H, e3 = e2 + H * H, e4 = e3 + H, e5 = e4 + out * H;
    const int n = e5 + out;
    load_scatter(W, n, [&](int i, float v) {
        if (i < e1) {
            const int j = i / in;
            b.W1s[j * LD1 + (i - j * in)] = v;
        } else if (i < e2) {
            b.b1[i - e1] = v;
        } else if (i < e3) {
            const int r = (i - e2) / H;
            b.W2s[r * b.ld2 + (i - e2 - r * H)] = v;
        } else if (i < e4) {
            b.b2[i - e3] = v;
        } else if (i < e5) {
            const int o = (i - e4) / H;
            b.W3s[o * b.hp + (i - e4 - o * H)] = v;
        } else {
            b.b3[i - e5] = v;
        }
    });
    for (int i = threadIdx.x; i < H * (K4 - in); i += LT) {
        const int j = i / (K4 - in);
        b.W1s[j * LD1 + in + (i - j * (K4 - in))] = 0.0f;
    }
    __syncthreads();
}

// Loads rows [r0, r0 + n) of X (global [rows][ldx]) into rows [d0, d0 + n) of the input
// chunk, zero-padded to a multiple of 4 columns (no barrier).
__device__ __forceinline__ void load_rows(int in, const float* X, int ldx, int r0, int n, int d0,
                                          const Buf& b) {
    const int K4 = k4(in);
    float* Xd = b.Xs + d0 * INP;
    if (ldx == in) {
        // rows contiguous: one range, float4 body
        load_scatter(X + (size_t)r0 * ldx, n * in, [&](int i, float v) {
            const int r = i / in;
            Xd[r * INP + (i - r * in)] = v;
        });
        for (int i = threadIdx.x; i < n * (K4 - in); i += LT) {
            const int r = i / (K4 - in);
            Xd[r * INP + in + (i - r * (K4 - in))] = 0.0f;
        }
    } else {
        batched_copy(n * K4, X + (size_t)r0 * ldx, Xd, [&](int i) { return (i / K4) * ldx + i % K4; },
                     [&](int i) { return (i / K4) * INP + i % K4; }, [&](int i) { return i % K4 < in; });
    }
}

// The layers of the mc-row chunk held in Xs: hidden activations stay in shared memory;
// emit(r, o, y) stores output o of chunk row r.
template <class Emit>
__device__ __forceinline__ void forward_core(int in, int H, int out, int mc, const Buf& b, bool tanh_out,
                                             Emit emit) {
    __syncthreads();
    const int as = b.as;
    gemm_nt(mc, H, k4(in), b.Xs, INP, b.W1s, LD1,
            [&](int m, int n, float v) { b.H1s[m * as + n] = fmaxf(v + b.b1[n], 0.0f); });
    gemm_nt(mc, H, H, b.H1s, as, b.W2s, b.ld2,
            [&](int m, int n, float v) { b.H2s[m * as + n] = fmaxf(v + b.b2[n], 0.0f); });
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int item = warp; item < mc * out; item += LT / 32) {
        const int r = item / out, o = item - r * out;
        float acc = 0.0f;
        for (int j = lane; j < H; j += 32) acc = fmaf(b.W3s[o * b.hp + j], b.H2s[r * as + j], acc);
        acc = warp_sum(acc) + b.b3[o];
        if (lane == 0) emit(r, o, tanh_out ? tanhf(acc) : acc);
    }
    __syncthreads();
}

// Forward of rows [r0, r0 + mc) of X (global [rows][ldx]); the outputs go to Y (global
// [rows][ldy]).
__device__ __forceinline__ void forward(int in, int H, int out, const float* X, int ldx, int r0,
                                        int mc, const Buf& b, float* Y, int ldy, bool tanh_out) {
    load_rows(in, X, ldx, r0, mc, 0, b);
    forward_core(in, H, out, mc, b, tanh_out,
                 [&](int r, int o, float y) { Y[(size_t)(r0 + r) * ldy + o] = y; });
}

// Forward of one chunk made of two row blocks: rows [0, n0) of X0 and [0, mc - n0) of X1
// (both [rows][ldx]); outputs to Y0 and Y1 ([rows][ldy]) in the same split.
__device__ __forceinline__ void forward2(int in, int H, int out, const float* X0, const float* X1, int ldx,
                                         int n0, int mc, const Buf& b, float* Y0, float* Y1, int ldy,
                                         bool tanh_out) {
    load_rows(in, X0, ldx, 0, n0, 0, b);
    load_rows(in, X1, ldx, 0, mc - n0, n0, b);
    forward_core(in, H, out, mc, b, tanh_out, [&](int r, int o, float y) {
        if (r < n0) Y0[(size_t)r * ldy + o] = y;
        else Y1[(size_t)(r - n0) * ldy + o] = y;
    });
}

// Reverse of the chunk just run by forward(); dZ3s [mc][4] holds dLoss/d(output
// pre-activation).  Accumulates the parameter gradient (first: overwrite) when want_w;
// writes dLoss/dX for columns [x_lo, in) to dX (global [rows][ldx]) when dX != nullptr.
__device__ __forceinline__ void backward(int in, int H, int out, int r0, int mc, const Buf& b,
                                         bool first, bool want_w, float* dX, int ldx, int x_lo) {
    const int as = b.as;
    if (want_w) {
        for (int i = threadIdx.x; i < out * H; i += LT) {
            const int o = i / H, j = i - o * H;
            float s = 0.0f;
            for (int r = 0; r < mc; ++r) s = fmaf(b.dZ3s[r * 4 + o], b.H2s[r * as + j], s);
            b.gW3[o * b.g3 + j] = first ? s : b.gW3[o * b.g3 + j] + s;
        }
        if (threadIdx.x < out) {
            float s = 0.0f;
            for (int r = 0; r < mc; ++r) s += b.dZ3s[r * 4 + threadIdx.x];
            b.gb3[threadIdx.x] = first ? s : b.gb3[threadIdx.x] + s;
        }
        if (b.dZ2s == b.H2s) __syncthreads();  // H2 read above, overwritten below
    }
    // dZ2 in place over H2 is safe: each element is read (mask) and written by one thread;
    // likewise dZ1 over H1 in gemm_mk's epilogue, whose operands are dZ2 and W2
    for (int i = threadIdx.x; i < mc * H; i += LT) {
        const int r = i / H, j = i - r * H;
        float v = 0.0f;
        for (int o = 0; o < out; ++o) v = fmaf(b.dZ3s[r * 4 + o], b.W3s[o * b.hp + j], v);
        b.dZ2s[r * as + j] = b.H2s[r * as + j] > 0.0f ? v : 0.0f;
    }
    __syncthreads();
    if (want_w) {
        gemm_km_acc(H, H, mc, b.dZ2s, as, b.H1s, as, b.gW2, b.g2, first);
        for (int j = threadIdx.x; j < H; j += LT) {
            float s = 0.0f;
            for (int r = 0; r < mc; ++r) s += b.dZ2s[r * as + j];
            b.gb2[j] = first ? s : b.gb2[j] + s;
        }
    }
    gemm_mk(mc, H, H, b.dZ2s, as, b.W2s, b.ld2, [&](int m, int n, float v) {
        b.dZ1s[m * as + n] = b.H1s[m * as + n] > 0.0f ? v : 0.0f;
    });
    if (want_w) {
        gemm_km_acc(H, in, mc, b.dZ1s, as, b.Xs, INP, b.gW1, b.g1, first);
        for (int j = threadIdx.x; j < H; j += LT) {
            float s = 0.0f;
            for (int r = 0; r < mc; ++r) s += b.dZ1s[r * as + j];
            b.gb1[j] = first ? s : b.gb1[j] + s;
        }
    }
    if (dX) {
        const int nc = in - x_lo;
        for (int i = threadIdx.x; i < mc * nc; i += LT) {
            const int r = i / nc, c = x_lo + (i - r * nc);
            float s = 0.0f;
            for (int j = 0; j < H; ++j) s = fmaf(b.dZ1s[r * as + j], b.W1s[j * LD1 + c], s);
            dX[(size_t)(r0 + r) * ldx + c] = s;
        }
    }
    __syncthreads();
}

// Writes the accumulated gradient in the parameter layout of W (global).
__device__ __forceinline__ void store_grads(float* G, int in, int H, int out, const Buf& b) {
    if (!b.gsm) {  // the accumulators were the output
        __syncthreads();
        return;
    }
    float* gW1 = G;
    float* gb1 = gW1 + H * in;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + out * H;
    for (int i = threadIdx.x; i < H * in; i += LT) {
        const int j = i / in, k = i - j * in;
        gW1[i] = b.gW1[j * INP + k];
    }
    for (int i = threadIdx.x; i < H * H; i += LT) {
        const int r = i / H, c = i - r * H;
        gW2[i] = b.gW2[r * b.g2 + c];
    }
    for (int i = threadIdx.x; i < H; i += LT) {
        gb1[i] = b.gb1[i];
        gb2[i] = b.gb2[i];
    }
    for (int i = threadIdx.x; i < out * H; i += LT) {
        const int o = i / H, j = i - o * H;
        gW3[i] = b.gW3[o * b.g3 + j];
    }
    if (threadIdx.x < out) gb3[threadIdx.x] = b.gb3[threadIdx.x];
    __syncthreads();
}

}  // namespace smlp
}  // namespace qsim
