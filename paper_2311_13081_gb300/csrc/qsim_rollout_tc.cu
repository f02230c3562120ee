// qsim_rollout_tc.cu -- fused env-step kernel with the actor's two hidden layers on the
// 5th-generation tensor cores (tcgen05.mma kind::tf32, accumulators in tensor memory).
//
// Same step as k_rollout (actor MLP + exploration + RK4 + reward + termination + reset +
// replay write, state in registers, one thread per env); what changes is where the
// 82 -> 64 -> 64 products run:
//   * a tile is 128 envs = the MMA's M = the 128 TMEM lanes; thread r of the tile owns env
//     r and TMEM lane r.  A CTA holds two tiles of 4 compute warps each plus one MMA warp
//     per tile (warp specialisation): issuing a tcgen05.mma costs its thread ~85 cycles
//     whatever N, so the 57 MMAs of a step are issued by the tile's MMA warp while the
//     compute warps draw the step's exploration noise and write the previous step's replay
//     record; compute and MMA warps hand over through mbarriers (A1 ready, D1 full, A2
//     ready, D2 full).  The two tiles run independently.
//   * FP32 accuracy from TF32 inputs by the three-term split x = x_hi + x_lo (x_hi: x with
//     the low 13 mantissa bits cleared, x_lo = x - x_hi exactly): A.W ~ A_hi.W_hi +
//     A_hi.W_lo + A_lo.W_hi, all accumulated in FP32 in tensor memory; the dropped
//     A_lo.W_lo term and the TF32 reading of the lo parts are ~2^-20 relative.
//   * layer-1 operand A (128 x 88) lives in TMEM (hi and lo halves): columns 0..17 the
//     observation, 18..23 zero, 24..87 a 16-slot ring of past actions (a_tau in slot
//     tau mod 16).  Nothing moves when the window slides: the ring's slot pairs (2h, 2h+1)
//     hold lags (i, i-1) (or (1, 16)), so each K=8 MMA step points its B descriptor at the
//     matching pair of lag blocks of a lag-reversed copy of W1 ([lag16 .. lag1, lag16]).
//   * layer-1 output: tcgen05.ld -> bias, ReLU, split -> layer-2 operand in shared memory
//     (canonical K-major layout) -> layer-2 MMAs -> tcgen05.ld -> bias, ReLU and the
//     64 -> 4 output layer in registers (SIMT), tanh.
// Shared-memory operands use the no-swizzle K-major layout: 8-row x 16-byte core matrices,
// K-adjacent core matrices 128 B apart (LBO), 8-row groups kc * 128 B apart (SBO).
// Every hand-over wait is bounded; on expiry the waiting warp records DEV_TIMEOUT in the
// status word and raises the CTA's abort flag, every warp leaves its step loop at its next
// wait, and TMEM is freed on every path.
#include <algorithm>

#include "qsim_internal.h"

namespace qsim {
namespace tcr {

constexpr int H = 64;            // hidden width handled here
constexpr int TILE = 128;        // envs per tile
constexpr int TILES = 2;         // tiles per CTA
constexpr int NCW = TILE * TILES / 32;  // compute warps per CTA
constexpr int NT = TILE * TILES + 32 * TILES;  // threads per CTA: compute + one MMA warp per tile
constexpr int K1 = 88;           // layer-1 A columns
constexpr int KW1 = 92;          // layer-1 B columns: 24 + 17 lag blocks of 4
constexpr int KC1 = KW1 / 4;     // core-matrix columns of W1
constexpr int KC2 = H / 4;       // core-matrix columns of W2 / A2
// TMEM columns of one tile (the CTA allocates 512 = 2 x 256)
constexpr int T_AHI = 0, T_ALO = K1, T_D = 2 * K1, T_COLS = 256;
// shared memory (bytes)
constexpr int SZ_W1 = H * KW1 * 4;
constexpr int SZ_W2 = H * H * 4;
constexpr int SZ_A2 = TILE * H * 4;
constexpr int OFF_W1HI = 0;
constexpr int OFF_W1LO = OFF_W1HI + SZ_W1;
constexpr int OFF_W2HI = OFF_W1LO + SZ_W1;
constexpr int OFF_W2LO = OFF_W2HI + SZ_W2;
constexpr int OFF_A2 = OFF_W2LO + SZ_W2;  // tile k: hi at + 2k SZ_A2, lo at + (2k+1) SZ_A2
constexpr int OFF_B1 = OFF_A2 + TILES * 2 * SZ_A2;
constexpr int OFF_B2 = OFF_B1 + 4 * H;
constexpr int OFF_W3 = OFF_B2 + 4 * H;  // [H] float4: W3[0..3][j]
constexpr int OFF_B3 = OFF_W3 + 16 * H;
constexpr int OFF_BAR = OFF_B3 + 16;     // per tile: A1 ready, D1 full, A2 ready, D2 full
constexpr int OFF_TSLOT = OFF_BAR + 32 * TILES;
constexpr int OFF_ABORT = OFF_TSLOT + 16;
constexpr int SMEM = OFF_ABORT + 16;
static_assert(SMEM <= 227 * 1024, "tensor-core rollout: shared memory");
static_assert(OFF_W1LO % 128 == 0 && OFF_W2HI % 128 == 0 && OFF_A2 % 128 == 0, "alignment");

constexpr int WAIT_LIMIT = 1 << 22;  // polls of a hand-over barrier before giving up

// instruction descriptor: D f32, A and B tf32, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

__device__ __forceinline__ int cano(int r, int k, int kc) {
    return ((r >> 3) * kc + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle, K-major: LBO = 128 B (next core matrix along
// K), SBO = kc * 128 B (next 8-row group)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, int kc) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(((uint32_t)kc * 128u) >> 4) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_tt(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}"
                 :: "r"(d), "r"(a_tmem), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar));
}

// Bounded wait for the completion of phase `parity` of an mbarrier; gives up early once the
// CTA's abort flag is set.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    for (int i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

// Lane 0 waits, the warp follows; false (warp-uniform) when the wait gave up.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        ok = mbar_wait(bar, parity, abort_flag);
        if (!ok) {
            *abort_flag = 1;
            if (status) atomicCAS(status, DEV_OK, DEV_TIMEOUT);
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

#define QSIM_R4(v, o) "r"(__float_as_uint(v[o])), "r"(__float_as_uint(v[o + 1])), "r"(__float_as_uint(v[o + 2])), "r"(__float_as_uint(v[o + 3]))

__device__ __forceinline__ void st16(uint32_t ta, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(ta), QSIM_R4(v, 0), QSIM_R4(v, 4), QSIM_R4(v, 8), QSIM_R4(v, 12) : "memory");
}
__device__ __forceinline__ void st8(uint32_t ta, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(ta), QSIM_R4(v, 0), QSIM_R4(v, 4) : "memory");
}
__device__ __forceinline__ void st4(uint32_t ta, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" :: "r"(ta), QSIM_R4(v, 0) : "memory");
}
#undef QSIM_R4

// 16 columns of this warp's lanes into registers; the wait sits in the same asm statement
// so that no use of the destination registers can be scheduled before the load completes.
__device__ __forceinline__ void ld16(uint32_t ta, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two 16-column loads in flight, one wait.
__device__ __forceinline__ void ld16x2(uint32_t ta, float* v, uint32_t tb, float* w) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
                 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(ta), "r"(tb) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) { v[i] = __uint_as_float(r[i]); w[i] = __uint_as_float(r[16 + i]); }
}

// Stores one 16-column chunk of the action ring (slots 4q .. 4q+3) as hi / lo halves.
__device__ __forceinline__ void ring_store16(uint32_t ta_hi, uint32_t ta_lo, const float* x) {
    float hi[16], lo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) { hi[i] = tf32_hi(x[i]); lo[i] = x[i] - hi[i]; }
    st16(ta_hi, hi);
    st16(ta_lo, lo);
}

}  // namespace tcr

using namespace tcr;

__global__ void __launch_bounds__(NT, 1) k_rollout_tc(EnvCfg C, EnvPtrs p, const float* __restrict__ actor,
                                                      int T, uint32_t t0, int64_t head0, int64_t capacity,
                                                      float sigma_in, int warp0, int warp_end) {
    extern __shared__ __align__(1024) unsigned char smb[];
    float* W1hi = reinterpret_cast<float*>(smb + OFF_W1HI);
    float* W1lo = reinterpret_cast<float*>(smb + OFF_W1LO);
    float* W2hi = reinterpret_cast<float*>(smb + OFF_W2HI);
    float* W2lo = reinterpret_cast<float*>(smb + OFF_W2LO);
    float* sB1 = reinterpret_cast<float*>(smb + OFF_B1);
    float* sB2 = reinterpret_cast<float*>(smb + OFF_B2);
    const float4* sW3 = reinterpret_cast<const float4*>(smb + OFF_W3);
    float* sB3 = reinterpret_cast<float*>(smb + OFF_B3);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smb + OFF_TSLOT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smb + OFF_ABORT);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp >= NCW;
    const int tile = mma_warp ? warp - NCW : warp >> 2;
    const int DA = C.obs_dim, nh = C.n_hist, ld = C.ld;

    // ---- stage W1 (lag-reversed, padded), W2 as hi / lo halves; b1, b2, W3, b3
    {
        const float* gW1 = actor;
        const float* gb1 = gW1 + H * DA;
        const float* gW2 = gb1 + H;
        const float* gb2 = gW2 + H * H;
        const float* gW3 = gb2 + H;
        const float* gb3 = gW3 + 4 * H;
        for (int i = tid; i < H * KW1; i += NT) {
            const int n = i / KW1, kk = i - n * KW1;
            float w = 0.0f;
            if (kk < 18) {
                w = gW1[n * DA + kk];
            } else if (kk >= 24) {
                const int b = (kk - 24) >> 2, c = (kk - 24) & 3;
                const int lag = b < 16 ? 16 - b : 16;
                if (lag <= nh) w = gW1[n * DA + 18 + 4 * (lag - 1) + c];
            }
            const float hi = tf32_hi(w);
            W1hi[cano(n, kk, KC1)] = hi;
            W1lo[cano(n, kk, KC1)] = w - hi;
        }
        for (int i = tid; i < H * H; i += NT) {
            const int n = i / H, k = i - n * H;
            const float w = gW2[i];
            const float hi = tf32_hi(w);
            W2hi[cano(n, k, KC2)] = hi;
            W2lo[cano(n, k, KC2)] = w - hi;
        }
        for (int i = tid; i < H; i += NT) {
            sB1[i] = gb1[i];
            sB2[i] = gb2[i];
            reinterpret_cast<float4*>(smb + OFF_W3)[i] = make_float4(gW3[i], gW3[H + i], gW3[2 * H + i], gW3[3 * H + i]);
        }
        if (tid < 4) sB3[tid] = gb3[tid];
        if (tid == 0) {
            for (int k = 0; k < TILES; ++k) {
                const uint32_t b0 = smem_addr(smb + OFF_BAR + 32 * k);
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(b0), "r"(4));        // A1 ready
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(b0 + 8), "r"(1));    // D1 full
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(b0 + 16), "r"(4));   // A2 ready
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(b0 + 24), "r"(1));   // D2 full
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            *abort_flag = 0;
        }
        if (warp == NCW) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(smem_addr(tslot)), "r"(TILES * T_COLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
    }
    const uint32_t tmem = *tslot + (uint32_t)(tile * T_COLS);  // this tile's columns, lane 0
    const uint32_t bar_a1 = smem_addr(smb + OFF_BAR + 32 * tile);
    const uint32_t bar_d1 = bar_a1 + 8, bar_a2 = bar_a1 + 16, bar_d2 = bar_a1 + 24;
    float* A2hi = reinterpret_cast<float*>(smb + OFF_A2 + (2 * tile) * SZ_A2);
    float* A2lo = reinterpret_cast<float*>(smb + OFF_A2 + (2 * tile + 1) * SZ_A2);

    if (mma_warp) {
        // ================= MMA warp of this tile: lane 0 issues, the warp follows the waits
        const uint32_t sW1hi = smem_addr(W1hi), sW1lo = smem_addr(W1lo);
        const uint32_t sW2hi = smem_addr(W2hi), sW2lo = smem_addr(W2lo);
        const uint32_t sA2hi = smem_addr(A2hi), sA2lo = smem_addr(A2lo);
        uint32_t ph = 0;
        int issued = 0;  // 0: nothing in flight, 1: layer 1 committed, 2: layer 2 committed
#pragma unroll 1
        for (int tt = 0; tt < T; ++tt) {
            const uint32_t t = t0 + (uint32_t)tt;
            if ((int64_t)t < (int64_t)C.learning_starts) continue;
            if (!warp_wait(bar_a1, ph, abort_flag, p.status)) break;
            fence_after();
            if (lane == 0) {
#pragma unroll 1
                for (int j = 0; j < K1 / 8; ++j) {
                    int wcol;  // first W1 column of this K-step
                    if (j < 3) {
                        wcol = 8 * j;
                    } else {
                        const int i0 = (int)((t - 1u - (uint32_t)(2 * (j - 3))) & 15u) + 1;  // lag of slot 2(j-3)
                        wcol = 24 + 4 * (16 - i0);
                    }
                    const uint64_t bhi = sdesc(sW1hi + (uint32_t)(wcol / 4) * 128u, KC1);
                    const uint64_t blo = sdesc(sW1lo + (uint32_t)(wcol / 4) * 128u, KC1);
                    mma_tt(tmem + T_D, tmem + T_AHI + 8 * j, bhi, j > 0);
                    mma_tt(tmem + T_D, tmem + T_AHI + 8 * j, blo, 1);
                    mma_tt(tmem + T_D, tmem + T_ALO + 8 * j, bhi, 1);
                }
                mma_commit(bar_d1);
            }
            __syncwarp();
            issued = 1;
            if (!warp_wait(bar_a2, ph, abort_flag, p.status)) break;
            fence_after();
            if (lane == 0) {
#pragma unroll 1
                for (int j = 0; j < H / 8; ++j) {
                    const uint32_t ko = (uint32_t)(2 * j) * 128u;
                    const uint64_t ahi = sdesc(sA2hi + ko, KC2), alo = sdesc(sA2lo + ko, KC2);
                    const uint64_t bhi = sdesc(sW2hi + ko, KC2), blo = sdesc(sW2lo + ko, KC2);
                    mma_ss(tmem + T_D, ahi, bhi, j > 0);
                    mma_ss(tmem + T_D, ahi, blo, 1);
                    mma_ss(tmem + T_D, alo, bhi, 1);
                }
                mma_commit(bar_d2);
            }
            __syncwarp();
            issued = 2;
            ph ^= 1u;
        }
        // on an abort, let the last committed batch finish before the memory is released
        if (*abort_flag && lane == 0 && issued) {
            for (int i = 0; i < WAIT_LIMIT; ++i) {
                uint32_t done;
                const uint32_t b = issued == 1 ? bar_d1 : bar_d2;
                const uint32_t par = issued == 1 ? ph : ph ^ 1u;
                asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                             "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(b), "r"(par) : "memory");
                if (done) break;
            }
        }
    } else {
        // ================= compute warps: thread r of the tile owns env r and TMEM lane r
        const int r = tid & (TILE - 1);
        const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
        const int gw = warp0 + blockIdx.x * NCW + warp;                  // global warp (32 envs)
        const bool active = gw < warp_end;                               // warp-uniform
        const int g = active ? gw * 32 + lane : lane;  // inactive warps: an in-range index, never stored to

        float s[NS], d[6];
        Prm P = make_prm(1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f);
        uint32_t ep_index = 0, ep_step = 0, n_done = 0, len_sum = 0;
        float ep_ret = 0.0f, ret_sum = 0.0f;
#pragma unroll
        for (int i = 0; i < NS; ++i) s[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = 0.0f;
        s[3] = 1.0f;
        if (active) {
#pragma unroll
            for (int i = 0; i < NS; ++i) s[i] = p.state[i * ld + g];
#pragma unroll
            for (int i = 0; i < 6; ++i) d[i] = p.dist[i * ld + g];
            P = make_prm(p.prm[g], p.prm[ld + g], p.prm[2 * ld + g], p.prm[3 * ld + g], p.prm[4 * ld + g],
                         p.prm[5 * ld + g], p.prm[6 * ld + g]);
            ep_index = p.ep_index[g]; ep_step = p.ep_step[g];
            n_done = p.n_done[g]; len_sum = p.len_sum[g];
            ep_ret = p.ep_ret[g]; ret_sum = p.ret_sum[g];
        }
        float Cr[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) Cr[i] = p.rewardC[i];
        const float sigma = sigma_in >= 0.0f ? sigma_in : p.rewardC[7];
        // action ring: slot (t0 - i) mod 16 holds a_{t0-i} (global history is newest first)
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            float x[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int sl = 4 * q + (j >> 2), c = j & 3;
                const int i0 = (int)((t0 - (uint32_t)sl) & 15u);
                const int i = i0 == 0 ? 16 : i0;
                x[j] = 0.0f;
                if (active && i <= nh) x[j] = p.hist[(4 * (i - 1) + c) * ld + g];
            }
            ring_store16(tl + T_AHI + 24 + 16 * q, tl + T_ALO + 24 + 16 * q, x);
        }
        int64_t slot = capacity > 0 ? head0 % capacity : 0;
        const int F = C.F;
        uint32_t ph = 0;
        // the previous step's transition, written while the next step's MMAs run
        bool pend = false;
        float ps[NS], ps2[NS], pa[4], pr = 0.0f;
        uint32_t pflags = 0;
        int64_t pslot = 0;
        Prm pP = P;
        float pd[6];
        auto flush = [&]() {
            if (pend && capacity > 0 && active) {
                float* rec = p.rec + (size_t)pslot * F * ld + g;
#pragma unroll
                for (int i = 0; i < NS; ++i) __stcs(rec + i * ld, ps[i]);
#pragma unroll
                for (int i = 0; i < 4; ++i) __stcs(rec + (17 + i) * ld, pa[i]);
                __stcs(rec + 21 * ld, pr);
                __stcs(rec + 22 * ld, __uint_as_float(pflags));
                if (C.n_priv) {
                    float pv[NPRIV];
                    priv_vals(C, pP, pd, pv);
#pragma unroll
                    for (int k = 0; k < NPRIV; ++k) __stcs(rec + (23 + k) * ld, pv[k]);
                }
                if (pflags & 3u) {
                    float* sd = p.side + (size_t)pslot * NS * ld + g;
#pragma unroll
                    for (int i = 0; i < NS; ++i) __stcs(sd + i * ld, ps2[i]);
                }
            }
            pend = false;
        };

#pragma unroll 1
        for (int tt = 0; tt < T; ++tt) {
            const uint32_t t = t0 + (uint32_t)tt;
            float a[4];
            if ((int64_t)t < (int64_t)C.learning_starts) {
                flush();
                const uint4 rr = draw(C, (uint32_t)g, t, TAG_WARM, 0);
                a[0] = 2.0f * u01(rr.x) - 1.0f;
                a[1] = 2.0f * u01(rr.y) - 1.0f;
                a[2] = 2.0f * u01(rr.z) - 1.0f;
                a[3] = 2.0f * u01(rr.w) - 1.0f;
            } else {
                // ---------------- observation -> A columns 0..23 (hi / lo); hand over
                {
                    float o[24];
                    obs_state(s, o);
                    if (C.any_noise) {
                        float nz[18];
                        obs_noise(C, (uint32_t)g, t, nz);
#pragma unroll
                        for (int k = 0; k < 18; ++k) o[k] += nz[k];
                    }
#pragma unroll
                    for (int k = 18; k < 24; ++k) o[k] = 0.0f;
                    float hi[24], lo[24];
#pragma unroll
                    for (int k = 0; k < 24; ++k) { hi[k] = tf32_hi(o[k]); lo[k] = o[k] - hi[k]; }
                    st16(tl + T_AHI, hi);
                    st8(tl + T_AHI + 16, hi + 16);
                    st16(tl + T_ALO, lo);
                    st8(tl + T_ALO + 16, lo + 16);
                    wait_st();
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_a1);
                // ---------------- while layer 1 runs: exploration noise, last step's record
                float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (sigma > 0.0f) {
                    const uint4 r0 = draw(C, (uint32_t)g, t, TAG_EXPL, 0);
                    const uint4 r1 = draw(C, (uint32_t)g, t, TAG_EXPL, 1);
                    z[0] = gauss(r0.x, r0.y); z[1] = gauss(r0.z, r0.w);
                    z[2] = gauss(r1.x, r1.y); z[3] = gauss(r1.z, r1.w);
                }
                flush();
                if (!warp_wait(bar_d1, ph, abort_flag, p.status)) break;
                fence_after();
                // ---------------- epilogue 1: bias, ReLU, split -> A2 (shared memory); hand over
#pragma unroll 1
                for (int c0 = 0; c0 < H; c0 += 32) {
                    float v[32];
                    ld16x2(tl + T_D + c0, v, tl + T_D + c0 + 16, v + 16);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float hv[4], lv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float x = fmaxf(v[4 * q + e] + sB1[c0 + 4 * q + e], 0.0f);
                            hv[e] = tf32_hi(x);
                            lv[e] = x - hv[e];
                        }
                        const int off = cano(r, c0 + 4 * q, KC2);
                        *reinterpret_cast<float4*>(A2hi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<float4*>(A2lo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_a2);
                if (!warp_wait(bar_d2, ph, abort_flag, p.status)) break;
                fence_after();
                ph ^= 1u;
                // ---------------- epilogue 2 + output layer (64 -> 4), tanh
                float pp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
                for (int c0 = 0; c0 < H; c0 += 32) {
                    float v[32];
                    ld16x2(tl + T_D + c0, v, tl + T_D + c0 + 16, v + 16);
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const float hcur = fmaxf(v[e] + sB2[c0 + e], 0.0f);
                        const float4 w3 = sW3[c0 + e];
                        pp[0] = fmaf(w3.x, hcur, pp[0]);
                        pp[1] = fmaf(w3.y, hcur, pp[1]);
                        pp[2] = fmaf(w3.z, hcur, pp[2]);
                        pp[3] = fmaf(w3.w, hcur, pp[3]);
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float mu = tanhf(pp[j] + sB3[j]);
                    a[j] = clampf(sigma > 0.0f ? fmaf(sigma, z[j], mu) : mu, -1.0f, 1.0f);
                }
            }
            // ---------------- dynamics, reward, termination
            float u[4], s2[NS];
            action_to_rpm(C.veh, a, u);
#pragma unroll
            for (int i = 0; i < NS; ++i) s2[i] = s[i];
            rk4(C.veh, C.dt, C.renorm, s2, u, P, d);
            const float rw = reward(Cr, s2, a);
            const bool term = terminated(C, s2);
            const uint32_t ep_after = ep_step + 1;
            const bool trunc = !term && (int)ep_after >= C.episode_len;
            // ---------------- transition: kept for the next step's MMA shadow
            if (capacity > 0) {
                pend = true;
#pragma unroll
                for (int i = 0; i < NS; ++i) { ps[i] = s[i]; ps2[i] = s2[i]; }
#pragma unroll
                for (int i = 0; i < 4; ++i) pa[i] = a[i];
                pr = rw;
                pflags = pack_flags(term, trunc, ep_step);
                pslot = slot;
                pP = P;
#pragma unroll
                for (int i = 0; i < 6; ++i) pd[i] = d[i];
                slot = (slot + 1 == capacity) ? 0 : slot + 1;
            }
            // ---------------- action ring: a_t into slot t mod 16; an episode end clears the ring
            const bool reset = term || trunc;
            const int hs = (int)(t & 15u);
            if (!__any_sync(0xffffffffu, reset)) {
                float hi[4], lo[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) { hi[c] = tf32_hi(a[c]); lo[c] = a[c] - hi[c]; }
                st4(tl + T_AHI + 24 + 4 * hs, hi);
                st4(tl + T_ALO + 24 + 4 * hs, lo);
            } else {
#pragma unroll 1
                for (int q = 0; q < 4; ++q) {
                    float vh[16], vl[16], x[16];
                    ld16x2(tl + T_AHI + 24 + 16 * q, vh, tl + T_ALO + 24 + 16 * q, vl);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int sl = 4 * q + (j >> 2);
                        x[j] = reset ? 0.0f : (sl == hs ? a[j & 3] : vh[j] + vl[j]);
                    }
                    ring_store16(tl + T_AHI + 24 + 16 * q, tl + T_ALO + 24 + 16 * q, x);
                }
            }
            ep_ret += rw;
            if (reset) {
                n_done += 1;
                len_sum += ep_after;
                ret_sum += ep_ret;
                ep_index += 1;
                float prm7[7];
                reset_env(C, (uint32_t)g, ep_index, s, prm7, d);
                P = make_prm(prm7[0], prm7[1], prm7[2], prm7[3], prm7[4], prm7[5], prm7[6]);
                ep_step = 0;
                ep_ret = 0.0f;
            } else {
#pragma unroll
                for (int i = 0; i < NS; ++i) s[i] = s2[i];
                ep_step = ep_after;
            }
        }
        flush();
        wait_st();

        // ---- write back (state, parameters, counters, history newest first)
        if (active) {
#pragma unroll
            for (int i = 0; i < NS; ++i) p.state[i * ld + g] = s[i];
            p.prm[g] = P.m; p.prm[ld + g] = P.Jx; p.prm[2 * ld + g] = P.Jy; p.prm[3 * ld + g] = P.Jz;
            p.prm[4 * ld + g] = P.kf; p.prm[5 * ld + g] = P.km; p.prm[6 * ld + g] = P.tm;
#pragma unroll
            for (int i = 0; i < 6; ++i) p.dist[i * ld + g] = d[i];
            p.ep_index[g] = ep_index; p.ep_step[g] = ep_step; p.ep_ret[g] = ep_ret;
            p.n_done[g] = n_done; p.len_sum[g] = len_sum; p.ret_sum[g] = ret_sum;
        }
        const uint32_t t_end = t0 + (uint32_t)T;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            float vh[16], vl[16];
            ld16x2(tl + T_AHI + 24 + 16 * q, vh, tl + T_ALO + 24 + 16 * q, vl);
            if (active) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int sl = 4 * q + (j >> 2), c = j & 3;
                    const int i0 = (int)((t_end - (uint32_t)sl) & 15u);
                    const int i = i0 == 0 ? 16 : i0;  // lag of slot sl after the last step
                    if (i <= nh) p.hist[(4 * (i - 1) + c) * ld + g] = vh[j] + vl[j];
                }
            }
        }
    }
    // ---- release tensor memory
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == NCW)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(*tslot), "r"(TILES * T_COLS) : "memory");
}

// Launches T steps on env warps [w0, w1) (8 env warps = 256 envs per CTA, plus 2 MMA warps).
qsim_status launch_rollout_tc_range(qsim_handle* h, const float* actor, int T, uint32_t t0, int64_t head,
                                    float sigma, int w0, int w1, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        QCHECK_CUDA(cudaFuncSetAttribute(k_rollout_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        configured = true;
    }
    const int grid = (w1 - w0 + NCW - 1) / NCW;
    k_rollout_tc<<<grid, NT, SMEM, st>>>(h->dc, h->p, actor, T, t0, head, h->capacity, sigma, w0, w1);
    QCHECK_LAUNCH("k_rollout_tc");
    return QSIM_OK;
}

}  // namespace qsim
