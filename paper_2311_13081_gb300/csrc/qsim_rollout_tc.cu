// qsim_rollout_tc.cu -- fused env-step kernel with the actor's two hidden layers on the
// 5th-generation tensor cores (tcgen05.mma kind::f16 with fp16 operands, FP32 accumulators
// in tensor memory).
//
// Same step as k_rollout (actor MLP + exploration + RK4 + reward + termination + reset +
// replay write, state in registers, one thread per env); what changes is where the
// 82 -> 64 -> 64 products run:
//   * a tile is 128 envs = the MMA's M = the 128 TMEM lanes; thread r of the tile owns env
//     r and TMEM lane r.  A CTA holds three tiles of 4 compute warps each plus one MMA warp
//     per tile (warp specialisation).  A chain of tcgen05.mma issued by one thread completes
//     one instruction per ~65 cycles whatever N (<= 128) -- chains of several warps proceed
//     in parallel -- so a tile's MMA latency per step is its instruction count x ~65 cycles
//     and the design minimises MMA instructions: fp16 operands give K = 16 per instruction,
//     and every operand is kept
//     as two halves, x = x_hi + x_lo (x_hi = fp16(x), x_lo = fp16(x - x_hi)), so that
//     A.W ~ A_hi.W_hi + A_hi.W_lo + A_lo.W_hi is FP32-accurate (the dropped A_lo.W_lo term
//     and the rounding of the lo halves are ~2^-22 relative): 18 MMAs for layer 1 and 12
//     for layer 2 per tile and step.  Compute and MMA warps hand over through mbarriers
//     (A1 ready, D1 full, A2 ready, D2 full); the compute warps draw the step's exploration
//     noise while layer 1 runs.  The tiles run independently.
//   * layer-1 operand A (128 x 96 halves) lives in TMEM as packed halves (element 2c in the
//     low 16 bits of column c), hi and lo: elements 0..17 the observation, 18 the constant 1
//     (its W1 column holds b1, so layer 1's bias comes out of the MMA), 19..31 zero, 32..95
//     a 16-slot ring of past actions (a_tau in slot tau mod 16).  Nothing moves when
//     the window slides: each K=16 MMA step covers ring slots 4s..4s+3, which hold lags
//     (i, i-1, i-2, i-3) (cyclically in 1..16), and points its B descriptor at the matching
//     four lag blocks of a lag-reversed copy of W1 ([lag16 .. lag1, lag16, lag15, lag14]).
//     A B descriptor must start on an 8-element core-matrix boundary while lag blocks are 4
//     elements wide, so W1 is staged twice, shifted by 4 elements: even and odd start
//     blocks each find an aligned copy.
//   * layer-1 output: tcgen05.ld -> ReLU, split -> layer-2 operand in shared memory
//     (canonical K-major layout) -> layer-2 MMAs -> tcgen05.ld -> bias, ReLU and the
//     64 -> 4 output layer in registers (SIMT), tanh.
//   * the half-precision range (|x| < 65504) holds for the observation of any state that
//     has not terminated and for the hidden activations of any sane actor; a value outside
//     it is reported as DEV_RANGE in the status word instead of being rounded silently.
// Shared-memory operands use the no-swizzle K-major layout: 8-row x 16-byte core matrices,
// K-adjacent core matrices 128 B apart (LBO), 8-row groups kc * 128 B apart (SBO).
// Every hand-over wait is bounded; on expiry the waiting warp records DEV_TIMEOUT in the
// status word and raises the CTA's abort flag, every warp leaves its step loop at its next
// wait, and TMEM is freed on every path.
// The kernel is a template on TRACK: the training step (false), or the trajectory-tracking
// flight of qsim_track (true; Sec. V): offset, clipped observation, tracking error instead
// of reward, no records or resets, the flights' state in per-call scratch.
#include <cuda_fp16.h>

#include <algorithm>

#include "qsim_internal.h"

namespace qsim {
namespace tcr {

constexpr int H = 64;                          // hidden width handled here
constexpr int TILE = 128;                      // envs per tile
constexpr int TILES = 3;                       // tiles per CTA
constexpr int NCW = TILE * TILES / 32;         // compute warps per CTA
constexpr int NT = TILE * TILES + 32 * TILES;  // threads per CTA: compute + one MMA warp per tile
constexpr int KA = 96;                         // layer-1 A elements: 32 observation + 64 ring
constexpr int KW = 112;                        // W1 copy: 32 obs | (4 zero, copy O) 19 lag blocks of 4 | pad
constexpr int KC1 = KW / 8;                    // core-matrix columns of a W1 copy
constexpr int KC2 = 64 / 8;                    // core-matrix columns of W2 / A2
// TMEM columns of one tile (32-bit columns; a column holds two halves)
constexpr int T_AHI = 0, T_ALO = KA / 2, T_D = KA, T_COLS = KA + H;  // 160
constexpr int T_ALLOC = 512;
static_assert(TILES * T_COLS <= T_ALLOC, "tensor memory");
// shared memory (bytes)
constexpr int SZ_W1 = H * KW * 2;
constexpr int SZ_W2 = H * H * 2;
constexpr int SZ_A2 = TILE * H * 2;
constexpr int OFF_W1 = 0;                   // [E hi, E lo, O hi, O lo]
constexpr int OFF_W2 = OFF_W1 + 4 * SZ_W1;  // [hi, lo]
constexpr int OFF_A2 = OFF_W2 + 2 * SZ_W2;  // tile k: hi at + 2k SZ_A2, lo at + (2k+1) SZ_A2
constexpr int OFF_B2 = OFF_A2 + TILES * 2 * SZ_A2;  // b1 is a column of W1
constexpr int OFF_W3 = OFF_B2 + 4 * H;  // [H/2][4] float2: (W3[o][2i], W3[o][2i+1])
constexpr int OFF_B3 = OFF_W3 + 16 * H;
constexpr int OFF_BAR = OFF_B3 + 16;  // per tile: A1 ready, D1 full, A2 ready, D2 full
constexpr int OFF_TSLOT = OFF_BAR + 32 * TILES;
constexpr int OFF_ABORT = OFF_TSLOT + 16;
constexpr int OFF_UNIT = OFF_ABORT + 16;
// precomputed B descriptors of layer 1 (hi, lo): [0..1] the observation K-steps, [2 + b0]
// the lag window starting at block b0 (b0 = 0..15); layer 2 per tile: (A hi, A lo, B hi,
// B lo) for each of its 4 K-steps
constexpr int OFF_DESC = (OFF_UNIT + 16 + 7) & ~7;
constexpr int N_DESC1 = 2 * (2 + 16), N_DESC2 = TILES * 4 * 4;
// the start of each compute thread's next episode, computed ahead (reset_env for episode
// ep_index + 1): [NXF][TILE * TILES] floats, field-major (state 17, parameters 7,
// disturbance 6)
constexpr int NXF = NS + 7 + 6;
constexpr int NX_LD = TILE * TILES;
constexpr int OFF_NXT = (OFF_DESC + 8 * (N_DESC1 + N_DESC2) + 15) & ~15;
constexpr int SMEM = OFF_NXT + 4 * NXF * NX_LD;
// steps between the passes that compute the next episodes' starts of the threads whose
// precomputed start was used (a power of two), besides the pass after a unit's first step.
// Measured on the 65,536 x 1,000 rollout (episodes of ~42 steps, 50-step units): every 4
// steps 8.1, 8: 8.38, 16: 8.54, 32: 8.61, 64: 8.65 x 10^9 env-steps/s -- a pass costs the
// warp a full reset for all its lanes, so a rare pass (mostly the one per unit) wins.
constexpr int NX_EVERY = 64;
static_assert(SMEM <= 227 * 1024, "tensor-core rollout: shared memory");
static_assert(SZ_W1 % 128 == 0 && OFF_A2 % 128 == 0 && SZ_A2 % 128 == 0, "alignment");

// polls of the wait that lets committed MMAs finish before an aborting CTA frees tensor
// memory (the hand-over and inter-CTA waits use the env set's run-time limit)
constexpr int WAIT_LIMIT = 1 << 22;
constexpr float HALF_MAX = 65504.0f;

// instruction descriptor: D f32, A and B f16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

// element (r, k) of a canonical K-major 16-bit operand with kc core-matrix columns
__device__ __forceinline__ int cano16(int r, int k, int kc) {
    return ((r >> 3) * kc + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

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
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}"
                 :: "r"(d), "r"(a_tmem), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar));
}

// The whole warp waits (try_wait suspends it in hardware between polls), kept uniform by a
// vote; false (warp-uniform) when the wait gave up.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          int limit) {
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (__any_sync(0xffffffffu, done)) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
    }
    if ((threadIdx.x & 31) == 0) {
        *abort_flag = 1;
        if (status) atomicCAS(status, DEV_OK, DEV_TIMEOUT);
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

#define QSIM_R4(v, o) "r"(v[o]), "r"(v[o + 1]), "r"(v[o + 2]), "r"(v[o + 3])
__device__ __forceinline__ void st16(uint32_t ta, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(ta), QSIM_R4(v, 0), QSIM_R4(v, 4), QSIM_R4(v, 8), QSIM_R4(v, 12) : "memory");
}
__device__ __forceinline__ void st2(uint32_t ta, uint32_t a, uint32_t b) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" :: "r"(ta), "r"(a), "r"(b) : "memory");
}
#undef QSIM_R4

// Two 16-column loads of this warp's lanes in flight, one wait; the wait sits in the same
// asm statement so that no use of the destination registers is scheduled before it.
__device__ __forceinline__ void ld16x2(uint32_t ta, uint32_t* r, uint32_t tb, uint32_t* q) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
                 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
                   "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
                 : "r"(ta), "r"(tb) : "memory");
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }

// Split a pair (x0, x1) into packed hi and lo halves; amax tracks the largest magnitude
// (checked against the half-precision range once per launch).
// max that propagates NaN (fmaxf would drop it), so a non-finite operand reaches the range check
__device__ __forceinline__ float fmax_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo, float& amax) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 f = __half22float2(h);
    hi = h2u(h);
    lo = h2u(__floats2half2_rn(x0 - f.x, x1 - f.y));
    amax = fmax_nan(amax, fmax_nan(fabsf(x0), fabsf(x1)));
}

// Value of a packed hi/lo pair.
__device__ __forceinline__ float2 join2(uint32_t hi, uint32_t lo) {
    const float2 a = __half22float2(u2h(hi)), b = __half22float2(u2h(lo));
    return make_float2(a.x + b.x, a.y + b.y);
}

}  // namespace tcr

using namespace tcr;

// Work units: (group g of NCW env warps, chunk k of `chunk` steps).  With `sched` (device
// counters [next unit, done chunks of group 0 .. n_groups-1], zeroed by the host) the grid is
// persistent: each CTA takes units in chunk-major order from the counter and starts chunk k
// of a group once chunk k-1 of that group has been published (a bounded wait); every unit
// it waits for was taken earlier by a running CTA, so the wait always ends.  Without
// `sched`, CTA b runs group b for all T steps.
// TRACK = true flies the deterministic actor along the figure-eight target of Sec. V
// instead (qsim_track): the observation's position and velocity are offset by the target's
// and clipped, the squared tracking error is accumulated, and there is no reward, record
// or reset; the flight's state, action ring and running sums live in per-call scratch
// (p) and in tr, carried from unit to unit like the training state.
template <bool TRACK>
__global__ void __launch_bounds__(NT, 1) k_rollout_tc(EnvCfg C, EnvPtrs p, const float* __restrict__ actor,
                                                      int T, uint32_t t0, int64_t head0, int64_t capacity,
                                                      float sigma_in, int warp0, int warp_end,
                                                      int n_groups, int chunk, int* sched, TrackArgs tr) {
    extern __shared__ __align__(1024) unsigned char smb[];
    __half* W1s = reinterpret_cast<__half*>(smb + OFF_W1);
    __half* W2s = reinterpret_cast<__half*>(smb + OFF_W2);
    float* sB2 = reinterpret_cast<float*>(smb + OFF_B2);
    const float4* sW3 = reinterpret_cast<const float4*>(smb + OFF_W3);  // [H/2][2]: outputs (0,1), (2,3)
    float* sB3 = reinterpret_cast<float*>(smb + OFF_B3);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smb + OFF_TSLOT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smb + OFF_ABORT);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp >= NCW;
    const int tile = mma_warp ? warp - NCW : warp >> 2;
    const int DA = C.obs_dim, nh = C.n_hist, ld = C.ld;

    // ---- stage W1 (two lag-reversed copies), W2 as hi / lo halves; b1, b2, W3, b3
    {
        const float* gW1 = actor;
        const float* gb1 = gW1 + H * DA;
        const float* gW2 = gb1 + H;
        const float* gb2 = gW2 + H * H;
        const float* gW3 = gb2 + H;
        const float* gb3 = gW3 + 4 * H;
        bool wbad = false;  // a weight outside the half-precision range (or not finite)
        for (int i = tid; i < 2 * H * KW; i += NT) {
            const int copy = i / (H * KW), j = i - copy * H * KW;  // copy 0: E, 1: O (shifted by 4)
            const int n = j / KW, kk = j - n * KW;
            float w = 0.0f;
            if (kk < 18) {
                w = gW1[n * DA + kk];
            } else if (kk == 18) {
                w = gb1[n];  // multiplies the constant-1 element of the observation block
            } else if (kk >= 32) {
                const int kb = kk - (copy ? 36 : 32);  // position inside the lag blocks
                if (kb >= 0 && kb < 4 * 19) {
                    const int b = kb >> 2, c = kb & 3;
                    const int lag = b < 16 ? 16 - b : 32 - b;  // blocks 16, 17, 18: lags 16, 15, 14
                    if (lag <= nh) w = gW1[n * DA + 18 + 4 * (lag - 1) + c];
                }
            }
            wbad |= !(fabsf(w) < HALF_MAX);
            const __half hi = __float2half_rn(w);
            __half* base = W1s + (size_t)(2 * copy) * (H * KW);
            base[cano16(n, kk, KC1)] = hi;
            base[H * KW + cano16(n, kk, KC1)] = __float2half_rn(w - __half2float(hi));
        }
        for (int i = tid; i < H * H; i += NT) {
            const int n = i / H, k = i - n * H;
            const float w = gW2[i];
            wbad |= !(fabsf(w) < HALF_MAX);
            const __half hi = __float2half_rn(w);
            W2s[cano16(n, k, KC2)] = hi;
            W2s[H * H + cano16(n, k, KC2)] = __float2half_rn(w - __half2float(hi));
        }
        for (int i = tid; i < H; i += NT) {
            sB2[i] = gb2[i];
            if (i < H / 2)
#pragma unroll
                for (int o = 0; o < 4; ++o)
                    reinterpret_cast<float2*>(smb + OFF_W3)[4 * i + o] = make_float2(gW3[o * H + 2 * i], gW3[o * H + 2 * i + 1]);
        }
        if (tid < 4) sB3[tid] = gb3[tid];
        if (wbad && p.status) atomicCAS(p.status, DEV_OK, DEV_RANGE);
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
        if (tid < 2 + 16) {
            // layer-1 B descriptors: observation K-steps (copy E) and the 16 lag windows
            uint64_t* d1 = reinterpret_cast<uint64_t*>(smb + OFF_DESC);
            const uint32_t sW1 = smem_addr(W1s);
            uint32_t wbase;
            int kk;
            if (tid < 2) {
                wbase = sW1;
                kk = 16 * tid;
            } else {
                const int b0 = tid - 2;
                wbase = sW1 + (uint32_t)((b0 & 1) * 2 * SZ_W1);
                kk = (b0 & 1) ? 36 + 4 * b0 : 32 + 4 * b0;
            }
            d1[2 * tid] = sdesc(wbase + (uint32_t)(kk / 8) * 128u, KC1);
            d1[2 * tid + 1] = sdesc(wbase + (uint32_t)SZ_W1 + (uint32_t)(kk / 8) * 128u, KC1);
        } else if (tid >= 32 && tid < 32 + TILES * 4) {
            // layer-2 descriptors of tile k, K-step j
            const int k = (tid - 32) >> 2, j = (tid - 32) & 3;
            uint64_t* d2 = reinterpret_cast<uint64_t*>(smb + OFF_DESC) + N_DESC1 + 16 * k + 4 * j;
            const uint32_t ko = (uint32_t)(2 * j) * 128u;
            const uint32_t a_hi = smem_addr(smb + OFF_A2 + (2 * k) * SZ_A2);
            const uint32_t a_lo = smem_addr(smb + OFF_A2 + (2 * k + 1) * SZ_A2);
            const uint32_t w2 = smem_addr(W2s);
            d2[0] = sdesc(a_hi + ko, KC2);
            d2[1] = sdesc(a_lo + ko, KC2);
            d2[2] = sdesc(w2 + ko, KC2);
            d2[3] = sdesc(w2 + (uint32_t)SZ_W2 + ko, KC2);
        }
        if (warp == NCW) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(smem_addr(tslot)), "r"(T_ALLOC) : "memory");
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
    __half* A2hi = reinterpret_cast<__half*>(smb + OFF_A2 + (2 * tile) * SZ_A2);
    __half* A2lo = reinterpret_cast<__half*>(smb + OFF_A2 + (2 * tile + 1) * SZ_A2);

    volatile int* unit_slot = reinterpret_cast<volatile int*>(smb + OFF_UNIT);
    const int n_chunks = (T + chunk - 1) / chunk;
    const int n_units = n_groups * n_chunks;
    uint32_t ph = 0;  // hand-over phase, advanced once per actor step (compute and MMA warps alike)
    int issued = 0;   // MMA warp: 0 nothing in flight, 1 layer 1 committed, 2 layer 2 committed
#pragma unroll 1
    for (int it = 0;; ++it) {
        if (tid == 0) {
            int u = sched ? atomicAdd(sched, 1) : (it == 0 ? (int)blockIdx.x : n_units);
            if (sched && u < n_units && u >= n_groups) {
                // chunk k of group g needs chunk k-1 of the same group published
                const int* done = sched + 1 + u % n_groups;
                const int need = u / n_groups;
                bool ok = false;
                for (int i = 0; i < C.wait_limit; ++i) {
                    int v;
                    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(done) : "memory");
                    if (v >= need) { ok = true; break; }
                    if (*abort_flag) break;
                    __nanosleep(256);
                }
                if (!ok) {
                    *abort_flag = 1;
                    if (p.status) atomicCAS(p.status, DEV_OK, DEV_TIMEOUT);
                }
            }
            *unit_slot = u;
        }
        __syncthreads();
        const int u = *unit_slot;
        if (u >= n_units || *abort_flag) break;
        const int ug = u % n_groups, uk = u / n_groups;
        const int Tu = min(chunk, T - uk * chunk);
        const uint32_t t0u = t0 + (uint32_t)(uk * chunk);
        const int64_t headu = head0 + (int64_t)uk * chunk;
        if (mma_warp) {
            // ================= MMA warp of this tile: lane 0 issues, the warp follows the waits
            // (descriptors from the table built at setup: the issue loops are MMAs only)
            const uint64_t* d1 = reinterpret_cast<const uint64_t*>(smb + OFF_DESC);
            const uint64_t* d2 = d1 + N_DESC1 + 16 * tile;
#pragma unroll 1
            for (int tt = 0; tt < Tu; ++tt) {
                const uint32_t t = t0u + (uint32_t)tt;
                if ((int64_t)t < (int64_t)C.learning_starts) continue;
                if (!warp_wait(bar_a1, ph, abort_flag, p.status, C.wait_limit)) break;
                fence_after();
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < KA / 16; ++j) {
                        // B window of K-step j: the observation block, or the lag window whose
                        // first block b0 holds the lag of ring slot 4(j-2)
                        const int e = j < 2 ? j : 2 + 15 - (int)((t - 1u - (uint32_t)(4 * (j - 2))) & 15u);
                        const uint64_t bhi = d1[2 * e], blo = d1[2 * e + 1];
                        mma_tt(tmem + T_D, tmem + T_AHI + 8 * j, bhi, j > 0);
                        mma_tt(tmem + T_D, tmem + T_AHI + 8 * j, blo, 1);
                        mma_tt(tmem + T_D, tmem + T_ALO + 8 * j, bhi, 1);
                    }
                    mma_commit(bar_d1);
                }
                __syncwarp();
                issued = 1;
                if (!warp_wait(bar_a2, ph, abort_flag, p.status, C.wait_limit)) break;
                fence_after();
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < H / 16; ++j) {
                        const uint64_t ahi = d2[4 * j], alo = d2[4 * j + 1], bhi = d2[4 * j + 2], blo = d2[4 * j + 3];
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
        } else {
            // ================= compute warps: thread r of the tile owns env r and TMEM lane r
            const int r = tid & (TILE - 1);
            const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
            const int gw = warp0 + ug * NCW + warp;                          // global warp (32 envs)
            const bool active = gw < warp_end;                               // warp-uniform
            const int g = active ? gw * 32 + lane : lane;  // inactive warps: an in-range index, never stored to

            float s[NS], d[6];
            Prm P = make_prm(1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f);
            // this thread's precomputed next-episode start (valid while nxt_ok)
            float* nx = reinterpret_cast<float*>(smb + OFF_NXT) + tid;
            bool nxt_ok = false;
            uint32_t ep_index = 0, ep_step = 0, n_done = 0, len_sum = 0;
            float ep_ret = 0.0f, ret_sum = 0.0f;
#pragma unroll
            for (int i = 0; i < NS; ++i) s[i] = 0.0f;
#pragma unroll
            for (int i = 0; i < 6; ++i) d[i] = 0.0f;
            s[3] = 1.0f;
            if (active) {
#pragma unroll
                for (int i = 0; i < NS; ++i) s[i] = __ldcg(p.state + i * ld + g);
#pragma unroll
                for (int i = 0; i < 6; ++i) d[i] = __ldcg(p.dist + i * ld + g);
                P = make_prm(__ldcg(p.prm + g), __ldcg(p.prm + ld + g), __ldcg(p.prm + 2 * ld + g),
                             __ldcg(p.prm + 3 * ld + g), __ldcg(p.prm + 4 * ld + g), __ldcg(p.prm + 5 * ld + g),
                             __ldcg(p.prm + 6 * ld + g));
                ep_index = __ldcg(p.ep_index + g); ep_step = __ldcg(p.ep_step + g);
                n_done = __ldcg(p.n_done + g); len_sum = __ldcg(p.len_sum + g);
                ep_ret = __ldcg(p.ep_ret + g); ret_sum = __ldcg(p.ret_sum + g);
            }
            const float sigma = sigma_in >= 0.0f ? sigma_in : p.rewardC[7];
            float Cr[7];  // reward weights, in registers for the whole unit
#pragma unroll
            for (int i = 0; i < 7; ++i) Cr[i] = __ldcg(p.rewardC + i);
            float amax = 0.0f;
            // tracking: this env's cycle time and the flight's running sums; ep_index holds
            // the flight's state (1 while it lasts)
            float Tp = 1.0f;
            double e3 = 0.0, exy = 0.0;
            int n_ok = 0;
            bool alive = false;
            if constexpr (TRACK) {
                if (active) {
                    Tp = __ldcg(tr.period + g);
                    e3 = __ldcg(tr.sq_err + g);
                    exy = __ldcg(tr.sq_err + ld + g);
                    n_ok = __ldcg(tr.steps_ok + g);
                    alive = ep_index != 0u;
                }
                if (!(Tp > 0.0f && isfinite(Tp))) {
                    Tp = 1.0f;
                    alive = false;
                }
            }
            const Target tg = make_target(C.dt, Tp, tr.amp);
            // action ring: slot (t0 - i) mod 16 holds a_{t0-i} (global history is newest first);
            // slot k = ring columns 2k, 2k + 1 (packed halves), after the 16 observation columns
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                uint32_t vh[16], vl[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    float x[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int el = 32 * q + 2 * c + e;  // element inside the ring
                        const int sl = el >> 2, cc = el & 3;
                        const int i0 = (int)((t0u - (uint32_t)sl) & 15u);
                        const int i = i0 == 0 ? 16 : i0;
                        x[e] = 0.0f;
                        if (active && i <= nh) x[e] = __ldcg(p.hist + (4 * (i - 1) + cc) * ld + g);
                    }
                    split2(x[0], x[1], vh[c], vl[c], amax);
                }
                st16(tl + T_AHI + 16 + 16 * q, vh);
                st16(tl + T_ALO + 16 + 16 * q, vl);
            }
            int64_t slot = capacity > 0 ? headu % capacity : 0;
            const int F = C.F;

#pragma unroll 1
            for (int tt = 0; tt < Tu; ++tt) {
                const uint32_t t = t0u + (uint32_t)tt;
                float a[4];
                if ((int64_t)t < (int64_t)C.learning_starts) {
                    const uint4 rr = draw(C, (uint32_t)g, t, TAG_WARM, 0);
                    a[0] = 2.0f * u01(rr.x) - 1.0f;
                    a[1] = 2.0f * u01(rr.y) - 1.0f;
                    a[2] = 2.0f * u01(rr.z) - 1.0f;
                    a[3] = 2.0f * u01(rr.w) - 1.0f;
                } else {
                    // ---------------- observation -> A elements 0..31 (hi / lo); hand over
                    {
                        float o[32];
                        obs_state(s, o);
                        if constexpr (TRACK) {
                            float pr[3], vr[3];
                            lissajous((int)t, tg, tr.amp, tr.z0, pr, vr);
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                o[k] = clampf(o[k] - pr[k], -tr.clip_p, tr.clip_p);
                                o[12 + k] = clampf(o[12 + k] - vr[k], -tr.clip_v, tr.clip_v);
                            }
                        }
                        if (C.any_noise) {
                            float nz[18];
                            obs_noise(C, (uint32_t)g, t, nz);
#pragma unroll
                            for (int k = 0; k < 18; ++k) o[k] += nz[k];
                        }
                        o[18] = 1.0f;  // bias input of layer 1
#pragma unroll
                        for (int k = 19; k < 32; ++k) o[k] = 0.0f;
                        uint32_t vh[16], vl[16];
#pragma unroll
                        for (int c = 0; c < 16; ++c) split2(o[2 * c], o[2 * c + 1], vh[c], vl[c], amax);
                        st16(tl + T_AHI, vh);
                        st16(tl + T_ALO, vl);
                        wait_st();
                    }
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_a1);
                    // ---------------- while layer 1 runs: exploration noise
                    float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    if (sigma > 0.0f) {
                        const uint4 r0 = draw(C, (uint32_t)g, t, TAG_EXPL, 0);
                        const uint4 r1 = draw(C, (uint32_t)g, t, TAG_EXPL, 1);
                        z[0] = gauss(r0.x, r0.y); z[1] = gauss(r0.z, r0.w);
                        z[2] = gauss(r1.x, r1.y); z[3] = gauss(r1.z, r1.w);
                    }
                    if (!warp_wait(bar_d1, ph, abort_flag, p.status, C.wait_limit)) break;
                    fence_after();
                    // ---------------- epilogue 1: bias, ReLU, split -> A2 (shared memory); hand over
#pragma unroll 1
                    for (int c0 = 0; c0 < H; c0 += 32) {
                        uint32_t v[32];
                        ld16x2(tl + T_D + c0, v, tl + T_D + c0 + 16, v + 16);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {  // 8 hidden units = one 16-byte core-matrix row
                            uint32_t hv[4], lv[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float x0 = fmaxf(__uint_as_float(v[8 * q + 2 * e]), 0.0f);
                                const float x1 = fmaxf(__uint_as_float(v[8 * q + 2 * e + 1]), 0.0f);
                                split2(x0, x1, hv[e], lv[e], amax);
                            }
                            const int off = cano16(r, c0 + 8 * q, KC2);
                            *reinterpret_cast<uint4*>(A2hi + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                            *reinterpret_cast<uint4*>(A2lo + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_a2);
                    if (!warp_wait(bar_d2, ph, abort_flag, p.status, C.wait_limit)) break;
                    fence_after();
                    ph ^= 1u;
                    // ---------------- epilogue 2 + output layer (64 -> 4), tanh
                    // hidden units in pairs (2i, 2i+1): bias and FMAs as f32x2; acc[o] holds the
                    // even- and odd-unit partial sums of output o, added at the end
                    unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
                    const unsigned long long* b2p = reinterpret_cast<const unsigned long long*>(sB2);
                    const unsigned long long* w3p = reinterpret_cast<const unsigned long long*>(sW3);
#pragma unroll 1
                    for (int c0 = 0; c0 < H; c0 += 32) {
                        uint32_t v[32];
                        ld16x2(tl + T_D + c0, v, tl + T_D + c0 + 16, v + 16);
#pragma unroll
                        for (int e = 0; e < 32; e += 2) {
                            const int i = (c0 + e) >> 1;
                            const unsigned long long z2 = f2add(f2pack(__uint_as_float(v[e]), __uint_as_float(v[e + 1])), b2p[i]);
                            float h0, h1;
                            f2unpack(z2, h0, h1);
                            const unsigned long long hh = f2pack(fmaxf(h0, 0.0f), fmaxf(h1, 0.0f));
                            const ulonglong2 w01 = reinterpret_cast<const ulonglong2*>(w3p)[2 * i];
                            const ulonglong2 w23 = reinterpret_cast<const ulonglong2*>(w3p)[2 * i + 1];
                            acc[0] = f2fma(w01.x, hh, acc[0]);
                            acc[1] = f2fma(w01.y, hh, acc[1]);
                            acc[2] = f2fma(w23.x, hh, acc[2]);
                            acc[3] = f2fma(w23.y, hh, acc[3]);
                        }
                    }
                    float pp[4];
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        float ev, od;
                        f2unpack(acc[o], ev, od);
                        pp[o] = ev + od;
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
                motor_lag_off(C, u, s2);
                rk4(C.veh, C.dt, C.renorm, s2, u, P, d);
                const float rw = reward(Cr, s2, a);
                const bool term = !TRACK && terminated(C, s2);
                const uint32_t ep_after = ep_step + 1;
                const bool trunc = !TRACK && !term && (int)ep_after >= C.episode_len;
                if constexpr (TRACK) {
                    // error against the target at the new time; a non-finite state or an error
                    // outside the termination box ends the flight (the lane then holds its
                    // last state while its tile finishes the steps)
                    float pr[3], vr[3];
                    lissajous((int)t + 1, tg, tr.amp, tr.z0, pr, vr);
                    const float ex = s2[0] - pr[0], ey = s2[1] - pr[1], ez = s2[2] - pr[2];
                    const bool crash = !finite_state(s2) || fabsf(ex) > C.term_pos ||
                                       fabsf(ey) > C.term_pos || fabsf(ez) > C.term_pos;
                    if (alive && crash) alive = false;
                    if (alive) {
                        const double exy2 = (double)ex * ex + (double)ey * ey;
                        exy += exy2;
                        e3 += exy2 + (double)ez * ez;
                        n_ok += 1;
                    }
                }
                // ---------------- transition record (field-major, streaming stores)
                if (capacity > 0) {
                    if (active && in_bounds(p.status, slot, p.rows, SITE_RING_WRITE) &&
                        in_bounds(p.status, g, ld, SITE_SOA)) {
                        float* rec = p.rec + (size_t)slot * F * ld + g;
#pragma unroll
                        for (int i = 0; i < NS; ++i) __stcs(rec + i * ld, s[i]);
#pragma unroll
                        for (int i = 0; i < 4; ++i) __stcs(rec + (17 + i) * ld, a[i]);
                        __stcs(rec + 21 * ld, rw);
                        __stcs(rec + 22 * ld, __uint_as_float(pack_flags(term, trunc, ep_step)));
                        if (C.n_priv) {
                            float pv[NPRIV];
                            priv_vals(C, P, d, pv);
#pragma unroll
                            for (int k = 0; k < NPRIV; ++k) __stcs(rec + (23 + k) * ld, pv[k]);
                        }
                        if (term || trunc) {
                            float* sd = p.side + ((size_t)slot * ld + g) * NS;
#pragma unroll
                            for (int i = 0; i < NS; ++i) __stcs(sd + i, s2[i]);
                        }
                    }
                    slot = (slot + 1 == capacity) ? 0 : slot + 1;
                }
                // ---------------- action ring: a_t into slot t mod 16; an episode end clears the ring
                const bool reset = term || trunc;
                const int hs = (int)(t & 15u);
                if (!__any_sync(0xffffffffu, reset)) {
                    uint32_t h0, h1, l0, l1;
                    split2(a[0], a[1], h0, l0, amax);
                    split2(a[2], a[3], h1, l1, amax);
                    st2(tl + T_AHI + 16 + 2 * hs, h0, h1);
                    st2(tl + T_ALO + 16 + 2 * hs, l0, l1);
                } else {
                    // some lane of the warp starts a new episode: rewrite the ring words (kept as
                    // they are, slot hs <- a_t, all zero for the lanes that reset)
                    uint32_t h0, h1, l0, l1;
                    split2(a[0], a[1], h0, l0, amax);
                    split2(a[2], a[3], h1, l1, amax);
#pragma unroll 1
                    for (int q = 0; q < 2; ++q) {
                        uint32_t vh[16], vl[16];
                        ld16x2(tl + T_AHI + 16 + 16 * q, vh, tl + T_ALO + 16 + 16 * q, vl);
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const int sl = (32 * q + 2 * c) >> 2;  // both halves of column c share a slot
                            if (sl == hs) { vh[c] = (c & 1) ? h1 : h0; vl[c] = (c & 1) ? l1 : l0; }
                            if (reset) { vh[c] = 0u; vl[c] = 0u; }
                        }
                        st16(tl + T_AHI + 16 + 16 * q, vh);
                        st16(tl + T_ALO + 16 + 16 * q, vl);
                    }
                }
                ep_ret += rw;
                // Episode starts (reset_env) depend only on (env, episode index), so each
                // thread's next one is computed ahead: a thread that resets takes its
                // precomputed start if it has one, else computes it now; after a unit's first
                // step (and every NX_EVERY steps) the threads without a precomputed start
                // compute their next one, together in one pass of the warp, so the first
                // reset of each env in a unit no longer makes the whole warp run reset_env.
                // (The sync below takes a value every lane has already computed.)
                bool now = false;
                if (reset) {
                    n_done += 1;
                    len_sum += ep_after;
                    ret_sum += ep_ret;
                    ep_index += 1;
                    if (nxt_ok) {
#pragma unroll
                        for (int i = 0; i < NS; ++i) s[i] = nx[i * NX_LD];
                        P = make_prm(nx[NS * NX_LD], nx[(NS + 1) * NX_LD], nx[(NS + 2) * NX_LD], nx[(NS + 3) * NX_LD],
                                     nx[(NS + 4) * NX_LD], nx[(NS + 5) * NX_LD], nx[(NS + 6) * NX_LD]);
#pragma unroll
                        for (int i = 0; i < 6; ++i) d[i] = nx[(NS + 7 + i) * NX_LD];
                        nxt_ok = false;
                    } else {
                        now = true;
                    }
                    ep_step = 0;
                    ep_ret = 0.0f;
                } else {
                    if (!TRACK || alive) {
#pragma unroll
                        for (int i = 0; i < NS; ++i) s[i] = s2[i];
                    }
                    ep_step = ep_after;
                }
                if constexpr (!TRACK) {
                    const bool fill = !now && !nxt_ok && active &&
                                      (tt == 0 || (t & (uint32_t)(NX_EVERY - 1)) == (uint32_t)(NX_EVERY - 1));
                    if (__any_sync(0xffffffffu, now || fill)) {
                        if (now || fill) {
                            float sn[NS], prm7[7], dn[6];
                            reset_env(C, (uint32_t)g, now ? ep_index : ep_index + 1u, sn, prm7, dn);
                            if (now) {
#pragma unroll
                                for (int i = 0; i < NS; ++i) s[i] = sn[i];
                                P = make_prm(prm7[0], prm7[1], prm7[2], prm7[3], prm7[4], prm7[5], prm7[6]);
#pragma unroll
                                for (int i = 0; i < 6; ++i) d[i] = dn[i];
                            } else {
#pragma unroll
                                for (int i = 0; i < NS; ++i) nx[i * NX_LD] = sn[i];
#pragma unroll
                                for (int i = 0; i < 7; ++i) nx[(NS + i) * NX_LD] = prm7[i];
#pragma unroll
                                for (int i = 0; i < 6; ++i) nx[(NS + 7 + i) * NX_LD] = dn[i];
                                nxt_ok = true;
                            }
                        }
                    }
                }
            }
            wait_st();
            const bool bad = !(amax < HALF_MAX);  // also catches a NaN that reached an operand
            if (__any_sync(0xffffffffu, bad) && lane == 0 && active && p.status) atomicCAS(p.status, DEV_OK, DEV_RANGE);

            if constexpr (TRACK) {
                if (active) {
                    tr.sq_err[g] = e3;
                    tr.sq_err[ld + g] = exy;
                    tr.steps_ok[g] = n_ok;
                }
                ep_index = alive ? 1u : 0u;
            }
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
            const uint32_t t_end = t0u + (uint32_t)Tu;
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                uint32_t vh[16], vl[16];
                ld16x2(tl + T_AHI + 16 + 16 * q, vh, tl + T_ALO + 16 + 16 * q, vl);
                if (active) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float2 x = join2(vh[c], vl[c]);
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int el = 32 * q + 2 * c + e;
                            const int sl = el >> 2, cc = el & 3;
                            const int i0 = (int)((t_end - (uint32_t)sl) & 15u);
                            const int i = i0 == 0 ? 16 : i0;  // lag of slot sl after the last step
                            if (i <= nh) p.hist[(4 * (i - 1) + cc) * ld + g] = e ? x.y : x.x;
                        }
                    }
                }
            }
        }
        // ---- unit done: publish it for the next chunk of this group
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0 && sched) {
            __threadfence();
            asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(sched + 1 + ug), "r"(uk + 1) : "memory");
        }
    }
    // on an abort, let the last committed MMA batch finish before the memory is released
    if (mma_warp && *abort_flag && lane == 0 && issued) {
        const uint32_t b = issued == 1 ? bar_d1 : bar_d2;
        const uint32_t par = issued == 1 ? ph : ph ^ 1u;
        for (int i = 0; i < WAIT_LIMIT; ++i) {
            uint32_t done;
            asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                         "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(b), "r"(par) : "memory");
            if (done) break;
        }
    }
    // ---- release tensor memory
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == NCW)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(*tslot), "r"(T_ALLOC) : "memory");
}

// Launches T steps on env warps [w0, w1) (12 env warps = 384 envs per CTA, plus 3 MMA warps):
// one CTA per group of 12 warps, or, with chunk > 0 and `sched` (1 + groups ints of device
// memory), a persistent grid of at most one CTA per SM walking (group, chunk) units.
qsim_status launch_rollout_tc_range(qsim_handle* h, const float* actor, int T, uint32_t t0, int64_t head,
                                    float sigma, int w0, int w1, cudaStream_t st, int chunk, int* sched) {
    static bool configured = false;
    if (!configured) {
        QCHECK_CUDA(cudaFuncSetAttribute(k_rollout_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        configured = true;
    }
    const int groups = (w1 - w0 + NCW - 1) / NCW;
    if (sched && chunk > 0) {
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        QCHECK_CUDA(cudaMemsetAsync(sched, 0, sizeof(int) * (size_t)(1 + groups), st));
        const int grid = std::min(sms, groups);
        k_rollout_tc<false><<<grid, NT, SMEM, st>>>(h->dc, h->p, actor, T, t0, head, h->capacity, sigma, w0, w1,
                                                    groups, std::min(chunk, T), sched, TrackArgs{});
    } else {
        k_rollout_tc<false><<<groups, NT, SMEM, st>>>(h->dc, h->p, actor, T, t0, head, h->capacity, sigma, w0, w1,
                                                      groups, T, nullptr, TrackArgs{});
    }
    QCHECK_LAUNCH("k_rollout_tc");
    return QSIM_OK;
}

// Start of every flight of a tracking call: on the target with its velocity, level, not
// rotating, motors at the env's hover speed, empty action history, running sums zero;
// ep_index = 1 marks a flight with a valid cycle time.
__global__ void k_track_init(EnvCfg C, EnvPtrs p, TrackArgs tr) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int ld = C.ld;
    if (g >= ld) return;
    float Tp = tr.period[g];
    const bool ok = Tp > 0.0f && isfinite(Tp);
    if (!ok) Tp = 1.0f;
    float pr[3], vr[3];
    lissajous(0, make_target(C.dt, Tp, tr.amp), tr.amp, tr.z0, pr, vr);
    const float m = p.prm[g], kf = p.prm[4 * ld + g];
    const float hover = clampf(sqrtf(m * C.veh.g / (4.0f * kf)), C.veh.rpm_min, C.veh.rpm_max);
    float s[NS];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        s[i] = pr[i];
        s[7 + i] = vr[i];
        s[10 + i] = 0.0f;
    }
    s[3] = 1.0f; s[4] = 0.0f; s[5] = 0.0f; s[6] = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) s[13 + i] = hover;
#pragma unroll
    for (int i = 0; i < NS; ++i) p.state[i * ld + g] = s[i];
    for (int i = 0; i < 4 * HMAX; ++i) p.hist[i * ld + g] = 0.0f;
    p.ep_index[g] = ok ? 1u : 0u;
    p.ep_step[g] = 0u; p.n_done[g] = 0u; p.len_sum[g] = 0u;
    p.ep_ret[g] = 0.0f; p.ret_sum[g] = 0.0f;
    tr.sq_err[g] = 0.0;
    tr.sq_err[ld + g] = 0.0;
    tr.steps_ok[g] = 0;
}

// Tracking flight of every env on the tensor-core kernel (hidden 64): the flights' states,
// rings and flags live in scratch allocated on the stream for this call (the env set is
// only read: its parameters and disturbances are copied), no observation noise, no
// exploration, no warm-up; persistent schedule in chunks of `chunk` steps.
qsim_status launch_track_tc(qsim_handle* h, const float* actor, int T, const TrackArgs& tr, int chunk,
                            cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        QCHECK_CUDA(cudaFuncSetAttribute(k_rollout_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        configured = true;
    }
    const int ld = h->ld, warps = ld / 32;
    const int groups = (warps + NCW - 1) / NCW;
    const size_t n = (size_t)ld;
    float* scr = nullptr;
    QCHECK_CUDA(cudaMallocAsync((void**)&scr, sizeof(float) * (n * (NS + 8 + 6 + 4 * HMAX + 6) + 1 + groups), st));
    EnvPtrs p = h->p;
    p.state = scr;
    p.prm = p.state + NS * n;
    p.dist = p.prm + 8 * n;
    p.hist = p.dist + 6 * n;
    p.ep_index = reinterpret_cast<uint32_t*>(p.hist + 4 * HMAX * n);
    p.ep_step = p.ep_index + n;
    p.n_done = p.ep_step + n;
    p.len_sum = p.n_done + n;
    p.ep_ret = reinterpret_cast<float*>(p.len_sum + n);
    p.ret_sum = p.ep_ret + n;
    int* sched = reinterpret_cast<int*>(p.ret_sum + n);  // this call's unit counters
    p.rec = nullptr;
    p.side = nullptr;
    QCHECK_CUDA(cudaMemcpyAsync(p.prm, h->p.prm, sizeof(float) * 8 * n, cudaMemcpyDeviceToDevice, st));
    QCHECK_CUDA(cudaMemcpyAsync(p.dist, h->p.dist, sizeof(float) * 6 * n, cudaMemcpyDeviceToDevice, st));
    EnvCfg C = h->dc;
    C.learning_starts = 0;
    C.any_noise = 0;
    k_track_init<<<(ld + 127) / 128, 128, 0, st>>>(C, p, tr);
    QCHECK_LAUNCH("k_track_init");
    if (T > 0) {
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        QCHECK_CUDA(cudaMemsetAsync(sched, 0, sizeof(int) * (size_t)(1 + groups), st));
        k_rollout_tc<true><<<std::min(sms, groups), NT, SMEM, st>>>(C, p, actor, T, 0u, 0, 0, 0.0f, 0, warps,
                                                                     groups, std::min(chunk, T), sched, tr);
        QCHECK_LAUNCH("k_rollout_tc<track>");
    }
    QCHECK_CUDA(cudaFreeAsync(scr, st));
    return QSIM_OK;
}

// Env warps per CTA of the tensor-core kernel (one CTA per SM).
int rollout_tc_warps_per_cta() { return NCW; }

// ------------------------------------------------------------------ MMA issue-rate probe
// One CTA: n_warps warps, lane 0 of each issues n_mma tcgen05.mma (kind::f16, M 128, N =
// n_cols / n_warps, K 16, A in TMEM, zero operands) into its own accumulator columns, then
// commits; cycles from the first issue to the completion of every chain -> out[0].
__global__ void __launch_bounds__(128) k_mma_probe(int n_mma, int n_cols, int n_warps, long long* out) {
    extern __shared__ __align__(1024) unsigned char smb[];
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smb + 16384);
    const uint32_t bar = smem_addr(smb + 16384 + 64);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 16384 / 4; i += blockDim.x) reinterpret_cast<float*>(smb)[i] = 0.0f;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(n_warps));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_addr(tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tm = *tslot;
    const int N = n_cols / n_warps;
    const long long c0 = clock64();
    if (warp < n_warps && lane == 0) {
        const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TILE >> 4) << 24);
        const uint64_t b = sdesc(smem_addr(smb), 2);  // N rows x 16 halves, zeros
        for (int i = 0; i < n_mma; ++i)
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}"
                         :: "r"(tm + (uint32_t)(warp * N)), "r"(tm + 256u), "l"(b), "r"(idesc), "r"((uint32_t)i));
        mma_commit(bar);
    }
    if (threadIdx.x == 0) {
        bool ok = false;
        for (int i = 0; i < WAIT_LIMIT && !ok; ++i) {
            uint32_t done;
            asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                         "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar) : "memory");
            ok = done != 0;
        }
        out[0] = ok ? clock64() - c0 : -1;
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tm) : "memory");
}

}  // namespace qsim

extern "C" qsim_status qsim_mma_probe(int32_t n_mma, int32_t n_cols, int32_t n_warps, int64_t* cycles,
                                      void* stream) {
    using namespace qsim;
    if (!cycles || n_mma < 1 || n_mma > 4096 || n_warps < 1 || n_warps > 4 || n_cols < 16 * n_warps ||
        n_cols > 256 || (n_cols / n_warps) % 16 != 0 || n_cols % n_warps != 0)
        return fail(QSIM_EINVAL, "qsim_mma_probe: bad arguments");
    k_mma_probe<<<1, 128, 16384 + 128, (cudaStream_t)stream>>>(n_mma, n_cols, n_warps,
                                                                reinterpret_cast<long long*>(cycles));
    QCHECK_LAUNCH("k_mma_probe");
    return QSIM_OK;
}
