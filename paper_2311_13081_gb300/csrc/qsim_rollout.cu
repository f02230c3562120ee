// qsim_rollout.cu -- fused env-step kernel: actor MLP + exploration + RK4 + reward +
// termination + reset + replay write, for n_steps steps with the state in registers.
//
// Work decomposition (one warp = 32 envs, warps fully independent after the weights are
// staged):
//   * dynamics, observation, reward, bookkeeping: lane l owns env 32*w + l, its 17-D
//     state, parameters and counters stay in registers across all steps.
//   * actor layers 1 and 2 (obs_dim -> H -> H): a register-blocked SIMT outer product per
//     warp.  Lane (tx = l >> 3, ty = l & 7) computes H/8 outputs (ty's slice) for 8 envs
//     (tx's slice): per k it loads H/8 weights and 8 activations with 128-bit shared
//     loads and issues H FFMA.  Weights are stored transposed and interleaved so that the
//     8 ty-lanes hit 8 distinct bank quads; hidden activations are stored with an XOR
//     swizzle of the bank quad so that the ty-lanes' stores are conflict free.
//   * actor layer 3 (H -> 4): each lane forms partial sums of its H/8 hidden units for
//     4 outputs x 8 envs and a 3-stage butterfly reduce-scatter over the ty-lanes leaves
//     lane l with the 4 pre-activations of ITS OWN env (env 8*tx + ty == l).
//   * action history: a 16-slot ring in shared memory (rows 18 + 4*slot of the obs tile),
//     slot of a_t = t mod 16; the first layer reads it in rotated order, so no data moves.
// Shared memory: actor weights once per CTA + per warp an obs tile [82][32] and a hidden
// tile [H][32].  Replay records go out as field-major streaming stores, 128 B per warp per
// field.
//
// The same kernel, instantiated with TRACK = true, flies the deterministic actor along the
// figure-eight target of Sec. V ("Trajectory tracking") instead: the observation's
// position and velocity are offset by the target's and clipped, and the squared tracking
// error is accumulated; there is no exploration, reward, replay write or reset.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "qsim_internal.h"

namespace qsim {

template <int H>
struct RollLayout {
    static constexpr int OBS_MAX = 18 + 4 * HMAX;  // 82
    static constexpr int W1 = 0;
    static constexpr int B1 = W1 + OBS_MAX * H;
    static constexpr int W2 = B1 + H;
    static constexpr int B2 = W2 + H * H;
    static constexpr int W3 = B2 + H;      // transposed [H][4]
    static constexpr int B3 = W3 + 4 * H;
    static constexpr int WEIGHTS = ((B3 + 4) + 3) & ~3;
    static constexpr int OBS = OBS_MAX * 32;
    static constexpr int HID = H * 32;
    static constexpr int PER_WARP = OBS + HID;
    static size_t bytes(int nw) { return sizeof(float) * (size_t)(WEIGHTS + nw * PER_WARP); }
};

// Position of output o of an H-wide layer inside a transposed weight row: lane-group
// ty = o / (H/8) owns H/8 consecutive outputs, stored as (H/32) float4 chunks that are
// interleaved across the 8 groups.
template <int H>
__device__ __forceinline__ int wpos(int o) {
    constexpr int OP = H / 8;
    const int ty = o / OP, r = o % OP;
    return (r >> 2) * 32 + ty * 4 + (r & 3);
}

template <int H, int NW, bool PK, bool TRACK = false>
__global__ void __launch_bounds__(NW * 32) k_rollout(EnvCfg C, EnvPtrs p,
                                                     const float* __restrict__ actor, int T,
                                                     uint32_t t0, int64_t head0,
                                                     int64_t capacity, float sigma_in,
                                                     int warp0, int warp_end, TrackArgs tr) {
    using L = RollLayout<H>;
    constexpr int OP = H / 8;  // outputs per lane
    constexpr int NQ = OP / 4; // float4 chunks per lane per weight row
    extern __shared__ __align__(16) float smem[];
    const int DA = C.obs_dim;
    const int ld = C.ld;

    // ---- stage the actor weights (canonical W1[H][DA] b1 W2[H][H] b2 W3[4][H] b3)
    {
        float* sW1 = smem + L::W1;
        float* sW2 = smem + L::W2;
        const float* gW1 = actor;
        const float* gb1 = gW1 + H * DA;
        const float* gW2 = gb1 + H;
        const float* gb2 = gW2 + H * H;
        const float* gW3 = gb2 + H;
        const float* gb3 = gW3 + 4 * H;
        for (int i = threadIdx.x; i < H * DA; i += NW * 32) {
            const int o = i / DA, k = i - o * DA;
            sW1[k * H + wpos<H>(o)] = gW1[i];
        }
        for (int i = threadIdx.x; i < H * H; i += NW * 32) {
            const int o = i / H, k = i - o * H;
            sW2[k * H + wpos<H>(o)] = gW2[i];
        }
        for (int i = threadIdx.x; i < H; i += NW * 32) {
            smem[L::B1 + i] = gb1[i];
            smem[L::B2 + i] = gb2[i];
        }
        for (int i = threadIdx.x; i < 4 * H; i += NW * 32) {
            const int j = i / H, k = i - j * H;
            smem[L::W3 + k * 4 + j] = gW3[i];
        }
        if (threadIdx.x < 4) smem[L::B3 + threadIdx.x] = gb3[threadIdx.x];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = warp0 + blockIdx.x * NW + warp;  // global warp (32 envs)
    const int g = gw * 32 + lane;                      // global env index
    if (gw >= warp_end) return;                        // warp-uniform
    const int tx = lane >> 3, ty = lane & 7;
    float* sObs = smem + L::WEIGHTS + warp * L::PER_WARP;
    float* sHid = sObs + L::OBS;
    const float* sW1 = smem + L::W1;
    const float* sW2 = smem + L::W2;
    const float* sW3 = smem + L::W3;

    // ---- per-env state into registers
    float s[NS], d[6];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = p.state[i * ld + g];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = p.dist[i * ld + g];
    Prm P = make_prm(p.prm[g], p.prm[ld + g], p.prm[2 * ld + g], p.prm[3 * ld + g],
                     p.prm[4 * ld + g], p.prm[5 * ld + g], p.prm[6 * ld + g]);
    // tracking: start on the target with its velocity, level, not rotating, motors at this
    // env's hover speed, empty action history
    Target tg{1.0, 0.0f};
    double e3 = 0.0, exy = 0.0;
    int n_ok = 0;
    bool alive = true;
    if constexpr (TRACK) {
        const float Tp = tr.period[g];
        alive = Tp > 0.0f && isfinite(Tp);
        tg = make_target(C.dt, alive ? Tp : 1.0f, tr.amp);
        float pr[3], vr[3];
        lissajous(0, tg, tr.amp, tr.z0, pr, vr);
        const float hover = clampf(sqrtf(P.m * C.veh.g / (4.0f * P.kf)), C.veh.rpm_min, C.veh.rpm_max);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            s[i] = pr[i];
            s[7 + i] = vr[i];
            s[10 + i] = 0.0f;
        }
        s[3] = 1.0f; s[4] = 0.0f; s[5] = 0.0f; s[6] = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) s[13 + i] = hover;
    }
    uint32_t ep_index = p.ep_index[g], ep_step = p.ep_step[g];
    uint32_t n_done = p.n_done[g], len_sum = p.len_sum[g];
    float ep_ret = p.ep_ret[g], ret_sum = p.ret_sum[g];
    float Cr[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Cr[i] = p.rewardC[i];
    const float sigma = sigma_in >= 0.0f ? sigma_in : p.rewardC[7];
    const int nh = C.n_hist;
    if constexpr (TRACK) {
        for (int k = 18; k < 18 + 4 * HMAX; ++k) sObs[k * 32 + lane] = 0.0f;
    } else
    // history (newest first in global) -> ring slot (t0 - i) mod 16
    for (int i = 1; i <= nh; ++i) {
        const int slot = (int)((t0 - (uint32_t)i) & 15u);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            sObs[(18 + 4 * slot + c) * 32 + lane] = p.hist[(4 * (i - 1) + c) * ld + g];
    }
    int64_t slot = capacity > 0 ? head0 % capacity : 0;
    const int F = C.F;
    __syncwarp();

    for (int tt = 0; tt < T; ++tt) {
        const uint32_t t = t0 + (uint32_t)tt;
        {
            float o[18];
            obs_state(s, o);
            if constexpr (TRACK) {
                float pr[3], vr[3];
                lissajous(tt, tg, tr.amp, tr.z0, pr, vr);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    o[k] = clampf(o[k] - pr[k], -tr.clip_p, tr.clip_p);
                    o[12 + k] = clampf(o[12 + k] - vr[k], -tr.clip_v, tr.clip_v);
                }
            } else if (C.any_noise) {
                float nz[18];
                obs_noise(C, (uint32_t)g, t, nz);
#pragma unroll
                for (int k = 0; k < 18; ++k) o[k] += nz[k];
            }
#pragma unroll
            for (int k = 0; k < 18; ++k) sObs[k * 32 + lane] = o[k];
        }
        __syncwarp();
        float a[4];
        if (!TRACK && (int64_t)t < (int64_t)C.learning_starts) {
            const uint4 r = draw(C, (uint32_t)g, t, TAG_WARM, 0);
            a[0] = 2.0f * u01(r.x) - 1.0f;
            a[1] = 2.0f * u01(r.y) - 1.0f;
            a[2] = 2.0f * u01(r.z) - 1.0f;
            a[3] = 2.0f * u01(r.w) - 1.0f;
        } else {
            // ---------------- layer 1: obs (DA) -> H, ReLU
            float acc[OP][8];
            if constexpr (PK) {
                // paired FMAs: acc2[q][e] holds outputs (2q, 2q+1) of env e; weight pairs come
                // straight from the 128-bit shared loads, activations are duplicated
                unsigned long long acc2[OP / 2][8];
#pragma unroll
                for (int q = 0; q < OP / 2; ++q) {
                    const unsigned long long b = f2pack(smem[L::B1 + ty * OP + 2 * q],
                                                        smem[L::B1 + ty * OP + 2 * q + 1]);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc2[q][e] = b;
                }
                auto fma_row2 = [&](const float* wrow, const float* xrow) {
                    unsigned long long w2[OP / 2];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float4 v = *reinterpret_cast<const float4*>(wrow + q * 32 + ty * 4);
                        w2[2 * q] = f2pack(v.x, v.y);
                        w2[2 * q + 1] = f2pack(v.z, v.w);
                    }
                    const float4 x0 = *reinterpret_cast<const float4*>(xrow + 8 * tx);
                    const float4 x1 = *reinterpret_cast<const float4*>(xrow + 8 * tx + 4);
                    const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const unsigned long long xb = f2pack(x[e], x[e]);
#pragma unroll
                        for (int q = 0; q < OP / 2; ++q) acc2[q][e] = f2fma(w2[q], xb, acc2[q][e]);
                    }
                };
#pragma unroll 2
                for (int k = 0; k < 18; ++k) fma_row2(sW1 + k * H, sObs + k * 32);
                for (int i = 1; i <= nh; ++i) {
                    const int base = 18 + 4 * (int)((t - (uint32_t)i) & 15u);
                    const int kw = 18 + 4 * (i - 1);
#pragma unroll
                    for (int c = 0; c < 4; ++c) fma_row2(sW1 + (kw + c) * H, sObs + (base + c) * 32);
                }
#pragma unroll
                for (int q = 0; q < OP / 2; ++q)
#pragma unroll
                    for (int e = 0; e < 8; ++e) f2unpack(acc2[q][e], acc[2 * q][e], acc[2 * q + 1][e]);
            } else {
#pragma unroll
            for (int i = 0; i < OP; ++i) {
                const float b = smem[L::B1 + ty * OP + i];
#pragma unroll
                for (int e = 0; e < 8; ++e) acc[i][e] = b;
            }
            auto fma_row = [&](const float* wrow, const float* xrow) {
                float w[OP];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 v = *reinterpret_cast<const float4*>(wrow + q * 32 + ty * 4);
                    w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
                }
                const float4 x0 = *reinterpret_cast<const float4*>(xrow + 8 * tx);
                const float4 x1 = *reinterpret_cast<const float4*>(xrow + 8 * tx + 4);
                const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int i = 0; i < OP; ++i)
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[i][e] = fmaf(w[i], x[e], acc[i][e]);
            };
#pragma unroll 2
            for (int k = 0; k < 18; ++k) fma_row(sW1 + k * H, sObs + k * 32);
            for (int i = 1; i <= nh; ++i) {
                const int base = 18 + 4 * (int)((t - (uint32_t)i) & 15u);
                const int kw = 18 + 4 * (i - 1);
#pragma unroll
                for (int c = 0; c < 4; ++c) fma_row(sW1 + (kw + c) * H, sObs + (base + c) * 32);
            }
            }
#pragma unroll
            for (int i = 0; i < OP; ++i) {
                const int o = ty * OP + i;
                float* row = sHid + o * 32;
                const float4 v0 = make_float4(fmaxf(acc[i][0], 0.f), fmaxf(acc[i][1], 0.f),
                                              fmaxf(acc[i][2], 0.f), fmaxf(acc[i][3], 0.f));
                const float4 v1 = make_float4(fmaxf(acc[i][4], 0.f), fmaxf(acc[i][5], 0.f),
                                              fmaxf(acc[i][6], 0.f), fmaxf(acc[i][7], 0.f));
                *reinterpret_cast<float4*>(row + 4 * ((2 * tx) ^ ty)) = v0;
                *reinterpret_cast<float4*>(row + 4 * ((2 * tx + 1) ^ ty)) = v1;
            }
            __syncwarp();
            // ---------------- layer 2: H -> H, ReLU (in registers)
            if constexpr (PK) {
                unsigned long long acc2[OP / 2][8];
#pragma unroll
                for (int q = 0; q < OP / 2; ++q) {
                    const unsigned long long b = f2pack(smem[L::B2 + ty * OP + 2 * q],
                                                        smem[L::B2 + ty * OP + 2 * q + 1]);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc2[q][e] = b;
                }
#pragma unroll 2
                for (int k = 0; k < H; ++k) {
                    const float* wrow = sW2 + k * H;
                    const float* xrow = sHid + k * 32;
                    const int sw = (k / OP) & 7;
                    unsigned long long w2[OP / 2];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float4 v = *reinterpret_cast<const float4*>(wrow + q * 32 + ty * 4);
                        w2[2 * q] = f2pack(v.x, v.y);
                        w2[2 * q + 1] = f2pack(v.z, v.w);
                    }
                    const float4 x0 = *reinterpret_cast<const float4*>(xrow + 4 * ((2 * tx) ^ sw));
                    const float4 x1 = *reinterpret_cast<const float4*>(xrow + 4 * ((2 * tx + 1) ^ sw));
                    const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const unsigned long long xb = f2pack(x[e], x[e]);
#pragma unroll
                        for (int q = 0; q < OP / 2; ++q) acc2[q][e] = f2fma(w2[q], xb, acc2[q][e]);
                    }
                }
#pragma unroll
                for (int q = 0; q < OP / 2; ++q)
#pragma unroll
                    for (int e = 0; e < 8; ++e) f2unpack(acc2[q][e], acc[2 * q][e], acc[2 * q + 1][e]);
            } else {
#pragma unroll
            for (int i = 0; i < OP; ++i) {
                const float b = smem[L::B2 + ty * OP + i];
#pragma unroll
                for (int e = 0; e < 8; ++e) acc[i][e] = b;
            }
#pragma unroll 2
            for (int k = 0; k < H; ++k) {
                const float* wrow = sW2 + k * H;
                const float* xrow = sHid + k * 32;
                const int sw = (k / OP) & 7;
                float w[OP];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 v = *reinterpret_cast<const float4*>(wrow + q * 32 + ty * 4);
                    w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
                }
                const float4 x0 = *reinterpret_cast<const float4*>(xrow + 4 * ((2 * tx) ^ sw));
                const float4 x1 = *reinterpret_cast<const float4*>(xrow + 4 * ((2 * tx + 1) ^ sw));
                const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int i = 0; i < OP; ++i)
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[i][e] = fmaf(w[i], x[e], acc[i][e]);
            }
            }
            // ---------------- layer 3: H -> 4, partial over this lane's H/8 units
            float pp[4][8];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 8; ++e) pp[j][e] = 0.0f;
#pragma unroll
            for (int i = 0; i < OP; ++i) {
                const float4 w3 = *reinterpret_cast<const float4*>(sW3 + (ty * OP + i) * 4);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float h = fmaxf(acc[i][e], 0.0f);
                    pp[0][e] = fmaf(w3.x, h, pp[0][e]);
                    pp[1][e] = fmaf(w3.y, h, pp[1][e]);
                    pp[2][e] = fmaf(w3.z, h, pp[2][e]);
                    pp[3][e] = fmaf(w3.w, h, pp[3][e]);
                }
            }
            // butterfly reduce-scatter over ty: lane ends with env 8*tx + ty == lane
            float q4[4][4];
            {
                const bool hi = (ty & 4) != 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float send = hi ? pp[j][e] : pp[j][e + 4];
                        const float keep = hi ? pp[j][e + 4] : pp[j][e];
                        q4[j][e] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                    }
            }
            float q2[4][2];
            {
                const bool hi = (ty & 2) != 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float send = hi ? q4[j][e] : q4[j][e + 2];
                        const float keep = hi ? q4[j][e + 2] : q4[j][e];
                        q2[j][e] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                    }
            }
            float mu[4];
            {
                const bool hi = (ty & 1) != 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float send = hi ? q2[j][0] : q2[j][1];
                    const float keep = hi ? q2[j][1] : q2[j][0];
                    mu[j] = tanhf(keep + __shfl_xor_sync(0xffffffffu, send, 1) + smem[L::B3 + j]);
                }
            }
            if (!TRACK && sigma > 0.0f) {
                const uint4 r0 = draw(C, (uint32_t)g, t, TAG_EXPL, 0);
                const uint4 r1 = draw(C, (uint32_t)g, t, TAG_EXPL, 1);
                a[0] = clampf(fmaf(sigma, gauss(r0.x, r0.y), mu[0]), -1.0f, 1.0f);
                a[1] = clampf(fmaf(sigma, gauss(r0.z, r0.w), mu[1]), -1.0f, 1.0f);
                a[2] = clampf(fmaf(sigma, gauss(r1.x, r1.y), mu[2]), -1.0f, 1.0f);
                a[3] = clampf(fmaf(sigma, gauss(r1.z, r1.w), mu[3]), -1.0f, 1.0f);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) a[j] = clampf(mu[j], -1.0f, 1.0f);
            }
        }
        // ---------------- dynamics, reward, termination
        float u[4], s2[NS];
        action_to_rpm(C.veh, a, u);
#pragma unroll
        for (int i = 0; i < NS; ++i) s2[i] = s[i];
        motor_lag_off(C, u, s2);
        rk4(C.veh, C.dt, C.renorm, s2, u, P, d);
        if constexpr (TRACK) {
            // error against the target at the new time; a non-finite state or an error
            // outside the training termination box ends the flight (the lane then holds its
            // last state while its warp finishes the steps)
            float pr[3], vr[3];
            lissajous(tt + 1, tg, tr.amp, tr.z0, pr, vr);
            const float ex = s2[0] - pr[0], ey = s2[1] - pr[1], ez = s2[2] - pr[2];
            const bool crash = !finite_state(s2) || fabsf(ex) > C.term_pos ||
                               fabsf(ey) > C.term_pos || fabsf(ez) > C.term_pos;
            if (alive && crash) alive = false;
            if (alive) {
                const double exy2 = (double)ex * ex + (double)ey * ey;
                exy += exy2;
                e3 += exy2 + (double)ez * ez;
                n_ok += 1;
#pragma unroll
                for (int i = 0; i < NS; ++i) s[i] = s2[i];
            }
            if (nh > 0) {
                const int hs = 18 + 4 * (int)(t & 15u);
#pragma unroll
                for (int c = 0; c < 4; ++c) sObs[(hs + c) * 32 + lane] = a[c];
            }
            __syncwarp();
            continue;
        }
        const float r = reward(Cr, s2, a);
        const bool term = terminated(C, s2);
        const uint32_t ep_after = ep_step + 1;
        const bool trunc = !term && (int)ep_after >= C.episode_len;
        // ---------------- transition record (field-major, streaming stores)
        if (capacity > 0) {
            if (in_bounds(p.status, slot, p.rows, SITE_RING_WRITE) && in_bounds(p.status, g, ld, SITE_SOA)) {
                float* rec = p.rec + (size_t)slot * F * ld + g;
#pragma unroll
                for (int i = 0; i < NS; ++i) __stcs(rec + i * ld, s[i]);
#pragma unroll
                for (int i = 0; i < 4; ++i) __stcs(rec + (17 + i) * ld, a[i]);
                __stcs(rec + 21 * ld, r);
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
        if (nh > 0) {
            const int hs = 18 + 4 * (int)(t & 15u);
#pragma unroll
            for (int c = 0; c < 4; ++c) sObs[(hs + c) * 32 + lane] = a[c];
        }
        ep_ret += r;
        if (term || trunc) {
            n_done += 1;
            len_sum += ep_after;
            ret_sum += ep_ret;
            ep_index += 1;
            float prm7[7];
            reset_env(C, (uint32_t)g, ep_index, s, prm7, d);
            P = make_prm(prm7[0], prm7[1], prm7[2], prm7[3], prm7[4], prm7[5], prm7[6]);
            for (int k = 18; k < 18 + 4 * HMAX; ++k) sObs[k * 32 + lane] = 0.0f;
            ep_step = 0;
            ep_ret = 0.0f;
        } else {
#pragma unroll
            for (int i = 0; i < NS; ++i) s[i] = s2[i];
            ep_step = ep_after;
        }
        __syncwarp();
    }

    if constexpr (TRACK) {
        tr.sq_err[g] = e3;
        tr.sq_err[ld + g] = exy;
        tr.steps_ok[g] = n_ok;
        return;
    }
    // ---- write back
    const uint32_t t_end = t0 + (uint32_t)T;
#pragma unroll
    for (int i = 0; i < NS; ++i) p.state[i * ld + g] = s[i];
    p.prm[g] = P.m; p.prm[ld + g] = P.Jx; p.prm[2 * ld + g] = P.Jy; p.prm[3 * ld + g] = P.Jz;
    p.prm[4 * ld + g] = P.kf; p.prm[5 * ld + g] = P.km; p.prm[6 * ld + g] = P.tm;
#pragma unroll
    for (int i = 0; i < 6; ++i) p.dist[i * ld + g] = d[i];
    for (int i = 1; i <= nh; ++i) {
        const int sl = (int)((t_end - (uint32_t)i) & 15u);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            p.hist[(4 * (i - 1) + c) * ld + g] = sObs[(18 + 4 * sl + c) * 32 + lane];
    }
    p.ep_index[g] = ep_index; p.ep_step[g] = ep_step; p.ep_ret[g] = ep_ret;
    p.n_done[g] = n_done; p.len_sum[g] = len_sum; p.ret_sum[g] = ret_sum;
}

using RollFn = void (*)(EnvCfg, EnvPtrs, const float*, int, uint32_t, int64_t, int64_t, float,
                        int, int, TrackArgs);

template <int H, bool PK>
static RollFn pick(int nw) {
    switch (nw) {
        case 2: return k_rollout<H, 2, PK>;
        case 4: return k_rollout<H, 4, PK>;
        case 6: return k_rollout<H, 6, PK>;
        case 8: return k_rollout<H, 8, PK>;
        case 10: return k_rollout<H, 10, PK>;
        default: return nullptr;
    }
}

static RollFn roll_fn(int hidden, int nw, bool pk = false) {
    if (hidden == 32) return pk ? pick<32, true>(nw) : pick<32, false>(nw);
    if (hidden == 64) return pk ? pick<64, true>(nw) : pick<64, false>(nw);
    if (hidden == 128) return pk ? pick<128, true>(nw) : pick<128, false>(nw);
    return nullptr;
}

static size_t roll_smem(int hidden, int nw) {
    if (hidden == 32) return RollLayout<32>::bytes(nw);
    if (hidden == 64) return RollLayout<64>::bytes(nw);
    return RollLayout<128>::bytes(nw);
}

static const int kWarpChoices[] = {2, 4, 6, 8, 10};
// steps per work unit of the persistent tensor-core schedule (parts = 1)
static const int kTcChunk = 50;

// Largest-smem-fitting default: the variant with most resident warps per SM whose grid
// needs the fewest waves.
static int default_warps(int hidden, int ld, int device) {
    int sms = 152, smem_sm = 228 * 1024, smem_blk = 227 * 1024;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const int warps_total = ld / 32;
    double best = -1.0;
    int best_nw = 4;
    for (int nw : kWarpChoices) {
        const size_t b = roll_smem(hidden, nw);
        if (b > (size_t)smem_blk) continue;
        const int per_sm = std::min(smem_sm / (int)(b + 1024), 2048 / (nw * 32));
        if (per_sm < 1) continue;
        const int blocks = (warps_total + nw - 1) / nw;
        const int slots = per_sm * sms;
        const int waves = (blocks + slots - 1) / slots;
        // modelled throughput: useful warp-waves, saturating at 8 resident warps per SM
        const double resident = std::min(8.0, (double)per_sm * nw);
        const double eff = (double)warps_total / ((double)waves * slots * nw) * resident;
        if (eff > best + 1e-9) {
            best = eff;
            best_nw = nw;
        }
    }
    return best_nw;
}

static int resident_warps(int hidden, int nw, int device, bool pk = false) {
    RollFn fn = roll_fn(hidden, nw, pk);
    int blocks = 0, sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, nw * 32, roll_smem(hidden, nw)) != cudaSuccess) {
        cudaGetLastError();
        blocks = 1;
    }
    return std::max(1, blocks) * nw * sms;
}

// Resident CTAs of the tensor-core kernel: one per SM (it allocates all 512 TMEM columns).
static int tc_resident_ctas(int device) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms;
}

static qsim_status ensure_streams(qsim_handle* h) {
    if (h->streams_ready) return QSIM_OK;
    for (int p = 0; p < 4; ++p) {
        QCHECK_CUDA(cudaStreamCreateWithFlags(&h->part_stream[p], cudaStreamNonBlocking));
        QCHECK_CUDA(cudaEventCreateWithFlags(&h->ev_join[p], cudaEventDisableTiming));
    }
    QCHECK_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    h->streams_ready = true;
    return QSIM_OK;
}

qsim_status launch_rollout_tc_range(qsim_handle* h, const float* actor, int T, uint32_t t0, int64_t head,
                                    float sigma, int w0, int w1, cudaStream_t st, int chunk, int* sched);
qsim_status launch_track_tc(qsim_handle* h, const float* actor, int T, const TrackArgs& tr, int chunk,
                            cudaStream_t st);
int rollout_tc_warps_per_cta();

// Launches T steps of the rollout as `parts` env partitions x chunks of `chunk` steps.
// Partition p owns warps [W p / parts, W (p+1) / parts); its chunks run in order on its
// own stream, chunks of different partitions are issued interleaved, and the caller's
// stream joins all partitions at the end.
// engine 2 (tensor cores) ignores nw.
qsim_status launch_rollout(qsim_handle* h, const float* actor, int hidden, int T, float sigma,
                           cudaStream_t st, int nw, int parts, int chunk, int engine) {
    const bool tc = engine == 2;
    const bool pk = engine == 1;
    if (tc && hidden != 64) return fail(QSIM_EINVAL, "qsim_rollout: tensor-core engine needs hidden=64");
    RollFn fn = tc ? nullptr : roll_fn(hidden, nw, pk);
    if (!tc && !fn) return fail(QSIM_EINVAL, "qsim_rollout: no kernel for hidden=%d warps=%d", hidden, nw);
    const size_t smem = tc ? 0 : roll_smem(hidden, nw);
    static bool configured[2][3][11] = {};
    const int hi = hidden == 32 ? 0 : (hidden == 64 ? 1 : 2);
    if (!tc && !configured[pk][hi][nw]) {
        QCHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured[pk][hi][nw] = true;
    }
    const int warps = h->ld / 32;
    parts = std::max(1, std::min(parts, std::min(4, warps)));
    if (chunk <= 0 || chunk > T) chunk = T;
    const uint32_t t0 = (uint32_t)h->t_now;
    if (tc) {
        if (parts == 1) {
            // one persistent launch walking (group of 384 envs, chunk of steps) units
            if (!h->tc_sched) {
                const int groups = (warps + rollout_tc_warps_per_cta() - 1) / rollout_tc_warps_per_cta();
                QCHECK_CUDA(cudaMalloc((void**)&h->tc_sched, sizeof(int) * (size_t)(1 + groups)));
            }
            return launch_rollout_tc_range(h, actor, T, t0, h->head, sigma, 0, warps, st,
                                           chunk < T ? chunk : kTcChunk, h->tc_sched);
        }
        qsim_status s = ensure_streams(h);
        if (s != QSIM_OK) return s;
        QCHECK_CUDA(cudaEventRecord(h->ev_fork, st));
        for (int p = 0; p < parts; ++p) QCHECK_CUDA(cudaStreamWaitEvent(h->part_stream[p], h->ev_fork, 0));
        for (int t = 0; t < T; t += chunk) {
            const int tcn = std::min(chunk, T - t);
            for (int p = 0; p < parts; ++p) {
                const int w0 = (int)((int64_t)warps * p / parts), w1 = (int)((int64_t)warps * (p + 1) / parts);
                if (w1 <= w0) continue;
                s = launch_rollout_tc_range(h, actor, tcn, t0 + (uint32_t)t, h->head + t, sigma, w0, w1,
                                            h->part_stream[p], 0, nullptr);
                if (s != QSIM_OK) return s;
            }
        }
        for (int p = 0; p < parts; ++p) {
            QCHECK_CUDA(cudaEventRecord(h->ev_join[p], h->part_stream[p]));
            QCHECK_CUDA(cudaStreamWaitEvent(st, h->ev_join[p], 0));
        }
        return QSIM_OK;
    }
    if (parts == 1 && chunk == T) {
        const int grid = (warps + nw - 1) / nw;
        fn<<<grid, nw * 32, smem, st>>>(h->dc, h->p, actor, T, t0, h->head, h->capacity, sigma, 0,
                                         warps, TrackArgs{});
        QCHECK_LAUNCH("k_rollout");
        return QSIM_OK;
    }
    qsim_status s = ensure_streams(h);
    if (s != QSIM_OK) return s;
    QCHECK_CUDA(cudaEventRecord(h->ev_fork, st));
    for (int p = 0; p < parts; ++p) QCHECK_CUDA(cudaStreamWaitEvent(h->part_stream[p], h->ev_fork, 0));
    for (int t = 0; t < T; t += chunk) {
        const int tc = std::min(chunk, T - t);
        for (int p = 0; p < parts; ++p) {
            const int w0 = (int)((int64_t)warps * p / parts), w1 = (int)((int64_t)warps * (p + 1) / parts);
            if (w1 <= w0) continue;
            const int grid = (w1 - w0 + nw - 1) / nw;
            fn<<<grid, nw * 32, smem, h->part_stream[p]>>>(h->dc, h->p, actor, tc, t0 + (uint32_t)t,
                                                            h->head + t, h->capacity, sigma, w0, w1,
                                                            TrackArgs{});
            QCHECK_LAUNCH("k_rollout");
        }
    }
    for (int p = 0; p < parts; ++p) {
        QCHECK_CUDA(cudaEventRecord(h->ev_join[p], h->part_stream[p]));
        QCHECK_CUDA(cudaStreamWaitEvent(st, h->ev_join[p], 0));
    }
    return QSIM_OK;
}

}  // namespace qsim

using namespace qsim;

extern "C" int32_t qsim_rollout_tune(qsim_handle* h, int32_t warps_per_block) {
    if (!h) return 0;
    if (warps_per_block > 0 && roll_fn(64, warps_per_block)) h->rollout_warps = warps_per_block;
    else if (warps_per_block == 0) h->rollout_warps = 0;
    return h->rollout_warps;
}

extern "C" qsim_status qsim_rollout(qsim_handle* h, const float* actor, int32_t hidden,
                                    int32_t n_steps, float sigma_e, void* stream) {
    if (!h || !actor) return fail(QSIM_EINVAL, "qsim_rollout: null pointer");
    if (n_steps < 0) return fail(QSIM_EINVAL, "qsim_rollout: n_steps < 0");
    if (hidden != 32 && hidden != 64 && hidden != 128)
        return fail(QSIM_EINVAL, "qsim_rollout: hidden=%d not in {32,64,128}", hidden);
    if (((h->t_now + n_steps) >> 32) != 0)
        return fail(QSIM_ESTATE, "qsim_rollout: step counter exhausted");
    if (n_steps == 0) return QSIM_OK;
    int nw = h->rollout_warps ? h->rollout_warps : default_warps(hidden, h->ld, h->device);
    if (roll_smem(hidden, nw) > 227 * 1024) nw = 2;
    // automatic (-1): the tensor-core engine where it exists (hidden 64), else paired-FMA SIMT
    int engine = h->rollout_packed >= 0 ? h->rollout_packed : (hidden == 64 ? 2 : 1);
    if (engine == 2 && hidden != 64) engine = 1;
    int parts = h->rollout_parts, chunk = h->rollout_chunk;
    if (parts <= 0) {
        if (engine == 2) {
            parts = 1;  // the persistent work-unit schedule
            chunk = 0;
        } else {
            // more than one wave of warps: pipeline two partitions in 100-step chunks
            parts = (h->ld / 32 > resident_warps(hidden, nw, h->device, engine == 1)) ? 2 : 1;
            chunk = parts > 1 ? 100 : 0;
        }
    }
    qsim_status s = launch_rollout(h, actor, hidden, n_steps, sigma_e, (cudaStream_t)stream, nw,
                                   parts, chunk, engine);
    if (s != QSIM_OK) return s;
    h->t_now += n_steps;
    if (h->capacity > 0) {
        h->head = (h->head + n_steps) % h->capacity;
        h->size = std::min<int64_t>(h->capacity, h->size + n_steps);
    }
    return QSIM_OK;
}

extern "C" int32_t qsim_rollout_autotune(qsim_handle* h, const float* actor, int32_t hidden,
                                         int32_t n_steps, void* stream) {
    if (!h || !actor || n_steps <= 0) return fail(QSIM_EINVAL, "qsim_rollout_autotune: bad argument");
    if (hidden != 32 && hidden != 64 && hidden != 128)
        return fail(QSIM_EINVAL, "qsim_rollout_autotune: hidden=%d not in {32,64,128}", hidden);
    int smem_blk = 227 * 1024;
    cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    QCHECK_CUDA(cudaEventCreate(&e0));
    QCHECK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_nw = 0, best_parts = 1, best_pk = 0, best_chunk = 0;
    struct Sched { int parts, chunk; };
    const int tc = std::max(1, std::min(100, n_steps / 4));
    // parts = 1 with chunk c: one launch (SIMT) or the persistent unit schedule with c-step
    // units (tensor cores; c = 0: the default unit)
    const Sched scheds[] = {{1, 0}, {1, std::max(1, n_steps / 4)}, {2, tc}, {3, tc}, {4, tc}};
    for (int pk = 0; pk < 3; ++pk)
    for (int nw : kWarpChoices) {
        if (pk == 2 && (hidden != 64 || nw != kWarpChoices[0])) continue;  // one tensor-core shape
        if (pk < 2 && roll_smem(hidden, nw) > (size_t)smem_blk) continue;
        if (h->rollout_packed >= 0 && pk != h->rollout_packed) continue;
        for (const Sched& sc : scheds) {
            if (((h->t_now + n_steps) >> 32) != 0) break;
            if (pk < 2 && sc.parts == 1 && sc.chunk > 0) continue;  // chunked single stream: SIMT gains nothing
            const int resident = pk == 2 ? rollout_tc_warps_per_cta() * tc_resident_ctas(h->device)
                                         : resident_warps(hidden, nw, h->device, pk == 1);
            if (sc.parts > 1 && h->ld / 32 <= resident) continue;
            cudaEventRecord(e0, st);
            qsim_status s = launch_rollout(h, actor, hidden, n_steps, -1.0f, st, nw, sc.parts, sc.chunk,
                                           pk);
            cudaEventRecord(e1, st);
            if (s != QSIM_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
            h->t_now += n_steps;
            if (h->capacity > 0) {
                h->head = (h->head + n_steps) % h->capacity;
                h->size = std::min<int64_t>(h->capacity, h->size + n_steps);
            }
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; best_nw = nw; best_parts = sc.parts; best_pk = pk; best_chunk = sc.chunk; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    QCHECK_LAUNCH("qsim_rollout_autotune");
    if (best_nw) {
        h->rollout_warps = best_nw;
        h->rollout_parts = best_parts;
        h->rollout_chunk = best_parts > 1 ? 100 : (best_pk == 2 ? best_chunk : 0);
        h->rollout_packed = best_pk;
    }
    return best_nw;
}

extern "C" int32_t qsim_rollout_packed(qsim_handle* h, int32_t packed) {
    if (!h) return 0;
    if (packed >= -1 && packed <= 1) h->rollout_packed = packed;
    return h->rollout_packed;
}

extern "C" int32_t qsim_rollout_engine(qsim_handle* h, int32_t engine) {
    if (!h) return 0;
    if (engine >= -1 && engine <= 2) h->rollout_packed = engine;
    return h->rollout_packed;
}

extern "C" int32_t qsim_rollout_schedule(qsim_handle* h, int32_t parts, int32_t chunk) {
    if (!h) return 0;
    if (parts >= 0 && parts <= 4) h->rollout_parts = parts;
    if (chunk >= 0) h->rollout_chunk = chunk;
    return h->rollout_parts;
}

namespace qsim {
template <int H>
static RollFn track_fn() { return k_rollout<H, 4, true, true>; }
}  // namespace qsim

extern "C" qsim_status qsim_track(qsim_handle* h, const float* actor, int32_t hidden,
                                  int32_t n_steps, const float* period, float amplitude, float z0,
                                  float clip_p, float clip_v, double* sq_err, int32_t* steps_ok,
                                  void* stream) {
    if (!h || !actor || !period || !sq_err || !steps_ok)
        return fail(QSIM_EINVAL, "qsim_track: null pointer");
    if (hidden != 32 && hidden != 64 && hidden != 128)
        return fail(QSIM_EINVAL, "qsim_track: hidden=%d not in {32,64,128}", hidden);
    if (n_steps < 0) return fail(QSIM_EINVAL, "qsim_track: n_steps < 0");
    if (!(std::fabs(amplitude) <= 1e6f) || !(std::fabs(z0) <= 1e6f) || !(clip_p >= 0.0f) ||
        !(clip_v >= 0.0f) || !(clip_p <= 1e30f) || !(clip_v <= 1e30f))
        return fail(QSIM_EINVAL, "qsim_track: amplitude, z0 and clips must be finite, clips >= 0");
    const float* ptrs[3] = {actor, period, reinterpret_cast<const float*>(steps_ok)};
    for (const float* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 4) return fail(QSIM_EINVAL, "qsim_track: misaligned pointer");
    if (reinterpret_cast<uintptr_t>(sq_err) % 8) return fail(QSIM_EINVAL, "qsim_track: misaligned pointer");
    TrackArgs tr{period, amplitude, z0, clip_p, clip_v, sq_err, steps_ok};
    // hidden 64 flies on the tensor-core kernel unless the handle pins a SIMT engine
    if (hidden == 64 && h->rollout_packed != 0 && h->rollout_packed != 1)
        return launch_track_tc(h, actor, n_steps, tr, kTcChunk, (cudaStream_t)stream);
    constexpr int nw = 4;
    RollFn fn = hidden == 32 ? track_fn<32>() : (hidden == 64 ? track_fn<64>() : track_fn<128>());
    const size_t smem = roll_smem(hidden, nw);
    static bool configured[3] = {};
    const int hi = hidden == 32 ? 0 : (hidden == 64 ? 1 : 2);
    if (!configured[hi]) {
        QCHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured[hi] = true;
    }
    const int warps = h->ld / 32;
    fn<<<(warps + nw - 1) / nw, nw * 32, smem, (cudaStream_t)stream>>>(
        h->dc, h->p, actor, n_steps, 0u, 0, 0, 0.0f, 0, warps, tr);
    QCHECK_LAUNCH("k_rollout<track>");
    return QSIM_OK;
}
