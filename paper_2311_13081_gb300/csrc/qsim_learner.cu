// qsim_learner.cu -- asymmetric TD3 learner (Sec. IV; TD3 of Fujimoto et al. 2018) and the
// batched multi-run training kernel.
//
// One run is processed by a thread-block cluster of S CTAs.  Each CTA owns B/S samples of
// the minibatch: it gathers them from the replay ring, rebuilds the actor and privileged
// critic observations, and runs every forward / backward GEMM of its slice with
// activations in its own scratch (L2-resident).  Weight gradients are reduced across the
// cluster in a fixed order (deterministic, no float atomics): each CTA sums one slice of
// the parameter vector over the S partials and applies Adam (and Polyak) to that slice,
// with hardware cluster barriers between phases.  A persistent grid of clusters walks a
// host-computed longest-processing-time-first list of runs; each run advances n_iters
// iterations of {env step of its envs, updates_per_step updates} before the cluster moves
// to its next run.  The same kernel launched for one run and one iteration is the plain
// (one-run-per-launch) form.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <numeric>
#include <vector>

#include <cooperative_groups.h>

#include "qsim_gemm.cuh"
#include "qsim_smlp.cuh"
#include "qsim_internal.h"
#include "qsim_recalc.cuh"
#include "qsim_tcgen05.cuh"

namespace cg = cooperative_groups;

namespace qsim {


constexpr int SMEM_ENGINE = smlp::floats() > smlp::floats2() ? smlp::floats() : smlp::floats2();
constexpr int SMEM_MAIN = GEMM_SMEM > SMEM_ENGINE ? GEMM_SMEM : SMEM_ENGINE;
// the small-run env step keeps an actor of hidden <= 128 and <= 128 inputs in shared memory
static_assert(SMEM_MAIN >= 128 * 128 + 128 + 128 * 128 + 128 + 4 * 128 + 4 + 4 + 8 * (132 + 2 * 132 + 4 + 32),
              "learner shared memory too small for the small-run env step");

struct LearnHyper {
    float gamma, tau, lr, beta1, beta2, eps, sigma_t, noise_clip;
    int policy_delay, updates_per_step;
};

// Everything the training kernel knows about one run.  Counters are updated in place by
// the kernel so that a captured graph can be replayed.
struct RunDesc {
    EnvCfg C;
    EnvPtrs E;
    int64_t capacity, head, size, t_now;
    int64_t next_curr, curr_interval;
    float cf[7], ct[7];
    float sig_f, sig_min;
    int recalc;
    int n_env;
    float *actor, *actor_t, *c1, *c1_t, *c2, *c2_t;
    float *m_a, *v_a, *m_c1, *v_c1, *m_c2, *v_c2;
    float* stats;
    int H, B, DA, DC, PA, PC;
    int64_t t_a, t_c, u;
    int64_t start_updates;
    LearnHyper hp;
    uint32_t* idx_log;  // [B] flat replay indices of the latest update, or null
};

// Forward of in -> H (ReLU) -> H (ReLU) -> out (tanh or linear) for M rows of X [M][ldx].
__device__ __noinline__ void mlp_fwd(const float* W, int in, int H, int out, const float* X, int ldx, int M,
                        float* H1, float* H2, float* Y, int ldy, bool tanh_out, float* sm) {
    const float* W1 = W;
    const float* b1 = W1 + H * in;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + out * H;
    cta_gemm(M, H, in, Mat{X, ldx, 1}, Mat{W1, 1, in}, sm,
             [&](int m, int n, float v) { H1[m * H + n] = fmaxf(v, 0.0f); }, b1);
    cta_gemm(M, H, H, Mat{H1, H, 1}, Mat{W2, 1, H}, sm,
             [&](int m, int n, float v) { H2[m * H + n] = fmaxf(v, 0.0f); }, b2);
    cta_gemm(M, out, H, Mat{H2, H, 1}, Mat{W3, 1, H}, sm, [&](int m, int n, float v) {
        Y[m * ldy + n] = tanh_out ? tanhf(v) : v;
    }, b3);
}

// Reverse through the MLP for M rows.  dZ3 [M][out] holds dLoss/d(pre-activation of the
// output layer).  Writes the parameter gradient (this CTA's partial) into G (layout of
// W) and, if dX != nullptr, dLoss/dX [M][in] (only columns [x_lo, in) are needed).
__device__ __noinline__ void mlp_bwd(const float* W, int in, int H, int out, const float* X, int ldx, int M,
                        const float* H1, const float* H2, const float* dZ3, float* dZ2,
                        float* dZ1, float* G, float* dX, int x_lo, float* sm) {
    const float* W2 = W + H * in + H;
    const float* W3 = W2 + H * H + H;
    float* gW1 = G;
    float* gb1 = gW1 + H * in;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + out * H;
    // dW3 = dZ3^T H2 ; db3 = colsum dZ3
    if (G) {
        cta_gemm(out, H, M, Mat{dZ3, 1, out}, Mat{H2, H, 1}, sm,
                 [&](int m, int n, float v) { gW3[m * H + n] = v; });
        for (int n = threadIdx.x; n < out; n += LT) {
            float s = 0.0f;
            for (int m = 0; m < M; ++m) s += ldcg(dZ3 + m * out + n);
            gb3[n] = s;
        }
    }
    // dZ2 = (dZ3 W3) * (H2 > 0)
    cta_gemm(M, H, out, Mat{dZ3, out, 1}, Mat{W3, H, 1}, sm, [&](int m, int n, float v) {
        dZ2[m * H + n] = H2[m * H + n] > 0.0f ? v : 0.0f;  // written by this CTA
    });
    if (G) {
        cta_gemm(H, H, M, Mat{dZ2, 1, H}, Mat{H1, H, 1}, sm,
                 [&](int m, int n, float v) { gW2[m * H + n] = v; });
        for (int n = threadIdx.x; n < H; n += LT) {
            float s = 0.0f;
            for (int m = 0; m < M; ++m) s += ldcg(dZ2 + m * H + n);
            gb2[n] = s;
        }
    }
    // dZ1 = (dZ2 W2) * (H1 > 0)
    cta_gemm(M, H, H, Mat{dZ2, H, 1}, Mat{W2, H, 1}, sm, [&](int m, int n, float v) {
        dZ1[m * H + n] = H1[m * H + n] > 0.0f ? v : 0.0f;  // written by this CTA
    });
    if (G) {
        cta_gemm(H, in, M, Mat{dZ1, 1, H}, Mat{X, ldx, 1}, sm,
                 [&](int m, int n, float v) { gW1[m * in + n] = v; });
        for (int n = threadIdx.x; n < H; n += LT) {
            float s = 0.0f;
            for (int m = 0; m < M; ++m) s += ldcg(dZ1 + m * H + n);
            gb1[n] = s;
        }
    }
    if (dX) {
        const float* W1 = W;
        cta_gemm(M, in - x_lo, H, Mat{dZ1, H, 1}, Mat{W1 + x_lo, in, 1}, sm,
                 [&](int m, int n, float v) { dX[m * in + x_lo + n] = v; });
    }
    __syncthreads();
}

// -------------------------------------------------------------------- cluster helpers
__device__ __forceinline__ void cluster_sync_all(int S) {
    if (S > 1) {
        __threadfence();
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

// Scratch layout of one CTA (floats), for Bc samples.
struct Scr {
    float *oa, *oa2, *oc, *oc2, *r, *term, *y, *q1, *q2, *mu, *da, *dz3, *X1, *X2, *H1a, *H2a,
        *H1b, *H2b, *dZ2, *dZ1, *ga, *g1, *g2, *loss, *env_obs, *env_h1, *env_h2, *env_mu;
};

__host__ __device__ inline size_t scratch_floats(int Bc, int H, int DA, int DC, int PA, int PC,
                                                 int n_env) {
    size_t f = 0;
    f += 2 * (size_t)Bc * DA + 2 * (size_t)Bc * DC;  // oa oa2 oc oc2
    f += 5 * (size_t)Bc;                              // r term y q1 q2
    f += 3 * 4 * (size_t)Bc;                          // mu da dz3
    f += 8 * (size_t)Bc * H;                          // X1 X2 H1a H2a H1b H2b dZ2 dZ1
    f += (size_t)PA + 2 * (size_t)PC + 8;             // partial grads + loss
    f += (size_t)n_env * (DA + 2 * H + 4);            // env-step tile
    return (f + 31) & ~(size_t)31;
}

__device__ Scr carve(float* base, int Bc, int H, int DA, int DC, int PA, int PC, int n_env) {
    Scr s;
    float* p = base;
    auto take = [&](size_t n) { float* q = p; p += n; return q; };
    s.oa = take((size_t)Bc * DA); s.oa2 = take((size_t)Bc * DA);
    s.oc = take((size_t)Bc * DC); s.oc2 = take((size_t)Bc * DC);
    s.r = take(Bc); s.term = take(Bc); s.y = take(Bc); s.q1 = take(Bc); s.q2 = take(Bc);
    s.mu = take(4 * (size_t)Bc); s.da = take(4 * (size_t)Bc); s.dz3 = take(4 * (size_t)Bc);
    s.X1 = take((size_t)Bc * H); s.X2 = take((size_t)Bc * H);
    s.H1a = take((size_t)Bc * H); s.H2a = take((size_t)Bc * H);
    s.H1b = take((size_t)Bc * H); s.H2b = take((size_t)Bc * H);
    s.dZ2 = take((size_t)Bc * H); s.dZ1 = take((size_t)Bc * H);
    s.ga = take(PA); s.g1 = take(PC); s.g2 = take(PC); s.loss = take(8);
    s.env_obs = take((size_t)n_env * DA); s.env_h1 = take((size_t)n_env * H);
    s.env_h2 = take((size_t)n_env * H); s.env_mu = take((size_t)n_env * 4);
    return s;
}

// ------------------------------------------------------------------- env-step helpers
__device__ __forceinline__ void load_env(const RunDesc& R, int e, float* s, float* d, Prm& P) {
    const int ld = R.C.ld;
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = ldcg(R.E.state + i * ld + e);
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = ldcg(R.E.dist + i * ld + e);
    const float* pr = R.E.prm;
    P = make_prm(ldcg(pr + e), ldcg(pr + ld + e), ldcg(pr + 2 * ld + e), ldcg(pr + 3 * ld + e),
                 ldcg(pr + 4 * ld + e), ldcg(pr + 5 * ld + e), ldcg(pr + 6 * ld + e));
}

// Actor forward for a handful of rows (n <= 8, hidden <= 64, input <= 128): one warp per
// output unit, lanes split the inputs, every weight load of a warp in flight at once, rows
// reduced with warp shuffles.  x, h: shared memory; the tanh outputs go to Y (global [n][4]).
template <int JT, int KC>
__device__ __forceinline__ void small_layer(const float* Wl, const float* bl, int in, int nout,
                                            const float* x, int ldx, int n, float* y, int ldy,
                                            bool last) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float w[JT][KC], bv[JT];
#pragma unroll
    for (int t = 0; t < JT; ++t) {
        const int j = warp + (LT / 32) * t;
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            const int k = lane + 32 * c;
            w[t][c] = j < nout && k < in ? ldcg(Wl + (size_t)j * in + k) : 0.0f;
        }
        bv[t] = j < nout ? ldcg(bl + j) : 0.0f;
    }
    for (int r = 0; r < n; ++r) {
        float xv[KC];
#pragma unroll
        for (int c = 0; c < KC; ++c) xv[c] = lane + 32 * c < in ? x[r * ldx + lane + 32 * c] : 0.0f;
#pragma unroll
        for (int t = 0; t < JT; ++t) {
            const int j = warp + (LT / 32) * t;
            if (j >= nout) continue;
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < KC; ++c) acc = fmaf(w[t][c], xv[c], acc);
            acc = smlp::warp_sum(acc) + bv[t];
            if (lane == 0) y[r * ldy + j] = last ? tanhf(acc) : fmaxf(acc, 0.0f);
        }
    }
}

__device__ __noinline__ void actor_small(const float* W, int in, int H, const float* X, int n,
                                         float* Y, float* sm) {
    constexpr int LX = 132, LH = 68;
    float* xs = sm;
    float* h1 = xs + 8 * LX;
    float* h2 = h1 + 8 * LH;
    for (int i = threadIdx.x; i < n * in; i += LT) xs[(i / in) * LX + i % in] = ldcg(X + i);
    __syncthreads();
    const float* b1 = W + (size_t)H * in;
    const float* W2 = b1 + H;
    const float* b2 = W2 + (size_t)H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + 4 * H;
    small_layer<8, 4>(W, b1, in, H, xs, LX, n, h1, LH, false);
    __syncthreads();
    small_layer<8, 2>(W2, b2, H, H, h1, LH, n, h2, LH, false);
    __syncthreads();
    small_layer<1, 2>(W3, b3, H, 4, h2, LH, n, Y, 4, true);
    __syncthreads();
}

// Actor forward of n rows through the shared-memory engine (hidden <= 64).
__device__ __noinline__ void actor_smem(const float* W, int in, int H, const float* X, int n,
                                        float* Y, float* sm) {
    const smlp::Buf b = smlp::carve(sm);
    smlp::stage(W, in, H, 4, b);
    for (int r0 = 0; r0 < n; r0 += smlp::MC)
        smlp::forward(in, H, 4, X, in, r0, min(smlp::MC, n - r0), b, Y, 4, true);
}

// One env step of all envs of run R (executed by one CTA): observation, actor forward
// (generic GEMM path), warm-up / exploration, RK4, reward, termination, record write,
// history update and reset.
__device__ __noinline__ void env_step_cta(RunDesc& R, const Scr& S, uint32_t t, int64_t slot, float* sm) {
    const EnvCfg& C = R.C;
    const int ld = C.ld, n = R.n_env, DA = R.DA, H = R.H;
    const bool warm = (int64_t)t < (int64_t)C.learning_starts;
    if (!warm) {
        for (int e = threadIdx.x; e < n; e += LT) {
            float s[NS], o[18];
#pragma unroll
            for (int i = 0; i < NS; ++i) s[i] = ldcg(R.E.state + i * ld + e);
            obs_state(s, o);
            if (C.any_noise) {
                float nz[18];
                obs_noise(C, (uint32_t)e, t, nz);
#pragma unroll
                for (int k = 0; k < 18; ++k) o[k] += nz[k];
            }
            float* row = S.env_obs + (size_t)e * DA;
#pragma unroll
            for (int k = 0; k < 18; ++k) row[k] = o[k];
            // history loads in two halves, each all in flight before its stores
            const int nh4 = 4 * C.n_hist;
#pragma unroll 1
            for (int h0 = 0; h0 < 4 * HMAX; h0 += 2 * HMAX) {
                float hv[2 * HMAX];
#pragma unroll
                for (int k = 0; k < 2 * HMAX; ++k)
                    hv[k] = h0 + k < nh4 ? ldcg(R.E.hist + (h0 + k) * ld + e) : 0.0f;
#pragma unroll
                for (int k = 0; k < 2 * HMAX; ++k)
                    if (h0 + k < nh4) row[18 + h0 + k] = hv[k];
            }
        }
        __syncthreads();
        if (n <= 8 && H <= 64 && DA <= 128) {
            actor_small(R.actor, DA, H, S.env_obs, n, S.env_mu, sm);
        } else if (H <= smlp::HP && DA <= smlp::INP) {
            actor_smem(R.actor, DA, H, S.env_obs, n, S.env_mu, sm);
        } else {
            mlp_fwd(R.actor, DA, H, 4, S.env_obs, DA, n, S.env_h1, S.env_h2, S.env_mu, 4, true, sm);
        }
    }
    const float sigma = ldcg(R.E.rewardC + 7);
    float Cr[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Cr[i] = ldcg(R.E.rewardC + i);
    for (int e = threadIdx.x; e < n; e += LT) {
        float s[NS], d[6], a[4];
        Prm P;
        load_env(R, e, s, d, P);
        // episode counters: loads in flight across the integration
        const uint32_t ep_step = ldcg(R.E.ep_step + e);
        const float ret0 = ldcg(R.E.ep_ret + e);
        if (warm) {
            const uint4 r = draw(C, (uint32_t)e, t, TAG_WARM, 0);
            a[0] = 2.0f * u01(r.x) - 1.0f; a[1] = 2.0f * u01(r.y) - 1.0f;
            a[2] = 2.0f * u01(r.z) - 1.0f; a[3] = 2.0f * u01(r.w) - 1.0f;
        } else {
            float mu[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) mu[j] = ldcg(S.env_mu + e * 4 + j);
            if (sigma > 0.0f) {
                const uint4 r0 = draw(C, (uint32_t)e, t, TAG_EXPL, 0);
                const uint4 r1 = draw(C, (uint32_t)e, t, TAG_EXPL, 1);
                a[0] = clampf(fmaf(sigma, gauss(r0.x, r0.y), mu[0]), -1.0f, 1.0f);
                a[1] = clampf(fmaf(sigma, gauss(r0.z, r0.w), mu[1]), -1.0f, 1.0f);
                a[2] = clampf(fmaf(sigma, gauss(r1.x, r1.y), mu[2]), -1.0f, 1.0f);
                a[3] = clampf(fmaf(sigma, gauss(r1.z, r1.w), mu[3]), -1.0f, 1.0f);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) a[j] = clampf(mu[j], -1.0f, 1.0f);
            }
        }
        float u[4], s2[NS];
        action_to_rpm(C.veh, a, u);
#pragma unroll
        for (int i = 0; i < NS; ++i) s2[i] = s[i];
        motor_lag_off(C, u, s2);
        rk4(C.veh, C.dt, C.renorm, s2, u, P, d);
        const float r = reward(Cr, s2, a);
        const bool term = terminated(C, s2);
        const uint32_t ep_after = ep_step + 1;
        const bool trunc = !term && (int)ep_after >= C.episode_len;
        if (R.capacity > 0 && in_bounds(R.E.status, slot, R.E.rows, SITE_RING_WRITE) &&
            in_bounds(R.E.status, e, ld, SITE_SOA)) {
            float* rec = R.E.rec + (size_t)slot * C.F * ld + e;
#pragma unroll
            for (int i = 0; i < NS; ++i) rec[i * ld] = s[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) rec[(17 + i) * ld] = a[i];
            rec[21 * ld] = r;
            rec[22 * ld] = __uint_as_float(pack_flags(term, trunc, ep_step));
            if (C.n_priv) {
                float pv[NPRIV];
                priv_vals(C, P, d, pv);
#pragma unroll
                for (int k = 0; k < NPRIV; ++k) rec[(23 + k) * ld] = pv[k];
            }
            if (term || trunc) {
                float* sd = R.E.side + ((size_t)slot * ld + e) * NS;
#pragma unroll
                for (int i = 0; i < NS; ++i) sd[i] = s2[i];
            }
        }
        {
            // shift the history (newest first) in two halves, the older half first so that
            // no entry is overwritten before it has been loaded: entries [h0, h0 + 30) move
            // to [h0 + 4, h0 + 34)
            const int nh4 = 4 * C.n_hist;
            constexpr int HH = 2 * HMAX - 2;
#pragma unroll 1
            for (int h0 = HH; h0 >= 0; h0 -= HH) {
                float hv[HH];
#pragma unroll
                for (int k = 0; k < HH; ++k)
                    hv[k] = h0 + k + 4 < nh4 ? ldcg(R.E.hist + (h0 + k) * ld + e) : 0.0f;
#pragma unroll
                for (int k = 0; k < HH; ++k)
                    if (h0 + k + 4 < nh4) R.E.hist[(h0 + k + 4) * ld + e] = hv[k];
            }
            if (C.n_hist > 0)
                for (int c = 0; c < 4; ++c) R.E.hist[c * ld + e] = a[c];
        }
        float ret = ret0 + r;
        uint32_t eps = ep_after;
        if (term || trunc) {
            R.E.n_done[e] = ldcg(R.E.n_done + e) + 1;
            R.E.len_sum[e] = ldcg(R.E.len_sum + e) + ep_after;
            R.E.ret_sum[e] = ldcg(R.E.ret_sum + e) + ret;
            const uint32_t epi = ldcg(R.E.ep_index + e) + 1;
            R.E.ep_index[e] = epi;
            float prm7[7];
            reset_env(C, (uint32_t)e, epi, s2, prm7, d);
            for (int i = 0; i < 7; ++i) R.E.prm[i * ld + e] = prm7[i];
            for (int i = 0; i < 6; ++i) R.E.dist[i * ld + e] = d[i];
            for (int i = 0; i < 4 * HMAX; ++i) R.E.hist[i * ld + e] = 0.0f;
            ret = 0.0f;
            eps = 0;
        }
        R.E.ep_ret[e] = ret;
        R.E.ep_step[e] = eps;
#pragma unroll
        for (int i = 0; i < NS; ++i) R.E.state[i * ld + e] = s2[i];
    }
    __syncthreads();
}

// Env step of a run with at most 8 envs (one CTA; a single run's env step sits on the
// critical path of every update): the actor's weights are copied into shared memory
// asynchronously (cp.async, L2 -> shared) while each env's thread loads its state and
// history and builds its observation in shared memory; the three layers then read
// shared memory only; the env's data stay in registers from the observation to the
// write-back, and the history shift reads the observation row already in shared memory.
__device__ __noinline__ void env_step_small(RunDesc& R, uint32_t t, int64_t slot, float* sm) {
    const EnvCfg& C = R.C;
    const int ld = C.ld, n = R.n_env, DA = R.DA, H = R.H, PA = R.PA;
    const bool warm = (int64_t)t < (int64_t)C.learning_starts;
    constexpr int LX = 132, LH = 132;
    float* Ws = sm;                                   // actor parameters, as stored
    float* xs = sm + ((PA + 3) & ~3);                 // [8][LX] observations
    float* h1 = xs + 8 * LX;                          // [8][LH]
    float* h2 = h1 + 8 * LH;                          // [8][LH]
    float* mus = h2 + 8 * LH;                         // [8][4]
    float* park = mus + 8 * 4;                        // [8][32]: env data across the layers
    if (!warm) {
        // 16-byte copies need a 16-byte aligned source (the actor opens the learner's
        // allocation, so it is); otherwise every element goes through the tail loop
        const int nv = ((uintptr_t)R.actor & 15u) == 0 ? PA >> 2 : 0;
        const uint32_t sW = (uint32_t)__cvta_generic_to_shared(Ws);
        for (int v = threadIdx.x; v < nv; v += LT)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(sW + 16u * (uint32_t)v),
                         "l"(R.actor + 4 * v) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int i = 4 * nv + threadIdx.x; i < PA; i += LT) Ws[i] = ldcg(R.actor + i);
    }
    const int e = threadIdx.x;
    const bool mine = e < n;
    if (mine) {
        // the env's data wait in shared memory while the layers run (no long live ranges)
        float* pk = park + 32 * e;
        float s[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) s[i] = pk[i] = ldcg(R.E.state + i * ld + e);
#pragma unroll
        for (int i = 0; i < 6; ++i) pk[NS + i] = ldcg(R.E.dist + i * ld + e);
#pragma unroll
        for (int i = 0; i < 7; ++i) pk[NS + 6 + i] = ldcg(R.E.prm + i * ld + e);
        pk[30] = __uint_as_float(ldcg(R.E.ep_step + e));
        pk[31] = ldcg(R.E.ep_ret + e);
        float* row = xs + e * LX;
        const int nh4 = 4 * C.n_hist;
        // history in two halves, each with all its loads in flight before its stores
#pragma unroll 1
        for (int h0 = 0; h0 < 4 * HMAX; h0 += 2 * HMAX) {
            float hv[2 * HMAX];
#pragma unroll
            for (int k = 0; k < 2 * HMAX; ++k) hv[k] = h0 + k < nh4 ? ldcg(R.E.hist + (h0 + k) * ld + e) : 0.0f;
#pragma unroll
            for (int k = 0; k < 2 * HMAX; ++k) row[18 + h0 + k] = hv[k];
        }
        float o[18];
        obs_state(s, o);
        if (!warm && C.any_noise) {
            float nz[18];
            obs_noise(C, (uint32_t)e, t, nz);
#pragma unroll
            for (int k = 0; k < 18; ++k) o[k] += nz[k];
        }
#pragma unroll
        for (int k = 0; k < 18; ++k) row[k] = o[k];
    }
    if (!warm) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        // layers: one warp per output unit; the warp's lanes split into n groups of L (one
        // group per env), each group's lanes over the inputs, group-wide shuffle sums
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int L = n <= 1 ? 32 : (n <= 2 ? 16 : (n <= 4 ? 8 : 4));
        const int r = lane / L, kq = lane - r * L;
        const bool on = r < n;
        auto gsum = [&](float v) {
            for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            return v;
        };
        const float* b1 = Ws + H * DA;
        const float* W2 = b1 + H;
        const float* b2 = W2 + H * H;
        const float* W3 = b2 + H;
        const float* b3 = W3 + 4 * H;
        for (int j = warp; j < H; j += LT / 32) {
            float acc = 0.0f;
            if (on)
                for (int k = kq; k < DA; k += L) acc = fmaf(Ws[j * DA + k], xs[r * LX + k], acc);
            acc = gsum(acc) + b1[j];
            if (on && kq == 0) h1[r * LH + j] = fmaxf(acc, 0.0f);
        }
        __syncthreads();
        for (int j = warp; j < H; j += LT / 32) {
            float acc = 0.0f;
            if (on)
                for (int k = kq; k < H; k += L) acc = fmaf(W2[j * H + k], h1[r * LH + k], acc);
            acc = gsum(acc) + b2[j];
            if (on && kq == 0) h2[r * LH + j] = fmaxf(acc, 0.0f);
        }
        __syncthreads();
        if (warp < 4) {
            const int o = warp;
            float acc = 0.0f;
            if (on)
                for (int k = kq; k < H; k += L) acc = fmaf(W3[o * H + k], h2[r * LH + k], acc);
            acc = gsum(acc) + b3[o];
            if (on && kq == 0) mus[r * 4 + o] = tanhf(acc);
        }
    }
    __syncthreads();
    if (!mine) return;
    float s[NS], d[6];
    const float* pk = park + 32 * e;
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = pk[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = pk[NS + i];
    const Prm P = make_prm(pk[23], pk[24], pk[25], pk[26], pk[27], pk[28], pk[29]);
    const uint32_t ep_step = __float_as_uint(pk[30]);
    const float ret0 = pk[31];
    const float sigma = ldcg(R.E.rewardC + 7);
    float Cr[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Cr[i] = ldcg(R.E.rewardC + i);
    float a[4];
    if (warm) {
        const uint4 r = draw(C, (uint32_t)e, t, TAG_WARM, 0);
        a[0] = 2.0f * u01(r.x) - 1.0f; a[1] = 2.0f * u01(r.y) - 1.0f;
        a[2] = 2.0f * u01(r.z) - 1.0f; a[3] = 2.0f * u01(r.w) - 1.0f;
    } else {
        const float* mu = mus + e * 4;
        if (sigma > 0.0f) {
            const uint4 r0 = draw(C, (uint32_t)e, t, TAG_EXPL, 0);
            const uint4 r1 = draw(C, (uint32_t)e, t, TAG_EXPL, 1);
            a[0] = clampf(fmaf(sigma, gauss(r0.x, r0.y), mu[0]), -1.0f, 1.0f);
            a[1] = clampf(fmaf(sigma, gauss(r0.z, r0.w), mu[1]), -1.0f, 1.0f);
            a[2] = clampf(fmaf(sigma, gauss(r1.x, r1.y), mu[2]), -1.0f, 1.0f);
            a[3] = clampf(fmaf(sigma, gauss(r1.z, r1.w), mu[3]), -1.0f, 1.0f);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] = clampf(mu[j], -1.0f, 1.0f);
        }
    }
    float u[4], s2[NS];
    action_to_rpm(C.veh, a, u);
#pragma unroll
    for (int i = 0; i < NS; ++i) s2[i] = s[i];
    motor_lag_off(C, u, s2);
    rk4(C.veh, C.dt, C.renorm, s2, u, P, d);
    const float r = reward(Cr, s2, a);
    const bool term = terminated(C, s2);
    const uint32_t ep_after = ep_step + 1;
    const bool trunc = !term && (int)ep_after >= C.episode_len;
    if (R.capacity > 0 && in_bounds(R.E.status, slot, R.E.rows, SITE_RING_WRITE) &&
        in_bounds(R.E.status, e, ld, SITE_SOA)) {
        float* rec = R.E.rec + (size_t)slot * C.F * ld + e;
#pragma unroll
        for (int i = 0; i < NS; ++i) rec[i * ld] = s[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) rec[(17 + i) * ld] = a[i];
        rec[21 * ld] = r;
        rec[22 * ld] = __uint_as_float(pack_flags(term, trunc, ep_step));
        if (C.n_priv) {
            float pv[NPRIV];
            priv_vals(C, P, d, pv);
#pragma unroll
            for (int k = 0; k < NPRIV; ++k) rec[(23 + k) * ld] = pv[k];
        }
        if (term || trunc) {
            float* sd = R.E.side + ((size_t)slot * ld + e) * NS;
#pragma unroll
            for (int i = 0; i < NS; ++i) sd[i] = s2[i];
        }
    }
    float ret = ret0 + r;
    uint32_t eps = ep_after;
    if (term || trunc) {
        R.E.n_done[e] = ldcg(R.E.n_done + e) + 1;
        R.E.len_sum[e] = ldcg(R.E.len_sum + e) + ep_after;
        R.E.ret_sum[e] = ldcg(R.E.ret_sum + e) + ret;
        const uint32_t epi = ldcg(R.E.ep_index + e) + 1;
        R.E.ep_index[e] = epi;
        float prm7[7];
        reset_env(C, (uint32_t)e, epi, s2, prm7, d);
        for (int i = 0; i < 7; ++i) R.E.prm[i * ld + e] = prm7[i];
        for (int i = 0; i < 6; ++i) R.E.dist[i * ld + e] = d[i];
        for (int i = 0; i < 4 * HMAX; ++i) R.E.hist[i * ld + e] = 0.0f;
        ret = 0.0f;
        eps = 0;
    } else {
        // history newest first: a_t, then the previous entries (from the observation row)
        const int nh4 = 4 * C.n_hist;
        const float* row = xs + e * LX + 18;
        for (int k = nh4 - 1; k >= 4; --k) R.E.hist[k * ld + e] = row[k - 4];
        if (C.n_hist > 0)
#pragma unroll
            for (int c = 0; c < 4; ++c) R.E.hist[c * ld + e] = a[c];
    }
    R.E.ep_ret[e] = ret;
    R.E.ep_step[e] = eps;
#pragma unroll
    for (int i = 0; i < NS; ++i) R.E.state[i * ld + e] = s2[i];
}

// ------------------------------------------------------------------------- TD3 update
// Ring index a mod m for a in [-m, 2m).
__device__ __forceinline__ int64_t ring(int64_t a, int64_t m) {
    return a < 0 ? a + m : (a >= m ? a - m : a);
}

// Gather samples [g0, g0 + G) (G <= 32) of this CTA's share of the minibatch: rebuilds o_a,
// o_a', o_c (with the stored action), o_c' (action slot filled later), r and the
// termination flag from the compact replay records.  Lane l handles sample g0 + l; warp 0
// builds the s_t part, warp 1 the s_{t+1} part and warps 2..7 the action history, each
// into a shared-memory tile laid out like the scratch rows, which is then written out with
// coalesced stores.
__device__ __noinline__ void gather_group(const RunDesc& R, int j0, int g0, int G, uint32_t u,
                                          int64_t head, int64_t size, int64_t t_now, const Scr& S,
                                          float* tile) {
    const EnvCfg& C = R.C;
    const int ld = C.ld, F = C.F, NE = R.n_env, DA = R.DA, DC = R.DC, nh = C.n_hist;
    const int64_t CAP = R.capacity;
    const int w = threadIdx.x >> 5, jl = threadIdx.x & 31;
    float* T_oa = tile;
    float* T_oa2 = T_oa + (size_t)G * DA;
    float* T_oc = T_oa2 + (size_t)G * DA;
    float* T_oc2 = T_oc + (size_t)G * DC;
    float* T_r = T_oc2 + (size_t)G * DC;
    float* T_term = T_r + G;
    int* T_env = reinterpret_cast<int*>(T_term + G);  // sample's env (-1: skipped) and t_rec,
    uint32_t* T_trec = reinterpret_cast<uint32_t*>(T_env + G);  // for the noise pass
    int* const bst = R.E.status;
    const int64_t rows = R.E.rows;
    if (jl < G) {
        const int j = j0 + g0 + jl;
        const int64_t lost = size == CAP ? nh : 0;
        const uint32_t nvalid = (uint32_t)((size - 1 - lost) * NE);
        const uint4 rr = draw(C, (uint32_t)j >> 2, u, TAG_REPLAY, 0);
        const uint32_t x = (j & 3) == 0 ? rr.x : ((j & 3) == 1 ? rr.y : ((j & 3) == 2 ? rr.z : rr.w));
        const uint32_t idx = (uint32_t)(((uint64_t)x * (uint64_t)nvalid) >> 32);
        if (w == 0 && R.idx_log) R.idx_log[j] = idx;
        const int64_t k = idx / (uint32_t)NE;
        const int env = (int)(idx % (uint32_t)NE);
        const int64_t slot = ring(head - size + lost + k, CAP);
        const uint32_t t_rec = (uint32_t)(t_now - size + lost + k);
        // (debug builds) a slot or env outside the ring skips the sample, status set
        const bool sample_ok = in_bounds(bst, slot, rows, SITE_RING_READ) && in_bounds(bst, env, ld, SITE_SOA);
        if (w == 0) {
            T_env[jl] = sample_ok ? env : -1;
            T_trec[jl] = t_rec;
        }
        if (sample_ok) {
            const float* rec = R.E.rec + (size_t)slot * F * ld + env;
            const uint32_t fl = __float_as_uint(ldcg(rec + 22 * ld));
            const bool done = (fl & 3u) != 0;
            const uint32_t ep = fl >> 8;
            float* oa = T_oa + (size_t)jl * DA;
            float* oa2 = T_oa2 + (size_t)jl * DA;
            float* oc = T_oc + (size_t)jl * DC;
            float* oc2 = T_oc2 + (size_t)jl * DC;
            const bool nxt_ok = w != 1 || done || in_bounds(bst, ring(slot + 1, CAP), rows, SITE_RING_READ);
            if (w < 2 && nxt_ok) {
                // w == 0: s_t -> o_a, o_c (+ stored action, reward, flag); w == 1: s_{t+1} -> o_a', o_c'
                // the side slot is env-major (an env's 17 values contiguous), the records field-major
                const bool from_side = w == 1 && done;
                const float* src = w == 0 ? rec
                                          : (from_side ? R.E.side + ((size_t)slot * ld + env) * NS
                                                       : R.E.rec + (size_t)ring(slot + 1, CAP) * F * ld + env);
                const size_t sst = from_side ? 1 : (size_t)ld;
                float st[NS], a[4], pv[NPRIV];
#pragma unroll
                for (int i = 0; i < NS; ++i) st[i] = ldcg(src + i * sst);
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = w == 0 ? ldcg(rec + (17 + i) * ld) : 0.0f;
#pragma unroll
                for (int q = 0; q < NPRIV; ++q) pv[q] = C.n_priv ? ldcg(rec + (23 + q) * ld) : 0.0f;
                const float r = w == 0 ? ldcg(rec + 21 * ld) : 0.0f;
                float* ocx = w == 0 ? oc : oc2;
                float* oax = w == 0 ? oa : oa2;
                float o[18];
                obs_state(st, o);
                // critic observations (noise-free; the symmetric layout 3 copies the actor's
                // noisy observation below)
                if (C.critic_layout != 3) {
#pragma unroll
                    for (int q = 0; q < 18; ++q) ocx[q] = o[q];
                    const int rpm_at = C.critic_layout == 2 ? 18 : DA;
#pragma unroll
                    for (int i = 0; i < 4; ++i) ocx[rpm_at + i] = rpm_norm(C.veh, st[13 + i]);
                    if (C.critic_layout != 0) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) ocx[rpm_at + 4 + q] = pv[q];
                    }
                }
                if (w == 0) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) oc[DC - 4 + i] = a[i];
                    T_r[jl] = r;
                    T_term[jl] = (fl & 1u) ? 1.0f : 0.0f;
                }
                // the observation noise is added by all warps below
#pragma unroll
                for (int q = 0; q < 18; ++q) oax[q] = o[q];
                if (C.critic_layout == 3) {
#pragma unroll
                    for (int q = 0; q < 18; ++q) ocx[q] = o[q];
                }
            } else if (w >= 2) {
                // history: o_a has a_{t-1..t-NH}, o_a' has a_t, a_{t-1..t-NH+1}; zeros before the
                // episode start.  Warp w handles lags i = w-1, w+5, w+11, all their loads issued
                // before the first store.
                static_assert(HMAX <= 18, "history lags: at most 3 per warp of 6");
                float h[3][4], h2[3][4];
#pragma unroll
                for (int u3 = 0; u3 < 3; ++u3) {
                    const int i = w - 1 + 6 * u3;
                    const bool lag = i <= nh;
                    const bool ok = lag && (uint32_t)i <= ep &&
                                    in_bounds(bst, ring(slot - i, CAP), rows, SITE_RING_READ);
                    const bool ok2 = lag && (i == 1 || ((uint32_t)(i - 1) <= ep &&
                                                        in_bounds(bst, ring(slot - i + 1, CAP), rows, SITE_RING_READ)));
                    const float* ap = R.E.rec + (size_t)ring(slot - i, CAP) * F * ld + env + 17 * ld;
                    const float* ap2 = i == 1 ? rec + 17 * ld
                                              : R.E.rec + (size_t)ring(slot - i + 1, CAP) * F * ld + env + 17 * ld;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        h[u3][c] = ok ? ldcg(ap + c * ld) : 0.0f;
                        h2[u3][c] = ok2 ? ldcg(ap2 + c * ld) : 0.0f;
                    }
                }
#pragma unroll
                for (int u3 = 0; u3 < 3; ++u3) {
                    const int i = w - 1 + 6 * u3;
                    if (i > nh) continue;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int q = 18 + 4 * (i - 1) + c;
                        oa[q] = h[u3][c];
                        oa2[q] = h2[u3][c];
                        if (C.critic_layout != 2) {
                            oc[q] = h[u3][c];
                            oc2[q] = h2[u3][c];
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (C.any_noise) {
        // the actor's observation noise of s_t (side 0, step t_rec) and s_{t+1} (side 1, step
        // t_rec + 1): 9 Philox blocks per side, the 18 (side, block) pairs over the 8 warps
        if (jl < G && T_env[jl] >= 0) {
            const uint32_t env = (uint32_t)T_env[jl], t_rec = T_trec[jl];
            for (int pr = w; pr < 18; pr += LT / 32) {
                const int side = pr >= 9, blk = pr - 9 * side;
                float n0, n1;
                obs_noise_pair(C, env, t_rec + (uint32_t)side, blk, n0, n1);
                float* oax = (side ? T_oa2 : T_oa) + (size_t)jl * DA;
                oax[2 * blk] += n0;
                oax[2 * blk + 1] += n1;
                if (C.critic_layout == 3) {
                    float* ocx = (side ? T_oc2 : T_oc) + (size_t)jl * DC;
                    ocx[2 * blk] += n0;
                    ocx[2 * blk + 1] += n1;
                }
            }
        }
        __syncthreads();
    }
    // coalesced write-out of the six scratch ranges of this group
    const int n1 = G * DA, n2 = G * DC;
    for (int i = threadIdx.x; i < n1; i += LT) {
        S.oa[(size_t)g0 * DA + i] = T_oa[i];
        S.oa2[(size_t)g0 * DA + i] = T_oa2[i];
    }
    for (int i = threadIdx.x; i < n2; i += LT) {
        S.oc[(size_t)g0 * DC + i] = T_oc[i];
        S.oc2[(size_t)g0 * DC + i] = T_oc2[i];
    }
    if (threadIdx.x < G) {
        S.r[g0 + threadIdx.x] = T_r[threadIdx.x];
        S.term[g0 + threadIdx.x] = T_term[threadIdx.x];
    }
    __syncthreads();
}

// Gather of this CTA's Bc samples in groups of 32 (tile: shared memory, free at this point).
__device__ __forceinline__ void gather_all(const RunDesc& R, int j0, int Bc, uint32_t u,
                                           int64_t head, int64_t size, int64_t t_now,
                                           const Scr& S, float* sm) {
    for (int g0 = 0; g0 < Bc; g0 += 32) gather_group(R, j0, g0, min(32, Bc - g0), u, head, size, t_now, S, sm);
}

// Adam on parameters [lo, hi) from the sum of S gradient partials (partial s at
// gpart_base + s * part_stride + goff, summed in the order s = 0..S-1); with tg != nullptr
// the target copy also takes its Polyak step tg = tau th + (1 - tau) tg from the new th
// (the fused form of polyak_slice, for steps that update the targets).
__device__ void adam_slice(float* th, const float* gpart_base, size_t part_stride, int S,
                           int goff, float* m, float* v, int lo, int hi, int64_t t,
                           const LearnHyper& hp, float gscale, float* tg = nullptr) {
    const float bc1 = 1.0f - powf(hp.beta1, (float)t);
    const float bc2 = 1.0f - powf(hp.beta2, (float)t);
    const float tau = hp.tau;
    // U elements per thread per pass, all their loads issued before the arithmetic (8 was
    // measured no faster on the batched runs and 2.4 % slower on the single run)
    constexpr int U = 4;
    for (int i0 = lo + threadIdx.x; i0 < hi; i0 += U * LT) {
        float g[U], mo[U], vo[U], to[U], tt[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = i0 + k * LT;
            g[k] = 0.0f; mo[k] = 0.0f; vo[k] = 0.0f; to[k] = 0.0f; tt[k] = 0.0f;
            if (i < hi) {
                mo[k] = m[i]; vo[k] = v[i]; to[k] = th[i];
                if (tg) tt[k] = tg[i];
            }
        }
        // partials in batches of 4 (4 x U loads in flight)
        for (int s0 = 0; s0 < S; s0 += 4) {
            float x[4][U];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float* gp = gpart_base + (size_t)(s0 + q) * part_stride + goff;
#pragma unroll
                for (int k = 0; k < U; ++k)
                    x[q][k] = s0 + q < S && i0 + k * LT < hi ? ldcg(gp + i0 + k * LT) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (s0 + q < S) g[k] += x[q][k];
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = i0 + k * LT;
            if (i >= hi) continue;
            const float gk = g[k] * gscale;
            const float mi = fmaf(hp.beta1, mo[k], (1.0f - hp.beta1) * gk);
            const float vi = fmaf(hp.beta2, vo[k], (1.0f - hp.beta2) * gk * gk);
            m[i] = mi;
            v[i] = vi;
            const float ti = to[k] - hp.lr * (mi / bc1) / (sqrtf(vi / bc2) + hp.eps);
            th[i] = ti;
            if (tg) tg[i] = fmaf(tau, ti, (1.0f - tau) * tt[k]);
        }
    }
}

__device__ void polyak_slice(float* tg, const float* src, int lo, int hi, float tau) {
    constexpr int U = 4;
    for (int i0 = lo + threadIdx.x; i0 < hi; i0 += U * LT) {
        float a[U], b[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = i0 + k * LT;
            a[k] = i < hi ? ldcg(src + i) : 0.0f;
            b[k] = i < hi ? tg[i] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (i0 + k * LT < hi) tg[i0 + k * LT] = fmaf(tau, a[k], (1.0f - tau) * b[k]);
    }
}

// Block-wide sum of v over threads (fixed order).
__device__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    float s = 0.0f;
    for (int i = 0; i < LT / 32; ++i) s += red[i];
    __syncthreads();
    return s;
}

// One TD3 update of run R by the cluster (rank `rk` of S).
__device__ __noinline__ void td3_update(RunDesc& R, int64_t head, int64_t size, int64_t t_now, uint32_t u,
                           int64_t& t_a, int64_t& t_c, const Scr& S, float* scr_base,
                           size_t scr_stride, int cl_base, int rk, int nS, float* sm) {
    const int B = R.B, Bc = B / nS, H = R.H, DA = R.DA, DC = R.DC, PA = R.PA, PC = R.PC;
    const LearnHyper& hp = R.hp;
    const int j0 = rk * Bc;
    // a9: gather
    gather_all(R, j0, Bc, u, head, size, t_now, S, sm);
    __syncthreads();
    // a10: target actor + smoothing
    mlp_fwd(R.actor_t, DA, H, 4, S.oa2, DA, Bc, S.X1, S.X2, S.mu, 4, true, sm);
    for (int jl = threadIdx.x; jl < Bc; jl += LT) {
        const uint32_t j = (uint32_t)(j0 + jl);
        const uint4 r0 = draw(R.C, j, u, TAG_SMOOTH, 0), r1 = draw(R.C, j, u, TAG_SMOOTH, 1);
        const float z[4] = {gauss(r0.x, r0.y), gauss(r0.z, r0.w), gauss(r1.x, r1.y), gauss(r1.z, r1.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float eps = clampf(hp.sigma_t * z[i], -hp.noise_clip, hp.noise_clip);
            S.oc2[(size_t)jl * DC + DC - 4 + i] = clampf(S.mu[jl * 4 + i] + eps, -1.0f, 1.0f);
        }
    }
    __syncthreads();
    // a11: twin target critics, clipped double-Q target
    mlp_fwd(R.c1_t, DC, H, 1, S.oc2, DC, Bc, S.X1, S.X2, S.q1, 1, false, sm);
    mlp_fwd(R.c2_t, DC, H, 1, S.oc2, DC, Bc, S.X1, S.X2, S.q2, 1, false, sm);
    for (int jl = threadIdx.x; jl < Bc; jl += LT) {
        const float qmin = fminf(S.q1[jl], S.q2[jl]);
        S.y[jl] = S.r[jl] + (S.term[jl] != 0.0f ? 0.0f : hp.gamma * qmin);
    }
    __syncthreads();
    // a12: critic regression, forward + backward on this CTA's samples
    mlp_fwd(R.c1, DC, H, 1, S.oc, DC, Bc, S.H1a, S.H2a, S.q1, 1, false, sm);
    mlp_fwd(R.c2, DC, H, 1, S.oc, DC, Bc, S.H1b, S.H2b, S.q2, 1, false, sm);
    float lsum = 0.0f;
    for (int jl = threadIdx.x; jl < Bc; jl += LT) {
        const float e1 = S.q1[jl] - S.y[jl], e2 = S.q2[jl] - S.y[jl];
        S.dz3[jl] = 2.0f * e1 / (float)B;
        S.da[jl] = 2.0f * e2 / (float)B;
        lsum += (e1 * e1 + e2 * e2) / (float)B;
    }
    lsum = block_sum(lsum, sm + SMEM_MAIN);
    if (threadIdx.x == 0) S.loss[0] = lsum;
    __syncthreads();
    mlp_bwd(R.c1, DC, H, 1, S.oc, DC, Bc, S.H1a, S.H2a, S.dz3, S.dZ2, S.dZ1, S.g1, nullptr, 0, sm);
    mlp_bwd(R.c2, DC, H, 1, S.oc, DC, Bc, S.H1b, S.H2b, S.da, S.dZ2, S.dZ1, S.g2, nullptr, 0, sm);
    cluster_sync_all(nS);
    // a14 (critics): reduce the partials over the cluster and apply Adam to this slice
    t_c += 1;
    {
        const size_t g1off = (size_t)(S.g1 - scr_base), g2off = (size_t)(S.g2 - scr_base);
        const float* cl0 = scr_base - (size_t)rk * scr_stride;  // scratch of cluster rank 0
        const int lo = (int)((int64_t)PC * rk / nS), hi = (int)((int64_t)PC * (rk + 1) / nS);
        adam_slice(R.c1, cl0, scr_stride, nS, (int)g1off, R.m_c1, R.v_c1, lo, hi, t_c, hp, 1.0f);
        adam_slice(R.c2, cl0, scr_stride, nS, (int)g2off, R.m_c2, R.v_c2, lo, hi, t_c, hp, 1.0f);
        if (rk == 0 && threadIdx.x == 0) {
            float l = 0.0f;
            for (int s = 0; s < nS; ++s) l += ldcg(cl0 + (size_t)s * scr_stride + (S.loss - scr_base));
            R.stats[0] = l;
        }
    }
    cluster_sync_all(nS);
    // a13: delayed actor update through the updated first critic
    if ((int64_t)(u % (uint32_t)hp.policy_delay) != (int64_t)(hp.policy_delay - 1)) return;
    mlp_fwd(R.actor, DA, H, 4, S.oa, DA, Bc, S.X1, S.X2, S.mu, 4, true, sm);
    for (int i = threadIdx.x; i < Bc * 4; i += LT) {
        const int jl = i >> 2, c = i & 3;
        S.oc[(size_t)jl * DC + DC - 4 + c] = S.mu[i];
    }
    __syncthreads();
    mlp_fwd(R.c1, DC, H, 1, S.oc, DC, Bc, S.H1a, S.H2a, S.q1, 1, false, sm);
    float qs = 0.0f;
    for (int jl = threadIdx.x; jl < Bc; jl += LT) {
        S.dz3[jl] = -1.0f / (float)B;
        qs += -S.q1[jl] / (float)B;
    }
    qs = block_sum(qs, sm + SMEM_MAIN);
    if (threadIdx.x == 0) S.loss[1] = qs;
    __syncthreads();
    // dQ1/d(input) restricted to the action columns [DC-4, DC) -> dX stored in oc2 rows
    mlp_bwd(R.c1, DC, H, 1, S.oc, DC, Bc, S.H1a, S.H2a, S.dz3, S.dZ2, S.dZ1, nullptr, S.oc2, DC - 4, sm);
    for (int i = threadIdx.x; i < Bc * 4; i += LT) {
        const int jl = i >> 2, c = i & 3;
        const float m = S.mu[i];
        S.da[i] = S.oc2[(size_t)jl * DC + DC - 4 + c] * (1.0f - m * m);
    }
    __syncthreads();
    mlp_bwd(R.actor, DA, H, 4, S.oa, DA, Bc, S.X1, S.X2, S.da, S.dZ2, S.dZ1, S.ga, nullptr, 0, sm);
    cluster_sync_all(nS);
    t_a += 1;
    {
        const size_t gaoff = (size_t)(S.ga - scr_base);
        const float* cl0 = scr_base - (size_t)rk * scr_stride;
        const int lo = (int)((int64_t)PA * rk / nS), hi = (int)((int64_t)PA * (rk + 1) / nS);
        adam_slice(R.actor, cl0, scr_stride, nS, (int)gaoff, R.m_a, R.v_a, lo, hi, t_a, hp, 1.0f);
        if (rk == 0 && threadIdx.x == 0) {
            float l = 0.0f;
            for (int s = 0; s < nS; ++s) l += ldcg(cl0 + (size_t)s * scr_stride + (S.loss - scr_base) + 1);
            R.stats[1] = l;
        }
        __syncthreads();
        polyak_slice(R.actor_t, R.actor, lo, hi, hp.tau);
        const int clo = (int)((int64_t)PC * rk / nS), chi = (int)((int64_t)PC * (rk + 1) / nS);
        polyak_slice(R.c1_t, R.c1, clo, chi, hp.tau);
        polyak_slice(R.c2_t, R.c2, clo, chi, hp.tau);
    }
    cluster_sync_all(nS);
}

// ------------------------------------------------ tensor-core forward pass (tcgen05)
// Forward of a CTA's Bc rows (Bc a multiple of 128) through a network in -> H -> H -> out
// (in <= 96, H in {32, 64, 128}): both hidden layers as tcgen05 MMAs (M 128 rows, N = H,
// K = 16) on fp16 hi/lo operands in shared memory (three products per FP32-accurate
// product), accumulators in tensor memory; bias, ReLU and the 4- or 1-wide output layer on
// the CUDA cores.  One thread issues the MMAs and commits them to an mbarrier that every
// thread waits on (bounded).  Shared memory is the learner's engine region, laid out here
// per call: W1 hi/lo [H][96], W2 hi/lo [H][H], the tile operand hi/lo (X [128][96], then the
// first hidden layer [128][H] in place), b1, b2, W3, b3, partial outputs, the mbarrier.
namespace tcf {
constexpr int KP = 96, KC1 = KP / 8;
constexpr int TMEM_COLS = 256;  // D1 [128 x H] at column 0, D2 at column H (H <= 128)
constexpr int WAIT_POLLS = 1 << 24;
struct Lay {
    int w1h, w1l, w2h, w2l, th, tl, b1, b2, w3, b3, part, bar, end;
};
__host__ __device__ constexpr Lay lay(int H) {
    const int w1 = H * KP * 2, w2 = H * H * 2, t = 128 * (H > KP ? H : KP) * 2;
    Lay L{};
    L.w1h = 0; L.w1l = w1; L.w2h = 2 * w1; L.w2l = 2 * w1 + w2; L.th = 2 * w1 + 2 * w2; L.tl = L.th + t;
    L.b1 = L.tl + t; L.b2 = L.b1 + 4 * H; L.w3 = L.b2 + 4 * H; L.b3 = L.w3 + 16 * H;
    L.part = L.b3 + 16; L.bar = L.part + 2 * 128 * 4 * 4; L.end = L.bar + 16;
    return L;
}
static_assert(lay(128).end <= 4 * SMEM_MAIN, "tensor-core forward: shared memory");

__device__ __forceinline__ bool eligible(const RunDesc& R, int Bc) {
    return Bc % 128 == 0 && (R.H == 32 || R.H == 64 || R.H == 128) && R.DA <= KP && R.DC <= KP;
}

// rows of 8 consecutive inputs -> packed hi / lo halves (zero beyond `in`)
__device__ __forceinline__ void split8(const float* src, int k0, int in, uint4& hi, uint4& lo) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = k0 + e < in ? ldcg(src + k0 + e) : 0.0f;
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) tc::split2(v[2 * e], v[2 * e + 1], h[e], l[e]);
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}
}  // namespace tcf

__device__ __noinline__ void tc_forward(const float* W, int in, int H, int out, const float* X, int ldx,
                                        int Bc, float* Y, int ldy, bool tanh_out, float* sm, uint32_t tmem,
                                        int* status) {
    using namespace tcf;
    unsigned char* smb = reinterpret_cast<unsigned char*>(sm);
    const Lay L = lay(H);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KC2 = H / 8;
    const float* gb1 = W + H * in;
    const float* gW2 = gb1 + H;
    const float* gb2 = gW2 + H * H;
    const float* gW3 = gb2 + H;
    const float* gb3 = gW3 + out * H;
    __half* w1h = reinterpret_cast<__half*>(smb + L.w1h);
    __half* w1l = reinterpret_cast<__half*>(smb + L.w1l);
    __half* w2h = reinterpret_cast<__half*>(smb + L.w2h);
    __half* w2l = reinterpret_cast<__half*>(smb + L.w2l);
    __half* th = reinterpret_cast<__half*>(smb + L.th);
    __half* tl = reinterpret_cast<__half*>(smb + L.tl);
    float* b1 = reinterpret_cast<float*>(smb + L.b1);
    float* b2 = reinterpret_cast<float*>(smb + L.b2);
    float* W3 = reinterpret_cast<float*>(smb + L.w3);
    float* b3 = reinterpret_cast<float*>(smb + L.b3);
    float* part = reinterpret_cast<float*>(smb + L.part);  // [2][128][4]
    const uint32_t bar = tc::smem_u32(smb + L.bar);
    // stage the weights as hi / lo halves in the canonical K-major layout
    for (int i = tid; i < H * KC1; i += LT) {
        const int n = i / KC1, kc = i - n * KC1;
        uint4 hi, lo;
        split8(W + (size_t)n * in, 8 * kc, in, hi, lo);
        *reinterpret_cast<uint4*>(w1h + tc::cano16(n, 8 * kc, KC1)) = hi;
        *reinterpret_cast<uint4*>(w1l + tc::cano16(n, 8 * kc, KC1)) = lo;
    }
    for (int i = tid; i < H * KC2; i += LT) {
        const int n = i / KC2, kc = i - n * KC2;
        uint4 hi, lo;
        split8(gW2 + (size_t)n * H, 8 * kc, H, hi, lo);
        *reinterpret_cast<uint4*>(w2h + tc::cano16(n, 8 * kc, KC2)) = hi;
        *reinterpret_cast<uint4*>(w2l + tc::cano16(n, 8 * kc, KC2)) = lo;
    }
    for (int i = tid; i < H; i += LT) {
        b1[i] = ldcg(gb1 + i);
        b2[i] = ldcg(gb2 + i);
    }
    for (int i = tid; i < out * H; i += LT) W3[i] = ldcg(gW3 + i);
    if (tid < out) b3[tid] = ldcg(gb3 + tid);
    if (tid == 0) tc::bar_init(bar, 1);
    uint32_t phase = 0;
    const uint32_t idesc = tc::idesc_f16(H);
    const uint32_t d1 = tmem, d2 = tmem + (uint32_t)H;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const int half = warp >> 2;                 // column half of the epilogues
    const int r = 32 * (warp & 3) + lane;       // tile row of this thread in the epilogues
    const int cbeg = half * (H / 2), cend = cbeg + H / 2;
    for (int t0 = 0; t0 < Bc; t0 += 128) {
        // input tile -> hi / lo halves
        for (int i = tid; i < 128 * KC1; i += LT) {
            const int rr = i / KC1, kc = i - rr * KC1;
            uint4 hi, lo;
            split8(X + (size_t)(t0 + rr) * ldx, 8 * kc, in, hi, lo);
            *reinterpret_cast<uint4*>(th + tc::cano16(rr, 8 * kc, KC1)) = hi;
            *reinterpret_cast<uint4*>(tl + tc::cano16(rr, 8 * kc, KC1)) = lo;
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < KP / 16; ++j) {
                const uint32_t ko = (uint32_t)j * 256u;
                const uint64_t ah = tc::sdesc(tc::smem_u32(th) + ko, KC1), al = tc::sdesc(tc::smem_u32(tl) + ko, KC1);
                const uint64_t bh = tc::sdesc(tc::smem_u32(w1h) + ko, KC1), bl = tc::sdesc(tc::smem_u32(w1l) + ko, KC1);
                tc::mma_ss(d1, ah, bh, idesc, j > 0);
                tc::mma_ss(d1, ah, bl, idesc, 1);
                tc::mma_ss(d1, al, bh, idesc, 1);
            }
            tc::commit(bar);
        }
        if (!tc::bar_wait(bar, phase, WAIT_POLLS) && lane == 0 && status) atomicCAS(status, DEV_OK, DEV_TIMEOUT);
        phase ^= 1u;
        tc::fence_after();
        // epilogue 1: bias, ReLU, split -> the tile buffer as the layer-2 operand
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            uint32_t v[16];
            tc::ld16(d1 + lane_off + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = c0 + 8 * q + 2 * e;
                    const float x0 = fmaxf(__uint_as_float(v[8 * q + 2 * e]) + b1[c], 0.0f);
                    const float x1 = fmaxf(__uint_as_float(v[8 * q + 2 * e + 1]) + b1[c + 1], 0.0f);
                    tc::split2(x0, x1, h[e], l[e]);
                }
                const int off = tc::cano16(r, c0 + 8 * q, KC2);
                *reinterpret_cast<uint4*>(th + off) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(tl + off) = make_uint4(l[0], l[1], l[2], l[3]);
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            for (int j = 0; j < H / 16; ++j) {
                const uint32_t ko = (uint32_t)j * 256u;
                const uint64_t ah = tc::sdesc(tc::smem_u32(th) + ko, KC2), al = tc::sdesc(tc::smem_u32(tl) + ko, KC2);
                const uint64_t bh = tc::sdesc(tc::smem_u32(w2h) + ko, KC2), bl = tc::sdesc(tc::smem_u32(w2l) + ko, KC2);
                tc::mma_ss(d2, ah, bh, idesc, j > 0);
                tc::mma_ss(d2, ah, bl, idesc, 1);
                tc::mma_ss(d2, al, bh, idesc, 1);
            }
            tc::commit(bar);
        }
        if (!tc::bar_wait(bar, phase, WAIT_POLLS) && lane == 0 && status) atomicCAS(status, DEV_OK, DEV_TIMEOUT);
        phase ^= 1u;
        tc::fence_after();
        // epilogue 2: bias, ReLU, the output layer's partial sums over this warp's columns
        float po[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            uint32_t v[16];
            tc::ld16(d2 + lane_off + (uint32_t)c0, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int c = c0 + e;
                const float h2 = fmaxf(__uint_as_float(v[e]) + b2[c], 0.0f);
#pragma unroll
                for (int o = 0; o < 4; ++o)
                    if (o < out) po[o] = fmaf(W3[o * H + c], h2, po[o]);
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) part[(half * 128 + r) * 4 + o] = po[o];
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid < 128) {
            for (int o = 0; o < out; ++o) {
                const float y = part[tid * 4 + o] + part[(128 + tid) * 4 + o] + b3[o];
                Y[(size_t)(t0 + tid) * ldy + o] = tanh_out ? tanhf(y) : y;
            }
        }
        __syncthreads();  // the tile buffer and the partials are reused by the next tile
    }
}

// One TD3 update with every network pass resident in shared memory (hidden <= 64, or the
// 128-wide engine shape for HT = 128): same phases and cluster reduction as td3_update.  HT/DAT/DCT fix the hidden width and the
// actor/critic input widths at compile time (0: taken from the run descriptor), so that the
// common shapes get fully unrolled shared-memory GEMMs.
template <int HT, int DAT, int DCT>
__device__ __noinline__ void td3_update_smem(RunDesc& R, int64_t head, int64_t size, int64_t t_now,
                                             uint32_t u, int64_t& t_a, int64_t& t_c, const Scr& S,
                                             float* scr_base, size_t scr_stride, int rk, int nS,
                                             float* sm, uint32_t tmem, bool tmem_ok) {
    using namespace smlp;
    const int B = R.B, Bc = B / nS, PA = R.PA, PC = R.PC;
    const int H = HT ? HT : R.H, DA = DAT ? DAT : R.DA, DC = DCT ? DCT : R.DC;
    const LearnHyper& hp = R.hp;
    const int j0 = rk * Bc;
    Buf b = HT == 128 ? carve2(sm) : carve(sm);  // the 64-wide shape is never re-bound
    const int MC = b.mc;
    float* red = sm + SMEM_MAIN;
    // a9: gather
    gather_all(R, j0, Bc, u, head, size, t_now, S, sm);
    __syncthreads();
    // the pure forward passes (target actor, target critics) on the tensor cores when the
    // CTA holds whole 128-row tiles
    const bool tcf_on = tmem_ok && tcf::eligible(R, Bc);
    // With an even cluster whose CTA pairs' rows fit one chunk, the twin critics are split
    // over the two halves: CTA rk runs critic cs = rk / half (target and current) on the
    // rows of the pair (rr, rr + half), rr = rk mod half, read from both owners' scratch.
    const int half = nS >> 1;
    const bool split = !tcf_on && half > 0 && (nS & 1) == 0 && 2 * Bc <= MC;
    const int cs = split ? rk / half : 0, rr = split ? rk - cs * half : rk;
    const ptrdiff_t d0 = (ptrdiff_t)(rr - rk) * (ptrdiff_t)scr_stride;
    const ptrdiff_t d1 = (ptrdiff_t)(rr + half - rk) * (ptrdiff_t)scr_stride;
    // a10: target actor + smoothing
    if (tcf_on) {
        tc_forward(R.actor_t, DA, H, 4, S.oa2, DA, Bc, S.mu, 4, true, sm, tmem, R.E.status);
    } else {
        stage(R.actor_t, DA, H, 4, b);
        for (int r0 = 0; r0 < Bc; r0 += MC) forward(DA, H, 4, S.oa2, DA, r0, min(MC, Bc - r0), b, S.mu, 4, true);
    }
    for (int jl = threadIdx.x; jl < Bc; jl += LT) {
        const uint32_t j = (uint32_t)(j0 + jl);
        const uint4 r0 = draw(R.C, j, u, TAG_SMOOTH, 0), r1 = draw(R.C, j, u, TAG_SMOOTH, 1);
        const float z[4] = {gauss(r0.x, r0.y), gauss(r0.z, r0.w), gauss(r1.x, r1.y), gauss(r1.z, r1.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float eps = clampf(hp.sigma_t * z[i], -hp.noise_clip, hp.noise_clip);
            S.oc2[(size_t)jl * DC + DC - 4 + i] = clampf(S.mu[jl * 4 + i] + eps, -1.0f, 1.0f);
        }
    }
    __syncthreads();
    // a11: twin target critics
    if (split) {
        cluster_sync_all(nS);  // the pair's o_c' rows are complete
        float* qt = cs ? S.q2 : S.q1;
        stage(cs ? R.c2_t : R.c1_t, DC, H, 1, b);
        forward2(DC, H, 1, S.oc2 + d0, S.oc2 + d1, DC, Bc, 2 * Bc, b, qt + d0, qt + d1, 1, false);
        cluster_sync_all(nS);  // both target values of the pair's rows are complete
    } else if (tcf_on) {
        tc_forward(R.c1_t, DC, H, 1, S.oc2, DC, Bc, S.q1, 1, false, sm, tmem, R.E.status);
        tc_forward(R.c2_t, DC, H, 1, S.oc2, DC, Bc, S.q2, 1, false, sm, tmem, R.E.status);
    } else {
        stage(R.c1_t, DC, H, 1, b);
        for (int r0 = 0; r0 < Bc; r0 += MC) forward(DC, H, 1, S.oc2, DC, r0, min(MC, Bc - r0), b, S.q1, 1, false);
        stage(R.c2_t, DC, H, 1, b);
        for (int r0 = 0; r0 < Bc; r0 += MC) forward(DC, H, 1, S.oc2, DC, r0, min(MC, Bc - r0), b, S.q2, 1, false);
    }
    if (!split) {
        for (int jl = threadIdx.x; jl < Bc; jl += LT) {
            const float qmin = fminf(S.q1[jl], S.q2[jl]);
            S.y[jl] = S.r[jl] + (S.term[jl] != 0.0f ? 0.0f : hp.gamma * qmin);
        }
    }
    __syncthreads();
    // a12: critic regression, forward + backward chunk by chunk
    float lsum = 0.0f;
    if (split) {
        // one chunk: the pair's 2 Bc rows through critic cs; Q into dz3 (scratch of this CTA)
        float* g = cs ? S.g2 : S.g1;
        stage(cs ? R.c2 : R.c1, DC, H, 1, b);
        if constexpr (HT == 128) bind_grads(b, g, DC, H, 1);
        forward2(DC, H, 1, S.oc + d0, S.oc + d1, DC, Bc, 2 * Bc, b, S.dz3, S.dz3 + Bc, 1, false);
        for (int r = threadIdx.x; r < 2 * Bc; r += LT) {
            const ptrdiff_t o = (r < Bc ? d0 : d1) + (r < Bc ? r : r - Bc);
            const float qmin = fminf(S.q1[o], S.q2[o]);
            const float y = S.r[o] + (S.term[o] != 0.0f ? 0.0f : hp.gamma * qmin);
            const float e = S.dz3[r] - y;
            b.dZ3s[r * 4] = 2.0f * e / (float)B;
            lsum += e * e / (float)B;
        }
        __syncthreads();
        backward(DC, H, 1, 0, 2 * Bc, b, true, true, nullptr, 0, 0);
        store_grads(g, DC, H, 1, b);
    }
    for (int c = 0; c < (split ? 0 : 2); ++c) {
        const float* W = c ? R.c2 : R.c1;
        float* q = c ? S.q2 : S.q1;
        stage(W, DC, H, 1, b);
        if constexpr (HT == 128) bind_grads(b, c ? S.g2 : S.g1, DC, H, 1);
        for (int r0 = 0; r0 < Bc; r0 += MC) {
            const int mc = min(MC, Bc - r0);
            forward(DC, H, 1, S.oc, DC, r0, mc, b, q, 1, false);
            for (int r = threadIdx.x; r < mc; r += LT) {
                const float e = q[r0 + r] - S.y[r0 + r];
                b.dZ3s[r * 4] = 2.0f * e / (float)B;
                lsum += e * e / (float)B;
            }
            __syncthreads();
            backward(DC, H, 1, r0, mc, b, r0 == 0, true, nullptr, 0, 0);
        }
        store_grads(c ? S.g2 : S.g1, DC, H, 1, b);
    }
    lsum = block_sum(lsum, red);
    if (threadIdx.x == 0) S.loss[0] = lsum;
    __syncthreads();
    cluster_sync_all(nS);
    // a14 (critics): reduce the partials over the cluster and apply Adam to this slice
    t_c += 1;
    {
        const size_t g1off = (size_t)(S.g1 - scr_base), g2off = (size_t)(S.g2 - scr_base);
        const float* cl0 = scr_base - (size_t)rk * scr_stride;
        const int lo = (int)((int64_t)PC * rk / nS), hi = (int)((int64_t)PC * (rk + 1) / nS);
        // split: critic 1's partials are in CTAs [0, half), critic 2's in [half, nS)
        const int np = split ? half : nS;
        // on steps that update the actor, the critics' targets take their Polyak step here
        // (the actor phase reads the critics, not their targets)
        const bool pol = (int64_t)(u % (uint32_t)hp.policy_delay) == (int64_t)(hp.policy_delay - 1);
        adam_slice(R.c1, cl0, scr_stride, np, (int)g1off, R.m_c1, R.v_c1, lo, hi, t_c, hp, 1.0f,
                   pol ? R.c1_t : nullptr);
        adam_slice(R.c2, cl0 + (split ? (size_t)half * scr_stride : 0), scr_stride, np, (int)g2off,
                   R.m_c2, R.v_c2, lo, hi, t_c, hp, 1.0f, pol ? R.c2_t : nullptr);
        if (rk == 0 && threadIdx.x == 0) {
            float l = 0.0f;
            for (int s2 = 0; s2 < nS; ++s2) l += ldcg(cl0 + (size_t)s2 * scr_stride + (S.loss - scr_base));
            R.stats[0] = l;
        }
    }
    cluster_sync_all(nS);
    // a13: delayed actor update through the updated first critic
    if ((int64_t)(u % (uint32_t)hp.policy_delay) != (int64_t)(hp.policy_delay - 1)) return;
    // mu(o_a) alone (no activations kept): a pure forward pass, on the tensor cores when the
    // CTA holds whole 128-row tiles
    if (tcf_on) {
        tc_forward(R.actor, DA, H, 4, S.oa, DA, Bc, S.mu, 4, true, sm, tmem, R.E.status);
    } else {
        stage(R.actor, DA, H, 4, b);
        for (int r0 = 0; r0 < Bc; r0 += MC) forward(DA, H, 4, S.oa, DA, r0, min(MC, Bc - r0), b, S.mu, 4, true);
    }
    for (int i = threadIdx.x; i < Bc * 4; i += LT) {
        const int jl = i >> 2, c = i & 3;
        S.oc[(size_t)jl * DC + DC - 4 + c] = S.mu[i];
    }
    __syncthreads();
    stage(R.c1, DC, H, 1, b);
    float qs = 0.0f;
    for (int r0 = 0; r0 < Bc; r0 += MC) {
        const int mc = min(MC, Bc - r0);
        forward(DC, H, 1, S.oc, DC, r0, mc, b, S.q1, 1, false);
        for (int r = threadIdx.x; r < mc; r += LT) {
            b.dZ3s[r * 4] = -1.0f / (float)B;
            qs += -S.q1[r0 + r] / (float)B;
        }
        __syncthreads();
        // dQ1/d(action columns) -> oc2 rows
        backward(DC, H, 1, r0, mc, b, false, false, S.oc2, DC, DC - 4);
    }
    qs = block_sum(qs, red);
    if (threadIdx.x == 0) S.loss[1] = qs;
    for (int i = threadIdx.x; i < Bc * 4; i += LT) {
        const int jl = i >> 2, c = i & 3;
        const float m = S.mu[i];
        S.da[i] = S.oc2[(size_t)jl * DC + DC - 4 + c] * (1.0f - m * m);
    }
    __syncthreads();
    stage(R.actor, DA, H, 4, b);
    if constexpr (HT == 128) bind_grads(b, S.ga, DA, H, 4);
    for (int r0 = 0; r0 < Bc; r0 += MC) {
        const int mc = min(MC, Bc - r0);
        forward(DA, H, 4, S.oa, DA, r0, mc, b, S.mu, 4, true);
        for (int i = threadIdx.x; i < mc * 4; i += LT) b.dZ3s[i] = S.da[r0 * 4 + i];
        __syncthreads();
        backward(DA, H, 4, r0, mc, b, r0 == 0, true, nullptr, 0, 0);
    }
    store_grads(S.ga, DA, H, 4, b);
    cluster_sync_all(nS);
    t_a += 1;
    {
        const size_t gaoff = (size_t)(S.ga - scr_base);
        const float* cl0 = scr_base - (size_t)rk * scr_stride;
        const int lo = (int)((int64_t)PA * rk / nS), hi = (int)((int64_t)PA * (rk + 1) / nS);
        adam_slice(R.actor, cl0, scr_stride, nS, (int)gaoff, R.m_a, R.v_a, lo, hi, t_a, hp, 1.0f, R.actor_t);
        if (rk == 0 && threadIdx.x == 0) {
            float l = 0.0f;
            for (int s2 = 0; s2 < nS; ++s2) l += ldcg(cl0 + (size_t)s2 * scr_stride + (S.loss - scr_base) + 1);
            R.stats[1] = l;
        }
    }
    cluster_sync_all(nS);
}

// Curriculum change + reward recalculation over the run's buffer, split over the cluster.
__device__ __noinline__ void curriculum_step(RunDesc& R, int64_t head, int64_t size, int rk, int nS) {
    if (rk == 0 && threadIdx.x == 0) {
        for (int i = 0; i < 7; ++i) {
            const float c = R.E.rewardC[i], x = c * R.cf[i];
            R.E.rewardC[i] = R.cf[i] >= 1.0f ? fminf(x, R.ct[i]) : fmaxf(x, R.ct[i]);
        }
        R.E.rewardC[7] = fmaxf(R.E.rewardC[7] * R.sig_f, R.sig_min);
    }
    cluster_sync_all(nS);
    if (!R.recalc || R.capacity == 0) return;
    float Cr[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Cr[i] = ldcg(R.E.rewardC + i);
    recalc_range(R.C, R.E, Cr, head, size, R.capacity, (uint64_t)rk * LT + threadIdx.x, (uint64_t)nS * LT);
    cluster_sync_all(nS);
}

// Persistent training kernel.  Cluster c walks runs order[off[c] .. off[c+1]).
__global__ void __launch_bounds__(LT) k_train(RunDesc* runs, const int* order, const int* off,
                                              int n_iters, int do_env, float* scratch,
                                              size_t scr_stride, int nS, int use_tc) {
    extern __shared__ __align__(16) float sm[];
    // tensor memory for the tensor-core forward passes, when some run of the launch has them
    __shared__ uint32_t tmem_slot;
    if (use_tc) {
        if ((threadIdx.x >> 5) == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(tc::smem_u32(&tmem_slot)), "r"(tcf::TMEM_COLS) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    const uint32_t tmem = use_tc ? tmem_slot : 0u;
    const int rk = nS > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int cl = blockIdx.x / nS;
    float* my = scratch + (size_t)blockIdx.x * scr_stride;
    for (int oi = off[cl]; oi < off[cl + 1]; ++oi) {
        RunDesc& R = runs[order[oi]];
        int64_t head = R.head, size = R.size, t_now = R.t_now, t_a = R.t_a, t_c = R.t_c, u = R.u;
        int64_t next_curr = R.next_curr;
        const int Bc = R.B / nS;
        const Scr S = carve(my, Bc, R.H, R.DA, R.DC, R.PA, R.PC, R.n_env);
        for (int it = 0; it < n_iters; ++it) {
            int n_upd = 1;
            if (do_env) {
                if (rk == 0) {
                    if (R.n_env <= 8 && R.H <= 128 && R.DA <= 128)
                        env_step_small(R, (uint32_t)t_now, head, sm);
                    else
                        env_step_cta(R, S, (uint32_t)t_now, head, sm);
                }
                t_now += 1;
                if (R.capacity > 0) {
                    head = head + 1 == R.capacity ? 0 : head + 1;
                    if (size < R.capacity) size += 1;
                }
                cluster_sync_all(nS);
                if (R.curr_interval > 0 && t_now * (int64_t)R.n_env >= next_curr) {
                    curriculum_step(R, head, size, rk, nS);
                    next_curr += R.curr_interval;
                }
                n_upd = t_now >= R.start_updates ? R.hp.updates_per_step : 0;
            }
            const bool resident = R.H <= smlp::HP && R.DC <= smlp::INP && R.DA <= smlp::INP;
            const bool resident128 = R.H == 128 && R.DA == 82 && R.DC == 90;
            for (int k = 0; k < n_upd; ++k) {
                if (resident) {
                    // specialised shapes: hidden 64 or 32 over 16 actions of history, and the
                    // privileged critic (82 + 4 + 6 motor/parameter inputs + 4 actions)
                    const int key = R.H * 1000000 + R.DA * 1000 + R.DC;
                    if (key == 64082090)
                        td3_update_smem<64, 82, 90>(R, head, size, t_now, (uint32_t)u, t_a, t_c, S,
                                                    my, scr_stride, rk, nS, sm, tmem, use_tc != 0);
                    else if (key == 32082090)
                        td3_update_smem<32, 82, 90>(R, head, size, t_now, (uint32_t)u, t_a, t_c, S,
                                                    my, scr_stride, rk, nS, sm, tmem, use_tc != 0);
                    else if (key == 64082096)
                        td3_update_smem<64, 82, 96>(R, head, size, t_now, (uint32_t)u, t_a, t_c, S,
                                                    my, scr_stride, rk, nS, sm, tmem, use_tc != 0);
                    else
                        td3_update_smem<0, 0, 0>(R, head, size, t_now, (uint32_t)u, t_a, t_c, S,
                                                 my, scr_stride, rk, nS, sm, tmem, use_tc != 0);
                } else if (resident128) {
                    // hidden 128 with 16 actions of history: the 128-wide engine shape
                    td3_update_smem<128, 82, 90>(R, head, size, t_now, (uint32_t)u, t_a, t_c, S, my,
                                                 scr_stride, rk, nS, sm, tmem, use_tc != 0);
                } else
                    td3_update(R, head, size, t_now, (uint32_t)u, t_a, t_c, S, my, scr_stride,
                               blockIdx.x - rk, rk, nS, sm);
                u += 1;
            }
        }
        cluster_sync_all(nS);
        if (rk == 0 && threadIdx.x == 0) {
            R.head = head; R.size = size; R.t_now = t_now; R.t_a = t_a; R.t_c = t_c; R.u = u;
            R.next_curr = next_curr;
        }
        cluster_sync_all(nS);
    }
    if (use_tc) {
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if ((threadIdx.x >> 5) == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tcf::TMEM_COLS) : "memory");
    }
}

// ------------------------------------------------------------------- initialisation
__global__ void k_init_params(float* P, int in, int h, int out, uint32_t net_id, uint32_t k0,
                              uint32_t k1, uint32_t run) {
    const int total = psize(in, h, out);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int sizes[6] = {h * in, h, h * h, h, out * h, out};
    const int fan[6] = {in, in, h, h, h, h};
    int blk = 0, acc = 0;
    while (blk < 5 && i >= acc + sizes[blk]) { acc += sizes[blk]; ++blk; }
    const float bound = 1.0f / sqrtf((float)fan[blk]);
    const uint4 r = philox((uint32_t)i >> 2, net_id, (TAG_INIT << 24), run, k0, k1);
    const uint32_t x = (i & 3) == 0 ? r.x : ((i & 3) == 1 ? r.y : ((i & 3) == 2 ? r.z : r.w));
    P[i] = bound * (2.0f * u01(x) - 1.0f);
}

static int grid_for(int64_t n, int b) { return (int)((n + b - 1) / b); }

static size_t learner_smem() { return sizeof(float) * (size_t)(SMEM_MAIN + 32); }


}  // namespace qsim

using namespace qsim;

// ---------------------------------------------------------------------------- ABI
static qsim_status fill_desc(ac_handle* a, qsim_handle* e, RunDesc& R) {
    memset(&R, 0, sizeof(R));
    if (!a || !e) return fail(QSIM_EINVAL, "null handle");
    R.C = e->dc;
    R.E = e->p;
    R.capacity = e->capacity; R.head = e->head; R.size = e->size; R.t_now = e->t_now;
    R.curr_interval = e->cfg.curriculum_interval;
    R.next_curr = e->next_curriculum;
    for (int i = 0; i < 7; ++i) { R.cf[i] = e->cfg.curriculum_factor[i]; R.ct[i] = e->cfg.curriculum_target[i]; }
    R.sig_f = e->cfg.sigma_factor; R.sig_min = e->cfg.sigma_min; R.recalc = e->cfg.recalc_rewards;
    R.n_env = e->n;
    R.actor = a->actor; R.actor_t = a->actor_t; R.c1 = a->c1; R.c1_t = a->c1_t; R.c2 = a->c2; R.c2_t = a->c2_t;
    R.m_a = a->m_a; R.v_a = a->v_a; R.m_c1 = a->m_c1; R.v_c1 = a->v_c1; R.m_c2 = a->m_c2; R.v_c2 = a->v_c2;
    R.stats = a->stats;
    R.H = a->hidden; R.B = a->batch; R.DA = a->obs_dim; R.DC = a->critic_in;
    R.PA = a->n_actor; R.PC = a->n_critic;
    R.t_a = a->t_actor; R.t_c = a->t_critic; R.u = a->updates;
    const int64_t lost = e->cfg.n_hist;
    R.start_updates = std::max<int64_t>((int64_t)e->cfg.learning_starts, 2 + lost);
    const ac_config& c = a->cfg;
    R.hp = LearnHyper{c.gamma, c.tau, c.lr, c.beta1, c.beta2, c.eps, c.sigma_target, c.noise_clip,
                      c.policy_delay, c.updates_per_step};
    R.idx_log = a->idx_log;
    return QSIM_OK;
}

static void read_back(ac_handle* a, qsim_handle* e, const RunDesc& R) {
    e->head = R.head; e->size = R.size; e->t_now = R.t_now; e->next_curriculum = R.next_curr;
    a->t_actor = R.t_a; a->t_critic = R.t_c; a->updates = R.u;
}

// Advances the counters of a run descriptor exactly as k_train does over n_iters
// iterations, so that the host knows them without reading the descriptor back.
static void advance_desc(RunDesc& R, int64_t n_iters, int do_env) {
    for (int64_t it = 0; it < n_iters; ++it) {
        int n_upd = 1;
        if (do_env) {
            R.t_now += 1;
            if (R.capacity > 0) {
                R.head = R.head + 1 == R.capacity ? 0 : R.head + 1;
                if (R.size < R.capacity) R.size += 1;
            }
            if (R.curr_interval > 0 && R.t_now * (int64_t)R.n_env >= R.next_curr) R.next_curr += R.curr_interval;
            n_upd = R.t_now >= R.start_updates ? R.hp.updates_per_step : 0;
        }
        for (int k = 0; k < n_upd; ++k) {
            R.t_c += 1;
            if ((int64_t)((uint32_t)R.u % (uint32_t)R.hp.policy_delay) == (int64_t)(R.hp.policy_delay - 1))
                R.t_a += 1;
            R.u += 1;
        }
    }
}

static int pick_cluster(const ac_handle* a, int n_runs) {
    if (a->cfg.cluster > 0) return a->cfg.cluster;
    if (n_runs >= 64) return 1;
    // a few runs: the widest cluster (16 CTAs, non-portable) that leaves each CTA >= 16
    // samples; at batch 256 that is 111.5 us per env step + update against 135.9 at 8 CTAs
    const int b = a->batch;
    int s = n_runs > 8 ? 2 : 16;
    while (s > 1 && (b % s || b / s < 16)) s >>= 1;
    return s;
}

static qsim_status validate_pair(const ac_handle* a, const qsim_handle* e) {
    if (!a || !e) return fail(QSIM_EINVAL, "null handle");
    int dev = -1;
    QCHECK_CUDA(cudaGetDevice(&dev));
    if (dev != a->device || dev != e->device)
        return fail(QSIM_EINVAL, "the current device (%d) is not the one the learner (%d) and env set (%d) "
                    "were created on", dev, a->device, e->device);
    if (e->capacity < 2) return fail(QSIM_ESTATE, "env set has no replay buffer");
    if (e->capacity < e->cfg.n_hist + 2)
        return fail(QSIM_EINVAL, "replay capacity %lld must exceed the history length + 1",
                    (long long)e->capacity);
    if (a->obs_dim != e->dc.obs_dim || a->critic_in != e->dc.cobs_dim + 4)
        return fail(QSIM_EINVAL, "learner and env set have different observation layouts");
    return QSIM_OK;
}

// Launch geometry of one run by itself: cluster size and per-CTA scratch (floats).
struct SingleRun {
    int nS = 1;
    size_t stride = 0;
};

// Checks shared by every single-run launch (ac_update, ac_update_static and the plain
// forms of ac_train).  do_env = 0: n_iters updates from the buffer as it is, which must
// already allow sampling.
static qsim_status prepare_single(const ac_handle* a, const qsim_handle* env, int do_env,
                                  int64_t n_iters, const char* who, SingleRun* out) {
    qsim_status s = validate_pair(a, env);
    if (s != QSIM_OK) return s;
    if (n_iters < 0) return fail(QSIM_EINVAL, "%s: negative count", who);
    if ((uint64_t)env->capacity * (uint64_t)env->n >= (1ull << 32))
        return fail(QSIM_EINVAL, "%s: replay buffer exceeds 2^32 transitions", who);
    if (do_env) {
        if (((env->t_now + n_iters) >> 32) != 0) return fail(QSIM_ESTATE, "%s: step counter exhausted", who);
    } else {
        const int64_t lost = env->size == env->capacity ? env->cfg.n_hist : 0;
        if (env->size - 1 - lost < 1)
            return fail(QSIM_ESTATE, "%s: replay buffer too small to sample (size=%lld)", who,
                        (long long)env->size);
        if (((a->updates + n_iters) >> 32) != 0) return fail(QSIM_ESTATE, "%s: update counter exhausted", who);
    }
    out->nS = pick_cluster(a, 1);
    if (a->batch % out->nS)
        return fail(QSIM_EINVAL, "%s: batch %d not divisible by cluster %d", who, a->batch, out->nS);
    out->stride = scratch_floats(a->batch / out->nS, a->hidden, a->obs_dim, a->critic_in, a->n_actor,
                                 a->n_critic, env->n);
    return QSIM_OK;
}

// Device image of one run's launch: the descriptor and a one-run schedule.
struct PackedRun {
    RunDesc run;
    int order[1];
    int off[2];
};
static_assert(sizeof(PackedRun) <= QSIM_STATIC_DESC_BYTES, "run descriptor exceeds its static area");
constexpr size_t kPackedBytes = (sizeof(PackedRun) + 255) & ~(size_t)255;

// Whether the run's pure forward passes go to the tensor cores (tcf::eligible on the device).
static bool tc_forward_wanted(const RunDesc& R, int nS) {
    const int Bc = R.B / nS;
    return Bc % 128 == 0 && (R.H == 32 || R.H == 64 || R.H == 128) && R.DA <= tcf::KP && R.DC <= tcf::KP;
}

static qsim_status launch_k_train(int grid, int nS, cudaStream_t st, RunDesc* d_runs, const int* d_order,
                                  const int* d_off, int64_t n_iters, int do_env, float* scratch,
                                  size_t stride, int use_tc) {
    if (n_iters > INT32_MAX) return fail(QSIM_EINVAL, "too many steps for one launch");
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(LT);
    lc.dynamicSmemBytes = learner_smem();
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (nS > 8) QCHECK_CUDA(cudaFuncSetAttribute(k_train, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    QCHECK_CUDA(cudaLaunchKernelEx(&lc, k_train, d_runs, d_order, d_off, (int)n_iters, do_env, scratch,
                                   stride, nS, use_tc));
    return QSIM_OK;
}

// One run, one launch of n_iters iterations.  desc_dev holds a PackedRun; when `mirror`
// is given it is the host copy of what desc_dev holds once the stream's earlier work has
// run, and the descriptor is uploaded only if the handles' state differs from it.
static qsim_status run_single(ac_handle* a, qsim_handle* env, int64_t n_iters, int do_env,
                              const SingleRun& L, unsigned char* desc_dev, float* scratch,
                              RunDesc* mirror, cudaStream_t st) {
    PackedRun pk;
    memset(&pk, 0, sizeof(pk));
    qsim_status s = fill_desc(a, env, pk.run);
    if (s != QSIM_OK) return s;
    pk.off[1] = 1;
    PackedRun* d_pk = reinterpret_cast<PackedRun*>(desc_dev);
    if (!mirror || memcmp(&pk.run, mirror, sizeof(RunDesc)) != 0) {
        // pageable source: the copy is staged before the call returns
        QCHECK_CUDA(cudaMemcpyAsync(d_pk, &pk, sizeof(pk), cudaMemcpyHostToDevice, st));
    }
    s = launch_k_train(L.nS, L.nS, st, &d_pk->run, d_pk->order, d_pk->off, n_iters, do_env, scratch, L.stride,
                       tc_forward_wanted(pk.run, L.nS) ? 1 : 0);
    if (s != QSIM_OK) {
        if (mirror) memset(mirror, 0xff, sizeof(RunDesc));  // unknown device state: upload next time
        return s;
    }
    advance_desc(pk.run, n_iters, do_env);
    read_back(a, env, pk.run);
    if (mirror) *mirror = pk.run;
    return QSIM_OK;
}

// The learner's own workspace for single-run launches: [PackedRun | scratch of the
// cluster], kept between calls, grown when a launch needs more.
struct LearnerCache {
    unsigned char* dev = nullptr;
    size_t bytes = 0;
    RunDesc mirror;
    LearnerCache() { memset(&mirror, 0xff, sizeof(mirror)); }
};

static qsim_status learner_run(ac_handle* a, qsim_handle* env, int64_t n_iters, int do_env,
                               const SingleRun& L, cudaStream_t st) {
    LearnerCache* c = static_cast<LearnerCache*>(a->cache);
    const size_t need = kPackedBytes + sizeof(float) * L.stride * (size_t)L.nS;
    if (c->bytes < need) {
        if (c->dev) {
            QCHECK_CUDA(cudaStreamSynchronize(st));
            cudaFree(c->dev);
            c->dev = nullptr;
            c->bytes = 0;
        }
        if (cudaMalloc((void**)&c->dev, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(QSIM_ENOMEM, "learner workspace of %zu bytes", need);
        }
        c->bytes = need;
        memset(&c->mirror, 0xff, sizeof(RunDesc));
    }
    return run_single(a, env, n_iters, do_env, L, c->dev, reinterpret_cast<float*>(c->dev + kPackedBytes),
                      &c->mirror, st);
}

// All runs in one persistent launch (clusters walk a longest-processing-time-first list).
// Estimated time of one training iteration of a run (microseconds; a fit to the persistent
// kernel's measured step times at one CTA per run and 8 envs, hidden 32-128, batch
// 128-512): the env step plus updates_per_step x (a part fixed per update: Adam over the
// parameters, barriers, weight staging; and a part per sample on a CTA: gather, the
// networks' passes).  Only its ratios matter: it balances the longest-processing-time-first
// assignment of runs to clusters, where a pure FLOP count left the small runs' fixed costs
// out and piled them onto the same clusters.
static double run_cost(const ac_handle* a, const qsim_handle* e, int nS) {
    const double h = a->hidden, b = (double)a->batch / std::max(1, nS);
    // the small-run env step (<= 8 envs, one env per lane group) or the CTA-wide one
    const double env = e->n <= 8 && a->hidden <= 128 ? 13.0 + 0.1 * h : 16.0 + 0.34 * h;
    const double per_sample = 1.042 + 3.98e-5 * (h * (a->obs_dim + a->critic_in) + 3.0 * h * h);
    const double upd = 32.3 + 0.71 * h + 0.0109 * h * h + b * per_sample;
    return env + std::max(1, (int)a->cfg.updates_per_step) * upd;
}

static qsim_status launch_train(std::vector<ac_handle*>& A, std::vector<qsim_handle*>& E,
                                int64_t n_iters, int do_env, int nS, cudaStream_t st,
                                int n_clusters_in) {
    const int n = (int)A.size();
    std::vector<RunDesc> D(n);
    size_t stride = 0;
    for (int i = 0; i < n; ++i) {
        qsim_status s = fill_desc(A[i], E[i], D[i]);
        if (s != QSIM_OK) return s;
        if (A[i]->batch % nS) return fail(QSIM_EINVAL, "batch %d not divisible by cluster %d", A[i]->batch, nS);
        stride = std::max(stride, scratch_floats(A[i]->batch / nS, A[i]->hidden, A[i]->obs_dim,
                                                 A[i]->critic_in, A[i]->n_actor, A[i]->n_critic, E[i]->n));
    }
    const int n_clusters = std::max(1, std::min(n, n_clusters_in));
    std::vector<int> order(n), off(n_clusters + 1, 0);
    {
        std::vector<double> cost(n);
        for (int i = 0; i < n; ++i) cost[i] = run_cost(A[i], E[i], nS);
        std::vector<int> idx(n);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<double> load(n_clusters, 0.0);
        std::vector<std::vector<int>> lists(n_clusters);
        for (int i : idx) {
            int best = 0;
            for (int c = 1; c < n_clusters; ++c)
                if (load[c] < load[best]) best = c;
            load[best] += cost[i];
            lists[best].push_back(i);
        }
        int k = 0;
        for (int c = 0; c < n_clusters; ++c) {
            off[c] = k;
            for (int i : lists[c]) order[k++] = i;
        }
        off[n_clusters] = k;
    }
    // device copies (stream-ordered; freed in stream order after the launch)
    RunDesc* d_runs;
    int *d_order, *d_off;
    float* scratch;
    const size_t scr_bytes = sizeof(float) * stride * (size_t)n_clusters * nS;
    QCHECK_CUDA(cudaMallocAsync((void**)&d_runs, sizeof(RunDesc) * n, st));
    QCHECK_CUDA(cudaMallocAsync((void**)&d_order, sizeof(int) * n, st));
    QCHECK_CUDA(cudaMallocAsync((void**)&d_off, sizeof(int) * (n_clusters + 1), st));
    QCHECK_CUDA(cudaMallocAsync((void**)&scratch, scr_bytes, st));
    QCHECK_CUDA(cudaMemcpyAsync(d_runs, D.data(), sizeof(RunDesc) * n, cudaMemcpyHostToDevice, st));
    QCHECK_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    QCHECK_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(int) * (n_clusters + 1), cudaMemcpyHostToDevice, st));
    int use_tc = 0;
    for (int i = 0; i < n; ++i) use_tc |= tc_forward_wanted(D[i], nS) ? 1 : 0;
    qsim_status s = launch_k_train(n_clusters * nS, nS, st, d_runs, d_order, d_off, n_iters, do_env,
                                   scratch, stride, use_tc);
    cudaFreeAsync(scratch, st);
    cudaFreeAsync(d_off, st);
    cudaFreeAsync(d_order, st);
    cudaFreeAsync(d_runs, st);
    if (s != QSIM_OK) return s;
    for (int i = 0; i < n; ++i) {
        advance_desc(D[i], n_iters, do_env);
        read_back(A[i], E[i], D[i]);
    }
    return QSIM_OK;
}

extern "C" qsim_status ac_create(const ac_config* cfg, const qsim_handle* env, ac_handle** out) {
    if (!cfg || !env || !out) return fail(QSIM_EINVAL, "ac_create: null pointer");
    *out = nullptr;
    if (cfg->hidden < 4 || cfg->hidden > 128 || (cfg->hidden % 4))
        return fail(QSIM_EINVAL, "ac_create: hidden=%d must be a multiple of 4 in [4,128]", cfg->hidden);
    if (cfg->batch < 1 || cfg->batch > 1024) return fail(QSIM_EINVAL, "ac_create: batch out of range");
    if (cfg->policy_delay < 1) return fail(QSIM_EINVAL, "ac_create: policy_delay < 1");
    if (cfg->cluster < 0 || cfg->cluster > 16 || (cfg->cluster & (cfg->cluster - 1)))
        return fail(QSIM_EINVAL, "ac_create: cluster must be 0 or a power of two <= 16");
    int dev = -1;
    QCHECK_CUDA(cudaGetDevice(&dev));
    if (dev != env->device)
        return fail(QSIM_EINVAL, "ac_create: the current device (%d) is not the env set's (%d)", dev, env->device);
    // the learner kernel needs more than the default 48 KB of dynamic shared memory (set on
    // the current device, where every launch for this learner happens)
    QCHECK_CUDA(cudaFuncSetAttribute(k_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)learner_smem()));
    ac_handle* a = new ac_handle();
    a->cfg = *cfg;
    if (a->cfg.updates_per_step < 1) a->cfg.updates_per_step = 1;
    a->device = dev;
    a->cache = new LearnerCache();
    a->idx_log = nullptr;
    a->obs_dim = env->dc.obs_dim;
    a->critic_in = env->dc.cobs_dim + 4;
    a->hidden = cfg->hidden;
    a->batch = cfg->batch;
    a->n_actor = a->hidden * a->obs_dim + a->hidden + a->hidden * a->hidden + a->hidden + 4 * a->hidden + 4;
    a->n_critic = a->hidden * a->critic_in + a->hidden + a->hidden * a->hidden + a->hidden + a->hidden + 1;
    a->t_actor = a->t_critic = a->updates = 0;
    const size_t PA = a->n_actor, PC = a->n_critic;
    const size_t total = 4 * PA + 8 * PC + 8;
    if (cudaMalloc((void**)&a->base, total * 4) != cudaSuccess ||
        cudaMalloc((void**)&a->status, 4) != cudaSuccess) {
        cudaGetLastError();
        ac_destroy(a);
        return fail(QSIM_ENOMEM, "ac_create: allocation failed");
    }
    cudaMemset(a->base, 0, total * 4);
    cudaMemset(a->status, 0, 4);
    float* p = a->base;
    a->actor = p; p += PA; a->actor_t = p; p += PA;
    a->c1 = p; p += PC; a->c1_t = p; p += PC; a->c2 = p; p += PC; a->c2_t = p; p += PC;
    a->m_a = p; p += PA; a->v_a = p; p += PA;
    a->m_c1 = p; p += PC; a->v_c1 = p; p += PC; a->m_c2 = p; p += PC; a->v_c2 = p; p += PC;
    a->stats = p;
    const uint32_t k0 = env->dc.key0, k1 = env->dc.key1, run = env->dc.run_id;
    k_init_params<<<grid_for(PA, 256), 256>>>(a->actor, a->obs_dim, a->hidden, 4, 0, k0, k1, run);
    k_init_params<<<grid_for(PC, 256), 256>>>(a->c1, a->critic_in, a->hidden, 1, 1, k0, k1, run);
    k_init_params<<<grid_for(PC, 256), 256>>>(a->c2, a->critic_in, a->hidden, 1, 2, k0, k1, run);
    cudaMemcpy(a->actor_t, a->actor, PA * 4, cudaMemcpyDeviceToDevice);
    cudaMemcpy(a->c1_t, a->c1, PC * 4, cudaMemcpyDeviceToDevice);
    cudaMemcpy(a->c2_t, a->c2, PC * 4, cudaMemcpyDeviceToDevice);
    cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        ac_destroy(a);
        return cuda_fail(err, "ac_create: init");
    }
    *out = a;
    return QSIM_OK;
}

extern "C" qsim_status ac_destroy(ac_handle* a) {
    if (!a) return QSIM_OK;
    LearnerCache* c = static_cast<LearnerCache*>(a->cache);
    if (c) {
        if (c->dev) {
            cudaDeviceSynchronize();
            cudaFree(c->dev);
        }
        delete c;
    }
    if (a->base) cudaFree(a->base);
    if (a->status) cudaFree(a->status);
    delete a;
    return QSIM_OK;
}

extern "C" qsim_status ac_info_get(const ac_handle* a, ac_info* o) {
    if (!a || !o) return fail(QSIM_EINVAL, "ac_info_get: null pointer");
    o->obs_dim = a->obs_dim; o->critic_in = a->critic_in; o->hidden = a->hidden; o->batch = a->batch;
    o->n_actor = a->n_actor; o->n_critic = a->n_critic;
    o->t_actor = a->t_actor; o->t_critic = a->t_critic; o->updates = a->updates;
    o->actor = a->actor; o->actor_t = a->actor_t; o->c1 = a->c1; o->c1_t = a->c1_t;
    o->c2 = a->c2; o->c2_t = a->c2_t; o->m_a = a->m_a; o->v_a = a->v_a;
    o->m_c1 = a->m_c1; o->v_c1 = a->v_c1; o->m_c2 = a->m_c2; o->v_c2 = a->v_c2;
    o->stats = a->stats;
    return QSIM_OK;
}

extern "C" qsim_status ac_set_counters(ac_handle* a, int64_t t_actor, int64_t t_critic, int64_t updates) {
    if (!a || t_actor < 0 || t_critic < 0 || updates < 0 || (updates >> 32))
        return fail(QSIM_EINVAL, "ac_set_counters: bad argument");
    a->t_actor = t_actor; a->t_critic = t_critic; a->updates = updates;
    return QSIM_OK;
}

extern "C" int32_t ac_set_cluster(ac_handle* a, int32_t cluster) {
    if (!a) return fail(QSIM_EINVAL, "ac_set_cluster: null handle");
    if (cluster < 0 || cluster > 16 || (cluster & (cluster - 1)))
        return fail(QSIM_EINVAL, "ac_set_cluster: cluster must be 0 or a power of two <= 16");
    const int32_t prev = a->cfg.cluster;
    a->cfg.cluster = cluster;
    return prev;
}

extern "C" qsim_status ac_set_index_log(ac_handle* a, uint32_t* idx) {
    if (!a) return fail(QSIM_EINVAL, "ac_set_index_log: null handle");
    if (reinterpret_cast<uintptr_t>(idx) & 3u) return fail(QSIM_EINVAL, "ac_set_index_log: misaligned pointer");
    a->idx_log = idx;
    return QSIM_OK;
}

extern "C" qsim_status ac_update(ac_handle* a, qsim_handle* env, int32_t n_updates, void* stream) {
    SingleRun L;
    qsim_status s = prepare_single(a, env, 0, n_updates, "ac_update", &L);
    if (s != QSIM_OK || n_updates == 0) return s;
    return learner_run(a, env, n_updates, 0, L, (cudaStream_t)stream);
}

// ------------------------------------------------- allocation-free learner update
// Scratch for ac_update_static(): a library-owned array in every device's global memory
// (held from library load until process exit), plus room for the run descriptor.
// Host code must not pass the symbol itself to a kernel (in host code it names a host-side
// stand-in); the device address comes from cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) float g_static_scratch[QSIM_STATIC_SCRATCH_BYTES / sizeof(float)];
static __device__ __align__(256) unsigned char g_static_desc[QSIM_STATIC_DESC_BYTES];

namespace {
struct StaticSlot {
    float* scratch = nullptr;
    unsigned char* desc = nullptr;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
StaticSlot g_static_slots[kMaxDevices];
std::mutex g_static_mutex;

// Resolves the device addresses of the static arrays for the current device (first call
// on each device only).
qsim_status static_slot(int device, StaticSlot** out) {
    if (device < 0 || device >= kMaxDevices) return fail(QSIM_EINVAL, "ac_update_static: device id %d", device);
    std::lock_guard<std::mutex> lock(g_static_mutex);
    StaticSlot& s = g_static_slots[device];
    if (!s.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "ac_update_static: cudaGetSymbolAddress(scratch)");
        s.scratch = static_cast<float*>(p);
        e = cudaGetSymbolAddress(&p, g_static_desc);
        if (e != cudaSuccess) return cuda_fail(e, "ac_update_static: cudaGetSymbolAddress(desc)");
        s.desc = static_cast<unsigned char*>(p);
        s.ready = true;
    }
    *out = &s;
    return QSIM_OK;
}
}  // namespace

extern "C" qsim_status ac_update_static(ac_handle* a, qsim_handle* env, int32_t n_updates,
                                        void* stream) {
    SingleRun L;
    qsim_status st = prepare_single(a, env, 0, n_updates, "ac_update_static", &L);
    if (st != QSIM_OK || n_updates == 0) return st;
    const size_t need = L.stride * sizeof(float) * (size_t)L.nS;
    if (need > QSIM_STATIC_SCRATCH_BYTES)
        return fail(QSIM_EINVAL,
                    "ac_update_static: needs %zu bytes of scratch (batch %d, hidden %d, cluster %d), "
                    "more than the static maximum of %d bytes; use ac_update",
                    need, a->batch, a->hidden, L.nS, (int)QSIM_STATIC_SCRATCH_BYTES);
    StaticSlot* slot = nullptr;
    st = static_slot(a->device, &slot);
    if (st != QSIM_OK) return st;
    // the shared descriptor area is rewritten on every call (no mirror)
    return run_single(a, env, n_updates, 0, L, slot->desc, slot->scratch, nullptr, (cudaStream_t)stream);
}

extern "C" qsim_status ac_train(ac_handle* const* runs, qsim_handle* const* envs, int32_t n_runs,
                                int64_t steps_per_run, int32_t persistent, void* stream) {
    if (!runs || !envs || n_runs < 1 || steps_per_run < 0 || persistent < 0 || persistent > 2)
        return fail(QSIM_EINVAL, "ac_train: bad argument");
    std::vector<ac_handle*> A(runs, runs + n_runs);
    std::vector<qsim_handle*> E(envs, envs + n_runs);
    std::vector<SingleRun> L(n_runs);
    for (int i = 0; i < n_runs; ++i) {
        qsim_status s = prepare_single(A[i], E[i], 1, steps_per_run, "ac_train", &L[i]);
        if (s != QSIM_OK) return s;
    }
    if (steps_per_run == 0) return QSIM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (persistent == 0) {
        // plain form: one launch per run and env step, each run on its own cluster size
        for (int64_t t = 0; t < steps_per_run; ++t)
            for (int i = 0; i < n_runs; ++i) {
                qsim_status s = learner_run(A[i], E[i], 1, 1, L[i], st);
                if (s != QSIM_OK) return s;
            }
        return QSIM_OK;
    }
    if (persistent == 2 || n_runs == 1) {
        // one launch per run for all its steps, runs one after another
        for (int i = 0; i < n_runs; ++i) {
            qsim_status s = learner_run(A[i], E[i], steps_per_run, 1, L[i], st);
            if (s != QSIM_OK) return s;
        }
        return QSIM_OK;
    }
    const int nS = pick_cluster(A[0], n_runs);
    for (int i = 1; i < n_runs; ++i)
        if (pick_cluster(A[i], n_runs) != nS) return fail(QSIM_EINVAL, "ac_train: runs need one cluster size");
    int max_clusters = 1;
    {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(nS * 1024);
        lc.blockDim = dim3(LT);
        lc.dynamicSmemBytes = learner_smem();
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = nS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        if (nS > 8) cudaFuncSetAttribute(k_train, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (cudaOccupancyMaxActiveClusters(&max_clusters, k_train, &lc) != cudaSuccess || max_clusters < 1) {
            cudaGetLastError();
            int sms = 152;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A[0]->device);
            max_clusters = std::max(1, sms / nS);
        }
    }
    return launch_train(A, E, steps_per_run, 1, nS, st, max_clusters);
}

// Autotuner of the batched launch: the cluster size S (CTAs per run) is timed on the runs
// themselves, every candidate that divides each run's batch with >= 16 samples per CTA.
extern "C" int32_t ac_train_autotune(ac_handle* const* runs, qsim_handle* const* envs, int32_t n_runs,
                                     int32_t trial_steps, void* stream) {
    if (!runs || !envs || n_runs < 1 || trial_steps < 1)
        return fail(QSIM_EINVAL, "ac_train_autotune: bad argument");
    for (int i = 0; i < n_runs; ++i)
        if (!runs[i] || !envs[i]) return fail(QSIM_EINVAL, "ac_train_autotune: null handle");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> saved(n_runs);
    for (int i = 0; i < n_runs; ++i) saved[i] = runs[i]->cfg.cluster;
    auto restore = [&]() { for (int i = 0; i < n_runs; ++i) runs[i]->cfg.cluster = saved[i]; };
    // one untimed call with the current setting: first-launch costs stay out of the trials
    qsim_status s0 = ac_train(runs, envs, n_runs, trial_steps, 1, stream);
    if (s0 != QSIM_OK) return s0;
    cudaEvent_t e0, e1;
    QCHECK_CUDA(cudaEventCreate(&e0));
    QCHECK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_s = 0;
    for (int cand : {1, 2, 4, 8, 16}) {
        bool ok = true;
        for (int i = 0; i < n_runs; ++i) {
            const int b = runs[i]->batch;
            if (b % cand || (cand > 1 && b / cand < 16)) ok = false;
        }
        if (!ok) continue;
        for (int i = 0; i < n_runs; ++i) runs[i]->cfg.cluster = cand;
        cudaEventRecord(e0, st);
        const qsim_status r = ac_train(runs, envs, n_runs, trial_steps, 1, stream);
        cudaEventRecord(e1, st);
        if (r != QSIM_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            restore();
            return r;
        }
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_s = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    QCHECK_LAUNCH("ac_train_autotune");
    for (int i = 0; i < n_runs; ++i) runs[i]->cfg.cluster = best_s;
    return best_s;
}

// ------------------------------------------------------------ graph-captured plans
struct ac_plan {
    std::vector<ac_handle*> A;
    std::vector<qsim_handle*> E;
    RunDesc* d_runs = nullptr;
    int* d_order = nullptr;
    int* d_off = nullptr;
    float* scratch = nullptr;
    size_t stride = 0;
    int nS = 1, n_clusters = 1, chunk = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t steps_run = 0;
};

extern "C" qsim_status ac_plan_destroy(ac_plan* p) {
    if (!p) return QSIM_OK;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_runs) cudaFree(p->d_runs);
    if (p->d_order) cudaFree(p->d_order);
    if (p->d_off) cudaFree(p->d_off);
    if (p->scratch) cudaFree(p->scratch);
    delete p;
    return QSIM_OK;
}

extern "C" qsim_status ac_plan_create(ac_handle* const* runs, qsim_handle* const* envs,
                                      int32_t n_runs, int32_t steps_per_chunk, ac_plan** out) {
    if (!runs || !envs || !out || n_runs < 1 || steps_per_chunk < 1)
        return fail(QSIM_EINVAL, "ac_plan_create: bad argument");
    *out = nullptr;
    ac_plan* p = new ac_plan();
    p->A.assign(runs, runs + n_runs);
    p->E.assign(envs, envs + n_runs);
    p->chunk = steps_per_chunk;
    for (int i = 0; i < n_runs; ++i) {
        qsim_status s = validate_pair(p->A[i], p->E[i]);
        if (s != QSIM_OK) { ac_plan_destroy(p); return s; }
        if ((uint64_t)p->E[i]->capacity * (uint64_t)p->E[i]->n >= (1ull << 32)) {
            ac_plan_destroy(p);
            return fail(QSIM_EINVAL, "ac_plan_create: replay buffer exceeds 2^32 transitions");
        }
    }
    p->nS = pick_cluster(p->A[0], n_runs);
    for (int i = 0; i < n_runs; ++i)
        if (pick_cluster(p->A[i], n_runs) != p->nS || p->A[i]->batch % p->nS) {
            ac_plan_destroy(p);
            return fail(QSIM_EINVAL, "ac_plan_create: runs need one cluster size dividing every batch");
        }
    const int nS = p->nS;
    int max_clusters = 1;
    {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(nS * 1024);
        lc.blockDim = dim3(LT);
        lc.dynamicSmemBytes = learner_smem();
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = nS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        if (nS > 8) cudaFuncSetAttribute(k_train, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (cudaOccupancyMaxActiveClusters(&max_clusters, k_train, &lc) != cudaSuccess || max_clusters < 1) {
            cudaGetLastError();
            int sms = 152;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->A[0]->device);
            max_clusters = std::max(1, sms / nS);
        }
    }
    const int n = n_runs;
    p->n_clusters = std::max(1, std::min(n, max_clusters));
    std::vector<RunDesc> D(n);
    for (int i = 0; i < n; ++i) {
        qsim_status s = fill_desc(p->A[i], p->E[i], D[i]);
        if (s != QSIM_OK) { ac_plan_destroy(p); return s; }
        p->stride = std::max(p->stride, scratch_floats(p->A[i]->batch / nS, p->A[i]->hidden,
                                                       p->A[i]->obs_dim, p->A[i]->critic_in,
                                                       p->A[i]->n_actor, p->A[i]->n_critic, p->E[i]->n));
    }
    int use_tc = 0;
    for (int i = 0; i < n; ++i) use_tc |= tc_forward_wanted(D[i], nS) ? 1 : 0;
    // longest-processing-time-first assignment of runs to clusters
    std::vector<int> order(n), off(p->n_clusters + 1, 0);
    {
        std::vector<double> cost(n);
        for (int i = 0; i < n; ++i) cost[i] = run_cost(p->A[i], p->E[i], nS);
        std::vector<int> idx(n);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<double> load(p->n_clusters, 0.0);
        std::vector<std::vector<int>> lists(p->n_clusters);
        for (int i : idx) {
            int best = 0;
            for (int c = 1; c < p->n_clusters; ++c)
                if (load[c] < load[best]) best = c;
            load[best] += cost[i];
            lists[best].push_back(i);
        }
        int k = 0;
        for (int c = 0; c < p->n_clusters; ++c) {
            off[c] = k;
            for (int i : lists[c]) order[k++] = i;
        }
        off[p->n_clusters] = k;
    }
    const size_t scr_bytes = sizeof(float) * p->stride * (size_t)p->n_clusters * nS;
    if (cudaMalloc((void**)&p->d_runs, sizeof(RunDesc) * n) != cudaSuccess ||
        cudaMalloc((void**)&p->d_order, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc((void**)&p->d_off, sizeof(int) * (p->n_clusters + 1)) != cudaSuccess ||
        cudaMalloc((void**)&p->scratch, scr_bytes) != cudaSuccess) {
        cudaGetLastError();
        ac_plan_destroy(p);
        return fail(QSIM_ENOMEM, "ac_plan_create: allocation failed");
    }
    cudaMemcpy(p->d_runs, D.data(), sizeof(RunDesc) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_off, off.data(), sizeof(int) * (p->n_clusters + 1), cudaMemcpyHostToDevice);
    // capture one chunk of the persistent launch
    cudaStream_t cs;
    QCHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(p->n_clusters * nS);
    lc.blockDim = dim3(LT);
    lc.dynamicSmemBytes = learner_smem();
    lc.stream = cs;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess)
        e = cudaLaunchKernelEx(&lc, k_train, p->d_runs, (const int*)p->d_order, (const int*)p->d_off,
                               steps_per_chunk, 1, p->scratch, p->stride, nS, use_tc);
    cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        ac_plan_destroy(p);
        return cuda_fail(e, "ac_plan_create: graph capture");
    }
    *out = p;
    return QSIM_OK;
}

extern "C" qsim_status ac_plan_run(ac_plan* p, int32_t n_chunks, void* stream) {
    if (!p || n_chunks < 0) return fail(QSIM_EINVAL, "ac_plan_run: bad argument");
    for (size_t i = 0; i < p->E.size(); ++i)
        if (((p->E[i]->t_now + p->steps_run + (int64_t)n_chunks * p->chunk) >> 32) != 0)
            return fail(QSIM_ESTATE, "ac_plan_run: step counter exhausted");
    for (int c = 0; c < n_chunks; ++c) QCHECK_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    p->steps_run += (int64_t)n_chunks * p->chunk;
    return QSIM_OK;
}

extern "C" qsim_status ac_plan_sync(ac_plan* p, void* stream) {
    if (!p) return fail(QSIM_EINVAL, "ac_plan_sync: null plan");
    const size_t n = p->A.size();
    std::vector<RunDesc> D(n);
    QCHECK_CUDA(cudaMemcpyAsync(D.data(), p->d_runs, sizeof(RunDesc) * n, cudaMemcpyDeviceToHost,
                                (cudaStream_t)stream));
    QCHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (size_t i = 0; i < n; ++i) read_back(p->A[i], p->E[i], D[i]);
    p->steps_run = 0;
    return QSIM_OK;
}

extern "C" qsim_status ac_sync(ac_handle* a) {
    if (!a) return fail(QSIM_EINVAL, "ac_sync: null handle");
    QCHECK_CUDA(cudaDeviceSynchronize());
    return QSIM_OK;
}

// ------------------------------------------------------------------------ checkpoints
namespace {
struct CkptHeader {
    char magic[8];
    int32_t abi, obs_dim, critic_in, hidden, n_actor, n_critic, n_env, ld;
    int64_t t_actor, t_critic, updates, t_now, head, size, next_curr;
};
}  // namespace

extern "C" qsim_status ac_save(const ac_handle* a, const qsim_handle* e, const char* path) {
    if (!a || !e || !path) return fail(QSIM_EINVAL, "ac_save: null pointer");
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "QSIMCKP1", 8);
    h.abi = QSIM_ABI_VERSION; h.obs_dim = a->obs_dim; h.critic_in = a->critic_in; h.hidden = a->hidden;
    h.n_actor = a->n_actor; h.n_critic = a->n_critic; h.n_env = e->n; h.ld = e->ld;
    h.t_actor = a->t_actor; h.t_critic = a->t_critic; h.updates = a->updates;
    h.t_now = e->t_now; h.head = e->head; h.size = e->size; h.next_curr = e->next_curriculum;
    const size_t nparam = 4 * (size_t)a->n_actor + 8 * (size_t)a->n_critic;
    std::vector<float> w(nparam);
    QCHECK_CUDA(cudaDeviceSynchronize());
    QCHECK_CUDA(cudaMemcpy(w.data(), a->base, nparam * 4, cudaMemcpyDeviceToHost));
    const size_t ld = e->ld;
    std::vector<float> env_f((NS + 8 + 6 + 4 * HMAX + 2) * ld + 8);
    std::vector<uint32_t> env_u(4 * ld);
    float* f = env_f.data();
    QCHECK_CUDA(cudaMemcpy(f, e->p.state, NS * ld * 4, cudaMemcpyDeviceToHost)); f += NS * ld;
    QCHECK_CUDA(cudaMemcpy(f, e->p.prm, 8 * ld * 4, cudaMemcpyDeviceToHost)); f += 8 * ld;
    QCHECK_CUDA(cudaMemcpy(f, e->p.dist, 6 * ld * 4, cudaMemcpyDeviceToHost)); f += 6 * ld;
    QCHECK_CUDA(cudaMemcpy(f, e->p.hist, 4 * HMAX * ld * 4, cudaMemcpyDeviceToHost)); f += 4 * HMAX * ld;
    QCHECK_CUDA(cudaMemcpy(f, e->p.ep_ret, ld * 4, cudaMemcpyDeviceToHost)); f += ld;
    QCHECK_CUDA(cudaMemcpy(f, e->p.ret_sum, ld * 4, cudaMemcpyDeviceToHost)); f += ld;
    QCHECK_CUDA(cudaMemcpy(f, e->p.rewardC, 8 * 4, cudaMemcpyDeviceToHost));
    QCHECK_CUDA(cudaMemcpy(env_u.data(), e->p.ep_index, ld * 4, cudaMemcpyDeviceToHost));
    QCHECK_CUDA(cudaMemcpy(env_u.data() + ld, e->p.ep_step, ld * 4, cudaMemcpyDeviceToHost));
    QCHECK_CUDA(cudaMemcpy(env_u.data() + 2 * ld, e->p.n_done, ld * 4, cudaMemcpyDeviceToHost));
    QCHECK_CUDA(cudaMemcpy(env_u.data() + 3 * ld, e->p.len_sum, ld * 4, cudaMemcpyDeviceToHost));
    std::ofstream os(path, std::ios::binary);
    if (!os) return fail(QSIM_EINVAL, "ac_save: cannot open %s", path);
    os.write((const char*)&h, sizeof(h));
    os.write((const char*)w.data(), w.size() * 4);
    os.write((const char*)env_f.data(), env_f.size() * 4);
    os.write((const char*)env_u.data(), env_u.size() * 4);
    if (!os) return fail(QSIM_EINVAL, "ac_save: write failed");
    return QSIM_OK;
}

extern "C" qsim_status ac_load(ac_handle* a, qsim_handle* e, const char* path) {
    if (!a || !e || !path) return fail(QSIM_EINVAL, "ac_load: null pointer");
    std::ifstream is(path, std::ios::binary);
    if (!is) return fail(QSIM_EINVAL, "ac_load: cannot open %s", path);
    CkptHeader h;
    is.read((char*)&h, sizeof(h));
    if (!is || memcmp(h.magic, "QSIMCKP1", 8) != 0) return fail(QSIM_EVERSION, "ac_load: not a checkpoint");
    if (h.abi != QSIM_ABI_VERSION || h.obs_dim != a->obs_dim || h.critic_in != a->critic_in ||
        h.hidden != a->hidden || h.n_actor != a->n_actor || h.n_critic != a->n_critic ||
        h.n_env != e->n || h.ld != e->ld)
        return fail(QSIM_EVERSION, "ac_load: checkpoint layout does not match the handles");
    const size_t nparam = 4 * (size_t)a->n_actor + 8 * (size_t)a->n_critic;
    const size_t ld = e->ld;
    std::vector<float> w(nparam), env_f((NS + 8 + 6 + 4 * HMAX + 2) * ld + 8);
    std::vector<uint32_t> env_u(4 * ld);
    is.read((char*)w.data(), w.size() * 4);
    is.read((char*)env_f.data(), env_f.size() * 4);
    is.read((char*)env_u.data(), env_u.size() * 4);
    if (!is) return fail(QSIM_EVERSION, "ac_load: truncated checkpoint");
    QCHECK_CUDA(cudaDeviceSynchronize());
    QCHECK_CUDA(cudaMemcpy(a->base, w.data(), nparam * 4, cudaMemcpyHostToDevice));
    const float* f = env_f.data();
    QCHECK_CUDA(cudaMemcpy(e->p.state, f, NS * ld * 4, cudaMemcpyHostToDevice)); f += NS * ld;
    QCHECK_CUDA(cudaMemcpy(e->p.prm, f, 8 * ld * 4, cudaMemcpyHostToDevice)); f += 8 * ld;
    QCHECK_CUDA(cudaMemcpy(e->p.dist, f, 6 * ld * 4, cudaMemcpyHostToDevice)); f += 6 * ld;
    QCHECK_CUDA(cudaMemcpy(e->p.hist, f, 4 * HMAX * ld * 4, cudaMemcpyHostToDevice)); f += 4 * HMAX * ld;
    QCHECK_CUDA(cudaMemcpy(e->p.ep_ret, f, ld * 4, cudaMemcpyHostToDevice)); f += ld;
    QCHECK_CUDA(cudaMemcpy(e->p.ret_sum, f, ld * 4, cudaMemcpyHostToDevice)); f += ld;
    QCHECK_CUDA(cudaMemcpy(e->p.rewardC, f, 8 * 4, cudaMemcpyHostToDevice));
    QCHECK_CUDA(cudaMemcpy(e->p.ep_index, env_u.data(), ld * 4, cudaMemcpyHostToDevice));
    QCHECK_CUDA(cudaMemcpy(e->p.ep_step, env_u.data() + ld, ld * 4, cudaMemcpyHostToDevice));
    QCHECK_CUDA(cudaMemcpy(e->p.n_done, env_u.data() + 2 * ld, ld * 4, cudaMemcpyHostToDevice));
    QCHECK_CUDA(cudaMemcpy(e->p.len_sum, env_u.data() + 3 * ld, ld * 4, cudaMemcpyHostToDevice));
    a->t_actor = h.t_actor; a->t_critic = h.t_critic; a->updates = h.updates;
    e->t_now = h.t_now; e->head = h.head; e->size = h.size; e->next_curriculum = h.next_curr;
    return QSIM_OK;
}
