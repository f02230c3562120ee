// qsim_env.cu -- env sets: create/reset, teacher-forced dynamics, single env step with
// external actions, observations, reward recalculation, statistics, Philox streams.
//
// Layouts are field-major [field][ld] (ld = env count padded to 32) so that one warp's
// access of one field is a single 128-byte transaction.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qsim_internal.h"
#include "qsim_recalc.cuh"

namespace qsim {

static thread_local std::string g_err;

qsim_status fail(qsim_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

qsim_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? QSIM_ENOMEM : QSIM_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

Vehicle make_vehicle(const qsim_params& v) {
    Vehicle V;
    for (int i = 0; i < 4; ++i) {
        V.rx[i] = v.rotor_pos[i][0];
        V.ry[i] = v.rotor_pos[i][1];
        V.dir[i] = v.rotor_dir[i];
    }
    V.rpm_min = v.rpm_min;
    V.rpm_max = v.rpm_max;
    V.g = v.g;
    return V;
}

static int critic_obs_dim(const qsim_config& c) {
    const int da = 18 + 4 * c.n_hist;
    if (c.critic_layout == QSIM_CRITIC_PAPER28) return 28;
    if (c.critic_layout == QSIM_CRITIC_PRIV) return da + 4 + NPRIV;
    if (c.critic_layout == QSIM_CRITIC_ACTOR) return da;
    return da + 4;
}

EnvCfg make_env_cfg(const qsim_config& c, const qsim_params& v, int n, int ld) {
    EnvCfg C;
    memset(&C, 0, sizeof(C));
    C.veh = make_vehicle(v);
    C.wait_limit = DEFAULT_WAIT_LIMIT;
    C.dt = c.dt;
    C.renorm = c.renorm_q;
    C.m0 = v.mass; C.Jx0 = v.J[0]; C.Jy0 = v.J[1]; C.Jz0 = v.J[2];
    C.kf0 = v.kf; C.km0 = v.km; C.tm0 = v.motor_tau;
    C.init_p = c.init_p; C.init_att = c.init_att; C.init_v = c.init_v; C.init_w = c.init_w;
    C.init_rpm_lo = c.init_rpm_lo; C.init_rpm_hi = c.init_rpm_hi;
    C.dr_mass = c.dr_mass; C.dr_J = c.dr_J; C.dr_kf = c.dr_kf; C.tm_lo = c.tm_lo; C.tm_hi = c.tm_hi;
    C.dist_f = c.dist_f; C.dist_tau = c.dist_tau;
    C.sig[0] = c.sig_p; C.sig[1] = c.sig_R; C.sig[2] = c.sig_v; C.sig[3] = c.sig_w;
    C.any_noise = (c.sig_p != 0.0f || c.sig_R != 0.0f || c.sig_v != 0.0f || c.sig_w != 0.0f);
    C.term_pos = c.term_pos;
    C.n_hist = c.n_hist;
    C.episode_len = c.episode_len;
    C.critic_layout = c.critic_layout;
    C.learning_starts = c.learning_starts;
    C.obs_dim = 18 + 4 * c.n_hist;
    C.cobs_dim = critic_obs_dim(c);
    C.n_priv = (c.critic_layout == QSIM_CRITIC_PRIV || c.critic_layout == QSIM_CRITIC_PAPER28) ? NPRIV : 0;
    C.no_lag = c.motor_lag_off ? 1 : 0;
    C.F = 23 + C.n_priv;
    C.key0 = (uint32_t)(c.seed & 0xffffffffu);
    C.key1 = (uint32_t)(c.seed >> 32);
    C.run_id = c.run_id;
    C.n = n;
    C.ld = ld;
    return C;
}

// ------------------------------------------------------------------------------ kernels
__global__ void k_philox_fill(uint32_t k0, uint32_t k1, uint32_t run, uint32_t tag, uint32_t sub,
                              uint32_t c1, int n, int kind, uint32_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox((uint32_t)i, c1, (tag << 24) | sub, run, k0, k1);
    uint4 o = r;
    if (kind == 1) {
        o = make_uint4(__float_as_uint(u01(r.x)), __float_as_uint(u01(r.y)),
                       __float_as_uint(u01(r.z)), __float_as_uint(u01(r.w)));
    } else if (kind == 2) {
        o = make_uint4(__float_as_uint(gauss(r.x, r.y)), __float_as_uint(gauss(r.z, r.w)), 0u, 0u);
    }
    reinterpret_cast<uint4*>(out)[i] = o;
}

__device__ __forceinline__ Prm load_prm(const float* prm, int ld, int e) {
    return make_prm(prm[e], prm[ld + e], prm[2 * ld + e], prm[3 * ld + e], prm[4 * ld + e],
                    prm[5 * ld + e], prm[6 * ld + e]);
}

__global__ void k_dynamics_step(Vehicle V, const float* __restrict__ prm,
                                const float* __restrict__ dist, const float* __restrict__ s_in,
                                const float* __restrict__ rpm, float dt, int renorm, int n, int ld,
                                int n_steps, float* __restrict__ s_out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float s[NS], u[4], d[6];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = s_in[i * ld + e];
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = rpm[i * ld + e];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = dist ? dist[i * ld + e] : 0.0f;
    const Prm P = load_prm(prm, ld, e);
    for (int t = 0; t < n_steps; ++t) rk4(V, dt, renorm, s, u, P, d);
#pragma unroll
    for (int i = 0; i < NS; ++i) s_out[i * ld + e] = s[i];
}

// Dynamics-only benchmark: env e starts near hover with a small env-dependent offset and
// integrates n_steps RK4 steps at the hover set-point, state in registers throughout.
__global__ void __launch_bounds__(128) k_dynamics_bench(Vehicle V, Prm P, float u_h, float dt,
                                                        int n, int ld, int n_steps,
                                                        float* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float s[NS];
    const float off = 1e-3f * (float)(e & 1023) / 1024.0f;
    s[0] = off; s[1] = -off; s[2] = 0.5f * off;
    s[3] = 1.0f; s[4] = 0.0f; s[5] = 0.0f; s[6] = 0.0f;
    s[7] = 0.0f; s[8] = 0.0f; s[9] = 0.0f;
    s[10] = off; s[11] = 0.0f; s[12] = -off;
#pragma unroll
    for (int i = 0; i < 4; ++i) s[13 + i] = u_h * (1.0f + off);
    const float u[4] = {u_h, u_h, u_h, u_h};
    const float d[6] = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < n_steps; ++t) rk4(V, dt, 1, s, u, P, d);
#pragma unroll
    for (int i = 0; i < NS; ++i) out[i * ld + e] = s[i];
}

__global__ void k_reset_all(EnvCfg C, EnvPtrs p) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int ld = C.ld;
    if (e >= ld) return;
    float s[NS], prm[7], d[6];
    reset_env(C, (uint32_t)e, 0u, s, prm, d);
#pragma unroll
    for (int i = 0; i < NS; ++i) p.state[i * ld + e] = s[i];
#pragma unroll
    for (int i = 0; i < 7; ++i) p.prm[i * ld + e] = prm[i];
    p.prm[7 * ld + e] = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) p.dist[i * ld + e] = d[i];
    for (int i = 0; i < 4 * HMAX; ++i) p.hist[i * ld + e] = 0.0f;
    p.ep_index[e] = 0; p.ep_step[e] = 0; p.ep_ret[e] = 0.0f;
    p.n_done[e] = 0; p.len_sum[e] = 0; p.ret_sum[e] = 0.0f;
}

// Critic observation of state s with history hist (4*n_hist, newest first) and priv.
__device__ __forceinline__ void write_critic_obs(const EnvCfg& C, const float* s, const float* pv,
                                                 const float* __restrict__ hist, int hist_ld,
                                                 float* out, int out_ld) {
    float o[18];
    obs_state(s, o);
    if (C.critic_layout == 2) {
        for (int k = 0; k < 18; ++k) out[k * out_ld] = o[k];
        for (int i = 0; i < 4; ++i) out[(18 + i) * out_ld] = rpm_norm(C.veh, s[13 + i]);
        for (int k = 0; k < 6; ++k) out[(22 + k) * out_ld] = pv[k];
        return;
    }
    for (int k = 0; k < 18; ++k) out[k * out_ld] = o[k];
    for (int k = 0; k < 4 * C.n_hist; ++k) out[(18 + k) * out_ld] = hist[k * hist_ld];
    const int da = C.obs_dim;
    for (int i = 0; i < 4; ++i) out[(da + i) * out_ld] = rpm_norm(C.veh, s[13 + i]);
    if (C.critic_layout == 1)
        for (int k = 0; k < NPRIV; ++k) out[(da + 4 + k) * out_ld] = pv[k];
}

__device__ __forceinline__ void write_actor_obs(const EnvCfg& C, const float* s, uint32_t env,
                                                uint32_t t, const float* __restrict__ hist,
                                                int hist_ld, float* out, int out_ld) {
    float o[18];
    obs_state(s, o);
    if (C.any_noise) {
        float nz[18];
        obs_noise(C, env, t, nz);
#pragma unroll
        for (int k = 0; k < 18; ++k) o[k] += nz[k];
    }
    for (int k = 0; k < 18; ++k) out[k * out_ld] = o[k];
    for (int k = 0; k < 4 * C.n_hist; ++k) out[(18 + k) * out_ld] = hist[k * hist_ld];
}

__global__ void k_observe(EnvCfg C, EnvPtrs p, uint32_t t, float* obs_a, float* obs_c) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int ld = C.ld;
    if (e >= C.n) return;
    float s[NS], d[6], pv[NPRIV];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = p.state[i * ld + e];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = p.dist[i * ld + e];
    const Prm P = load_prm(p.prm, ld, e);
    priv_vals(C, P, d, pv);
    if (obs_a) write_actor_obs(C, s, (uint32_t)e, t, p.hist + e, ld, obs_a + e, ld);
    if (obs_c) {
        if (C.critic_layout == 3) write_actor_obs(C, s, (uint32_t)e, t, p.hist + e, ld, obs_c + e, ld);
        else write_critic_obs(C, s, pv, p.hist + e, ld, obs_c + e, ld);
    }
}

// One env step with external actions (thread per env).
__global__ void k_step(EnvCfg C, EnvPtrs p, const float* __restrict__ actions, uint32_t t,
                       int64_t slot, int has_buffer, float* obs_a, float* obs_c, float* rew_out,
                       uint8_t* term_out, uint8_t* trunc_out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int ld = C.ld;
    if (e >= C.n) return;
    float s[NS], d[6], a[4], u[4], pv[NPRIV];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = p.state[i * ld + e];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = p.dist[i * ld + e];
    Prm P = load_prm(p.prm, ld, e);
    float Cr[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Cr[i] = p.rewardC[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = clampf(actions[i * ld + e], -1.0f, 1.0f);
    action_to_rpm(C.veh, a, u);
    float s2[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) s2[i] = s[i];
    motor_lag_off(C, u, s2);
    rk4(C.veh, C.dt, C.renorm, s2, u, P, d);
    const float r = reward(Cr, s2, a);
    const uint32_t ep_before = p.ep_step[e];
    const uint32_t ep_after = ep_before + 1;
    const bool term = terminated(C, s2);
    const bool trunc = !term && (int)ep_after >= C.episode_len;
    if (has_buffer && in_bounds(p.status, slot, p.rows, SITE_RING_WRITE) &&
        in_bounds(p.status, e, ld, SITE_SOA)) {
        float* rec = p.rec + (size_t)slot * C.F * ld;
#pragma unroll
        for (int i = 0; i < NS; ++i) rec[i * ld + e] = s[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) rec[(17 + i) * ld + e] = a[i];
        rec[21 * ld + e] = r;
        rec[22 * ld + e] = __uint_as_float(pack_flags(term, trunc, ep_before));
        if (C.n_priv) {
            priv_vals(C, P, d, pv);
            for (int k = 0; k < NPRIV; ++k) rec[(23 + k) * ld + e] = pv[k];
        }
        if (term || trunc) {
            float* sd = p.side + ((size_t)slot * ld + e) * NS;
#pragma unroll
            for (int i = 0; i < NS; ++i) sd[i] = s2[i];
        }
    }
    // history: newest first
    for (int i = C.n_hist - 1; i >= 1; --i)
        for (int c = 0; c < 4; ++c) p.hist[(4 * i + c) * ld + e] = p.hist[(4 * (i - 1) + c) * ld + e];
    if (C.n_hist > 0)
        for (int c = 0; c < 4; ++c) p.hist[c * ld + e] = a[c];
    float ret = p.ep_ret[e] + r;
    uint32_t ep_step = ep_after;
    if (term || trunc) {
        p.n_done[e] += 1;
        p.len_sum[e] += ep_after;
        p.ret_sum[e] += ret;
        const uint32_t epi = p.ep_index[e] + 1;
        p.ep_index[e] = epi;
        float prm7[7];
        reset_env(C, (uint32_t)e, epi, s2, prm7, d);
        for (int i = 0; i < 7; ++i) p.prm[i * ld + e] = prm7[i];
        for (int i = 0; i < 6; ++i) p.dist[i * ld + e] = d[i];
        for (int i = 0; i < 4 * HMAX; ++i) p.hist[i * ld + e] = 0.0f;
        P = make_prm(prm7[0], prm7[1], prm7[2], prm7[3], prm7[4], prm7[5], prm7[6]);
        ret = 0.0f;
        ep_step = 0;
    }
    p.ep_ret[e] = ret;
    p.ep_step[e] = ep_step;
#pragma unroll
    for (int i = 0; i < NS; ++i) p.state[i * ld + e] = s2[i];
    if (rew_out) rew_out[e] = r;
    if (term_out) term_out[e] = term ? 1 : 0;
    if (trunc_out) trunc_out[e] = trunc ? 1 : 0;
    priv_vals(C, P, d, pv);
    if (obs_a) write_actor_obs(C, s2, (uint32_t)e, t + 1, p.hist + e, ld, obs_a + e, ld);
    if (obs_c) {
        if (C.critic_layout == 3) write_actor_obs(C, s2, (uint32_t)e, t + 1, p.hist + e, ld, obs_c + e, ld);
        else write_critic_obs(C, s2, pv, p.hist + e, ld, obs_c + e, ld);
    }
}

// Reward recalculation over every stored record (HBM streaming: reads s', a, flags,
// writes r), four envs of one slot per thread (recalc_range).
__global__ void __launch_bounds__(256) k_recalc(EnvCfg C, EnvPtrs p, int64_t head, int64_t size,
                                                int64_t capacity) {
    float Cr[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Cr[i] = p.rewardC[i];
    recalc_range(C, p, Cr, head, size, capacity, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (uint64_t)gridDim.x * blockDim.x);
}

// The same over several env sets in one launch: blockIdx.y selects the set.
struct RecalcJob {
    EnvCfg C;
    EnvPtrs p;
    int64_t head, size, capacity;
};

__global__ void __launch_bounds__(256) k_recalc_batch(const RecalcJob* __restrict__ jobs) {
    const RecalcJob& J = jobs[blockIdx.y];
    float Cr[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Cr[i] = J.p.rewardC[i];
    recalc_range(J.C, J.p, Cr, J.head, J.size, J.capacity, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (uint64_t)gridDim.x * blockDim.x);
}

__global__ void k_set_reward(float* rewardC, float c0, float c1, float c2, float c3, float c4,
                             float c5, float c6, float sigma) {
    rewardC[0] = c0; rewardC[1] = c1; rewardC[2] = c2; rewardC[3] = c3;
    rewardC[4] = c4; rewardC[5] = c5; rewardC[6] = c6; rewardC[7] = sigma;
}

// 16 independent FMA chains per thread: issue-bound on the FP32 pipe.
__global__ void __launch_bounds__(256) k_ffma_probe(int iters, float* out) {
    float a[16];
    const float x = 1.0f + 1e-7f * (float)threadIdx.x, y = 0.999999f;
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = (float)(i + blockIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < 16; ++i) a[i] = fmaf(a[i], y, x);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += a[i];
    if (s == 12345.678f) out[0] = s;  // keeps the chains live
}

// Same with paired FMAs: 16 independent f32x2 chains (32 FMAs per 16 instructions).
__global__ void __launch_bounds__(256) k_ffma2_probe(int iters, float* out) {
    unsigned long long a[16];
    const unsigned long long x = f2pack(1.0f + 1e-7f * (float)threadIdx.x, 1.0f),
                             y = f2pack(0.999999f, 0.999999f);
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = f2pack((float)(i + blockIdx.x), (float)i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < 16; ++i) a[i] = f2fma(a[i], y, x);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float lo, hi;
        f2unpack(a[i], lo, hi);
        s += lo + hi;
    }
    if (s == 12345.678f) out[0] = s;
}

static int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

}  // namespace qsim

using namespace qsim;

// ------------------------------------------------------------------------------- ABI
extern "C" const char* qsim_last_error(void) { return g_err.c_str(); }
extern "C" int32_t qsim_abi_version(void) { return QSIM_ABI_VERSION; }

extern "C" qsim_status qsim_memcpy(void* dst, const void* src, size_t bytes, void* stream) {
    if (!dst || !src) return fail(QSIM_EINVAL, "qsim_memcpy: null pointer");
    QCHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, (cudaStream_t)stream));
    return QSIM_OK;
}

extern "C" qsim_status qsim_stream_sync(void* stream) {
    QCHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return QSIM_OK;
}

extern "C" void qsim_philox_host(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

extern "C" qsim_status qsim_philox_fill(uint64_t seed, uint32_t run, uint32_t tag, uint32_t sub,
                                        uint32_t c1, int32_t n, int32_t kind, uint32_t* out,
                                        void* stream) {
    if (!out || n < 0 || kind < 0 || kind > 2 || !aligned16(out))
        return fail(QSIM_EINVAL, "qsim_philox_fill: bad argument");
    if (n == 0) return QSIM_OK;
    k_philox_fill<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), run, tag, sub, c1, n, kind, out);
    QCHECK_LAUNCH("k_philox_fill");
    return QSIM_OK;
}

extern "C" qsim_status qsim_dynamics_step(const qsim_params* veh, const float* params,
                                          const float* dist, const float* state_in,
                                          const float* rpm, float dt, int32_t renorm, int32_t n,
                                          int32_t ld, int32_t n_steps, float* state_out,
                                          void* stream) {
    if (!veh || !params || !state_in || !rpm || !state_out)
        return fail(QSIM_EINVAL, "qsim_dynamics_step: null pointer");
    if (n < 0 || ld < n || (ld & 3) || n_steps < 0 || !(dt > 0.0f))
        return fail(QSIM_EINVAL, "qsim_dynamics_step: bad size (n=%d ld=%d steps=%d)", n, ld,
                    n_steps);
    if (!aligned16(params) || !aligned16(state_in) || !aligned16(rpm) || !aligned16(state_out) ||
        (dist && !aligned16(dist)))
        return fail(QSIM_EINVAL, "qsim_dynamics_step: pointers must be 16-byte aligned");
    if (n == 0) return QSIM_OK;
    k_dynamics_step<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(
        make_vehicle(*veh), params, dist, state_in, rpm, dt, renorm, n, ld, n_steps, state_out);
    QCHECK_LAUNCH("k_dynamics_step");
    return QSIM_OK;
}

extern "C" qsim_status qsim_dynamics_bench(const qsim_params* veh, int32_t n, int32_t ld,
                                           int32_t n_steps, float dt, float* state_out,
                                           void* stream) {
    if (!veh || !state_out || n <= 0 || ld < n || n_steps < 0)
        return fail(QSIM_EINVAL, "qsim_dynamics_bench: bad argument");
    Prm P;
    P.m = veh->mass; P.Jx = veh->J[0]; P.Jy = veh->J[1]; P.Jz = veh->J[2]; P.kf = veh->kf;
    P.km = veh->km; P.tm = veh->motor_tau;
    P.im = 1.0f / P.m; P.iJx = 1.0f / P.Jx; P.iJy = 1.0f / P.Jy; P.iJz = 1.0f / P.Jz;
    P.itm = 1.0f / P.tm;
    const float u_h = sqrtf(veh->mass * veh->g / (4.0f * veh->kf));
    // blocks of 128 threads, halved (to 32) while they would not cover every SM: the paper's
    // shape (8,192 envs) then runs on all SMs instead of 64
    int sms = 152, bs = 128, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    while (bs > 32 && grid_for(n, bs) < sms) bs >>= 1;
    k_dynamics_bench<<<grid_for(n, bs), bs, 0, (cudaStream_t)stream>>>(
        make_vehicle(*veh), P, u_h, dt, n, ld, n_steps, state_out);
    QCHECK_LAUNCH("k_dynamics_bench");
    return QSIM_OK;
}

static qsim_status validate_cfg(const qsim_config* c, const qsim_params* v) {
    if (!c || !v) return fail(QSIM_EINVAL, "qsim_create: null config");
    if (c->n_envs < 1 || c->n_envs > (1 << 26))
        return fail(QSIM_EINVAL, "qsim_create: n_envs=%d out of range", c->n_envs);
    if (c->n_hist < 0 || c->n_hist > HMAX)
        return fail(QSIM_EINVAL, "qsim_create: n_hist=%d not in 0..16", c->n_hist);
    if (c->episode_len < 1) return fail(QSIM_EINVAL, "qsim_create: episode_len < 1");
    if (c->critic_layout < 0 || c->critic_layout > 3)
        return fail(QSIM_EINVAL, "qsim_create: bad critic_layout");
    if (c->replay_capacity < 0 || (c->replay_capacity > 0 && c->replay_capacity < 2))
        return fail(QSIM_EINVAL, "qsim_create: replay_capacity must be 0 or >= 2");
    if (!(c->dt > 0.0f)) return fail(QSIM_EINVAL, "qsim_create: dt must be > 0");
    if (!(v->mass > 0.0f) || !(v->J[0] > 0.0f) || !(v->J[1] > 0.0f) || !(v->J[2] > 0.0f) ||
        !(v->motor_tau > 0.0f) || !(v->kf > 0.0f) || !(v->rpm_max > v->rpm_min))
        return fail(QSIM_EINVAL, "qsim_create: non-physical vehicle parameters");
    if (!(c->tm_lo > 0.0f) || c->tm_hi < c->tm_lo)
        return fail(QSIM_EINVAL, "qsim_create: bad motor time-constant range");
    if (c->dr_mass < 0 || c->dr_mass >= 1 || c->dr_J < 0 || c->dr_J >= 1 || c->dr_kf < 0 ||
        c->dr_kf >= 1)
        return fail(QSIM_EINVAL, "qsim_create: randomisation widths must be in [0,1)");
    return QSIM_OK;
}

extern "C" qsim_status qsim_create(const qsim_config* cfg, const qsim_params* veh,
                                   qsim_handle** out) {
    if (!out) return fail(QSIM_EINVAL, "qsim_create: null out");
    *out = nullptr;
    qsim_status st = validate_cfg(cfg, veh);
    if (st != QSIM_OK) return st;
    qsim_handle* h = new qsim_handle();
    memset(&h->p, 0, sizeof(h->p));
    h->cfg = *cfg;
    h->veh = *veh;
    h->n = cfg->n_envs;
    h->ld = (cfg->n_envs + 31) & ~31;
    h->dc = make_env_cfg(*cfg, *veh, h->n, h->ld);
    h->capacity = cfg->replay_capacity;
    h->p.rows = h->capacity;
    h->t_now = h->head = h->size = 0;
    h->next_curriculum = cfg->curriculum_interval > 0 ? cfg->curriculum_interval : -1;
    h->rollout_warps = 0;
    h->rollout_parts = 0;
    h->rollout_chunk = 0;
    h->rollout_packed = -1;
    h->streams_ready = false;
    h->tc_sched = nullptr;
    cudaGetDevice(&h->device);
    const size_t ld = (size_t)h->ld;
    auto alloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        return cudaMemset(*p, 0, bytes) == cudaSuccess;
    };
    bool ok = alloc((void**)&h->p.state, NS * ld * 4) && alloc((void**)&h->p.prm, 8 * ld * 4) &&
              alloc((void**)&h->p.dist, 6 * ld * 4) && alloc((void**)&h->p.hist, 4 * HMAX * ld * 4) &&
              alloc((void**)&h->p.ep_ret, ld * 4) && alloc((void**)&h->p.ret_sum, ld * 4) &&
              alloc((void**)&h->p.ep_index, ld * 4) && alloc((void**)&h->p.ep_step, ld * 4) &&
              alloc((void**)&h->p.n_done, ld * 4) && alloc((void**)&h->p.len_sum, ld * 4) &&
              alloc((void**)&h->p.rewardC, 8 * 4) &&
              alloc((void**)&h->p.status, STATUS_WORDS * 4);
    if (ok && h->capacity > 0) {
        ok = alloc((void**)&h->p.rec, (size_t)h->capacity * h->dc.F * ld * 4) &&
             alloc((void**)&h->p.side, (size_t)h->capacity * NS * ld * 4);
    }
    if (!ok) {
        cudaGetLastError();
        qsim_destroy(h);
        return fail(QSIM_ENOMEM, "qsim_create: device allocation failed (%d envs, %lld slots)",
                    h->n, (long long)h->capacity);
    }
    k_set_reward<<<1, 1>>>(h->p.rewardC, cfg->reward[0], cfg->reward[1], cfg->reward[2],
                           cfg->reward[3], cfg->reward[4], cfg->reward[5], cfg->reward[6],
                           cfg->sigma_e);
    k_reset_all<<<grid_for(h->ld, 128), 128>>>(h->dc, h->p);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        qsim_destroy(h);
        return cuda_fail(e, "qsim_create: reset");
    }
    *out = h;
    return QSIM_OK;
}

extern "C" qsim_status qsim_destroy(qsim_handle* h) {
    if (!h) return QSIM_OK;
    void* ptrs[] = {h->p.state, h->p.prm, h->p.dist, h->p.hist, h->p.ep_ret, h->p.ret_sum,
                    h->p.ep_index, h->p.ep_step, h->p.n_done, h->p.len_sum, h->p.rec,
                    h->p.side, h->p.rewardC, h->p.status, h->tc_sched};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->streams_ready) {
        for (int i = 0; i < 4; ++i) {
            cudaStreamDestroy(h->part_stream[i]);
            cudaEventDestroy(h->ev_join[i]);
        }
        cudaEventDestroy(h->ev_fork);
    }
    delete h;
    return QSIM_OK;
}

extern "C" qsim_status qsim_info_get(const qsim_handle* h, qsim_info* o) {
    if (!h || !o) return fail(QSIM_EINVAL, "qsim_info_get: null pointer");
    o->n_envs = h->n; o->ld = h->ld;
    o->obs_dim = h->dc.obs_dim; o->critic_obs_dim = h->dc.cobs_dim;
    o->record_fields = h->dc.F; o->n_priv = h->dc.n_priv;
    o->capacity = h->capacity; o->t_now = h->t_now; o->head = h->head; o->size = h->size;
    o->state = h->p.state; o->params = h->p.prm; o->dist = h->p.dist; o->hist = h->p.hist;
    o->ep_index = h->p.ep_index; o->ep_step = h->p.ep_step; o->ep_ret = h->p.ep_ret;
    o->n_done = h->p.n_done; o->len_sum = h->p.len_sum; o->ret_sum = h->p.ret_sum;
    o->records = h->p.rec; o->side = h->p.side; o->reward_c = h->p.rewardC;
    return QSIM_OK;
}

extern "C" qsim_status qsim_set_counters(qsim_handle* h, int64_t t_now, int64_t head,
                                         int64_t size) {
    if (!h) return fail(QSIM_EINVAL, "qsim_set_counters: null handle");
    if (t_now < 0 || size < 0 || size > h->capacity || head < 0 ||
        (h->capacity > 0 && head >= h->capacity) || (t_now >> 32) != 0)
        return fail(QSIM_EINVAL, "qsim_set_counters: counters out of range");
    h->t_now = t_now; h->head = head; h->size = size;
    return QSIM_OK;
}

// Reads the flag word of (slot, env) through the debug bounds check (a one-thread probe of
// the status path: out-of-range indices reach it only in the checked build).
__global__ void k_bounds_probe(EnvCfg C, EnvPtrs p, int64_t slot, int64_t env, uint32_t* out) {
    if (in_bounds(p.status, slot, p.rows, SITE_PROBE) && in_bounds(p.status, env, C.ld, SITE_SOA))
        *out = __float_as_uint(p.rec[((size_t)slot * C.F + 22) * (size_t)C.ld + (size_t)env]);
}

extern "C" int32_t qsim_bounds_checked(void) { return QSIM_BOUNDS_CHECK ? 1 : 0; }

extern "C" qsim_status qsim_bounds_probe(qsim_handle* h, int64_t slot, int64_t env, uint32_t* flags_out,
                                         void* stream) {
    if (!h || !flags_out) return fail(QSIM_EINVAL, "qsim_bounds_probe: null argument");
    if (h->capacity == 0) return fail(QSIM_ESTATE, "qsim_bounds_probe: env set has no replay buffer");
    const bool inside = slot >= 0 && slot < h->capacity && env >= 0 && env < h->dc.ld;
    if (!QSIM_BOUNDS_CHECK && !inside)
        return fail(QSIM_EINVAL, "qsim_bounds_probe: (%lld, %lld) outside the ring (library built "
                                 "without bounds checks)", (long long)slot, (long long)env);
    k_bounds_probe<<<1, 1, 0, (cudaStream_t)stream>>>(h->dc, h->p, slot, env, flags_out);
    QCHECK_CUDA(cudaGetLastError());
    return QSIM_OK;
}

extern "C" int32_t qsim_set_wait_limit(qsim_handle* h, int32_t polls) {
    if (!h) return fail(QSIM_EINVAL, "qsim_set_wait_limit: null handle");
    if (polls < 0 || polls > (1 << 30)) return fail(QSIM_EINVAL, "qsim_set_wait_limit: %d polls", polls);
    const int32_t prev = h->dc.wait_limit;
    h->dc.wait_limit = polls == 0 ? DEFAULT_WAIT_LIMIT : polls;
    return prev;
}

extern "C" qsim_status qsim_sync(qsim_handle* h) {
    if (!h) return fail(QSIM_EINVAL, "qsim_sync: null handle");
    int st[STATUS_WORDS] = {};
    QCHECK_CUDA(cudaMemcpy(st, h->p.status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st[0] != DEV_OK) {
        cudaMemset(h->p.status, 0, sizeof(st));
        if (st[0] == DEV_TIMEOUT) return fail(QSIM_ETIMEOUT, "device-side wait ran out");
        if (st[0] == DEV_RANGE)
            return fail(QSIM_ESTATE, "tensor-core rollout: an actor weight, input or hidden activation "
                                     "was outside the half-precision range (|x| >= 65504) or not finite");
        if (st[0] == DEV_BOUNDS) {
            static const char* const sites[] = {"index", "replay-ring write slot", "replay-ring read slot",
                                                "SoA env index", "probe slot"};
            const int site = st[1] >= 1 && st[1] <= 4 ? st[1] : 0;
            const long long idx = (long long)(((uint64_t)(uint32_t)st[3] << 32) | (uint32_t)st[2]);
            const long long lim = (long long)(((uint64_t)(uint32_t)st[5] << 32) | (uint32_t)st[4]);
            return fail(QSIM_ESTATE, "bounds check: %s %lld outside [0, %lld)", sites[site], idx, lim);
        }
        return fail(QSIM_ESTATE, "device reported status %d", st[0]);
    }
    return QSIM_OK;
}

extern "C" qsim_status qsim_observe(qsim_handle* h, float* obs_a, float* obs_c, void* stream) {
    if (!h) return fail(QSIM_EINVAL, "qsim_observe: null handle");
    k_observe<<<grid_for(h->n, 128), 128, 0, (cudaStream_t)stream>>>(h->dc, h->p,
                                                                       (uint32_t)h->t_now, obs_a, obs_c);
    QCHECK_LAUNCH("k_observe");
    return QSIM_OK;
}

extern "C" qsim_status qsim_step(qsim_handle* h, const float* actions, float* obs_a, float* obs_c,
                                 float* reward, uint8_t* terminated, uint8_t* truncated,
                                 void* stream) {
    if (!h || !actions) return fail(QSIM_EINVAL, "qsim_step: null pointer");
    if ((h->t_now + 1) >> 32) return fail(QSIM_ESTATE, "qsim_step: step counter exhausted");
    const int has_buf = h->capacity > 0;
    k_step<<<grid_for(h->n, 128), 128, 0, (cudaStream_t)stream>>>(
        h->dc, h->p, actions, (uint32_t)h->t_now, has_buf ? h->head : 0, has_buf, obs_a, obs_c,
        reward, terminated, truncated);
    QCHECK_LAUNCH("k_step");
    h->t_now += 1;
    if (has_buf) {
        h->head = (h->head + 1) % h->capacity;
        if (h->size < h->capacity) h->size += 1;
    }
    return QSIM_OK;
}

extern "C" qsim_status qsim_recalc_rewards(qsim_handle* h, void* stream) {
    if (!h) return fail(QSIM_EINVAL, "qsim_recalc_rewards: null handle");
    if (h->capacity == 0 || h->size == 0) return QSIM_OK;
    const int64_t total = h->size * (int64_t)((h->n + 3) / 4);  // quads of four envs
    if (total >= (int64_t)1 << 32) return fail(QSIM_EINVAL, "qsim_recalc_rewards: ring too large");
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device);
    const int64_t want = (total + 255) / 256;
    const int grid = (int)(want < (int64_t)dev_sms * 16 ? want : (int64_t)dev_sms * 16);
    k_recalc<<<grid, 256, 0, (cudaStream_t)stream>>>(h->dc, h->p, h->head, h->size, h->capacity);
    QCHECK_LAUNCH("k_recalc");
    return QSIM_OK;
}

extern "C" qsim_status qsim_recalc_rewards_batch(qsim_handle* const* hs, int32_t n, void* stream) {
    if (!hs || n < 1 || n > 65535) return fail(QSIM_EINVAL, "qsim_recalc_rewards_batch: bad argument");
    int dev = -1;
    QCHECK_CUDA(cudaGetDevice(&dev));
    std::vector<RecalcJob> jobs;
    int64_t most = 0, total = 0;
    for (int i = 0; i < n; ++i) {
        const qsim_handle* h = hs[i];
        if (!h) return fail(QSIM_EINVAL, "qsim_recalc_rewards_batch: null handle %d", i);
        if (h->device != dev) return fail(QSIM_EINVAL, "qsim_recalc_rewards_batch: handle %d is on another device", i);
        if (h->capacity == 0 || h->size == 0) continue;
        const int64_t quads = h->size * (int64_t)((h->n + 3) / 4);
        if (quads >= (int64_t)1 << 32) return fail(QSIM_EINVAL, "qsim_recalc_rewards_batch: ring %d too large", i);
        jobs.push_back(RecalcJob{h->dc, h->p, h->head, h->size, h->capacity});
        most = std::max(most, quads);
        total += quads;
    }
    if (jobs.empty()) return QSIM_OK;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // blocks per set: its share of 16 blocks per SM, at least one, at most one per 256 quads
    const int64_t want = std::max<int64_t>(1, (int64_t)sms * 16 * most / std::max<int64_t>(total, 1));
    const int gx = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (most + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    RecalcJob* d_jobs = nullptr;
    QCHECK_CUDA(cudaMallocAsync((void**)&d_jobs, sizeof(RecalcJob) * jobs.size(), st));
    QCHECK_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(RecalcJob) * jobs.size(), cudaMemcpyHostToDevice, st));
    k_recalc_batch<<<dim3(gx, (unsigned)jobs.size()), 256, 0, st>>>(d_jobs);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d_jobs, st);
    if (e != cudaSuccess) return cuda_fail(e, "k_recalc_batch");
    return QSIM_OK;
}

extern "C" qsim_status qsim_set_reward(qsim_handle* h, const float c[7], float sigma_e,
                                       void* stream) {
    if (!h || !c) return fail(QSIM_EINVAL, "qsim_set_reward: null pointer");
    k_set_reward<<<1, 1, 0, (cudaStream_t)stream>>>(h->p.rewardC, c[0], c[1], c[2], c[3], c[4],
                                                    c[5], c[6], sigma_e);
    QCHECK_LAUNCH("k_set_reward");
    return QSIM_OK;
}

extern "C" qsim_status qsim_stats_get(qsim_handle* h, qsim_stats* out, void* stream) {
    if (!h || !out) return fail(QSIM_EINVAL, "qsim_stats_get: null pointer");
    std::vector<uint32_t> nd(h->n), ls(h->n);
    std::vector<float> rs(h->n);
    QCHECK_CUDA(cudaMemcpyAsync(nd.data(), h->p.n_done, 4 * (size_t)h->n, cudaMemcpyDeviceToHost,
                                (cudaStream_t)stream));
    QCHECK_CUDA(cudaMemcpyAsync(ls.data(), h->p.len_sum, 4 * (size_t)h->n, cudaMemcpyDeviceToHost,
                                (cudaStream_t)stream));
    QCHECK_CUDA(cudaMemcpyAsync(rs.data(), h->p.ret_sum, 4 * (size_t)h->n, cudaMemcpyDeviceToHost,
                                (cudaStream_t)stream));
    QCHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int64_t ep = 0;
    double len = 0.0, ret = 0.0;
    for (int i = 0; i < h->n; ++i) {
        ep += nd[i];
        len += ls[i];
        ret += rs[i];
    }
    out->episodes = ep;
    out->mean_length = ep ? len / (double)ep : 0.0;
    out->mean_return = ep ? ret / (double)ep : 0.0;
    return QSIM_OK;
}

extern "C" qsim_status qsim_ffma_probe(int32_t n_blocks, int32_t iters, float* out, void* stream) {
    if (n_blocks <= 0 || !out || iters == 0) return fail(QSIM_EINVAL, "qsim_ffma_probe: bad argument");
    if (iters < 0) k_ffma2_probe<<<n_blocks, 256, 0, (cudaStream_t)stream>>>(-iters, out);
    else k_ffma_probe<<<n_blocks, 256, 0, (cudaStream_t)stream>>>(iters, out);
    QCHECK_LAUNCH("k_ffma_probe");
    return QSIM_OK;
}
