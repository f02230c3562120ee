// qsim_device.cuh -- device-side building blocks of the quadrotor hot path (sm_103a).
//
// Single-precision implementations of: Philox4x32-10 (Salmon et al., SC'11), the
// uniform / Box-Muller conversions, the multirotor rigid-body derivative with first-order
// motor lag and its RK4 step (Sec. IV "Methodology"), the actor / critic observations
// (Sec. IV: o_a = {p, R, v, omega, H}, privileged critic), the reward (Sec. IV reward
// formula), termination and the domain-randomised reset.  Every kernel of the library
// builds on these; state lives in registers as float[17] with compile-time indices.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qsim {

constexpr int NS = 17;    // p(3) q(4: w,x,y,z) v(3) omega(3) omega_m(4)
constexpr int HMAX = 16;  // longest action history
constexpr int NPRIV = 6;

enum : uint32_t { TAG_RESET = 0, TAG_DR = 1, TAG_OBS = 2, TAG_EXPL = 3, TAG_REPLAY = 4,
                  TAG_SMOOTH = 5, TAG_DIST = 6, TAG_INIT = 7, TAG_WARM = 8 };

// Vehicle geometry and limits.
struct Vehicle {
    float rx[4], ry[4], dir[4];
    float rpm_min, rpm_max, g;
};

// Everything an env kernel needs, passed by value.
struct EnvCfg {
    Vehicle veh;
    float dt;
    int renorm;
    float m0, Jx0, Jy0, Jz0, kf0, km0, tm0;
    float init_p, init_att, init_v, init_w, init_rpm_lo, init_rpm_hi;
    float dr_mass, dr_J, dr_kf, tm_lo, tm_hi, dist_f, dist_tau;
    float sig[4];
    int any_noise;
    float term_pos;
    int n_hist, episode_len, critic_layout, learning_starts;
    int no_lag;  // motor model ablated: rotors at the set-point at once
    int obs_dim, cobs_dim, n_priv, F;  // F: floats per transition record
    uint32_t key0, key1, run_id;
    int wait_limit;  // polls of a bounded device-side wait before it gives up
    int n, ld;
};

constexpr int DEFAULT_WAIT_LIMIT = 1 << 22;

// Per-env parameters with the reciprocals the derivative needs.
struct Prm {
    float m, Jx, Jy, Jz, kf, km, tm;
    float im, iJx, iJy, iJz, itm;
};

__device__ __forceinline__ Prm make_prm(float m, float Jx, float Jy, float Jz, float kf, float km,
                                        float tm) {
    Prm p;
    p.m = m; p.Jx = Jx; p.Jy = Jy; p.Jz = Jz; p.kf = kf; p.km = km; p.tm = tm;
    p.im = 1.0f / m; p.iJx = 1.0f / Jx; p.iJy = 1.0f / Jy; p.iJz = 1.0f / Jz; p.itm = 1.0f / tm;
    return p;
}

// ------------------------------------------------------------------------------- Philox
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint4 draw(const EnvCfg& C, uint32_t c0, uint32_t c1, uint32_t tag,
                                      uint32_t sub) {
    return philox(c0, c1, (tag << 24) | sub, C.run_id, C.key0, C.key1);
}

// Same stream with the rounds kept as a loop: for cold paths (resets, observation noise)
// whose unrolled copies would only bloat the hot loop's instruction footprint.
__device__ __forceinline__ uint4 draw_rolled(const EnvCfg& C, uint32_t c0, uint32_t c1,
                                             uint32_t tag, uint32_t sub) {
    uint32_t x0 = c0, x1 = c1, x2 = (tag << 24) | sub, x3 = C.run_id, k0 = C.key0, k1 = C.key1;
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
        const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
        const uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(x0, x1, x2, x3);
}

// N blocks of the same stream with counters (c0, c1, c2[n], run), computed together round
// by round: the independent blocks interleave (instruction-level parallelism) in one
// rolled loop; each block equals draw_rolled's.
template <int N>
__device__ __forceinline__ void draw_rolled_n(const EnvCfg& C, uint32_t c0, uint32_t c1,
                                              const uint32_t (&c2)[N], uint4 (&out)[N]) {
    uint32_t x0[N], x1[N], x2[N], x3[N];
#pragma unroll
    for (int n = 0; n < N; ++n) { x0[n] = c0; x1[n] = c1; x2[n] = c2[n]; x3[n] = C.run_id; }
    uint32_t k0 = C.key0, k1 = C.key1;
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const uint32_t lo0 = 0xD2511F53u * x0[n], hi0 = __umulhi(0xD2511F53u, x0[n]);
            const uint32_t lo1 = 0xCD9E8D57u * x2[n], hi1 = __umulhi(0xCD9E8D57u, x2[n]);
            const uint32_t n0 = hi1 ^ x1[n] ^ k0, n2 = hi0 ^ x3[n] ^ k1;
            x0[n] = n0; x1[n] = lo1; x2[n] = n2; x3[n] = lo0;
        }
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
#pragma unroll
    for (int n = 0; n < N; ++n) out[n] = make_uint4(x0[n], x1[n], x2[n], x3[n]);
}

// ((x >> 9) + 1/2) * 2^-23: exact in float, strictly inside (0, 1).
__device__ __forceinline__ float u01(uint32_t x) {
    return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// Box-Muller, cosine branch.
__device__ __forceinline__ float gauss(uint32_t a, uint32_t b) {
    return sqrtf(-2.0f * logf(u01(a))) * cospif(2.0f * u01(b));
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) {
    return fminf(fmaxf(x, lo), hi);
}

__device__ __forceinline__ bool finitef(float x) {
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

__device__ __forceinline__ bool finite_state(const float* s) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < NS; ++i) ok &= finitef(s[i]);
    return ok;
}

// ----------------------------------------------------------------------------- dynamics
// Time derivative of the 17-vector at held, already clipped RPM set-point uc.
__device__ __forceinline__ void deriv(const Vehicle& V, const float* s, const float* uc,
                                      const Prm& P, const float* d, float* ds) {
    const float qw = s[3], qx = s[4], qy = s[5], qz = s[6];
    const float wx = s[10], wy = s[11], wz = s[12];
    float f[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = P.kf * s[13 + i] * s[13 + i];
    const float F = (f[0] + f[1]) + (f[2] + f[3]);
    float tx = d[3], ty = d[4], tz = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        tx = fmaf(V.ry[i], f[i], tx);
        ty = fmaf(-V.rx[i], f[i], ty);
        tz = fmaf(V.dir[i], f[i], tz);
    }
    tz = fmaf(P.km, tz, d[5]);
    // third column of R(q): body z axis in the world frame
    const float r02 = 2.0f * (qx * qz + qw * qy);
    const float r12 = 2.0f * (qy * qz - qw * qx);
    const float r22 = 1.0f - 2.0f * (qx * qx + qy * qy);
    ds[0] = s[7]; ds[1] = s[8]; ds[2] = s[9];
    ds[7] = fmaf(r02, F, d[0]) * P.im;
    ds[8] = fmaf(r12, F, d[1]) * P.im;
    ds[9] = fmaf(r22, F, d[2]) * P.im - V.g;
    ds[3] = 0.5f * (-qx * wx - qy * wy - qz * wz);
    ds[4] = 0.5f * (qw * wx + qy * wz - qz * wy);
    ds[5] = 0.5f * (qw * wy - qx * wz + qz * wx);
    ds[6] = 0.5f * (qw * wz + qx * wy - qy * wx);
    ds[10] = (tx - (P.Jz - P.Jy) * wy * wz) * P.iJx;
    ds[11] = (ty - (P.Jx - P.Jz) * wz * wx) * P.iJy;
    ds[12] = (tz - (P.Jy - P.Jx) * wx * wy) * P.iJz;
#pragma unroll
    for (int i = 0; i < 4; ++i) ds[13 + i] = (uc[i] - s[13 + i]) * P.itm;
}

// Classic RK4 over the 17-vector (in place), then optional quaternion renormalisation.
__device__ __forceinline__ void rk4(const Vehicle& V, float dt, int renorm, float* s,
                                    const float* u, const Prm& P, const float* d) {
    float uc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) uc[i] = clampf(u[i], V.rpm_min, V.rpm_max);
    float k[NS], acc[NS], y[NS];
    deriv(V, s, uc, P, d, k);
    const float h2 = 0.5f * dt;
#pragma unroll
    for (int i = 0; i < NS; ++i) { acc[i] = k[i]; y[i] = fmaf(h2, k[i], s[i]); }
    deriv(V, y, uc, P, d, k);
#pragma unroll
    for (int i = 0; i < NS; ++i) { acc[i] = fmaf(2.0f, k[i], acc[i]); y[i] = fmaf(h2, k[i], s[i]); }
    deriv(V, y, uc, P, d, k);
#pragma unroll
    for (int i = 0; i < NS; ++i) { acc[i] = fmaf(2.0f, k[i], acc[i]); y[i] = fmaf(dt, k[i], s[i]); }
    deriv(V, y, uc, P, d, k);
    const float h6 = dt * (1.0f / 6.0f);
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = fmaf(h6, acc[i] + k[i], s[i]);
    if (renorm) {
        const float inv = rsqrtf(s[3] * s[3] + s[4] * s[4] + s[5] * s[5] + s[6] * s[6]);
        s[3] *= inv; s[4] *= inv; s[5] *= inv; s[6] *= inv;
    }
}

// Motor-model ablation (Sec. VI, the study without rotor delay): the rotors run at the
// clipped set-point from the start of the step, so the lag term of the motor equation is
// zero in every RK4 stage.
__device__ __forceinline__ void motor_lag_off(const EnvCfg& C, const float* u, float* s) {
    if (C.no_lag) {
#pragma unroll
        for (int i = 0; i < 4; ++i) s[13 + i] = clampf(u[i], C.veh.rpm_min, C.veh.rpm_max);
    }
}

// Arguments of the trajectory-tracking instantiations of the env-step kernels.
struct TrackArgs {
    const float* period;  // [ld] cycle time T of each env's target, s
    float amp, z0;        // target amplitude A and height
    float clip_p, clip_v; // observation offsets clipped to +-clip per component
    double* sq_err;       // [2][ld] out: sums of |e|^2 and e_x^2 + e_y^2
    int32_t* steps_ok;    // [ld] out: steps completed before the flight ended
};

// Figure-eight target of Sec. V at step k: p* = (A cos th, (A/2) sin 2 th, z0) with
// th = 2 pi k dt / T, and its time derivative v*.  Per env the cycles per step dt / T
// (double) and the velocity scale A 2 pi / T are formed once; per step the cycle fraction
// k dt / T is one double product reduced to [0, 1) before the single-precision sin / cos,
// so the phase stays exact over long flights.
struct Target {
    double cyc;  // dt / T
    float aw;    // A 2 pi / T
};

__device__ __forceinline__ Target make_target(float dt, float T, float A) {
    return Target{(double)dt / (double)T, A * (6.283185307179586f / T)};
}

__device__ __forceinline__ void lissajous(int k, const Target& tg, float A, float z0, float* pr,
                                          float* vr) {
    const double x = (double)k * tg.cyc;
    const float f1 = (float)(x - floor(x));
    const float f2 = (float)(2.0 * x - floor(2.0 * x));
    float s1, c1, s2, c2;
    sincospif(2.0f * f1, &s1, &c1);
    sincospif(2.0f * f2, &s2, &c2);
    pr[0] = A * c1;
    pr[1] = 0.5f * A * s2;
    pr[2] = z0;
    vr[0] = -tg.aw * s1;
    vr[1] = tg.aw * c2;
    vr[2] = 0.0f;
}

// Rotation matrix of q, row-major.
__device__ __forceinline__ void rotmat(const float* q, float* R) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0f - 2.0f * (y * y + z * z); R[1] = 2.0f * (x * y - w * z); R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z); R[4] = 1.0f - 2.0f * (x * x + z * z); R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y); R[7] = 2.0f * (y * z + w * x); R[8] = 1.0f - 2.0f * (x * x + y * y);
}

// The 18 state entries of the actor observation: p, R row-major, v, omega.
__device__ __forceinline__ void obs_state(const float* s, float* o) {
    o[0] = s[0]; o[1] = s[1]; o[2] = s[2];
    rotmat(s + 3, o + 3);
    o[12] = s[7]; o[13] = s[8]; o[14] = s[9];
    o[15] = s[10]; o[16] = s[11]; o[17] = s[12];
}

// Observation noise of env `env` at global step t: 18 normals, two per Philox block.
// Observation noise components 2b and 2b + 1 (b < 9) of env `env` at step t: one Philox
// block, two Box-Muller normals scaled by their component's sigma.
__device__ __forceinline__ void obs_noise_pair(const EnvCfg& C, uint32_t env, uint32_t t, int b, float& n0,
                                               float& n1) {
    const uint4 r = draw_rolled(C, env, t, TAG_OBS, (uint32_t)b);
    const int k = 2 * b;
    const float s0 = k < 3 ? C.sig[0] : (k < 12 ? C.sig[1] : (k < 15 ? C.sig[2] : C.sig[3]));
    const float s1 = (k + 1) < 3 ? C.sig[0]
                     : ((k + 1) < 12 ? C.sig[1] : ((k + 1) < 15 ? C.sig[2] : C.sig[3]));
    n0 = s0 * gauss(r.x, r.y);
    n1 = s1 * gauss(r.z, r.w);
}

__device__ __forceinline__ void obs_noise(const EnvCfg& C, uint32_t env, uint32_t t, float* nz) {
#pragma unroll 1
    for (int b = 0; b < 9; ++b) obs_noise_pair(C, env, t, b, nz[2 * b], nz[2 * b + 1]);
}

__device__ __forceinline__ float rpm_norm(const Vehicle& V, float w) {
    return 2.0f * (w - V.rpm_min) / (V.rpm_max - V.rpm_min) - 1.0f;
}

// Privileged extras of the critic: true parameters relative to nominal, or scaled
// disturbances for the 28-D layout.
__device__ __forceinline__ void priv_vals(const EnvCfg& C, const Prm& P, const float* d,
                                          float* pv) {
    if (C.critic_layout == 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) pv[k] = C.dist_f > 0.0f ? d[k] / C.dist_f : 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) pv[3 + k] = C.dist_tau > 0.0f ? d[3 + k] / C.dist_tau : 0.0f;
    } else {
        pv[0] = P.m / C.m0 - 1.0f;
        pv[1] = P.Jx / C.Jx0 - 1.0f;
        pv[2] = P.Jy / C.Jy0 - 1.0f;
        pv[3] = P.Jz / C.Jz0 - 1.0f;
        pv[4] = P.kf / C.kf0 - 1.0f;
        pv[5] = P.tm / C.tm0 - 1.0f;
    }
}

// Reward on s' with normalised action a; 0 for a non-finite s'.
__device__ __forceinline__ float reward(const float* Cr, const float* s, const float* a) {
    if (!finite_state(s)) return 0.0f;
    const float p2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
    const float v2 = s[7] * s[7] + s[8] * s[8] + s[9] * s[9];
    const float w2 = s[10] * s[10] + s[11] * s[11] + s[12] * s[12];
    float a2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float e = a[i] - Cr[5];
        a2 = fmaf(e, e, a2);
    }
    return -Cr[0] * p2 - Cr[1] * (1.0f - s[3] * s[3]) - Cr[2] * v2 - Cr[3] * w2 - Cr[4] * a2 + Cr[6];
}

__device__ __forceinline__ bool terminated(const EnvCfg& C, const float* s) {
    return !finite_state(s) || fabsf(s[0]) > C.term_pos || fabsf(s[1]) > C.term_pos ||
           fabsf(s[2]) > C.term_pos;
}

__device__ __forceinline__ void qmul(const float* a, const float* b, float* o) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Initial state, domain-randomised parameters and disturbance of episode `ep` of env.
__device__ __forceinline__ void reset_env(const EnvCfg& C, uint32_t env, uint32_t ep, float* s,
                                          float* prm7, float* d) {
    // the four initial-state blocks and the two domain-randomisation blocks, interleaved
    const uint32_t c2[6] = {TAG_RESET << 24, (TAG_RESET << 24) | 1u, (TAG_RESET << 24) | 2u,
                            (TAG_RESET << 24) | 3u, TAG_DR << 24, (TAG_DR << 24) | 1u};
    uint4 R6[6];
    draw_rolled_n<6>(C, env, ep, c2, R6);
    float U[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint4 r = R6[b];
        U[4 * b] = u01(r.x); U[4 * b + 1] = u01(r.y); U[4 * b + 2] = u01(r.z); U[4 * b + 3] = u01(r.w);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = C.init_p * (2.0f * U[k] - 1.0f);
    float sr, cr, sp, cp, sy, cy;
    sincosf(0.5f * C.init_att * (2.0f * U[3] - 1.0f), &sr, &cr);
    sincosf(0.5f * C.init_att * (2.0f * U[4] - 1.0f), &sp, &cp);
    sincosf(0.5f * C.init_att * (2.0f * U[5] - 1.0f), &sy, &cy);
    const float qz[4] = {cy, 0.0f, 0.0f, sy}, qy[4] = {cp, 0.0f, sp, 0.0f}, qx[4] = {cr, sr, 0.0f, 0.0f};
    float t1[4];
    qmul(qz, qy, t1);
    qmul(t1, qx, s + 3);
#pragma unroll
    for (int k = 0; k < 3; ++k) s[7 + k] = C.init_v * (2.0f * U[6 + k] - 1.0f);
#pragma unroll
    for (int k = 0; k < 3; ++k) s[10 + k] = C.init_w * (2.0f * U[9 + k] - 1.0f);
#pragma unroll
    for (int i = 0; i < 4; ++i) s[13 + i] = fmaf(C.init_rpm_hi - C.init_rpm_lo, U[12 + i], C.init_rpm_lo);
    const uint4 a = R6[4], b = R6[5];
    prm7[0] = C.m0 * (1.0f + C.dr_mass * (2.0f * u01(a.x) - 1.0f));
    prm7[1] = C.Jx0 * (1.0f + C.dr_J * (2.0f * u01(a.y) - 1.0f));
    prm7[2] = C.Jy0 * (1.0f + C.dr_J * (2.0f * u01(a.z) - 1.0f));
    prm7[3] = C.Jz0 * (1.0f + C.dr_J * (2.0f * u01(a.w) - 1.0f));
    prm7[4] = C.kf0 * (1.0f + C.dr_kf * (2.0f * u01(b.x) - 1.0f));
    prm7[5] = C.km0;
    prm7[6] = fmaf(C.tm_hi - C.tm_lo, u01(b.y), C.tm_lo);
    if (C.dist_f > 0.0f || C.dist_tau > 0.0f) {
        const uint4 x = draw_rolled(C, env, ep, TAG_DIST, 0), y = draw_rolled(C, env, ep, TAG_DIST, 1);
        d[0] = C.dist_f * (2.0f * u01(x.x) - 1.0f);
        d[1] = C.dist_f * (2.0f * u01(x.y) - 1.0f);
        d[2] = C.dist_f * (2.0f * u01(x.z) - 1.0f);
        d[3] = C.dist_tau * (2.0f * u01(x.w) - 1.0f);
        d[4] = C.dist_tau * (2.0f * u01(y.x) - 1.0f);
        d[5] = C.dist_tau * (2.0f * u01(y.y) - 1.0f);
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) d[k] = 0.0f;
    }
}

// Normalised action -> RPM set-point, linear over the RPM range.
__device__ __forceinline__ void action_to_rpm(const Vehicle& V, const float* a, float* u) {
    const float half = 0.5f * (V.rpm_max - V.rpm_min);
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = fmaf(a[i] + 1.0f, half, V.rpm_min);
}

__device__ __forceinline__ uint32_t pack_flags(bool term, bool trunc, uint32_t ep_step) {
    return (term ? 1u : 0u) | (trunc ? 2u : 0u) | (ep_step << 8);
}

// ------------------------------------------------------------- packed FP32 (f32x2) ops
// Blackwell's paired FP32 FMA: two IEEE single-precision FMAs (round to nearest) per
// instruction on a 64-bit register pair; element results equal fmaf's.
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Device status codes (first error wins).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADSIZE = 2, DEV_RANGE = 3, DEV_BOUNDS = 4 };

// A handle's status is STATUS_WORDS ints: [0] the code above; with DEV_BOUNDS also [1] the
// site, [2..3] the index and [4..5] the bound (64-bit, low word first).
constexpr int STATUS_WORDS = 8;

__device__ __forceinline__ void set_status(int* st, int code) {
    if (st) atomicCAS(st, DEV_OK, code);
}

// Debug bounds checks, compiled in with -DQSIM_BOUNDS_CHECK=1 (a separate build of the
// library) and out otherwise.  Every replay-ring slot and every SoA env index that a kernel
// computes before touching the ring is checked against its allocation; the first index
// outside [0, n) records DEV_BOUNDS, the site, the index and n in the status words, and the
// access is skipped.
#ifndef QSIM_BOUNDS_CHECK
#define QSIM_BOUNDS_CHECK 0
#endif
enum : int { SITE_RING_WRITE = 1, SITE_RING_READ = 2, SITE_SOA = 3, SITE_PROBE = 4 };

__device__ __forceinline__ bool in_bounds(int* st, int64_t i, int64_t n, int site) {
#if QSIM_BOUNDS_CHECK
    if (i >= 0 && i < n) return true;
    if (st && atomicCAS(st, DEV_OK, DEV_BOUNDS) == DEV_OK) {
        st[1] = site;
        st[2] = (int)(uint32_t)(uint64_t)i;
        st[3] = (int)(uint32_t)((uint64_t)i >> 32);
        st[4] = (int)(uint32_t)(uint64_t)n;
        st[5] = (int)(uint32_t)((uint64_t)n >> 32);
    }
    return false;
#else
    (void)st; (void)i; (void)n; (void)site;
    return true;
#endif
}

}  // namespace qsim
