// qsim_diff.cu -- reverse-mode gradients through an H-step RK4 rollout (differentiable
// simulation of the Sec. IV dynamics, with or without the actor in the loop).
//
// Schedule (thread per env, state in registers):
//   forward   : integrate H steps, store the state every `ckpt` steps and the actions,
//               accumulate the loss.
//   backward  : for each segment, last to first: recompute the segment's states from its
//               checkpoint (in closed loop also the actor's inputs and hidden activations,
//               two steps per pass through the layers), then sweep it in reverse --
//               vector-Jacobian product of RK4 (four stage derivatives recomputed,
//               quaternion renormalisation included), of the action -> RPM map, and in
//               closed loop of the actor (backprop with weights in shared memory; history
//               inputs pass their adjoint to earlier actions).  The adjoint state and
//               parameter gradients carry over between segments in the workspace.
//   weights   : closed loop only -- the per-(step, env) activations and deltas of a
//               segment are reduced into the actor gradient over env chunks (on a side
//               stream while the next segment's reverse sweep runs, with two record
//               buffers in turn), then summed over chunks in a fixed order
//               (deterministic).
// Memory: O(H/ckpt + ckpt) states per env instead of O(H).
#include <algorithm>
#include <cstring>

#include "qsim_gemm.cuh"
#include "qsim_internal.h"

namespace qsim {

struct VjpArgs {
    Vehicle V;
    int n, ld, H, ckpt, mode, nh, hid, DA, PA, nseg, nchunk, chunk, npart;  // npart: weight-gradient partials
    float w_p, w_q, w_v, w_a, dt;
    int renorm;
    const float *s0, *prm, *actions, *actor, *seed;
    float *loss, *g_actions, *g_actor, *g_params, *actions_out;
    // workspace
    float *ck, *A, *la, *segs, *lam, *gp, *rec, *fo, *part;
};

constexpr int VT = 128;  // threads per CTA of the per-env kernels

__device__ __forceinline__ void load_vehicle_prm(const VjpArgs& a, int e, Prm& P) {
    const float* p = a.prm;
    const int ld = a.ld;
    P = make_prm(p[e], p[ld + e], p[2 * ld + e], p[3 * ld + e], p[4 * ld + e], p[5 * ld + e],
                 p[6 * ld + e]);
}

__device__ __forceinline__ float state_loss(const VjpArgs& a, const float* s) {
    return a.w_p * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) + a.w_q * (1.0f - s[3] * s[3]) +
           a.w_v * (s[7] * s[7] + s[8] * s[8] + s[9] * s[9]);
}

__device__ __forceinline__ void state_loss_grad(const VjpArgs& a, const float* s, float* g) {
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] += 2.0f * a.w_p * s[k];
    g[3] += -2.0f * a.w_q * s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[7 + k] += 2.0f * a.w_v * s[7 + k];
}

// d(derivative)^T lam, added into gs (state), gu (unclipped set-point) and gp (m, Jx, Jy,
// Jz, kf, km, T_m).  No disturbance in the differentiable rollout.
__device__ __forceinline__ void deriv_vjp(const Vehicle& V, const float* s, const float* u,
                                          const Prm& P, const float* lam, float* gs, float* gu,
                                          float* gp) {
    const float qw = s[3], qx = s[4], qy = s[5], qz = s[6];
    const float wx = s[10], wy = s[11], wz = s[12];
    float f[4], F = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) { f[i] = P.kf * s[13 + i] * s[13 + i]; F += f[i]; }
    const float r02 = 2.0f * (qx * qz + qw * qy);
    const float r12 = 2.0f * (qy * qz - qw * qx);
    const float r22 = 1.0f - 2.0f * (qx * qx + qy * qy);
    // p' = v
    gs[7] += lam[0]; gs[8] += lam[1]; gs[9] += lam[2];
    // v' = R e_z F / m - g e_z
    const float lv0 = lam[7], lv1 = lam[8], lv2 = lam[9];
    const float gF = (lv0 * r02 + lv1 * r12 + lv2 * r22) * P.im;
    gp[0] += -(lv0 * r02 + lv1 * r12 + lv2 * r22) * F * P.im * P.im;
    const float G2 = lv0 * F * P.im, G5 = lv1 * F * P.im, G8 = lv2 * F * P.im;
    gs[3] += 2.0f * (qy * G2 - qx * G5);
    gs[4] += 2.0f * (qz * G2 - qw * G5 - 2.0f * qx * G8);
    gs[5] += 2.0f * (qw * G2 + qz * G5 - 2.0f * qy * G8);
    gs[6] += 2.0f * (qx * G2 + qy * G5);
    // q' = 1/2 q (x) (0, w)
    const float l0 = lam[3], l1 = lam[4], l2 = lam[5], l3 = lam[6];
    gs[3] += 0.5f * (l1 * wx + l2 * wy + l3 * wz);
    gs[4] += 0.5f * (-l0 * wx - l2 * wz + l3 * wy);
    gs[5] += 0.5f * (-l0 * wy + l1 * wz - l3 * wx);
    gs[6] += 0.5f * (-l0 * wz - l1 * wy + l2 * wx);
    gs[10] += 0.5f * (-qx * l0 + qw * l1 + qz * l2 - qy * l3);
    gs[11] += 0.5f * (-qy * l0 - qz * l1 + qw * l2 + qx * l3);
    gs[12] += 0.5f * (-qz * l0 + qy * l1 - qx * l2 + qw * l3);
    // w' = J^-1 (tau - w x J w)
    const float mx = lam[10] * P.iJx, my = lam[11] * P.iJy, mz = lam[12] * P.iJz;
    float tx = 0.0f, ty = 0.0f, tz = 0.0f, sdf = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        tx = fmaf(V.ry[i], f[i], tx);
        ty = fmaf(-V.rx[i], f[i], ty);
        sdf = fmaf(V.dir[i], f[i], sdf);
    }
    tz = P.km * sdf;
    const float wdx = (tx - (P.Jz - P.Jy) * wy * wz) * P.iJx;
    const float wdy = (ty - (P.Jx - P.Jz) * wz * wx) * P.iJy;
    const float wdz = (tz - (P.Jy - P.Jx) * wx * wy) * P.iJz;
    gs[10] += -my * (P.Jx - P.Jz) * wz - mz * (P.Jy - P.Jx) * wy;
    gs[11] += -mx * (P.Jz - P.Jy) * wz - mz * (P.Jy - P.Jx) * wx;
    gs[12] += -mx * (P.Jz - P.Jy) * wy - my * (P.Jx - P.Jz) * wx;
    gp[1] += -mx * wdx - my * wz * wx + mz * wx * wy;
    gp[2] += -my * wdy + mx * wy * wz - mz * wx * wy;
    gp[3] += -mz * wdz - mx * wy * wz + my * wz * wx;
    // rotor forces
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float gf = gF + mx * V.ry[i] - my * V.rx[i] + mz * V.dir[i] * P.km;
        gs[13 + i] += gf * 2.0f * P.kf * s[13 + i];
        gp[4] += gf * s[13 + i] * s[13 + i];
    }
    gp[5] += mz * sdf;
    // motor lag
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float uc = clampf(u[i], V.rpm_min, V.rpm_max);
        const float lm = lam[13 + i];
        gs[13 + i] += -lm * P.itm;
        if (u[i] > V.rpm_min && u[i] < V.rpm_max) gu[i] += lm * P.itm;
        gp[6] += -lm * (uc - s[13 + i]) * P.itm * P.itm;
    }
}

// Reverse of one RK4 step: lam_out = dL/ds'; gs receives dL/ds (overwritten), gu and gp
// are accumulated.
__device__ __forceinline__ void rk4_vjp(const Vehicle& V, float dt, int renorm, const float* s,
                                        const float* u, const Prm& P, const float* lam_out,
                                        float* gs, float* gu, float* gp) {
    float uc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) uc[i] = clampf(u[i], V.rpm_min, V.rpm_max);
    const float d0[6] = {0, 0, 0, 0, 0, 0};
    float k1[NS], k2[NS], k3[NS], y2[NS], y3[NS], y4[NS];
    deriv(V, s, uc, P, d0, k1);
#pragma unroll
    for (int i = 0; i < NS; ++i) y2[i] = fmaf(0.5f * dt, k1[i], s[i]);
    deriv(V, y2, uc, P, d0, k2);
#pragma unroll
    for (int i = 0; i < NS; ++i) y3[i] = fmaf(0.5f * dt, k2[i], s[i]);
    deriv(V, y3, uc, P, d0, k3);
#pragma unroll
    for (int i = 0; i < NS; ++i) y4[i] = fmaf(dt, k3[i], s[i]);
    float lam[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) lam[i] = lam_out[i];
    if (renorm) {
        float k4[NS];
        deriv(V, y4, uc, P, d0, k4);
        float pre[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            pre[i] = s[3 + i] + dt * (1.0f / 6.0f) * (k1[3 + i] + 2.0f * k2[3 + i] + 2.0f * k3[3 + i] + k4[3 + i]);
        const float inv = rsqrtf(pre[0] * pre[0] + pre[1] * pre[1] + pre[2] * pre[2] + pre[3] * pre[3]);
        float dot = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) dot += pre[i] * inv * lam_out[3 + i];
#pragma unroll
        for (int i = 0; i < 4; ++i) lam[3 + i] = (lam_out[3 + i] - pre[i] * inv * dot) * inv;
    }
    float lk[NS], ly[NS], lk2[NS], lk3[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        gs[i] = lam[i];
        lk[i] = dt * (1.0f / 6.0f) * lam[i];   // k4 and k1 weight
        lk2[i] = dt * (1.0f / 3.0f) * lam[i];  // k2 weight
        lk3[i] = lk2[i];                       // k3 weight
        ly[i] = 0.0f;
    }
    deriv_vjp(V, y4, u, P, lk, ly, gu, gp);       // k4 = f(y4), y4 = s + dt k3
#pragma unroll
    for (int i = 0; i < NS; ++i) { gs[i] += ly[i]; lk3[i] = fmaf(dt, ly[i], lk3[i]); ly[i] = 0.0f; }
    deriv_vjp(V, y3, u, P, lk3, ly, gu, gp);      // k3 = f(y3), y3 = s + dt/2 k2
#pragma unroll
    for (int i = 0; i < NS; ++i) { gs[i] += ly[i]; lk2[i] = fmaf(0.5f * dt, ly[i], lk2[i]); ly[i] = 0.0f; }
    deriv_vjp(V, y2, u, P, lk2, ly, gu, gp);      // k2 = f(y2), y2 = s + dt/2 k1
#pragma unroll
    for (int i = 0; i < NS; ++i) { gs[i] += ly[i]; lk[i] = fmaf(0.5f * dt, ly[i], lk[i]); ly[i] = 0.0f; }
    deriv_vjp(V, s, u, P, lk, ly, gu, gp);        // k1 = f(s)
#pragma unroll
    for (int i = 0; i < NS; ++i) gs[i] += ly[i];
}

// Reverse of the observation's state entries {p, R(q) row-major, v, omega}.
__device__ __forceinline__ void obs_vjp(const float* s, const float* go, float* gs) {
    const float qw = s[3], qx = s[4], qy = s[5], qz = s[6];
    const float* G = go + 3;
    gs[0] += go[0]; gs[1] += go[1]; gs[2] += go[2];
    gs[3] += 2.0f * (-qz * G[1] + qy * G[2] + qz * G[3] - qx * G[5] - qy * G[6] + qx * G[7]);
    gs[4] += 2.0f * (qy * G[1] + qz * G[2] + qy * G[3] - 2.0f * qx * G[4] - qw * G[5] + qz * G[6] +
                     qw * G[7] - 2.0f * qx * G[8]);
    gs[5] += 2.0f * (-2.0f * qy * G[0] + qx * G[1] + qw * G[2] + qx * G[3] + qz * G[5] - qw * G[6] +
                     qz * G[7] - 2.0f * qy * G[8]);
    gs[6] += 2.0f * (-2.0f * qz * G[0] - qw * G[1] + qx * G[2] + qw * G[3] - 2.0f * qz * G[4] +
                     qy * G[5] + qx * G[6] + qy * G[7]);
    gs[7] += go[12]; gs[8] += go[13]; gs[9] += go[14];
    gs[10] += go[15]; gs[11] += go[16]; gs[12] += go[17];
}

// Actor observation of env e at step t into O [DA][ld] column e: state part from s, then
// the rollout's own previous actions (zeros before t = 0).
__device__ __forceinline__ void build_obs(const VjpArgs& a, int e, int t, const float* s, float* O) {
    const int ld = a.ld;
    float o[18];
    obs_state(s, o);
#pragma unroll
    for (int k = 0; k < 18; ++k) O[k * ld] = o[k];
    for (int i = 1; i <= a.nh; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            O[(18 + 4 * (i - 1) + c) * ld] = (t - i >= 0) ? a.A[((size_t)(t - i) * 4 + c) * ld + e] : 0.0f;
}

// Per-thread actor forward with weights in shared memory; vectors live in column e of
// field-major global arrays (coalesced across the warp, L1-resident).
__device__ __forceinline__ void actor_fwd_thread(const float* sW, int DA, int H, const float* O,
                                                 float* H1, float* H2, int ld, float* mu) {
    const float* W1 = sW;
    const float* b1 = W1 + H * DA;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + 4 * H;
    for (int j = 0; j < H; ++j) {
        float acc = b1[j];
        for (int k = 0; k < DA; ++k) acc = fmaf(W1[j * DA + k], O[k * ld], acc);
        H1[j * ld] = fmaxf(acc, 0.0f);
    }
    for (int j = 0; j < H; ++j) {
        float acc = b2[j];
        for (int k = 0; k < H; ++k) acc = fmaf(W2[j * H + k], H1[k * ld], acc);
        H2[j * ld] = fmaxf(acc, 0.0f);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float acc = b3[j];
        for (int k = 0; k < H; ++k) acc = fmaf(W3[j * H + k], H2[k * ld], acc);
        mu[j] = tanhf(acc);
    }
}

__global__ void __launch_bounds__(VT) k_vjp_forward(VjpArgs a) {
    extern __shared__ __align__(16) float sW[];
    if (a.mode == 1) {
        for (int i = threadIdx.x; i < a.PA; i += VT) sW[i] = a.actor[i];
        __syncthreads();
    }
    const int e = blockIdx.x * VT + threadIdx.x;
    if (e >= a.n) return;
    const int ld = a.ld;
    float s[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = a.s0[i * ld + e];
    Prm P;
    load_vehicle_prm(a, e, P);
    const float d0[6] = {0, 0, 0, 0, 0, 0};
    const float half = 0.5f * (a.V.rpm_max - a.V.rpm_min);
    float loss = 0.0f;
    for (int t = 0; t < a.H; ++t) {
        if (t % a.ckpt == 0) {
            float* c = a.ck + (size_t)(t / a.ckpt) * NS * ld + e;
#pragma unroll
            for (int i = 0; i < NS; ++i) c[i * ld] = s[i];
        }
        float act[4];
        if (a.mode == 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) act[c] = a.actions[((size_t)t * 4 + c) * ld + e];
        } else {
            float* O = a.fo + e;
            build_obs(a, e, t, s, O);
            actor_fwd_thread(sW, a.DA, a.hid, O, O + (size_t)a.DA * ld, O + (size_t)(a.DA + a.hid) * ld,
                             ld, act);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            a.A[((size_t)t * 4 + c) * ld + e] = act[c];
            if (a.actions_out) a.actions_out[((size_t)t * 4 + c) * ld + e] = act[c];
        }
        float u[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) u[c] = fmaf(act[c] + 1.0f, half, a.V.rpm_min);
        rk4(a.V, a.dt, a.renorm, s, u, P, d0);
        loss += state_loss(a, s) + a.w_a * (act[0] * act[0] + act[1] * act[1] + act[2] * act[2] + act[3] * act[3]);
    }
    if (a.loss) a.loss[e] = loss;
}

// Reverse sweep over segment g.
__global__ void __launch_bounds__(VT) k_vjp_backward(VjpArgs a, int g) {
    extern __shared__ __align__(16) float sW[];
    if (a.mode == 1) {
        for (int i = threadIdx.x; i < a.PA; i += VT) sW[i] = a.actor[i];
        __syncthreads();
    }
    const int e = blockIdx.x * VT + threadIdx.x;
    if (e >= a.n) return;
    const int ld = a.ld, DA = a.DA, H = a.hid;
    const int t0 = g * a.ckpt, t1 = min(a.H, t0 + a.ckpt);
    const bool last = (t1 == a.H);
    const float seed = a.seed ? a.seed[e] : 1.0f;
    Prm P;
    load_vehicle_prm(a, e, P);
    const float d0[6] = {0, 0, 0, 0, 0, 0};
    const float half = 0.5f * (a.V.rpm_max - a.V.rpm_min);
    // recompute the segment's states from its checkpoint
    float s[NS];
    {
        const float* c = a.ck + (size_t)g * NS * ld + e;
#pragma unroll
        for (int i = 0; i < NS; ++i) s[i] = c[i * ld];
    }
    float lam[NS], gp[7];
    for (int t = t0; t < t1; ++t) {
        float* ss = a.segs + (size_t)(t - t0) * NS * ld + e;
#pragma unroll
        for (int i = 0; i < NS; ++i) ss[i * ld] = s[i];
        float u[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) u[c] = fmaf(a.A[((size_t)t * 4 + c) * ld + e] + 1.0f, half, a.V.rpm_min);
        rk4(a.V, a.dt, a.renorm, s, u, P, d0);
    }
    if (last) {
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] = 0.0f;
        state_loss_grad(a, s, lam);
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] *= seed;
#pragma unroll
        for (int i = 0; i < 7; ++i) gp[i] = 0.0f;
    } else {
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] = a.lam[i * ld + e];
#pragma unroll
        for (int i = 0; i < 7; ++i) gp[i] = a.gp[i * ld + e];
    }
    const size_t NR = (size_t)DA + 4 * H + 4;  // O, H1, H2, dZ1, dZ2, dZ3 per (step, env)
    for (int t = t1 - 1; t >= t0; --t) {
        float st[NS];
        const float* ss = a.segs + (size_t)(t - t0) * NS * ld + e;
#pragma unroll
        for (int i = 0; i < NS; ++i) st[i] = ss[i * ld];
        float act[4], u[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            act[c] = a.A[((size_t)t * 4 + c) * ld + e];
            u[c] = fmaf(act[c] + 1.0f, half, a.V.rpm_min);
        }
        float gs[NS], gu[4] = {0, 0, 0, 0};
        rk4_vjp(a.V, a.dt, a.renorm, st, u, P, lam, gs, gu, gp);
        float ga[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ga[c] = gu[c] * half + seed * 2.0f * a.w_a * act[c];
        if (a.mode == 0) {
            if (a.g_actions)
#pragma unroll
                for (int c = 0; c < 4; ++c) a.g_actions[((size_t)t * 4 + c) * ld + e] = ga[c];
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) ga[c] += a.la[((size_t)t * 4 + c) * ld + e];
            float* R = a.rec + (size_t)(t - t0) * NR * ld + e;
            float* O = R;
            float* H1 = R + (size_t)DA * ld;
            float* H2 = H1 + (size_t)H * ld;
            float* dZ1 = H2 + (size_t)H * ld;
            float* dZ2 = dZ1 + (size_t)H * ld;
            float* dZ3 = dZ2 + (size_t)H * ld;
            build_obs(a, e, t, st, O);
            float mu[4];
            actor_fwd_thread(sW, DA, H, O, H1, H2, ld, mu);
            const float* W1 = sW;
            const float* W2 = W1 + H * DA + H;
            const float* W3 = W2 + H * H + H;
            float z3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                z3[c] = ga[c] * (1.0f - mu[c] * mu[c]);
                dZ3[c * ld] = z3[c];
            }
            for (int k = 0; k < H; ++k) {
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < 4; ++c) acc = fmaf(W3[c * H + k], z3[c], acc);
                dZ2[k * ld] = H2[k * ld] > 0.0f ? acc : 0.0f;
            }
            for (int k = 0; k < H; ++k) {
                float acc = 0.0f;
                for (int j = 0; j < H; ++j) acc = fmaf(W2[j * H + k], dZ2[j * ld], acc);
                dZ1[k * ld] = H1[k * ld] > 0.0f ? acc : 0.0f;
            }
            float go[18];
            for (int k = 0; k < 18; ++k) {
                float acc = 0.0f;
                for (int j = 0; j < H; ++j) acc = fmaf(W1[j * DA + k], dZ1[j * ld], acc);
                go[k] = acc;
            }
            obs_vjp(st, go, gs);
            for (int i = 1; i <= a.nh && t - i >= 0; ++i)
                for (int c = 0; c < 4; ++c) {
                    const int k = 18 + 4 * (i - 1) + c;
                    float acc = 0.0f;
                    for (int j = 0; j < H; ++j) acc = fmaf(W1[j * DA + k], dZ1[j * ld], acc);
                    a.la[((size_t)(t - i) * 4 + c) * ld + e] += acc;
                }
        }
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] = gs[i];
        if (t >= 1) {
            float lg[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) lg[i] = 0.0f;
            state_loss_grad(a, st, lg);
#pragma unroll
            for (int i = 0; i < NS; ++i) lam[i] = fmaf(seed, lg[i], lam[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) a.lam[i * ld + e] = lam[i];
#pragma unroll
    for (int i = 0; i < 7; ++i) a.gp[i * ld + e] = gp[i];
    if (g == 0 && a.g_params)
#pragma unroll
        for (int i = 0; i < 4; ++i) a.g_params[i * ld + e] = gp[i];
}

// ------------------------------------------------------- closed loop, lane group per env
// The thread-per-env kernels above leave the GPU nearly idle at a few thousand envs (one
// warp per SM) and re-read every activation from memory for each output.  For hidden 32 or
// 64 (and at most 96 actor inputs) the closed loop runs one env per group of LPE lanes
// instead (LPE = 32, 16 or 8; 32 / LPE envs per warp): every lane of a group keeps the full
// state and runs RK4 and its vector-Jacobian product redundantly (no communication), while
// the actor's layers are split across the group's lanes (lane l of the group owns hidden
// units l + LPE j and inputs l + LPE m), with broadcasts by group-wide shuffles and the
// weights in shared memory (odd row strides: conflict-free for lane-varying rows and
// columns alike; the groups of a warp read the same weights, a broadcast).  Narrower groups
// spend fewer instructions per env on the redundant integration.  The action history and
// the history-input adjoints live in per-env rings of 16 x 4 floats in shared memory.
// Activation records for the weight gradient are written env-major ([step][env][field]:
// one contiguous row per env).
// Warps per CTA of the lane-group kernels: 4 (two CTAs per SM), or 7 at 8 lanes per env
// (one CTA per SM), whichever leaves the fewest warps on the busiest SM for the env count
// (host: lane_group_warps).  At 4,096 envs 7 gives 147 CTAs of 7 warps, one wave, against
// 256 CTAs of 4 that put 8 warps on most SMs.
constexpr int kWvSmall = 4, kWvWide = 7;
constexpr int SB = 2;  // steps per pass through the hidden layers in the reverse sweep's recompute

// Row stride (floats) for 16-byte loads of consecutive rows by the lanes of a group: a
// multiple of 4 whose quarter is odd, so that 8 consecutive rows start in 8 distinct bank
// quads (conflict-free).
__host__ __device__ constexpr int vstride(int n) {
    return (((n + 3) & ~3) >> 2) & 1 ? ((n + 3) & ~3) : ((n + 3) & ~3) + 4;
}

// Weights in shared memory, one copy each: W1 [H][l1] and W2 [H][l2] (row padding zero),
// W3 [4][H], biases.  Forward products: a lane reads 4 consecutive inputs of one of its
// rows with one 16-byte load (rows of the group's lanes in distinct bank quads); reverse
// products: the group's lanes read consecutive columns of one row (conflict-free).
struct WarpActor {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
    int l1, l2;  // row strides
};

__device__ __forceinline__ WarpActor stage_warp_actor(const float* actor, int DA, int H, float* sm) {
    WarpActor w;
    const int l1 = vstride(DA), l2 = vstride(H);
    float* W1 = sm;
    float* W2 = W1 + H * l1;
    float* b1 = W2 + H * l2;
    float* b2 = b1 + H;
    float* W3 = b2 + H;
    float* b3 = W3 + 4 * H;
    const float* gW1 = actor;
    const float* gb1 = gW1 + H * DA;
    const float* gW2 = gb1 + H;
    const float* gb2 = gW2 + H * H;
    const float* gW3 = gb2 + H;
    const float* gb3 = gW3 + 4 * H;
    for (int i = threadIdx.x; i < H * l1; i += blockDim.x) {
        const int j = i / l1, k = i - j * l1;
        const float v = k < DA ? gW1[j * DA + k] : 0.0f;
        W1[i] = v;
    }
    for (int i = threadIdx.x; i < H * l2; i += blockDim.x) {
        const int j = i / l2, k = i - j * l2;
        W2[i] = k < H ? gW2[j * H + k] : 0.0f;
    }
    for (int i = threadIdx.x; i < H; i += blockDim.x) { b1[i] = gb1[i]; b2[i] = gb2[i]; }
    for (int i = threadIdx.x; i < 4 * H; i += blockDim.x) W3[i] = gW3[i];
    if (threadIdx.x < 4) b3[threadIdx.x] = gb3[threadIdx.x];
    w.W1 = W1; w.b1 = b1; w.W2 = W2; w.b2 = b2; w.W3 = W3; w.b3 = b3;
    w.l1 = l1; w.l2 = l2;
    return w;
}

__host__ __device__ inline int warp_actor_floats(int DA, int H) {
    return H * vstride(DA) + H * vstride(H) + 2 * H + 4 * H + 4;
}

// Per-lane shape of the lane-group kernels.
template <int H, int LPE>
struct Grp {
    static constexpr int HPL = H / LPE;               // hidden units per lane
    static constexpr int NX = (96 + LPE - 1) / LPE;   // actor inputs per lane (at most 96 inputs)
    static constexpr int G = 32 / LPE;                // envs per warp
    static_assert(H % LPE == 0 && 32 % LPE == 0, "lane-group shape");
};

// Value of v[i] for a run-time index i (select chain; v stays in registers).
template <int N>
__device__ __forceinline__ float pick(const float* v, int i) {
    float r = v[0];
#pragma unroll
    for (int k = 1; k < N; ++k) r = i == k ? v[k] : r;
    return r;
}

template <int LPE>
__device__ __forceinline__ float grp_sum(float v) {
#pragma unroll
    for (int o = LPE / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// This lane's actor inputs x[m] = input (group lane + LPE m): the observation of state s
// (inputs < 18) then the action history a_{t-i} (zero before the rollout starts or beyond
// n_hist), read through `hist(step, component)`.
template <int LPE, int NX, class Hist>
__device__ __forceinline__ void grp_actor_input(const float* s, int t, int DA, int nh, Hist hist, float* x) {
    const int gl = threadIdx.x & (LPE - 1);
    float o[18];
    obs_state(s, o);
#pragma unroll
    for (int m = 0; m < NX; ++m) {
        const int k = gl + LPE * m;
        float v = 0.0f;
        if (LPE * m < 18) {
            const float ok = pick<18>(o, k);
            if (k < 18) v = ok;
        }
        if (k >= 18 && k < DA) {
            const int i = ((k - 18) >> 2) + 1, c = (k - 18) & 3;
            if (i <= nh && t - i >= 0) v = hist(t - i, c);
        }
        x[m] = v;
    }
}

// Actor forward for this group's env: h1, h2 for the lane's hidden units, mu on every lane.
template <int H, int LPE>
__device__ __forceinline__ void grp_actor_fwd(const WarpActor& w, int DA, const float* x, float* h1,
                                              float* h2, float* mu) {
    using S = Grp<H, LPE>;
    const int gl = threadIdx.x & (LPE - 1);
    float acc[S::HPL];
#pragma unroll
    for (int j = 0; j < S::HPL; ++j) acc[j] = w.b1[gl + LPE * j];
    // inputs in fours: four broadcasts, then one 16-byte weight load and four FMAs (in input
    // order) per hidden unit; past DA both the inputs and the padded weights are zero
#pragma unroll
    for (int m = 0; m < S::NX; ++m) {
        for (int kk = 0; kk < LPE && LPE * m + kk < DA; kk += 4) {
            float xk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) xk[q] = __shfl_sync(0xffffffffu, x[m], kk + q, LPE);
            const float* wr = w.W1 + gl * w.l1 + LPE * m + kk;
#pragma unroll
            for (int j = 0; j < S::HPL; ++j) {
                const float4 wv = *reinterpret_cast<const float4*>(wr + LPE * j * w.l1);
                acc[j] = fmaf(wv.x, xk[0], acc[j]);
                acc[j] = fmaf(wv.y, xk[1], acc[j]);
                acc[j] = fmaf(wv.z, xk[2], acc[j]);
                acc[j] = fmaf(wv.w, xk[3], acc[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < S::HPL; ++j) { h1[j] = fmaxf(acc[j], 0.0f); acc[j] = w.b2[gl + LPE * j]; }
#pragma unroll
    for (int m = 0; m < S::HPL; ++m)
        for (int kk = 0; kk < LPE; kk += 4) {
            float hk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) hk[q] = __shfl_sync(0xffffffffu, h1[m], kk + q, LPE);
            const float* wr = w.W2 + gl * w.l2 + LPE * m + kk;
#pragma unroll
            for (int j = 0; j < S::HPL; ++j) {
                const float4 wv = *reinterpret_cast<const float4*>(wr + LPE * j * w.l2);
                acc[j] = fmaf(wv.x, hk[0], acc[j]);
                acc[j] = fmaf(wv.y, hk[1], acc[j]);
                acc[j] = fmaf(wv.z, hk[2], acc[j]);
                acc[j] = fmaf(wv.w, hk[3], acc[j]);
            }
        }
#pragma unroll
    for (int j = 0; j < S::HPL; ++j) h2[j] = fmaxf(acc[j], 0.0f);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float pc = 0.0f;
#pragma unroll
        for (int j = 0; j < S::HPL; ++j) pc = fmaf(w.W3[c * H + gl + LPE * j], h2[j], pc);
        mu[c] = tanhf(grp_sum<LPE>(pc) + w.b3[c]);
    }
}

// The actor's hidden layers h1, h2 (this lane's units) for SB steps of this group's env at
// once, from their inputs x[b]: each 16-byte weight load serves SB steps.  Every unit sums
// in the same order as grp_actor_fwd (bias, then the inputs in order), so h1 and h2 are
// bitwise those of the forward pass.
template <int H, int LPE, int SB>
__device__ __forceinline__ void grp_actor_hidden_steps(const WarpActor& w, int DA,
                                                       const float (&x)[SB][Grp<H, LPE>::NX],
                                                       float (&h1)[SB][Grp<H, LPE>::HPL],
                                                       float (&h2)[SB][Grp<H, LPE>::HPL]) {
    using S = Grp<H, LPE>;
    const int gl = threadIdx.x & (LPE - 1);
    float acc[SB][S::HPL];
#pragma unroll
    for (int j = 0; j < S::HPL; ++j) {
        const float b = w.b1[gl + LPE * j];
#pragma unroll
        for (int q = 0; q < SB; ++q) acc[q][j] = b;
    }
#pragma unroll
    for (int m = 0; m < S::NX; ++m) {
        for (int kk = 0; kk < LPE && LPE * m + kk < DA; kk += 4) {
            float xk[SB][4];
#pragma unroll
            for (int q = 0; q < SB; ++q)
#pragma unroll
                for (int i = 0; i < 4; ++i) xk[q][i] = __shfl_sync(0xffffffffu, x[q][m], kk + i, LPE);
            const float* wr = w.W1 + gl * w.l1 + LPE * m + kk;
#pragma unroll
            for (int j = 0; j < S::HPL; ++j) {
                const float4 wv = *reinterpret_cast<const float4*>(wr + LPE * j * w.l1);
#pragma unroll
                for (int q = 0; q < SB; ++q) {
                    acc[q][j] = fmaf(wv.x, xk[q][0], acc[q][j]);
                    acc[q][j] = fmaf(wv.y, xk[q][1], acc[q][j]);
                    acc[q][j] = fmaf(wv.z, xk[q][2], acc[q][j]);
                    acc[q][j] = fmaf(wv.w, xk[q][3], acc[q][j]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < S::HPL; ++j) {
        const float b = w.b2[gl + LPE * j];
#pragma unroll
        for (int q = 0; q < SB; ++q) { h1[q][j] = fmaxf(acc[q][j], 0.0f); acc[q][j] = b; }
    }
#pragma unroll
    for (int m = 0; m < S::HPL; ++m)
        for (int kk = 0; kk < LPE; kk += 4) {
            float hk[SB][4];
#pragma unroll
            for (int q = 0; q < SB; ++q)
#pragma unroll
                for (int i = 0; i < 4; ++i) hk[q][i] = __shfl_sync(0xffffffffu, h1[q][m], kk + i, LPE);
            const float* wr = w.W2 + gl * w.l2 + LPE * m + kk;
#pragma unroll
            for (int j = 0; j < S::HPL; ++j) {
                const float4 wv = *reinterpret_cast<const float4*>(wr + LPE * j * w.l2);
#pragma unroll
                for (int q = 0; q < SB; ++q) {
                    acc[q][j] = fmaf(wv.x, hk[q][0], acc[q][j]);
                    acc[q][j] = fmaf(wv.y, hk[q][1], acc[q][j]);
                    acc[q][j] = fmaf(wv.z, hk[q][2], acc[q][j]);
                    acc[q][j] = fmaf(wv.w, hk[q][3], acc[q][j]);
                }
            }
        }
#pragma unroll
    for (int j = 0; j < S::HPL; ++j)
#pragma unroll
        for (int q = 0; q < SB; ++q) h2[q][j] = fmaxf(acc[q][j], 0.0f);
}

// Env handled by this lane's group, whether it exists, and whether any group of the warp
// has an env (warp-uniform).  A group past the last env runs on a valid index (the last
// env) so that the warp's shuffles stay complete, and stores nothing.
template <int LPE, int WV>
__device__ __forceinline__ void grp_env(int n, int& e, bool& live, bool& warp_live) {
    constexpr int G = 32 / LPE;
    const int warp = threadIdx.x >> 5, sub = (threadIdx.x & 31) / LPE;
    const int e0 = (blockIdx.x * WV + warp) * G;
    e = e0 + sub;
    live = e < n;
    warp_live = e0 < n;
    if (!live) e = n - 1;
}

template <int H, int LPE, int WV>
__global__ void __launch_bounds__(32 * WV) k_vjp_forward_w(VjpArgs a) {
    using S = Grp<H, LPE>;
    extern __shared__ __align__(16) float sm[];
    const int DA = a.DA, ld = a.ld;
    const WarpActor w = stage_warp_actor(a.actor, DA, H, sm);
    const int gl = threadIdx.x & (LPE - 1);
    float* ring = sm + warp_actor_floats(DA, H) + 64 * (threadIdx.x / LPE);  // a_tau at (tau & 15)
    __syncthreads();
    int e;
    bool live, warp_live;
    grp_env<LPE, WV>(a.n, e, live, warp_live);
    if (!warp_live) return;  // warp-uniform
    float s[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = a.s0[i * ld + e];
    Prm P;
    load_vehicle_prm(a, e, P);
    const float d0[6] = {0, 0, 0, 0, 0, 0};
    const float half = 0.5f * (a.V.rpm_max - a.V.rpm_min);
    float loss = 0.0f;
    for (int t = 0; t < a.H; ++t) {
        if (t % a.ckpt == 0) {
#pragma unroll
            for (int r = 0; r < (NS + LPE - 1) / LPE; ++r) {
                const int i = gl + LPE * r;
                const float v = pick<NS>(s, i);
                if (live && i < NS) a.ck[(size_t)(t / a.ckpt) * NS * ld + (size_t)i * ld + e] = v;
            }
        }
        float x[S::NX], h1[S::HPL], h2[S::HPL], act[4];
        grp_actor_input<LPE, S::NX>(s, t, DA, a.nh, [&](int tau, int c) { return ring[(tau & 15) * 4 + c]; }, x);
        grp_actor_fwd<H, LPE>(w, DA, x, h1, h2, act);
        __syncwarp();
        if (gl < 4) {
            const float v = pick<4>(act, gl);
            ring[(t & 15) * 4 + gl] = v;
            if (live) {
                a.A[((size_t)t * 4 + gl) * ld + e] = v;
                if (a.actions_out) a.actions_out[((size_t)t * 4 + gl) * ld + e] = v;
            }
        }
        __syncwarp();
        float u[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) u[c] = fmaf(act[c] + 1.0f, half, a.V.rpm_min);
        rk4(a.V, a.dt, a.renorm, s, u, P, d0);
        loss += state_loss(a, s) + a.w_a * (act[0] * act[0] + act[1] * act[1] + act[2] * act[2] + act[3] * act[3]);
    }
    if (a.loss && gl == 0 && live) a.loss[e] = loss;
}

// Reverse sweep over segment g, one env per lane group.
template <int H, int LPE, int WV>
__global__ void __launch_bounds__(32 * WV, WV == kWvSmall ? 2 : 1) k_vjp_backward_w(VjpArgs a, int g) {
    using S = Grp<H, LPE>;
    constexpr int HPL = S::HPL, NX = S::NX;
    extern __shared__ __align__(16) float sm[];
    const int DA = a.DA, ld = a.ld, nh = a.nh;
    const WarpActor w = stage_warp_actor(a.actor, DA, H, sm);
    float* adj = sm + warp_actor_floats(DA, H) + 64 * (threadIdx.x / LPE);  // dL/da_tau at (tau & 15)
    const int gl = threadIdx.x & (LPE - 1);
    int e;
    bool live, warp_live;
    grp_env<LPE, WV>(a.n, e, live, warp_live);
    const int t0 = g * a.ckpt, t1 = min(a.H, t0 + a.ckpt);
    const bool last = (t1 == a.H);
    // history adjoints carried over from the later segments (zero for the last one)
    for (int i = gl; i < 64; i += LPE) adj[i] = live ? a.la[(size_t)i * ld + e] : 0.0f;
    __syncthreads();
    if (!warp_live) return;  // warp-uniform
    const float seed = a.seed ? a.seed[e] : 1.0f;
    Prm P;
    load_vehicle_prm(a, e, P);
    const float d0[6] = {0, 0, 0, 0, 0, 0};
    const float half = 0.5f * (a.V.rpm_max - a.V.rpm_min);
    const size_t NR = (size_t)DA + 4 * H + 4;
    // Recompute the segment from its checkpoint: the states (RK4 with the rollout's stored
    // actions), and the actor's inputs and hidden activations at every step, which go
    // into the step's activation record (x | h1 | h2) for the reverse sweep and the weight
    // gradient.  Steps go SB at a time through the hidden layers, so that each weight read
    // from shared memory serves SB steps.
    float s[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = a.ck[(size_t)g * NS * ld + (size_t)i * ld + e];
    auto histA = [&](int tau, int c) { return a.A[((size_t)tau * 4 + c) * ld + e]; };
    for (int tb = t0; tb < t1; tb += SB) {
        float xb[SB][NX];
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            const int t = tb + q;
            if (t < t1) {
                float* ss = a.segs + (size_t)(t - t0) * NS * ld + e;
#pragma unroll
                for (int r = 0; r < (NS + LPE - 1) / LPE; ++r) {
                    const int i = gl + LPE * r;
                    const float v = pick<NS>(s, i);
                    if (live && i < NS) ss[(size_t)i * ld] = v;
                }
                grp_actor_input<LPE, NX>(s, t, DA, nh, histA, xb[q]);
                float u[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) u[c] = fmaf(a.A[((size_t)t * 4 + c) * ld + e] + 1.0f, half, a.V.rpm_min);
                rk4(a.V, a.dt, a.renorm, s, u, P, d0);
            } else {
#pragma unroll
                for (int m = 0; m < NX; ++m) xb[q][m] = 0.0f;
            }
        }
        float h1b[SB][HPL], h2b[SB][HPL];
        grp_actor_hidden_steps<H, LPE, SB>(w, DA, xb, h1b, h2b);
        if (live) {
#pragma unroll
            for (int q = 0; q < SB; ++q) {
                if (tb + q >= t1) break;
                float* R = a.rec + ((size_t)e * (t1 - t0) + (tb + q - t0)) * NR;
#pragma unroll
                for (int m = 0; m < NX; ++m)
                    if (gl + LPE * m < DA) R[gl + LPE * m] = xb[q][m];
#pragma unroll
                for (int j = 0; j < HPL; ++j) {
                    R[DA + gl + LPE * j] = h1b[q][j];
                    R[DA + H + gl + LPE * j] = h2b[q][j];
                }
            }
        }
    }
    __syncwarp();
    float lam[NS], gp[7];
    if (last) {
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] = 0.0f;
        state_loss_grad(a, s, lam);
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] *= seed;
#pragma unroll
        for (int i = 0; i < 7; ++i) gp[i] = 0.0f;
    } else {
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] = a.lam[i * ld + e];
#pragma unroll
        for (int i = 0; i < 7; ++i) gp[i] = a.gp[i * ld + e];
    }
    for (int t = t1 - 1; t >= t0; --t) {
        float st[NS];
        const float* ss = a.segs + (size_t)(t - t0) * NS * ld + e;
#pragma unroll
        for (int i = 0; i < NS; ++i) st[i] = ss[(size_t)i * ld];
        float act[4], u[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            act[c] = a.A[((size_t)t * 4 + c) * ld + e];
            u[c] = fmaf(act[c] + 1.0f, half, a.V.rpm_min);
        }
        float gs[NS], gu[4] = {0, 0, 0, 0};
        rk4_vjp(a.V, a.dt, a.renorm, st, u, P, lam, gs, gu, gp);
        float ga[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ga[c] = gu[c] * half + seed * 2.0f * a.w_a * act[c] + adj[(t & 15) * 4 + c];
        __syncwarp();
        if (gl < 4) adj[(t & 15) * 4 + gl] = 0.0f;  // slot now belongs to step t - 16
        // the actor at step t: its hidden activations from the step's record (written by
        // this lane in the recompute above; a group without an env reads env n - 1's), its
        // output mu = the stored action (the closed loop adds no noise)
        float* R = a.rec + ((size_t)e * (t1 - t0) + (t - t0)) * NR;
        float h1[HPL], h2[HPL];
#pragma unroll
        for (int j = 0; j < HPL; ++j) {
            h1[j] = R[DA + gl + LPE * j];
            h2[j] = R[DA + H + gl + LPE * j];
        }
        // reverse: output layer, layer 2, layer 1, inputs
        float dz3[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) dz3[c] = ga[c] * (1.0f - act[c] * act[c]);
        float dz2[HPL], dz1[HPL];
#pragma unroll
        for (int j = 0; j < HPL; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) acc = fmaf(w.W3[c * H + gl + LPE * j], dz3[c], acc);
            dz2[j] = h2[j] > 0.0f ? acc : 0.0f;
        }
        {
            float acc[HPL];
#pragma unroll
            for (int i = 0; i < HPL; ++i) acc[i] = 0.0f;
#pragma unroll
            for (int m = 0; m < HPL; ++m)
                for (int jj = 0; jj < LPE; jj += 4) {
                    float dj[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) dj[q] = __shfl_sync(0xffffffffu, dz2[m], jj + q, LPE);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float* wr = w.W2 + (LPE * m + jj + q) * w.l2 + gl;
#pragma unroll
                        for (int i = 0; i < HPL; ++i) acc[i] = fmaf(wr[LPE * i], dj[q], acc[i]);
                    }
                }
#pragma unroll
            for (int i = 0; i < HPL; ++i) dz1[i] = h1[i] > 0.0f ? acc[i] : 0.0f;
        }
        float dx[NX];
#pragma unroll
        for (int q = 0; q < NX; ++q) dx[q] = 0.0f;
#pragma unroll
        for (int m = 0; m < HPL; ++m)
            for (int jj = 0; jj < LPE; jj += 4) {
                float dj[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) dj[q] = __shfl_sync(0xffffffffu, dz1[m], jj + q, LPE);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float* wr = w.W1 + (LPE * m + jj + r) * w.l1 + gl;
#pragma unroll
                    for (int q = 0; q < NX; ++q)
                        if (gl + LPE * q < DA) dx[q] = fmaf(wr[LPE * q], dj[r], dx[q]);
                }
            }
        // observation part -> state adjoint (every lane), history part -> earlier actions
        float go[18];
#pragma unroll
        for (int k = 0; k < 18; ++k) go[k] = __shfl_sync(0xffffffffu, dx[k / LPE], k % LPE, LPE);
        obs_vjp(st, go, gs);
#pragma unroll
        for (int q = 0; q < NX; ++q) {
            const int k = gl + LPE * q;
            if (k >= 18 && k < DA) {
                const int i = ((k - 18) >> 2) + 1, c = (k - 18) & 3;
                if (t - i >= 0) adj[((t - i) & 15) * 4 + c] += dx[q];
            }
        }
        // the rest of the activation record of (step t, env e): x | h1 | h2 | dZ1 | dZ2 | dZ3,
        // env-major over the segment ([env][step][field]): a chunk of envs is one contiguous
        // run of rows
        if (live) {
#pragma unroll
            for (int j = 0; j < HPL; ++j) {
                R[DA + 2 * H + gl + LPE * j] = dz1[j];
                R[DA + 3 * H + gl + LPE * j] = dz2[j];
            }
            if (gl < 4) R[DA + 4 * H + gl] = pick<4>(dz3, gl);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < NS; ++i) lam[i] = gs[i];
        if (t >= 1) {
            float lg[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) lg[i] = 0.0f;
            state_loss_grad(a, st, lg);
#pragma unroll
            for (int i = 0; i < NS; ++i) lam[i] = fmaf(seed, lg[i], lam[i]);
        }
    }
    if (live) {
        if (gl == 0) {
#pragma unroll
            for (int i = 0; i < NS; ++i) a.lam[i * ld + e] = lam[i];
#pragma unroll
            for (int i = 0; i < 7; ++i) a.gp[i * ld + e] = gp[i];
            if (g == 0 && a.g_params)
#pragma unroll
                for (int i = 0; i < 4; ++i) a.g_params[i * ld + e] = gp[i];
        }
        for (int i = gl; i < 64; i += LPE) a.la[(size_t)i * ld + e] = adj[i];
    }
}

// Partial actor-weight gradient of segment g over env chunk blockIdx.x (closed loop).
// Records are field-major per step (fs = ld, es = 1: the thread-per-env kernels; one GEMM
// pass per step) or env-major over the whole segment (fs = 1, es = NR: the lane-group
// kernels; the chunk's env x step rows are contiguous, one GEMM pass over all of them).
__global__ void __launch_bounds__(LT) k_vjp_wgrad(VjpArgs a, int g, int fs, int es) {
    extern __shared__ __align__(16) float sm[];
    const int ld = a.ld, DA = a.DA, H = a.hid;
    const int t0 = g * a.ckpt, t1 = min(a.H, t0 + a.ckpt);
    const int e0 = blockIdx.x * a.chunk;
    const int ne = min(a.chunk, a.n - e0);
    if (ne <= 0) return;
    const size_t NR = (size_t)DA + 4 * H + 4;
    // the chunk's partial gradient accumulates in shared memory over the segment's steps and
    // is written out once
    float* P = sm + GEMM_SMEM;
    float* gW1 = P;
    float* gb1 = gW1 + H * DA;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + 4 * H;
    const bool seg_rows = fs == 1;  // env-major over the segment
    const int steps = seg_rows ? 1 : t1 - t0;
    const int nk = seg_rows ? ne * (t1 - t0) : ne;  // reduction rows per pass
    for (int t = t0; t < t0 + steps; ++t) {
        const float* R = seg_rows ? a.rec + (size_t)e0 * (t1 - t0) * NR
                                  : a.rec + (size_t)(t - t0) * NR * ld + (size_t)e0 * es;
        const float* O = R;
        const float* H1 = R + (size_t)DA * fs;
        const float* H2 = H1 + (size_t)H * fs;
        const float* dZ1 = H2 + (size_t)H * fs;
        const float* dZ2 = dZ1 + (size_t)H * fs;
        const float* dZ3 = dZ2 + (size_t)H * fs;
        const bool first = (t == t0);
        cta_gemm(H, DA, nk, Mat{dZ1, fs, es}, Mat{O, es, fs}, sm, [&](int m, int n, float v) {
            float* p = gW1 + m * DA + n;
            *p = first ? v : *p + v;
        });
        cta_gemm(H, H, nk, Mat{dZ2, fs, es}, Mat{H1, es, fs}, sm, [&](int m, int n, float v) {
            float* p = gW2 + m * H + n;
            *p = first ? v : *p + v;
        });
        cta_gemm(4, H, nk, Mat{dZ3, fs, es}, Mat{H2, es, fs}, sm, [&](int m, int n, float v) {
            float* p = gW3 + m * H + n;
            *p = first ? v : *p + v;
        });
        for (int j = threadIdx.x; j < 2 * H + 4; j += LT) {
            const float* src = j < H ? dZ1 + (size_t)j * fs : (j < 2 * H ? dZ2 + (size_t)(j - H) * fs
                                                                         : dZ3 + (size_t)(j - 2 * H) * fs);
            float* dst = j < H ? gb1 + j : (j < 2 * H ? gb2 + (j - H) : gb3 + (j - 2 * H));
            // 8 loads in flight per thread, 8 running sums added in a fixed order
            float acc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            int q = 0;
            for (; q + 8 <= nk; q += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = ldcg(src + (size_t)(q + u) * es);
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] += v[u];
            }
            for (; q < nk; ++q) acc[0] += ldcg(src + (size_t)q * es);
            const float s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
            *dst = first ? s : *dst + s;
        }
        __syncthreads();
    }
    float* out = a.part + (size_t)blockIdx.x * a.PA;
    for (int i = threadIdx.x; i < a.PA; i += LT) out[i] = P[i];
}

// Actor-weight gradient of segment g over env chunk blockIdx.x from the lane-group kernels'
// env-major records: the chunk's env x step rows are contiguous, NR floats each
// [x (DA) | h1 | h2 | dz1 | dz2 | dz3 (4)].  The rows stream through shared memory in blocks
// of WB (cp.async, double-buffered) and every thread keeps its outputs in registers over
// its rows: dW1 = dz1^T x and dW2 = dz2^T h1 on an (H/4) x TN thread grid (4 rows x J
// columns each, columns tn + TN j), dW3 = dz3^T h2 one element per thread, and the bias
// sums; each element sums its rows in order (deterministic).  Two CTAs share a chunk (the
// first and second half of its rows, split at a multiple of WB), each writing its own
// partial: twice the CTAs of the chunk count, so that every SM has work.
template <int H>
__global__ void __launch_bounds__(LT) k_vjp_wgrad_rows(VjpArgs a, int g) {
    constexpr int MT = H / 4, TN = LT / MT, J1 = (96 + TN - 1) / TN, J2 = H / TN, WB = 32;
    static_assert(MT * TN == LT && J2 * TN == H, "thread grid");
    extern __shared__ __align__(16) float sm[];
    const int DA = a.DA, NR = DA + 4 * H + 4;
    const int t0 = g * a.ckpt, t1 = min(a.H, t0 + a.ckpt);
    const int e0 = (blockIdx.x >> 1) * a.chunk, half = blockIdx.x & 1;
    const int ne = min(a.chunk, a.n - e0);
    if (ne <= 0) return;
    const int nrow_all = ne * (t1 - t0);
    const int split = ((nrow_all / 2 + WB - 1) / WB) * WB;
    const int rbeg = half ? min(split, nrow_all) : 0, nrow = half ? nrow_all - rbeg : min(split, nrow_all);
    const int nblk = (nrow + WB - 1) / WB;
    // 16-byte aligned: the records start aligned and a chunk, half or block offset is a
    // multiple of 32 rows of NR floats (128 NR bytes)
    const float* base = a.rec + ((size_t)e0 * (t1 - t0) + rbeg) * NR;
    const int tid = threadIdx.x, tm = tid / TN, tn = tid - tm * TN;
    auto issue = [&](int blk) {
        float* dst = sm + (size_t)(blk & 1) * WB * NR;
        const int r0 = blk * WB, n = min(WB, nrow - r0) * NR, n4 = n >> 2;
        const float* src = base + (size_t)r0 * NR;
        const uint32_t sd = (uint32_t)__cvta_generic_to_shared(dst);
        for (int v = tid; v < n4; v += LT)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(sd + 16u * (uint32_t)v),
                         "l"(src + 4 * v) : "memory");
        for (int i = 4 * n4 + tid; i < n; i += LT) dst[i] = ldcg(src + i);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float acc1[4][J1], acc2[4][J2], acc3 = 0.0f, accb = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < J1; ++j) acc1[i][j] = 0.0f;
#pragma unroll
        for (int j = 0; j < J2; ++j) acc2[i][j] = 0.0f;
    }
    // dW3 element (o3, j3) for tid < 4 H; bias element tid < 2 H + 4 (b1, b2, b3)
    const int o3 = tid / H, j3 = tid - o3 * H;
    const int boff = tid < H ? DA + 2 * H + tid : (tid < 2 * H ? DA + 3 * H + (tid - H) : DA + 4 * H + (tid - 2 * H));
    if (nblk > 0) issue(0);
    for (int blk = 0; blk < nblk; ++blk) {
        if (blk + 1 < nblk) {
            issue(blk + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float* Rb = sm + (size_t)(blk & 1) * WB * NR;
        const int nr = min(WB, nrow - blk * WB);
        for (int r = 0; r < nr; ++r) {
            const float* R = Rb + r * NR;
            const float* D1 = R + DA + 2 * H;
            const float* D2 = D1 + H;
            const float2 d1a = *reinterpret_cast<const float2*>(D1 + 4 * tm);
            const float2 d1b = *reinterpret_cast<const float2*>(D1 + 4 * tm + 2);
            const float2 d2a = *reinterpret_cast<const float2*>(D2 + 4 * tm);
            const float2 d2b = *reinterpret_cast<const float2*>(D2 + 4 * tm + 2);
            const float d1[4] = {d1a.x, d1a.y, d1b.x, d1b.y}, d2[4] = {d2a.x, d2a.y, d2b.x, d2b.y};
            float xv[J1], hv[J2];
#pragma unroll
            for (int j = 0; j < J1; ++j) xv[j] = R[min(tn + TN * j, DA - 1)];
#pragma unroll
            for (int j = 0; j < J2; ++j) hv[j] = R[DA + tn + TN * j];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int j = 0; j < J1; ++j) acc1[i][j] = fmaf(d1[i], xv[j], acc1[i][j]);
#pragma unroll
                for (int j = 0; j < J2; ++j) acc2[i][j] = fmaf(d2[i], hv[j], acc2[i][j]);
            }
            if (tid < 4 * H) acc3 = fmaf(R[DA + 4 * H + o3], R[DA + H + j3], acc3);
            if (tid < 2 * H + 4) accb += R[boff];
        }
        __syncthreads();  // the buffer is refilled two blocks later
    }
    float* out = a.part + (size_t)blockIdx.x * a.PA;
    float* oW1 = out;
    float* ob1 = oW1 + H * DA;
    float* oW2 = ob1 + H;
    float* ob2 = oW2 + H * H;
    float* oW3 = ob2 + H;
    float* ob3 = oW3 + 4 * H;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = 4 * tm + i;
#pragma unroll
        for (int j = 0; j < J1; ++j)
            if (tn + TN * j < DA) oW1[m * DA + tn + TN * j] = acc1[i][j];
#pragma unroll
        for (int j = 0; j < J2; ++j) oW2[m * H + tn + TN * j] = acc2[i][j];
    }
    if (tid < 4 * H) oW3[o3 * H + j3] = acc3;
    if (tid < H) ob1[tid] = accb;
    else if (tid < 2 * H) ob2[tid - H] = accb;
    else if (tid < 2 * H + 4) ob3[tid - 2 * H] = accb;
}

// g_actor += sum over the partials (fixed order): a CTA takes 32 parameters; warp w sums
// partials w, w + 8, ... (coalesced over the parameters), then the 8 warp sums are added
// in order.
__global__ void __launch_bounds__(256) k_vjp_wreduce(VjpArgs a) {
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    float s = 0.0f;
    if (p < a.PA) {
#pragma unroll 4
        for (int c = w; c < a.npart; c += 8) s += a.part[(size_t)c * a.PA + p];
    }
    red[w][lane] = s;
    __syncthreads();
    if (w != 0 || p >= a.PA) return;
    s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += red[k][lane];
    a.g_actor[p] += s;
}

static size_t align_up(size_t x) { return (x + 63) & ~(size_t)63; }

struct WsLayout {
    size_t ck, A, la, segs, lam, gp, rec, fo, part, total;
};

static WsLayout ws_layout(const qsim_vjp_desc& d, int DA, int PA, int nchunk) {
    WsLayout w;
    const size_t ld = d.ld, nseg = (d.H + d.ckpt - 1) / d.ckpt;
    size_t off = 0;
    auto take = [&](size_t floats) { size_t o = off; off += align_up(floats); return o; };
    w.ck = take(nseg * NS * ld);
    w.A = take((size_t)d.H * 4 * ld);
    w.la = take(d.mode == 1 ? (size_t)std::max(d.H, 16) * 4 * ld : 0);  // >= the warp path's 64-float ring
    w.segs = take((size_t)d.ckpt * NS * ld);
    w.lam = take(NS * ld);
    w.gp = take(8 * ld);
    const size_t NR = (size_t)DA + 4 * (size_t)d.hidden + 4;
    // closed loop: the records of two segments (the weight gradient of one segment runs
    // while the next segment's reverse sweep writes the other half)
    w.rec = take(d.mode == 1 ? 2 * (size_t)d.ckpt * NR * ld : 0);
    w.fo = take(d.mode == 1 ? ((size_t)DA + 2 * (size_t)d.hidden) * ld : 0);
    w.part = take(d.mode == 1 ? 2 * (size_t)nchunk * PA : 0);  // up to two partials per chunk
    w.total = off;
    return w;
}

// The calling host thread's side stream on one device (lowest priority, so that the block
// scheduler prefers the reverse sweep's blocks) and its fork / join events, created on the
// first closed-loop gradient call and kept for the thread's life.  The weight gradient of
// segment g runs there while segment g - 1's reverse sweep runs on the caller's stream.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork[2] = {nullptr, nullptr}, join[2] = {nullptr, nullptr};
};

static SideStream* side_stream() {
    constexpr int kMaxDev = 16;
    thread_local SideStream side[kMaxDev];
    thread_local bool tried[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return nullptr;
    }
    SideStream& x = side[dev];
    if (!tried[dev]) {
        tried[dev] = true;
        int least = 0, greatest = 0;
        bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
                  cudaStreamCreateWithPriority(&x.s, cudaStreamNonBlocking, least) == cudaSuccess;
        for (int i = 0; ok && i < 2; ++i)
            ok = cudaEventCreateWithFlags(&x.fork[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&x.join[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            x.s = nullptr;  // the weight gradient then runs on the caller's stream
        }
    }
    return x.s ? &x : nullptr;
}

static constexpr int kChunk = 32;  // envs per weight-gradient CTA
static constexpr int kAutoLanesPerEnv = 8;  // lane-group width of the closed loop by default

// The lane-group kernels of one (hidden, lanes per env, warps per CTA) shape.
struct GrpKernels {
    void (*fw)(VjpArgs);
    void (*bw)(VjpArgs, int);
    int wv;
};

static GrpKernels grp_kernels(int hidden64, int lanes_index, bool wide) {
    static const GrpKernels tab[2][4] = {
        {{k_vjp_forward_w<32, 32, kWvSmall>, k_vjp_backward_w<32, 32, kWvSmall>, kWvSmall},
         {k_vjp_forward_w<32, 16, kWvSmall>, k_vjp_backward_w<32, 16, kWvSmall>, kWvSmall},
         {k_vjp_forward_w<32, 8, kWvSmall>, k_vjp_backward_w<32, 8, kWvSmall>, kWvSmall},
         {k_vjp_forward_w<32, 8, kWvWide>, k_vjp_backward_w<32, 8, kWvWide>, kWvWide}},
        {{k_vjp_forward_w<64, 32, kWvSmall>, k_vjp_backward_w<64, 32, kWvSmall>, kWvSmall},
         {k_vjp_forward_w<64, 16, kWvSmall>, k_vjp_backward_w<64, 16, kWvSmall>, kWvSmall},
         {k_vjp_forward_w<64, 8, kWvSmall>, k_vjp_backward_w<64, 8, kWvSmall>, kWvSmall},
         {k_vjp_forward_w<64, 8, kWvWide>, k_vjp_backward_w<64, 8, kWvWide>, kWvWide}}};
    return tab[hidden64][lanes_index == 2 && wide ? 3 : lanes_index];
}

// Whether the 7-warp CTAs leave fewer warps on the busiest SM than the 4-warp ones (two
// resident per SM) for n envs at lpe lanes per env: warps per SM ~ ceil(CTAs / SMs) x warps
// per CTA.
static bool lane_group_wide(int n, int lpe) {
    if (lpe != 8) return false;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else
            sms = 152;
    }
    const long warps = (n + 3) / 4;  // 4 envs per warp at 8 lanes per env
    auto busiest = [&](long wv) { return ((warps + wv - 1) / wv + sms - 1) / sms * wv; };
    return busiest(kWvWide) < busiest(kWvSmall);
}

}  // namespace qsim

using namespace qsim;

static qsim_status check_desc(const qsim_vjp_desc* d) {
    if (!d) return fail(QSIM_EINVAL, "qsim_rollout_vjp: null descriptor");
    if (d->n < 1 || d->ld < d->n || (d->ld & 3) || d->H < 1 || d->ckpt < 1 || d->mode < 0 ||
        d->mode > 1 || !(d->dt > 0.0f))
        return fail(QSIM_EINVAL, "qsim_rollout_vjp: bad sizes (n=%d ld=%d H=%d ckpt=%d mode=%d)",
                    d->n, d->ld, d->H, d->ckpt, d->mode);
    if (d->mode == 1 && (d->n_hist < 0 || d->n_hist > HMAX || d->hidden < 4 || d->hidden > 128))
        return fail(QSIM_EINVAL, "qsim_rollout_vjp: bad actor shape (n_hist=%d hidden=%d)", d->n_hist,
                    d->hidden);
    if (d->lanes_per_env != 0 && d->lanes_per_env != 8 && d->lanes_per_env != 16 && d->lanes_per_env != 32)
        return fail(QSIM_EINVAL, "qsim_rollout_vjp: lanes per env %d not 0, 8, 16 or 32", d->lanes_per_env);
    return QSIM_OK;
}

extern "C" size_t qsim_vjp_workspace(const qsim_vjp_desc* d) {
    if (check_desc(d) != QSIM_OK) return 0;
    const int DA = 18 + 4 * d->n_hist;
    const int PA = d->hidden * DA + d->hidden + d->hidden * d->hidden + d->hidden + 4 * d->hidden + 4;
    const int nchunk = (d->n + kChunk - 1) / kChunk;
    return ws_layout(*d, DA, PA, nchunk).total * sizeof(float);
}

extern "C" qsim_status qsim_rollout_vjp(const qsim_vjp_desc* d, const qsim_params* veh,
                                        const float* s0, const float* params, const float* actions,
                                        const float* actor, const float* seed, float* loss,
                                        float* g_actions, float* g_actor, float* g_params,
                                        float* actions_out, void* workspace, void* stream) {
    qsim_status st = check_desc(d);
    if (st != QSIM_OK) return st;
    if (!veh || !s0 || !params || !workspace) return fail(QSIM_EINVAL, "qsim_rollout_vjp: null pointer");
    if (d->mode == 0 && !actions) return fail(QSIM_EINVAL, "qsim_rollout_vjp: open loop needs actions");
    if (d->mode == 1 && !actor) return fail(QSIM_EINVAL, "qsim_rollout_vjp: closed loop needs actor");
    if (!aligned16(s0) || !aligned16(params) || !aligned16(workspace))
        return fail(QSIM_EINVAL, "qsim_rollout_vjp: pointers must be 16-byte aligned");
    VjpArgs a;
    memset(&a, 0, sizeof(a));
    a.V = make_vehicle(*veh);
    a.n = d->n; a.ld = d->ld; a.H = d->H; a.ckpt = d->ckpt; a.mode = d->mode;
    a.nh = d->mode == 1 ? d->n_hist : 0;
    a.hid = d->hidden;
    a.DA = 18 + 4 * a.nh;
    a.PA = a.hid * a.DA + a.hid + a.hid * a.hid + a.hid + 4 * a.hid + 4;
    a.nseg = (d->H + d->ckpt - 1) / d->ckpt;
    a.chunk = kChunk;
    a.nchunk = (d->n + kChunk - 1) / kChunk;
    a.npart = a.nchunk;
    a.w_p = d->w_p; a.w_q = d->w_q; a.w_v = d->w_v; a.w_a = d->w_a; a.dt = d->dt;
    a.renorm = d->renorm;
    a.s0 = s0; a.prm = params; a.actions = actions; a.actor = actor; a.seed = seed;
    a.loss = loss; a.g_actions = g_actions; a.g_actor = g_actor; a.g_params = g_params;
    a.actions_out = actions_out;
    qsim_vjp_desc dd = *d;
    dd.n_hist = a.nh;
    const WsLayout w = ws_layout(dd, a.DA, a.PA, a.nchunk);
    float* base = static_cast<float*>(workspace);
    a.ck = base + w.ck; a.A = base + w.A; a.la = base + w.la; a.segs = base + w.segs;
    a.lam = base + w.lam; a.gp = base + w.gp; a.rec = base + w.rec; a.fo = base + w.fo;
    a.part = base + w.part;
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t smem = d->mode == 1 ? sizeof(float) * (size_t)a.PA : 0;
    if (smem > 48 * 1024) {
        QCHECK_CUDA(cudaFuncSetAttribute(k_vjp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        QCHECK_CUDA(cudaFuncSetAttribute(k_vjp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    const int grid = (d->n + VT - 1) / VT;
    // closed loop at hidden 32 / 64: one env per group of lpe lanes
    const bool warp_path = d->mode == 1 && (a.hid == 32 || a.hid == 64) && a.DA <= 96;
    const int lpe = d->lanes_per_env == 0 ? kAutoLanesPerEnv : d->lanes_per_env;
    const bool wide = warp_path && lane_group_wide(d->n, lpe);
    const int WV = wide ? kWvWide : kWvSmall;
    const int envs_per_cta = WV * (32 / lpe);
    const int gridw = (d->n + envs_per_cta - 1) / envs_per_cta;
    const size_t smem_fw = sizeof(float) * (size_t)(warp_actor_floats(a.DA, a.hid) + 64 * envs_per_cta);
    const size_t smem_bw = smem_fw;
    GrpKernels gk{};
    if (warp_path) {
        const int hi = a.hid == 64, li = lpe == 32 ? 0 : (lpe == 16 ? 1 : 2);
        gk = grp_kernels(hi, li, wide);
        static bool configured[2][4] = {};
        const int ci = li == 2 && wide ? 3 : li;
        if (!configured[hi][ci]) {
            QCHECK_CUDA(cudaFuncSetAttribute(gk.fw, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
            QCHECK_CUDA(cudaFuncSetAttribute(gk.bw, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
            configured[hi][ci] = true;
        }
        gk.fw<<<gridw, 32 * WV, smem_fw, cs>>>(a);
    } else {
        k_vjp_forward<<<grid, VT, smem, cs>>>(a);
    }
    QCHECK_LAUNCH("k_vjp_forward");
    const bool want_grad = g_actions || g_actor || g_params;
    if (!want_grad) return QSIM_OK;
    if (d->mode == 1) {
        QCHECK_CUDA(cudaMemsetAsync(a.la, 0, sizeof(float) * (size_t)std::max(d->H, 16) * 4 * d->ld, cs));
        if (g_actor) QCHECK_CUDA(cudaMemsetAsync(g_actor, 0, sizeof(float) * (size_t)a.PA, cs));
    }
    const int NR = a.DA + 4 * a.hid + 4;
    const size_t smem_wg = sizeof(float) * (size_t)(GEMM_SMEM + a.PA);
    // the lane-group path's row-streaming weight gradient: two blocks of 32 records
    const size_t smem_wr = sizeof(float) * 2 * 32 * (size_t)NR;
    if (d->mode == 1 && g_actor && warp_path) {
        static bool wr_configured[2] = {false, false};
        const int hi = a.hid == 64;
        if (!wr_configured[hi]) {
            QCHECK_CUDA(cudaFuncSetAttribute(hi ? k_vjp_wgrad_rows<64> : k_vjp_wgrad_rows<32>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 32 * (96 + 4 * 64 + 4) * 4));
            wr_configured[hi] = true;
        }
    }
    if (d->mode == 1 && g_actor) {
        static size_t wg_configured = 0;
        if (smem_wg > 48 * 1024 && smem_wg > wg_configured) {
            QCHECK_CUDA(cudaFuncSetAttribute(k_vjp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_wg));
            wg_configured = smem_wg;
        }
    }
    // Lane-group closed loop: segment g's records go to half (g & 1) of the record area,
    // and its weight gradient (+ the fixed-order reduction into g_actor) runs on the side
    // stream while segment g - 1's reverse sweep runs: it is submitted after that sweep,
    // so the sweep's blocks are queued first.  Segment g - 2 reuses the half once the
    // weight gradient is done; the last one (segment 0) runs on `stream` after the side
    // stream's, which joins the side stream back (also under stream capture).
    SideStream* side = (d->mode == 1 && g_actor && warp_path && a.nseg > 1) ? side_stream() : nullptr;
    const size_t rec_seg = (size_t)a.ckpt * NR * a.ld;
    auto weight_grad = [&](int g, cudaStream_t ws) -> qsim_status {
        VjpArgs ag = a;
        if (side) ag.rec = a.rec + (size_t)(g & 1) * rec_seg;
        if (warp_path) {
            ag.npart = 2 * a.nchunk;  // two CTAs (row halves) per chunk
            if (a.hid == 64) k_vjp_wgrad_rows<64><<<ag.npart, LT, smem_wr, ws>>>(ag, g);
            else k_vjp_wgrad_rows<32><<<ag.npart, LT, smem_wr, ws>>>(ag, g);
        } else {
            k_vjp_wgrad<<<a.nchunk, LT, smem_wg, ws>>>(ag, g, a.ld, 1);
        }
        QCHECK_LAUNCH("k_vjp_wgrad");
        k_vjp_wreduce<<<(a.PA + 31) / 32, 256, 0, ws>>>(ag);
        QCHECK_LAUNCH("k_vjp_wreduce");
        return QSIM_OK;
    };
    for (int g = a.nseg - 1; g >= 0; --g) {
        VjpArgs ag = a;
        if (side) {
            ag.rec = a.rec + (size_t)(g & 1) * rec_seg;
            if (g <= a.nseg - 3) QCHECK_CUDA(cudaStreamWaitEvent(cs, side->join[g & 1], 0));
        }
        if (warp_path) {
            gk.bw<<<gridw, 32 * WV, smem_bw, cs>>>(ag, g);
        } else {
            k_vjp_backward<<<grid, VT, smem, cs>>>(ag, g);
        }
        QCHECK_LAUNCH("k_vjp_backward");
        if (d->mode == 1 && g_actor) {
            if (side) {
                QCHECK_CUDA(cudaEventRecord(side->fork[g & 1], cs));
                if (g + 1 < a.nseg) {  // segment g + 1's weight gradient, behind sweep g
                    QCHECK_CUDA(cudaStreamWaitEvent(side->s, side->fork[(g + 1) & 1], 0));
                    qsim_status st2 = weight_grad(g + 1, side->s);
                    if (st2 != QSIM_OK) return st2;
                    QCHECK_CUDA(cudaEventRecord(side->join[(g + 1) & 1], side->s));
                }
                if (g == 0) {
                    QCHECK_CUDA(cudaStreamWaitEvent(cs, side->join[1], 0));
                    qsim_status st2 = weight_grad(0, cs);
                    if (st2 != QSIM_OK) return st2;
                }
            } else {
                qsim_status st2 = weight_grad(g, cs);
                if (st2 != QSIM_OK) return st2;
            }
        }
    }
    return QSIM_OK;
}
