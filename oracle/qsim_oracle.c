/*
 * qsim_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the header).
 *
 * Citations name the paper's section / equation; "TD3" is Fujimoto, van Hoof & Meger,
 * ICML 2018 (cited by the paper for its RL algorithm); "Adam" is Kingma & Ba, ICLR 2015;
 * "Philox" is Salmon, Moraes, Dror & Shaw, SC'11 ("Parallel Random Numbers: As Easy as
 * 1, 2, 3").  Where the paper leaves a choice open, the reading taken is named inline.
 */
#include "qsim_oracle.h"
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11, Sec. 4): ten rounds of two 32x32->64 multiplies   */
/* with a Weyl-sequence key schedule.                                                    */
/* ------------------------------------------------------------------------------------ */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;  /* golden ratio */
            k1 += 0xBB67AE85u;  /* sqrt(3) - 1 */
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in the open interval (0,1) from the top 23 bits: ((x >> 9) + 1/2) * 2^-23. */
double or_uniform(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box & Muller (1958), cosine branch only: one normal from one pair of uniforms. */
double or_gauss(uint32_t x1, uint32_t x2) {
    double u1 = or_uniform(x1), u2 = or_uniform(x2);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Replay index: floor(x * n / 2^32), exact in 64-bit integers. */
uint32_t or_replay_index(uint32_t x, uint32_t n) {
    return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
}

/* Counter layout shared by every random draw: (c0, c1, tag<<24 | sub, run); key = seed. */
static void draw(const or_cfg* c, uint32_t c0, uint32_t c1, uint32_t tag, uint32_t sub,
                 uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, (tag << 24) | sub, c->run_id};
    uint32_t key[2] = {(uint32_t)(c->seed & 0xffffffffu), (uint32_t)(c->seed >> 32)};
    or_philox(ctr, key, out);
}

enum { TAG_RESET = 0, TAG_DR = 1, TAG_OBS = 2, TAG_EXPL = 3, TAG_REPLAY = 4, TAG_SMOOTH = 5,
       TAG_DIST = 6, TAG_INIT = 7, TAG_WARM = 8 };

/* ------------------------------------------------------------------------------------ */
/* Dimensions                                                                           */
/* ------------------------------------------------------------------------------------ */
int or_net_size(int in, int hid, int out) { return hid * in + hid + hid * hid + hid + out * hid + out; }

/* Actor observation o_a = {p, R, v, omega, H}: 18 + 4 N_H (Sec. IV). */
int or_actor_in(const or_cfg* c) { return 18 + 4 * c->n_hist; }

static int critic_obs_dim(const or_cfg* c) {
    if (c->critic_layout == OR_CRITIC_PAPER28) return 28;      /* {p,R,v,w,w_m,f_r,tau_r} */
    if (c->critic_layout == OR_CRITIC_PRIV) return or_actor_in(c) + 4 + OR_NPRIV;
    if (c->critic_layout == OR_CRITIC_ACTOR) return or_actor_in(c);  /* symmetric critic */
    return or_actor_in(c) + 4;                                  /* actor obs + motor speeds */
}
/* The critic sees its observation followed by the action (Q(o_c, a)). */
int or_critic_in(const or_cfg* c) { return critic_obs_dim(c) + 4; }

/* PyTorch-style default initialisation: W, b ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)). */
void or_init_params(const or_cfg* c, int net_id, int in, int hid, int out, double* P) {
    int sizes[6] = {hid * in, hid, hid * hid, hid, out * hid, out};
    int fan[6] = {in, in, hid, hid, hid, hid};
    int i = 0;
    for (int blk = 0; blk < 6; ++blk) {
        double bound = 1.0 / sqrt((double)fan[blk]);
        for (int k = 0; k < sizes[blk]; ++k, ++i) {
            uint32_t r[4];
            draw(c, (uint32_t)i >> 2, (uint32_t)net_id, TAG_INIT, 0, r);
            P[i] = bound * (2.0 * or_uniform(r[i & 3]) - 1.0);
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Rigid-body multirotor dynamics with first-order motor lag (Sec. IV, "standard        */
/* dynamics of a quadrotor subject to motor delays").  Reading: world z up; q=(w,x,y,z)  */
/* rotates body to world; omega in the body frame; thrust k_f w_m^2 along body z; yaw   */
/* torque dir_i * k_m * f_i; motor lag d(w_m)/dt = (u - w_m)/T_m with u clipped to the   */
/* RPM range.                                                                           */
/* ------------------------------------------------------------------------------------ */
static void quat_rot(const double* q, double* R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

void or_deriv(const or_cfg* c, const double* s, const double* u, const double* prm,
              const double* dist, double* ds) {
    const double m = prm[0], J[3] = {prm[1], prm[2], prm[3]}, kf = prm[4], km = prm[5],
                 tm = prm[6];
    const double* q = s + 3;
    const double* v = s + 7;
    const double* w = s + 10;
    const double* wm = s + 13;
    double F = 0.0, tau[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 4; ++i) {
        double f = kf * wm[i] * wm[i];
        const double* r = c->rotor_pos + 3 * i;
        /* r x (0,0,f) = (r_y f, -r_x f, 0) */
        tau[0] += r[1] * f;
        tau[1] += -r[0] * f;
        tau[2] += c->rotor_dir[i] * km * f;
        F += f;
    }
    for (int k = 0; k < 3; ++k) tau[k] += dist[3 + k];
    double R[9];
    quat_rot(q, R);
    /* p' = v */
    for (int k = 0; k < 3; ++k) ds[k] = v[k];
    /* v' = R (0,0,F)/m + f_r/m - g e_z */
    for (int k = 0; k < 3; ++k) ds[7 + k] = R[3 * k + 2] * F / m + dist[k] / m;
    ds[9] -= c->g;
    /* q' = 1/2 q (x) (0, omega) */
    ds[3] = 0.5 * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
    ds[4] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    ds[5] = 0.5 * (q[0] * w[1] - q[1] * w[2] + q[3] * w[0]);
    ds[6] = 0.5 * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
    /* omega' = J^-1 (tau - omega x J omega) */
    double Jw[3] = {J[0] * w[0], J[1] * w[1], J[2] * w[2]};
    double cr[3] = {w[1] * Jw[2] - w[2] * Jw[1], w[2] * Jw[0] - w[0] * Jw[2],
                    w[0] * Jw[1] - w[1] * Jw[0]};
    for (int k = 0; k < 3; ++k) ds[10 + k] = (tau[k] - cr[k]) / J[k];
    /* omega_m' = (u - omega_m) / T_m */
    for (int i = 0; i < 4; ++i)
        ds[13 + i] = (clampd(u[i], c->rpm_min, c->rpm_max) - wm[i]) / tm;
}

/* Classic fourth-order Runge-Kutta over the 17-vector with the set-point held over dt,
 * then (reading) renormalisation of the quaternion; stage states are not renormalised. */
void or_rk4(const or_cfg* c, const double* s, const double* u, const double* prm,
            const double* dist, double dt, int renorm, double* out) {
    double k1[OR_NS], k2[OR_NS], k3[OR_NS], k4[OR_NS], y[OR_NS];
    or_deriv(c, s, u, prm, dist, k1);
    for (int i = 0; i < OR_NS; ++i) y[i] = s[i] + 0.5 * dt * k1[i];
    or_deriv(c, y, u, prm, dist, k2);
    for (int i = 0; i < OR_NS; ++i) y[i] = s[i] + 0.5 * dt * k2[i];
    or_deriv(c, y, u, prm, dist, k3);
    for (int i = 0; i < OR_NS; ++i) y[i] = s[i] + dt * k3[i];
    or_deriv(c, y, u, prm, dist, k4);
    for (int i = 0; i < OR_NS; ++i)
        out[i] = s[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    if (renorm) {
        double n = sqrt(out[3] * out[3] + out[4] * out[4] + out[5] * out[5] + out[6] * out[6]);
        for (int i = 3; i < 7; ++i) out[i] /= n;
    }
}

/* n independent envs ([n][17] etc.) stepped n_steps times with a held set-point. */
void or_dynamics_batch(const or_cfg* c, int n, const double* s, const double* u,
                       const double* prm, const double* dist, double dt, int renorm,
                       int n_steps, double* out) {
    for (int e = 0; e < n; ++e) {
        double cur[OR_NS], nxt[OR_NS];
        memcpy(cur, s + OR_NS * e, sizeof(cur));
        for (int t = 0; t < n_steps; ++t) {
            or_rk4(c, cur, u + 4 * e, prm + OR_NPRM * e, dist + OR_NDIST * e, dt, renorm, nxt);
            memcpy(cur, nxt, sizeof(cur));
        }
        memcpy(out + OR_NS * e, cur, sizeof(cur));
    }
}

/* ------------------------------------------------------------------------------------ */
/* Initial-state distribution + domain randomisation + disturbances (Sec. IV: diverse    */
/* positions, orientations, velocities, rotor speeds; f_r, tau_r sampled per episode).  */
/* ------------------------------------------------------------------------------------ */
static void quat_mul(const double* a, const double* b, double* o) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

void or_reset_env(const or_cfg* c, uint32_t env, uint32_t episode, double* s, double* prm,
                  double* dist) {
    double U[16];
    for (int sub = 0; sub < 4; ++sub) {
        uint32_t r[4];
        draw(c, env, episode, TAG_RESET, (uint32_t)sub, r);
        for (int k = 0; k < 4; ++k) U[4 * sub + k] = or_uniform(r[k]);
    }
    for (int k = 0; k < 3; ++k) s[k] = c->init_p * (2.0 * U[k] - 1.0);
    /* attitude: roll, pitch, yaw uniform, composed q = q_z(yaw) q_y(pitch) q_x(roll) */
    double roll = c->init_att * (2.0 * U[3] - 1.0);
    double pitch = c->init_att * (2.0 * U[4] - 1.0);
    double yaw = c->init_att * (2.0 * U[5] - 1.0);
    double qx[4] = {cos(0.5 * roll), sin(0.5 * roll), 0, 0};
    double qy[4] = {cos(0.5 * pitch), 0, sin(0.5 * pitch), 0};
    double qz[4] = {cos(0.5 * yaw), 0, 0, sin(0.5 * yaw)};
    double t1[4];
    quat_mul(qz, qy, t1);
    quat_mul(t1, qx, s + 3);
    for (int k = 0; k < 3; ++k) s[7 + k] = c->init_v * (2.0 * U[6 + k] - 1.0);
    for (int k = 0; k < 3; ++k) s[10 + k] = c->init_w * (2.0 * U[9 + k] - 1.0);
    for (int i = 0; i < 4; ++i)
        s[13 + i] = c->init_rpm_lo + (c->init_rpm_hi - c->init_rpm_lo) * U[12 + i];

    double D[8];
    for (int sub = 0; sub < 2; ++sub) {
        uint32_t r[4];
        draw(c, env, episode, TAG_DR, (uint32_t)sub, r);
        for (int k = 0; k < 4; ++k) D[4 * sub + k] = or_uniform(r[k]);
    }
    prm[0] = c->mass * (1.0 + c->dr_mass * (2.0 * D[0] - 1.0));
    prm[1] = c->Jx * (1.0 + c->dr_J * (2.0 * D[1] - 1.0));
    prm[2] = c->Jy * (1.0 + c->dr_J * (2.0 * D[2] - 1.0));
    prm[3] = c->Jz * (1.0 + c->dr_J * (2.0 * D[3] - 1.0));
    prm[4] = c->kf * (1.0 + c->dr_kf * (2.0 * D[4] - 1.0));
    prm[5] = c->km;
    prm[6] = c->tm_lo + (c->tm_hi - c->tm_lo) * D[5];
    prm[7] = 0.0;

    double X[8];
    for (int sub = 0; sub < 2; ++sub) {
        uint32_t r[4];
        draw(c, env, episode, TAG_DIST, (uint32_t)sub, r);
        for (int k = 0; k < 4; ++k) X[4 * sub + k] = or_uniform(r[k]);
    }
    for (int k = 0; k < 3; ++k) dist[k] = c->dist_f * (2.0 * X[k] - 1.0);
    for (int k = 0; k < 3; ++k) dist[3 + k] = c->dist_tau * (2.0 * X[3 + k] - 1.0);
}

/* ------------------------------------------------------------------------------------ */
/* Observations (Sec. IV): actor o_a = {p, R, v, omega, H} (+ Gaussian noise on the      */
/* first 18 entries); critic: privileged, noise-free.                                    */
/* ------------------------------------------------------------------------------------ */
void or_obs_noise(const or_cfg* c, uint32_t env, uint64_t t, double* noise) {
    for (int k = 0; k < 18; ++k) {
        uint32_t r[4];
        draw(c, env, (uint32_t)t, TAG_OBS, (uint32_t)(k / 2), r);
        double z = (k & 1) ? or_gauss(r[2], r[3]) : or_gauss(r[0], r[1]);
        double sig = k < 3 ? c->sig_p : (k < 12 ? c->sig_R : (k < 15 ? c->sig_v : c->sig_w));
        noise[k] = sig * z;
    }
}

void or_obs_actor(const or_cfg* c, const double* s, const double* hist, const double* noise,
                  double* o) {
    double R[9];
    quat_rot(s + 3, R);
    for (int k = 0; k < 3; ++k) o[k] = s[k];
    for (int k = 0; k < 9; ++k) o[3 + k] = R[k];
    for (int k = 0; k < 3; ++k) o[12 + k] = s[7 + k];
    for (int k = 0; k < 3; ++k) o[15 + k] = s[10 + k];
    for (int k = 0; k < 4 * c->n_hist; ++k) o[18 + k] = hist[k];
    if (noise)
        for (int k = 0; k < 18; ++k) o[k] += noise[k];
}

/* Privileged extras stored with each transition: true parameters relative to nominal
 * (PRIV layout) or the per-episode disturbances scaled to [-1,1] (28-D layout). */
void or_priv(const or_cfg* c, const double* prm, const double* dist, double* priv) {
    if (c->critic_layout == OR_CRITIC_PAPER28) {
        for (int k = 0; k < 3; ++k) priv[k] = c->dist_f > 0 ? dist[k] / c->dist_f : 0.0;
        for (int k = 0; k < 3; ++k) priv[3 + k] = c->dist_tau > 0 ? dist[3 + k] / c->dist_tau : 0.0;
    } else {
        priv[0] = prm[0] / c->mass - 1.0;
        priv[1] = prm[1] / c->Jx - 1.0;
        priv[2] = prm[2] / c->Jy - 1.0;
        priv[3] = prm[3] / c->Jz - 1.0;
        priv[4] = prm[4] / c->kf - 1.0;
        priv[5] = prm[6] / c->tm - 1.0;
    }
}

static double rpm_norm(const or_cfg* c, double w) {
    return 2.0 * (w - c->rpm_min) / (c->rpm_max - c->rpm_min) - 1.0;
}

void or_obs_critic(const or_cfg* c, const double* s, const double* hist, const double* priv,
                   double* o) {
    if (c->critic_layout == OR_CRITIC_PAPER28) {
        double R[9];
        quat_rot(s + 3, R);
        for (int k = 0; k < 3; ++k) o[k] = s[k];
        for (int k = 0; k < 9; ++k) o[3 + k] = R[k];
        for (int k = 0; k < 3; ++k) o[12 + k] = s[7 + k];
        for (int k = 0; k < 3; ++k) o[15 + k] = s[10 + k];
        for (int i = 0; i < 4; ++i) o[18 + i] = rpm_norm(c, s[13 + i]);
        for (int k = 0; k < 6; ++k) o[22 + k] = priv[k];
        return;
    }
    int da = or_actor_in(c);
    or_obs_actor(c, s, hist, NULL, o);
    if (c->critic_layout == OR_CRITIC_ACTOR) return; /* symmetric: the actor's observation */
    for (int i = 0; i < 4; ++i) o[da + i] = rpm_norm(c, s[13 + i]);
    if (c->critic_layout == OR_CRITIC_PRIV)
        for (int k = 0; k < OR_NPRIV; ++k) o[da + 4 + k] = priv[k];
}

/* ------------------------------------------------------------------------------------ */
/* Reward (Sec. IV): r = -C_rp|p|^2 - C_rq(1-q_w^2) - C_rv|v|^2 - C_rw|w|^2             */
/*                       - C_ra|a - C_rab|^2 + C_rs, evaluated on s' (reading).          */
/* A non-finite s' earns 0 (reading: the transition terminates).                        */
/* ------------------------------------------------------------------------------------ */
static int finite_state(const double* s) {
    for (int i = 0; i < OR_NS; ++i)
        if (!isfinite(s[i])) return 0;
    return 1;
}

double or_reward(const or_reward_c* C, const double* s, const double* a) {
    if (!finite_state(s)) return 0.0;
    double p2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
    double v2 = s[7] * s[7] + s[8] * s[8] + s[9] * s[9];
    double w2 = s[10] * s[10] + s[11] * s[11] + s[12] * s[12];
    double a2 = 0.0;
    for (int i = 0; i < 4; ++i) a2 += (a[i] - C->c[5]) * (a[i] - C->c[5]);
    return -C->c[0] * p2 - C->c[1] * (1.0 - s[3] * s[3]) - C->c[2] * v2 - C->c[3] * w2 -
           C->c[4] * a2 + C->c[6];
}

/* ------------------------------------------------------------------------------------ */
/* Multilayer perceptrons: in -> hid (ReLU) -> hid (ReLU) -> out (tanh or linear).      */
/* Parameter layout W1[hid][in] b1 W2[hid][hid] b2 W3[out][hid] b3.                     */
/* ------------------------------------------------------------------------------------ */
void or_mlp_forward(const or_net* net, const double* P, const double* x, double* h1,
                    double* h2, double* y, int tanh_out) {
    int in = net->in, hid = net->hid, out = net->out;
    const double *W1 = P, *b1 = W1 + hid * in, *W2 = b1 + hid, *b2 = W2 + hid * hid,
                 *W3 = b2 + hid, *b3 = W3 + out * hid;
    for (int j = 0; j < hid; ++j) {
        double acc = b1[j];
        for (int k = 0; k < in; ++k) acc += W1[j * in + k] * x[k];
        h1[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int j = 0; j < hid; ++j) {
        double acc = b2[j];
        for (int k = 0; k < hid; ++k) acc += W2[j * hid + k] * h1[k];
        h2[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int j = 0; j < out; ++j) {
        double acc = b3[j];
        for (int k = 0; k < hid; ++k) acc += W3[j * hid + k] * h2[k];
        y[j] = tanh_out ? tanh(acc) : acc;
    }
}

/* Reverse mode through the MLP; dy is dLoss/dy (post output activation).  Parameter
 * gradients are ADDED into dP; dx (if non-NULL) receives dLoss/dx. */
static void mlp_backward(const or_net* net, const double* P, const double* x, const double* h1,
                         const double* h2, const double* y, const double* dy, int tanh_out,
                         double* dP, double* dx) {
    int in = net->in, hid = net->hid, out = net->out;
    const double *W1 = P, *b1 = W1 + hid * in, *W2 = b1 + hid, *b2 = W2 + hid * hid,
                 *W3 = b2 + hid;
    (void)b1; (void)b2;
    double *dW1 = dP, *db1 = dW1 + hid * in, *dW2 = db1 + hid, *db2 = dW2 + hid * hid,
           *dW3 = db2 + hid, *db3 = dW3 + out * hid;
    double* dz3 = (double*)malloc(sizeof(double) * (size_t)out);
    double* dz2 = (double*)malloc(sizeof(double) * (size_t)hid);
    double* dz1 = (double*)malloc(sizeof(double) * (size_t)hid);
    for (int j = 0; j < out; ++j) dz3[j] = tanh_out ? dy[j] * (1.0 - y[j] * y[j]) : dy[j];
    for (int j = 0; j < out; ++j) {
        for (int k = 0; k < hid; ++k) dW3[j * hid + k] += dz3[j] * h2[k];
        db3[j] += dz3[j];
    }
    for (int k = 0; k < hid; ++k) {
        double acc = 0.0;
        for (int j = 0; j < out; ++j) acc += W3[j * hid + k] * dz3[j];
        dz2[k] = h2[k] > 0.0 ? acc : 0.0;
    }
    for (int j = 0; j < hid; ++j) {
        for (int k = 0; k < hid; ++k) dW2[j * hid + k] += dz2[j] * h1[k];
        db2[j] += dz2[j];
    }
    for (int k = 0; k < hid; ++k) {
        double acc = 0.0;
        for (int j = 0; j < hid; ++j) acc += W2[j * hid + k] * dz2[j];
        dz1[k] = h1[k] > 0.0 ? acc : 0.0;
    }
    for (int j = 0; j < hid; ++j) {
        for (int k = 0; k < in; ++k) dW1[j * in + k] += dz1[j] * x[k];
        db1[j] += dz1[j];
    }
    if (dx) {
        for (int k = 0; k < in; ++k) {
            double acc = 0.0;
            for (int j = 0; j < hid; ++j) acc += W1[j * in + k] * dz1[j];
            dx[k] = acc;
        }
    }
    free(dz3); free(dz2); free(dz1);
}

/* ------------------------------------------------------------------------------------ */
/* Environment step (Sec. IV + Sec. V "Training"): observation -> actor -> exploration   */
/* -> RPM set-point -> RK4 -> reward -> termination -> transition record -> history ->  */
/* reset when the episode ended.                                                        */
/* ------------------------------------------------------------------------------------ */
/* One env step of the dynamics at set-point u.  With the motor model ablated (Sec. VI,
 * "rotor delay" removed) the rotors run at the clipped set-point from the start of the
 * step, so the lag term of the motor equation is zero throughout. */
static void step_dynamics(const or_cfg* c, const double* s, const double* u, const double* prm,
                          const double* dist, double* s2) {
    double sm[OR_NS];
    memcpy(sm, s, sizeof(sm));
    if (c->motor_lag_off)
        for (int i = 0; i < 4; ++i) sm[13 + i] = clampd(u[i], c->rpm_min, c->rpm_max);
    or_rk4(c, sm, u, prm, dist, c->dt, c->renorm_q, s2);
}

typedef struct roll_job {
    const or_cfg* c;
    const or_reward_c* C;
    or_envs* e;
    const double* actor;
    int hidden, T, k0, k1;
    uint64_t t0;
    double sigma_e;
    const double* ext;
    or_roll_out* out;
} roll_job;

static void env_reset_local(const or_cfg* c, or_envs* e, int k) {
    or_reset_env(c, e->env_id[k], e->ep_index[k], e->s + OR_NS * k, e->prm + OR_NPRM * k,
                 e->dist + OR_NDIST * k);
    memset(e->hist + 4 * OR_HMAX * k, 0, sizeof(double) * 4 * OR_HMAX);
    e->ep_step[k] = 0;
    e->ep_ret[k] = 0.0;
}

static void roll_env(const roll_job* J, int k) {
    const or_cfg* c = J->c;
    or_envs* e = J->e;
    int n = e->n, da = or_actor_in(c);
    uint32_t env = e->env_id[k];
    double* s = e->s + OR_NS * k;
    double* prm = e->prm + OR_NPRM * k;
    double* dist = e->dist + OR_NDIST * k;
    double* hist = e->hist + 4 * OR_HMAX * k;
    or_net actor = {da, J->hidden, 4};
    double* h1 = (double*)malloc(sizeof(double) * (size_t)J->hidden * 2);
    double* h2 = h1 + J->hidden;
    for (int tt = 0; tt < J->T; ++tt) {
        uint64_t t = J->t0 + (uint64_t)tt;
        double a[4], mu[4] = {0, 0, 0, 0};
        if (J->ext) {
            if (J->out->obs) {
                double noise[18];
                or_obs_noise(c, env, t, noise);
                or_obs_actor(c, s, hist, noise, J->out->obs + (size_t)((size_t)tt * n + k) * da);
            }
            for (int i = 0; i < 4; ++i)
                a[i] = clampd(J->ext[((size_t)tt * n + k) * 4 + i], -1.0, 1.0);
        } else {
            if ((int64_t)t < (int64_t)c->learning_starts) {
                /* warm-up: uniform random actions (reading of the TD3 start phase) */
                if (J->out->obs) {
                    /* the observation of this step, for callers that record it */
                    double noise[18];
                    or_obs_noise(c, env, t, noise);
                    or_obs_actor(c, s, hist, noise, J->out->obs + (size_t)((size_t)tt * n + k) * da);
                }
                uint32_t r[4];
                draw(c, env, (uint32_t)t, TAG_WARM, 0, r);
                for (int i = 0; i < 4; ++i) a[i] = 2.0 * or_uniform(r[i]) - 1.0;
            } else {
                double noise[18], o[18 + 4 * OR_HMAX];
                or_obs_noise(c, env, t, noise);
                or_obs_actor(c, s, hist, noise, o);
                if (J->out->obs) memcpy(J->out->obs + (size_t)((size_t)tt * n + k) * da, o,
                                        sizeof(double) * (size_t)da);
                or_mlp_forward(&actor, J->actor, o, h1, h2, mu, 1);
                double z[4];
                for (int sub = 0; sub < 2; ++sub) {
                    uint32_t r[4];
                    draw(c, env, (uint32_t)t, TAG_EXPL, (uint32_t)sub, r);
                    z[2 * sub] = or_gauss(r[0], r[1]);
                    z[2 * sub + 1] = or_gauss(r[2], r[3]);
                }
                for (int i = 0; i < 4; ++i) a[i] = clampd(mu[i] + J->sigma_e * z[i], -1.0, 1.0);
            }
        }
        /* normalised action -> RPM set-point, linear over the RPM range (reading) */
        double u[4];
        for (int i = 0; i < 4; ++i)
            u[i] = c->rpm_min + 0.5 * (a[i] + 1.0) * (c->rpm_max - c->rpm_min);
        double s2[OR_NS];
        step_dynamics(c, s, u, prm, dist, s2);
        double r = or_reward(J->C, s2, a);
        uint32_t ep_before = e->ep_step[k];
        e->ep_step[k] += 1;
        int term = !finite_state(s2) || fabs(s2[0]) > c->term_pos || fabs(s2[1]) > c->term_pos ||
                   fabs(s2[2]) > c->term_pos;
        int trunc = !term && (int64_t)e->ep_step[k] >= (int64_t)c->episode_len;
        size_t rk = (size_t)tt * n + k;
        memcpy(J->out->rec_s + OR_NS * rk, s, sizeof(double) * OR_NS);
        memcpy(J->out->rec_a + 4 * rk, a, sizeof(double) * 4);
        J->out->rec_r[rk] = r;
        J->out->rec_flags[rk] = (uint32_t)term | ((uint32_t)trunc << 1) | (ep_before << 8);
        or_priv(c, prm, dist, J->out->rec_priv + OR_NPRIV * rk);
        if (J->out->mu) memcpy(J->out->mu + 4 * rk, mu, sizeof(double) * 4);
        if (term || trunc) memcpy(J->out->side + OR_NS * rk, s2, sizeof(double) * OR_NS);
        e->ep_ret[k] += r;
        /* history: newest first */
        memmove(hist + 4, hist, sizeof(double) * 4 * (OR_HMAX - 1));
        memcpy(hist, a, sizeof(double) * 4);
        memcpy(s, s2, sizeof(double) * OR_NS);
        if (term || trunc) {
            e->n_done[k] += 1;
            e->len_sum[k] += e->ep_step[k];
            e->ret_sum[k] += e->ep_ret[k];
            e->ep_index[k] += 1;
            env_reset_local(c, e, k);
        }
    }
    free(h1);
}

static void* roll_thread(void* arg) {
    roll_job* J = (roll_job*)arg;
    for (int k = J->k0; k < J->k1; ++k) roll_env(J, k);
    return NULL;
}

int or_rollout(const or_cfg* c, const or_reward_c* C, or_envs* e, const double* actor,
               int hidden, int T, uint64_t t0, double sigma_e, const double* ext_actions,
               or_roll_out* out, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > e->n) n_threads = e->n > 0 ? e->n : 1;
    roll_job* jobs = (roll_job*)calloc((size_t)n_threads, sizeof(roll_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int i = 0; i < n_threads; ++i) {
        roll_job J = {c, C, e, actor, hidden, T, (int)((int64_t)e->n * i / n_threads),
                      (int)((int64_t)e->n * (i + 1) / n_threads), t0, sigma_e, ext_actions, out};
        jobs[i] = J;
    }
    if (n_threads == 1) {
        roll_thread(&jobs[0]);
    } else {
        for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, roll_thread, &jobs[i]);
        for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    }
    free(jobs); free(th);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Trajectory tracking in simulation (Sec. V "Trajectory tracking").  The trained
 * position controller is steered along a moving target by offsetting its observation:
 * Sec. IV reaches any position / velocity set-point by shifting the current position and
 * velocity, with the offsets clipped to the size the controller met in training.  The
 * target of Sec. V is the figure-eight Lissajous curve
 *   p*(t) = (A cos(2 pi t / T), (A / 2) sin(4 pi t / T), z0)
 * (A = 1 m in the paper); v*(t) is its time derivative. */
void or_lissajous(double t, double T, double A, double z0, double* p, double* v) {
    const double w = 2.0 * M_PI / T;
    p[0] = A * cos(w * t);
    p[1] = 0.5 * A * sin(2.0 * w * t);
    p[2] = z0;
    v[0] = -A * w * sin(w * t);
    v[1] = A * w * cos(2.0 * w * t);
    v[2] = 0.0;
}

typedef struct track_job {
    const or_cfg* c;
    const or_track* J;
    int k0, k1;
} track_job;

static void track_env(const or_cfg* c, const or_track* J, int k) {
    const double* prm = J->prm + OR_NPRM * k;
    const double* dist = J->dist + OR_NDIST * k;
    const double T = J->period[k];
    J->sq_err[2 * k] = 0.0;
    J->sq_err[2 * k + 1] = 0.0;
    J->steps_ok[k] = 0;
    if (!(T > 0.0) || !isfinite(T)) return; /* no target: no flight */
    or_net actor = {or_actor_in(c), J->hidden, 4};
    double* h1 = (double*)malloc(sizeof(double) * (size_t)J->hidden * 2);
    double* h2 = h1 + J->hidden;
    double s[OR_NS], pr[3], vr[3], hist[4 * OR_HMAX];
    memset(s, 0, sizeof(s));
    memset(hist, 0, sizeof(hist));
    /* start (reading): on the target with its velocity, level, not rotating, motors at
     * the hover speed of this env's mass and thrust coefficient, no action history */
    or_lissajous(0.0, T, J->amp, J->z0, pr, vr);
    for (int i = 0; i < 3; ++i) { s[i] = pr[i]; s[7 + i] = vr[i]; }
    s[3] = 1.0;
    double hover = clampd(sqrt(prm[0] * c->g / (4.0 * prm[4])), c->rpm_min, c->rpm_max);
    for (int i = 0; i < 4; ++i) s[13 + i] = hover;
    if (J->traj) memcpy(J->traj + (size_t)k * (J->n_steps + 1) * OR_NS, s, sizeof(s));
    double e3 = 0.0, exy = 0.0;
    int ok = 0;
    for (int kk = 0; kk < J->n_steps; ++kk) {
        /* shifted, clipped observation; no observation noise, no exploration (reading) */
        or_lissajous(kk * c->dt, T, J->amp, J->z0, pr, vr);
        double sh[OR_NS], o[18 + 4 * OR_HMAX], mu[4], a[4], u[4], s2[OR_NS];
        memcpy(sh, s, sizeof(sh));
        for (int i = 0; i < 3; ++i) {
            sh[i] = clampd(s[i] - pr[i], -J->clip_p, J->clip_p);
            sh[7 + i] = clampd(s[7 + i] - vr[i], -J->clip_v, J->clip_v);
        }
        or_obs_actor(c, sh, hist, NULL, o);
        or_mlp_forward(&actor, J->actor, o, h1, h2, mu, 1);
        for (int i = 0; i < 4; ++i) {
            a[i] = clampd(mu[i], -1.0, 1.0);
            u[i] = c->rpm_min + 0.5 * (a[i] + 1.0) * (c->rpm_max - c->rpm_min);
        }
        step_dynamics(c, s, u, prm, dist, s2);
        /* tracking error against the target at the new time; a non-finite state or an
         * error outside the training termination box ends the flight (reading) */
        or_lissajous((kk + 1) * c->dt, T, J->amp, J->z0, pr, vr);
        double e[3] = {s2[0] - pr[0], s2[1] - pr[1], s2[2] - pr[2]};
        if (J->traj) memcpy(J->traj + ((size_t)k * (J->n_steps + 1) + kk + 1) * OR_NS, s2, sizeof(s2));
        if (!finite_state(s2) || fabs(e[0]) > c->term_pos || fabs(e[1]) > c->term_pos ||
            fabs(e[2]) > c->term_pos)
            break;
        e3 += e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        exy += e[0] * e[0] + e[1] * e[1];
        ok += 1;
        memmove(hist + 4, hist, sizeof(double) * 4 * (OR_HMAX - 1));
        memcpy(hist, a, sizeof(double) * 4);
        memcpy(s, s2, sizeof(s));
    }
    J->sq_err[2 * k] = e3;
    J->sq_err[2 * k + 1] = exy;
    J->steps_ok[k] = ok;
    free(h1);
}

static void* track_thread(void* arg) {
    track_job* t = (track_job*)arg;
    for (int k = t->k0; k < t->k1; ++k) track_env(t->c, t->J, k);
    return NULL;
}

int or_track_run(const or_cfg* c, const or_track* J, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > J->n) n_threads = J->n > 0 ? J->n : 1;
    track_job* jobs = (track_job*)calloc((size_t)n_threads, sizeof(track_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int i = 0; i < n_threads; ++i) {
        track_job t = {c, J, (int)((int64_t)J->n * i / n_threads),
                       (int)((int64_t)J->n * (i + 1) / n_threads)};
        jobs[i] = t;
    }
    if (n_threads == 1) {
        track_thread(&jobs[0]);
    } else {
        for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, track_thread, &jobs[i]);
        for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    }
    free(jobs); free(th);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* TD3 update with an asymmetric (privileged) critic (Sec. IV; TD3).                    */
/* ------------------------------------------------------------------------------------ */
static int64_t pmod(int64_t a, int64_t m) { int64_t r = a % m; return r < 0 ? r + m : r; }

static void adam_step(double* th, const double* g, double* m, double* v, int P, int64_t t,
                      const or_td3* L) {
    double bc1 = 1.0 - pow(L->beta1, (double)t), bc2 = 1.0 - pow(L->beta2, (double)t);
    for (int i = 0; i < P; ++i) {
        m[i] = L->beta1 * m[i] + (1.0 - L->beta1) * g[i];
        v[i] = L->beta2 * v[i] + (1.0 - L->beta2) * g[i] * g[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        th[i] -= L->lr * mh / (sqrt(vh) + L->eps);
    }
}

static void polyak(double* tgt, const double* src, int P, double tau) {
    for (int i = 0; i < P; ++i) tgt[i] = tau * src[i] + (1.0 - tau) * tgt[i];
}

int or_td3_update(const or_cfg* c, or_td3* L, const or_buffer* b, or_td3_diag* d) {
    const int B = L->batch, H = L->hidden, DA = or_actor_in(c), DC = or_critic_in(c);
    const int PA = or_net_size(DA, H, 4), PC = or_net_size(DC, H, 1);
    const int NE = b->n_env, CAP = b->capacity;
    const int64_t lost = (b->size == b->capacity) ? c->n_hist : 0;
    const int64_t nslot = b->size - 1 - lost;
    if (nslot <= 0 || (uint64_t)nslot * (uint64_t)NE >= (1ull << 32)) return -1;
    const uint32_t nvalid = (uint32_t)(nslot * NE);
    const uint32_t u = (uint32_t)L->update_idx;
    or_net actor = {DA, H, 4}, critic = {DC, H, 1};

    double* oa = (double*)calloc((size_t)B * DA, sizeof(double));
    double* oa2 = (double*)calloc((size_t)B * DA, sizeof(double));
    double* oc = (double*)calloc((size_t)B * DC, sizeof(double));
    double* oc2 = (double*)calloc((size_t)B * DC, sizeof(double));
    double* rr = (double*)calloc((size_t)B, sizeof(double));
    int* term = (int*)calloc((size_t)B, sizeof(int));
    double* y = (double*)calloc((size_t)B, sizeof(double));
    double* h1 = (double*)calloc((size_t)H, sizeof(double));
    double* h2 = (double*)calloc((size_t)H, sizeof(double));
    double* gin = (double*)calloc((size_t)DC, sizeof(double));
    double* ga = (double*)calloc((size_t)PA, sizeof(double));
    double* g1 = (double*)calloc((size_t)PC, sizeof(double));
    double* g2 = (double*)calloc((size_t)PC, sizeof(double));
    double* ha1 = (double*)calloc((size_t)H, sizeof(double));
    double* ha2 = (double*)calloc((size_t)H, sizeof(double));

    /* a9: minibatch sample + gather, observations rebuilt from the compact records */
    for (int j = 0; j < B; ++j) {
        uint32_t r4[4];
        draw(c, (uint32_t)j >> 2, u, TAG_REPLAY, 0, r4);
        uint32_t idx = or_replay_index(r4[j & 3], nvalid);
        if (d && d->idx) d->idx[j] = idx;
        int64_t k = idx / (uint32_t)NE;
        int env = (int)(idx % (uint32_t)NE);
        int64_t slot = pmod(b->head - b->size + lost + k, CAP);
        int64_t t_rec = b->t_now - b->size + lost + k;
        size_t rk = (size_t)slot * NE + env;
        uint32_t fl = b->flags[rk];
        int done = (fl & 3u) != 0;
        uint32_t ep = fl >> 8;
        const double* s = b->s + OR_NS * rk;
        const double* a = b->a + 4 * rk;
        const double* priv = b->priv + OR_NPRIV * rk;
        const double* s2 = done ? b->side + OR_NS * rk
                                : b->s + OR_NS * ((size_t)pmod(slot + 1, CAP) * NE + env);
        double hist[4 * OR_HMAX], hist2[4 * OR_HMAX];
        memset(hist, 0, sizeof(hist));
        memset(hist2, 0, sizeof(hist2));
        for (int i = 1; i <= c->n_hist; ++i) {
            if ((uint32_t)i <= ep) {
                const double* ap = b->a + 4 * ((size_t)pmod(slot - i, CAP) * NE + env);
                for (int cc = 0; cc < 4; ++cc) hist[4 * (i - 1) + cc] = ap[cc];
            }
            if (i == 1) {
                for (int cc = 0; cc < 4; ++cc) hist2[cc] = a[cc];
            } else if ((uint32_t)(i - 1) <= ep) {
                const double* ap = b->a + 4 * ((size_t)pmod(slot - (i - 1), CAP) * NE + env);
                for (int cc = 0; cc < 4; ++cc) hist2[4 * (i - 1) + cc] = ap[cc];
            }
        }
        double n1[18], n2[18];
        or_obs_noise(c, (uint32_t)env, (uint64_t)t_rec, n1);
        or_obs_noise(c, (uint32_t)env, (uint64_t)(t_rec + 1), n2);
        or_obs_actor(c, s, hist, n1, oa + (size_t)j * DA);
        or_obs_actor(c, s2, hist2, n2, oa2 + (size_t)j * DA);
        if (c->critic_layout == OR_CRITIC_ACTOR) {
            /* ablation of the asymmetric actor-critic: the critic sees exactly what the
             * actor sees, observation noise included */
            memcpy(oc + (size_t)j * DC, oa + (size_t)j * DA, sizeof(double) * (size_t)DA);
            memcpy(oc2 + (size_t)j * DC, oa2 + (size_t)j * DA, sizeof(double) * (size_t)DA);
        } else {
            or_obs_critic(c, s, hist, priv, oc + (size_t)j * DC);
            or_obs_critic(c, s2, hist2, priv, oc2 + (size_t)j * DC);
        }
        for (int cc = 0; cc < 4; ++cc) oc[(size_t)j * DC + DC - 4 + cc] = a[cc];
        rr[j] = b->r[rk];
        term[j] = (int)(fl & 1u);
    }

    /* a10: target actor + target-policy smoothing */
    for (int j = 0; j < B; ++j) {
        double mu2[4], z[4];
        or_mlp_forward(&actor, L->actor_t, oa2 + (size_t)j * DA, h1, h2, mu2, 1);
        for (int sub = 0; sub < 2; ++sub) {
            uint32_t r4[4];
            draw(c, (uint32_t)j, u, TAG_SMOOTH, (uint32_t)sub, r4);
            z[2 * sub] = or_gauss(r4[0], r4[1]);
            z[2 * sub + 1] = or_gauss(r4[2], r4[3]);
        }
        for (int i = 0; i < 4; ++i) {
            double eps = clampd(L->sigma_t * z[i], -L->noise_clip, L->noise_clip);
            double a2 = clampd(mu2[i] + eps, -1.0, 1.0);
            oc2[(size_t)j * DC + DC - 4 + i] = a2;
            if (d && d->a2) d->a2[4 * j + i] = a2;
        }
    }
    if (d) {
        if (d->oa) memcpy(d->oa, oa, sizeof(double) * (size_t)B * DA);
        if (d->oa2) memcpy(d->oa2, oa2, sizeof(double) * (size_t)B * DA);
        if (d->oc) memcpy(d->oc, oc, sizeof(double) * (size_t)B * DC);
        if (d->oc2) memcpy(d->oc2, oc2, sizeof(double) * (size_t)B * DC);
    }
    /* a11: twin target critics, clipped double-Q target; no bootstrap on termination */
    for (int j = 0; j < B; ++j) {
        double q1t, q2t;
        or_mlp_forward(&critic, L->c1_t, oc2 + (size_t)j * DC, h1, h2, &q1t, 0);
        or_mlp_forward(&critic, L->c2_t, oc2 + (size_t)j * DC, h1, h2, &q2t, 0);
        double qmin = q1t < q2t ? q1t : q2t;
        y[j] = rr[j] + (term[j] ? 0.0 : L->gamma * qmin);
        if (d && d->y) d->y[j] = y[j];
    }
    /* a12: critic regression L = mean (Q1-y)^2 + mean (Q2-y)^2 */
    double lc = 0.0;
    for (int j = 0; j < B; ++j) {
        double q;
        const double* x = oc + (size_t)j * DC;
        or_mlp_forward(&critic, L->c1, x, h1, h2, &q, 0);
        if (d && d->q1) d->q1[j] = q;
        double dq = 2.0 * (q - y[j]) / B;
        lc += (q - y[j]) * (q - y[j]) / B;
        mlp_backward(&critic, L->c1, x, h1, h2, &q, &dq, 0, g1, NULL);
        or_mlp_forward(&critic, L->c2, x, h1, h2, &q, 0);
        if (d && d->q2) d->q2[j] = q;
        dq = 2.0 * (q - y[j]) / B;
        lc += (q - y[j]) * (q - y[j]) / B;
        mlp_backward(&critic, L->c2, x, h1, h2, &q, &dq, 0, g2, NULL);
    }
    if (d) {
        d->critic_loss = lc;
        if (d->g_c1) memcpy(d->g_c1, g1, sizeof(double) * PC);
        if (d->g_c2) memcpy(d->g_c2, g2, sizeof(double) * PC);
    }
    /* a14 (critics): Adam */
    L->t_c += 1;
    adam_step(L->c1, g1, L->m_c1, L->v_c1, PC, L->t_c, L);
    adam_step(L->c2, g2, L->m_c2, L->v_c2, PC, L->t_c, L);

    /* a13: delayed actor update through the (updated) first critic */
    int do_actor = (L->update_idx % L->policy_delay) == (L->policy_delay - 1);
    if (d) d->actor_updated = do_actor;
    if (do_actor) {
        double la = 0.0;
        double* xpi = (double*)calloc((size_t)DC, sizeof(double));
        for (int j = 0; j < B; ++j) {
            double mu[4], q;
            const double* xo = oa + (size_t)j * DA;
            or_mlp_forward(&actor, L->actor, xo, ha1, ha2, mu, 1);
            memcpy(xpi, oc + (size_t)j * DC, sizeof(double) * DC);
            for (int i = 0; i < 4; ++i) xpi[DC - 4 + i] = mu[i];
            or_mlp_forward(&critic, L->c1, xpi, h1, h2, &q, 0);
            la += -q / B;
            double dq = -1.0 / B;
            double* dummy = (double*)calloc((size_t)PC, sizeof(double));
            mlp_backward(&critic, L->c1, xpi, h1, h2, &q, &dq, 0, dummy, gin);
            free(dummy);
            mlp_backward(&actor, L->actor, xo, ha1, ha2, mu, gin + DC - 4, 1, ga, NULL);
        }
        free(xpi);
        if (d) {
            d->actor_loss = la;
            if (d->g_a) memcpy(d->g_a, ga, sizeof(double) * PA);
        }
        L->t_a += 1;
        adam_step(L->actor, ga, L->m_a, L->v_a, PA, L->t_a, L);
        polyak(L->actor_t, L->actor, PA, L->tau);
        polyak(L->c1_t, L->c1, PC, L->tau);
        polyak(L->c2_t, L->c2, PC, L->tau);
    }
    L->update_idx += 1;
    free(oa); free(oa2); free(oc); free(oc2); free(rr); free(term); free(y); free(h1);
    free(h2); free(gin); free(ga); free(g1); free(g2); free(ha1); free(ha2);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Curriculum + reward recalculation (Sec. IV: every 100,000 steps multiply the reward   */
/* weights by their factors until the targets; Sec. VI: recompute every stored reward   */
/* after each change).                                                                  */
/* ------------------------------------------------------------------------------------ */
void or_curriculum(const double* factor, const double* target, double* C, int n) {
    for (int i = 0; i < n; ++i) {
        double x = C[i] * factor[i];
        if (factor[i] >= 1.0) C[i] = x < target[i] ? x : target[i];
        else C[i] = x > target[i] ? x : target[i];
    }
}

int or_recalc_rewards(const or_reward_c* C, or_buffer* b, const double* cur_state) {
    const int NE = b->n_env, CAP = b->capacity;
    for (int64_t k = 0; k < b->size; ++k) {
        int64_t slot = pmod(b->head - b->size + k, CAP);
        for (int env = 0; env < NE; ++env) {
            size_t rk = (size_t)slot * NE + env;
            int done = (b->flags[rk] & 3u) != 0;
            const double* s2;
            if (done) s2 = b->side + OR_NS * rk;
            else if (k == b->size - 1) s2 = cur_state + OR_NS * env;
            else s2 = b->s + OR_NS * ((size_t)pmod(slot + 1, CAP) * NE + env);
            b->r[rk] = or_reward(C, s2, b->a + 4 * rk);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Differentiation through the simulator: reverse mode of RK4 (with renormalisation)    */
/* and of the actor, over a fixed horizon with no resets.                                */
/* Loss = sum_{t=1..H} [w_p|p_t|^2 + w_q(1-q_w,t^2) + w_v|v_t|^2] + w_a sum_{t<H} |a_t|^2 */
/* ------------------------------------------------------------------------------------ */
/* Vector-Jacobian product of the derivative f(s,u,prm,dist): given lam = dL/df, ADD
 * dL/ds, dL/du (u inside the RPM range only) and dL/dprm. */
static void deriv_vjp(const or_cfg* c, const double* s, const double* u, const double* prm,
                      const double* dist, const double* lam, double* gs, double* gu,
                      double* gp) {
    const double m = prm[0], J[3] = {prm[1], prm[2], prm[3]}, kf = prm[4], km = prm[5],
                 tm = prm[6];
    const double *q = s + 3, *w = s + 10, *wm = s + 13;
    double f[4], F = 0.0;
    for (int i = 0; i < 4; ++i) { f[i] = kf * wm[i] * wm[i]; F += f[i]; }
    double R[9];
    quat_rot(q, R);
    /* p' = v */
    for (int k = 0; k < 3; ++k) gs[7 + k] += lam[k];
    /* v'_k = R[k][2] F/m + d_k/m - g e_z */
    const double* lv = lam + 7;
    double gF = 0.0;
    for (int k = 0; k < 3; ++k) gF += lv[k] * R[3 * k + 2] / m;
    for (int k = 0; k < 3; ++k) gp[0] += -lv[k] * (R[3 * k + 2] * F + dist[k]) / (m * m);
    /* dR[k][2]/dq scaled by F/m */
    double G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    G[2] = lv[0] * F / m; G[5] = lv[1] * F / m; G[8] = lv[2] * F / m;
    {
        double qw = q[0], qx = q[1], qy = q[2], qz = q[3];
        gs[3] += 2 * (-qz * G[1] + qy * G[2] + qz * G[3] - qx * G[5] - qy * G[6] + qx * G[7]);
        gs[4] += 2 * (qy * G[1] + qz * G[2] + qy * G[3] - 2 * qx * G[4] - qw * G[5] + qz * G[6] +
                      qw * G[7] - 2 * qx * G[8]);
        gs[5] += 2 * (-2 * qy * G[0] + qx * G[1] + qw * G[2] + qx * G[3] + qz * G[5] - qw * G[6] +
                      qz * G[7] - 2 * qy * G[8]);
        gs[6] += 2 * (-2 * qz * G[0] - qw * G[1] + qx * G[2] + qw * G[3] - 2 * qz * G[4] +
                      qy * G[5] + qx * G[6] + qy * G[7]);
    }
    /* q' = 1/2 q (x) (0, w) */
    const double* lq = lam + 3;
    gs[3] += 0.5 * (lq[1] * w[0] + lq[2] * w[1] + lq[3] * w[2]);
    gs[4] += 0.5 * (-lq[0] * w[0] - lq[2] * w[2] + lq[3] * w[1]);
    gs[5] += 0.5 * (-lq[0] * w[1] + lq[1] * w[2] - lq[3] * w[0]);
    gs[6] += 0.5 * (-lq[0] * w[2] - lq[1] * w[1] + lq[2] * w[0]);
    gs[10] += 0.5 * (-q[1] * lq[0] + q[0] * lq[1] + q[3] * lq[2] - q[2] * lq[3]);
    gs[11] += 0.5 * (-q[2] * lq[0] - q[3] * lq[1] + q[0] * lq[2] + q[1] * lq[3]);
    gs[12] += 0.5 * (-q[3] * lq[0] + q[2] * lq[1] - q[1] * lq[2] + q[0] * lq[3]);
    /* w'_x = (tau_x - (Jz-Jy) w_y w_z)/Jx, cyclic */
    const double* lw = lam + 10;
    double mu[3] = {lw[0] / J[0], lw[1] / J[1], lw[2] / J[2]};
    double wd[3];
    {
        double tau[3] = {dist[3], dist[4], dist[5]};
        for (int i = 0; i < 4; ++i) {
            const double* r = c->rotor_pos + 3 * i;
            tau[0] += r[1] * f[i]; tau[1] += -r[0] * f[i]; tau[2] += c->rotor_dir[i] * km * f[i];
        }
        wd[0] = (tau[0] - (J[2] - J[1]) * w[1] * w[2]) / J[0];
        wd[1] = (tau[1] - (J[0] - J[2]) * w[2] * w[0]) / J[1];
        wd[2] = (tau[2] - (J[1] - J[0]) * w[0] * w[1]) / J[2];
    }
    gs[10] += -mu[1] * (J[0] - J[2]) * w[2] - mu[2] * (J[1] - J[0]) * w[1];
    gs[11] += -mu[0] * (J[2] - J[1]) * w[2] - mu[2] * (J[1] - J[0]) * w[0];
    gs[12] += -mu[0] * (J[2] - J[1]) * w[1] - mu[1] * (J[0] - J[2]) * w[0];
    gp[1] += -lw[0] * wd[0] / J[0] - mu[1] * w[2] * w[0] + mu[2] * w[0] * w[1];
    gp[2] += -lw[1] * wd[1] / J[1] + mu[0] * w[1] * w[2] - mu[2] * w[0] * w[1];
    gp[3] += -lw[2] * wd[2] / J[2] - mu[0] * w[1] * w[2] + mu[1] * w[2] * w[0];
    /* rotor forces feed F and tau */
    double sdf = 0.0;
    for (int i = 0; i < 4; ++i) {
        const double* r = c->rotor_pos + 3 * i;
        double gf = gF + mu[0] * r[1] - mu[1] * r[0] + mu[2] * c->rotor_dir[i] * km;
        gs[13 + i] += gf * 2.0 * kf * wm[i];
        gp[4] += gf * wm[i] * wm[i];
        sdf += c->rotor_dir[i] * f[i];
    }
    gp[5] += mu[2] * sdf;
    /* w_m' = (clip(u) - w_m)/T_m */
    const double* lm = lam + 13;
    for (int i = 0; i < 4; ++i) {
        double uc = clampd(u[i], c->rpm_min, c->rpm_max);
        gs[13 + i] += -lm[i] / tm;
        if (u[i] > c->rpm_min && u[i] < c->rpm_max) gu[i] += lm[i] / tm;
        gp[6] += -lm[i] * (uc - wm[i]) / (tm * tm);
    }
}

/* Reverse of one RK4 step (+ renormalisation): given lam' = dL/ds', ADD dL/ds, dL/du,
 * dL/dprm. */
static void rk4_vjp(const or_cfg* c, const double* s, const double* u, const double* prm,
                    const double* dist, double dt, int renorm, const double* lam_out,
                    double* gs, double* gu, double* gp) {
    double k1[OR_NS], k2[OR_NS], k3[OR_NS], k4[OR_NS], y2[OR_NS], y3[OR_NS], y4[OR_NS],
        pre[OR_NS];
    or_deriv(c, s, u, prm, dist, k1);
    for (int i = 0; i < OR_NS; ++i) y2[i] = s[i] + 0.5 * dt * k1[i];
    or_deriv(c, y2, u, prm, dist, k2);
    for (int i = 0; i < OR_NS; ++i) y3[i] = s[i] + 0.5 * dt * k2[i];
    or_deriv(c, y3, u, prm, dist, k3);
    for (int i = 0; i < OR_NS; ++i) y4[i] = s[i] + dt * k3[i];
    or_deriv(c, y4, u, prm, dist, k4);
    for (int i = 0; i < OR_NS; ++i)
        pre[i] = s[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    double lam[OR_NS];
    memcpy(lam, lam_out, sizeof(lam));
    if (renorm) {
        double n = sqrt(pre[3] * pre[3] + pre[4] * pre[4] + pre[5] * pre[5] + pre[6] * pre[6]);
        double qn[4] = {pre[3] / n, pre[4] / n, pre[5] / n, pre[6] / n};
        double dot = 0.0;
        for (int i = 0; i < 4; ++i) dot += qn[i] * lam_out[3 + i];
        for (int i = 0; i < 4; ++i) lam[3 + i] = (lam_out[3 + i] - qn[i] * dot) / n;
    }
    double lk1[OR_NS], lk2[OR_NS], lk3[OR_NS], lk4[OR_NS], ly[OR_NS];
    for (int i = 0; i < OR_NS; ++i) {
        gs[i] += lam[i];
        lk1[i] = dt / 6.0 * lam[i];
        lk2[i] = dt / 3.0 * lam[i];
        lk3[i] = dt / 3.0 * lam[i];
        lk4[i] = dt / 6.0 * lam[i];
    }
    memset(ly, 0, sizeof(ly));
    deriv_vjp(c, y4, u, prm, dist, lk4, ly, gu, gp);
    for (int i = 0; i < OR_NS; ++i) { gs[i] += ly[i]; lk3[i] += dt * ly[i]; }
    memset(ly, 0, sizeof(ly));
    deriv_vjp(c, y3, u, prm, dist, lk3, ly, gu, gp);
    for (int i = 0; i < OR_NS; ++i) { gs[i] += ly[i]; lk2[i] += 0.5 * dt * ly[i]; }
    memset(ly, 0, sizeof(ly));
    deriv_vjp(c, y2, u, prm, dist, lk2, ly, gu, gp);
    for (int i = 0; i < OR_NS; ++i) { gs[i] += ly[i]; lk1[i] += 0.5 * dt * ly[i]; }
    deriv_vjp(c, s, u, prm, dist, lk1, gs, gu, gp);
}

/* Reverse of the observation's state part {p, R(q), v, omega}: ADD into gs. */
static void obs_vjp(const double* s, const double* go, double* gs) {
    const double* q = s + 3;
    const double* G = go + 3;
    double qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    for (int k = 0; k < 3; ++k) gs[k] += go[k];
    gs[3] += 2 * (-qz * G[1] + qy * G[2] + qz * G[3] - qx * G[5] - qy * G[6] + qx * G[7]);
    gs[4] += 2 * (qy * G[1] + qz * G[2] + qy * G[3] - 2 * qx * G[4] - qw * G[5] + qz * G[6] +
                  qw * G[7] - 2 * qx * G[8]);
    gs[5] += 2 * (-2 * qy * G[0] + qx * G[1] + qw * G[2] + qx * G[3] + qz * G[5] - qw * G[6] +
                  qz * G[7] - 2 * qy * G[8]);
    gs[6] += 2 * (-2 * qz * G[0] - qw * G[1] + qx * G[2] + qw * G[3] - 2 * qz * G[4] + qy * G[5] +
                  qx * G[6] + qy * G[7]);
    for (int k = 0; k < 3; ++k) gs[7 + k] += go[12 + k];
    for (int k = 0; k < 3; ++k) gs[10 + k] += go[15 + k];
}

static double state_loss(const or_diff* d, const double* s) {
    return d->w_p * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) + d->w_q * (1.0 - s[3] * s[3]) +
           d->w_v * (s[7] * s[7] + s[8] * s[8] + s[9] * s[9]);
}

static void state_loss_grad(const or_diff* d, const double* s, double* g) {
    for (int k = 0; k < 3; ++k) g[k] += 2.0 * d->w_p * s[k];
    g[3] += -2.0 * d->w_q * s[3];
    for (int k = 0; k < 3; ++k) g[7 + k] += 2.0 * d->w_v * s[7 + k];
}

int or_diff_run(const or_cfg* c0, or_diff* d) {
    or_cfg cc = *c0;
    cc.n_hist = d->n_hist;
    const or_cfg* c = &cc;
    const int H = d->H, DA = 18 + 4 * d->n_hist, HID = d->hidden;
    const int PA = or_net_size(DA, HID, 4);
    or_net actor = {DA, HID, 4};
    const double zero_dist[OR_NDIST] = {0, 0, 0, 0, 0, 0};
    double* S = (double*)malloc(sizeof(double) * (size_t)(H + 1) * OR_NS);
    double* A = (double*)malloc(sizeof(double) * (size_t)H * 4);
    double* O = (double*)malloc(sizeof(double) * (size_t)H * (DA > 0 ? DA : 1));
    double* h1 = (double*)malloc(sizeof(double) * (size_t)H * (HID > 0 ? HID : 1));
    double* h2 = (double*)malloc(sizeof(double) * (size_t)H * (HID > 0 ? HID : 1));
    double* la = (double*)malloc(sizeof(double) * (size_t)H * 4);
    if (d->mode == 1 && d->g_actor) memset(d->g_actor, 0, sizeof(double) * PA);
    for (int e = 0; e < d->n; ++e) {
        const double* prm = d->prm + OR_NPRM * e;
        memcpy(S, d->s0 + OR_NS * e, sizeof(double) * OR_NS);
        double loss = 0.0;
        /* forward */
        for (int t = 0; t < H; ++t) {
            double* a = A + 4 * t;
            if (d->mode == 0) {
                memcpy(a, d->actions + ((size_t)e * H + t) * 4, sizeof(double) * 4);
            } else {
                double hist[4 * OR_HMAX];
                memset(hist, 0, sizeof(hist));
                for (int i = 1; i <= d->n_hist; ++i)
                    if (t - i >= 0) memcpy(hist + 4 * (i - 1), A + 4 * (t - i), sizeof(double) * 4);
                or_obs_actor(c, S + OR_NS * t, hist, NULL, O + (size_t)t * DA);
                or_mlp_forward(&actor, d->actor, O + (size_t)t * DA, h1 + (size_t)t * HID,
                               h2 + (size_t)t * HID, a, 1);
            }
            double u[4];
            for (int i = 0; i < 4; ++i)
                u[i] = c->rpm_min + 0.5 * (a[i] + 1.0) * (c->rpm_max - c->rpm_min);
            or_rk4(c, S + OR_NS * t, u, prm, zero_dist, c->dt, c->renorm_q, S + OR_NS * (t + 1));
            loss += state_loss(d, S + OR_NS * (t + 1));
            loss += d->w_a * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
        }
        if (d->loss) d->loss[e] = loss;
        if (d->traj) memcpy(d->traj + (size_t)e * (H + 1) * OR_NS, S, sizeof(double) * (H + 1) * OR_NS);
        if (d->act_out) memcpy(d->act_out + (size_t)e * H * 4, A, sizeof(double) * H * 4);
        /* reverse */
        double lam[OR_NS];
        memset(lam, 0, sizeof(lam));
        memset(la, 0, sizeof(double) * (size_t)H * 4);
        double gp[OR_NPRM];
        memset(gp, 0, sizeof(gp));
        state_loss_grad(d, S + OR_NS * H, lam);
        for (int t = H - 1; t >= 0; --t) {
            const double* a = A + 4 * t;
            double u[4], gu[4] = {0, 0, 0, 0}, gs[OR_NS];
            memset(gs, 0, sizeof(gs));
            for (int i = 0; i < 4; ++i)
                u[i] = c->rpm_min + 0.5 * (a[i] + 1.0) * (c->rpm_max - c->rpm_min);
            rk4_vjp(c, S + OR_NS * t, u, prm, zero_dist, c->dt, c->renorm_q, lam, gs, gu, gp);
            double gat[4];
            for (int i = 0; i < 4; ++i)
                gat[i] = la[4 * t + i] + gu[i] * 0.5 * (c->rpm_max - c->rpm_min) + 2.0 * d->w_a * a[i];
            if (d->mode == 0) {
                if (d->g_actions) memcpy(d->g_actions + ((size_t)e * H + t) * 4, gat, sizeof(gat));
            } else {
                double* go = (double*)calloc((size_t)DA, sizeof(double));
                mlp_backward(&actor, d->actor, O + (size_t)t * DA, h1 + (size_t)t * HID,
                             h2 + (size_t)t * HID, a, gat, 1, d->g_actor, go);
                obs_vjp(S + OR_NS * t, go, gs);
                for (int i = 1; i <= d->n_hist; ++i)
                    if (t - i >= 0)
                        for (int k = 0; k < 4; ++k) la[4 * (t - i) + k] += go[18 + 4 * (i - 1) + k];
                free(go);
            }
            memcpy(lam, gs, sizeof(lam));
            if (t >= 1) state_loss_grad(d, S + OR_NS * t, lam);
        }
        if (d->g_prm) memcpy(d->g_prm + OR_NPRM * e, gp, sizeof(gp));
    }
    free(S); free(A); free(O); free(h1); free(h2); free(la);
    return 0;
}
