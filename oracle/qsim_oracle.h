/*
 * qsim_oracle.h -- plain FP64 CPU oracle for the quadrotor training hot path of
 * "Learning to Fly in Seconds" (Eschmann et al., arXiv 2311.13081).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this code; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no header, helper or table with the CUDA path.
 *
 * Everything is double precision, one environment / one sample at a time, in
 * the order the method states it (Sec. IV "Methodology" of the paper for the
 * MDP; Fujimoto et al. 2018 for TD3; Kingma & Ba 2015 for Adam; Salmon et al.
 * SC'11 for Philox4x32-10).  Memory layouts here are array-of-structs
 * ([env][field]); the CUDA path uses field-major layouts and the Python test
 * wrapper converts.
 */
#ifndef QSIM_ORACLE_H
#define QSIM_ORACLE_H
#include <stdint.h>

#define OR_NS 17      /* state: p(3) q(4: w,x,y,z) v(3) omega(3) omega_m(4) */
#define OR_NPRM 8     /* per-env params: m, Jx, Jy, Jz, kf, km, Tm, unused */
#define OR_NDIST 6    /* f_r(3), tau_r(3) */
#define OR_NPRIV 6
#define OR_HMAX 16    /* longest action history */

enum { OR_CRITIC_HIST = 0, OR_CRITIC_PRIV = 1, OR_CRITIC_PAPER28 = 2, OR_CRITIC_ACTOR = 3 };

typedef struct or_cfg {
    /* nominal vehicle */
    double mass, Jx, Jy, Jz, kf, km, tm;
    double rotor_pos[12];  /* 4 rotors x (x,y,z), body frame */
    double rotor_dir[4];   /* yaw-torque sign per rotor */
    double rpm_min, rpm_max, g;
    /* integration */
    double dt;
    int32_t renorm_q, n_hist, episode_len, critic_layout;
    /* initial-state distribution */
    double init_p, init_att, init_v, init_w, init_rpm_lo, init_rpm_hi;
    /* domain randomisation (relative half-widths; motor time constant range) */
    double dr_mass, dr_J, dr_kf, tm_lo, tm_hi;
    /* per-episode disturbance half-widths */
    double dist_f, dist_tau;
    /* actor observation noise (std-dev per group) */
    double sig_p, sig_R, sig_v, sig_w;
    /* termination box half-width on position */
    double term_pos;
    /* random stream */
    uint64_t seed;
    uint32_t run_id;
    int32_t learning_starts;
    /* ablation of the motor model: 1 = the rotors run at their set-point at once */
    int32_t motor_lag_off, pad_;
} or_cfg;

/* Reward constants, in the order of the reward formula: C_rp C_rq C_rv C_rw C_ra C_rab C_rs */
typedef struct or_reward_c { double c[7]; } or_reward_c;

typedef struct or_envs {
    int32_t n;
    const uint32_t* env_id;  /* [n] env index used in the random counters */
    double* s;               /* [n][17] */
    double* prm;             /* [n][8] */
    double* dist;            /* [n][6] */
    double* hist;            /* [n][64] newest first: hist[4(i-1)+c] = a_{t-i}[c] */
    uint32_t* ep_index;      /* [n] */
    uint32_t* ep_step;       /* [n] */
    double* ep_ret;          /* [n] */
    uint32_t* n_done;        /* [n] completed episodes */
    uint32_t* len_sum;       /* [n] */
    double* ret_sum;         /* [n] */
} or_envs;

typedef struct or_roll_out {
    double* rec_s;      /* [T][n][17] */
    double* rec_a;      /* [T][n][4] */
    double* rec_r;      /* [T][n] */
    uint32_t* rec_flags;/* [T][n] */
    double* rec_priv;   /* [T][n][6] */
    double* side;       /* [T][n][17], written where the episode ended */
    double* mu;         /* [T][n][4] deterministic actor output (may be NULL) */
    double* obs;        /* [T][n][18 + 4 n_hist] actor observation at each step, noise
                           included, also during warm-up (may be NULL) */
} or_roll_out;

typedef struct or_net {
    int32_t in, hid, out;
} or_net;

typedef struct or_td3 {
    double gamma, tau, lr, beta1, beta2, eps, sigma_t, noise_clip;
    int32_t policy_delay, batch, hidden, pad_;
    double *actor, *actor_t, *c1, *c1_t, *c2, *c2_t;
    double *m_a, *v_a, *m_c1, *v_c1, *m_c2, *v_c2;
    int64_t t_a, t_c, update_idx;
} or_td3;

typedef struct or_buffer {
    int32_t n_env, capacity;
    const double* s;        /* [C][n_env][17] */
    const double* a;        /* [C][n_env][4] */
    double* r;              /* [C][n_env] (rewritten by the recalculation) */
    const uint32_t* flags;  /* [C][n_env] */
    const double* priv;     /* [C][n_env][6] */
    const double* side;     /* [C][n_env][17] */
    int64_t head, size, t_now;
} or_buffer;

typedef struct or_td3_diag {
    uint32_t* idx;      /* [B] sampled flat index */
    double *y, *q1, *q2;/* [B] */
    double* a2;         /* [B][4] smoothed target action */
    double *oa, *oa2;   /* [B][18 + 4 n_hist] rebuilt actor observations at s and s' */
    double *oc, *oc2;   /* [B][critic input] rebuilt critic inputs: o_c with the stored
                           action, o_c' with the smoothed target action */
    double *g_c1, *g_c2, *g_a; /* gradients of the losses */
    double critic_loss, actor_loss;
    int32_t actor_updated, pad_;
} or_td3_diag;

typedef struct or_diff {
    int32_t n, H, mode, n_hist;  /* mode 0: open loop (actions given); 1: closed loop (actor) */
    double w_p, w_q, w_v, w_a;
    const double* s0;       /* [n][17] */
    const double* prm;      /* [n][8] */
    const double* actions;  /* [n][H][4] (open loop) */
    const double* actor;    /* actor params (closed loop) */
    int32_t hidden, pad_;
    double* loss;           /* [n] */
    double* g_actions;      /* [n][H][4] */
    double* g_actor;        /* [P_actor], summed over envs */
    double* g_prm;          /* [n][8] */
    double* traj;           /* [n][H+1][17] (may be NULL) */
    double* act_out;        /* [n][H][4] (may be NULL) */
} or_diff;

/* Simulated trajectory tracking (Sec. V): n envs with their own parameters follow the
 * Lissajous target of cycle time period[k] for n_steps steps. */
typedef struct or_track {
    int32_t n, n_steps, hidden, pad_;
    const double* prm;      /* [n][8] */
    const double* dist;     /* [n][6] */
    const double* period;   /* [n] cycle time T, s */
    const double* actor;    /* actor params */
    double amp, z0, clip_p, clip_v;
    double* sq_err;         /* [n][2]: sum |e|^2, sum e_x^2 + e_y^2 over completed steps */
    int32_t* steps_ok;      /* [n] steps completed before the flight ended */
    double* traj;           /* [n][n_steps + 1][17] (may be NULL): start, then the state after
                               each step up to the one that ended the flight */
} or_track;

#ifdef __cplusplus
extern "C" {
#endif
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform(uint32_t x);
double or_gauss(uint32_t x1, uint32_t x2);
uint32_t or_replay_index(uint32_t x, uint32_t n);
int or_net_size(int in, int hid, int out);
int or_actor_in(const or_cfg* c);
int or_critic_in(const or_cfg* c);
void or_init_params(const or_cfg* c, int net_id, int in, int hid, int out, double* P);

void or_deriv(const or_cfg* c, const double* s, const double* u, const double* prm,
              const double* dist, double* ds);
void or_rk4(const or_cfg* c, const double* s, const double* u, const double* prm,
            const double* dist, double dt, int renorm, double* out);
void or_dynamics_batch(const or_cfg* c, int n, const double* s, const double* u,
                       const double* prm, const double* dist, double dt, int renorm,
                       int n_steps, double* out);
void or_reset_env(const or_cfg* c, uint32_t env, uint32_t episode, double* s, double* prm,
                  double* dist);
void or_obs_noise(const or_cfg* c, uint32_t env, uint64_t t, double* noise);
void or_obs_actor(const or_cfg* c, const double* s, const double* hist, const double* noise,
                  double* o);
void or_priv(const or_cfg* c, const double* prm, const double* dist, double* priv);
void or_obs_critic(const or_cfg* c, const double* s, const double* hist, const double* priv,
                   double* o);
double or_reward(const or_reward_c* C, const double* s, const double* a);
void or_mlp_forward(const or_net* net, const double* P, const double* x, double* h1,
                    double* h2, double* y, int tanh_out);

int or_rollout(const or_cfg* c, const or_reward_c* C, or_envs* e, const double* actor,
               int hidden, int T, uint64_t t0, double sigma_e, const double* ext_actions,
               or_roll_out* out, int n_threads);
int or_td3_update(const or_cfg* c, or_td3* L, const or_buffer* b, or_td3_diag* d);
int or_recalc_rewards(const or_reward_c* C, or_buffer* b, const double* cur_state);
void or_curriculum(const double* factor, const double* target, double* C, int n);
int or_diff_run(const or_cfg* c, or_diff* d);
void or_lissajous(double t, double T, double A, double z0, double* p, double* v);
int or_track_run(const or_cfg* c, const or_track* J, int n_threads);
#ifdef __cplusplus
}
#endif
#endif
