/*
 * qsim.h -- C ABI of the GB300 quadrotor-training hot path of "Learning to Fly in
 * Seconds" (Eschmann, Albani, Loianno; arXiv 2311.13081).
 *
 * The library simulates batches of quadrotors (Sec. IV "Methodology": 17-D state
 * {p, q, v, omega, omega_m}, first-order motor lag, RK4 at 100 Hz), steps them with an
 * actor MLP and exploration noise, stores transitions in a device replay buffer and
 * trains an asymmetric TD3 actor-critic on them (Sec. IV; TD3 of Fujimoto et al. 2018),
 * including the reward curriculum and reward recalculation (Sec. IV, Sec. VI "Ablation
 * study"), many independent runs per launch, and reverse-mode gradients through the
 * simulator.
 *
 * Conventions for every entry point:
 *  - All sizes are element counts.  "Device pointer" means memory of the current CUDA
 *    device (e.g. torch.Tensor.data_ptr()); "host pointer" means pageable or pinned
 *    host memory.  Field-major layouts are written [field][env]: element (f, e) lives
 *    at f * ld + e, where ld is the padded env count returned by qsim_info().
 *  - Calls that take a `stream` (a cudaStream_t; NULL = legacy default stream) are
 *    asynchronous: argument errors found on the host return at once; device-side
 *    conditions (bounded waits that ran out, non-finite states) are recorded in the
 *    handle's status word and returned by qsim_sync()/ac_sync().
 *  - Nothing throws across the ABI.  On failure the return value is negative and
 *    qsim_last_error() holds a message (thread-local, owned by the library).
 *  - Handles own their device buffers (allocated at create, freed at destroy).  Pointer
 *    arguments stay owned by the caller and are only borrowed for the stream-ordered
 *    call.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QSIM_ABI_VERSION 1

typedef enum qsim_status {
    QSIM_OK = 0,
    QSIM_EINVAL = -1,   /* bad argument: null/misaligned pointer, size out of range */
    QSIM_ENOMEM = -2,   /* device allocation failed */
    QSIM_ECUDA = -3,    /* a CUDA call failed (message in qsim_last_error) */
    QSIM_ETIMEOUT = -4, /* a bounded device-side wait ran out */
    QSIM_ESTATE = -5,   /* handle not in a state that allows the call */
    QSIM_EVERSION = -6  /* checkpoint written by another ABI / layout */
} qsim_status;

/* Critic observation layouts (Sec. IV: the critic sees privileged information). */
typedef enum qsim_critic_layout {
    QSIM_CRITIC_HIST = 0,    /* actor obs (noise-free) + 4 normalised motor speeds        */
    QSIM_CRITIC_PRIV = 1,    /* ... + true mass, inertia, thrust coeff., motor T (rel.)  */
    QSIM_CRITIC_PAPER28 = 2, /* {p, R, v, omega, omega_m, f_r, tau_r}: the 28-D vector   */
    QSIM_CRITIC_ACTOR = 3    /* the actor's own observation, noise included: no privileged
                                information (Sec. VI ablation of the asymmetric critic)  */
} qsim_critic_layout;

/* Nominal vehicle (Sec. IV "standard dynamics of a quadrotor subject to motor delays";
 * values for the Crazyflie-class platform of the paper: 27 g, 0.15 s motor constant). */
typedef struct qsim_params {
    float mass;          /* kg */
    float J[3];          /* principal inertia, kg m^2 */
    float kf;            /* thrust per rotor = kf * rpm^2, N / rpm^2 */
    float km;            /* yaw torque per rotor = dir * km * thrust, m */
    float motor_tau;     /* first-order motor time constant, s */
    float rotor_pos[4][3]; /* body-frame rotor positions, m */
    float rotor_dir[4];  /* +1 / -1 yaw-torque sign per rotor */
    float rpm_min, rpm_max;
    float g;             /* m/s^2, world z up */
} qsim_params;

/* Environment-set configuration (Sec. IV MDP; constants of the supplement replaced by
 * the values documented with each field). */
typedef struct qsim_config {
    int32_t n_envs;          /* >= 1 */
    int32_t n_hist;          /* action-history length N_H, 0..16 (obs = 18 + 4 N_H) */
    int32_t episode_len;     /* truncation length in steps */
    int32_t critic_layout;   /* qsim_critic_layout */
    int32_t renorm_q;        /* renormalise q after each RK4 step (1) or not (0) */
    int32_t learning_starts; /* global steps with uniform random actions (TD3 warm-up) */
    int32_t replay_capacity; /* time slots per env in the replay ring (0 = no buffer) */
    int32_t motor_lag_off;   /* 1: no motor model (Sec. VI ablation "rotor delay"): the
                                rotors run at the clipped set-point from the start of each
                                step; 0: first-order lag.  Env-set kernels only
                                (qsim_dynamics_* and qsim_rollout_vjp always model the lag) */
    float dt;                /* integration step, s (0.01 = 100 Hz) */
    uint32_t run_id;         /* random-stream id of this run */
    uint64_t seed;           /* Philox key */
    /* initial-state distribution: p, attitude angles, v, omega uniform in +-range */
    float init_p, init_att, init_v, init_w, init_rpm_lo, init_rpm_hi;
    /* domain randomisation: relative half-widths and motor-time-constant range */
    float dr_mass, dr_J, dr_kf, tm_lo, tm_hi;
    /* per-episode force / torque disturbance half-widths (N, N m) */
    float dist_f, dist_tau;
    /* actor observation noise std-devs: position, rotation matrix, velocity, omega */
    float sig_p, sig_R, sig_v, sig_w;
    float term_pos;          /* episode terminates when any |p_i| exceeds this, m */
    /* reward constants C_rp C_rq C_rv C_rw C_ra C_rab C_rs (Sec. IV reward formula) */
    float reward[7];
    /* curriculum (Sec. IV): every `curriculum_interval` env interactions multiply each
     * constant by its factor until it reaches its target; the exploration std-dev is
     * multiplied by sigma_factor down to sigma_min.  interval 0 disables it. */
    float curriculum_factor[7];
    float curriculum_target[7];
    float sigma_e;           /* exploration std-dev at start */
    float sigma_factor, sigma_min;
    int32_t recalc_rewards;  /* recompute stored rewards after each change (1) */
    int64_t curriculum_interval;
} qsim_config;

typedef struct qsim_handle qsim_handle;
typedef struct ac_handle ac_handle;

/* Sizes and device pointers of an env set (for inspection and teacher forcing).
 * All arrays are field-major with leading dimension `ld` unless noted. */
typedef struct qsim_info {
    int32_t n_envs, ld;       /* env count and padded leading dimension (multiple of 32) */
    int32_t obs_dim;          /* actor observation dims, 18 + 4 N_H */
    int32_t critic_obs_dim;   /* critic observation dims without the action */
    int32_t record_fields;    /* floats per transition record: 17 s, 4 a, r, flags, priv */
    int32_t n_priv;
    int64_t capacity;         /* replay time slots */
    int64_t t_now;            /* global steps taken */
    int64_t head, size;       /* replay ring head (next slot) and filled slots */
    float* state;             /* [17][ld] p(3) q(4: w,x,y,z) v(3) omega(3) omega_m(4) */
    float* params;            /* [8][ld]  m Jx Jy Jz kf km T_m 0 */
    float* dist;              /* [6][ld]  f_r(3) tau_r(3) */
    float* hist;              /* [64][ld] a_{t-1} .. a_{t-16}, newest first */
    uint32_t* ep_index;       /* [ld] episodes started so far (random counter) */
    uint32_t* ep_step;        /* [ld] steps into the current episode */
    float* ep_ret;            /* [ld] return of the current episode */
    uint32_t* n_done;         /* [ld] completed episodes */
    uint32_t* len_sum;        /* [ld] sum of completed episode lengths */
    float* ret_sum;           /* [ld] sum of completed episode returns */
    float* records;           /* [capacity][record_fields][ld]; flags are uint32 bits:
                                 bit0 terminated, bit1 truncated, bits 8.. episode step */
    float* side;              /* [capacity][ld][17] s' where the episode ended (env-major) */
    float* reward_c;          /* [8] device: current C_* (7) and exploration std-dev */
} qsim_info;

/* ---------------------------------------------------------------- library / errors */
const char* qsim_last_error(void);
int32_t qsim_abi_version(void);
/* Plain cudaMemcpyAsync (kind = cudaMemcpyDefault) for bindings without a CUDA runtime. */
qsim_status qsim_memcpy(void* dst, const void* src, size_t bytes, void* stream);
qsim_status qsim_stream_sync(void* stream);

/* --------------------------------------------------------------------- random streams
 * Philox4x32-10 (Salmon et al., SC'11) with key = (seed lo, seed hi) and counter
 * (c0 = i, c1, tag << 24 | sub, run).  Writes n blocks of 4 uint32 to `out` (device).
 * kind 0: raw uint32; 1: uniforms ((x >> 9) + 1/2) 2^-23 as float bits;
 * 2: Box-Muller normals (cosine branch, two per block) as float bits. */
qsim_status qsim_philox_fill(uint64_t seed, uint32_t run, uint32_t tag, uint32_t sub,
                             uint32_t c1, int32_t n, int32_t kind, uint32_t* out,
                             void* stream);
/* Host-side Philox (same stream) for small draws such as per-run hyper-parameters. */
void qsim_philox_host(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ------------------------------------------------------------------------- dynamics
 * One or more teacher-forced RK4 steps (Sec. IV dynamics; Sec. V 100 Hz) of n
 * independent bodies with the RPM set-point `rpm` held constant:
 *   state_in/out [17][ld], params [8][ld] (m Jx Jy Jz kf km T_m -), dist [6][ld] or
 *   NULL (no disturbance), rpm [4][ld].  All device pointers, 16-byte aligned, ld >= n
 *   and a multiple of 4.  state_out may alias state_in.  Vehicle geometry comes from
 *   `veh` (host pointer).  renorm: renormalise q after each step. */
qsim_status qsim_dynamics_step(const qsim_params* veh, const float* params, const float* dist,
                               const float* state_in, const float* rpm, float dt,
                               int32_t renorm, int32_t n, int32_t ld, int32_t n_steps,
                               float* state_out, void* stream);

/* Dynamics-only throughput kernel in the shape of the paper's simulator benchmark
 * (Sec. V "Simulation": envs x steps of forward dynamics, no policy): every env holds
 * its state in registers for n_steps RK4 steps at the hover set-point of `veh`;
 * final states are written to state_out [17][ld] (device). */
qsim_status qsim_dynamics_bench(const qsim_params* veh, int32_t n, int32_t ld,
                                int32_t n_steps, float dt, float* state_out, void* stream);

/* ----------------------------------------------------------------------- env sets
 * qsim_create allocates n_envs environments (+ a replay ring when replay_capacity > 0)
 * on the current device and resets every env to episode 0 (state, domain-randomised
 * parameters, disturbance, empty history).  Synchronous. */
qsim_status qsim_create(const qsim_config* cfg, const qsim_params* veh, qsim_handle** out);
qsim_status qsim_destroy(qsim_handle* h);
qsim_status qsim_info_get(const qsim_handle* h, qsim_info* out);
/* Overwrite host-side counters (used when teacher-forcing a buffer): t_now, head, size. */
qsim_status qsim_set_counters(qsim_handle* h, int64_t t_now, int64_t head, int64_t size);
/* Device status word: QSIM_OK or the first device-side error since the last call
 * (synchronous; clears the word): QSIM_ETIMEOUT when a bounded wait of the tensor-core
 * rollout ran out, QSIM_ESTATE when it met a value outside the half-precision range or
 * not finite. */
qsim_status qsim_sync(qsim_handle* h);

/* Polls a bounded device-side wait of this env set's kernels makes before it gives up:
 * the tensor-core rollout's hand-over waits between its compute and MMA warps and its
 * waits for the previous chunk of an env group (1..2^30; 0 restores the default 2^22).
 * A wait that runs out records QSIM_ETIMEOUT for qsim_sync; every warp of the block then
 * leaves its step loop, the MMAs already committed are allowed to finish (a separate wait
 * of the default length), tensor memory is released and the kernel returns, so later
 * calls run normally.  The env set's contents are then those of a partly completed call
 * (unspecified, finite if the inputs were), with the counters advanced as for a full
 * call.  A limit far below the
 * MMA latency (a few thousand cycles) makes the waits run out on purpose, which is how
 * the failure path is tested.  Returns the previous limit, or a negative qsim_status.
 * (No counterpart in the paper.) */
int32_t qsim_set_wait_limit(qsim_handle* h, int32_t polls);

/* Debug bounds checks (no counterpart in the paper).  The library built with
 * -DQSIM_BOUNDS_CHECK=1 (paper_2311_13081_gb300.build.build(bounds_check=True), a separate
 * shared object) checks every replay-ring slot and SoA env index that a kernel computes
 * before it reads or writes the ring (rollouts, env step, learner env step and replay
 * gather, reward recalculation) against the allocation; the first index outside [0, n)
 * skips that access and is reported by qsim_sync as QSIM_ESTATE, with the site, the index
 * and n in qsim_last_error().  qsim_bounds_checked() returns 1 in that build, 0 otherwise.
 * qsim_bounds_probe reads the packed flag word of (slot, env) into *flags_out (device,
 * 4 bytes) through the same check: in the checked build an index outside the ring is
 * passed to the kernel, which records it and skips the read; in the default build it is
 * refused on the host with QSIM_EINVAL.  Asynchronous on `stream`. */
int32_t qsim_bounds_checked(void);
qsim_status qsim_bounds_probe(qsim_handle* h, int64_t slot, int64_t env, uint32_t* flags_out,
                              void* stream);

/* Actor and critic observations of the current states (Sec. IV: o_a = {p, R, v, omega,
 * H} with noise of the current step; o_c privileged and noise-free, except in the
 * symmetric layout QSIM_CRITIC_ACTOR, where o_c = o_a).  obs_a
 * [obs_dim][ld], obs_c [critic_obs_dim][ld] (either may be NULL); device pointers. */
qsim_status qsim_observe(qsim_handle* h, float* obs_a, float* obs_c, void* stream);

/* One environment step with external normalised actions [4][ld] in [-1,1] (clipped):
 * RPM set-point, RK4, reward, termination/truncation, transition write into the replay
 * ring, history update, reset of finished envs.  Outputs (device, any may be NULL):
 * reward [ld], terminated [ld], truncated [ld] (uint8), and the observations of the
 * next step as qsim_observe would return them. */
qsim_status qsim_step(qsim_handle* h, const float* actions, float* obs_a, float* obs_c,
                      float* reward, uint8_t* terminated, uint8_t* truncated, void* stream);

/* Fused rollout of n_steps steps for every env (the ENV STEP of the hot path): actor
 * MLP (obs_dim -> hidden -> hidden -> 4, ReLU/ReLU/tanh; parameters `actor` in the
 * layout W1[h][in] b1 W2[h][h] b2 W3[4][h] b3, device) with Gaussian exploration of
 * std-dev sigma_e (sigma_e < 0: the handle's current value) or uniform warm-up actions
 * while t < learning_starts, then RK4 dynamics, reward, termination, reset and the
 * transition write.  hidden is 32, 64 or 128 (every width runs on the SIMT kernel; 64
 * also on the tensor-core kernel, see qsim_rollout_engine). */
qsim_status qsim_rollout(qsim_handle* h, const float* actor, int32_t hidden, int32_t n_steps,
                         float sigma_e, void* stream);

/* Simulated trajectory tracking (Sec. V "Trajectory tracking"): every env of the set flies
 * the deterministic actor (no exploration, no observation noise) along the figure-eight
 * target p*(t) = (A cos(2 pi t / T), (A / 2) sin(4 pi t / T), z0) for n_steps steps of dt,
 * with its own domain-randomised parameters and disturbances (the set's current ones).  As
 * Sec. IV prescribes for set-points, the actor observes its position and velocity offset
 * by the target's p*(t) and velocity v*(t) (the time derivative of p*), each component
 * clipped to +-clip_p (m) and +-clip_v (m/s).  Start: on the target with its velocity, level, not rotating, motors at
 * the env's hover speed sqrt(m g / (4 k_f)) clipped to the RPM range, empty action history.
 * After each step the error e = p - p*(t + dt) is accumulated; a non-finite state or any
 * |e_i| > term_pos (the config's termination box) ends that env's flight, whose error is
 * not counted.  The env set itself (states, counters, replay) is not modified.
 *   actor     device, layout as in qsim_rollout; hidden 32, 64 or 128.  Hidden 64 flies on
 *             the tensor-core kernel (its state in scratch allocated on `stream` with
 *             cudaMallocAsync for the call) unless qsim_rollout_engine pins engine 0 or 1;
 *             the other widths, and pinned SIMT engines, on the SIMT kernel.  The two
 *             engines agree to FP32 rounding, not bitwise.
 *   period    device float [ld]: cycle time T > 0 of each env, s (T <= 0, infinite or NaN
 *             flies no step)
 *   sq_err    device double [2][ld] out: sum of |e|^2 and sum of e_x^2 + e_y^2 over the
 *             completed steps; RMSE = sqrt(sq_err / steps_ok) (the paper's e and e_xy)
 *   steps_ok  device int32 [ld] out: steps completed before the flight ended (<= n_steps)
 * Pointers must be 4-byte aligned (sq_err 8-byte); amplitude, z0 and the clips finite,
 * clips >= 0; otherwise QSIM_EINVAL. */
qsim_status qsim_track(qsim_handle* h, const float* actor, int32_t hidden, int32_t n_steps,
                       const float* period, float amplitude, float z0, float clip_p,
                       float clip_v, double* sq_err, int32_t* steps_ok, void* stream);

/* Warps per block for the rollout kernel (0 = autotuned choice).  Returns the value in
 * effect. */
int32_t qsim_rollout_tune(qsim_handle* h, int32_t warps_per_block);

/* Rollout schedule: split the envs into `parts` partitions (1..4) run on internal streams,
 * each advancing in chunks of `chunk` steps (0 = whole call), joined on the caller's stream
 * at the end of every qsim_rollout call.  Partitions keep the SMs busy while another
 * partition's last blocks finish.  parts 0 = automatic (2 partitions in 100-step chunks
 * when the env set needs more than one wave of resident warps).  Returns the parts in
 * effect; a negative argument leaves that setting unchanged. */
int32_t qsim_rollout_schedule(qsim_handle* h, int32_t parts, int32_t chunk);

/* Rollout kernel variant: packed = 1 uses Blackwell's paired FP32 FMA (fma.rn.f32x2: two
 * single-precision FMAs per instruction, results identical to the scalar kernel), 0 the
 * scalar kernel, -1 automatic (see qsim_rollout_engine).  Returns the
 * setting in effect. */
int32_t qsim_rollout_packed(qsim_handle* h, int32_t packed);  /* engines 0/1 of qsim_rollout_engine */

/* Rollout engine: 0 the SIMT kernel (scalar FMA), 1 the SIMT kernel with paired FMA (same
 * results as 0), 2 the tensor-core kernel (hidden = 64 only: the two hidden layers as
 * tcgen05 fp16 MMAs on hi/lo halves of every operand, three products per layer that keep
 * FP32 accuracy, accumulators in tensor memory, 384 envs per block; results agree with 0
 * to FP32 rounding, not bitwise; an actor weight of W1 or W2, actor input or hidden
 * activation of magnitude >= 65504 or not finite is reported by qsim_sync as QSIM_ESTATE),
 * -1 automatic (the autotuner's choice once it has run; before that the tensor-core engine
 * at hidden 64 and the paired-FMA SIMT kernel otherwise).  Any other value
 * leaves the setting unchanged.  Returns the setting in effect.  The paper's environment
 * step has no counterpart of this switch: it selects among kernels computing the same step
 * (Sec. IV: the quadrotor dynamics and the actor). */
int32_t qsim_rollout_engine(qsim_handle* h, int32_t engine);

/* Autotuner: times every (warps-per-block, schedule) variant of the rollout kernel that fits
 * on this device with n_steps-step rollouts (CUDA events on `stream`; these are real env
 * steps that advance the env set), keeps the fastest for this handle and returns its warps
 * per block (negative qsim_status on error).  Synchronises the stream. */
int32_t qsim_rollout_autotune(qsim_handle* h, const float* actor, int32_t hidden,
                              int32_t n_steps, void* stream);

/* FP32 FMA throughput probe: every thread of n_blocks x 256 runs |iters| iterations of 16
 * independent FMA chains (iters < 0: paired f32x2 FMAs, 2 per instruction); out is a
 * device scratch word.  Used to confirm the FP32 roofline peak. */
qsim_status qsim_ffma_probe(int32_t n_blocks, int32_t iters, float* out, void* stream);

/* Tensor-core issue-rate probe (one block): n_warps (1..4) warps each issue a chain of n_mma
 * (1..4096) tcgen05.mma instructions (kind::f16, M 128, N = n_cols / n_warps (a multiple of
 * 16, n_cols <= 256), K 16, zero operands) into disjoint accumulator columns; *cycles
 * (device int64) receives the SM cycles from the first issue until every chain has
 * completed, or -1 if the completion wait ran out.  Shows that one issuing thread completes
 * one such MMA per ~65 cycles for any N <= 128 while chains of several warps overlap, which
 * shapes the tensor-core rollout (no counterpart in the paper). */
qsim_status qsim_mma_probe(int32_t n_mma, int32_t n_cols, int32_t n_warps, int64_t* cycles, void* stream);

/* Recompute every stored reward from (s', a) with the current reward constants (Sec. VI
 * reward recalculation). */
qsim_status qsim_recalc_rewards(qsim_handle* h, void* stream);
/* The same for n env sets (1..65535, all on the current device) in one launch, each with
 * its own constants; results equal qsim_recalc_rewards on each set.  The launch's set
 * descriptors are staged in memory allocated on `stream` (cudaMallocAsync, freed in
 * stream order). */
qsim_status qsim_recalc_rewards_batch(qsim_handle* const* hs, int32_t n, void* stream);
/* Set the current reward constants (7 floats) and exploration std-dev (host values). */
qsim_status qsim_set_reward(qsim_handle* h, const float c[7], float sigma_e, void* stream);

/* Reduced episode statistics (host out; synchronises the stream). */
typedef struct qsim_stats {
    int64_t episodes;       /* completed episodes */
    double mean_length;     /* mean completed-episode length, steps */
    double mean_return;     /* mean completed-episode return */
} qsim_stats;
qsim_status qsim_stats_get(qsim_handle* h, qsim_stats* out, void* stream);

/* ---------------------------------------------------------------------- learner
 * TD3 with an asymmetric critic (Sec. IV; TD3): actor obs_dim -> H -> H -> 4 (tanh),
 * twin critics (critic_obs_dim + 4) -> H -> H -> 1, target networks, Adam. */
typedef struct ac_config {
    int32_t hidden;          /* H in {32, 64, 128} (any multiple of 32 up to 128) */
    int32_t batch;           /* minibatch B, multiple of 32, <= 1024 */
    int32_t policy_delay;    /* actor + target update every d-th critic update */
    int32_t updates_per_step;/* updates per env step in ac_train (update-to-data) */
    float gamma, tau, lr, beta1, beta2, eps;
    float sigma_target;      /* target-policy smoothing std-dev */
    float noise_clip;        /* smoothing noise clip */
    int32_t cluster;         /* CTAs that cooperate on one update (1..16; 0 = auto: 16 for up
                                to 8 runs, 2 for up to 63, 1 beyond, halved while a CTA would
                                get < 16 samples; ac_train_autotune sets the timed best) */
    int32_t reserved0;
} ac_config;

/* Sizes and device pointers of a learner (all float32, device). */
typedef struct ac_info {
    int32_t obs_dim, critic_in, hidden, batch;
    int32_t n_actor, n_critic;      /* parameter counts */
    int64_t t_actor, t_critic;      /* Adam steps taken */
    int64_t updates;                /* updates taken (random counter) */
    float *actor, *actor_t, *c1, *c1_t, *c2, *c2_t;
    float *m_a, *v_a, *m_c1, *v_c1, *m_c2, *v_c2;
    float* stats;                   /* [4] last critic loss, last actor loss, -, - */
} ac_info;

/* Create a learner sized for env set `env` (observation layouts), initialise the three
 * online networks with PyTorch-style U(+-1/sqrt(fan_in)) from Philox tag 7 (networks
 * 0 actor, 1 critic 1, 2 critic 2) and copy them into the targets.  Synchronous. */
qsim_status ac_create(const ac_config* cfg, const qsim_handle* env, ac_handle** out);
qsim_status ac_destroy(ac_handle* a);
qsim_status ac_info_get(const ac_handle* a, ac_info* out);
qsim_status ac_set_counters(ac_handle* a, int64_t t_actor, int64_t t_critic, int64_t updates);

/* n_updates TD3 updates (the AC UPDATE of the hot path): minibatch sample + gather from
 * `env`'s replay ring, target actor + smoothing, twin target critics, critic regression,
 * Adam on the critics, and every policy_delay-th update the actor gradient through
 * critic 1, Adam on the actor and Polyak averaging of all targets (Sec. IV; TD3).
 * One launch on a cluster of the learner's single-run size (ac_config.cluster).
 * Asynchronous: the learner keeps a device workspace (its run descriptor and the
 * cluster's scratch) between calls, allocated with cudaMalloc on the first call and
 * whenever a later call needs a larger one, and the host advances its copy of the
 * counters without reading the device.  Calls on one learner (ac_update, ac_train,
 * ac_update_static) must be ordered on the GPU: one stream, or streams ordered by events.
 * The learner and the env set must belong to the current device (else QSIM_EINVAL). */
qsim_status ac_update(ac_handle* a, qsim_handle* env, int32_t n_updates, void* stream);

/* Debug output of the replay sampler: while idx is non-null (device, batch uint32,
 * 4-byte aligned), every update writes the flat index k * n_envs + env of each minibatch
 * sample j (k = time slot counted from the oldest sampled slot) to idx[j], so the latest
 * update's indices can be compared with the reference sampler bit for bit.  NULL turns
 * the log off.  Affects launches issued after the call. */
qsim_status ac_set_index_log(ac_handle* a, uint32_t* idx);

/* Set the learner's cluster size (CTAs per update: 0 = automatic, else a power of two
 * <= 16), as ac_config.cluster.  Returns the previous setting, or a negative
 * qsim_status. */
int32_t ac_set_cluster(ac_handle* a, int32_t cluster);

/* Allocation-free variant of ac_update, for callers that cannot allocate device memory
 * while they run updates -- for example an embedded trainer that reserves all memory up
 * front, code running under a custom allocator that forbids cudaMalloc, or a host thread
 * that must not take the driver's allocation locks.  The paper has no counterpart; this is
 * a deployment convenience of this library.  Same arguments, semantics and results as
 * ac_update; the learner and env handles still supply every input and output.
 * Differences:
 *  - Scratch (activations, partial gradients, the run descriptor) lives in a static
 *    device array of QSIM_STATIC_SCRATCH_BYTES (+ QSIM_STATIC_DESC_BYTES) that every GPU
 *    which loads the library holds until the process exits.  Configurations needing more
 *    scratch (large batch x hidden, see the error message) return QSIM_EINVAL.
 *  - The call makes no cudaMalloc / cudaFree and calls no allocating library routine.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before any
 *    stream capture.  The address is kept for the life of the process: like every
 *    handle of this library, it does not survive a cudaDeviceReset.
 *  - Every call shares the one array: calls whose work overlaps on the GPU (other streams,
 *    other threads) race and must be serialised by the caller.  The array keeps the last
 *    call's contents; nothing in it needs to start at zero.
 *  - The run descriptor is copied from host stack memory into the array on every call
 *    (cudaMemcpyAsync from pageable memory). */
#define QSIM_STATIC_SCRATCH_BYTES (8u << 20)
#define QSIM_STATIC_DESC_BYTES (4u << 10)
qsim_status ac_update_static(ac_handle* a, qsim_handle* env, int32_t n_updates, void* stream);

/* Train n_runs independent runs for steps_per_run env steps each: per step, the fused
 * env step of each run's envs (actor, exploration, dynamics, reward, reset, transition
 * write) followed by updates_per_step updates once the buffer allows sampling, plus the
 * curriculum with reward recalculation when configured (Sec. IV, Sec. VI).
 *   persistent = 1: one persistent launch of all the steps for all runs (clusters of the
 *     size every run shares walk the runs longest first; ac_plan_* below captures such a
 *     launch in a CUDA graph for repeated use);
 *   persistent = 0: the plain form: the same kernel launched per run and per step;
 *   persistent = 2: one launch per run for all of its steps, runs one after another.
 * Forms 0 and 2 give each run its own single-run cluster size (as ac_update); a single
 * run with persistent = 1 runs as form 2.  Results are bit-identical between the forms
 * whenever the cluster sizes agree (e.g. ac_config.cluster set); otherwise they differ in
 * the order of the cross-CTA gradient sums (FP32 rounding).  Asynchronous for a single
 * run and in forms 0 and 2 (the learners' workspaces, as ac_update); the multi-run
 * persistent form allocates its descriptors and scratch on `stream` (cudaMallocAsync,
 * freed in stream order), without synchronising. */
qsim_status ac_train(ac_handle* const* runs, qsim_handle* const* envs, int32_t n_runs,
                     int64_t steps_per_run, int32_t persistent, void* stream);

/* Autotuner of the batched launch: times the persistent ac_train over trial_steps steps
 * for every cluster size S in {1, 2, 4, 8, 16} (CTAs per run) that divides every run's
 * batch with at least 16 samples per CTA (S = 1 always qualifies), after one untimed call
 * with the current setting, with CUDA events on `stream`, and sets every run's cluster
 * size to the fastest (what ac_config.cluster = S would have chosen).  The trials are real
 * training steps: every run advances by (1 + number of candidates) x trial_steps steps.
 * Results depend on S only through the order of the cross-CTA gradient reduction (FP32
 * rounding); for a fixed S they are reproducible bit for bit.  Returns the chosen S, or a
 * negative qsim_status (the runs keep their previous setting).  Synchronises the stream.
 * The paper has no counterpart: it trains one run on a CPU. */
int32_t ac_train_autotune(ac_handle* const* runs, qsim_handle* const* envs, int32_t n_runs,
                          int32_t trial_steps, void* stream);
qsim_status ac_sync(ac_handle* a);

/* Graph-captured batched training.  ac_plan_create builds, once, everything ac_train's
 * persistent form builds per call (run descriptors, per-cluster scratch, the longest-
 * processing-time-first run schedule) and captures one persistent launch of
 * steps_per_chunk steps for all runs into a CUDA graph (synchronous).  ac_plan_run replays
 * it n_chunks times on `stream` (asynchronous); the runs' counters advance in device memory,
 * so consecutive replays continue where the last one stopped.  ac_plan_sync copies the
 * counters back into the handles (synchronises `stream`); call it before using the handles
 * with any other entry point.  The handles must outlive the plan and must not be used by
 * other calls between ac_plan_create and ac_plan_sync. */
typedef struct ac_plan ac_plan;
qsim_status ac_plan_create(ac_handle* const* runs, qsim_handle* const* envs, int32_t n_runs,
                           int32_t steps_per_chunk, ac_plan** out);
qsim_status ac_plan_run(ac_plan* p, int32_t n_chunks, void* stream);
qsim_status ac_plan_sync(ac_plan* p, void* stream);
qsim_status ac_plan_destroy(ac_plan* p);

/* Checkpoint: weights, targets, Adam moments and counters, the env set's states and
 * counters and current reward constants (not the replay buffer).  Versioned binary. */
qsim_status ac_save(const ac_handle* a, const qsim_handle* env, const char* path);
qsim_status ac_load(ac_handle* a, qsim_handle* env, const char* path);

/* ------------------------------------------------------------------ differentiation
 * Reverse-mode gradient through an H-step RK4 rollout of n envs without resets or
 * disturbances (differentiable form of the Sec. IV dynamics):
 *   loss_e = sum_{t=1..H} [w_p |p_t|^2 + w_q (1 - q_w,t^2) + w_v |v_t|^2]
 *            + w_a sum_{t=0..H-1} |a_t|^2
 * mode 0 (open loop): actions [H][4][ld] given (normalised, mapped linearly to RPM and
 * clipped to the RPM range); g_actions [H][4][ld] receives d L / d a_t.
 * mode 1 (closed loop): a_t = actor(o_a,t), o_a built from the state and the rollout's
 * own previous n_hist actions (zeros before t = 0, no noise); g_actor [P_actor] receives
 * d L / d actor (summed over envs; overwritten).
 * L = sum_e seed_e loss_e with seed [ld] (device; NULL = all ones), so a caller can pass
 * the upstream gradient of each env's loss.  Both modes write loss [ld] (unweighted),
 * d L / d (m, Jx, Jy, Jz) into g_params [4][ld], and the actions used into actions_out
 * [H][4][ld] (either may be NULL).  If g_actions, g_actor and g_params are all NULL only
 * the forward pass runs.
 * States are checkpointed every `ckpt` steps and recomputed inside each segment, so the
 * workspace (device, 16-byte aligned, qsim_vjp_workspace() bytes, caller-owned) grows with
 * H/ckpt + ckpt, not H.  s0 [17][ld], params [8][ld] (m Jx Jy Jz kf km T_m -).
 * Asynchronous on `stream`.  In closed loop with g_actor, each segment's weight gradient
 * runs on an internal low-priority stream of the calling host thread (created on its first
 * such call on the device) while the next segment's reverse sweep runs; it forks from and
 * joins back into `stream` through events, so the call completes in `stream` order and
 * can be captured in a CUDA graph once that stream exists (make one uncaptured call first).
 * Like every handle of this library, that stream does not survive a cudaDeviceReset.
 * Results are bitwise reproducible for a given descriptor. */
typedef struct qsim_vjp_desc {
    int32_t n, ld, H, ckpt, mode, n_hist, hidden;
    int32_t lanes_per_env;  /* closed loop at hidden 32 / 64 with <= 96 actor inputs: lanes
                               that share one env (32, 16 or 8; 0 = automatic, 8); each
                               group integrates its env redundantly and splits the actor's
                               layers over its lanes.  Results agree between settings to FP32
                               rounding (the order of the group sums differs). */
    float w_p, w_q, w_v, w_a;
    float dt;
    int32_t renorm;
} qsim_vjp_desc;
size_t qsim_vjp_workspace(const qsim_vjp_desc* d);
qsim_status qsim_rollout_vjp(const qsim_vjp_desc* d, const qsim_params* veh, const float* s0,
                             const float* params, const float* actions, const float* actor,
                             const float* seed, float* loss, float* g_actions, float* g_actor,
                             float* g_params, float* actions_out, void* workspace, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
