"""Workload presets and seeded synthetic-input generators.

This module holds configuration VALUES (vehicle constants, ranges, hyper-parameters) and
seeded numpy generators for test inputs.  It holds none of the method's arithmetic and
serves both the CUDA library's tests/benchmark and the oracle, which share nothing else.

Presets follow the five workloads the method is exercised on:
  c1  plain single run: 1 env, fixed Crazyflie-class parameters, 10,000 steps, batch 256
  c2  batched rollout: 65,536 envs x 1,000 steps, per-env domain randomisation
  c3  differentiation: 4,096 envs, 200-step horizon, checkpoint every 20 steps
  c4  batched training: 512 runs, widths {32,64,128}, batches {128,256,512}, 8 envs/run
  c5  asymmetric critic + curriculum: 128 runs x 64 envs, privileged critic, 300,000 steps
"""
from __future__ import annotations

import math

import numpy as np

ARM = 0.028
_A = ARM / math.sqrt(2.0)

# Crazyflie-class nano quadrotor (27 g), X configuration, rotors ordered front-right,
# back-right, back-left, front-left (x forward, y left, z up), alternating spin.
VEHICLE = dict(
    mass=0.027, Jx=1.4e-5, Jy=1.4e-5, Jz=2.2e-5, kf=3.16e-10, km=0.005, tm=0.15,
    rotor_pos=[_A, -_A, 0.0, -_A, -_A, 0.0, -_A, _A, 0.0, _A, _A, 0.0],
    rotor_dir=[-1.0, 1.0, -1.0, 1.0],
    rpm_min=0.0, rpm_max=21702.0, g=9.81,
)


def hover_rpm(v=VEHICLE) -> float:
    """RPM at which four rotors carry the weight: k_f w^2 * 4 = m g."""
    return math.sqrt(v["mass"] * v["g"] / (4.0 * v["kf"]))


def hover_action(v=VEHICLE) -> float:
    """Normalised action of the hover RPM under the linear action -> RPM map."""
    return 2.0 * (hover_rpm(v) - v["rpm_min"]) / (v["rpm_max"] - v["rpm_min"]) - 1.0


# reward constants C_rp C_rq C_rv C_rw C_ra C_rab C_rs (builder defaults; the paper's
# values are in a supplement that is not available)
REWARD = [1.0, 1.0, 0.1, 0.01, 0.01, hover_action(), 1.5]

SIM = dict(
    dt=0.01, renorm_q=1, n_hist=16, episode_len=500, critic_layout=0,
    init_p=0.2, init_att=math.radians(30.0), init_v=1.0, init_w=1.0,
    init_rpm_lo=0.0, init_rpm_hi=21702.0,
    dr_mass=0.0, dr_J=0.0, dr_kf=0.0, tm_lo=0.15, tm_hi=0.15,
    dist_f=0.0, dist_tau=0.0,
    sig_p=0.0, sig_R=0.0, sig_v=0.0, sig_w=0.0,
    term_pos=0.6, seed=0, run_id=0, learning_starts=1000,
)

DR = dict(dr_mass=0.2, dr_J=0.2, dr_kf=0.1, tm_lo=0.03, tm_hi=0.15)

TD3 = dict(gamma=0.99, tau=0.005, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, sigma_t=0.2,
           noise_clip=0.5, policy_delay=2, batch=256, hidden=64, sigma_e=0.1)

# Curriculum on the action weight: 0.01 -> 0.5 in three multiplicative steps, one per
# 100,000 steps; exploration noise decays with the inverse factor down to a floor.
CURRICULUM = dict(interval=100_000,
                  factor=[1.0, 1.0, 1.0, 1.0, (0.5 / 0.01) ** (1.0 / 3.0), 1.0, 1.0],
                  target=[1.0, 1.0, 0.1, 0.01, 0.5, REWARD[5], 1.5],
                  sigma_factor=(0.01 / 0.5) ** (1.0 / 3.0), sigma_min=0.02)


# Ablation study (Sec. VI): the full method and the variants that each remove one
# component (the last removes two).  The observation-noise and disturbance scales of the
# full method are the builder's values (the paper's are in the unavailable supplement).
ABLATION_BASE = dict(critic_layout=0, sig_p=0.002, sig_R=0.01, sig_v=0.01, sig_w=0.01,
                     dist_f=0.0027, dist_tau=1.0e-6, motor_lag_off=0, learning_starts=1000)
ABLATIONS = {
    "all_components": {},
    "observation_noise": dict(sig_p=0.0, sig_R=0.0, sig_v=0.0, sig_w=0.0),
    "reward_recalculation": dict(recalc_rewards=0),
    "exploration_noise_decay": dict(sigma_factor=1.0),
    "disturbances": dict(dist_f=0.0, dist_tau=0.0),
    "asymmetric_actor_critic": dict(critic_layout=3),
    "action_history": dict(n_hist=0),
    "curriculum": dict(curriculum=False),
    "rotor_delay": dict(motor_lag_off=1),
    "aac_and_curriculum": dict(critic_layout=3, curriculum=False),
}


def ablation(name: str):
    """(sim config, curriculum, recalc_rewards) of one variant of the ablation study.
    Without the curriculum the reward constants keep their initial values while the
    exploration noise still decays; without the decay the noise stays at its start value."""
    c = config("c2")
    c.update(ABLATION_BASE)
    v = dict(ABLATIONS[name])
    cur = dict(CURRICULUM)
    if v.pop("curriculum", True) is False:
        cur["factor"] = [1.0] * 7
        cur["target"] = list(REWARD)
    if "sigma_factor" in v:
        cur["sigma_factor"] = v.pop("sigma_factor")
    recalc = v.pop("recalc_rewards", 1)
    c.update(v)
    return c, cur, recalc


def config(name: str = "c1") -> dict:
    """Full simulation config (vehicle + sim + preset overrides) as a plain dict."""
    c = dict(VEHICLE)
    c.update(SIM)
    if name in ("c2", "c5"):
        c.update(DR)
    if name == "c5":
        c["critic_layout"] = 1
    if name == "c3":
        c["learning_starts"] = 0
    return c


PRESETS = {
    "c1": dict(n_envs=1, steps=10_000, batch=256, capacity=10_000, hidden=64, seed=0),
    "c2": dict(n_envs=65_536, steps=1_000, capacity=1_000, hidden=64, seed=0, sigma_e=0.1),
    "c3": dict(n_envs=4_096, horizon=200, ckpt=20, hidden=64, weights=(1.0, 0.1, 0.1, 0.01)),
    "c4": dict(n_runs=512, n_envs=8, steps=100_000, widths=(32, 64, 128),
               batches=(128, 256, 512)),
    "c5": dict(n_runs=128, n_envs=64, steps=300_000, capacity_per_run=1_000_000, hidden=64),
}


# ---------------------------------------------------------------------------------------
# Seeded generators (numpy PCG64) for test inputs
# ---------------------------------------------------------------------------------------
def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_quat(g: np.random.Generator, n: int) -> np.ndarray:
    q = g.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def random_states(seed: int, n: int, p=0.2, v=1.0, w=1.0, rpm=(0.0, 21702.0)) -> np.ndarray:
    """[n][17] states with the magnitudes of the initial-state distribution."""
    g = rng(seed)
    s = np.zeros((n, 17))
    s[:, 0:3] = g.uniform(-p, p, (n, 3))
    s[:, 3:7] = random_quat(g, n)
    s[:, 7:10] = g.uniform(-v, v, (n, 3))
    s[:, 10:13] = g.uniform(-w, w, (n, 3))
    s[:, 13:17] = g.uniform(rpm[0], rpm[1], (n, 4))
    return s


def random_params(seed: int, n: int, v=VEHICLE, rel=0.2) -> np.ndarray:
    """[n][8] per-env params around the nominal vehicle."""
    g = rng(seed)
    P = np.zeros((n, 8))
    P[:, 0] = v["mass"] * g.uniform(1 - rel, 1 + rel, n)
    P[:, 1] = v["Jx"] * g.uniform(1 - rel, 1 + rel, n)
    P[:, 2] = v["Jy"] * g.uniform(1 - rel, 1 + rel, n)
    P[:, 3] = v["Jz"] * g.uniform(1 - rel, 1 + rel, n)
    P[:, 4] = v["kf"] * g.uniform(1 - rel / 2, 1 + rel / 2, n)
    P[:, 5] = v["km"]
    P[:, 6] = g.uniform(0.03, 0.15, n)
    return P


def nominal_params(n: int, v=VEHICLE) -> np.ndarray:
    P = np.zeros((n, 8))
    P[:, 0], P[:, 1], P[:, 2], P[:, 3] = v["mass"], v["Jx"], v["Jy"], v["Jz"]
    P[:, 4], P[:, 5], P[:, 6] = v["kf"], v["km"], v["tm"]
    return P


def random_actions(seed: int, shape, lo=-1.0, hi=1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, shape)


def random_net(seed: int, size: int, scale: float) -> np.ndarray:
    return rng(seed).uniform(-scale, scale, size)
