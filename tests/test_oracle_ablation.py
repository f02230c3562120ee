"""Pins of the oracle's ablation switches (Sec. VI, ablation study): the motor model switched
off ("rotor delay" removed) and the symmetric critic (asymmetric actor-critic removed).

The other ablations of the study are configuration values whose effect the existing pins
already cover (no action history: n_hist 0; no curriculum: reward factors 1 with the
exploration decay kept; no reward recalculation: recalc off; no disturbances /
observation noise: zero scales; no exploration-noise decay: sigma factor 1); the last test
pins that each preset changes only its component.
"""
import copy

import numpy as np
import pytest

import oracle as O
import workloads as W
from test_oracle_learner import hyper, make_buffer, make_learner, small_cfg


def level_rest_envs(c, n, rpm):
    e = O.new_envs(c, np.arange(n))
    e["s"][:] = 0.0
    e["s"][:, 3] = 1.0
    e["s"][:, 13:] = rpm
    e["prm"][:] = [c["mass"], c["Jx"], c["Jy"], c["Jz"], c["kf"], c["km"], c["tm"], 0.0]
    e["dist"][:] = 0.0
    return e


def test_without_motor_lag_the_thrust_is_there_at_once():
    """From rest with the rotors stopped, hover set-points hold the vehicle exactly when the
    motors follow at once; with the first-order lag it first drops."""
    T = 12
    acts = np.full((T, 1, 4), W.hover_action())
    for off in (1, 0):
        c = small_cfg(motor_lag_off=off, term_pos=10.0, episode_len=1000)
        e = level_rest_envs(c, 1, 0.0)
        rec = O.rollout(c, W.REWARD, e, T, 0, ext_actions=acts)
        if off:
            assert np.allclose(e["s"][0, :3], 0.0, atol=1e-12)
            assert np.allclose(e["s"][0, 7:10], 0.0, atol=1e-12)
            assert np.allclose(e["s"][0, 13:], W.hover_rpm(), rtol=1e-12)
            # the stored state before step 1 already carries the set-point speeds
            assert np.allclose(rec["rec_s"][1, 0, 13:], W.hover_rpm(), rtol=1e-12)
        else:
            assert e["s"][0, 9] < -0.05  # fell while the rotors spun up


def test_without_motor_lag_constant_thrust_closed_form():
    """Constant thrust from the first instant: z(t) = (4 k_f u^2 / m - g) t^2 / 2 and
    v_z = (4 k_f u^2 / m - g) t, which RK4 integrates exactly."""
    c = small_cfg(motor_lag_off=1, term_pos=10.0, episode_len=1000)
    u_rpm = 1.1 * W.hover_rpm()
    a = 2.0 * (u_rpm - c["rpm_min"]) / (c["rpm_max"] - c["rpm_min"]) - 1.0
    T = 7
    e = level_rest_envs(c, 1, 3000.0)
    O.rollout(c, W.REWARD, e, T, 0, ext_actions=np.full((T, 1, 4), a))
    acc = 4.0 * c["kf"] * u_rpm ** 2 / c["mass"] - c["g"]
    t = T * c["dt"]
    assert e["s"][0, 2] == pytest.approx(0.5 * acc * t * t, rel=1e-10)
    assert e["s"][0, 9] == pytest.approx(acc * t, rel=1e-10)
    assert np.allclose(e["s"][0, :2], 0.0, atol=1e-14)


def _strip_rpm_columns(P, dc_hist, da, H):
    """Critic parameters of the HIST layout (inputs: actor obs, 4 motor speeds, action) with
    the 4 motor-speed columns of W1 removed: the same network on the symmetric layout."""
    W1 = P[:H * dc_hist].reshape(H, dc_hist)
    W1s = np.concatenate([W1[:, :da], W1[:, da + 4:]], axis=1)
    return np.concatenate([W1s.ravel(), P[H * dc_hist:]])


@pytest.mark.parametrize("noise", [False, True])
def test_symmetric_critic_is_the_history_critic_without_motor_speeds(noise):
    """Without observation noise, a symmetric critic equals the privileged history critic
    whose motor-speed weights are zero: same Q-values, targets and losses.  With noise the
    symmetric critic sees the noisy observation, so the two differ."""
    kw = dict(sig_p=0.01, sig_R=0.02, sig_v=0.05, sig_w=0.05) if noise else {}
    ch = small_cfg(episode_len=9, **kw)
    cs = dict(ch)
    cs["critic_layout"] = 3
    da = O.actor_in(ch)
    assert O.critic_in(cs) == da + 4 and O.critic_in(ch) == da + 8
    buf, _, _ = make_buffer(ch, n_env=3, T=60, capacity=64)
    H = 6
    Lh = make_learner(ch, H)
    dch = O.critic_in(ch)
    for k in ("c1", "c1_t", "c2", "c2_t"):
        W1 = Lh[k][:H * dch].reshape(H, dch)
        W1[:, da:da + 4] = 0.0
    Ls = copy.deepcopy(Lh)
    for k in ("c1", "c1_t", "c2", "c2_t"):
        Ls[k] = _strip_rpm_columns(Lh[k], dch, da, H)
    for k in ("m_c1", "v_c1", "m_c2", "v_c2"):
        Ls[k] = np.zeros(Ls["c1"].size)
    dh = O.td3_update(ch, hyper(B=16, H=H), Lh, copy.deepcopy(buf))
    ds = O.td3_update(cs, hyper(B=16, H=H), Ls, copy.deepcopy(buf))
    assert np.array_equal(dh["idx"], ds["idx"])
    same = all(np.allclose(dh[k], ds[k], rtol=1e-12, atol=1e-12) for k in ("q1", "q2", "y"))
    assert same != noise
    if not noise:
        assert dh["critic_loss"] == pytest.approx(ds["critic_loss"], rel=1e-12)
        # the updated critics agree too, column for column
        assert np.allclose(_strip_rpm_columns(Lh["c1"], dch, da, H), Ls["c1"], rtol=1e-10,
                           atol=1e-13)


def test_ablation_presets_remove_one_component_each():
    """The ten variants of the study: each differs from the full method in exactly the
    component it names (the last in two)."""
    full, fcur, frec = W.ablation("all_components")
    assert set(W.ABLATIONS) == {"all_components", "observation_noise", "reward_recalculation",
                                "exploration_noise_decay", "disturbances",
                                "asymmetric_actor_critic", "action_history", "curriculum",
                                "rotor_delay", "aac_and_curriculum"}
    assert frec == 1 and full["critic_layout"] == 0 and full["n_hist"] == 16
    assert full["motor_lag_off"] == 0 and full["dist_f"] > 0 and full["sig_p"] > 0
    assert fcur["factor"][4] > 1.0 and fcur["sigma_factor"] < 1.0

    def diff(name):
        c, cur, rec = W.ablation(name)
        keys = {k for k in full if c.get(k) != full[k]}
        if rec != frec:
            keys.add("recalc_rewards")
        if cur["factor"] != fcur["factor"] or cur["target"] != fcur["target"]:
            keys.add("curriculum")
        if cur["sigma_factor"] != fcur["sigma_factor"]:
            keys.add("sigma_factor")
        return keys

    assert diff("all_components") == set()
    assert diff("observation_noise") == {"sig_p", "sig_R", "sig_v", "sig_w"}
    assert diff("reward_recalculation") == {"recalc_rewards"}
    assert diff("exploration_noise_decay") == {"sigma_factor"}
    assert diff("disturbances") == {"dist_f", "dist_tau"}
    assert diff("asymmetric_actor_critic") == {"critic_layout"}
    assert diff("action_history") == {"n_hist"}
    assert diff("curriculum") == {"curriculum"}
    assert diff("rotor_delay") == {"motor_lag_off"}
    assert diff("aac_and_curriculum") == {"critic_layout", "curriculum"}
    # without the curriculum the reward constants stay at their start values
    _, cur, _ = W.ablation("curriculum")
    assert cur["factor"] == [1.0] * 7 and cur["target"] == list(W.REWARD)
