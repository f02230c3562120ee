"""Pins of the oracle's replay gather and of its MLP forward pass.

The learner rebuilds each sampled transition's actor observation o_a and the next one o_a'
from the compact replay records: the state, the last N_H executed actions of the same env
(zeros before the episode start) and observation noise regenerated from its random counter
(Sec. IV: actor observation = position, rotation matrix, linear and angular velocity and
the action history; TD3 samples transitions (s, a, r, s') uniformly).  Here the rebuilt
vectors are checked against what the actor actually saw during the rollout, recorded step
by step from the live history, and against the actor output recorded there: an
off-by-one in the history lag, a wrong noise counter or a wrong s' source fails these.

The forward pass (ReLU hidden layers, tanh or linear output, parameter layout W1 b1 W2 b2
W3 b3 with W[out][in]) is pinned on a hand-computed two-unit network with pre-activations
of both signs.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def noisy_cfg(**kw):
    c = W.config("c1")
    c.update(dict(n_hist=16, learning_starts=0, episode_len=9, term_pos=0.23,
                  sig_p=0.002, sig_R=0.01, sig_v=0.01, sig_w=0.01))
    c.update(kw)
    return c


def actor_rollout(c, n_env, T, hidden=8, sigma_e=0.3, seed=5):
    e = O.new_envs(c, np.arange(n_env))
    actor = O.init_params(c, 0, O.actor_in(c), hidden, 4)
    # larger output weights than the default init: the envs leave the box now and then
    actor[-4 * hidden - 4:] *= 8.0
    rec = O.rollout(c, W.REWARD, e, T, 0, actor=actor, hidden=hidden, sigma_e=sigma_e,
                    obs=True)
    return rec, actor, e


def ring_of(rec, T, cap):
    n_env = rec["rec_s"].shape[1]
    buf = dict(s=np.zeros((cap, n_env, 17)), a=np.zeros((cap, n_env, 4)),
               r=np.zeros((cap, n_env)), flags=np.zeros((cap, n_env), np.uint32),
               priv=np.zeros((cap, n_env, 6)), side=np.zeros((cap, n_env, 17)),
               head=T % cap, size=min(T, cap), t_now=T)
    for t in range(T):
        sl = t % cap
        for k, src in (("s", "rec_s"), ("a", "rec_a"), ("r", "rec_r"), ("flags", "rec_flags"),
                       ("priv", "rec_priv"), ("side", "side")):
            buf[k][sl] = np.nan_to_num(rec[src][t]) if k == "side" else rec[src][t]
    return buf


def learner(c, hidden, actor):
    da, dc = O.actor_in(c), O.critic_in(c)
    L = dict(actor=actor.copy(), actor_t=actor.copy(), c1=O.init_params(c, 1, dc, hidden, 1),
             c2=O.init_params(c, 2, dc, hidden, 1), t_a=0, t_c=0, update_idx=0)
    L["c1_t"], L["c2_t"] = L["c1"].copy(), L["c2"].copy()
    for k, n in (("a", "actor"), ("c1", "c1"), ("c2", "c2")):
        L["m_" + k] = np.zeros(L[n].size)
        L["v_" + k] = np.zeros(L[n].size)
    assert da == 18 + 4 * c["n_hist"]
    return L


def hyper(B, H):
    h = dict(W.TD3)
    h.update(batch=B, hidden=H)
    return h


def sampled_steps(c, buf, d, n_env):
    """Global step t and env of every sampled transition, from the flat index alone."""
    lost = c["n_hist"] if buf["size"] == buf["s"].shape[0] else 0
    out = []
    for idx in d["idx"]:
        k, env = int(idx) // n_env, int(idx) % n_env
        out.append((buf["t_now"] - buf["size"] + lost + k, env))
    return out


@pytest.mark.parametrize("cap", [60, 37])
def test_rebuilt_observations_are_what_the_actor_saw(cap):
    """o_a of a sampled transition equals the observation recorded at its step; o_a' equals
    the next step's observation, or, where the episode ended, the observation of the
    side-slot state s' with the executed action pushed into the history and the noise of
    the next step's counter."""
    c = noisy_cfg()
    T, n_env, H = 60, 3, 8
    rec, actor, _ = actor_rollout(c, n_env, T, hidden=H)
    flags = rec["rec_flags"]
    assert np.any(flags & 1) and np.any(flags & 2), "case needs terminations and truncations"
    buf = ring_of(rec, T, cap)
    L = learner(c, H, actor)
    L["update_idx"] = 3
    B = 512
    d = O.td3_update(c, hyper(B, H), L, buf)
    nh = c["n_hist"]
    seen_done = seen_mid = seen_start = 0
    for j, (t, env) in enumerate(sampled_steps(c, buf, d, n_env)):
        assert 0 <= t < T - 1
        obs_t = rec["obs"][t, env]
        assert np.array_equal(d["oa"][j], obs_t), (j, t, env)
        # the actor output recorded at that step follows from the rebuilt observation
        mu, _, _ = O.mlp_forward(actor, d["oa"][j], O.actor_in(c), H, 4, True)
        assert np.allclose(mu, rec["mu"][t, env], rtol=0, atol=1e-12)
        fl = int(flags[t, env])
        if fl & 3:
            seen_done += 1
            hist2 = np.zeros(4 * O.HMAX)
            hist2[:4] = rec["rec_a"][t, env]
            hist2[4:4 * nh] = obs_t[18:18 + 4 * (nh - 1)]
            exp = O.obs_actor(c, rec["side"][t, env], hist2, O.obs_noise(c, env, t + 1))
            assert np.array_equal(d["oa2"][j], exp), (j, t, env)
        else:
            assert np.array_equal(d["oa2"][j], rec["obs"][t + 1, env]), (j, t, env)
            mu2, _, _ = O.mlp_forward(actor, d["oa2"][j], O.actor_in(c), H, 4, True)
            assert np.allclose(mu2, rec["mu"][t + 1, env], rtol=0, atol=1e-12)
        ep = fl >> 8
        if ep == 0:
            seen_start += 1
            assert not np.any(d["oa"][j][18:]), "no history at the episode start"
        elif ep < nh:
            seen_mid += 1
            assert not np.any(d["oa"][j][18 + 4 * ep:]), "zeros before the episode start"
    assert seen_done and seen_mid and seen_start


@pytest.mark.parametrize("layout", [O.CRITIC_HIST, O.CRITIC_PRIV])
def test_rebuilt_critic_inputs(layout):
    """o_c = noise-free observation, normalised motor speeds, (privileged parameters), and
    the stored action; o_c' the same at s' with the smoothed target action."""
    c = noisy_cfg(critic_layout=layout, dr_mass=0.2, dr_J=0.2, dr_kf=0.1, tm_lo=0.03,
                  dist_f=0.0027, dist_tau=1e-6)
    T, n_env, H = 50, 2, 8
    rec, actor, _ = actor_rollout(c, n_env, T, hidden=H, seed=7)
    buf = ring_of(rec, T, 64)
    L = learner(c, H, actor)
    B = 256
    d = O.td3_update(c, hyper(B, H), L, buf)
    da, dc = O.actor_in(c), O.critic_in(c)
    rng = c["rpm_max"] - c["rpm_min"]
    for j, (t, env) in enumerate(sampled_steps(c, buf, d, n_env)):
        for x, obs_row, s, sub in ((d["oc"][j], d["oa"][j], rec["rec_s"][t, env], t),
                                   (d["oc2"][j], d["oa2"][j], None, t + 1)):
            noise = O.obs_noise(c, env, sub)
            # the critic sees the actor's observation without its noise
            assert np.allclose(x[:18], obs_row[:18] - noise[:18], rtol=0, atol=1e-15)
            assert np.array_equal(x[18:da], obs_row[18:da])
            st = s if s is not None else (rec["side"][t, env] if rec["rec_flags"][t, env] & 3
                                          else rec["rec_s"][t + 1, env])
            assert np.allclose(x[da:da + 4], 2.0 * (st[13:17] - c["rpm_min"]) / rng - 1.0,
                               rtol=0, atol=1e-15)
            if layout == O.CRITIC_PRIV:
                assert np.array_equal(x[da + 4:da + 10], rec["rec_priv"][t, env])
        assert np.array_equal(d["oc"][j][dc - 4:], rec["rec_a"][t, env])
        assert np.array_equal(d["oc2"][j][dc - 4:], d["a2"][j])


def test_recorded_observation_matches_live_state():
    """The recorded observation is p, R(q) row-major, v, omega of the state the step
    started from, plus noise, then the executed actions newest first."""
    c = noisy_cfg(episode_len=500, term_pos=0.6)
    T = 6
    rec, _, _ = actor_rollout(c, 1, T)
    for t in range(T):
        s = rec["rec_s"][t, 0]
        w, x, y, z = s[3:7]
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        clean = np.concatenate([s[0:3], R.ravel(), s[7:10], s[10:13]])
        o = rec["obs"][t, 0]
        assert np.allclose(o[:18] - O.obs_noise(c, 0, t), clean, rtol=0, atol=1e-14)
        for i in range(1, 17):
            exp = rec["rec_a"][t - i, 0] if i <= t else np.zeros(4)
            assert np.array_equal(o[18 + 4 * (i - 1):18 + 4 * i], exp)


# ----------------------------------------------------------------------------- forward
def two_unit_net():
    """in = 2, hidden = 2, out = 2, laid out W1[2][2] b1 W2[2][2] b2 W3[2][2] b3."""
    W1, b1 = [1.0, -2.0, 0.5, 1.0], [0.5, -1.0]
    W2, b2 = [2.0, 3.0, -1.0, -4.0], [0.25, 1.0]
    W3, b3 = [1.0, 2.0, -2.0, 0.5], [-1.0, 0.5]
    return np.array(W1 + b1 + W2 + b2 + W3 + b3)


def test_mlp_forward_hand_computed():
    P = two_unit_net()
    assert P.size == O.net_size(2, 2, 2)
    # x = (1, 1):
    #   z1 = (1 - 2 + 0.5, 0.5 + 1 - 1) = (-0.5, 0.5)  -> h1 = (0, 0.5)   (first unit clipped)
    #   z2 = (0 + 1.5 + 0.25, 0 - 2 + 1) = (1.75, -1) -> h2 = (1.75, 0)  (second unit clipped)
    #   z3 = (1.75 + 0 - 1, -3.5 + 0 + 0.5) = (0.75, -3)
    y, h1, h2 = O.mlp_forward(P, [1.0, 1.0], 2, 2, 2, False)
    assert h1.tolist() == [0.0, 0.5]
    assert h2.tolist() == [1.75, 0.0]
    assert y.tolist() == [0.75, -3.0]
    y, _, _ = O.mlp_forward(P, [1.0, 1.0], 2, 2, 2, True)
    assert y[0] == pytest.approx(math.tanh(0.75), rel=1e-15)
    assert y[1] == pytest.approx(math.tanh(-3.0), rel=1e-15)
    # x = (-2, 0.5):
    #   z1 = (-2 - 1 + 0.5, -1 + 0.5 - 1) = (-2.5, -1.5) -> h1 = (0, 0)
    #   z2 = b2 = (0.25, 1)                              -> h2 = (0.25, 1)
    #   z3 = (0.25 + 2 - 1, -0.5 + 0.5 + 0.5) = (1.25, 0.5)
    y, h1, h2 = O.mlp_forward(P, [-2.0, 0.5], 2, 2, 2, False)
    assert h1.tolist() == [0.0, 0.0]
    assert h2.tolist() == [0.25, 1.0]
    assert y.tolist() == [1.25, 0.5]


def test_mlp_forward_single_output_critic_shape():
    """out = 1 (the critics): the output row is W3[0] . h2 + b3, no activation."""
    P = np.array([1.0, 0.0, 0.0, 1.0,  # W1 = identity
                  0.0, 0.0,            # b1
                  1.0, 1.0, 1.0, -1.0,  # W2
                  0.0, 0.0,            # b2
                  3.0, -5.0,           # W3[0]
                  0.125])              # b3
    assert P.size == O.net_size(2, 2, 1)
    # x = (2, 1): h1 = (2, 1); z2 = (3, 1) -> h2 = (3, 1); y = 9 - 5 + 0.125
    y, _, h2 = O.mlp_forward(P, [2.0, 1.0], 2, 2, 1, False)
    assert h2.tolist() == [3.0, 1.0] and y.tolist() == [4.125]
    # x = (1, 3): h1 = (1, 3); z2 = (4, -2) -> h2 = (4, 0); y = 12 + 0.125
    y, _, h2 = O.mlp_forward(P, [1.0, 3.0], 2, 2, 1, False)
    assert h2.tolist() == [4.0, 0.0] and y.tolist() == [12.125]
