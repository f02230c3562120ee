"""Pins of the oracle's rollout, TD3 learner, reward recalculation and adjoint.

Finite differences in FP64 on small networks, closed forms (first Adam step, Polyak at
tau in {0,1}, TD targets with constant target critics), and structural invariants of the
episode bookkeeping.
"""
import copy

import numpy as np
import pytest

import oracle as O
import workloads as W


def small_cfg(**kw):
    c = W.config("c1")
    c.update(dict(n_hist=4, learning_starts=0))
    c.update(kw)
    return c


def make_learner(c, hidden, seed=0):
    da, dc = O.actor_in(c), O.critic_in(c)
    L = dict(actor=O.init_params(c, 0, da, hidden, 4), c1=O.init_params(c, 1, dc, hidden, 1),
             c2=O.init_params(c, 2, dc, hidden, 1), t_a=0, t_c=0, update_idx=0)
    # perturb targets away from the online nets so that every term is exercised
    g = W.rng(seed)
    L["actor_t"] = L["actor"] + 0.05 * g.standard_normal(L["actor"].size)
    L["c1_t"] = L["c1"] + 0.05 * g.standard_normal(L["c1"].size)
    L["c2_t"] = L["c2"] + 0.05 * g.standard_normal(L["c2"].size)
    for k, n in (("a", "actor"), ("c1", "c1"), ("c2", "c2")):
        L["m_" + k] = np.zeros(L[n].size)
        L["v_" + k] = np.zeros(L[n].size)
    return L


def make_buffer(c, n_env=3, T=80, seed=1, capacity=None):
    """Oracle rollout of T steps with random actions, stored in a ring of ``capacity``."""
    e = O.new_envs(c, np.arange(n_env))
    acts = W.random_actions(seed, (T, n_env, 4))
    rec = O.rollout(c, W.REWARD, e, T, 0, ext_actions=acts)
    cap = capacity or T
    buf = dict(s=np.zeros((cap, n_env, 17)), a=np.zeros((cap, n_env, 4)),
               r=np.zeros((cap, n_env)), flags=np.zeros((cap, n_env), np.uint32),
               priv=np.zeros((cap, n_env, 6)), side=np.zeros((cap, n_env, 17)),
               head=T % cap, size=min(T, cap), t_now=T)
    for t in range(T):
        sl = t % cap
        for k, src in (("s", "rec_s"), ("a", "rec_a"), ("r", "rec_r"), ("flags", "rec_flags"),
                       ("priv", "rec_priv"), ("side", "side")):
            buf[k][sl] = np.nan_to_num(rec[src][t]) if k == "side" else rec[src][t]
    return buf, e, rec


def hyper(B=8, H=8, **kw):
    h = dict(W.TD3)
    h.update(batch=B, hidden=H)
    h.update(kw)
    return h


# ----------------------------------------------------------------------------- rollout logic
def test_rollout_bookkeeping():
    c = small_cfg(episode_len=7, term_pos=0.6)
    e = O.new_envs(c, [0, 1])
    T = 40
    acts = W.random_actions(2, (T, 2, 4))
    rec = O.rollout(c, W.REWARD, e, T, 0, ext_actions=acts)
    for k in range(2):
        ep = 0
        for t in range(T):
            fl = int(rec["rec_flags"][t, k])
            assert fl >> 8 == ep
            term, trunc = fl & 1, (fl >> 1) & 1
            assert not (term and trunc)
            if trunc:
                assert ep + 1 == 7
            done = term or trunc
            if not done and t + 1 < T:
                # next record's state is this transition's s'
                s2 = O.rk4(c, rec["rec_s"][t, k], 10851.0 * (rec["rec_a"][t, k] + 1.0),
                           W.nominal_params(1)[0])
                assert np.allclose(rec["rec_s"][t + 1, k], s2, rtol=1e-12, atol=1e-12)
                ep += 1
            else:
                ep = 0
            assert np.allclose(rec["rec_a"][t, k], np.clip(acts[t, k], -1, 1))
    # history is newest first and of length n_hist (4 here)
    h = e["hist"][0]
    steps = int(e["ep_step"][0])
    for i in range(1, min(steps, 4) + 1):
        assert np.allclose(h[4 * (i - 1):4 * i], rec["rec_a"][T - i, 0])


def test_termination_box_and_reset():
    c = small_cfg(term_pos=0.21, episode_len=500)
    e = O.new_envs(c, [5])
    # full throttle on one side: flips and leaves the box quickly
    acts = np.tile(np.array([1.0, 1.0, -1.0, -1.0]), (60, 1, 1))
    rec = O.rollout(c, W.REWARD, e, 60, 0, ext_actions=acts)
    fl = rec["rec_flags"][:, 0]
    t_end = int(np.argmax(fl & 1))
    assert fl[t_end] & 1
    assert np.max(np.abs(rec["side"][t_end, 0, 0:3])) > 0.21
    assert e["ep_index"][0] >= 1
    # the state after the terminal step is the reset state of episode 1
    s1, _, _ = O.reset_env(c, 5, 1)
    assert np.allclose(rec["rec_s"][t_end + 1, 0], s1)


def test_actor_rollout_warmup_and_exploration():
    c = small_cfg(learning_starts=3)
    actor = O.init_params(c, 0, O.actor_in(c), 8, 4)
    e = O.new_envs(c, [0, 1, 2])
    rec = O.rollout(c, W.REWARD, e, 6, 0, actor=actor, hidden=8, sigma_e=0.0)
    # warm-up actions are uniform draws (tag 8), afterwards the deterministic actor
    for t in range(3):
        for k in range(3):
            r = O.philox([k, t, 8 << 24, 0], [0, 0])
            assert np.allclose(rec["rec_a"][t, k], [2 * O.uniform(x) - 1 for x in r])
    assert np.allclose(rec["rec_a"][3:], rec["mu"][3:])
    assert np.all(np.abs(rec["mu"][3:]) < 1)


def test_recalc_invariance_and_linkage():
    c = small_cfg(episode_len=9)
    buf, e, rec = make_buffer(c, n_env=2, T=30)
    r0 = buf["r"].copy()
    O.recalc_rewards(W.REWARD, buf, e["s"])
    # same constants: the newest non-terminal record uses the live env state
    assert np.allclose(buf["r"], r0, rtol=1e-14, atol=1e-14)
    C2 = list(W.REWARD)
    C2[4] = 0.5
    O.recalc_rewards(C2, buf, e["s"])
    expect = r0 - (0.5 - W.REWARD[4]) * np.sum((buf["a"] - W.REWARD[5]) ** 2, axis=-1)
    assert np.allclose(buf["r"], expect, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- TD3
def test_td3_target_with_constant_target_critics():
    c = small_cfg(episode_len=6)
    buf, _, _ = make_buffer(c, n_env=2, T=40, capacity=50)  # not full: no excluded window
    H = 3
    L = make_learner(c, H)
    dc = O.critic_in(c)
    for name, q in (("c1_t", 3.0), ("c2_t", 5.0)):
        P = np.zeros_like(L[name])
        # W1 = 0, b1 = 1 -> h1 = 1; W2 = 0, b2 = 1 -> h2 = 1; W3 = q/H, b3 = 0 -> Q = q
        P[H * dc:H * dc + H] = 1.0
        o = H * dc + H + H * H
        P[o:o + H] = 1.0
        P[o + H:o + 2 * H] = q / H
        L[name] = P
    d = O.td3_update(c, hyper(B=32, H=H, gamma=0.9), L, buf)
    n = buf["s"].shape[1]
    for j in range(32):
        idx = int(d["idx"][j])
        slot, env = idx // n, idx % n
        fl = int(buf["flags"][slot, env])
        exp = buf["r"][slot, env] + (0.0 if fl & 1 else 0.9 * 3.0)
        assert d["y"][j] == pytest.approx(exp, rel=1e-14, abs=1e-14)
    assert np.any(buf["flags"] & 2), "case should contain truncated transitions"


def test_replay_indices_follow_philox():
    c = small_cfg()
    buf, _, _ = make_buffer(c, n_env=3, T=50, capacity=64)
    L = make_learner(c, 4)
    L["update_idx"] = 17
    d = O.td3_update(c, hyper(B=10, H=4), L, buf)
    nvalid = (50 - 1) * 3
    for j in range(10):
        r = O.philox([j >> 2, 17, 4 << 24, 0], [0, 0])
        assert int(d["idx"][j]) == (int(r[j & 3]) * nvalid) >> 32


def test_critic_and_actor_gradients_match_finite_differences():
    c = small_cfg(episode_len=11)
    buf, _, _ = make_buffer(c, n_env=2, T=40)
    H = 5
    L0 = make_learner(c, H)
    L0["update_idx"] = 1  # actor update happens on this call (policy_delay 2)
    hp = hyper(B=6, H=H)
    d0 = O.td3_update(c, hp, copy.deepcopy(L0), buf)
    assert d0["actor_updated"]
    g = W.rng(9)
    h = 1e-6
    for name, gk, lk in (("c1", "g_c1", "critic_loss"), ("c2", "g_c2", "critic_loss"),
                         ("actor", "g_a", "actor_loss")):
        for i in g.choice(L0[name].size, 12, replace=False):
            Lp, Lm = copy.deepcopy(L0), copy.deepcopy(L0)
            Lp[name][i] += h
            Lm[name][i] -= h
            fd = (O.td3_update(c, hp, Lp, buf)[lk] - O.td3_update(c, hp, Lm, buf)[lk]) / (2 * h)
            an = d0[gk][i]
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (name, i, fd, an)


def test_adam_first_step_and_polyak_closed_forms():
    c = small_cfg()
    buf, _, _ = make_buffer(c, n_env=2, T=30)
    L0 = make_learner(c, 6)
    L0["update_idx"] = 1
    for tau in (0.0, 1.0, 0.3):
        L = copy.deepcopy(L0)
        d = O.td3_update(c, hyper(B=8, H=6, tau=tau), L, buf)
        lr, eps = W.TD3["lr"], W.TD3["eps"]
        for name, gk in (("c1", "g_c1"), ("c2", "g_c2"), ("actor", "g_a")):
            gg = d[gk]
            exp = L0[name] - lr * gg / (np.abs(gg) + eps)
            assert np.allclose(L[name], exp, rtol=1e-12, atol=1e-15)
            tgt = tau * L[name] + (1 - tau) * L0[name + "_t"]
            assert np.allclose(L[name + "_t"], tgt, rtol=1e-12, atol=1e-15)
        assert L["t_a"] == 1 and L["t_c"] == 1 and L["update_idx"] == 2


def test_actor_is_delayed():
    c = small_cfg()
    buf, _, _ = make_buffer(c, n_env=2, T=30)
    L = make_learner(c, 4)
    flags = []
    for _ in range(6):
        a_before = L["actor"].copy()
        t_before = L["actor_t"].copy()
        d = O.td3_update(c, hyper(B=4, H=4), L, buf)
        flags.append(d["actor_updated"])
        if not d["actor_updated"]:
            assert np.array_equal(L["actor"], a_before) and np.array_equal(L["actor_t"], t_before)
    assert flags == [False, True] * 3
    assert L["t_c"] == 6 and L["t_a"] == 3


def test_wrapped_buffer_excludes_oldest_history_window():
    c = small_cfg(n_hist=4)
    buf, _, _ = make_buffer(c, n_env=2, T=50, capacity=20)
    assert buf["size"] == 20 and buf["head"] == 10
    L = make_learner(c, 4)
    d = O.td3_update(c, hyper(B=64, H=4), L, buf)
    nvalid = (20 - 1 - 4) * 2
    assert int(d["idx"].max()) < nvalid


# ----------------------------------------------------------------------------- adjoint
def _fd_check(fun, x, grad, idxs, h, tol):
    for i in idxs:
        xp, xm = x.copy(), x.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        fd = (fun(xp) - fun(xm)) / (2 * h)
        an = grad.flat[i]
        assert abs(fd - an) <= tol * max(abs(an), 1e-8 * 0 + 1e-6), (i, fd, an)


def test_adjoint_open_loop_matches_fd():
    c = small_cfg()
    n, H = 2, 30
    s0 = W.random_states(21, n)
    prm = W.random_params(22, n)
    acts = W.random_actions(23, (n, H, 4), -0.6, 0.6)
    wts = (1.0, 0.5, 0.2, 0.01)
    out = O.diff_run(c, s0, prm, H, wts, mode=0, actions=acts)

    def loss_a(a):
        return O.diff_run(c, s0, prm, H, wts, mode=0, actions=a)["loss"].sum()

    g = W.rng(1)
    _fd_check(loss_a, acts, out["g_actions"], g.choice(acts.size, 16, replace=False), 1e-4, 1e-6)

    def loss_p(p):
        return O.diff_run(c, s0, p, H, wts, mode=0, actions=acts)["loss"].sum()

    for k in range(n):
        for j in range(7):
            i = k * 8 + j
            pp, pm = prm.copy(), prm.copy()
            hh = 1e-4 * abs(prm.flat[i])
            pp.flat[i] += hh
            pm.flat[i] -= hh
            fd = (loss_p(pp) - loss_p(pm)) / (2 * hh)
            an = out["g_prm"].flat[i]
            assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9 * abs(fd) + 1e-12, (j, fd, an)


def test_adjoint_closed_loop_matches_fd():
    c = small_cfg()
    n, H, hid, nh = 2, 25, 6, 3
    s0 = W.random_states(31, n)
    prm = W.nominal_params(n)
    da = 18 + 4 * nh
    actor = O.init_params(c, 0, da, hid, 4)
    wts = (1.0, 0.5, 0.2, 0.05)
    out = O.diff_run(c, s0, prm, H, wts, mode=1, actor=actor, hidden=hid, n_hist=nh)

    def loss_w(w):
        return O.diff_run(c, s0, prm, H, wts, mode=1, actor=w, hidden=hid,
                          n_hist=nh)["loss"].sum()

    g = W.rng(2)
    _fd_check(loss_w, actor, out["g_actor"], g.choice(actor.size, 20, replace=False), 1e-5, 1e-6)


def test_adjoint_free_fall_closed_form():
    """Rotors off: p_t = p0 + v0 t - g t^2/2 e_z, so dL/dm = dL/dJ = 0 and the loss is
    the closed-form sum."""
    c = small_cfg(renorm_q=1)
    s0 = np.zeros((1, 17))
    s0[0, 3] = 1.0
    s0[0, 0:3] = [0.1, 0.0, 0.2]
    s0[0, 7:10] = [0.0, 0.5, 0.0]
    prm = W.nominal_params(1)
    H = 20
    acts = np.full((1, H, 4), -1.0)  # rpm_min = 0
    out = O.diff_run(c, s0, prm, H, (1.0, 0.0, 0.0, 0.0), mode=0, actions=acts)
    ts = np.arange(1, H + 1) * c["dt"]
    p = s0[0, 0:3][None] + s0[0, 7:10][None] * ts[:, None]
    p[:, 2] -= 0.5 * c["g"] * ts ** 2
    assert out["loss"][0] == pytest.approx(np.sum(p ** 2), rel=1e-12)
    assert np.all(out["g_prm"][0, :4] == 0.0)
