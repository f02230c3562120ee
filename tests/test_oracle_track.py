"""Pins of the oracle's simulated trajectory tracking (Sec. V "Trajectory tracking").

The target is the paper's figure-eight p*(t) = (A cos(2 pi t/T), (A/2) sin(4 pi t/T), z0);
the controller sees its position and velocity offset by the target's (Sec. IV set-point
shifting), clipped.  The pins use facts that hold independently of the tracking code: hand
values of the curve, its derivative by finite differences, the translation invariance of
the dynamics (a fixed target is a plain rollout of the shifted state), the zero offsets of
a start on the target, and the Galilean structure of the equations of motion (a blind
controller flies the same attitude history whatever the target's speed).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

NS = 17


def cfg(**kw):
    c = W.config("c2")
    c.update(sig_p=0.0, sig_R=0.0, sig_v=0.0, sig_w=0.0, learning_starts=0)
    c.update(kw)
    return c


def hover_actor(d, hidden=32, seed=3, gain=0.05):
    """Random actor whose output sits near the hover action: the flights last a while."""
    dd = dict(d)
    dd["seed"] = seed
    da = O.actor_in(d)
    P = O.init_params(dd, 0, da, hidden, 4)
    w3 = hidden * da + hidden + hidden * hidden + hidden
    P[w3:w3 + 4 * hidden] *= gain
    P[w3 + 4 * hidden:] = math.atanh(W.hover_action())
    return P


def params(d, n, seed=5):
    prm = W.random_params(seed, n)
    dist = np.zeros((n, 6))
    return prm, dist


# ------------------------------------------------------------------------------ target
def test_lissajous_hand_values():
    A, z0, T = 1.3, 0.4, 5.5
    s2 = math.sqrt(0.5)
    cases = {0.0: (A, 0.0), T / 8: (A * s2, A / 2), T / 4: (0.0, 0.0), 3 * T / 8: (-A * s2, -A / 2),
             T / 2: (-A, 0.0), 3 * T / 4: (0.0, 0.0)}
    for t, (x, y) in cases.items():
        p, _ = O.lissajous(t, T, A, z0)
        assert np.allclose(p, [x, y, z0], atol=1e-12), (t, p)
    _, v = O.lissajous(0.0, T, A, z0)
    assert np.allclose(v, [0.0, 2 * math.pi * A / T, 0.0], atol=1e-12)
    # one cycle later the curve repeats; half a cycle later it is mirrored in x
    for t in np.linspace(0.0, T, 7):
        p0, v0 = O.lissajous(t, T, A, z0)
        p1, v1 = O.lissajous(t + T, T, A, z0)
        ph, _ = O.lissajous(t + T / 2, T, A, z0)
        assert np.allclose(p0, p1, atol=1e-12) and np.allclose(v0, v1, atol=1e-12)
        assert np.allclose(ph, [-p0[0], p0[1], z0], atol=1e-12)


def test_lissajous_velocity_is_the_time_derivative():
    rng = np.random.default_rng(0)
    for _ in range(20):
        T = rng.uniform(2.0, 20.0)
        t = rng.uniform(0.0, 3 * T)
        h = 1e-6
        pp, v = O.lissajous(t, T, 1.0, 0.0)
        pa, _ = O.lissajous(t + h, T, 1.0, 0.0)
        pb, _ = O.lissajous(t - h, T, 1.0, 0.0)
        assert np.allclose((pa - pb) / (2 * h), v, atol=1e-7)


# ------------------------------------------------------------------------------ flights
def test_fixed_target_is_a_shifted_plain_rollout():
    """T -> infinity: the target rests at (A, 0, z0).  The dynamics are translation
    invariant, so the tracking flight is the deterministic rollout of the state shifted by
    -(A, 0, z0), and the accumulated error is that rollout's |p|^2 summed over its steps
    before it leaves the termination box."""
    d = cfg()
    n, steps, hid = 6, 120, 32
    prm, dist = params(d, n)
    actor = hover_actor(d, hid)
    A, z0 = 1.0, 0.3
    out = O.track(d, prm, dist, np.full(n, 1e12), actor, hid, steps, amp=A, z0=z0, clip_p=50.0,
                  clip_v=50.0, traj=True)
    # the plain rollout from the shifted start
    s0 = out["traj"][:, 0].copy()
    s0[:, 0] -= A
    s0[:, 2] -= z0
    e = dict(env_id=np.arange(n, dtype=np.uint32), s=s0, prm=prm.copy(), dist=dist.copy(),
             hist=np.zeros((n, 64)), ep_index=np.zeros(n, np.uint32),
             ep_step=np.zeros(n, np.uint32), ep_ret=np.zeros(n), n_done=np.zeros(n, np.uint32),
             len_sum=np.zeros(n, np.uint32), ret_sum=np.zeros(n))
    d2 = dict(d)
    d2["episode_len"] = 10 ** 6
    ref = O.rollout(d2, W.REWARD, e, steps, 0, actor=actor, hidden=hid, sigma_e=0.0)
    for k in range(n):
        ok = int(out["steps_ok"][k])
        flags = ref["rec_flags"][:, k]
        term = np.nonzero(flags & 1)[0]
        assert ok == (int(term[0]) if term.size else steps), (k, ok, term[:3])
        # states: rec_s[j] is the state before step j; the flight's traj[j]
        shifted = out["traj"][k, :ok + 1].copy()
        shifted[:, 0] -= A
        shifted[:, 2] -= z0
        assert np.allclose(shifted[:ok], ref["rec_s"][:ok, k], rtol=1e-9, atol=1e-9)
        pos = ref["rec_s"][1:ok, k, :3]
        last = shifted[ok, :3] if ok else np.zeros(3)
        e3 = float(np.sum(pos ** 2)) + (float(np.sum(last ** 2)) if ok else 0.0)
        exy = float(np.sum(pos[:, :2] ** 2)) + (float(np.sum(last[:2] ** 2)) if ok else 0.0)
        assert np.isclose(out["sq_err"][k, 0], e3, rtol=1e-9, atol=1e-12)
        assert np.isclose(out["sq_err"][k, 1], exy, rtol=1e-9, atol=1e-12)
    assert out["steps_ok"].max() > 20  # the flights are long enough to mean something


def test_start_on_the_target_sees_zero_offsets():
    """At t = 0 the vehicle sits on the target with the target's velocity, so the first
    observation is that of a level vehicle at rest at the origin whatever T: the first step
    is the actor's action for that observation, integrated by RK4 from the start state."""
    d = cfg()
    n, hid = 3, 32
    prm, dist = params(d, n)
    actor = hover_actor(d, hid)
    for T in (3.5, 15.0):
        out = O.track(d, prm, dist, np.full(n, T), actor, hid, 1, traj=True)
        rest = np.zeros(NS)
        rest[3] = 1.0
        o = O.obs_actor(d, rest, np.zeros(64))
        mu, _, _ = O.mlp_forward(actor, o, O.actor_in(d), hid, 4, True)
        a = np.clip(mu, -1.0, 1.0)
        u = d["rpm_min"] + 0.5 * (a + 1.0) * (d["rpm_max"] - d["rpm_min"])
        for k in range(n):
            s0 = out["traj"][k, 0]
            p0, v0 = O.lissajous(0.0, T)
            assert np.allclose(s0[:3], p0) and np.allclose(s0[7:10], v0)
            assert np.allclose(s0[3:7], [1, 0, 0, 0]) and np.allclose(s0[10:13], 0)
            hover = math.sqrt(prm[k, 0] * d["g"] / (4 * prm[k, 4]))
            assert np.allclose(s0[13:], hover, rtol=1e-12)
            s1 = O.rk4(d, s0, u, prm[k], dist[k])
            assert np.allclose(out["traj"][k, 1], s1, rtol=1e-12, atol=1e-13)
            p1, _ = O.lissajous(d["dt"], T)
            assert np.isclose(out["sq_err"][k, 0], np.sum((s1[:3] - p1) ** 2), rtol=1e-12)


def test_zero_clips_make_the_flight_independent_of_the_target_speed():
    """With both clips 0 the actor never sees position or velocity.  The attitude, rate and
    motor equations do not involve p or v, so every cycle time yields the same attitude
    history, and the positions differ only by the start velocity times the elapsed time
    (RK4 integrates the p' = v shift exactly)."""
    d = cfg(term_pos=1e6)
    n, hid, steps = 2, 32, 60
    prm, dist = params(d, n)
    actor = hover_actor(d, hid)
    a = O.track(d, prm, dist, np.full(n, 3.5), actor, hid, steps, clip_p=0.0, clip_v=0.0, traj=True)
    b = O.track(d, prm, dist, np.full(n, 11.0), actor, hid, steps, clip_p=0.0, clip_v=0.0, traj=True)
    assert np.array_equal(a["steps_ok"], [steps] * n) and np.array_equal(b["steps_ok"], [steps] * n)
    assert np.allclose(a["traj"][:, :, 3:7], b["traj"][:, :, 3:7], atol=1e-12)
    assert np.allclose(a["traj"][:, :, 10:], b["traj"][:, :, 10:], rtol=1e-12, atol=1e-9)
    dv = a["traj"][:, 0, 7:10] - b["traj"][:, 0, 7:10]
    tk = d["dt"] * np.arange(steps + 1)
    dp = a["traj"][:, :, :3] - b["traj"][:, :, :3]
    assert np.allclose(dp, dv[:, None, :] * tk[None, :, None], atol=1e-9)
    # with the offsets visible the flights differ
    c = O.track(d, prm, dist, np.full(n, 11.0), actor, hid, steps, traj=True)
    assert not np.allclose(c["traj"][:, -1, 3:7], b["traj"][:, -1, 3:7], atol=1e-6)


def test_flight_ends_outside_the_box_and_without_a_target():
    d = cfg(term_pos=1e-7)
    prm, dist = params(d, 2)
    actor = hover_actor(d, 32)
    out = O.track(d, prm, dist, [5.5, 5.5], actor, 32, 10)
    assert np.array_equal(out["steps_ok"], [0, 0]) and np.all(out["sq_err"] == 0.0)
    d = cfg()
    out = O.track(d, prm, dist, [0.0, -1.0], actor, 32, 10)
    assert np.array_equal(out["steps_ok"], [0, 0]) and np.all(out["sq_err"] == 0.0)
    out = O.track(d, prm, dist, [np.inf, np.nan], actor, 32, 10)
    assert np.array_equal(out["steps_ok"], [0, 0]) and np.all(out["sq_err"] == 0.0)
