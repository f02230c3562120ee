"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: published known-answer
vectors, closed-form solutions, conservation laws, convergence orders, finite differences
and hand-built special cases.  A plausible slip (a dropped term, a wrong sign or index, a
transposed operand) should fail at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def cfg(**kw):
    c = W.config("c1")
    c.update(kw)
    return c


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_is_open_interval_and_exact():
    assert O.uniform(0) == 0.5 * 2.0 ** -23
    assert O.uniform(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -23
    # the conversion keeps only the top 23 bits
    assert O.uniform(0x1FF) == O.uniform(0)
    assert O.uniform(0x200) == 1.5 * 2.0 ** -23


def test_gauss_box_muller_cos_branch():
    # uniforms are odd multiples of 2^-24; the one just below 1/4 puts the angle a hair
    # before pi/2, so z = r cos(angle) ~ r * 2 pi 2^-24
    xq = (1 << 30) - (1 << 9)
    assert O.uniform(xq) == 0.25 - 2.0 ** -24
    x1 = 0x80000000
    r = math.sqrt(-2.0 * math.log(O.uniform(x1)))
    assert 0.0 < O.gauss(x1, xq) < 4e-7 * r
    assert O.gauss(x1, 0) == pytest.approx(r, rel=1e-12)  # angle ~ 0
    # distribution over a Philox stream: Kolmogorov-Smirnov against N(0,1)
    from scipy import stats
    zs = []
    for i in range(20000):
        o = O.philox([i, 7, 3 << 24, 0], [1, 2])
        zs += [O.gauss(o[0], o[1]), O.gauss(o[2], o[3])]
    zs = np.array(zs)
    assert stats.kstest(zs, "norm").pvalue > 1e-3
    assert abs(zs.mean()) < 0.02 and abs(zs.var() - 1.0) < 0.03


def test_replay_index_integer_map():
    n = 999 * 65536
    assert O.replay_index(0, n) == 0
    assert O.replay_index(0xFFFFFFFF, n) == n - 1
    for x in (1, 12345, 0x80000000, 0xDEADBEEF):
        assert O.replay_index(x, n) == (x * n) >> 32
    # chi-square sanity of uniformity over 16 bins from a Philox stream
    counts = np.zeros(16)
    for i in range(40000):
        counts[O.replay_index(int(O.philox([i, 0, 4 << 24, 0], [0, 0])[0]), 16)] += 1
    chi2 = ((counts - 2500.0) ** 2 / 2500.0).sum()
    assert chi2 < 45.0  # 15 dof, p ~ 1e-4


# ----------------------------------------------------------------------------- dynamics
def test_free_fall_closed_form():
    c = cfg(renorm_q=0)
    s = W.random_states(1, 1, rpm=(0.0, 0.0))[0]
    s[10:13] = 0.0
    u = np.zeros(4)
    prm = W.nominal_params(1)[0]
    T = 500
    out = O.dynamics_batch(c, s[None], u[None], prm[None], n_steps=T)[0]
    t = T * c["dt"]
    p = s[0:3] + s[7:10] * t
    p[2] -= 0.5 * c["g"] * t * t
    v = s[7:10].copy()
    v[2] -= c["g"] * t
    assert np.allclose(out[0:3], p, rtol=1e-12, atol=1e-12)
    assert np.allclose(out[7:10], v, rtol=1e-12, atol=1e-12)
    assert np.allclose(out[3:7], s[3:7], atol=1e-15)


def test_exact_hover_is_invariant():
    c = cfg()
    prm = W.nominal_params(1)[0]
    wh = W.hover_rpm()
    s = np.zeros(17)
    s[3] = 1.0
    s[13:17] = wh
    ds = O.deriv(c, s, np.full(4, wh), prm)
    assert np.all(np.abs(ds[7:10]) <= 1e-13)
    assert np.all(np.abs(ds[10:13]) <= 1e-13)
    assert np.all(np.abs(ds[13:17]) == 0.0)
    out = O.dynamics_batch(c, s[None], np.full((1, 4), wh), prm[None], n_steps=500)[0]
    assert np.allclose(out, s, atol=1e-10, rtol=0)


def test_tilted_thrust_direction():
    """Body z axis of q = rot_x(theta) points to (0, -sin, cos): pins R(q) (not R^T)."""
    c = cfg()
    prm = W.nominal_params(1)[0]
    th = 0.3
    s = np.zeros(17)
    s[3:7] = [math.cos(th / 2), math.sin(th / 2), 0, 0]
    w = 15000.0
    s[13:17] = w
    F = 4 * prm[4] * w * w
    ds = O.deriv(c, s, np.full(4, w), prm)
    assert ds[7] == pytest.approx(0.0, abs=1e-12)
    assert ds[8] == pytest.approx(-math.sin(th) * F / prm[0], rel=1e-12)
    assert ds[9] == pytest.approx(math.cos(th) * F / prm[0] - c["g"], rel=1e-12)


def test_single_rotor_torque_matches_cross_product():
    c = cfg()
    prm = W.nominal_params(1)[0]
    pos = np.array(c["rotor_pos"]).reshape(4, 3)
    for i in range(4):
        s = np.zeros(17)
        s[3] = 1.0
        s[13 + i] = 12000.0
        f = prm[4] * 12000.0 ** 2
        tau = np.cross(pos[i], [0, 0, f]) + np.array([0, 0, c["rotor_dir"][i] * prm[5] * f])
        ds = O.deriv(c, s, s[13:17], prm)
        assert np.allclose(ds[10:13], tau / prm[1:4], rtol=1e-12, atol=1e-9)


def test_motor_lag_one_step_factor_and_time_constant():
    c = cfg()
    prm = W.nominal_params(1)[0]
    h = c["dt"] / prm[6]
    phi = 1 - h + h * h / 2 - h ** 3 / 6 + h ** 4 / 24
    assert phi == pytest.approx(0.935506996, abs=1e-9)
    s = np.zeros(17)
    s[3] = 1.0
    s[13:17] = [0.0, 1000.0, 5000.0, 20000.0]
    u = np.array([10000.0, 10000.0, 0.0, 21702.0])
    out = O.rk4(c, s, u, prm)
    assert np.allclose(out[13:17] - u, (s[13:17] - u) * phi, rtol=1e-13, atol=1e-9)
    assert abs(phi - math.exp(-h)) < 2e-8  # O(h^5) agreement, |diff| ~ 1.1e-8
    # after t = T the set-point step is 63.2 % covered (Sec. IV, RC time constant)
    n = int(round(prm[6] / 1e-4))
    s[13:17] = 0.0
    out = O.dynamics_batch(c, s[None], np.full((1, 4), 10000.0), prm[None], dt=1e-4,
                           n_steps=n)[0]
    assert np.allclose(out[13:17] / 10000.0, 1 - math.exp(-1), atol=1e-9)


def _angmom_energy(s, prm):
    q = s[3:7]
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    Jw = prm[1:4] * s[10:13]
    return R @ Jw, 0.5 * np.dot(s[10:13], Jw), np.linalg.norm(q)


def test_torque_free_conservation_and_order():
    c = cfg(renorm_q=0)
    prm = W.nominal_params(1)[0]
    prm[1:4] = [1.4e-5, 1.9e-5, 2.6e-5]  # asymmetric body, generic tumbling
    s = np.zeros(17)
    s[3:7] = W.random_quat(W.rng(3), 1)[0]
    s[10:13] = [3.0, -2.0, 4.0]
    L0, E0, n0 = _angmom_energy(s, prm)
    drifts = []
    for dt in (0.01, 0.005):
        n = int(round(1.0 / dt))
        out = O.dynamics_batch(c, s[None], np.zeros((1, 4)), prm[None], dt=dt, renorm=0,
                               n_steps=n)[0]
        L, E, nq = _angmom_energy(out, prm)
        assert np.linalg.norm(L - L0) < 1e-6 * np.linalg.norm(L0)
        assert abs(E - E0) < 1e-6 * E0
        assert abs(nq - 1.0) < 1e-6
        drifts.append(np.linalg.norm(L - L0) + abs(E - E0) / E0 * np.linalg.norm(L0))
    assert 12.0 < drifts[0] / drifts[1] < 20.0  # fourth order: ratio ~16


def test_axisymmetric_precession_closed_form():
    c = cfg(renorm_q=1)
    prm = W.nominal_params(1)[0]  # Jx = Jy
    s = np.zeros(17)
    s[3] = 1.0
    s[10:13] = [0.7, -0.4, 5.0]
    T = 1.0
    out = O.dynamics_batch(c, s[None], np.zeros((1, 4)), prm[None], dt=1e-3, n_steps=1000)[0]
    Om = (prm[3] - prm[1]) / prm[1] * s[12]
    wxy0 = complex(s[10], s[11])
    wxy = wxy0 * np.exp(1j * Om * T)
    assert out[12] == pytest.approx(s[12], abs=1e-12)
    assert out[10] == pytest.approx(wxy.real, abs=1e-9)
    assert out[11] == pytest.approx(wxy.imag, abs=1e-9)


def test_single_axis_rotation_quaternion_body_frame():
    """Spin about one principal axis: q(t) = q0 (x) exp(w t / 2) (body-frame rate)."""
    c = cfg(renorm_q=0)
    prm = W.nominal_params(1)[0]
    q0 = W.random_quat(W.rng(5), 1)[0]
    for axis in range(3):
        s = np.zeros(17)
        s[3:7] = q0
        s[10 + axis] = 2.5
        out = O.dynamics_batch(c, s[None], np.zeros((1, 4)), prm[None], dt=1e-3, n_steps=800)[0]
        th = 2.5 * 0.8
        e = np.zeros(4)
        e[0] = math.cos(th / 2)
        e[1 + axis] = math.sin(th / 2)
        w0, x0, y0, z0 = q0
        w1, x1, y1, z1 = e
        ref = np.array([w0 * w1 - x0 * x1 - y0 * y1 - z0 * z1,
                        w0 * x1 + x0 * w1 + y0 * z1 - z0 * y1,
                        w0 * y1 - x0 * z1 + y0 * w1 + z0 * x1,
                        w0 * z1 + x0 * y1 - y0 * x1 + z0 * w1])
        assert np.allclose(out[3:7], ref, atol=1e-12)


def test_rk4_fourth_order_convergence():
    c = cfg(renorm_q=0)
    s = W.random_states(11, 1)[0]
    prm = W.nominal_params(1)[0]
    u = np.array([9000.0, 16000.0, 12000.0, 20000.0])
    T = 0.5
    dt0 = 0.01

    def run(dt):
        return O.dynamics_batch(c, s[None], u[None], prm[None], dt=dt, renorm=0,
                                n_steps=int(round(T / dt)))[0]

    ref = run(dt0 / 64)
    errs = [np.linalg.norm((run(dt0 / k) - ref) / np.maximum(np.abs(ref), 1.0))
            for k in (1, 2, 4)]
    for a, b in zip(errs, errs[1:]):
        assert 16 * 0.9 < a / b < 16 * 1.1


def test_renormalisation_keeps_unit_quaternion():
    c = cfg(renorm_q=1)
    s = W.random_states(2, 4)
    prm = W.nominal_params(4)
    out = O.dynamics_batch(c, s, np.full((4, 4), 12000.0), prm, n_steps=50)
    assert np.allclose(np.linalg.norm(out[:, 3:7], axis=1), 1.0, atol=1e-15)


# ----------------------------------------------------------------------------- MDP pieces
def test_reward_algebra():
    C = W.REWARD
    s = np.zeros(17)
    s[3] = 1.0
    a = np.full(4, C[5])
    assert O.reward(C, s, a) == pytest.approx(C[6], abs=1e-15)
    s[3] = -1.0  # double cover: q_w = -1 is the same attitude, zero cost
    assert O.reward(C, s, a) == pytest.approx(C[6], abs=1e-15)
    s2 = np.zeros(17)
    s2[0:3] = [0.1, -0.2, 0.3]
    s2[3:7] = [math.cos(0.2), math.sin(0.2), 0, 0]
    s2[7:10] = [1, 2, 3]
    s2[10:13] = [-1, 0.5, 2]
    a2 = np.array([0.1, -0.5, 0.9, 0.0])
    exp = (-C[0] * 0.14 - C[1] * math.sin(0.2) ** 2 - C[2] * 14 - C[3] * 5.25
           - C[4] * np.sum((a2 - C[5]) ** 2) + C[6])
    assert O.reward(C, s2, a2) == pytest.approx(exp, rel=1e-14)
    s2[5] = np.nan
    assert O.reward(C, s2, a2) == 0.0


def test_reset_distribution_and_euler_composition():
    c = W.config("c2")
    S, P = [], []
    for env in range(400):
        s, prm, dist = O.reset_env(c, env, 3)
        S.append(s)
        P.append(prm)
        assert np.all(dist == 0.0)
    S, P = np.array(S), np.array(P)
    assert np.all(np.abs(S[:, 0:3]) <= 0.2)
    assert np.all(np.abs(S[:, 7:10]) <= 1.0) and np.all(np.abs(S[:, 10:13]) <= 1.0)
    assert np.all((S[:, 13:17] >= 0) & (S[:, 13:17] <= 21702.0))
    assert np.allclose(np.linalg.norm(S[:, 3:7], axis=1), 1.0, atol=1e-15)
    assert np.all(np.abs(P[:, 0] / 0.027 - 1) <= 0.2)
    assert np.all((P[:, 6] >= 0.03) & (P[:, 6] <= 0.15))
    assert np.all(np.abs(P[:, 4] / 3.16e-10 - 1) <= 0.1)
    # R(q) equals Rz(yaw) Ry(pitch) Rx(roll) for the recovered angles (all within 30 deg)
    for s in S[:20]:
        o = O.obs_actor(c, s, np.zeros(64))
        R = o[3:12].reshape(3, 3)
        pitch = -math.asin(R[2, 0])
        roll = math.atan2(R[2, 1], R[2, 2])
        yaw = math.atan2(R[1, 0], R[0, 0])
        for ang in (roll, pitch, yaw):
            assert abs(ang) <= math.radians(30) + 1e-12

        def rx(a):
            return np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])

        def ry(a):
            return np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])

        def rz(a):
            return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])

        assert np.allclose(rz(yaw) @ ry(pitch) @ rx(roll), R, atol=1e-12)
    # nominal config (no DR) gives the nominal parameters exactly
    _, prm, _ = O.reset_env(W.config("c1"), 5, 0)
    assert prm[0] == 0.027 and prm[6] == 0.15 and prm[4] == 3.16e-10


def test_actor_observation_layout():
    c = cfg()
    s = W.random_states(4, 1)[0]
    hist = np.arange(64, dtype=float)
    o = O.obs_actor(c, s, hist)
    assert o.size == 82
    assert np.array_equal(o[0:3], s[0:3]) and np.array_equal(o[12:15], s[7:10])
    assert np.array_equal(o[15:18], s[10:13]) and np.array_equal(o[18:], hist)
    R = o[3:12].reshape(3, 3)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) == pytest.approx(1.0)
    nz = O.obs_noise(dict(c, sig_p=0.1, sig_R=0.0, sig_v=0.2, sig_w=0.3), 3, 17)
    assert np.all(nz[3:12] == 0.0) and np.all(nz[0:3] != 0.0)
    assert np.all(O.obs_noise(c, 3, 17) == 0.0)


def test_critic_observation_layouts():
    s = W.random_states(6, 1)[0]
    hist = np.linspace(-1, 1, 64)
    c = cfg()
    oc = O.obs_critic(c, s, hist, np.zeros(6))
    assert oc.size == 86 and O.critic_in(c) == 90
    assert np.array_equal(oc[:82], O.obs_actor(c, s, hist))
    assert np.allclose(oc[82:], 2 * s[13:17] / 21702.0 - 1)
    cp = cfg(critic_layout=1)
    assert O.critic_in(cp) == 96
    pv = O.priv(cp, [0.027 * 1.1, 1.4e-5, 1.4e-5 * 0.9, 2.2e-5, 3.16e-10, 0.005, 0.03, 0], np.zeros(6))
    assert np.allclose(pv, [0.1, 0, -0.1, 0, 0, 0.03 / 0.15 - 1])
    c28 = cfg(critic_layout=2, dist_f=0.01, dist_tau=1e-4)
    assert O.critic_in(c28) == 32  # 28 privileged dims + 4 action dims
    pv = O.priv(c28, W.nominal_params(1)[0], [0.005, 0, -0.01, 1e-4, 0, 0])
    assert np.allclose(pv, [0.5, 0, -1, 1, 0, 0])


def test_curriculum_reaches_target_in_three_steps():
    f, t = W.CURRICULUM["factor"], W.CURRICULUM["target"]
    Cv = np.array(W.REWARD)
    seq = []
    for _ in range(5):
        Cv = O.curriculum(f, t, Cv)
        seq.append(Cv[4])
    assert seq[0] == pytest.approx(0.01 * 50 ** (1 / 3), rel=1e-12)
    assert seq[2] == pytest.approx(0.5, rel=1e-12) and seq[3] == seq[4] == 0.5
    assert np.allclose(Cv[[0, 1, 2, 3, 5, 6]], np.array(W.REWARD)[[0, 1, 2, 3, 5, 6]])
