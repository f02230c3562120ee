"""GPU parity of the env-side entry points against the FP64 oracle (teacher-forced: each
call's FP32 inputs are read back and promoted to FP64 for the oracle)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from helpers import (STATE_SCALE, assert_close, compare_records, cpu, f64, gpu_records,
                     lib_config, oracle_envs, u32)

pytestmark = pytest.mark.gpu

SIMT = 1  # qsim_rollout_engine: the SIMT kernel (paired FMA); the tensor-core engine has its own file


def test_philox_streams_bit_exact(gpu):
    q = gpu
    seed = 0x123456789ABCDEF0
    for tag, sub, c1, run in ((0, 0, 0, 0), (3, 1, 777, 5), (4, 0, 2**31 + 3, 511)):
        out = torch.empty(4 * 1000, dtype=torch.int32, device="cuda")
        q.qsim_philox_fill(seed, run, tag, sub, c1, out, kind=0)
        g = u32(out).reshape(-1, 4)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i in list(range(0, 1000, 37)) + [999]:
            ref = O.philox([i, c1, (tag << 24) | sub, run], key)
            assert [int(x) for x in g[i]] == [int(x) for x in ref]
        # uniforms: exact in float32
        q.qsim_philox_fill(seed, run, tag, sub, c1, out, kind=1)
        uf = cpu(out).view(np.float32).reshape(-1, 4)
        ref_u = np.array([[O.uniform(int(x)) for x in row] for row in g], dtype=np.float64)
        assert np.array_equal(uf.astype(np.float64), ref_u)
        # Box-Muller normals: float32 vs float64
        q.qsim_philox_fill(seed, run, tag, sub, c1, out, kind=2)
        z = cpu(out).view(np.float32).reshape(-1, 4)[:, :2].astype(np.float64)
        ref_z = np.array([[O.gauss(r[0], r[1]), O.gauss(r[2], r[3])] for r in g])
        assert_close(z, ref_z, 1.0, rtol=1e-5, what="gauss")
    # host-side Philox is the same stream
    assert q.qsim_philox_host([1, 2, 3, 4], [5, 6]) == [int(x) for x in O.philox([1, 2, 3, 4], [5, 6])]


@pytest.mark.parametrize("n,steps", [(1, 1), (1000, 1), (333, 25), (4096, 3)])
def test_dynamics_step_parity(gpu, n, steps):
    q = gpu
    d = W.config("c1")
    veh = q.make_params(d)
    ld = q.padded(n)
    s = W.random_states(7 + n, n)
    prm = W.random_params(8 + n, n)
    u = W.random_actions(9 + n, (n, 4), 0.0, 21702.0)
    dist = W.random_actions(10 + n, (n, 6), -1e-3, 1e-3)

    def dev(x, rows):
        t = torch.zeros(rows, ld, dtype=torch.float32)
        t[:, :n] = torch.tensor(x.T, dtype=torch.float32)
        return t.cuda()

    S, Pm, U, D = dev(s, 17), dev(prm, 8), dev(u, 4), dev(dist, 6)
    out = torch.empty_like(S)
    q.qsim_dynamics_step(veh, Pm, D, S, U, 0.01, 1, n, ld, steps, out)
    torch.cuda.synchronize()
    ref = O.dynamics_batch(d, f64(S)[:, :n].T, f64(U)[:, :n].T, f64(Pm)[:, :n].T,
                           f64(D)[:, :n].T, dt=np.float64(np.float32(0.01)), renorm=1,
                           n_steps=steps)
    assert_close(f64(out)[:, :n].T, ref, STATE_SCALE, what="state")


def _bench_start(d, n):
    """Initial states of the dynamics benchmark kernel, formed in FP32 as it forms them: a
    per-env offset off = 1e-3 (e mod 1024) / 1024 on position, roll/yaw rate and the
    motor speeds around the hover set-point, level attitude, zero velocity."""
    f32 = np.float32
    off = (f32(1e-3) * (np.arange(n) % 1024).astype(f32)) / f32(1024)
    uh = np.sqrt(f32(d["mass"]) * f32(d["g"]) / (f32(4) * f32(d["kf"])))
    s = np.zeros((n, 17), f32)
    s[:, 0], s[:, 1], s[:, 2] = off, -off, f32(0.5) * off
    s[:, 3] = 1
    s[:, 10], s[:, 12] = off, -off
    s[:, 13:17] = (uh * (f32(1) + off))[:, None]
    u = np.full((n, 4), uh, f32)
    prm = np.zeros((n, 8), f32)
    prm[:, :7] = [d["mass"], d["Jx"], d["Jy"], d["Jz"], d["kf"], d["km"], d["tm"]]
    return s.astype(np.float64), u.astype(np.float64), prm.astype(np.float64)


def _fp32_config(d):
    """The vehicle constants as the GPU holds them (FP32), promoted to FP64."""
    dd = {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in d.items()}
    dd["rotor_pos"] = [float(np.float32(x)) for x in d["rotor_pos"]]
    dd["rotor_dir"] = [float(np.float32(x)) for x in d["rotor_dir"]]
    return dd


@pytest.mark.parametrize("n,steps", [(8192, 1), (1000, 10), (3000, 100)])
def test_dynamics_bench_parity(gpu, n, steps):
    """The kernel timed as the simulator benchmark (Sec. V: forward dynamics only, hover
    set-point) against the oracle's batch dynamics from the same initial states, element by
    element at the per-call tolerance.  Up to 100 steps the FP32 rounding accumulated in
    the hover balance (thrust / mass - g) stays below a fifth of it."""
    q = gpu
    d = W.config("c1")
    veh = q.make_params(d)
    ld = q.padded(n)
    out = torch.full((17, ld), float("nan"), device="cuda")
    q.qsim_dynamics_bench(veh, n, ld, steps, 0.01, out)
    torch.cuda.synchronize()
    s, u, prm = _bench_start(d, n)
    ref = O.dynamics_batch(_fp32_config(d), s, u, prm, None, dt=np.float64(np.float32(0.01)),
                           renorm=1, n_steps=steps)
    assert_close(f64(out)[:, :n].T, ref, STATE_SCALE, what=f"bench {steps} steps")


def test_dynamics_bench_long_run_invariants(gpu):
    """1,000 steps (10 s) of the open-loop hover, beyond per-call range: the hover is
    unstable, so an FP32 rounding of the torque balance (one ulp of a rotor moment,
    ~1e-10 N m, e.g. from a fused multiply-add that breaks the exact cancellation of the
    symmetric rotors) grows like g (dtau / J) t^4 / 24 into ~3 cm of horizontal drift over
    10 s, and the thrust balance (thrust / m - g) accumulates ~5e-4 m in height.  Checked
    by invariants: finite, unit quaternion, motor speeds settled on the set-point (the lag
    factor 0.9355 per step leaves < 1e-28 of the initial offset; an FP32 increment below
    half an ulp rounds away, which can leave the speed up to 7 ulps = 5e-7 relative off the
    set-point); against the oracle within those drift bounds (height 1e-2 m, horizontal
    0.1 m, velocity 0.1 m/s)."""
    q = gpu
    d = W.config("c1")
    veh = q.make_params(d)
    n, steps = 2048, 1000
    ld = q.padded(n)
    out = torch.full((17, ld), float("nan"), device="cuda")
    q.qsim_dynamics_bench(veh, n, ld, steps, 0.01, out)
    torch.cuda.synchronize()
    g = f64(out)[:, :n].T
    s, u, prm = _bench_start(d, n)
    ref = O.dynamics_batch(_fp32_config(d), s, u, prm, None, dt=np.float64(np.float32(0.01)),
                           renorm=1, n_steps=steps)
    assert np.isfinite(g).all()
    assert np.allclose(np.linalg.norm(g[:, 3:7], axis=1), 1.0, atol=1e-6)
    assert np.allclose(g[:, 13:17], u, rtol=1e-6, atol=0)
    assert np.max(np.abs(g[:, 2] - ref[:, 2])) < 1e-2
    assert np.max(np.abs(g[:, 0:2] - ref[:, 0:2])) < 0.1
    assert np.max(np.abs(g[:, 7:10] - ref[:, 7:10])) < 0.1


def test_dynamics_rejects_bad_arguments(gpu):
    q = gpu
    veh = q.make_params(W.config("c1"))
    S = torch.zeros(17, 32, device="cuda")
    with pytest.raises(q.QsimError):
        q.qsim_dynamics_step(veh, S, None, S, S, 0.01, 1, 40, 32, 1, S)  # ld < n
    with pytest.raises(q.QsimError):
        q.qsim_dynamics_step(veh, S, None, S, S, -0.01, 1, 8, 32, 1, S)  # dt <= 0
    with pytest.raises(q.QsimError):
        q.qsim_dynamics_step(veh, S[:, 1:], None, S, S, 0.01, 1, 8, 32, 1, S)  # misaligned


def test_create_resets_like_oracle(gpu):
    q = gpu
    d, cfg, veh = lib_config(q, "c2", n_envs=200, capacity=0)
    h = q.qsim_create(cfg, veh)
    try:
        info = q.qsim_info_get(h)
        st, prm = f64(info["state"]), f64(info["params"])
        for e in (0, 1, 17, 199):
            s_ref, p_ref, _ = O.reset_env(d, e, 0)
            assert_close(st[:, e], s_ref, STATE_SCALE, what="reset state")
            assert_close(prm[:7, e], p_ref[:7], np.abs(p_ref[:7]) + 1e-30, what="reset params")
        assert np.all(f64(info["hist"]) == 0)
    finally:
        q.qsim_destroy(h)


@pytest.mark.parametrize("layout,lag_off", [(0, 0), (1, 0), (2, 0), (3, 1)])
def test_step_and_observe_parity(gpu, layout, lag_off):
    """Every critic layout (3: the symmetric critic of the ablation study, whose o_c is the
    noisy o_a); the last case also with the motor model ablated."""
    q = gpu
    n = 70
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=16, critic_layout=layout,
                             episode_len=9, sig_p=0.01, sig_R=0.02, sig_v=0.03, sig_w=0.04,
                             dist_f=0.01, dist_tau=1e-4, motor_lag_off=lag_off)
    h = q.qsim_create(cfg, veh)
    try:
        info = q.qsim_info_get(h)
        ld = info["ld"]
        da, dc = info["obs_dim"], info["critic_obs_dim"]
        for step in range(12):
            acts = torch.tensor(W.random_actions(100 + step, (4, ld), -1.3, 1.3), dtype=torch.float32,
                                device="cuda")
            info = q.qsim_info_get(h)
            ids = np.arange(n)
            e = oracle_envs(info, ids)
            t0, head0 = info["t_now"], info["head"]
            oa = torch.zeros(da, ld, device="cuda")
            oc = torch.zeros(dc, ld, device="cuda")
            rw = torch.zeros(ld, device="cuda")
            te = torch.zeros(ld, dtype=torch.uint8, device="cuda")
            tr = torch.zeros(ld, dtype=torch.uint8, device="cuda")
            q.qsim_step(h, acts, oa, oc, rw, te, tr)
            torch.cuda.synchronize()
            ref = O.rollout(d, W.REWARD, e, 1, t0, ext_actions=f64(acts)[:, :n].T[None])
            info = q.qsim_info_get(h)
            compare_records(gpu_records(info, [head0], ids), ref, what=f"step{step}")
            assert_close(f64(info["state"])[:, :n].T, e["s"], STATE_SCALE, what="next state")
            assert np.array_equal(u32(info["ep_index"])[:n], e["ep_index"])
            assert np.array_equal(u32(info["ep_step"])[:n], e["ep_step"])
            assert_close(f64(rw)[:n], ref["rec_r"][0], 1.0, what="reward out")
            assert np.array_equal(cpu(te)[:n], (ref["rec_flags"][0] & 1).astype(np.uint8))
            assert np.array_equal(cpu(tr)[:n], ((ref["rec_flags"][0] >> 1) & 1).astype(np.uint8))
            # observations of the next step
            for k in range(0, n, 7):
                o_ref = O.obs_actor(d, e["s"][k], e["hist"][k], O.obs_noise(d, k, t0 + 1))
                assert_close(f64(oa)[:, k], o_ref, 1.0, what="obs_a")
                pv = O.priv(d, e["prm"][k], e["dist"][k])
                c_ref = o_ref if layout == 3 else O.obs_critic(d, e["s"][k], e["hist"][k], pv)
                assert_close(f64(oc)[:, k], c_ref, 1.0, what="obs_c")
        st = q.qsim_stats_get(h)
        assert st["episodes"] > 0 and st["mean_length"] <= 9
    finally:
        q.qsim_destroy(h)


def _actor(d, hidden, seed=0):
    dd = dict(d)
    dd["seed"] = seed
    return O.init_params(dd, 0, O.actor_in(d), hidden, 4).astype(np.float32)


@pytest.mark.parametrize("hidden,n,warps,lag_off", [(64, 300, 0, 0), (64, 1000, 4, 0),
                                                    (32, 100, 0, 0), (128, 200, 2, 0),
                                                    (64, 64, 10, 0), (64, 300, 0, 1)])
def test_rollout_parity(gpu, hidden, n, warps, lag_off):
    """Widths, warps per block, ragged env counts; the last case without the motor model
    (the ablation study's variant without rotor delay)."""
    q = gpu
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=6, learning_starts=3, episode_len=40,
                             sig_p=0.005, sig_R=0.01, sig_v=0.02, sig_w=0.02,
                             motor_lag_off=lag_off)
    h = q.qsim_create(cfg, veh)
    q.qsim_rollout_engine(h, SIMT)
    try:
        if warps:
            q.qsim_rollout_tune(h, warps)
        actor = _actor(d, hidden)
        A = torch.tensor(actor, device="cuda")
        ids = np.arange(n)
        for call, T in enumerate((2, 1, 3, 1)):
            info = q.qsim_info_get(h)
            e = oracle_envs(info, ids)
            t0, head0 = info["t_now"], info["head"]
            q.qsim_rollout(h, A, hidden, T, 0.1)
            torch.cuda.synchronize()
            ref = O.rollout(d, W.REWARD, e, T, t0, actor=actor.astype(np.float64), hidden=hidden,
                            sigma_e=0.1, n_threads=8)
            info = q.qsim_info_get(h)
            slots = [(head0 + k) % 6 for k in range(T)]
            if T == 1:
                compare_records(gpu_records(info, slots, ids), ref, what=f"rollout{call}")
                assert_close(f64(info["state"])[:, :n].T, e["s"], STATE_SCALE, what="state")
                assert_close(f64(info["hist"])[:, :n].T, e["hist"], 1.0, what="hist")
                assert np.array_equal(u32(info["ep_step"])[:n], e["ep_step"])
            else:
                # several steps in one call: first step strictly, later steps where the
                # trajectories have not been separated by a termination decision
                g = gpu_records(info, slots, ids)
                compare_records({k: v[:1] for k, v in g.items()}, {k: v[:1] for k, v in ref.items()},
                                what=f"rollout{call}.0")
                same = np.all(g["rec_flags"] == ref["rec_flags"], axis=0)
                assert same.mean() > 0.99
                assert_close(g["rec_s"][:, same], ref["rec_s"][:, same], STATE_SCALE, what="multi s")
    finally:
        q.qsim_destroy(h)


def test_rollout_full_size_sampled(gpu):
    """65,536 envs in the benchmark's launch configuration; 256 sampled envs checked."""
    q = gpu
    n = 65536
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=4, learning_starts=0)
    h = q.qsim_create(cfg, veh)
    q.qsim_rollout_engine(h, SIMT)
    try:
        actor = _actor(d, 64)
        A = torch.tensor(actor, device="cuda")
        q.qsim_rollout(h, A, 64, 3, 0.1)
        ids = np.unique([O.replay_index(int(O.philox([i, 0, 4 << 24, 0], [0, 0])[0]), n)
                         for i in range(256)])
        info = q.qsim_info_get(h)
        e = oracle_envs(info, ids)
        t0, head0 = info["t_now"], info["head"]
        q.qsim_rollout(h, A, 64, 1, 0.1)
        torch.cuda.synchronize()
        ref = O.rollout(d, W.REWARD, e, 1, t0, actor=actor.astype(np.float64), hidden=64,
                        sigma_e=0.1, n_threads=8)
        info = q.qsim_info_get(h)
        compare_records(gpu_records(info, [head0], ids), ref, what="c2 sampled")
        assert_close(f64(info["state"])[:, ids].T, e["s"], STATE_SCALE, what="c2 state")
    finally:
        q.qsim_destroy(h)


def test_rollout_deterministic(gpu):
    q = gpu
    d, cfg, veh = lib_config(q, "c2", n_envs=500, capacity=20, learning_starts=0)
    A = torch.tensor(_actor(d, 64), device="cuda")
    outs = []
    for _ in range(2):
        h = q.qsim_create(cfg, veh)
        q.qsim_rollout_engine(h, SIMT)
        q.qsim_rollout(h, A, 64, 17, 0.1)
        info = q.qsim_info_get(h)
        outs.append((cpu(info["records"]).copy(), cpu(info["state"]).copy()))
        q.qsim_destroy(h)
    assert np.array_equal(outs[0][0].view(np.uint32), outs[1][0].view(np.uint32))
    assert np.array_equal(outs[0][1].view(np.uint32), outs[1][1].view(np.uint32))


def test_recalc_rewards_parity(gpu):
    q = gpu
    n = 40
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=30, episode_len=7, learning_starts=0)
    h = q.qsim_create(cfg, veh)
    q.qsim_rollout_engine(h, SIMT)
    try:
        A = torch.tensor(_actor(d, 64), device="cuda")
        q.qsim_rollout(h, A, 64, 45, 0.3)  # wraps the ring
        C2 = list(W.REWARD)
        C2[4] = 0.37
        C2[0] = 2.0
        q.qsim_set_reward(h, C2, 0.1)
        q.qsim_recalc_rewards(h)
        torch.cuda.synchronize()
        info = q.qsim_info_get(h)
        cap = info["capacity"]
        rec = f64(info["records"])
        raw = cpu(info["records"]).view(np.uint32)
        buf = dict(s=rec[:, 0:17, :n].transpose(0, 2, 1), a=rec[:, 17:21, :n].transpose(0, 2, 1),
                   r=np.zeros((cap, n)), flags=raw[:, 22, :n], priv=np.zeros((cap, n, 6)),
                   side=np.nan_to_num(f64(info["side"])[:, :, :n].transpose(0, 2, 1)),
                   head=info["head"], size=info["size"], t_now=info["t_now"])
        O.recalc_rewards(C2, buf, f64(info["state"])[:, :n].T)
        assert_close(rec[:, 21, :n], buf["r"], 1.0, what="recalc")
    finally:
        q.qsim_destroy(h)


def test_recalc_rewards_batch_equals_per_set(gpu):
    """One launch over several env sets (different sizes, fill levels and reward constants)
    gives bit for bit what qsim_recalc_rewards gives on each set."""
    q = gpu
    sets = []
    try:
        for k, (n, cap, steps) in enumerate(((40, 30, 45), (7, 16, 9), (300, 12, 20), (64, 8, 0))):
            d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=cap, episode_len=7, learning_starts=0,
                                     seed=k, run_id=k)
            pair = []
            for _ in range(2):
                h = q.qsim_create(cfg, veh)
                q.qsim_rollout_engine(h, SIMT)
                if steps:
                    q.qsim_rollout(h, torch.tensor(_actor(d, 64), device="cuda"), 64, steps, 0.3)
                C2 = list(W.REWARD)
                C2[4] = 0.2 + 0.1 * k
                q.qsim_set_reward(h, C2, 0.1)
                pair.append(h)
            sets.append(pair)
        for a, _ in sets:
            q.qsim_recalc_rewards(a)
        q.qsim_recalc_rewards_batch([b for _, b in sets])
        torch.cuda.synchronize()
        for a, b in sets:
            ra, rb = cpu(q.qsim_info_get(a)["records"]), cpu(q.qsim_info_get(b)["records"])
            assert np.array_equal(ra.view(np.uint32), rb.view(np.uint32))
    finally:
        for pair in sets:
            for h in pair:
                q.qsim_destroy(h)


def test_partitioned_schedule_is_bitwise_identical(gpu):
    """Env partitions on internal streams, advanced in time chunks, give exactly the
    single-launch results (same per-env arithmetic, different launch grouping)."""
    q = gpu
    n = 65536
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=8, learning_starts=2)
    A = torch.tensor(_actor(d, 64), device="cuda")
    outs = []
    for parts, chunk in ((1, 0), (3, 2), (2, 1)):
        h = q.qsim_create(cfg, veh)
        q.qsim_rollout_engine(h, SIMT)
        q.qsim_rollout_schedule(h, parts, chunk)
        q.qsim_rollout(h, A, 64, 5, 0.1)
        torch.cuda.synchronize()
        info = q.qsim_info_get(h)
        outs.append([cpu(info[k]).copy() for k in ("records", "side", "state", "hist", "ep_step")])
        q.qsim_destroy(h)
    for o in outs[1:]:
        for x, y in zip(o, outs[0]):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


@pytest.mark.parametrize("hidden", [32, 64, 128])
def test_packed_fma_kernel_is_bitwise_identical(gpu, hidden):
    """The paired-FMA (f32x2) rollout variant performs the same IEEE FMAs in the same order
    as the scalar variant: results must match bit for bit."""
    q = gpu
    n = 3000
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=12, learning_starts=2,
                             sig_p=0.01, sig_v=0.01)
    A = torch.tensor(_actor(d, hidden), device="cuda")
    outs = []
    for packed in (0, 1):
        h = q.qsim_create(cfg, veh)
        q.qsim_rollout_packed(h, packed)
        q.qsim_rollout_tune(h, 2 if hidden == 128 else 4)
        q.qsim_rollout(h, A, hidden, 20, 0.1)
        torch.cuda.synchronize()
        info = q.qsim_info_get(h)
        outs.append([cpu(info[k]).copy() for k in ("records", "side", "state", "hist")])
        q.qsim_destroy(h)
    for x, y in zip(outs[0], outs[1]):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
