"""Tensor-core rollout engine (tcgen05 TF32 with the hi/lo split) against the FP64 oracle,
teacher-forced per call; schedule invariance and determinism of the engine itself."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from helpers import (STATE_SCALE, assert_close, compare_records, cpu, f64, gpu_records,
                     lib_config, oracle_envs, u32)

pytestmark = pytest.mark.gpu

TC = 2  # qsim_rollout_engine: tensor cores


def _actor(d, hidden=64, seed=0):
    dd = dict(d)
    dd["seed"] = seed
    return O.init_params(dd, 0, O.actor_in(d), hidden, 4).astype(np.float32)


def _run_parity(q, n, calls, n_hist=None, **over):
    kw = dict(capacity=6, learning_starts=3, episode_len=40, sig_p=0.005, sig_R=0.01,
              sig_v=0.02, sig_w=0.02)
    kw.update(over)
    if n_hist is not None:
        kw["n_hist"] = n_hist
    d, cfg, veh = lib_config(q, "c2", n_envs=n, **kw)
    h = q.qsim_create(cfg, veh)
    cap = kw["capacity"]
    try:
        assert q.qsim_rollout_engine(h, TC) == TC
        actor = _actor(d)
        A = torch.tensor(actor, device="cuda")
        ids = np.arange(n)
        for call, T in enumerate(calls):
            info = q.qsim_info_get(h)
            e = oracle_envs(info, ids)
            t0, head0 = info["t_now"], info["head"]
            q.qsim_rollout(h, A, 64, T, 0.1)
            q.qsim_sync(h)
            ref = O.rollout(d, W.REWARD, e, T, t0, actor=actor.astype(np.float64), hidden=64,
                            sigma_e=0.1, n_threads=8)
            info = q.qsim_info_get(h)
            slots = [(head0 + k) % cap for k in range(T)]
            g = gpu_records(info, slots, ids)
            compare_records({k: v[:1] for k, v in g.items()}, {k: v[:1] for k, v in ref.items()},
                            what=f"tc rollout{call}.0")
            if T == 1:
                assert_close(f64(info["state"])[:, :n].T, e["s"], STATE_SCALE, what="state")
                nh4 = 4 * d["n_hist"]  # only the entries that are actor inputs
                assert_close(f64(info["hist"])[:nh4, :n].T, e["hist"][:, :nh4], 1.0, what="hist")
                assert np.array_equal(u32(info["ep_step"])[:n], e["ep_step"])
            else:
                same = np.all(g["rec_flags"] == ref["rec_flags"], axis=0)
                assert same.mean() > 0.99
                assert_close(g["rec_s"][:, same], ref["rec_s"][:, same], STATE_SCALE, what="multi s")
                assert_close(g["rec_a"][:, same], ref["rec_a"][:, same], 1.0, what="multi a")
    finally:
        q.qsim_destroy(h)


@pytest.mark.parametrize("n", [300, 1000, 64, 257])
def test_tc_rollout_parity(gpu, n):
    """Ragged tiles (300, 257: partial 128-env tiles and inactive warps), a single partial
    tile (64), several 256-env blocks (1000); warm-up steps then actor steps."""
    _run_parity(gpu, n, (2, 1, 3, 1))


def test_tc_rollout_parity_short_history(gpu):
    """History shorter than the 16-slot ring: the lag blocks past n_hist carry zero weights."""
    _run_parity(gpu, 300, (4, 1, 2), n_hist=5)


def test_tc_rollout_parity_without_motor_lag(gpu):
    """The ablation study's variant without rotor delay on the tensor-core engine."""
    _run_parity(gpu, 300, (2, 1, 3, 1), motor_lag_off=1)


def test_tc_rollout_parity_without_history(gpu):
    """No action history (18-input actor): every lag block of W1 is zero."""
    _run_parity(gpu, 200, (3, 1), n_hist=0)


def test_tc_rollout_without_replay_and_noise(gpu):
    """No replay ring (nothing recorded) and sigma_e = 0 (deterministic actions): the state
    and the episode counters still follow the oracle."""
    q = gpu
    n = 150
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=0, learning_starts=0, episode_len=6)
    h = q.qsim_create(cfg, veh)
    try:
        q.qsim_rollout_engine(h, TC)
        actor = _actor(d)
        A = torch.tensor(actor, device="cuda")
        ids = np.arange(n)
        for T in (1, 4, 1):
            info = q.qsim_info_get(h)
            e = oracle_envs(info, ids)
            t0 = info["t_now"]
            q.qsim_rollout(h, A, 64, T, 0.0)
            q.qsim_sync(h)
            O.rollout(d, W.REWARD, e, T, t0, actor=actor.astype(np.float64), hidden=64,
                      sigma_e=0.0, n_threads=8)
            info = q.qsim_info_get(h)
            same = (u32(info["ep_step"])[:n] == e["ep_step"]) & (u32(info["n_done"])[:n] == e["n_done"])
            if T == 1:  # one step from identical inputs: counters exact
                assert same.all()
                assert_close(f64(info["state"])[:, :n].T, e["s"], STATE_SCALE, what="state")
            else:  # several steps: a termination decision may differ where |p| sits at the box
                assert same.mean() > 0.98
    finally:
        q.qsim_destroy(h)


def test_tc_episode_ends_clear_the_action_ring(gpu):
    """Episodes of 4 steps inside one 10-step call: the ring is cleared at every episode end
    (per lane, inside a warp where other lanes continue) and refilled step by step."""
    _run_parity(gpu, 200, (10, 1), capacity=12, learning_starts=0, episode_len=4)


def test_tc_full_size_sampled(gpu):
    """65,536 envs, default schedule of the engine; 256 sampled envs checked."""
    q = gpu
    n = 65536
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=4, learning_starts=0)
    h = q.qsim_create(cfg, veh)
    try:
        q.qsim_rollout_engine(h, TC)
        actor = _actor(d)
        A = torch.tensor(actor, device="cuda")
        q.qsim_rollout(h, A, 64, 3, 0.1)
        ids = np.unique([O.replay_index(int(O.philox([i, 0, 4 << 24, 0], [0, 0])[0]), n)
                         for i in range(256)])
        info = q.qsim_info_get(h)
        e = oracle_envs(info, ids)
        t0, head0 = info["t_now"], info["head"]
        q.qsim_rollout(h, A, 64, 1, 0.1)
        q.qsim_sync(h)
        ref = O.rollout(d, W.REWARD, e, 1, t0, actor=actor.astype(np.float64), hidden=64,
                        sigma_e=0.1, n_threads=8)
        info = q.qsim_info_get(h)
        compare_records(gpu_records(info, [head0], ids), ref, what="c2 tc sampled")
        assert_close(f64(info["state"])[:, ids].T, e["s"], STATE_SCALE, what="c2 tc state")
    finally:
        q.qsim_destroy(h)


def test_tc_schedule_invariant_and_deterministic(gpu):
    """Each env's arithmetic does not depend on which envs share its tile: a repeated launch
    grouping reproduces the run bit for bit, and other groupings (partitions, chunks) agree
    to FP32 rounding.  They are not bitwise equal because each launch writes the action
    history back as the value of its fp16 hi/lo pair (within 2^-22 relative of the action)
    and the next launch splits it again."""
    q = gpu
    n = 40000
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=8, learning_starts=2)
    A = torch.tensor(_actor(d), device="cuda")
    outs = []
    for parts, chunk in ((1, 0), (1, 0), (3, 2), (2, 1), (1, 2)):
        h = q.qsim_create(cfg, veh)
        q.qsim_rollout_engine(h, TC)
        q.qsim_rollout_schedule(h, parts, chunk)
        q.qsim_rollout(h, A, 64, 5, 0.1)
        q.qsim_sync(h)
        info = q.qsim_info_get(h)
        outs.append([cpu(info[k]).copy() for k in ("records", "side", "state", "hist", "ep_step")])
        q.qsim_destroy(h)
    for x, y in zip(outs[1], outs[0]):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    for o in outs[2:]:
        for k, (x, y) in enumerate(zip(o, outs[0])):
            if x.dtype == np.float32:
                np.testing.assert_allclose(x, y, rtol=1e-5, atol=1e-6)
            else:
                assert np.array_equal(x, y)


def test_tc_persistent_units_beyond_one_wave(gpu):
    """65,536 envs = 171 groups of 384 on at most one CTA per SM, 2-step units: chunk k of a
    group starts after chunk k-1 of that group, on whichever CTA takes it.  Compared with
    one launch per group for the same 7 steps (FP32-rounding agreement, see above) and, on
    sampled envs, with the oracle for the last step."""
    q = gpu
    n = 65536
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=16, learning_starts=0)
    actor = _actor(d)
    A = torch.tensor(actor, device="cuda")
    outs = []
    for parts, chunk in ((1, 2), (4, 100)):
        h = q.qsim_create(cfg, veh)
        q.qsim_rollout_engine(h, TC)
        q.qsim_rollout_schedule(h, parts, chunk)
        q.qsim_rollout(h, A, 64, 7, 0.1)
        q.qsim_sync(h)
        info = q.qsim_info_get(h)
        outs.append([cpu(info[k]).copy() for k in ("records", "state", "hist", "ep_step")])
        if parts == 1:
            ids = np.unique([O.replay_index(int(O.philox([i, 0, 4 << 24, 0], [0, 0])[0]), n)
                             for i in range(256)])
            e = oracle_envs(info, ids)
            t0, head0 = info["t_now"], info["head"]
            q.qsim_rollout(h, A, 64, 1, 0.1)
            q.qsim_sync(h)
            ref = O.rollout(d, W.REWARD, e, 1, t0, actor=actor.astype(np.float64), hidden=64,
                            sigma_e=0.1, n_threads=8)
            info = q.qsim_info_get(h)
            compare_records(gpu_records(info, [head0], ids), ref, what="persistent sampled")
        q.qsim_destroy(h)
    for x, y in zip(outs[0], outs[1]):
        if x.dtype == np.float32:
            np.testing.assert_allclose(x, y, rtol=1e-5, atol=1e-6)
        else:
            assert np.array_equal(x, y)


def test_tc_engine_other_widths_run_on_simt(gpu):
    q = gpu
    d, cfg, veh = lib_config(q, "c2", n_envs=64, capacity=4)
    h = q.qsim_create(cfg, veh)
    try:
        q.qsim_rollout_engine(h, TC)
        A = torch.tensor(_actor(d, 32), device="cuda")
        # hidden 32 has no tensor-core kernel: the SIMT engine runs instead
        q.qsim_rollout(h, A, 32, 2, 0.1)
        q.qsim_sync(h)
        assert q.qsim_rollout_engine(h, 5) == TC
    finally:
        q.qsim_destroy(h)


def test_tc_persistent_1000_steps_every_step_teacher_forced(gpu):
    """The benchmark's call: 65,536 envs x 1,000 steps in one persistent launch of 50-step
    units (each unit reloads its envs' state and action ring from HBM), observation noise
    on.  Every step of 256 sampled envs is replayed on the oracle from the GPU's own ring:
    state s_t from record t, action history from the records of the same episode, the
    episode's domain-randomised parameters from the oracle's reset of (env, episode); the
    action, reward, flags and successor state (record t+1, the side slot at episode ends,
    the final state after the last step) are compared per step.  Termination decisions may
    differ only where the oracle's successor sits within 1e-5 m of the box edge."""
    q = gpu
    n, T = 65536, 1000
    d, cfg, veh = lib_config(q, "c2", n_envs=n, capacity=T, learning_starts=0, sig_p=0.005,
                             sig_R=0.01, sig_v=0.02, sig_w=0.02)
    h = q.qsim_create(cfg, veh)
    try:
        q.qsim_rollout_engine(h, TC)
        q.qsim_rollout_schedule(h, 1, 50)
        actor = _actor(d)
        A = torch.tensor(actor, device="cuda")
        ids = np.unique([O.replay_index(int(O.philox([i, 0, 4 << 24, 0], [0, 0])[0]), n)
                         for i in range(256)])
        k = ids.size
        q.qsim_rollout(h, A, 64, T, 0.1)
        q.qsim_sync(h)
        info = q.qsim_info_get(h)
        assert info["t_now"] == T and info["size"] == T
        idt = torch.tensor(ids, device="cuda")
        R = info["records"][:, :, idt]
        rec = f64(R)                                   # [T][F][k]
        flags = cpu(R).view(np.uint32)[:, 22]          # [T][k]
        side = f64(info["side"][:, :, idt])            # [T][17][k]
        final = f64(info["state"][:, idt]).T           # [k][17]
        del R
        rs, ra, rr = rec[:, 0:17].transpose(0, 2, 1), rec[:, 17:21].transpose(0, 2, 1), rec[:, 21]
        resets = {}

        def episode_params(env, ep):
            if (env, ep) not in resets:
                resets[(env, ep)] = O.reset_env(d, env, ep)[1:]
            return resets[(env, ep)]

        ep_index = np.zeros(k, np.uint32)
        actor64 = actor.astype(np.float64)
        edge = 0
        worst = 0.0
        for t in range(T):
            ep_step = flags[t] >> 8
            hist = np.zeros((k, 64))
            for i in range(1, 17):
                has = ep_step >= i
                if t - i >= 0:
                    hist[has, 4 * (i - 1):4 * i] = ra[t - i][has]
                else:
                    assert not has.any()
            prm = np.array([episode_params(int(e), int(p))[0] for e, p in zip(ids, ep_index)])
            dist = np.array([episode_params(int(e), int(p))[1] for e, p in zip(ids, ep_index)])
            e = dict(env_id=ids.astype(np.uint32), s=rs[t].copy(), prm=prm, dist=dist, hist=hist,
                     ep_index=ep_index.copy(), ep_step=ep_step.astype(np.uint32),
                     ep_ret=np.zeros(k), n_done=np.zeros(k, np.uint32),
                     len_sum=np.zeros(k, np.uint32), ret_sum=np.zeros(k))
            ref = O.rollout(d, W.REWARD, e, 1, t, actor=actor64, hidden=64, sigma_e=0.1)
            of, gf = ref["rec_flags"][0], flags[t]
            odone = (of & 3) != 0
            # successor the oracle computed: side slot if done, else its new state
            s_ref = np.where(odone[:, None], np.nan_to_num(ref["side"][0]), e["s"])
            mism = gf != of
            if mism.any():
                pos = np.abs(s_ref[mism, 0:3])
                assert np.all(np.min(np.abs(pos - d["term_pos"]), axis=1) < 1e-5), \
                    f"step {t}: flags differ away from the box edge: {gf[mism]} vs {of[mism]}"
                edge += int(mism.sum())
            ok = ~mism
            assert_close(ra[t][ok], ref["rec_a"][0][ok], 1.0, what=f"step {t} a")
            assert_close(rr[t][ok], ref["rec_r"][0][ok], 1.0, what=f"step {t} r")
            gdone = (gf & 3) != 0
            if t + 1 < T:
                s_gpu = np.where(gdone[:, None], side[t].T, rs[t + 1])
            else:
                s_gpu = np.where(gdone[:, None], side[t].T, final)
            sel = ok & ~np.isnan(s_ref).any(axis=1)
            assert_close(s_gpu[sel], s_ref[sel], STATE_SCALE, what=f"step {t} s'")
            worst = max(worst, float(np.max(np.abs(ra[t][ok] - ref["rec_a"][0][ok]))))
            ep_index = ep_index + gdone.astype(np.uint32)
        assert edge <= 3, edge
        assert worst < 1e-3
    finally:
        q.qsim_destroy(h)
