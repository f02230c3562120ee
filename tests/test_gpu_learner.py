"""GPU parity of the TD3 learner (ac_update), the fused training iteration (ac_train) and
the plain-vs-persistent equivalence."""
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from helpers import (STATE_SCALE, assert_close, assert_norm_close, compare_records, cpu, f64,
                     gpu_records, lib_config, oracle_envs, u32)

pytestmark = pytest.mark.gpu


def oracle_buffer(info, n):
    cap = info["capacity"]
    rec = f64(info["records"])
    raw = cpu(info["records"]).view(np.uint32)
    priv = (rec[:, 23:29, :n].transpose(0, 2, 1).copy() if info["n_priv"]
            else np.zeros((cap, n, 6)))
    return dict(s=rec[:, 0:17, :n].transpose(0, 2, 1).copy(),
                a=rec[:, 17:21, :n].transpose(0, 2, 1).copy(), r=rec[:, 21, :n].copy(),
                flags=raw[:, 22, :n].copy(), priv=priv,
                side=np.nan_to_num(f64(info["side"])[:, :, :n].transpose(0, 2, 1)).copy(),
                head=info["head"], size=info["size"], t_now=info["t_now"])


NETS = ("actor", "actor_t", "c1", "c1_t", "c2", "c2_t", "m_a", "v_a", "m_c1", "v_c1", "m_c2",
        "v_c2")


def oracle_learner(ai):
    L = {k: f64(ai[k]).copy() for k in NETS}
    L.update(t_a=ai["t_actor"], t_c=ai["t_critic"], update_idx=ai["updates"])
    return L


def check_update(ai, Lref, dg, hp, what):
    lr, eps, b1, b2 = hp["lr"], hp["eps"], hp["beta1"], hp["beta2"]
    pairs = [("c1", "g_c1", "m_c1", "v_c1"), ("c2", "g_c2", "m_c2", "v_c2")]
    if dg["actor_updated"]:
        pairs.append(("actor", "g_a", "m_a", "v_a"))
    for name, gk, mk, vk in pairs:
        g = dg[gk]
        tol_g = 1e-4 * np.abs(g) + 1e-4 * np.sqrt(np.mean(g * g))
        # Adam's step lr * m/(sqrt(v)+eps) moves by at most this much when g moves by tol_g
        atol = np.minimum(lr * (1e-3 + eps * tol_g / (np.abs(g) + eps) ** 2), 2 * lr)
        th = f64(ai[name])
        bad = np.abs(th - Lref[name]) > atol + 1e-4 * np.abs(Lref[name]) * 1e-3
        assert not bad.any(), f"{what}.{name}: {bad.sum()} params off, e.g. {th[bad][:3]} vs {Lref[name][bad][:3]}"
        assert_close(f64(ai[mk]), Lref[mk], (1 - b1) * tol_g / 1e-4, rtol=1e-4, what=f"{what}.{mk}")
        assert_close(f64(ai[vk]), Lref[vk], (1 - b2) * 2 * (np.abs(g) + tol_g) * tol_g / 1e-4,
                     rtol=2e-4, what=f"{what}.{vk}")
        tgt = name + "_t"
        if dg["actor_updated"]:
            assert_close(f64(ai[tgt]), Lref[tgt], hp["tau"] * atol / 1e-4 + 1e-7 / 1e-4,
                         what=f"{what}.{tgt}")
    if not dg["actor_updated"]:
        assert np.array_equal(f64(ai["actor"]), Lref["actor"])


def make_run(q, n_env=3, cap=64, hidden=32, batch=64, cluster=1, layout=0, steps=40, seed=0,
             episode_len=12, **over):
    d, cfg, veh = lib_config(q, "c2" if layout == 1 else "c1", n_envs=n_env, capacity=cap,
                             critic_layout=layout, episode_len=episode_len, learning_starts=0,
                             seed=seed, sig_p=0.003, sig_R=0.003, sig_v=0.01, sig_w=0.01,
                             dist_f=0.002 if layout == 2 else 0.0, dist_tau=1e-5 if layout == 2 else 0.0,
                             **over)
    h = q.qsim_create(cfg, veh)
    hp = dict(W.TD3)
    hp.update(hidden=hidden, batch=batch)
    a = q.ac_create(q.make_ac_config(hp, cluster=cluster), h)
    info = q.qsim_info_get(h)
    for k in range(steps):
        acts = torch.tensor(W.random_actions(500 + k, (4, info["ld"])), dtype=torch.float32,
                            device="cuda")
        q.qsim_step(h, acts)
    torch.cuda.synchronize()
    return d, h, a, hp


@pytest.mark.parametrize("cluster,layout,hidden,batch", [(1, 0, 32, 64), (2, 0, 64, 64),
                                                         (4, 1, 32, 128), (1, 2, 16, 32),
                                                         (8, 0, 128, 256), (1, 0, 128, 128),
                                                         (2, 3, 64, 64), (16, 0, 64, 256),
                                                         (1, 0, 128, 512), (0, 1, 64, 256),
                                                         (1, 0, 64, 256), (1, 1, 64, 128),
                                                         (1, 0, 32, 128), (2, 0, 64, 256),
                                                         (4, 2, 32, 64)])
def test_ac_update_parity(gpu, cluster, layout, hidden, batch):
    """Cluster 16 at hidden 64 / batch 256 is the single run's automatic choice; hidden 128
    with batch 512 on one CTA is the largest shape of the batched workload; cluster 0 is
    the automatic choice with the privileged critic.  CTAs holding whole 128-sample tiles
    (1 x 128 .. 512, 2 x 128) run the target actor and target critics on the tensor cores,
    at hidden 32, 64 and 128 and with the privileged critic.  Even clusters whose CTA pairs
    hold at most 64 rows (2 x 64, 4 x 128, 8 x 256, 16 x 256, 2 x 64 symmetric, 4 x 64
    with the 28-D critic) split the twin critics over the cluster's two halves."""
    q = gpu
    d, h, a, hp = make_run(q, hidden=hidden, batch=batch, cluster=cluster, layout=layout)
    try:
        # perturb the targets away from the online nets so every term is exercised
        ai = q.ac_info_get(a)
        g = torch.Generator(device="cuda").manual_seed(3)
        for k in ("actor_t", "c1_t", "c2_t"):
            ai[k] += 0.02 * torch.randn(ai[k].shape, device="cuda", generator=g)
        torch.cuda.synchronize()
        for call in range(3):
            info = q.qsim_info_get(h)
            buf = oracle_buffer(info, info["n_envs"])
            ai = q.ac_info_get(a)
            L = oracle_learner(ai)
            q.ac_update(a, h, 1)
            torch.cuda.synchronize()
            dg = O.td3_update(d, hp, L, buf)
            ai = q.ac_info_get(a)
            assert ai["updates"] == L["update_idx"] and ai["t_actor"] == L["t_a"]
            check_update(ai, L, dg, hp, f"update{call}")
            assert_close(f64(ai["stats"])[0], dg["critic_loss"], 1.0, what="critic loss")
            if dg["actor_updated"]:
                assert_close(f64(ai["stats"])[1], dg["actor_loss"], 10.0, what="actor loss")
    finally:
        q.ac_destroy(a)
        q.qsim_destroy(h)


@pytest.mark.parametrize("lag_off,layout", [(0, 0), (1, 3)])
def test_train_iteration_parity(gpu, lag_off, layout):
    """One ac_train step = one env step (generic tile path) + one update, vs the oracle;
    also with the motor model ablated and the symmetric critic."""
    q = gpu
    d, h, a, hp = make_run(q, n_env=5, cap=32, hidden=32, batch=32, cluster=2, steps=20,
                           layout=layout, motor_lag_off=lag_off)
    try:
        for it in range(3):
            info = q.qsim_info_get(h)
            n = info["n_envs"]
            e = oracle_envs(info, np.arange(n))
            ai = q.ac_info_get(a)
            L = oracle_learner(ai)
            t0, head0 = info["t_now"], info["head"]
            q.ac_train([a], [h], 1, persistent=1)
            torch.cuda.synchronize()
            ref = O.rollout(d, W.REWARD, e, 1, t0, actor=L["actor"], hidden=32, sigma_e=0.1)
            info = q.qsim_info_get(h)
            compare_records(gpu_records(info, [head0], np.arange(n)), ref, what=f"it{it}.env")
            assert_close(f64(info["state"])[:, :n].T, e["s"], STATE_SCALE, what="state")
            buf = oracle_buffer(info, n)
            dg = O.td3_update(d, hp, L, buf)
            check_update(q.ac_info_get(a), L, dg, hp, f"it{it}.upd")
    finally:
        q.ac_destroy(a)
        q.qsim_destroy(h)


def _train_pair(q, persistent, n_runs=3, steps=25, cluster=1):
    runs, envs = [], []
    for r in range(n_runs):
        d, cfg, veh = lib_config(q, "c1", n_envs=2 + r, capacity=40, learning_starts=6,
                                 episode_len=15, seed=r, run_id=r)
        h = q.qsim_create(cfg, veh)
        hp = dict(W.TD3)
        hp.update(hidden=[32, 64, 16][r % 3], batch=[32, 64, 32][r % 3])
        a = q.ac_create(q.make_ac_config(hp, cluster=cluster), h)
        runs.append(a)
        envs.append(h)
    q.ac_train(runs, envs, steps, persistent=persistent)
    torch.cuda.synchronize()
    snap = []
    for a, h in zip(runs, envs):
        ai, info = q.ac_info_get(a), q.qsim_info_get(h)
        snap.append({k: cpu(ai[k]).copy() for k in NETS} |
                    {k: cpu(info[k]).copy() for k in ("state", "records", "hist", "ep_step")})
        q.ac_destroy(a)
        q.qsim_destroy(h)
    return snap


def test_plain_and_persistent_training_are_bitwise_equal(gpu):
    """Same cluster size: the batched launch, one launch per run and step, and one launch
    per run give the same bits."""
    q = gpu
    s1 = _train_pair(q, persistent=1)
    for form in (0, 2):
        s0 = _train_pair(q, persistent=form)
        for a, b in zip(s1, s0):
            for k in a:
                assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), (form, k)


def test_plain_forms_use_each_runs_own_cluster(gpu):
    """Automatic cluster sizes: the two one-run-at-a-time forms give each run its
    single-run size (2 CTAs for batch 32, 4 for batch 64) and agree bit for bit; split
    into several calls they continue where they stopped (the learners keep their
    workspaces and host-side counters between calls)."""
    q = gpu
    s0 = _train_pair(q, persistent=0, cluster=0)
    s2 = _train_pair(q, persistent=2, cluster=0)
    for a, b in zip(s0, s2):
        for k in a:
            assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k
    # 25 steps as 10 + 1 + 14 in the per-run form
    runs, envs = [], []
    for r in range(3):
        d, cfg, veh = lib_config(q, "c1", n_envs=2 + r, capacity=40, learning_starts=6,
                                 episode_len=15, seed=r, run_id=r)
        h = q.qsim_create(cfg, veh)
        hp = dict(W.TD3)
        hp.update(hidden=[32, 64, 16][r % 3], batch=[32, 64, 32][r % 3])
        runs.append(q.ac_create(q.make_ac_config(hp, cluster=0), h))
        envs.append(h)
    for steps in (10, 1, 14):
        q.ac_train(runs, envs, steps, persistent=2)
    torch.cuda.synchronize()
    for r, (a, h) in enumerate(zip(runs, envs)):
        ai, info = q.ac_info_get(a), q.qsim_info_get(h)
        # updates start once t_now >= max(learning_starts, n_hist + 2) = 18
        assert ai["updates"] == 25 - 18 + 1 and info["t_now"] == 25
        for k in NETS:
            assert np.array_equal(cpu(ai[k]).view(np.uint8), s2[r][k].view(np.uint8)), k
        for k in ("state", "records"):
            assert np.array_equal(cpu(info[k]).view(np.uint8), s2[r][k].view(np.uint8)), k
        q.ac_destroy(a)
        q.qsim_destroy(h)


@pytest.mark.parametrize("cluster,cap,steps", [(4, 64, 40), (2, 24, 60), (1, 200, 30)])
def test_replay_indices_bit_exact(gpu, cluster, cap, steps):
    """The sampled flat replay indices of every update equal the oracle sampler's bit for
    bit (Philox tag 4 words scaled by the number of valid transitions), before and after
    the ring wraps, on several CTAs of a cluster."""
    q = gpu
    d, h, a, hp = make_run(q, hidden=32, batch=128, cluster=cluster, cap=cap, steps=steps)
    try:
        idx = torch.zeros(128, dtype=torch.int32, device="cuda")
        q.ac_set_index_log(a, idx)
        for call in range(3):
            info = q.qsim_info_get(h)
            buf = oracle_buffer(info, info["n_envs"])
            L = oracle_learner(q.ac_info_get(a))
            q.ac_update(a, h, 1)
            torch.cuda.synchronize()
            dg = O.td3_update(d, hp, L, buf)
            got = cpu(idx).view(np.uint32)
            assert np.array_equal(got, dg["idx"]), (call, got[:8], dg["idx"][:8])
            # one more env step between updates moves the window
            acts = torch.tensor(W.random_actions(70 + call, (4, info["ld"])),
                                dtype=torch.float32, device="cuda")
            q.qsim_step(h, acts)
        q.ac_set_index_log(a, None)
    finally:
        q.ac_destroy(a)
        q.qsim_destroy(h)


def test_curriculum_inside_training(gpu):
    q = gpu
    cur = dict(W.CURRICULUM)
    cur["interval"] = 30  # env interactions
    d, cfg, veh = lib_config(q, "c1", n_envs=3, capacity=64, learning_starts=4, curriculum=cur)
    h = q.qsim_create(cfg, veh)
    hp = dict(W.TD3)
    hp.update(hidden=16, batch=32)
    a = q.ac_create(q.make_ac_config(hp), h)
    try:
        q.ac_train([a], [h], 25, persistent=1)  # 75 interactions -> 2 changes
        torch.cuda.synchronize()
        info = q.qsim_info_get(h)
        C = f64(info["reward_c"])
        Cref = np.array(W.REWARD)
        for _ in range(2):
            Cref = O.curriculum(cur["factor"], cur["target"], Cref)
        assert_close(C[:7], Cref, np.abs(Cref) + 1e-3, what="curriculum constants")
        sig = 0.1 * cur["sigma_factor"] ** 2
        assert abs(C[7] - max(sig, cur["sigma_min"])) < 1e-6
        # rewards were recalculated with the changed constants
        n = info["n_envs"]
        buf = oracle_buffer(info, n)
        r_gpu = buf["r"].copy()
        O.recalc_rewards(C[:7], buf, f64(info["state"])[:, :n].T)
        stored = info["size"]
        # every record written before the last change was recalculated; later ones were
        # written with the same constants
        assert_close(r_gpu[:stored], buf["r"][:stored], 1.0, what="recalculated rewards")
    finally:
        q.ac_destroy(a)
        q.qsim_destroy(h)


def test_checkpoint_resume_is_bitwise(gpu):
    q = gpu

    def setup():
        d, cfg, veh = lib_config(q, "c1", n_envs=4, capacity=50, learning_starts=5, episode_len=20)
        h = q.qsim_create(cfg, veh)
        hp = dict(W.TD3)
        hp.update(hidden=32, batch=32)
        return h, q.ac_create(q.make_ac_config(hp), h)

    h1, a1 = setup()
    q.ac_train([a1], [h1], 30, persistent=1)
    h2, a2 = setup()
    q.ac_train([a2], [h2], 15, persistent=1)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "ck.bin")
        q.ac_save(a2, h2, path)
        h3, a3 = setup()
        # the replay buffer is not part of the checkpoint: copy it device-to-device
        i2, i3 = q.qsim_info_get(h2), q.qsim_info_get(h3)
        i3["records"].copy_(i2["records"])
        i3["side"].copy_(i2["side"])
        q.ac_load(a3, h3, path)
        q.ac_train([a3], [h3], 15, persistent=1)
        torch.cuda.synchronize()
        A1, A3 = q.ac_info_get(a1), q.ac_info_get(a3)
        for k in NETS:
            assert np.array_equal(cpu(A1[k]).view(np.uint32), cpu(A3[k]).view(np.uint32)), k
        I1, I3 = q.qsim_info_get(h1), q.qsim_info_get(h3)
        assert np.array_equal(cpu(I1["state"]).view(np.uint32), cpu(I3["state"]).view(np.uint32))
        with open(path, "r+b") as f:
            f.write(b"XXXX")
        with pytest.raises(q.QsimError):
            q.ac_load(a3, h3, path)
    for a, h in ((a1, h1), (a2, h2), (a3, h3)):
        q.ac_destroy(a)
        q.qsim_destroy(h)


def test_update_rejects_empty_buffer(gpu):
    q = gpu
    d, cfg, veh = lib_config(q, "c1", n_envs=2, capacity=10)
    h = q.qsim_create(cfg, veh)
    hp = dict(W.TD3)
    hp.update(hidden=16, batch=32)
    a = q.ac_create(q.make_ac_config(hp), h)
    try:
        with pytest.raises(q.QsimError):
            q.ac_update(a, h, 1)
    finally:
        q.ac_destroy(a)
        q.qsim_destroy(h)


def test_graph_plan_equals_persistent_training(gpu):
    """A captured plan replayed in chunks gives bitwise the single persistent launch."""
    q = gpu

    def make():
        runs, envs = [], []
        for r in range(4):
            d, cfg, veh = lib_config(q, "c1", n_envs=3, capacity=40, learning_starts=5,
                                     episode_len=15, seed=10 + r, run_id=r)
            h = q.qsim_create(cfg, veh)
            hp = dict(W.TD3)
            hp.update(hidden=[32, 16][r % 2], batch=32)
            runs.append(q.ac_create(q.make_ac_config(hp, cluster=1), h))
            envs.append(h)
        return runs, envs

    r1, e1 = make()
    q.ac_train(r1, e1, 24, persistent=1)
    r2, e2 = make()
    plan = q.ac_plan_create(r2, e2, 8)
    q.ac_plan_run(plan, 3)
    q.ac_plan_sync(plan)
    torch.cuda.synchronize()
    try:
        for a, b, ha, hb in zip(r1, r2, e1, e2):
            A, B = q.ac_info_get(a), q.ac_info_get(b)
            assert A["updates"] == B["updates"] and A["t_actor"] == B["t_actor"]
            for k in NETS:
                assert np.array_equal(cpu(A[k]).view(np.uint32), cpu(B[k]).view(np.uint32)), k
            IA, IB = q.qsim_info_get(ha), q.qsim_info_get(hb)
            assert IA["t_now"] == IB["t_now"] == 24 and IA["head"] == IB["head"]
            for k in ("state", "records"):
                assert np.array_equal(cpu(IA[k]).view(np.uint32), cpu(IB[k]).view(np.uint32)), k
    finally:
        q.ac_plan_destroy(plan)
        for a, h in zip(r1 + r2, e1 + e2):
            q.ac_destroy(a)
            q.qsim_destroy(h)


def test_ablation_study_runs_in_one_persistent_launch(gpu):
    """The ablation study's ten variants (different critic layouts, history lengths, motor
    models, noise, disturbances, curricula) as runs of one persistent training launch give
    bit for bit what each run gives when launched on its own."""
    q = gpu

    def make(r, name):
        c, cur, recalc = W.ablation(name)
        c.update(seed=r, run_id=r, learning_starts=8)
        cur = dict(cur, interval=12)
        cfg = q.make_config(c, 1, 40, reward=W.REWARD, sigma_e=0.1, curriculum=cur,
                            recalc_rewards=recalc)
        h = q.qsim_create(cfg, q.make_params(c))
        hp = dict(W.TD3)
        hp.update(hidden=32, batch=32)
        return q.ac_create(q.make_ac_config(hp, cluster=1), h), h

    def snap(a, h):
        return (cpu(q.ac_info_get(a)["c1"]).copy(), cpu(q.ac_info_get(a)["actor"]).copy(),
                cpu(q.qsim_info_get(h)["records"]).copy())

    names = list(W.ABLATIONS)
    pairs = [make(r, name) for r, name in enumerate(names)]
    q.ac_train([a for a, _ in pairs], [h for _, h in pairs], 30, persistent=1)
    torch.cuda.synchronize()
    together = [snap(a, h) for a, h in pairs]
    for a, h in pairs:
        q.ac_destroy(a)
        q.qsim_destroy(h)
    for r, name in enumerate(names):
        a, h = make(r, name)
        q.ac_train([a], [h], 30, persistent=1)
        torch.cuda.synchronize()
        alone = snap(a, h)
        for x, y in zip(alone, together[r]):
            assert np.array_equal(x, y), name
        q.ac_destroy(a)
        q.qsim_destroy(h)


def test_train_autotune_picks_an_admissible_cluster(gpu):
    """The batched-launch autotuner times the admissible cluster sizes on the runs themselves
    (batch 64: 1, 2 and 4 CTAs per run), keeps the fastest, and the runs advance by the trial
    steps (one untimed call plus one per candidate); training then goes on at that size."""
    q = gpu
    runs, envs = [], []
    for r in range(3):
        d, cfg, veh = lib_config(q, "c1", n_envs=2, capacity=64, learning_starts=4,
                                 episode_len=15, seed=r, run_id=r)
        h = q.qsim_create(cfg, veh)
        hp = dict(W.TD3)
        hp.update(hidden=[32, 64, 32][r], batch=64)
        runs.append(q.ac_create(q.make_ac_config(hp, cluster=0), h))
        envs.append(h)
    try:
        q.ac_train(runs, envs, 10, persistent=1)
        torch.cuda.synchronize()
        t0 = [q.qsim_info_get(h)["t_now"] for h in envs]
        S = q.ac_train_autotune(runs, envs, 3)
        assert S in (1, 2, 4)
        assert [q.qsim_info_get(h)["t_now"] for h in envs] == [t + 3 * 4 for t in t0]
        q.ac_train(runs, envs, 5, persistent=1)
        torch.cuda.synchronize()
        for a in runs:
            ai = q.ac_info_get(a)
            assert all(bool(torch.isfinite(ai[k]).all()) for k in NETS)
        with pytest.raises(q.QsimError):
            q.ac_train_autotune(runs, envs, 0)
    finally:
        for a, h in zip(runs, envs):
            q.ac_destroy(a)
            q.qsim_destroy(h)
