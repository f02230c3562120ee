"""GPU reverse-mode gradients through the RK4 rollout (qsim_rollout_vjp) against the FP64
oracle adjoint and central finite differences of the oracle forward.

Tolerance (the differentiation workload's stated bar): relative error <= 1e-3, norm-wise
per gradient tensor, and element-wise |g - g_ref| <= 1e-3 |g_ref| + 1e-3 rms(g_ref).
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from helpers import f64

pytestmark = pytest.mark.gpu

TOL = 1e-3


def close(g, r, what):
    g, r = np.asarray(g, np.float64), np.asarray(r, np.float64)
    rms = np.sqrt(np.mean(r * r)) + 1e-30
    assert np.linalg.norm(g - r) <= TOL * np.linalg.norm(r) + 1e-30, \
        f"{what}: norm rel err {np.linalg.norm(g - r) / np.linalg.norm(r):.2e}"
    bad = np.abs(g - r) > TOL * np.abs(r) + TOL * rms
    assert not bad.any(), f"{what}: {bad.sum()} elements off, e.g. {g[bad][:3]} vs {r[bad][:3]}"


def setup(n, H, mode, seed=0, n_hist=16, hidden=64, ckpt=7, lanes=0):
    q = __import__("paper_2311_13081_gb300")
    from paper_2311_13081_gb300 import diff
    d = W.config("c1")
    veh = q.make_params(d)
    ld = q.padded(n)
    s0 = np.zeros((17, ld), np.float32)
    s0[:, :n] = W.random_states(seed, n, p=0.1, v=0.5, w=0.5, rpm=(12000.0, 17000.0)).T
    prm = np.zeros((8, ld), np.float32)
    prm[:, :n] = W.random_params(seed + 1, n).T
    prm[:, n:] = prm[:, :1]
    wts = (1.0, 0.5, 0.2, 0.05)
    desc = diff.make_desc(n, ld, H, ckpt, mode, wts, n_hist=n_hist, hidden=hidden,
                          lanes_per_env=lanes)
    S0, PR = torch.tensor(s0, device="cuda"), torch.tensor(prm, device="cuda")
    return q, diff, d, veh, ld, S0, PR, desc, wts


@pytest.mark.parametrize("n,H,ckpt", [(37, 30, 7), (64, 20, 20), (5, 9, 1)])
def test_open_loop_vjp_matches_oracle(gpu, n, H, ckpt):
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 0, seed=n, ckpt=ckpt)
    acts = np.zeros((H, 4, ld), np.float32)
    acts[:, :, :n] = W.random_actions(n + 5, (H, 4, n), -0.3, 0.5)
    A = torch.tensor(acts, device="cuda")
    loss = torch.zeros(ld, device="cuda")
    ga = torch.zeros_like(A)
    gp = torch.zeros(4, ld, device="cuda")
    ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
    q.qsim_rollout_vjp(desc, veh, S0, PR, A, None, None, loss, ga, None, gp, None, ws)
    torch.cuda.synchronize()
    ref = O.diff_run(d, f64(S0)[:, :n].T, f64(PR)[:, :n].T, H, wts, mode=0,
                     actions=f64(A)[:, :, :n].transpose(2, 0, 1))
    close(f64(loss)[:n], ref["loss"], "loss")
    close(f64(ga)[:, :, :n].transpose(2, 0, 1), ref["g_actions"], "g_actions")
    close(f64(gp)[:, :n].T, ref["g_prm"][:, :4], "g_params")


def test_closed_loop_vjp_matches_oracle(gpu):
    n, H, nh, hid = 40, 25, 4, 16
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 1, seed=3, n_hist=nh, hidden=hid, ckpt=6)
    dd = dict(d, n_hist=nh)
    actor = O.init_params(dd, 0, 18 + 4 * nh, hid, 4).astype(np.float32)
    AW = torch.tensor(actor, device="cuda")
    loss = torch.zeros(ld, device="cuda")
    gw = torch.zeros_like(AW)
    gp = torch.zeros(4, ld, device="cuda")
    aout = torch.zeros(H, 4, ld, device="cuda")
    ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
    q.qsim_rollout_vjp(desc, veh, S0, PR, None, AW, None, loss, None, gw, gp, aout, ws)
    torch.cuda.synchronize()
    ref = O.diff_run(d, f64(S0)[:, :n].T, f64(PR)[:, :n].T, H, wts, mode=1,
                     actor=actor.astype(np.float64), hidden=hid, n_hist=nh)
    close(f64(loss)[:n], ref["loss"], "loss")
    close(f64(aout)[:, :, :n].transpose(2, 0, 1), ref["act_out"], "actions")
    close(f64(gw), ref["g_actor"], "g_actor")
    close(f64(gp)[:, :n].T, ref["g_prm"][:, :4], "g_params")


@pytest.mark.parametrize("hid,lanes,n", [(64, 32, 45), (64, 16, 45), (64, 8, 45), (32, 16, 45),
                                         (32, 8, 45), (64, 8, 2601), (32, 8, 2601)])
def test_closed_loop_lane_groups_match_oracle(gpu, hid, lanes, n):
    """The lane-group kernels (hidden 32 / 64, 16 actions of history): one env per 32, 16 or
    8 lanes.  45 envs leave the last warp's groups partly without an env (they run on a
    valid index and store nothing).  2,601 envs at 8 lanes take the 7-warp CTAs (one per
    SM; 93 CTAs, the last one ragged) instead of the 4-warp ones."""
    H, nh = 23, 16
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 1, seed=5, n_hist=nh, hidden=hid,
                                                   ckpt=6, lanes=lanes)
    actor = O.init_params(d, 0, 18 + 4 * nh, hid, 4).astype(np.float32)
    AW = torch.tensor(actor, device="cuda")
    loss = torch.zeros(ld, device="cuda")
    gw = torch.zeros_like(AW)
    gp = torch.zeros(4, ld, device="cuda")
    aout = torch.zeros(H, 4, ld, device="cuda")
    ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
    q.qsim_rollout_vjp(desc, veh, S0, PR, None, AW, None, loss, None, gw, gp, aout, ws)
    torch.cuda.synchronize()
    ref = O.diff_run(d, f64(S0)[:, :n].T, f64(PR)[:, :n].T, H, wts, mode=1,
                     actor=actor.astype(np.float64), hidden=hid, n_hist=nh)
    close(f64(loss)[:n], ref["loss"], "loss")
    close(f64(aout)[:, :, :n].transpose(2, 0, 1), ref["act_out"], "actions")
    close(f64(gw), ref["g_actor"], "g_actor")
    close(f64(gp)[:, :n].T, ref["g_prm"][:, :4], "g_params")


def test_vjp_rejects_bad_lane_groups(gpu):
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(8, 5, 1, lanes=12)
    assert q.qsim_vjp_workspace(desc) == 0


def test_vjp_matches_finite_differences_of_oracle_forward(gpu):
    """GPU adjoint vs central differences (h = 1e-4, FP64) of the oracle's forward."""
    n, H = 3, 15
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 0, seed=9, ckpt=4)
    acts = np.zeros((H, 4, ld), np.float32)
    acts[:, :, :n] = W.random_actions(19, (H, 4, n), -0.2, 0.4)
    A = torch.tensor(acts, device="cuda")
    loss = torch.zeros(ld, device="cuda")
    ga = torch.zeros_like(A)
    gp = torch.zeros(4, ld, device="cuda")
    ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
    q.qsim_rollout_vjp(desc, veh, S0, PR, A, None, None, loss, ga, None, gp, None, ws)
    torch.cuda.synchronize()
    s0, prm = f64(S0)[:, :n].T, f64(PR)[:, :n].T
    a64 = f64(A)[:, :, :n].transpose(2, 0, 1).copy()
    g = f64(ga)[:, :, :n].transpose(2, 0, 1)
    rng = W.rng(4)
    for _ in range(10):
        e, t, c = rng.integers(n), rng.integers(H), rng.integers(4)
        ap, am = a64.copy(), a64.copy()
        ap[e, t, c] += 1e-4
        am[e, t, c] -= 1e-4
        fd = (O.diff_run(d, s0, prm, H, wts, mode=0, actions=ap)["loss"][e]
              - O.diff_run(d, s0, prm, H, wts, mode=0, actions=am)["loss"][e]) / 2e-4
        assert abs(g[e, t, c] - fd) <= TOL * abs(fd) + 1e-6, (e, t, c, g[e, t, c], fd)
    gpar = f64(gp)[:, :n].T
    for e in range(n):
        for j in range(4):
            pp, pm = prm.copy(), prm.copy()
            h = 1e-4 * prm[e, j]
            pp[e, j] += h
            pm[e, j] -= h
            fd = (O.diff_run(d, s0, pp, H, wts, mode=0, actions=a64)["loss"][e]
                  - O.diff_run(d, s0, pm, H, wts, mode=0, actions=a64)["loss"][e]) / (2 * h)
            assert abs(gpar[e, j] - fd) <= TOL * abs(fd) + 1e-9 * abs(fd / prm[e, j]), (e, j, gpar[e, j], fd)


def test_checkpoint_interval_does_not_change_results(gpu):
    n, H = 50, 24
    outs = []
    for ckpt in (1, 5, 24):
        q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 1, seed=2, n_hist=16, hidden=32, ckpt=ckpt)
        actor = O.init_params(d, 0, 82, 32, 4).astype(np.float32)
        AW = torch.tensor(actor, device="cuda")
        loss = torch.zeros(ld, device="cuda")
        gw = torch.zeros_like(AW)
        gp = torch.zeros(4, ld, device="cuda")
        ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
        q.qsim_rollout_vjp(desc, veh, S0, PR, None, AW, None, loss, None, gw, gp, None, ws)
        torch.cuda.synchronize()
        outs.append((f64(loss), f64(gw), f64(gp)))
    for o in outs[1:]:
        # recomputed states are bit-identical, so loss and parameter gradients are too;
        # the actor gradient is summed per segment, so its FP32 sums regroup
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[2], outs[0][2])
        assert np.linalg.norm(o[1] - outs[0][1]) <= 1e-5 * np.linalg.norm(outs[0][1])


def test_autograd_function_routes_upstream_gradient(gpu):
    n, H = 33, 12
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 0, seed=5, ckpt=5)
    acts = torch.tensor(W.random_actions(8, (H, 4, ld), -0.3, 0.3), dtype=torch.float32,
                        device="cuda", requires_grad=True)
    prm = PR.clone().requires_grad_(True)
    w = torch.linspace(0.5, 2.0, n, device="cuda")
    L = diff.RolloutLoss.apply(prm, acts, S0, veh, desc)
    (L * w).sum().backward()
    # reference: the library call with the same seed
    seed = torch.zeros(ld, device="cuda")
    seed[:n] = w
    loss = torch.zeros(ld, device="cuda")
    ga = torch.zeros(H, 4, ld, device="cuda")
    gp = torch.zeros(4, ld, device="cuda")
    ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
    q.qsim_rollout_vjp(desc, veh, S0, PR, acts.detach(), None, seed, loss, ga, None, gp, None, ws)
    torch.cuda.synchronize()
    assert torch.equal(acts.grad, ga)
    assert torch.equal(prm.grad[0:4], gp) and torch.all(prm.grad[4:] == 0)


def test_c3_full_size_sampled(gpu):
    """4,096 envs, 200 steps, checkpoint every 20, closed loop with the 82-64-64-4 actor;
    loss and parameter gradients of 6 sampled envs against the oracle, actor gradient
    checked on a 6-env rollout."""
    n, H = 4096, 200
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 1, seed=11, n_hist=16, hidden=64, ckpt=20)
    actor = O.init_params(d, 0, 82, 64, 4).astype(np.float32)
    AW = torch.tensor(actor, device="cuda")
    loss = torch.zeros(ld, device="cuda")
    gw = torch.zeros_like(AW)
    gp = torch.zeros(4, ld, device="cuda")
    ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
    q.qsim_rollout_vjp(desc, veh, S0, PR, None, AW, None, loss, None, gw, gp, None, ws)
    torch.cuda.synchronize()
    assert torch.isfinite(gw).all()
    ids = np.array([0, 1, 777, 2048, 3000, 4095])
    ref = O.diff_run(d, f64(S0)[:, ids].T, f64(PR)[:, ids].T, H, wts, mode=1,
                     actor=actor.astype(np.float64), hidden=64, n_hist=16)
    close(f64(loss)[ids], ref["loss"], "loss")
    close(f64(gp)[:, ids].T, ref["g_prm"][:, :4], "g_params")
    # actor gradient of exactly these 6 envs through the same launch configuration
    seed = torch.zeros(ld, device="cuda")
    seed[torch.tensor(ids, device="cuda")] = 1.0
    q.qsim_rollout_vjp(desc, veh, S0, PR, None, AW, seed, loss, None, gw, gp, None, ws)
    torch.cuda.synchronize()
    close(f64(gw), ref["g_actor"], "g_actor (6 envs)")


def test_closed_loop_gradient_is_reproducible_and_captures_in_a_graph(gpu):
    """The closed loop's weight gradient of each segment runs on a side stream while the
    next segment's reverse sweep runs, with two record buffers in turn.  Over 5 segments
    (both buffers reused) repeated calls, a call on another stream and a replay of the
    call captured in a CUDA graph give bitwise the same results."""
    n, H = 300, 50
    q, diff, d, veh, ld, S0, PR, desc, wts = setup(n, H, 1, seed=4, n_hist=16, hidden=64,
                                                   ckpt=10, lanes=8)
    actor = O.init_params(d, 0, 82, 64, 4).astype(np.float32)
    AW = torch.tensor(actor, device="cuda")
    loss = torch.zeros(ld, device="cuda")
    gw = torch.zeros_like(AW)
    gp = torch.zeros(4, ld, device="cuda")
    ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
    args = (desc, veh, S0, PR, None, AW, None, loss, None, gw, gp, None, ws)
    q.qsim_rollout_vjp(*args)
    torch.cuda.synchronize()
    ref = (loss.clone(), gw.clone(), gp.clone())
    assert torch.isfinite(ref[1]).all() and ref[1].abs().sum() > 0
    for t in (loss, gw, gp):
        t.zero_()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        q.qsim_rollout_vjp(*args)
    torch.cuda.synchronize()
    assert torch.equal(loss, ref[0]) and torch.equal(gw, ref[1]) and torch.equal(gp, ref[2])
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        q.qsim_rollout_vjp(*args)
    for t in (loss, gw, gp):
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(loss, ref[0]) and torch.equal(gw, ref[1]) and torch.equal(gp, ref[2])
