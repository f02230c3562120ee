"""Failure detection on the GPU without a fault: bounded device-side waits that run out,
values outside the half-precision range of the tensor-core rollout, and non-finite
inputs.  Each failure is made by the host (a wait limit far below the MMA latency, an
actor scaled out of range, a NaN written into an input); the kernel records a status
that the host reads, the context stays usable and later calls run normally."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from helpers import STATE_SCALE, assert_close, compare_records, f64, gpu_records, lib_config, oracle_envs

pytestmark = pytest.mark.gpu

TC = 2
QSIM_ETIMEOUT, QSIM_ESTATE = -4, -5


def _env(q, n=1000, **over):
    kw = dict(capacity=8, learning_starts=0, episode_len=40)
    kw.update(over)
    d, cfg, veh = lib_config(q, "c2", n_envs=n, **kw)
    h = q.qsim_create(cfg, veh)
    assert q.qsim_rollout_engine(h, TC) == TC
    actor = O.init_params(d, 0, O.actor_in(d), 64, 4).astype(np.float32)
    return d, h, actor


def _one_step_parity(q, d, h, actor, n, what):
    A = torch.tensor(actor, device="cuda")
    info = q.qsim_info_get(h)
    ids = np.arange(0, n, 7)
    e = oracle_envs(info, ids)
    t0, head0 = info["t_now"], info["head"]
    q.qsim_rollout(h, A, 64, 1, 0.1)
    q.qsim_sync(h)
    ref = O.rollout(d, W.REWARD, e, 1, t0, actor=actor.astype(np.float64), hidden=64,
                    sigma_e=0.1, n_threads=8)
    info = q.qsim_info_get(h)
    compare_records(gpu_records(info, [head0 % info["capacity"]], ids), ref, what=what)


@pytest.mark.parametrize("sched", [(1, 0), (1, 2), (2, 0)])
def test_tc_wait_that_runs_out_is_reported_and_the_next_call_runs(gpu, sched):
    """A one-poll wait limit: the hand-over waits (and, with 2-step units, the waits for a
    group's previous chunk) give up before the MMAs complete; persistent schedule with one
    unit per group, with 2-step units, and two partitions without the unit counter.  qsim_sync reports
    QSIM_ETIMEOUT; with the default limit restored the next call matches the oracle, which
    also shows that the aborted blocks released their tensor memory (every block of the
    next launch allocates all of it)."""
    q = gpu
    n = 4000
    d, h, actor = _env(q, n)
    try:
        q.qsim_rollout_schedule(h, *sched)
        A = torch.tensor(actor, device="cuda")
        q.qsim_rollout(h, A, 64, 2, 0.1)
        q.qsim_sync(h)
        assert q.qsim_set_wait_limit(h, 1) == 1 << 22
        q.qsim_rollout(h, A, 64, 4, 0.1)
        with pytest.raises(q.QsimError) as ei:
            q.qsim_sync(h)
        assert ei.value.status == QSIM_ETIMEOUT
        q.qsim_sync(h)  # the status word was cleared
        assert q.qsim_set_wait_limit(h, 0) == 1
        for k in range(2):
            _one_step_parity(q, d, h, actor, n, f"after timeout {k}")
    finally:
        q.qsim_destroy(h)


@pytest.mark.parametrize("scale", [3e5, 1e6])
def test_tc_half_precision_overflow_is_reported(gpu, scale):
    """First-layer weights scaled by 3e5 (at most 3.3e4, still inside the fp16 range)
    drive the first hidden activations of a fresh env set to ~1.7e5, past it (the FP64
    oracle's largest is 5.7e4 at 1e5, 1.7e5 at 3e5); scaled by 1e6 the weights themselves
    leave it.  Either way the
    kernel reports QSIM_ESTATE rather than rounding silently; an ordinary actor afterwards
    runs and matches the oracle."""
    q = gpu
    n = 600
    d, h, actor = _env(q, n)
    try:
        big = actor.copy()
        H, DA = 64, O.actor_in(d)
        big[:H * DA] *= scale
        q.qsim_rollout(h, torch.tensor(big, device="cuda"), 64, 1, 0.1)
        with pytest.raises(q.QsimError) as ei:
            q.qsim_sync(h)
        assert ei.value.status == QSIM_ESTATE and "half-precision" in str(ei.value)
        # the out-of-range step may have sent states anywhere: start the envs afresh
        q.qsim_destroy(h)
        d, h, actor = _env(q, n)
        _one_step_parity(q, d, h, actor, n, "after overflow")
    finally:
        q.qsim_destroy(h)


def test_dynamics_with_nan_input_is_contained(gpu):
    """A NaN written into one body's state: that body's result is NaN, every other body
    matches the oracle, nothing traps, and the next call runs normally."""
    q = gpu
    n = 256
    d = W.config("c1")
    veh = q.make_params(d)
    ld = q.padded(n)
    s = W.random_states(3, n)
    prm = W.random_params(4, n)
    u = W.random_actions(5, (n, 4), 0.0, 21702.0)
    s[17, 8] = np.nan
    S = torch.zeros(17, ld, dtype=torch.float32)
    S[:, :n] = torch.tensor(s.T, dtype=torch.float32)
    Pm = torch.zeros(8, ld, dtype=torch.float32)
    Pm[:, :n] = torch.tensor(prm.T, dtype=torch.float32)
    U = torch.zeros(4, ld, dtype=torch.float32)
    U[:, :n] = torch.tensor(u.T, dtype=torch.float32)
    S, Pm, U = S.cuda(), Pm.cuda(), U.cuda()
    out = torch.empty_like(S)
    for call in range(2):
        q.qsim_dynamics_step(veh, Pm, None, S, U, 0.01, 1, n, ld, 3, out)
        torch.cuda.synchronize()
        g = f64(out)[:, :n].T
        ok = np.arange(n) != 17 if call == 0 else np.ones(n, bool)
        if call == 0:
            assert np.isnan(g[17]).any()
        ref = O.dynamics_batch(d, f64(S)[:, :n].T[ok], f64(U)[:, :n].T[ok], f64(Pm)[:, :n].T[ok],
                               None, dt=np.float64(np.float32(0.01)), renorm=1, n_steps=3)
        assert_close(g[ok], ref, STATE_SCALE, what=f"call {call}")
        # repaired input (level, at rest): the next call runs normally on every body
        S[:13, 17] = 0.0
        S[3, 17] = 1.0


def test_nan_state_in_rollout_terminates_that_env(gpu):
    """A NaN written into one env's velocity before a tensor-core rollout step: the NaN
    reaches an MMA operand, which the kernel reports (QSIM_ESTATE, like any value outside
    the half-precision range); the step's successor state is non-finite, so that env
    terminates (flag bit 0), receives reward 0 and starts a new episode; the other envs
    (their own rows of every MMA) are unaffected."""
    q = gpu
    n = 300
    d, h, actor = _env(q, n)
    try:
        A = torch.tensor(actor, device="cuda")
        q.qsim_rollout(h, A, 64, 2, 0.1)
        info = q.qsim_info_get(h)
        info["state"][7, 5] = float("nan")
        torch.cuda.synchronize()
        head0 = info["head"]
        ids = np.array([4, 6, 100])
        e = oracle_envs(info, ids)
        t0 = info["t_now"]
        q.qsim_rollout(h, A, 64, 1, 0.1)
        with pytest.raises(q.QsimError) as ei:
            q.qsim_sync(h)
        assert ei.value.status == QSIM_ESTATE
        info = q.qsim_info_get(h)
        rec = gpu_records(info, [head0], np.array([5]))
        assert int(rec["rec_flags"][0, 0]) & 1
        assert rec["rec_r"][0, 0] == 0.0
        assert int(info["ep_step"][5].item()) == 0
        assert np.isfinite(f64(info["state"])[:, 5]).all()
        ref = O.rollout(d, W.REWARD, e, 1, t0, actor=actor.astype(np.float64), hidden=64,
                        sigma_e=0.1, n_threads=4)
        compare_records(gpu_records(info, [head0], ids), ref, what="neighbours")
    finally:
        q.qsim_destroy(h)
