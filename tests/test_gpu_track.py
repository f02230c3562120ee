"""Simulated trajectory tracking (Sec. V) on the GPU against the FP64 oracle: per env the
completed-step count (exact, unless the oracle's flight ends within FP32 reach of the
termination box) and the accumulated squared errors."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from helpers import cpu, f64, lib_config

pytestmark = pytest.mark.gpu

PERIODS = (3.5, 5.5, 15.0, 1000.0)


def hover_actor(d, hidden, seed=3, gain=0.05):
    """Random actor whose output sits near the hover action (float32 values)."""
    dd = dict(d)
    dd["seed"] = seed
    da = O.actor_in(d)
    P = O.init_params(dd, 0, da, hidden, 4)
    w3 = hidden * da + hidden + hidden * hidden + hidden
    P[w3:w3 + 4 * hidden] *= gain
    P[w3 + 4 * hidden:] = math.atanh(W.hover_action())
    return P.astype(np.float32)


def fly(q, n, hidden, steps, periods=PERIODS, sample=None, clip_p=0.2, clip_v=1.0, amp=1.0,
        z0=0.0, engine=None, **over):
    """engine None: the library's choice (tensor cores at hidden 64); 1: the SIMT kernel."""
    kw = dict(dist_f=0.004, dist_tau=2e-6)
    kw.update(over)
    d, cfg, veh = lib_config(q, "c2", n_envs=n, **kw)
    h = q.qsim_create(cfg, veh)
    try:
        if engine is not None:
            assert q.qsim_rollout_engine(h, engine) == engine
        info = q.qsim_info_get(h)
        ld = info["ld"]
        per = np.array([periods[i % len(periods)] for i in range(ld)], np.float32)
        actor = hover_actor(d, hidden)
        A = torch.tensor(actor, device="cuda")
        P = torch.tensor(per, device="cuda")
        sq = torch.full((2, ld), -1.0, dtype=torch.float64, device="cuda")
        ok = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
        state_before = cpu(info["state"]).copy()
        q.qsim_track(h, A, hidden, steps, P, sq, ok, amplitude=amp, z0=z0, clip_p=clip_p,
                     clip_v=clip_v)
        q.qsim_sync(h)
        torch.cuda.synchronize()
        info = q.qsim_info_get(h)
        assert np.array_equal(cpu(info["state"]), state_before)  # the env set is untouched
        ids = np.arange(n) if sample is None else np.asarray(sample)
        prm = f64(info["params"])[:, ids].T.copy()
        dist = f64(info["dist"])[:, ids].T.copy()
        ref = O.track(d, prm, dist, per[ids].astype(np.float64), actor.astype(np.float64), hidden,
                      steps, amp=amp, z0=z0, clip_p=clip_p, clip_v=clip_v, traj=True, n_threads=8)
        return d, cpu(sq)[:, ids].T, cpu(ok)[ids], ref, per[ids]
    finally:
        q.qsim_destroy(h)


def compare(d, sq, ok, ref, periods, steps, what, amp=1.0, z0=0.0):
    """steps_ok equal, except where the oracle's state at the step at which the earlier of
    the two flights ended lies within 1 mm of the termination box (FP32 trajectories differ
    from FP64 ones by ~1e-5 m over these flights); squared errors within 2e-3 relative."""
    rok = ref["steps_ok"]
    same = ok == rok
    for k in np.nonzero(~same)[0]:
        j = int(min(ok[k], rok[k])) + 1
        assert j <= steps, (what, k, ok[k], rok[k])
        p = ref["traj"][k, j, :3]
        pt, _ = O.lissajous(j * d["dt"], float(periods[k]), amp, z0)
        margin = np.max(np.abs(p - pt)) - d["term_pos"]
        assert np.isfinite(margin) and abs(margin) < 1e-3, \
            f"{what}: env {k} steps_ok gpu={ok[k]} ref={rok[k]} (box margin {margin:.2e} m)"
    assert (~same).mean() <= 0.02, (what, int((~same).sum()))
    n = np.maximum(rok, 1)[:, None]
    err = np.abs(sq - ref["sq_err"])[same]
    lim = (2e-3 * np.abs(ref["sq_err"]) + 1e-4 * 0.04 * n)[same]
    bad = err > lim
    assert not bad.any(), (what, np.argwhere(bad)[:3], sq[same][bad][:3], ref["sq_err"][same][bad][:3])


@pytest.mark.parametrize("hidden,n,engine", [(64, 300, None), (64, 300, 1), (64, 1000, None),
                                             (32, 97, None), (128, 130, None)])
def test_track_parity(gpu, hidden, n, engine):
    """Ragged env counts (partial warps, blocks and 128-env tiles), every actor width, both
    engines at hidden 64 (tensor cores by default, the SIMT kernel when pinned), four cycle
    times (agile 3.5 s to a slowly moving 1000 s target), disturbances on."""
    steps = 300
    d, sq, ok, ref, per = fly(gpu, n, hidden, steps, engine=engine)
    compare(d, sq, ok, ref, per, steps, f"track h{hidden} n{n}")
    assert ok.max() >= 100  # some flights last long enough to exercise the history ring
    assert (ok < steps).any()  # and some end


@pytest.mark.parametrize("engine", [None, 1])
def test_track_parity_without_history_and_with_binding_clips(gpu, engine):
    """18-input actor; tight clips that bind on most steps."""
    steps = 200
    d, sq, ok, ref, per = fly(gpu, 130, 64, steps, n_hist=0, clip_p=0.02, clip_v=0.05,
                              engine=engine)
    compare(d, sq, ok, ref, per, steps, "track nh0 clips")


@pytest.mark.parametrize("engine", [None, 1])
def test_track_invalid_periods_and_empty_flight(gpu, engine):
    """Periods <= 0, infinite or NaN fly no step; n_steps = 0 writes zeros."""
    d, sq, ok, ref, _ = fly(gpu, 40, 64, 50, periods=(0.0, -2.0, float("inf"), float("nan"), 5.5),
                            engine=engine)
    assert np.array_equal(ok, ref["steps_ok"])
    dead = np.arange(40) % 5 != 4
    assert np.all(ok[dead] == 0) and np.all(sq[dead] == 0.0)
    d, sq, ok, ref, _ = fly(gpu, 40, 64, 0, engine=engine)
    assert np.all(ok == 0) and np.all(sq == 0.0)


def test_track_argument_errors(gpu):
    q = gpu
    d, cfg, veh = lib_config(q, "c2", n_envs=32)
    h = q.qsim_create(cfg, veh)
    try:
        A = torch.zeros(20000, device="cuda")
        P = torch.ones(32, device="cuda")
        sq = torch.zeros((2, 32), dtype=torch.float64, device="cuda")
        ok = torch.zeros(32, dtype=torch.int32, device="cuda")
        for kw in (dict(hidden=48), dict(n_steps=-1), dict(clip_p=-1.0),
                   dict(amplitude=float("nan"))):
            args = dict(hidden=64, n_steps=10, clip_p=0.2, amplitude=1.0)
            args.update(kw)
            with pytest.raises(q.QsimError):
                q.qsim_track(h, A, args["hidden"], args["n_steps"], P, sq, ok,
                             amplitude=args["amplitude"], clip_p=args["clip_p"])
    finally:
        q.qsim_destroy(h)


def test_track_full_size_sampled(gpu):
    """The measured workload: 65,536 envs x 1,000 steps (10 s of flight), cycle times 15,
    5.5 and 3.5 s; 48 envs spread over the set checked against the oracle."""
    n, steps = 65536, 1000
    sample = np.linspace(0, n - 1, 48).astype(int)
    d, sq, ok, ref, per = fly(gpu, n, 64, steps, periods=(15.0, 5.5, 3.5), sample=sample)
    compare(d, sq, ok, ref, per, steps, "track full")
