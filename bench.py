"""Benchmark of the quadrotor training hot path on GB300.

Default workload (one bench step): the fused env step of 65,536 domain-randomised
quadrotors for 1,000 steps each (actor MLP 82-64-64-4 with Gaussian exploration, RK4
dynamics with motor lag, reward, termination, reset) writing every transition into a
65,536 x 1,000 device replay ring -- 65.5 M env-steps per bench step.

Printed as ONE JSON line (rank 0).  Besides the headline env-steps/s it carries the
roofline of the dominant kernel (FP32 FMA bound), the end-to-end number through the C ABI
with host buffers, the FP64 oracle timed on this host's cores, and secondary measurements
of the other hot-path pieces: the learner (wall time to N actor-critic updates, batched
persistent launch vs the plain one-run-per-launch form), reward recalculation bandwidth,
the dynamics-only benchmark in the paper's shape, and reverse-mode gradients.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank simulates its own 65,536 envs (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("env-steps/s (sim+policy) and wall time to N actor-critic updates on 1 GB300, "
          "vs plain")
FLOP_ACTOR = lambda da, h: 2 * (da * h + h * h + 4 * h)  # noqa: E731
# tensor-core engine: the two hidden layers as fp16 MMAs on hi/lo halves, three products
# per FP32-accurate product (A_hi W_hi + A_hi W_lo + A_lo W_hi); fp16 and bf16 dense
# tensor rates are equal on this part, so the measured bf16 peak is the fp16 peak
FLOP_TC_MMA = lambda da, h: 3 * 2 * (da * h + h * h)  # noqa: E731
FLOP_DYN = 672        # RK4 (4 derivative evaluations + stage/accumulation arithmetic)
FLOP_MISC = 60        # observation rotation matrix, reward, termination, action map
BYTES_STEP = 92       # transition record written per env-step (17 s, 4 a, r, flags)
# DRAM bytes per env-step of k_rollout<64,*> measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum).  Set to None whenever the kernel changes until it is captured
# again: its side-ring stores changed since the last capture.
NCU_DRAM_BYTES_PER_ENV_STEP = None
# same for the tensor-core kernel k_rollout_tc: one-pass capture of a full-size timed launch,
# 65,536 envs x 1,000 steps (profiles/k_rollout_tc_c2_65536x1000.md)
NCU_DRAM_BYTES_PER_ENV_STEP_TC = (110.884864e6 + 6301.343488e6) / (65536 * 1000)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=65536)
    ap.add_argument("--horizon", type=int, default=1000)
    ap.add_argument("--no-extras", action="store_true", help="headline measurement only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--only-learner", type=int, default=0, metavar="RUNS",
                    help="only the batched-learner sample with RUNS runs (for profiling)")
    ap.add_argument("--learner-steps", type=int, default=1000)
    ap.add_argument("--only-recalc", type=int, default=0, metavar="SLOTS",
                    help="only reward recalculation over a filled ring of --envs x SLOTS records")
    ap.add_argument("--only-dynamics", type=int, default=0, metavar="STEPS",
                    help="only the dynamics-only kernel, 8,192 envs x STEPS steps (profiling)")
    ap.add_argument("--dyn-envs", type=int, default=8192, help="with --only-dynamics: envs")
    ap.add_argument("--only-c5", action="store_true",
                    help="only the c5 sample (full replay rings, recalculation), for profiling")
    ap.add_argument("--only-diff", action="store_true",
                    help="only the differentiation sample (c3 shape), for profiling")
    ap.add_argument("--only-c1", action="store_true",
                    help="only the single-run learner sample (1 env, batch 256), for profiling")
    ap.add_argument("--only-ablation", action="store_true",
                    help="only the ablation-study sample (ten variants in one launch)")
    ap.add_argument("--only-track", action="store_true",
                    help="only the Lissajous tracking sample, for profiling")
    ap.add_argument("--warps", type=int, default=0,
                    help="pin the rollout's warps per block and skip the autotuner (profiling)")
    ap.add_argument("--parts", type=int, default=1, help="with --warps: env partitions")
    ap.add_argument("--chunk", type=int, default=100, help="with --warps: steps per chunk")
    ap.add_argument("--packed", type=int, default=1, help="with --warps: paired-FMA variant")
    ap.add_argument("--engine", type=int, default=-1,
                    help="rollout engine: 0 SIMT, 1 SIMT paired FMA, 2 tensor cores, -1 autotuned")
    return ap.parse_args()


# ---------------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------- multi-GPU
def rank_workload(W, rank):
    """The c2 env set of one rank (weak scaling): every rank simulates its own 65,536 envs
    with its own random streams (run id = rank), so no data crosses ranks."""
    d = W.config("c2")
    d.update(learning_starts=0, seed=0, run_id=rank)
    return d


def max_over_ranks(torch, dist, x, world, device):
    """Largest of a per-rank time over all ranks -- the only collective of the bench."""
    if world <= 1:
        return float(x)
    tt = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def flush_l2(buf):
    buf.zero_()


def device_peaks(torch, q):
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        max_mhz = float(mp.get("sm_max_mhz", max_mhz))
        hbm = float(mp["hbm_gbs"])
        hbm_src = "measured"
        bf16_sus = float(mp["bf16_tflops_sustained"])
        tc_src = "measured"
    except Exception:
        hbm, hbm_src = 6800.0, "fallback"
        bf16_sus, tc_src = 1700.0, "fallback"
    fp32 = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    return sms, max_mhz, fp32, hbm, hbm_src, bf16_sus, tc_src


# -------------------------------------------------------------------------- measurements
def measure_ffma(torch, q):
    out = torch.zeros(4, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, iters = sms * 8, 4096
    q.qsim_ffma_probe(blocks, 64, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    q.qsim_ffma_probe(blocks, iters, out)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    flops = blocks * 256 * iters * 8 * 16 * 2
    e0.record()
    q.qsim_ffma_probe(blocks, -iters // 2, out)  # paired f32x2 FMAs, same FMA count
    e1.record()
    e1.synchronize()
    ms2 = e0.elapsed_time(e1)
    return {"ffma": flops / (ms * 1e-3) / 1e12, "ffma2": flops / (ms2 * 1e-3) / 1e12}


def measure_mma_rate(torch, q):
    """SM cycles per tcgen05.mma (kind::f16, M 128, K 16) in a chain of 64, by accumulator
    width N and by the number of warps issuing chains into disjoint columns."""
    cyc = torch.zeros(1, dtype=torch.int64, device="cuda")
    res = {}
    for n_cols, n_warps in ((64, 1), (128, 1), (256, 1), (64, 2), (128, 4)):
        q.qsim_mma_probe(64, n_cols, n_warps, cyc)  # warm-up
        q.qsim_mma_probe(64, n_cols, n_warps, cyc)
        torch.cuda.synchronize()
        c = int(cyc.item())
        res[f"N{n_cols // n_warps}_x{n_warps}warps"] = {
            "cycles": c, "cycles_per_mma": c / (64 * n_warps) if c > 0 else None}
    return res


def measure_dynamics(torch, q, veh):
    """Paper's simulator benchmark shape: 8,192 envs x 1e6 RK4 steps, no policy."""
    res = {}
    for n, steps, tag in ((8192, 1_000_000, "paper_shape_8192x1e6"),
                          (155_648, 50_000, "saturating_155648x5e4")):
        ld = (n + 31) // 32 * 32
        out = torch.empty(17, ld, device="cuda")
        q.qsim_dynamics_bench(veh, n, ld, 1000, 0.01, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        q.qsim_dynamics_bench(veh, n, ld, steps, 0.01, out)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        res[tag] = {"env_steps_per_s": n * steps / (ms * 1e-3), "ms": ms,
                    "tflops": n * steps * FLOP_DYN / (ms * 1e-3) / 1e12,
                    "finite": bool(torch.isfinite(out[:, :n]).all())}
    return res


def measure_track(torch, q, W, fp32_peak, n=65536, steps=1000, hidden=64):
    """Simulated Lissajous tracking (Sec. V): every env flies the deterministic actor for
    `steps` steps (10 s) along the figure-eight, cycle times 15, 5.5 and 3.5 s over the
    envs, domain-randomised vehicles.  The actor is random (PyTorch-style init) with its
    output layer scaled down around the hover action, so flights last a while; no trained
    weights exist here, so the errors say nothing about the paper's controller."""
    d = W.config("c2")
    cfg = q.make_config(d, n, 0, reward=W.REWARD, sigma_e=0.0)
    h = q.qsim_create(cfg, q.make_params(d))
    try:
        ld = q.qsim_info_get(h)["ld"]
        g = torch.Generator().manual_seed(11)
        da = 18 + 4 * d["n_hist"]
        parts = []
        for fan_in, shape in ((da, (hidden, da)), (da, (hidden,)), (hidden, (hidden, hidden)),
                              (hidden, (hidden,)), (hidden, (4, hidden))):
            b = fan_in ** -0.5
            parts.append((torch.rand(shape, generator=g) * 2 - 1).mul(b).flatten())
        parts[-1] *= 0.05
        parts.append(torch.full((4,), math.atanh(W.hover_action())))
        actor = torch.cat(parts).float().cuda()
        per = torch.tensor([(15.0, 5.5, 3.5)[i % 3] for i in range(ld)], device="cuda")
        sq = torch.empty((2, ld), dtype=torch.float64, device="cuda")
        ok = torch.empty(ld, dtype=torch.int32, device="cuda")
        # the SIMT kernel first (for comparison), then the default engine (tensor cores)
        times = {}
        for engine in (1, -1):
            q.qsim_rollout_engine(h, engine)
            q.qsim_track(h, actor, hidden, 100, per, sq, ok)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record()
            for _ in range(reps):
                q.qsim_track(h, actor, hidden, steps, per, sq, ok)
            e1.record()
            e1.synchronize()
            q.qsim_sync(h)
            times[engine] = e0.elapsed_time(e1) / reps
        ms = times[-1]
        okc = ok[:n].double().cpu()
        sqc = sq[:, :n].cpu()
        res = {"workload": f"{n} envs x {steps} steps, cycle times 15 / 5.5 / 3.5 s",
               "env_steps_per_s": n * steps / (ms * 1e-3), "ms": ms,
               "fp32_equivalent_tflops": n * steps * (FLOP_ACTOR(da, hidden) + FLOP_DYN + FLOP_MISC)
               / (ms * 1e-3) / 1e12, "fp32_peak": fp32_peak, "kernel": "k_rollout_tc<true>",
               "simt_kernel": {"kernel": "k_rollout<64, 4, 1, 1>", "ms": times[1],
                               "env_steps_per_s": n * steps / (times[1] * 1e-3),
                               "fp32_frac": n * steps * (FLOP_ACTOR(da, hidden) + FLOP_DYN + FLOP_MISC)
                               / (times[1] * 1e-3) / 1e12 / fp32_peak}}
        for j, T in enumerate((15.0, 5.5, 3.5)):
            sel = torch.arange(n) % 3 == j
            k = okc[sel]
            flown = k > 0
            rmse = torch.sqrt(sqc[0, sel][flown] / k[flown])
            res[f"T{T:g}"] = {"mean_steps_completed": float(k.mean()),
                              "flights_completed": float((k == steps).double().mean()),
                              "median_rmse_m": float(rmse.median()) if flown.any() else None}
        return res
    finally:
        q.qsim_destroy(h)


def measure_ablation(torch, q, W, seeds=5, steps=3000):
    """The ablation study's ten variants (Sec. VI) x `seeds` seeds as runs of ONE persistent
    training launch (1 env per run, width 64, batch 256, 1,000 warm-up steps, then one
    update per env step).  Reports the launch's throughput and, per variant, the mean
    length and return of the episodes completed so far: at a few thousand steps these are
    early-training numbers, not the paper's 300,000-step checkpoint."""
    names = list(W.ABLATIONS)
    runs, envs, tags = [], [], []
    for i, name in enumerate(names):
        for k in range(seeds):
            r = i * seeds + k
            c, cur, recalc = W.ablation(name)
            c.update(seed=k, run_id=r)
            cfg = q.make_config(c, 1, steps, reward=W.REWARD, sigma_e=0.1, curriculum=cur,
                                recalc_rewards=recalc)
            h = q.qsim_create(cfg, q.make_params(c))
            runs.append(q.ac_create(q.make_ac_config(dict(W.TD3), cluster=0), h))
            envs.append(h)
            tags.append(name)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.ac_train(runs, envs, steps, persistent=1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        updates = len(runs) * (steps - 1000)
        res = {"runs": len(runs), "steps_per_run": steps, "s": dt,
               "env_steps_per_s": len(runs) * steps / dt, "updates_per_s": updates / dt,
               "variants": {}}
        for name in names:
            st = [q.qsim_stats_get(h) for h, t in zip(envs, tags) if t == name]
            eps = sum(x["episodes"] for x in st)
            res["variants"][name] = {
                "episodes": eps,
                "mean_length": (sum(x["mean_length"] * x["episodes"] for x in st) / eps
                                if eps else None),
                "mean_return": (sum(x["mean_return"] * x["episodes"] for x in st) / eps
                                if eps else None)}
        return res
    finally:
        for a, h in zip(runs, envs):
            q.ac_destroy(a)
            q.qsim_destroy(h)


def measure_recalc(torch, q, h, n, horizon, hbm):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q.qsim_recalc_rewards(h)
    st.synchronize()
    reps = 3
    e0.record()
    for _ in range(reps):
        q.qsim_recalc_rewards(h)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    records = n * horizon
    byts = records * (17 * 4 + 4 * 4 + 4 + 4)  # read s', a, flags; write r
    return {"records": records, "ms": ms, "gbs": byts / (ms * 1e-3) / 1e9,
            "frac_of_measured_hbm": byts / (ms * 1e-3) / 1e9 / hbm, "bytes_per_record": 92}


def _c4_runs(q, W, n_runs, capacity, learning_starts):
    """The batched-training workload: n_runs independent runs, hidden width and minibatch
    drawn per run from Philox (tag 9, seed r) over {32,64,128} x {128,256,512}, 8 envs
    each, the domain-randomised vehicle; cluster size automatic (0)."""
    widths, batches = (32, 64, 128), (128, 256, 512)
    runs, envs, flop_per_step = [], [], 0.0
    for r in range(n_runs):
        x = q.qsim_philox_host([0, 0, 9 << 24, r], [r, 0])
        hid, B = widths[x[0] % 3], batches[x[1] % 3]
        d = W.config("c2")
        d.update(seed=r, run_id=r, learning_starts=learning_starts)
        cfg = q.make_config(d, 8, capacity, reward=W.REWARD, sigma_e=0.1)
        h = q.qsim_create(cfg, q.make_params(d))
        hp = dict(W.TD3)
        hp.update(hidden=hid, batch=B)
        runs.append(q.ac_create(q.make_ac_config(hp, cluster=0), h))
        envs.append(h)
        flop_per_step += 2 * B * update_macs(82, 90, hid)
    return runs, envs, flop_per_step


def update_macs(da, dc, h):
    """Multiply-adds per sample of one TD3 update (target actor, 2 target critics, 2 critics
    forward + backward (input and weight gradients), and every second update the actor
    phase: actor forward, critic 1 forward and input gradient, actor backward)."""
    actor = da * h + h * h + 4 * h
    critic = dc * h + h * h + h
    return actor + 2 * critic + 2 * critic + 2 * 2 * critic + 0.5 * (actor + 2 * critic + 2 * actor)


def measure_training(torch, q, W, n_runs=512, capacity=2048, long_steps=1000, equal_steps=40):
    """Batched training (the c4 workload, bounded): n_runs runs of mixed widths and batches,
    8 envs each, replay rings of `capacity` slots filled past wrapping (random warm-up
    actions, no updates) before anything is timed.  Wall time to N actor-critic updates:
      * persistent: all runs in one persistent launch, graph-captured (ac_plan), cluster
        size from the autotuner; timed directly over long_steps steps (n_runs x long_steps
        updates) and over equal_steps steps;
      * plain forms, the same runs launched one at a time, each on its own single-run
        cluster size (automatic), no per-launch allocation or synchronisation: one launch
        per run and env step (ac_train persistent=0), and one launch per run for all its
        steps (persistent=2); timed over equal_steps steps (n_runs x equal_steps updates).
    speedup = plain wall time / persistent wall time for the same N."""
    prefill = capacity + 16
    runs, envs, flop_step = _c4_runs(q, W, n_runs, capacity, learning_starts=prefill)
    res = {}
    try:
        q.ac_train(runs, envs, prefill, persistent=1)  # rings wrap; warm-up actions only
        torch.cuda.synchronize()
        info = q.qsim_info_get(envs[0])
        assert info["size"] == capacity and info["t_now"] == prefill
        # persistent arm first (its launches come early, for profiling), then the plain forms
        cluster = q.ac_train_autotune(runs, envs, 4)
        torch.cuda.synchronize()
        for steps, tag in ((long_steps, "persistent"), (equal_steps, "persistent_equal_n")):
            plan = q.ac_plan_create(runs, envs, steps)  # persistent launch captured in a graph
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q.ac_plan_run(plan, 1)
            q.ac_plan_sync(plan)
            dt = time.perf_counter() - t0
            q.ac_plan_destroy(plan)
            res[tag] = {"s": dt, "updates": n_runs * steps, "updates_per_s": n_runs * steps / dt,
                        "tflops": flop_step * steps / dt / 1e12}
        # plain forms, each run on its automatic single-run cluster (the header's rule: 16
        # CTAs, halved while a CTA would get fewer than 16 samples)
        per_run = {}
        for a in runs:
            q.ac_set_cluster(a, 0)
            b = q.ac_info_get(a)["batch"]
            s_ = 16
            while s_ > 1 and (b % s_ or b // s_ < 16):
                s_ //= 2
            per_run[f"batch{b}"] = s_
        for form, tag in ((0, "plain_launch_per_run_step"), (2, "plain_launch_per_run")):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q.ac_train(runs, envs, equal_steps, persistent=form)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            res[tag] = {"s": dt, "updates": n_runs * equal_steps,
                        "updates_per_s": n_runs * equal_steps / dt,
                        "tflops": flop_step * equal_steps / dt / 1e12}
    finally:
        for a, h in zip(runs, envs):
            q.ac_destroy(a)
            q.qsim_destroy(h)
    fp32_peak = device_peaks(torch, q)[2]
    for k in ("persistent", "persistent_equal_n"):
        res[k]["fp32_frac"] = res[k]["tflops"] / fp32_peak
    eq = res["persistent_equal_n"]["s"]
    res["speedup_vs_plain_launch_per_run_step"] = res["plain_launch_per_run_step"]["s"] / eq
    res["speedup_vs_plain_launch_per_run"] = res["plain_launch_per_run"]["s"] / eq
    res["speedup_vs_plain"] = min(res["speedup_vs_plain_launch_per_run_step"],
                                  res["speedup_vs_plain_launch_per_run"])
    res["fp32_peak"] = fp32_peak
    res["config"] = {"runs": n_runs, "envs_per_run": 8, "replay_slots_per_run": capacity,
                     "prefill_steps": prefill, "rings_wrapped": True, "updates_per_step": 1,
                     "equal_n_steps": equal_steps, "long_steps": long_steps,
                     "cluster_persistent_autotuned": cluster,
                     "cluster_plain_per_run": per_run,
                     "flop_count": "2 x B x update_macs(82, 90, hidden) per run and update"}
    return res


def measure_c1(torch, q, W, steps=10_000):
    """The plain single run (c1): 1 env with the fixed vehicle, batch 256, replay 10,000,
    1,000 warm-up steps, then one update per env step: wall time of the whole 10,000-step
    training (9,000 updates) in one call, timed directly on a fresh run.  The cluster size
    comes from the autotuner run beforehand on a separate run of the same shape."""
    d = W.config("c1")
    hp = dict(W.TD3)

    def new_run():
        cfg = q.make_config(d, 1, 10_000, reward=W.REWARD, sigma_e=0.1)
        h = q.qsim_create(cfg, q.make_params(d))
        return q.ac_create(q.make_ac_config(hp), h), h

    a, h = new_run()
    q.ac_train([a], [h], 1100, persistent=1)
    cluster = q.ac_train_autotune([a], [h], 20)
    q.ac_destroy(a)
    q.qsim_destroy(h)
    a, h = new_run()
    q.ac_set_cluster(a, cluster)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q.ac_train([a], [h], steps, persistent=1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ai = q.ac_info_get(a)
    upd = int(ai["updates"])
    q.ac_destroy(a)
    q.qsim_destroy(h)
    return {"env_steps": steps, "updates": upd, "s": dt, "updates_per_s": upd / dt,
            "env_steps_per_s": steps / dt, "cluster_autotuned": cluster,
            "learning_starts": d["learning_starts"]}


def measure_diff(torch, q, W, n=4096, H=200, ckpt=20):
    """Differentiation workload: gradients of the H-step loss w.r.t. the actor weights and
    (m, J) of n envs, closed loop with the 82-64-64-4 actor, checkpoint every ckpt steps;
    and w.r.t. the action sequence in open loop."""
    import numpy as np
    from paper_2311_13081_gb300 import diff
    d = W.config("c1")
    veh = q.make_params(d)
    ld = (n + 31) // 32 * 32
    s0 = torch.tensor(W.random_states(0, ld, p=0.1, v=0.5, w=0.5, rpm=(12000.0, 17000.0)).T.copy(),
                      dtype=torch.float32, device="cuda")
    prm = torch.tensor(W.random_params(1, ld).T.copy(), dtype=torch.float32, device="cuda")
    res = {}
    for mode, lanes in ((1, 32), (1, 16), (1, 0), (0, 0)):
        desc = diff.make_desc(n, ld, H, ckpt, mode, (1.0, 0.5, 0.2, 0.05), n_hist=16, hidden=64,
                              lanes_per_env=lanes)
        ws = torch.empty(q.qsim_vjp_workspace(desc) // 4 + 1, device="cuda")
        loss = torch.zeros(ld, device="cuda")
        gp = torch.zeros(4, ld, device="cuda")
        if mode == 1:
            hp = dict(W.TD3)
            cfg = q.make_config(d, 1, 32, reward=W.REWARD)
            h = q.qsim_create(cfg, veh)
            a = q.ac_create(q.make_ac_config(hp), h)
            x = q.ac_info_get(a)["actor"].clone()
            q.ac_destroy(a)
            q.qsim_destroy(h)
            gx = torch.zeros_like(x)
            args = (None, x, None, loss, None, gx, gp, None, ws)
        else:
            x = torch.tensor(W.random_actions(2, (H, 4, ld), -0.3, 0.4), dtype=torch.float32,
                             device="cuda")
            gx = torch.zeros_like(x)
            args = (x, None, None, loss, gx, None, gp, None, ws)
        q.qsim_rollout_vjp(desc, veh, s0, prm, *args)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        q.qsim_rollout_vjp(desc, veh, s0, prm, *args)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        tag = ("closed_loop_actor" if lanes == 0 else f"closed_loop_actor_{lanes}_lanes_per_env") \
            if mode == 1 else "open_loop_actions"
        res[tag] = {"ms": ms, "env_steps_per_s": n * H / (ms * 1e-3),
                    "finite": bool(torch.isfinite(gx).all() and torch.isfinite(gp).all())}
        if mode == 1 and lanes == 0:
            res[tag]["lanes_per_env"] = 8
    res["config"] = {"envs": n, "horizon": H, "ckpt": ckpt,
                     "workspace_mb": q.qsim_vjp_workspace(desc) / 1e6}
    return res


def measure_c5(torch, q, W, hbm, n_runs=128, n_envs=64, records=1_000_000, iters=40,
               updates_per_step=64):
    """Asymmetric privileged critic + curriculum at scale (c5, bounded): 128 runs x 64 envs,
    replay rings of 1,000,000 records per run (15,625 slots x 64 envs), filled completely
    with warm-up steps before anything is timed.
      * reward recalculation (Sec. VI) over every run's full ring, the stand-alone kernel
        once per run: 128 x 10^6 records, GB/s against the measured HBM copy bandwidth;
      * training: iters steps of all runs in one graph-captured persistent launch, 64
        updates per step (update-to-data ratio 1), with the curriculum interval shortened to
        1,024 interactions so that the sample contains curriculum changes, each followed
        by the recalculation over the run's full ring inside the training kernel."""
    runs, envs = [], []
    cur = dict(W.CURRICULUM)
    cur["interval"] = 1024
    slots = records // n_envs
    for r in range(n_runs):
        d = W.config("c5")
        d.update(seed=r, run_id=r, learning_starts=slots + 20)
        cfg = q.make_config(d, n_envs, slots, reward=W.REWARD, sigma_e=0.1, curriculum=cur)
        h = q.qsim_create(cfg, q.make_params(d))
        hp = dict(W.TD3)
        hp.update(hidden=64, batch=256)
        runs.append(q.ac_create(q.make_ac_config(hp, cluster=1, updates_per_step=updates_per_step), h))
        envs.append(h)
    res = {}
    try:
        q.ac_train(runs, envs, slots + 20, persistent=1)  # fills every ring (warm-up actions)
        torch.cuda.synchronize()
        info = q.qsim_info_get(envs[0])
        assert info["size"] == slots
        q.qsim_recalc_rewards_batch(envs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record()
        for _ in range(reps):
            q.qsim_recalc_rewards_batch(envs)  # every run's ring in one launch
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        total = n_runs * slots * n_envs
        gbs = total * 92 / (ms * 1e-3) / 1e9
        res["reward_recalc_full_rings"] = {
            "records": total, "ms": ms, "launches": 1, "gbs": gbs,
            "frac_of_measured_hbm": gbs / hbm, "bytes_per_record": 92}
        plan = q.ac_plan_create(runs, envs, iters)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.ac_plan_run(plan, 1)
        q.ac_plan_sync(plan)
        dt = time.perf_counter() - t0
        q.ac_plan_destroy(plan)
        rc = q.qsim_info_get(envs[0])["reward_c"].tolist()
        upd = n_runs * iters * updates_per_step
        res.update({"s": dt, "env_steps": n_runs * n_envs * iters, "updates": upd,
                    "updates_per_s": upd / dt, "env_steps_per_s": n_runs * n_envs * iters / dt,
                    "C_ra_after": rc[4], "sigma_e_after": rc[7]})
    finally:
        for a, h in zip(runs, envs):
            q.ac_destroy(a)
            q.qsim_destroy(h)
    res["config"] = {"runs": n_runs, "envs_per_run": n_envs, "iters": iters,
                     "updates_per_step": updates_per_step, "replay_per_run": slots * n_envs,
                     "rings_filled": True, "curriculum_interval": 1024,
                     "critic": "privileged (96 inputs)"}
    return res


def cpu_baseline(n_envs=4096, horizon=1000, chunk=50):
    """The FP64 oracle (as it stands) on this host's cores: a bounded sample of the
    rollout workload (n_envs x horizon env-steps, all cores)."""
    import numpy as np

    import oracle as O
    import workloads as W
    O.build()
    cores = os.cpu_count() or 1
    d = W.config("c2")
    d.update(learning_starts=0)
    actor = O.init_params(d, 0, 82, 64, 4)
    e = O.new_envs(d, np.arange(n_envs))
    t0 = time.perf_counter()
    for c in range(0, horizon, chunk):
        O.rollout(d, W.REWARD, e, min(chunk, horizon - c), c, actor=actor, hidden=64,
                  sigma_e=0.1, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_envs * horizon / dt, "unit": "env-steps/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{n_envs} envs x {horizon} steps of the same rollout workload "
                      f"(FP64 C oracle, {cores} threads), {dt:.1f} s"}


# ------------------------------------------------------------------------------ main arms
def arm_config(n, horizon, **extra):
    """The workload the headline is quoted on (both arms report it)."""
    c = {"workload": f"c2 batched rollout: {n} domain-randomised quadrotors x {horizon} steps per "
                     f"bench step, actor 82-64-64-4, replay {n}x{horizon} in HBM",
         "envs_per_gpu": n, "steps_per_bench_step": horizon}
    c.update(extra)
    return c


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    import workloads as W
    O.build()
    cores = os.cpu_count() or 1
    d = W.config("c2")
    d.update(learning_starts=0)
    actor = O.init_params(d, 0, 82, 64, 4)
    n, T = 4096, 40
    e = O.new_envs(d, np.arange(n))
    t = 0
    for _ in range(args.warmup):
        O.rollout(d, W.REWARD, e, T, t, actor=actor, hidden=64, sigma_e=0.1, n_threads=cores)
        t += T
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.rollout(d, W.REWARD, e, T, t, actor=actor, hidden=64, sigma_e=0.1, n_threads=cores)
        t += T
    dt = time.perf_counter() - t0
    v = n * T * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args.envs, args.horizon),
            "cpu_baseline": {"value": v, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} of the {args.envs} envs x {T} of the {args.horizon} steps "
                                       f"per bench step (a bounded sample of the workload; "
                                       f"env-steps/s is per env-step), {cores} threads"},
            "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2311_13081_gb300 as q
    import workloads as W

    if args.only_diff:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        print(json.dumps({"differentiation_c3": measure_diff(torch, q, W)}))
        return
    if args.only_c1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        print(json.dumps({"learner_single_run_c1": measure_c1(torch, q, W)}))
        return
    if args.only_recalc:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        hbm = device_peaks(torch, q)[3]
        d = rank_workload(W, 0)
        cfg = q.make_config(d, args.envs, args.only_recalc, reward=W.REWARD, sigma_e=0.1)
        h = q.qsim_create(cfg, q.make_params(d))
        a = q.ac_create(q.make_ac_config(dict(W.TD3)), h)
        q.qsim_rollout(h, q.ac_info_get(a)["actor"], 64, args.only_recalc + 1)  # fills the ring
        print(json.dumps({"reward_recalc": measure_recalc(torch, q, h, args.envs, args.only_recalc, hbm)}))
        q.ac_destroy(a)
        q.qsim_destroy(h)
        return
    if args.only_dynamics:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        veh = q.make_params(W.config("c1"))
        n = args.dyn_envs
        out = torch.empty(17, q.padded(n), device="cuda")
        for _ in range(2):
            q.qsim_dynamics_bench(veh, n, q.padded(n), args.only_dynamics, 0.01, out)
        torch.cuda.synchronize()
        print(json.dumps({"dynamics_only": {"envs": n, "steps": args.only_dynamics,
                                            "finite": bool(torch.isfinite(out).all())}}))
        return
    if args.only_c5:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        hbm = device_peaks(torch, q)[3]
        print(json.dumps({"asymmetric_curriculum_c5": measure_c5(torch, q, W, hbm)}))
        return
    if args.only_ablation:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        print(json.dumps({"ablation_study": measure_ablation(torch, q, W)}))
        return
    if args.only_track:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        fp32_peak = device_peaks(torch, q)[2]
        print(json.dumps({"lissajous_tracking": measure_track(torch, q, W, fp32_peak)}))
        return
    if args.only_learner:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        q.load()
        print(json.dumps({"learner_batched": measure_training(torch, q, W, n_runs=args.only_learner,
                                                              long_steps=args.learner_steps)}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    q.load()
    n, horizon = args.envs, args.horizon
    d = rank_workload(W, rank)
    veh = q.make_params(d)
    cfg = q.make_config(d, n, horizon, reward=W.REWARD, sigma_e=0.1)
    h = q.qsim_create(cfg, veh)
    hp = dict(W.TD3)
    a = q.ac_create(q.make_ac_config(hp), h)  # random-init actor (Philox tag 7, seed 0)
    actor = q.ac_info_get(a)["actor"]
    hidden = 64
    info = q.qsim_info_get(h)
    l2 = torch.empty(512 * 1024 * 1024 // 4, device="cuda")
    if args.warps:
        tuned = q.qsim_rollout_tune(h, args.warps)
        q.qsim_rollout_schedule(h, args.parts, args.chunk if args.parts > 1 else 0)
        q.qsim_rollout_engine(h, args.engine if args.engine >= 0 else args.packed)
    else:
        if args.engine >= 0:
            q.qsim_rollout_engine(h, args.engine)
        tuned = q.qsim_rollout_autotune(h, actor, hidden, 100)
    for _ in range(args.warmup):
        q.qsim_rollout(h, actor, hidden, horizon)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with Clocks(local) as clk:
        time.sleep(0.3)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush_l2(l2)
            starts[k].record()
            q.qsim_rollout(h, actor, hidden, horizon)
            ends[k].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    packed_used = q.qsim_rollout_engine(h, -2)
    parts_used = q.qsim_rollout_schedule(h, -1, -1)
    t_dev = max_over_ranks(torch, dist, sum(ms) / 1e3, world, "cuda")
    if world > 1:
        dist.barrier()
    env_steps = n * horizon * args.steps * world
    value = env_steps / t_dev
    sms, max_mhz, fp32_peak, hbm, hbm_src, f16_peak, tc_src = device_peaks(torch, q)
    flop_step = FLOP_ACTOR(82, hidden) + FLOP_DYN + FLOP_MISC
    achieved = n * horizon * flop_step / (sum(ms) / args.steps * 1e-3) / 1e12
    clocks = clk.summary()

    # end to end through the C ABI with host buffers: pinned actor weights in, episode
    # statistics out, every step
    host_actor = actor.detach().cpu().pin_memory()
    dev_actor = torch.empty_like(actor)
    host_stats = torch.empty(3, info["ld"], dtype=torch.int32).pin_memory()
    stats_dev = torch.stack([info["n_done"], info["len_sum"], info["ret_sum"].view(torch.int32)])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    w0 = time.perf_counter()
    for k in range(args.steps):
        dev_actor.copy_(host_actor, non_blocking=True)
        q.qsim_rollout(h, dev_actor, hidden, horizon)
        stats_dev = torch.stack([info["n_done"], info["len_sum"], info["ret_sum"].view(torch.int32)])
        host_stats.copy_(stats_dev, non_blocking=True)
        torch.cuda.synchronize()
    e2e_t = max_over_ranks(torch, dist, time.perf_counter() - w0, world, "cuda")
    e2e = {"value": env_steps / max(e2e_t, 1e-9), "unit": "env-steps/s",
           "h2d_bytes_per_step": host_actor.numel() * 4,
           "d2h_bytes_per_step": host_stats.numel() * 4}

    extras = {}
    if rank == 0 and not args.no_extras:
        extras["fp32_fma_probe_tflops"] = measure_ffma(torch, q)
        extras["tcgen05_mma_issue_probe"] = measure_mma_rate(torch, q)
        extras["reward_recalc"] = measure_recalc(torch, q, h, n, horizon, hbm)
        st = q.qsim_stats_get(h)
        extras["episodes"] = st
    q.ac_destroy(a)
    q.qsim_destroy(h)
    del l2
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_extras:
        extras["dynamics_only"] = measure_dynamics(torch, q, veh)
        extras["lissajous_tracking"] = measure_track(torch, q, W, fp32_peak)
        extras["learner_batched"] = measure_training(torch, q, W)
        extras["learner_single_run_c1"] = measure_c1(torch, q, W)
        extras["differentiation_c3"] = measure_diff(torch, q, W)
        extras["asymmetric_curriculum_c5"] = measure_c5(torch, q, W, hbm)
        extras["ablation_study"] = measure_ablation(torch, q, W)
    step_s = sum(ms) / args.steps * 1e-3
    hbm_ach = n * horizon * BYTES_STEP / step_s / 1e9
    if packed_used == 2:
        # tensor-core engine: the dominant kernel's MLP runs on the tensor pipe; achieved =
        # the method's work (actor 19,200 + RK4 672 + misc 60 flop per env-step) / time,
        # against the fp16 dense tensor peak (the emulated fp16 MMA flops are reported
        # separately)
        tc_flop = FLOP_TC_MMA(82, hidden)
        ach = n * horizon * flop_step / step_s / 1e12
        mma = n * horizon * tc_flop / step_s / 1e12
        roofline = {"bound": "tensor", "achieved": ach, "peak": f16_peak, "unit": "TFLOP/s",
                    "frac": ach / f16_peak,
                    "traffic": (None if NCU_DRAM_BYTES_PER_ENV_STEP_TC is None
                                else NCU_DRAM_BYTES_PER_ENV_STEP_TC * n * horizon),
                    "peak_source": f"fp16 dense tensor, sustained ({tc_src} bf16 sustained; equal rates)",
                    "flop_per_env_step": flop_step,
                    "fp32_equivalent_frac": ach / fp32_peak,
                    "fp32_peak": fp32_peak,
                    "fp32_peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                    "mma_instructions_per_env_step": 30 / 128,
                    "mma_flop_per_env_step": tc_flop,
                    "mma_tflops": mma, "mma_frac": mma / f16_peak,
                    "simt_fp32_tflops": n * horizon * (FLOP_DYN + FLOP_MISC + 2 * 4 * hidden) / step_s / 1e12,
                    "hbm_gbs_achieved": hbm_ach, "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                    "traffic": (None if NCU_DRAM_BYTES_PER_ENV_STEP is None
                                else NCU_DRAM_BYTES_PER_ENV_STEP * n * horizon),
                    "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                    "flop_per_env_step": flop_step,
                    "hbm_gbs_achieved": hbm_ach, "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src}
    chunk_used = args.chunk if args.warps else 100
    launches = args.steps * (parts_used * -(-horizon // max(1, min(chunk_used, horizon)))
                             if parts_used > 1 else 1)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": arm_config(n, horizon, l2="flushed before every timed step (512 MB write)",
                                 rollout_warps_per_block=tuned, rollout_engine=packed_used,
                                 rollout_partitions=parts_used),
            "roofline": roofline,
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
            "cpu_baseline": cpu, "step_ms": ms, "wall_s": wall,
        }
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
