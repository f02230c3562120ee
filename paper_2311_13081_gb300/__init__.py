"""Thin Python binding of libqsim (the C ABI in ``include/qsim.h``).

Argument marshalling only: every step of the simulation and training hot path runs in
the library's CUDA kernels.  PyTorch is used for device memory (tensors passed by
``data_ptr()``) and streams.  There is no CPU fallback: if the library is not built,
:func:`load` raises.

Function names follow the C ABI (``qsim_create``, ``qsim_step``, ``qsim_rollout``,
``ac_update``, ``ac_train`` ...).  Handles are returned as opaque ``ctypes.c_void_p``.
Device arrays owned by a handle are exposed zero-copy through ``qsim_info_get`` /
``ac_info_get`` as torch tensors (field-major ``[field][ld]``).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

from . import build as _build

_lib = None
P = C.c_void_p


class QsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qsim status {status}: {msg}")
        self.status = status


# ------------------------------------------------------------------------- ABI structs
class QsimParams(C.Structure):
    _fields_ = [("mass", C.c_float), ("J", C.c_float * 3), ("kf", C.c_float), ("km", C.c_float),
                ("motor_tau", C.c_float), ("rotor_pos", C.c_float * 12),
                ("rotor_dir", C.c_float * 4), ("rpm_min", C.c_float), ("rpm_max", C.c_float),
                ("g", C.c_float)]


class QsimConfig(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("n_hist", C.c_int32), ("episode_len", C.c_int32),
                ("critic_layout", C.c_int32), ("renorm_q", C.c_int32),
                ("learning_starts", C.c_int32), ("replay_capacity", C.c_int32),
                ("motor_lag_off", C.c_int32), ("dt", C.c_float), ("run_id", C.c_uint32),
                ("seed", C.c_uint64),
                ("init_p", C.c_float), ("init_att", C.c_float), ("init_v", C.c_float),
                ("init_w", C.c_float), ("init_rpm_lo", C.c_float), ("init_rpm_hi", C.c_float),
                ("dr_mass", C.c_float), ("dr_J", C.c_float), ("dr_kf", C.c_float),
                ("tm_lo", C.c_float), ("tm_hi", C.c_float), ("dist_f", C.c_float),
                ("dist_tau", C.c_float), ("sig_p", C.c_float), ("sig_R", C.c_float),
                ("sig_v", C.c_float), ("sig_w", C.c_float), ("term_pos", C.c_float),
                ("reward", C.c_float * 7), ("curriculum_factor", C.c_float * 7),
                ("curriculum_target", C.c_float * 7), ("sigma_e", C.c_float),
                ("sigma_factor", C.c_float), ("sigma_min", C.c_float),
                ("recalc_rewards", C.c_int32), ("curriculum_interval", C.c_int64)]


class QsimInfo(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("ld", C.c_int32), ("obs_dim", C.c_int32),
                ("critic_obs_dim", C.c_int32), ("record_fields", C.c_int32),
                ("n_priv", C.c_int32), ("capacity", C.c_int64), ("t_now", C.c_int64),
                ("head", C.c_int64), ("size", C.c_int64),
                ("state", P), ("params", P), ("dist", P), ("hist", P), ("ep_index", P),
                ("ep_step", P), ("ep_ret", P), ("n_done", P), ("len_sum", P), ("ret_sum", P),
                ("records", P), ("side", P), ("reward_c", P)]


class QsimStats(C.Structure):
    _fields_ = [("episodes", C.c_int64), ("mean_length", C.c_double),
                ("mean_return", C.c_double)]


class AcConfig(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("batch", C.c_int32), ("policy_delay", C.c_int32),
                ("updates_per_step", C.c_int32), ("gamma", C.c_float), ("tau", C.c_float),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("sigma_target", C.c_float), ("noise_clip", C.c_float),
                ("cluster", C.c_int32), ("reserved0", C.c_int32)]


class AcInfo(C.Structure):
    _fields_ = [("obs_dim", C.c_int32), ("critic_in", C.c_int32), ("hidden", C.c_int32),
                ("batch", C.c_int32), ("n_actor", C.c_int32), ("n_critic", C.c_int32),
                ("t_actor", C.c_int64), ("t_critic", C.c_int64), ("updates", C.c_int64),
                ("actor", P), ("actor_t", P), ("c1", P), ("c1_t", P), ("c2", P), ("c2_t", P),
                ("m_a", P), ("v_a", P), ("m_c1", P), ("v_c1", P), ("m_c2", P), ("v_c2", P),
                ("stats", P)]


class QsimVjpDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("ld", C.c_int32), ("H", C.c_int32), ("ckpt", C.c_int32),
                ("mode", C.c_int32), ("n_hist", C.c_int32), ("hidden", C.c_int32),
                ("lanes_per_env", C.c_int32), ("w_p", C.c_float), ("w_q", C.c_float),
                ("w_v", C.c_float), ("w_a", C.c_float), ("dt", C.c_float),
                ("renorm", C.c_int32)]


_SIGS = {
    "qsim_last_error": (C.c_char_p, []),
    "qsim_abi_version": (C.c_int32, []),
    "qsim_memcpy": (C.c_int, [P, P, C.c_size_t, P]),
    "qsim_stream_sync": (C.c_int, [P]),
    "qsim_philox_fill": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.c_int32, C.c_int32, P, P]),
    "qsim_philox_host": (None, [P, P, P]),
    "qsim_dynamics_step": (C.c_int, [C.POINTER(QsimParams), P, P, P, P, C.c_float, C.c_int32,
                                     C.c_int32, C.c_int32, C.c_int32, P, P]),
    "qsim_dynamics_bench": (C.c_int, [C.POINTER(QsimParams), C.c_int32, C.c_int32, C.c_int32,
                                      C.c_float, P, P]),
    "qsim_create": (C.c_int, [C.POINTER(QsimConfig), C.POINTER(QsimParams), C.POINTER(P)]),
    "qsim_destroy": (C.c_int, [P]),
    "qsim_info_get": (C.c_int, [P, C.POINTER(QsimInfo)]),
    "qsim_set_counters": (C.c_int, [P, C.c_int64, C.c_int64, C.c_int64]),
    "qsim_sync": (C.c_int, [P]),
    "qsim_set_wait_limit": (C.c_int32, [P, C.c_int32]),
    "qsim_bounds_checked": (C.c_int32, []),
    "qsim_bounds_probe": (C.c_int, [P, C.c_int64, C.c_int64, P, P]),
    "qsim_observe": (C.c_int, [P, P, P, P]),
    "qsim_step": (C.c_int, [P, P, P, P, P, P, P, P]),
    "qsim_rollout": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_float, P]),
    "qsim_track": (C.c_int, [P, P, C.c_int32, C.c_int32, P, C.c_float, C.c_float, C.c_float,
                             C.c_float, P, P, P]),
    "qsim_rollout_tune": (C.c_int32, [P, C.c_int32]),
    "qsim_rollout_autotune": (C.c_int32, [P, P, C.c_int32, C.c_int32, P]),
    "qsim_rollout_schedule": (C.c_int32, [P, C.c_int32, C.c_int32]),
    "qsim_rollout_packed": (C.c_int32, [P, C.c_int32]),
    "qsim_rollout_engine": (C.c_int32, [P, C.c_int32]),
    "qsim_ffma_probe": (C.c_int, [C.c_int32, C.c_int32, P, P]),
    "qsim_mma_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, P]),
    "qsim_recalc_rewards": (C.c_int, [P, P]),
    "qsim_recalc_rewards_batch": (C.c_int, [P, C.c_int32, P]),
    "qsim_set_reward": (C.c_int, [P, P, C.c_float, P]),
    "qsim_stats_get": (C.c_int, [P, C.POINTER(QsimStats), P]),
    "ac_create": (C.c_int, [C.POINTER(AcConfig), P, C.POINTER(P)]),
    "ac_destroy": (C.c_int, [P]),
    "ac_info_get": (C.c_int, [P, C.POINTER(AcInfo)]),
    "ac_set_counters": (C.c_int, [P, C.c_int64, C.c_int64, C.c_int64]),
    "ac_set_cluster": (C.c_int32, [P, C.c_int32]),
    "ac_set_index_log": (C.c_int, [P, P]),
    "ac_update": (C.c_int, [P, P, C.c_int32, P]),
    "ac_update_static": (C.c_int, [P, P, C.c_int32, P]),
    "ac_train": (C.c_int, [P, P, C.c_int32, C.c_int64, C.c_int32, P]),
    "ac_train_autotune": (C.c_int32, [P, P, C.c_int32, C.c_int32, P]),
    "ac_sync": (C.c_int, [P]),
    "ac_plan_create": (C.c_int, [P, P, C.c_int32, C.c_int32, C.POINTER(P)]),
    "ac_plan_run": (C.c_int, [P, C.c_int32, P]),
    "ac_plan_sync": (C.c_int, [P, P]),
    "ac_plan_destroy": (C.c_int, [P]),
    "ac_save": (C.c_int, [P, P, C.c_char_p]),
    "ac_load": (C.c_int, [P, P, C.c_char_p]),
    "qsim_vjp_workspace": (C.c_size_t, [C.POINTER(QsimVjpDesc)]),
    "qsim_rollout_vjp": (C.c_int, [C.POINTER(QsimVjpDesc), C.POINTER(QsimParams), P, P, P, P,
                                   P, P, P, P, P, P, P, P]),
}


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libqsim (built by ``build.build()``).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libqsim not built ({path}); run paper_2311_13081_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)  # every declared entry point must be exported
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _chk(status):
    if status != 0:
        raise QsimError(status, _lib.qsim_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream=None):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


class _Dev:
    """Zero-copy device array descriptor (CUDA array interface)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape),
                                         "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def view(ptr: int, shape, dtype: str = "f4") -> torch.Tensor:
    """Torch view of a library-owned device array (float32 "f4" or int32 "i4")."""
    return torch.as_tensor(_Dev(ptr, shape, "<" + dtype), device="cuda")


# ---------------------------------------------------------------------- config helpers
def make_params(d: dict) -> QsimParams:
    p = QsimParams()
    p.mass = d["mass"]
    p.J[0], p.J[1], p.J[2] = d["Jx"], d["Jy"], d["Jz"]
    p.kf, p.km, p.motor_tau = d["kf"], d["km"], d["tm"]
    for i, x in enumerate(d["rotor_pos"]):
        p.rotor_pos[i] = x
    for i, x in enumerate(d["rotor_dir"]):
        p.rotor_dir[i] = x
    p.rpm_min, p.rpm_max, p.g = d["rpm_min"], d["rpm_max"], d["g"]
    return p


def make_config(d: dict, n_envs: int, replay_capacity: int = 0, reward=None, sigma_e=0.1,
                curriculum: dict | None = None, recalc_rewards: int = 1) -> QsimConfig:
    c = QsimConfig()
    c.n_envs, c.replay_capacity = int(n_envs), int(replay_capacity)
    for k in ("n_hist", "episode_len", "critic_layout", "renorm_q", "learning_starts"):
        setattr(c, k, int(d[k]))
    c.motor_lag_off = int(d.get("motor_lag_off", 0))
    c.dt, c.run_id, c.seed = d["dt"], int(d.get("run_id", 0)), int(d.get("seed", 0))
    for k in ("init_p", "init_att", "init_v", "init_w", "init_rpm_lo", "init_rpm_hi", "dr_mass",
              "dr_J", "dr_kf", "tm_lo", "tm_hi", "dist_f", "dist_tau", "sig_p", "sig_R", "sig_v",
              "sig_w", "term_pos"):
        setattr(c, k, float(d[k]))
    rw = reward if reward is not None else d.get("reward")
    for i, x in enumerate(rw):
        c.reward[i] = x
    c.sigma_e = float(sigma_e)
    if curriculum:
        c.curriculum_interval = int(curriculum["interval"])
        for i in range(7):
            c.curriculum_factor[i] = curriculum["factor"][i]
            c.curriculum_target[i] = curriculum["target"][i]
        c.sigma_factor = float(curriculum.get("sigma_factor", 1.0))
        c.sigma_min = float(curriculum.get("sigma_min", 0.0))
    else:
        c.curriculum_interval = 0
        for i in range(7):
            c.curriculum_factor[i] = 1.0
            c.curriculum_target[i] = c.reward[i]
        c.sigma_factor, c.sigma_min = 1.0, 0.0
    c.recalc_rewards = int(recalc_rewards)
    return c


def make_ac_config(d: dict, cluster: int = 0, updates_per_step: int = 1) -> AcConfig:
    a = AcConfig()
    a.hidden, a.batch, a.policy_delay = int(d["hidden"]), int(d["batch"]), int(d["policy_delay"])
    a.updates_per_step = int(updates_per_step)
    a.gamma, a.tau, a.lr = d["gamma"], d["tau"], d["lr"]
    a.beta1, a.beta2, a.eps = d["beta1"], d["beta2"], d["eps"]
    a.sigma_target, a.noise_clip = d["sigma_t"], d["noise_clip"]
    a.cluster = int(cluster)
    return a


# ---------------------------------------------------------------------------- ABI calls
def qsim_philox_fill(seed, run, tag, sub, c1, out: torch.Tensor, kind=0, stream=None):
    load()
    n = out.numel() // 4
    _chk(_lib.qsim_philox_fill(seed, run, tag, sub, c1, n, kind, _ptr(out), _stream(stream)))


def qsim_philox_host(ctr, key):
    load()
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    _lib.qsim_philox_host(C.cast(c, P), C.cast(k, P), C.cast(o, P))
    return [int(x) for x in o]


def qsim_dynamics_step(veh: QsimParams, params, dist, state_in, rpm, dt, renorm, n, ld,
                       n_steps, state_out, stream=None):
    load()
    _chk(_lib.qsim_dynamics_step(C.byref(veh), _ptr(params), _ptr(dist), _ptr(state_in),
                                 _ptr(rpm), dt, renorm, n, ld, n_steps, _ptr(state_out),
                                 _stream(stream)))


def qsim_dynamics_bench(veh: QsimParams, n, ld, n_steps, dt, state_out, stream=None):
    load()
    _chk(_lib.qsim_dynamics_bench(C.byref(veh), n, ld, n_steps, dt, _ptr(state_out),
                                  _stream(stream)))


def qsim_create(cfg: QsimConfig, veh: QsimParams):
    load()
    h = P()
    _chk(_lib.qsim_create(C.byref(cfg), C.byref(veh), C.byref(h)))
    return h


def qsim_destroy(h):
    if h:
        _chk(_lib.qsim_destroy(h))


def qsim_info_get(h) -> dict:
    inf = QsimInfo()
    _chk(_lib.qsim_info_get(h, C.byref(inf)))
    ld, cap, F = inf.ld, inf.capacity, inf.record_fields
    out = dict(n_envs=inf.n_envs, ld=ld, obs_dim=inf.obs_dim, critic_obs_dim=inf.critic_obs_dim,
               record_fields=F, n_priv=inf.n_priv, capacity=cap, t_now=inf.t_now,
               head=inf.head, size=inf.size)
    out["state"] = view(inf.state, (17, ld))
    out["params"] = view(inf.params, (8, ld))
    out["dist"] = view(inf.dist, (6, ld))
    out["hist"] = view(inf.hist, (64, ld))
    for k in ("ep_index", "ep_step", "n_done", "len_sum"):
        out[k] = view(getattr(inf, k), (ld,), "i4")
    out["ep_ret"] = view(inf.ep_ret, (ld,))
    out["ret_sum"] = view(inf.ret_sum, (ld,))
    out["reward_c"] = view(inf.reward_c, (8,))
    if cap > 0:
        out["records"] = view(inf.records, (cap, F, ld))
        # env-major on the device; returned as a [capacity][17][ld] view like the records
        out["side"] = view(inf.side, (cap, ld, 17)).permute(0, 2, 1)
    return out


def qsim_set_counters(h, t_now, head, size):
    _chk(_lib.qsim_set_counters(h, t_now, head, size))


def qsim_sync(h):
    _chk(_lib.qsim_sync(h))


def qsim_set_wait_limit(h, polls) -> int:
    """Polls of a bounded device-side wait before it gives up (0 = default); returns the
    previous limit."""
    r = _lib.qsim_set_wait_limit(h, int(polls))
    if r < 0:
        _chk(r)
    return r


def qsim_bounds_checked() -> bool:
    """True when the loaded library was built with the debug bounds checks."""
    load()
    return bool(_lib.qsim_bounds_checked())


def qsim_bounds_probe(h, slot, env, out: torch.Tensor, stream=None):
    """Flag word of ring record (slot, env) into out (int32, 1 element) through the debug
    bounds check (out-of-range indices: see include/qsim.h)."""
    _chk(_lib.qsim_bounds_probe(h, int(slot), int(env), _ptr(out), _stream(stream)))


def qsim_observe(h, obs_a=None, obs_c=None, stream=None):
    _chk(_lib.qsim_observe(h, _ptr(obs_a), _ptr(obs_c), _stream(stream)))


def qsim_step(h, actions, obs_a=None, obs_c=None, reward=None, terminated=None, truncated=None,
              stream=None):
    _chk(_lib.qsim_step(h, _ptr(actions), _ptr(obs_a), _ptr(obs_c), _ptr(reward),
                        _ptr(terminated), _ptr(truncated), _stream(stream)))


def qsim_rollout(h, actor, hidden, n_steps, sigma_e=-1.0, stream=None):
    _chk(_lib.qsim_rollout(h, _ptr(actor), hidden, n_steps, sigma_e, _stream(stream)))


def qsim_track(h, actor, hidden, n_steps, period, sq_err, steps_ok, amplitude=1.0, z0=0.0,
               clip_p=0.2, clip_v=1.0, stream=None):
    """Lissajous tracking flight of every env (period float32 [ld], sq_err float64 [2][ld],
    steps_ok int32 [ld]; device tensors)."""
    _chk(_lib.qsim_track(h, _ptr(actor), hidden, n_steps, _ptr(period), amplitude, z0, clip_p,
                         clip_v, _ptr(sq_err), _ptr(steps_ok), _stream(stream)))


def qsim_rollout_tune(h, warps_per_block=0) -> int:
    return _lib.qsim_rollout_tune(h, warps_per_block)


def qsim_rollout_autotune(h, actor, hidden, n_steps, stream=None) -> int:
    r = _lib.qsim_rollout_autotune(h, _ptr(actor), hidden, n_steps, _stream(stream))
    if r < 0:
        _chk(r)
    return int(r)


def qsim_rollout_schedule(h, parts=-1, chunk=-1) -> int:
    return int(_lib.qsim_rollout_schedule(h, parts, chunk))


def qsim_rollout_packed(h, packed=-1) -> int:
    return int(_lib.qsim_rollout_packed(h, packed))


def qsim_rollout_engine(h, engine=-2) -> int:
    """0 SIMT, 1 SIMT paired FMA, 2 tensor cores (hidden 64), -1 automatic; other values
    only query."""
    return int(_lib.qsim_rollout_engine(h, engine))


def qsim_mma_probe(n_mma, n_cols, n_warps, cycles, stream=None):
    load()
    _chk(_lib.qsim_mma_probe(n_mma, n_cols, n_warps, _ptr(cycles), _stream(stream)))


def qsim_ffma_probe(n_blocks, iters, out, stream=None):
    load()
    _chk(_lib.qsim_ffma_probe(n_blocks, iters, _ptr(out), _stream(stream)))


def qsim_recalc_rewards(h, stream=None):
    _chk(_lib.qsim_recalc_rewards(h, _stream(stream)))


def qsim_recalc_rewards_batch(hs, stream=None):
    """Reward recalculation of several env sets in one launch."""
    n = len(hs)
    ha = (P * n)(*[h.value if isinstance(h, P) else h for h in hs])
    _chk(_lib.qsim_recalc_rewards_batch(C.cast(ha, P), n, _stream(stream)))


def qsim_set_reward(h, c7, sigma_e, stream=None):
    arr = (C.c_float * 7)(*[float(x) for x in c7])
    _chk(_lib.qsim_set_reward(h, C.cast(arr, P), float(sigma_e), _stream(stream)))
    torch.cuda.current_stream().synchronize()


def qsim_stats_get(h, stream=None) -> dict:
    s = QsimStats()
    _chk(_lib.qsim_stats_get(h, C.byref(s), _stream(stream)))
    return dict(episodes=s.episodes, mean_length=s.mean_length, mean_return=s.mean_return)


def ac_create(cfg: AcConfig, env):
    load()
    h = P()
    _chk(_lib.ac_create(C.byref(cfg), env, C.byref(h)))
    return h


def ac_destroy(a):
    if a:
        _chk(_lib.ac_destroy(a))


def ac_info_get(a) -> dict:
    inf = AcInfo()
    _chk(_lib.ac_info_get(a, C.byref(inf)))
    out = dict(obs_dim=inf.obs_dim, critic_in=inf.critic_in, hidden=inf.hidden, batch=inf.batch,
               n_actor=inf.n_actor, n_critic=inf.n_critic, t_actor=inf.t_actor,
               t_critic=inf.t_critic, updates=inf.updates)
    for k in ("actor", "actor_t", "m_a", "v_a"):
        out[k] = view(getattr(inf, k), (inf.n_actor,))
    for k in ("c1", "c1_t", "c2", "c2_t", "m_c1", "v_c1", "m_c2", "v_c2"):
        out[k] = view(getattr(inf, k), (inf.n_critic,))
    out["stats"] = view(inf.stats, (4,))
    return out


def ac_set_counters(a, t_actor, t_critic, updates):
    _chk(_lib.ac_set_counters(a, t_actor, t_critic, updates))


def ac_update(a, env, n_updates, stream=None):
    _chk(_lib.ac_update(a, env, n_updates, _stream(stream)))


def ac_set_cluster(a, cluster) -> int:
    """Set the learner's cluster size (0 = automatic); returns the previous setting."""
    r = _lib.ac_set_cluster(a, int(cluster))
    if r < 0:
        _chk(r)
    return r


def ac_set_index_log(a, idx):
    """Log the replay indices of every update into ``idx`` (uint32/int32 cuda tensor of
    batch elements), or stop logging with ``None``."""
    if idx is not None:
        assert idx.is_cuda and idx.dtype in (torch.int32, torch.uint32) and idx.is_contiguous()
    _chk(_lib.ac_set_index_log(a, None if idx is None else idx.data_ptr()))


def ac_update_static(a, env, n_updates, stream=None):
    """ac_update without any device allocation (library-owned static scratch)."""
    _chk(_lib.ac_update_static(a, env, n_updates, _stream(stream)))


def ac_train(runs, envs, steps_per_run, persistent=1, stream=None):
    """persistent 1: all runs in one launch; 0: one launch per run and step (plain form);
    2: one launch per run for all of its steps, runs one after another."""
    n = len(runs)
    ra = (P * n)(*[r.value if isinstance(r, P) else r for r in runs])
    ea = (P * n)(*[e.value if isinstance(e, P) else e for e in envs])
    _chk(_lib.ac_train(C.cast(ra, P), C.cast(ea, P), n, steps_per_run, persistent,
                       _stream(stream)))


def ac_train_autotune(runs, envs, trial_steps=4, stream=None) -> int:
    """Time the persistent launch at every admissible cluster size; keep the fastest."""
    n = len(runs)
    ra = (P * n)(*[r.value if isinstance(r, P) else r for r in runs])
    ea = (P * n)(*[e.value if isinstance(e, P) else e for e in envs])
    r = _lib.ac_train_autotune(C.cast(ra, P), C.cast(ea, P), n, trial_steps, _stream(stream))
    if r < 0:
        _chk(r)
    return r


def ac_plan_create(runs, envs, steps_per_chunk):
    n = len(runs)
    ra = (P * n)(*[r.value if isinstance(r, P) else r for r in runs])
    ea = (P * n)(*[e.value if isinstance(e, P) else e for e in envs])
    p = P()
    _chk(_lib.ac_plan_create(C.cast(ra, P), C.cast(ea, P), n, steps_per_chunk, C.byref(p)))
    return p


def ac_plan_run(plan, n_chunks, stream=None):
    _chk(_lib.ac_plan_run(plan, n_chunks, _stream(stream)))


def ac_plan_sync(plan, stream=None):
    _chk(_lib.ac_plan_sync(plan, _stream(stream)))


def ac_plan_destroy(plan):
    if plan:
        _chk(_lib.ac_plan_destroy(plan))


def ac_sync(a):
    _chk(_lib.ac_sync(a))


def ac_save(a, env, path):
    _chk(_lib.ac_save(a, env, path.encode()))


def ac_load(a, env, path):
    _chk(_lib.ac_load(a, env, path.encode()))


def qsim_vjp_workspace(desc: QsimVjpDesc) -> int:
    load()
    return int(_lib.qsim_vjp_workspace(C.byref(desc)))


def qsim_rollout_vjp(desc: QsimVjpDesc, veh: QsimParams, s0, params, actions, actor, seed,
                     loss, g_actions, g_actor, g_params, actions_out, workspace, stream=None):
    load()
    _chk(_lib.qsim_rollout_vjp(C.byref(desc), C.byref(veh), _ptr(s0), _ptr(params),
                               _ptr(actions), _ptr(actor), _ptr(seed), _ptr(loss),
                               _ptr(g_actions), _ptr(g_actor), _ptr(g_params),
                               _ptr(actions_out), _ptr(workspace), _stream(stream)))


def param_count(inp: int, hid: int, out: int) -> int:
    return hid * inp + hid + hid * hid + hid + out * hid + out


def padded(n: int) -> int:
    return int(math.ceil(n / 32.0) * 32)
