"""FP64 CPU oracle for the quadrotor training hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product library never does: it shares no code, header,
table or helper with this oracle.

The arithmetic lives in ``qsim_oracle.c`` (plain C, double precision, built with
``-O2`` and without ``-ffast-math``).  This module only marshals numpy arrays.
Layouts here are array-of-structs (``[env][field]``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libqsim_oracle.so")
_lib = None

NS, NPRM, NDIST, NPRIV, HMAX = 17, 8, 6, 6, 16
CRITIC_HIST, CRITIC_PRIV, CRITIC_PAPER28 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math).  Returns the .so path."""
    src = os.path.join(_HERE, "qsim_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "qsim_oracle.h"))):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, _SO)
    return _SO


class Cfg(C.Structure):
    _fields_ = [
        ("mass", C.c_double), ("Jx", C.c_double), ("Jy", C.c_double), ("Jz", C.c_double),
        ("kf", C.c_double), ("km", C.c_double), ("tm", C.c_double),
        ("rotor_pos", C.c_double * 12), ("rotor_dir", C.c_double * 4),
        ("rpm_min", C.c_double), ("rpm_max", C.c_double), ("g", C.c_double),
        ("dt", C.c_double),
        ("renorm_q", C.c_int32), ("n_hist", C.c_int32), ("episode_len", C.c_int32),
        ("critic_layout", C.c_int32),
        ("init_p", C.c_double), ("init_att", C.c_double), ("init_v", C.c_double),
        ("init_w", C.c_double), ("init_rpm_lo", C.c_double), ("init_rpm_hi", C.c_double),
        ("dr_mass", C.c_double), ("dr_J", C.c_double), ("dr_kf", C.c_double),
        ("tm_lo", C.c_double), ("tm_hi", C.c_double),
        ("dist_f", C.c_double), ("dist_tau", C.c_double),
        ("sig_p", C.c_double), ("sig_R", C.c_double), ("sig_v", C.c_double),
        ("sig_w", C.c_double),
        ("term_pos", C.c_double),
        ("seed", C.c_uint64), ("run_id", C.c_uint32), ("learning_starts", C.c_int32),
        ("motor_lag_off", C.c_int32), ("pad_", C.c_int32),
    ]


class RewardC(C.Structure):
    _fields_ = [("c", C.c_double * 7)]


_P = C.c_void_p


class Envs(C.Structure):
    _fields_ = [("n", C.c_int32), ("env_id", _P), ("s", _P), ("prm", _P), ("dist", _P),
                ("hist", _P), ("ep_index", _P), ("ep_step", _P), ("ep_ret", _P),
                ("n_done", _P), ("len_sum", _P), ("ret_sum", _P)]


class RollOut(C.Structure):
    _fields_ = [("rec_s", _P), ("rec_a", _P), ("rec_r", _P), ("rec_flags", _P),
                ("rec_priv", _P), ("side", _P), ("mu", _P), ("obs", _P)]


class Net(C.Structure):
    _fields_ = [("in_", C.c_int32), ("hid", C.c_int32), ("out", C.c_int32)]


class TD3(C.Structure):
    _fields_ = [("gamma", C.c_double), ("tau", C.c_double), ("lr", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("sigma_t", C.c_double), ("noise_clip", C.c_double),
                ("policy_delay", C.c_int32), ("batch", C.c_int32), ("hidden", C.c_int32),
                ("pad_", C.c_int32),
                ("actor", _P), ("actor_t", _P), ("c1", _P), ("c1_t", _P), ("c2", _P),
                ("c2_t", _P), ("m_a", _P), ("v_a", _P), ("m_c1", _P), ("v_c1", _P),
                ("m_c2", _P), ("v_c2", _P),
                ("t_a", C.c_int64), ("t_c", C.c_int64), ("update_idx", C.c_int64)]


class Buffer(C.Structure):
    _fields_ = [("n_env", C.c_int32), ("capacity", C.c_int32), ("s", _P), ("a", _P),
                ("r", _P), ("flags", _P), ("priv", _P), ("side", _P),
                ("head", C.c_int64), ("size", C.c_int64), ("t_now", C.c_int64)]


class TD3Diag(C.Structure):
    _fields_ = [("idx", _P), ("y", _P), ("q1", _P), ("q2", _P), ("a2", _P), ("oa", _P),
                ("oa2", _P), ("oc", _P), ("oc2", _P), ("g_c1", _P),
                ("g_c2", _P), ("g_a", _P), ("critic_loss", C.c_double),
                ("actor_loss", C.c_double), ("actor_updated", C.c_int32), ("pad_", C.c_int32)]


class Diff(C.Structure):
    _fields_ = [("n", C.c_int32), ("H", C.c_int32), ("mode", C.c_int32), ("n_hist", C.c_int32),
                ("w_p", C.c_double), ("w_q", C.c_double), ("w_v", C.c_double),
                ("w_a", C.c_double), ("s0", _P), ("prm", _P), ("actions", _P), ("actor", _P),
                ("hidden", C.c_int32), ("pad_", C.c_int32),
                ("loss", _P), ("g_actions", _P), ("g_actor", _P), ("g_prm", _P), ("traj", _P),
                ("act_out", _P)]


class Track(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_steps", C.c_int32), ("hidden", C.c_int32),
                ("pad_", C.c_int32), ("prm", _P), ("dist", _P), ("period", _P), ("actor", _P),
                ("amp", C.c_double), ("z0", C.c_double), ("clip_p", C.c_double),
                ("clip_v", C.c_double), ("sq_err", _P), ("steps_ok", _P), ("traj", _P)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_uniform.restype = C.c_double
        L.or_uniform.argtypes = [C.c_uint32]
        L.or_gauss.restype = C.c_double
        L.or_gauss.argtypes = [C.c_uint32, C.c_uint32]
        L.or_replay_index.restype = C.c_uint32
        L.or_replay_index.argtypes = [C.c_uint32, C.c_uint32]
        L.or_reward.restype = C.c_double
        L.or_reward.argtypes = [C.POINTER(RewardC), _P, _P]
        for fn in ("or_net_size", "or_actor_in", "or_critic_in", "or_rollout", "or_td3_update",
                   "or_recalc_rewards", "or_diff_run", "or_track_run"):
            getattr(L, fn).restype = C.c_int
        L.or_net_size.argtypes = [C.c_int, C.c_int, C.c_int]
        L.or_actor_in.argtypes = [C.POINTER(Cfg)]
        L.or_critic_in.argtypes = [C.POINTER(Cfg)]
        L.or_rk4.argtypes = [C.POINTER(Cfg), _P, _P, _P, _P, C.c_double, C.c_int, _P]
        L.or_deriv.argtypes = [C.POINTER(Cfg), _P, _P, _P, _P, _P]
        L.or_dynamics_batch.argtypes = [C.POINTER(Cfg), C.c_int, _P, _P, _P, _P, C.c_double,
                                        C.c_int, C.c_int, _P]
        L.or_reset_env.argtypes = [C.POINTER(Cfg), C.c_uint32, C.c_uint32, _P, _P, _P]
        L.or_obs_noise.argtypes = [C.POINTER(Cfg), C.c_uint32, C.c_uint64, _P]
        L.or_obs_actor.argtypes = [C.POINTER(Cfg), _P, _P, _P, _P]
        L.or_obs_critic.argtypes = [C.POINTER(Cfg), _P, _P, _P, _P]
        L.or_priv.argtypes = [C.POINTER(Cfg), _P, _P, _P]
        L.or_mlp_forward.argtypes = [C.POINTER(Net), _P, _P, _P, _P, _P, C.c_int]
        L.or_init_params.argtypes = [C.POINTER(Cfg), C.c_int, C.c_int, C.c_int, C.c_int, _P]
        L.or_rollout.argtypes = [C.POINTER(Cfg), C.POINTER(RewardC), C.POINTER(Envs), _P,
                                 C.c_int, C.c_int, C.c_uint64, C.c_double, _P,
                                 C.POINTER(RollOut), C.c_int]
        L.or_td3_update.argtypes = [C.POINTER(Cfg), C.POINTER(TD3), C.POINTER(Buffer),
                                    C.POINTER(TD3Diag)]
        L.or_recalc_rewards.argtypes = [C.POINTER(RewardC), C.POINTER(Buffer), _P]
        L.or_curriculum.argtypes = [_P, _P, _P, C.c_int]
        L.or_diff_run.argtypes = [C.POINTER(Cfg), C.POINTER(Diff)]
        L.or_lissajous.restype = None
        L.or_lissajous.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _P, _P]
        L.or_track_run.argtypes = [C.POINTER(Cfg), C.POINTER(Track), C.c_int]
        L.or_philox.argtypes = [_P, _P, _P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_cfg(d: dict) -> Cfg:
    c = Cfg()
    for name, _ in Cfg._fields_:
        if name in d:
            v = d[name]
            if name in ("rotor_pos", "rotor_dir"):
                arr = getattr(c, name)
                for i, x in enumerate(np.asarray(v, dtype=np.float64).ravel()):
                    arr[i] = float(x)
            else:
                setattr(c, name, v)
    return c


def reward_c(vals) -> RewardC:
    r = RewardC()
    for i, x in enumerate(vals):
        r.c[i] = float(x)
    return r


# ---------------------------------------------------------------------------------------
# Small primitives
# ---------------------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_p(c), _p(k), _p(o))
    return o


def uniform(x: int) -> float:
    return lib().or_uniform(int(x) & 0xFFFFFFFF)


def gauss(x1: int, x2: int) -> float:
    return lib().or_gauss(int(x1) & 0xFFFFFFFF, int(x2) & 0xFFFFFFFF)


def replay_index(x: int, n: int) -> int:
    return lib().or_replay_index(int(x) & 0xFFFFFFFF, int(n) & 0xFFFFFFFF)


def net_size(i, h, o) -> int:
    return lib().or_net_size(i, h, o)


def actor_in(cfg) -> int:
    return lib().or_actor_in(C.byref(make_cfg(cfg)))


def critic_in(cfg) -> int:
    return lib().or_critic_in(C.byref(make_cfg(cfg)))


def deriv(cfg, s, u, prm, dist=None):
    s, u, prm = _f64(s, (NS,)), _f64(u, (4,)), _f64(prm, (NPRM,))
    dist = _f64(np.zeros(NDIST) if dist is None else dist, (NDIST,))
    ds = np.zeros(NS)
    lib().or_deriv(C.byref(make_cfg(cfg)), _p(s), _p(u), _p(prm), _p(dist), _p(ds))
    return ds


def rk4(cfg, s, u, prm, dist=None, dt=None, renorm=None):
    c = make_cfg(cfg)
    s, u, prm = _f64(s, (NS,)), _f64(u, (4,)), _f64(prm, (NPRM,))
    dist = _f64(np.zeros(NDIST) if dist is None else dist, (NDIST,))
    out = np.zeros(NS)
    lib().or_rk4(C.byref(c), _p(s), _p(u), _p(prm), _p(dist),
                 c.dt if dt is None else float(dt), c.renorm_q if renorm is None else int(renorm),
                 _p(out))
    return out


def dynamics_batch(cfg, s, u, prm, dist=None, dt=None, renorm=None, n_steps=1):
    """[n][17] states, [n][4] held RPM set-points, [n][8] params -> [n][17] after n_steps."""
    c = make_cfg(cfg)
    s = _f64(s)
    n = s.shape[0]
    u, prm = _f64(u, (n, 4)), _f64(prm, (n, NPRM))
    dist = _f64(np.zeros((n, NDIST)) if dist is None else dist, (n, NDIST))
    out = np.zeros((n, NS))
    lib().or_dynamics_batch(C.byref(c), n, _p(s), _p(u), _p(prm), _p(dist),
                            c.dt if dt is None else float(dt),
                            c.renorm_q if renorm is None else int(renorm), int(n_steps), _p(out))
    return out


def reset_env(cfg, env: int, episode: int):
    s, prm, dist = np.zeros(NS), np.zeros(NPRM), np.zeros(NDIST)
    lib().or_reset_env(C.byref(make_cfg(cfg)), env, episode, _p(s), _p(prm), _p(dist))
    return s, prm, dist


def obs_noise(cfg, env: int, t: int):
    o = np.zeros(18)
    lib().or_obs_noise(C.byref(make_cfg(cfg)), env, t, _p(o))
    return o


def obs_actor(cfg, s, hist, noise=None):
    c = make_cfg(cfg)
    o = np.zeros(18 + 4 * c.n_hist)
    s, hist = _f64(s, (NS,)), _f64(hist, (4 * HMAX,))
    nz = None if noise is None else _f64(noise, (18,))
    lib().or_obs_actor(C.byref(c), _p(s), _p(hist), _p(nz), _p(o))
    return o


def priv(cfg, prm, dist):
    out = np.zeros(NPRIV)
    lib().or_priv(C.byref(make_cfg(cfg)), _p(_f64(prm, (NPRM,))), _p(_f64(dist, (NDIST,))),
                  _p(out))
    return out


def obs_critic(cfg, s, hist, pv):
    c = make_cfg(cfg)
    o = np.zeros(lib().or_critic_in(C.byref(c)) - 4)
    lib().or_obs_critic(C.byref(c), _p(_f64(s, (NS,))), _p(_f64(hist, (4 * HMAX,))),
                        _p(_f64(pv, (NPRIV,))), _p(o))
    return o


def reward(Cvals, s, a) -> float:
    rc = reward_c(Cvals)
    return lib().or_reward(C.byref(rc), _p(_f64(s, (NS,))), _p(_f64(a, (4,))))


def mlp_forward(P, x, inp, hid, out, tanh_out):
    net = Net(inp, hid, out)
    P, x = _f64(P), _f64(x, (inp,))
    h1, h2, y = np.zeros(hid), np.zeros(hid), np.zeros(out)
    lib().or_mlp_forward(C.byref(net), _p(P), _p(x), _p(h1), _p(h2), _p(y), int(tanh_out))
    return y, h1, h2


def init_params(cfg, net_id, inp, hid, out):
    P = np.zeros(net_size(inp, hid, out))
    lib().or_init_params(C.byref(make_cfg(cfg)), net_id, inp, hid, out, _p(P))
    return P


# ---------------------------------------------------------------------------------------
# Environment sets and rollouts
# ---------------------------------------------------------------------------------------
def new_envs(cfg, env_ids) -> dict:
    """Fresh env set: every env reset to episode 0 (state, params, disturbance, history)."""
    ids = np.ascontiguousarray(env_ids, dtype=np.uint32)
    n = ids.size
    e = dict(env_id=ids, s=np.zeros((n, NS)), prm=np.zeros((n, NPRM)),
             dist=np.zeros((n, NDIST)), hist=np.zeros((n, 4 * HMAX)),
             ep_index=np.zeros(n, np.uint32), ep_step=np.zeros(n, np.uint32),
             ep_ret=np.zeros(n), n_done=np.zeros(n, np.uint32), len_sum=np.zeros(n, np.uint32),
             ret_sum=np.zeros(n))
    for k in range(n):
        e["s"][k], e["prm"][k], e["dist"][k] = reset_env(cfg, int(ids[k]), 0)
    return e


def _envs_struct(e):
    for k in ("s", "prm", "dist", "hist", "ep_ret", "ret_sum"):
        e[k] = np.ascontiguousarray(e[k], dtype=np.float64)
    for k in ("env_id", "ep_index", "ep_step", "n_done", "len_sum"):
        e[k] = np.ascontiguousarray(e[k], dtype=np.uint32)
    return Envs(int(e["env_id"].size), _p(e["env_id"]), _p(e["s"]), _p(e["prm"]), _p(e["dist"]),
                _p(e["hist"]), _p(e["ep_index"]), _p(e["ep_step"]), _p(e["ep_ret"]),
                _p(e["n_done"]), _p(e["len_sum"]), _p(e["ret_sum"]))


def rollout(cfg, Cvals, e: dict, T: int, t0: int, actor=None, hidden=64, sigma_e=0.0,
            ext_actions=None, n_threads=1, obs=False) -> dict:
    """Advance env set ``e`` (modified in place) by T steps starting at global step t0.

    ``ext_actions`` ([T][n][4], normalised) replaces the actor, warm-up and exploration.
    Returns the transition records ([T][n][...]) and the side slots; with ``obs`` also the
    actor observation of every step ([T][n][18 + 4 n_hist], noise included).
    """
    c = make_cfg(cfg)
    st = _envs_struct(e)
    n = st.n
    out = dict(rec_s=np.zeros((T, n, NS)), rec_a=np.zeros((T, n, 4)), rec_r=np.zeros((T, n)),
               rec_flags=np.zeros((T, n), np.uint32), rec_priv=np.zeros((T, n, NPRIV)),
               side=np.full((T, n, NS), np.nan), mu=np.zeros((T, n, 4)))
    if obs:
        out["obs"] = np.zeros((T, n, 18 + 4 * c.n_hist))
    ro = RollOut(*[_p(out.get(k)) for k in ("rec_s", "rec_a", "rec_r", "rec_flags", "rec_priv",
                                            "side", "mu", "obs")])
    act = None if actor is None else _f64(actor)
    ext = None if ext_actions is None else _f64(ext_actions, (T, n, 4))
    rc = reward_c(Cvals)
    lib().or_rollout(C.byref(c), C.byref(rc), C.byref(st), _p(act), int(hidden), int(T),
                     int(t0), float(sigma_e), _p(ext), C.byref(ro), int(n_threads))
    return out


# ---------------------------------------------------------------------------------------
# Learner
# ---------------------------------------------------------------------------------------
def td3_update(cfg, hyper: dict, L: dict, buf: dict, diag: bool = True) -> dict:
    """One TD3 update.  ``L`` holds float64 arrays actor, actor_t, c1, c1_t, c2, c2_t, m_*,
    v_* and ints t_a, t_c, update_idx (all modified in place).  ``buf`` holds the replay
    arrays s [C][n][17], a, r, flags, priv, side and ints head, size, t_now."""
    c = make_cfg(cfg)
    B, H = int(hyper["batch"]), int(hyper["hidden"])
    for k in ("actor", "actor_t", "c1", "c1_t", "c2", "c2_t", "m_a", "v_a", "m_c1", "v_c1",
              "m_c2", "v_c2"):
        L[k] = np.ascontiguousarray(L[k], dtype=np.float64)
    td = TD3(hyper["gamma"], hyper["tau"], hyper["lr"], hyper["beta1"], hyper["beta2"],
             hyper["eps"], hyper["sigma_t"], hyper["noise_clip"], int(hyper["policy_delay"]),
             B, H, 0, *[_p(L[k]) for k in ("actor", "actor_t", "c1", "c1_t", "c2", "c2_t",
                                           "m_a", "v_a", "m_c1", "v_c1", "m_c2", "v_c2")],
             int(L["t_a"]), int(L["t_c"]), int(L["update_idx"]))
    for k in ("s", "a", "r", "priv", "side"):
        buf[k] = np.ascontiguousarray(buf[k], dtype=np.float64)
    buf["flags"] = np.ascontiguousarray(buf["flags"], dtype=np.uint32)
    capn = buf["s"].shape
    bs = Buffer(int(capn[1]), int(capn[0]), _p(buf["s"]), _p(buf["a"]), _p(buf["r"]),
                _p(buf["flags"]), _p(buf["priv"]), _p(buf["side"]), int(buf["head"]),
                int(buf["size"]), int(buf["t_now"]))
    PA = L["actor"].size
    PC = L["c1"].size
    DA, DC = lib().or_actor_in(C.byref(c)), lib().or_critic_in(C.byref(c))
    dg = dict(idx=np.zeros(B, np.uint32), y=np.zeros(B), q1=np.zeros(B), q2=np.zeros(B),
              a2=np.zeros((B, 4)), oa=np.zeros((B, DA)), oa2=np.zeros((B, DA)),
              oc=np.zeros((B, DC)), oc2=np.zeros((B, DC)), g_c1=np.zeros(PC),
              g_c2=np.zeros(PC), g_a=np.zeros(PA))
    ds = TD3Diag(*[_p(dg[k]) for k in ("idx", "y", "q1", "q2", "a2", "oa", "oa2", "oc", "oc2",
                                       "g_c1", "g_c2", "g_a")],
                 0.0, 0.0, 0, 0)
    rc = lib().or_td3_update(C.byref(c), C.byref(td), C.byref(bs), C.byref(ds))
    if rc != 0:
        raise ValueError("oracle td3_update: replay buffer too small to sample")
    L["t_a"], L["t_c"], L["update_idx"] = td.t_a, td.t_c, td.update_idx
    dg.update(critic_loss=ds.critic_loss, actor_loss=ds.actor_loss,
              actor_updated=bool(ds.actor_updated))
    return dg


def recalc_rewards(Cvals, buf: dict, cur_state) -> None:
    rc = reward_c(Cvals)
    for k in ("s", "a", "r", "priv", "side"):
        buf[k] = np.ascontiguousarray(buf[k], dtype=np.float64)
    buf["flags"] = np.ascontiguousarray(buf["flags"], dtype=np.uint32)
    capn = buf["s"].shape
    bs = Buffer(int(capn[1]), int(capn[0]), _p(buf["s"]), _p(buf["a"]), _p(buf["r"]),
                _p(buf["flags"]), _p(buf["priv"]), _p(buf["side"]), int(buf["head"]),
                int(buf["size"]), int(buf["t_now"]))
    cs = _f64(cur_state, (capn[1], NS))
    lib().or_recalc_rewards(C.byref(rc), C.byref(bs), _p(cs))


def curriculum(factor, target, Cvals):
    f, t = _f64(factor), _f64(target)
    Cv = _f64(Cvals).copy()
    lib().or_curriculum(_p(f), _p(t), _p(Cv), int(Cv.size))
    return Cv


# ---------------------------------------------------------------------------------------
# Differentiation
# ---------------------------------------------------------------------------------------
def diff_run(cfg, s0, prm, H, weights, mode=0, actions=None, actor=None, hidden=64,
             n_hist=16) -> dict:
    c = make_cfg(cfg)
    s0 = _f64(s0)
    n = s0.shape[0]
    prm = _f64(prm, (n, NPRM))
    da = 18 + 4 * n_hist
    pa = net_size(da, hidden, 4)
    out = dict(loss=np.zeros(n), g_actions=np.zeros((n, H, 4)), g_actor=np.zeros(pa),
               g_prm=np.zeros((n, NPRM)), traj=np.zeros((n, H + 1, NS)),
               act_out=np.zeros((n, H, 4)))
    act = None if actions is None else _f64(actions, (n, H, 4))
    aw = None if actor is None else _f64(actor)
    d = Diff(n, int(H), int(mode), int(n_hist), float(weights[0]), float(weights[1]),
             float(weights[2]), float(weights[3]), _p(s0), _p(prm), _p(act), _p(aw),
             int(hidden), 0, _p(out["loss"]), _p(out["g_actions"]), _p(out["g_actor"]),
             _p(out["g_prm"]), _p(out["traj"]), _p(out["act_out"]))
    lib().or_diff_run(C.byref(c), C.byref(d))
    return out


# ---------------------------------------------------------------------------------------
# Simulated trajectory tracking (Sec. V)
# ---------------------------------------------------------------------------------------
def lissajous(t: float, T: float, A: float = 1.0, z0: float = 0.0):
    """Figure-eight target of Sec. V and its velocity at time t (s), cycle time T (s)."""
    p, v = np.zeros(3), np.zeros(3)
    lib().or_lissajous(float(t), float(T), float(A), float(z0), _p(p), _p(v))
    return p, v


def track(cfg, prm, dist, period, actor, hidden, n_steps, amp=1.0, z0=0.0, clip_p=0.2,
          clip_v=1.0, traj=False, n_threads=1) -> dict:
    """Fly n envs (params ``prm`` [n][8], disturbances ``dist`` [n][6]) along the target.

    Returns sq_err [n][2] (sums of |e|^2 and e_x^2 + e_y^2 over the completed steps),
    steps_ok [n] and, if requested, the states traj [n][n_steps + 1][17]."""
    c = make_cfg(cfg)
    prm = _f64(prm)
    n = prm.shape[0]
    dist = _f64(dist, (n, NDIST))
    per = _f64(period, (n,))
    aw = _f64(actor)
    out = dict(sq_err=np.zeros((n, 2)), steps_ok=np.zeros(n, np.int32),
               traj=np.full((n, n_steps + 1, NS), np.nan) if traj else None)
    J = Track(n, int(n_steps), int(hidden), 0, _p(prm), _p(dist), _p(per), _p(aw), float(amp),
              float(z0), float(clip_p), float(clip_v), _p(out["sq_err"]), _p(out["steps_ok"]),
              _p(out["traj"]))
    lib().or_track_run(C.byref(c), C.byref(J), int(n_threads))
    return out
