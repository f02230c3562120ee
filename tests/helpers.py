"""Shared test helpers: conversions between the library's field-major device arrays and
the oracle's array-of-structs, and the tolerance rule used by every parity test.

Tolerance (FP32 result vs FP64 oracle on the same FP32 inputs): element-wise
    |x_gpu - x_ref| <= RTOL * |x_ref| + atol_field
with RTOL = 1e-4 and atol_field = 1e-4 x the field's typical scale (position 0.2 m,
velocity 1 m/s, rates 1 rad/s, quaternion / rotation entries 1, motor speed 1e4 rpm,
reward 1, Q-value 10), and the norm-wise rule ||x_gpu - x_ref|| / ||x_ref|| <= 1e-4 for
vectors of gradients.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
import workloads as W

RTOL = 1e-4
STATE_SCALE = np.array([0.2] * 3 + [1.0] * 4 + [1.0] * 3 + [1.0] * 3 + [1e4] * 4)


def assert_close(gpu, ref, scale=1.0, rtol=RTOL, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    atol = 1e-4 * np.asarray(scale, dtype=np.float64)
    err = np.abs(gpu - ref)
    lim = rtol * np.abs(ref) + atol
    bad = err > lim
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} elements out of tolerance; "
                             f"first at {tuple(i)}: gpu={gpu[tuple(i)]!r} ref={ref[tuple(i)]!r}")


def assert_norm_close(gpu, ref, tol=1e-4, what=""):
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    n = np.linalg.norm(ref)
    d = np.linalg.norm(gpu - ref)
    assert d <= tol * max(n, 1e-30), f"{what}: relative norm error {d / max(n, 1e-30):.3e}"


def cpu(t):
    return t.detach().cpu().numpy()


def f64(t):
    return cpu(t).astype(np.float64)


def u32(t):
    return cpu(t).view(np.uint32) if t.dtype == torch.int32 else cpu(t).astype(np.uint32)


def lib_config(q, preset="c1", n_envs=1, capacity=0, sigma_e=0.1, curriculum=None, **over):
    d = W.config(preset)
    d.update(over)
    cfg = q.make_config(d, n_envs, capacity, reward=W.REWARD, sigma_e=sigma_e,
                        curriculum=curriculum)
    return d, cfg, q.make_params(d)


def oracle_envs(info: dict, ids) -> dict:
    """Oracle env set mirroring GPU envs ``ids`` (FP32 values promoted to FP64)."""
    ids = np.asarray(ids)
    st = f64(info["state"])[:, ids].T.copy()
    prm = f64(info["params"])[:, ids].T.copy()
    dist = f64(info["dist"])[:, ids].T.copy()
    hist = f64(info["hist"])[:, ids].T.copy()
    return dict(env_id=ids.astype(np.uint32), s=st, prm=prm, dist=dist, hist=hist,
                ep_index=u32(info["ep_index"])[ids].copy(), ep_step=u32(info["ep_step"])[ids].copy(),
                ep_ret=f64(info["ep_ret"])[ids].copy(), n_done=u32(info["n_done"])[ids].copy(),
                len_sum=u32(info["len_sum"])[ids].copy(), ret_sum=f64(info["ret_sum"])[ids].copy())


def gpu_records(info: dict, slots, ids):
    """Records at ring slots ``slots`` for envs ``ids`` as oracle-shaped arrays."""
    rec = f64(info["records"])  # [cap][F][ld]
    raw = cpu(info["records"]).view(np.uint32)
    side = f64(info["side"])
    slots = np.asarray(slots)
    ids = np.asarray(ids)
    R = rec[slots][:, :, ids]  # [T][F][n]
    out = dict(rec_s=R[:, 0:17].transpose(0, 2, 1), rec_a=R[:, 17:21].transpose(0, 2, 1),
               rec_r=R[:, 21], rec_flags=raw[slots][:, 22][:, ids],
               side=side[slots][:, :, ids].transpose(0, 2, 1))
    if info["n_priv"]:
        out["rec_priv"] = R[:, 23:29].transpose(0, 2, 1)
    return out


def compare_records(g, o, what="records"):
    """Flags bit-exact (termination reported separately if s' sits on the box edge)."""
    assert_close(g["rec_s"], o["rec_s"], STATE_SCALE, what=what + ".s")
    assert_close(g["rec_a"], o["rec_a"], 1.0, what=what + ".a")
    assert_close(g["rec_r"], o["rec_r"], 1.0, what=what + ".r")
    gf, of = np.asarray(g["rec_flags"]), np.asarray(o["rec_flags"])
    mism = gf != of
    if mism.any():
        raise AssertionError(f"{what}.flags: {mism.sum()} mismatches, e.g. gpu={gf[mism][:4]} "
                             f"ref={of[mism][:4]}")
    done = (of & 3) != 0
    if done.any():
        assert_close(g["side"][done], o["side"][done], STATE_SCALE, what=what + ".side")
    if "rec_priv" in g:
        assert_close(g["rec_priv"], o["rec_priv"], 1.0, what=what + ".priv")
