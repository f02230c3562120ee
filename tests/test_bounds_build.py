"""The debug variant of the library with device-side bounds checks of replay-ring slots and
SoA env indices (built with -DQSIM_BOUNDS_CHECK=1).

CPU: both variants build, export every declared symbol and report which one they are.
GPU (each case in a child process, since one process loads one variant): on valid inputs
the checked build reports no violation and gives results bitwise equal to the default
build (rollouts on both engines, env steps, learner updates with replay gathers, reward
recalculation); an out-of-range index given to the probe, whose only access is behind the
check, is reported with its site, index and bound, and the status is clean afterwards."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from test_abi import declared_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_both_variants_export_every_symbol_and_say_which_they_are():
    from paper_2311_13081_gb300 import build as b
    for checked in (False, True):
        lib = ctypes.CDLL(b.build(bounds_check=checked))
        missing = [n for n in declared_functions() if not hasattr(lib, n)]
        assert not missing, missing
        assert lib.qsim_bounds_checked() == (1 if checked else 0)


# Child program: runs a fixed seeded workload through the library at argv[1] and writes
# the results (and, for the checked build, the probe outcomes) to argv[2].
_CHILD = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import paper_2311_13081_gb300 as q
import workloads as W

q.load(sys.argv[1])
out = {"checked": q.qsim_bounds_checked()}
res = {}
d = W.config("c2")
d.update(learning_starts=0)
n = 200
h = q.qsim_create(q.make_config(d, n, 48, reward=W.REWARD, sigma_e=0.1), q.make_params(d))
hp = dict(W.TD3)
hp.update(hidden=64, batch=64)
a = q.ac_create(q.make_ac_config(hp, cluster=2), h)
ai = q.ac_info_get(a)
for engine in (2, 1):
    q.qsim_rollout_engine(h, engine)
    q.qsim_rollout(h, ai["actor"], 64, 30, 0.1)
acts = torch.zeros(4, q.qsim_info_get(h)["state"].shape[1], device="cuda")
q.qsim_step(h, acts)
q.ac_train([a], [h], 25, persistent=1)
q.ac_update(a, h, 3)
q.qsim_recalc_rewards(h)
torch.cuda.synchronize()
q.qsim_sync(h)
info = q.qsim_info_get(h)
for k in ("state", "records", "side"):
    if k in info:
        res[k] = info[k].float().cpu().numpy().view(np.uint32).tolist()
ai = q.ac_info_get(a)
for k in ("actor", "c1", "c2"):
    res[k] = ai[k].float().cpu().numpy().view(np.uint32).tolist()
out["results"] = res
if out["checked"]:
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    q.qsim_bounds_probe(h, 5, 7, flag)
    torch.cuda.synchronize()
    q.qsim_sync(h)
    msgs = []
    for slot, env in ((48, 0), (-1, 3), (0, 1 << 20)):
        q.qsim_bounds_probe(h, slot, env, flag)
        torch.cuda.synchronize()
        try:
            q.qsim_sync(h)
            msgs.append("")
        except q.QsimError as e:
            msgs.append(str(e))
    q.qsim_sync(h)  # reset by the read above
    out["probe"] = msgs
else:
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    try:
        q.qsim_bounds_probe(h, 48, 0, flag)
        out["refused"] = False
    except q.QsimError as e:
        out["refused"] = "outside the ring" in str(e)
json.dump(out, open(sys.argv[2], "w"))
'''


def _run_child(lib, path):
    code = "ROOT = " + repr(ROOT) + "\n" + _CHILD
    r = subprocess.run([sys.executable, "-c", code, lib, path], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.load(open(path))


@pytest.mark.gpu
def test_checked_build_matches_default_and_reports_violations(tmp_path):
    from paper_2311_13081_gb300 import build as b
    plain = _run_child(b.build(), str(tmp_path / "plain.json"))
    checked = _run_child(b.build(bounds_check=True), str(tmp_path / "checked.json"))
    assert plain["checked"] == 0 and checked["checked"] == 1
    # the default build refuses an out-of-range probe on the host
    assert plain["refused"] is True
    # no false positive, and the checks change no result
    assert plain["results"].keys() == checked["results"].keys()
    for k in plain["results"]:
        assert np.array_equal(np.array(plain["results"][k]), np.array(checked["results"][k])), k
    m = checked["probe"]
    assert "probe slot 48 outside [0, 48)" in m[0], m
    assert "probe slot -1 outside [0, 48)" in m[1], m
    assert "SoA env index 1048576 outside [0, 224)" in m[2], m
