"""ac_update_static -- the allocation-free learner update -- against ac_update.

Callers that cannot allocate device memory while they train (an embedded trainer with
all memory reserved up front, a custom allocator that forbids cudaMalloc) use
ac_update_static, whose scratch is a library-owned static device array.  Its results
must be those of ac_update on the same inputs; checked on two calls in a row (the second
call reuses the array left over from the first).  This file is collected last so that a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import cpu, lib_config

pytestmark = pytest.mark.gpu

NETS = ("actor", "actor_t", "c1", "c1_t", "c2", "c2_t", "m_a", "v_a", "m_c1", "v_c1", "m_c2",
        "v_c2")


def _setup(q, hidden, batch, cluster):
    d, cfg, veh = lib_config(q, "c1", n_envs=3, capacity=64, learning_starts=0, episode_len=12,
                             sig_p=0.003, sig_v=0.01)
    h = q.qsim_create(cfg, veh)
    hp = dict(W.TD3)
    hp.update(hidden=hidden, batch=batch)
    a = q.ac_create(q.make_ac_config(hp, cluster=cluster), h)
    ld = q.qsim_info_get(h)["ld"]
    for k in range(30):
        acts = torch.tensor(W.random_actions(900 + k, (4, ld)), dtype=torch.float32, device="cuda")
        q.qsim_step(h, acts)
    torch.cuda.synchronize()
    return h, a


@pytest.mark.parametrize("hidden,batch,cluster", [(64, 64, 2), (128, 128, 1), (64, 256, 0)])
def test_static_update_matches_ac_update(gpu, hidden, batch, cluster):
    """Both entry points launch the same kernel on the same cluster size, so the results
    are equal bit for bit (cluster 0: the automatic single-run size, 16 CTAs here)."""
    q = gpu
    h1, a1 = _setup(q, hidden, batch, cluster)
    h2, a2 = _setup(q, hidden, batch, cluster)
    try:
        for call in range(2):
            q.ac_update(a1, h1, 1)
            q.ac_update_static(a2, h2, 1)
            torch.cuda.synchronize()
            A1, A2 = q.ac_info_get(a1), q.ac_info_get(a2)
            assert A1["updates"] == A2["updates"] == call + 1
            assert A1["t_actor"] == A2["t_actor"] and A1["t_critic"] == A2["t_critic"]
            for k in NETS + ("stats",):
                x, y = cpu(A2[k]), cpu(A1[k])
                assert np.array_equal(x.view(np.uint32), y.view(np.uint32)), f"call{call}.{k}"
    finally:
        for a, h in ((a1, h1), (a2, h2)):
            q.ac_destroy(a)
            q.qsim_destroy(h)


def test_static_update_rejects_oversized_configuration(gpu):
    q = gpu
    # 4,096 envs x (obs + 2 hidden + 4) floats of env-step tile plus a 1,024-sample
    # batch at width 128 need more than the static maximum
    d, cfg, veh = lib_config(q, "c1", n_envs=4096, capacity=64, learning_starts=0)
    h = q.qsim_create(cfg, veh)
    hp = dict(W.TD3)
    hp.update(hidden=128, batch=1024)
    a = q.ac_create(q.make_ac_config(hp, cluster=1), h)
    try:
        ld = q.qsim_info_get(h)["ld"]
        for k in range(25):
            q.qsim_step(h, torch.zeros(4, ld, device="cuda"))
        with pytest.raises(q.QsimError, match="static maximum"):
            q.ac_update_static(a, h, 1)
    finally:
        q.ac_destroy(a)
        q.qsim_destroy(h)
