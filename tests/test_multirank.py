"""The bench's N>1 host logic on CPU ranks (gloo, world size 2): each rank's workload is its
own independent env set, and the only collective -- the max of the per-rank time -- gives
every rank the same value."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle as O
import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.0 + 0.5 * rank  # a per-rank time
        out[rank] = bench.max_over_ranks(torch, dist, t, world, "cpu")
        d = bench.rank_workload(W, rank)
        # the first reset of envs 0..7 of this rank (the oracle's Philox streams)
        st = np.stack([O.reset_env(d, e, 0)[0] for e in range(8)])
        out[world + rank] = float(np.abs(st).sum())
        out[2 * world + rank] = float(d["run_id"])
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_cpu():
    world = 2
    out = mp.get_context("spawn").Array("d", 3 * world)
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert list(out[:world]) == [1.5, 1.5]          # max over ranks, on every rank
    assert out[2 * world:] == [0.0, 1.0]            # run id = rank
    assert out[world] != out[world + 1]             # independent env sets per rank


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(torch, None, 2.5, 1, "cpu") == 2.5
