"""Host logic of the multi-GPU replica path, run as two gloo ranks on the CPU.

The product shards by whole problems (one periodic box per rank, no data-path collective);
these tests cover what crosses ranks: distinct particle draws per rank, the barrier, the
maximum of the per-rank times and the whole-job rate formed from it.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2210_01837_gb300.replicas import Collective, rank_env, replica_seed_offset, whole_job_rate
from paper_2210_01837_gb300.workloads import rollers_1m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    env = rank_env()
    assert (env.rank, env.world, env.local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    coll = Collective(dist, "cpu")
    # a small replica workload; each rank draws its own suspension
    params, pos, F, T = rollers_1m(n=256, nxy=48, L=32.0, seed_offset=replica_seed_offset(rank))
    coll.barrier()
    t_local = 0.5 + rank  # stand-in elapsed times: rank 1 is the slow one
    t_max = coll.max(t_local)
    rate = whole_job_rate(world, 10, t_max)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), pos=pos, t_max=t_max, rate=rate)
    coll.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{i}.npz") for i in range(world)]
    # every rank saw the slowest rank's time and the same whole-job rate
    assert float(r[0]["t_max"]) == float(r[1]["t_max"]) == 1.5
    assert float(r[0]["rate"]) == float(r[1]["rate"]) == pytest.approx(world * 10 / 1.5)
    # replicas are different suspensions of the same shape
    assert r[0]["pos"].shape == r[1]["pos"].shape
    assert not np.array_equal(r[0]["pos"], r[1]["pos"])


def test_single_rank_defaults():
    env = rank_env({})
    assert (env.rank, env.world, env.local) == (0, 1, 0)
    c = Collective()
    c.barrier()
    assert c.max(2.5) == 2.5
    assert whole_job_rate(1, 4, 2.0) == 2.0
    assert replica_seed_offset(0) == 3 and replica_seed_offset(5) == 8


@pytest.mark.parametrize("bad", [(0, 1, 1.0), (1, -1, 1.0), (1, 1, 0.0)])
def test_whole_job_rate_rejects(bad):
    with pytest.raises(ValueError):
        whole_job_rate(*bad)
