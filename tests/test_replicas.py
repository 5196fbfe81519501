"""Multi-process host logic of replica runs on CPU: two gloo ranks split a
job list, prove their shares independently (the oracle stands in for a
GPU), and reduce their timings with the same helpers bench.py uses."""
import json
import os
import socket

import numpy as np
import pytest

from paper_1202_1350_gb300 import replicas

torch = pytest.importorskip("torch")


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    import torch.distributed as dist

    import oracle
    from paper_1202_1350_gb300 import inputs as I

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = [(3 + k % 3, 100 + k) for k in range(7)]
    mine = replicas.shard(jobs, rank, world)
    done = []
    for logn, seed in mine:
        c = oracle.Circuit(*oracle.f2_layers(logn))
        x = I.f2_inputs(logn, 1 << 16, replicas.replica_seed(seed, rank))
        tr = c.prove(x, seed)
        ok, _ = c.verify(x, seed, tr)
        done.append([logn, seed, bool(ok)])
    # a rank's "elapsed time"; the job's time is the slowest rank's
    t_max = replicas.max_over_ranks(1.0 + rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, done)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"t_max": t_max, "all": gathered}, f)


def test_two_gloo_ranks_split_jobs_and_reduce_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["t_max"] == float(world)  # max over ranks of 1.0 + rank
        seeds = sorted(s for part in r["all"] for _, s, _ in part)
        assert seeds == list(range(100, 107))  # every job proved exactly once
        assert all(ok for part in r["all"] for _, _, ok in part)
    assert replicas.whole_job_rate(10.0, world, 2.0) == 10.0


def test_shard_properties():
    jobs = list(range(11))
    parts = [replicas.shard(jobs, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == jobs
    assert all(abs(len(p) - len(jobs) / 3) < 1 for p in parts)
    with pytest.raises(ValueError):
        replicas.shard(jobs, 3, 3)
    assert replicas.replica_seed(7, 0) != replicas.replica_seed(7, 1)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert np.isclose(replicas.whole_job_rate(5.0, 4, 2.0), 10.0)
