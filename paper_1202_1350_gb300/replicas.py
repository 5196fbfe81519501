"""Host logic of multi-GPU runs: independent replicas, one process per GPU.

Proofs share nothing, so N GPUs run N independent provers: each rank proves
its own instances (its own inputs and seeds), the only collective is the
timing reduction (barrier, then the maximum of the ranks' elapsed times), and
whole-job throughput is the work of all ranks over that maximum.  Job lists
(batches, serving traces) are split across ranks round-robin.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, local_rank, world_size) from the torch.distributed launcher's
    environment (1 process when unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(jobs, rank: int, world: int):
    """This rank's share of a job list: every world-th job from position rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(jobs)[rank::world]


def replica_seed(seed0: int, rank: int) -> int:
    """Input seed of a rank's replica (distinct per rank)."""
    return seed0 + rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of x over all ranks (x itself without a process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(work_per_rank: float, world: int, max_seconds: float) -> float:
    """Throughput of the whole job: every rank's work over the slowest rank's time."""
    return world * work_per_rank / max_seconds
