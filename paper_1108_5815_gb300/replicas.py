"""Multi-GPU execution of the solve: independent replicas, one per rank.

A single FMM system does not split across GPUs without exchanging coarse
multipoles and halo particles (the paper's local essential tree), so each rank
solves its own copy of the workload and no collective touches the data path.
The only communication is the timing aggregation: the job's time is the slowest
rank's, and the job's throughput is the work of all ranks over that time.
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment (1 process if absent)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(local_ms: float, local_units: int, group=None, device=None):
    """Slowest rank's time and total units over all ranks.

    Returns (max_ms, total_units, throughput = total_units / max_ms in units per second)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return local_ms, local_units, local_units / (local_ms / 1e3)
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    max_ms, units = float(t.item()), int(u.item())
    return max_ms, units, units / (max_ms / 1e3)
