"""Replicas on several GPUs: one process per GPU, each running an independent copy of the
workload (the path shards over independent cells, so no collective touches the data).
The only cross-rank steps are the barriers around a timed region and the maximum of the
per-rank times; whole-job throughput is the units all ranks processed over that time."""
from __future__ import annotations

import os


def ranks_from_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) as torchrun sets them (1 process without it)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world: int, backend: str, device=None):
    """Join the process group of the replicas (None for a single process)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    if device is not None:
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float, device="cpu") -> float:
    """Largest value of x over the ranks (x itself for a single process)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Throughput of all replicas together: every rank processed units_per_rank in at
    most `seconds` (the maximum over ranks)."""
    return units_per_rank * world / seconds
