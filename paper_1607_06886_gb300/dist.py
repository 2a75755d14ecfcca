"""Replica sharding of independent planning queries across ranks (one process per GPU).

Queries are independent problems, so ranks share nothing on the data path: rank r plans the
query with seed `base_seed + r`, and only the timing and the partial-plan counts are reduced
(maximum of the timed region, sum of the work).  The reductions run on whatever backend the
process group uses (gloo on CPU tensors, NCCL on CUDA tensors).
"""
from __future__ import annotations

import os
from typing import Tuple


def world() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def query_seed(rank: int, base_seed: int = 0) -> int:
    return base_seed + rank


def _reduce(x: float, op: str, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def reduce_max(x: float, device="cpu") -> float:
    return _reduce(x, "max", device)


def reduce_sum(x: float, device="cpu") -> float:
    return _reduce(x, "sum", device)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def aggregate(work: float, seconds: float, device="cpu") -> Tuple[float, float, float]:
    """Whole-job throughput: (total work, max seconds over ranks, total work / max seconds)."""
    tot = reduce_sum(work, device)
    t = reduce_max(seconds, device)
    return tot, t, (tot / t if t > 0 else 0.0)
