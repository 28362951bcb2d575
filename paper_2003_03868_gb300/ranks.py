"""Whole-job timing of runs on several GPUs, one process per GPU (host logic only).

Every rank solves its own work: a replica of the same system (a single system does not
shard), or its own set of independent systems (the batched solve).  No data moves
between ranks; the only collective is this reduction of the timings: the job's time is
the slowest rank's, its work the sum of the ranks' work."""
from __future__ import annotations


def job_timing(ms: float, flops: float, dist=None, device: str = "cpu") -> tuple[float, float]:
    """(max over ranks of ms, sum over ranks of flops); the inputs unchanged without dist."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(flops)
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    f = torch.tensor([flops], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t.item()), float(f.item())
