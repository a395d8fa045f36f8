"""One process per GPU: rank bookkeeping of the weakly scaled search.

Every rank searches its own data (a segment drawn with its own seed): maps, sub-bands and data
segments are independent, so the data path has no exchange.  Only the timing is combined: the step
time is the maximum over ranks and the work is the sum, so the reported rate is the whole job's.
"""
from __future__ import annotations

import os

SEED_STRIDE = 7919          # rank r draws its segment with seed base + SEED_STRIDE * r


def rank_env() -> tuple:
    """(rank, world size, local rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_seed(base: int, rank: int) -> int:
    return base + SEED_STRIDE * rank


def combine(ms: float, work: float, device="cpu") -> tuple:
    """(max over ranks of ms, sum over ranks of work) through torch.distributed when it is
    initialised with more than one rank, else the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(work)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
