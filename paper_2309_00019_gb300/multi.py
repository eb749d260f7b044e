"""Multi-GPU layout: one process per GPU, weak scaling.

The hot path partitions into independent segments, so every rank filters its
own segment (its own seeded synthetic data and banks) and no collective
touches the data path.  The only collectives are a barrier around the timed
region and two scalar reductions of the timing: the job's time is the
slowest rank's device time and its work is the sum of the ranks'
template-seconds.
"""

from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) from the launcher's environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def segment_seed(base, rank):
    """Seed of the rank's own segment: independent data per rank."""
    return base + rank


def reduce_timing(dist, seconds, work, device=None):
    """(max over ranks of seconds, sum over ranks of work), as floats."""
    import torch

    t = torch.tensor([seconds, work], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])
