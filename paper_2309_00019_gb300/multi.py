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


def merge_triggers(parts):
    """Trigger lists of template-range shards, each ordered by (det, tmpl,
    sample), merged into the order of the unsharded run."""
    import numpy as np

    parts = [p for p in parts if p is not None and len(p)]
    if not parts:
        return None
    return np.sort(np.concatenate(parts), order=["det", "tmpl", "sample"], kind="stable")


def gather_triggers(dist, trig):
    """Variable-size gather of every rank's trigger list, merged (every rank
    gets the merge): the one collective a bank sharded by template range needs."""
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, trig)
    return merge_triggers(parts)
