"""The N > 1 layout on CPU: two gloo ranks, each with its own segment, and the
timing reductions bench.py applies (max of the time, sum of the work)."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import synth
    from paper_2309_00019_gb300.multi import reduce_timing, segment_seed

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = synth.make_config1(seed=segment_seed(0, rank))
        digest = float(np.abs(cfg.strain).sum())
        seconds, work = 1.0 + 0.5 * rank, 10.0 * (rank + 1)
        dist.barrier()
        t_max, w_sum = reduce_timing(dist, seconds, work)
        digests = [None] * world
        dist.all_gather_object(digests, digest)
        out.put((rank, t_max, w_sum, digests))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_reduction():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, w_sum, digests in res:
        assert t_max == 1.5          # the slowest rank's time
        assert w_sum == 30.0         # every rank's work
        assert w_sum / t_max == 20.0  # the job's throughput as bench.py reports it
        assert digests[0] != digests[1]  # independent segments per rank


def _gather_worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2309_00019_gb300.mf import TRIGGER_NP
    from paper_2309_00019_gb300.multi import gather_triggers

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(rank)
        n = 5 + 3 * rank  # variable sizes
        t = np.zeros(n, dtype=TRIGGER_NP)
        t["det"] = rng.integers(0, 2, n)
        t["tmpl"] = rank * 100 + rng.integers(0, 100, n)  # this rank's template range
        t["sample"] = rng.integers(0, 1 << 14, n)
        t["snr"] = rng.uniform(5, 10, n)
        t = np.sort(t, order=["det", "tmpl", "sample"])
        out.put((rank, t, gather_triggers(dist, t)))
    finally:
        dist.destroy_process_group()


def test_sharded_trigger_gather_equals_merged_lists():
    import torch.multiprocessing as mp

    from paper_2309_00019_gb300.multi import merge_triggers

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = merge_triggers([res[0][1], res[1][1]])
    assert len(expect) == 5 + 8
    for _, _, merged in res:
        assert np.array_equal(merged, expect)
    assert np.all(np.diff(expect["det"]) >= 0)
