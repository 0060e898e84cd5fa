"""The multi-rank host logic on the CPU: two gloo ranks (one process per rank, as on one GPU
per rank), the max / sum over ranks used for whole-job timings, and the split of a batched
ensemble's scenarios between ranks (no data-path collective)."""
import os
import socket

import numpy as np

from paper_1410_0753_gb300.ranks import max_over_ranks, shard_scenarios, sum_over_ranks, world_rank


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r = world_rank()
        durations = np.random.default_rng(4).integers(500, 4001, 256)
        mine = shard_scenarios(durations, w, r)
        work = float(durations[mine].sum())
        q.put((r, w, max_over_ranks(1.5 + r), sum_over_ranks(10.0 * (r + 1)), mine.tolist(),
               max_over_ranks(work), sum_over_ranks(work)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_split_the_ensemble():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    durations = np.random.default_rng(4).integers(500, 4001, 256)
    (r0, w0, m0, s0, a, mx0, sm0), (r1, w1, m1, s1, b, mx1, sm1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert m0 == m1 == 2.5 and s0 == s1 == 30.0
    assert not set(a) & set(b) and sorted(a + b) == list(range(256))
    assert sm0 == sm1 == float(durations.sum())
    assert mx0 - (sm0 - mx0) <= durations.max()          # the ranks' work differs by <= one scenario


def test_single_process_and_degenerate_splits():
    assert max_over_ranks(3.0) == 3.0 and sum_over_ranks(3.0) == 3.0 and world_rank() == (1, 0)
    d = [5, 5, 5]
    assert list(shard_scenarios(d, 1, 0)) == [0, 1, 2]
    parts = [list(shard_scenarios(d, 4, r)) for r in range(4)]
    assert parts == [[0], [1], [2], []]                  # more ranks than scenarios: one idles
    assert list(shard_scenarios([], 2, 0)) == []
