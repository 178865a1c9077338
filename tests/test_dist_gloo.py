"""Multi-process host logic of bench.py on CPU (gloo, world_size 2): the batch of surfaces is
split over the ranks with no data-path collective, and the job's time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_1805_06106_gb300 import dist as D

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, lr = D.env()
        shard = D.lpt_shards(costs, ws)[r]
        load = sum(costs[i] for i in shard)
        all_shards = [None] * ws
        dist.all_gather_object(all_shards, shard)
        D.barrier()
        q.put((r, shard, all_shards, D.max_over_ranks(load), D.sum_over_ranks(load), (ws, r, lr)))
    finally:
        dist.destroy_process_group()


def test_batch_split_over_two_gloo_ranks():
    from synth import batched_specs

    costs = [300 * n * n for n, _, _ in batched_specs(64, seed=5)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shards = [r[1] for r in res]
    # every rank saw the same split; it partitions the batch
    assert res[0][2] == res[1][2] == shards
    assert sorted(shards[0] + shards[1]) == list(range(len(costs)))
    loads = [sum(costs[i] for i in s) for s in shards]
    # LPT: the heavier rank exceeds the lighter by at most the largest item
    assert max(loads) - min(loads) <= max(costs)
    assert all(r[3] == max(loads) for r in res) and all(r[4] == sum(costs) for r in res)
    assert [r[5] for r in res] == [(2, 0, 0), (2, 1, 1)]


def test_lpt_single_rank_and_ties():
    from paper_1805_06106_gb300 import dist as D

    assert D.lpt_shards([3, 1, 2], 1) == [[0, 1, 2]]
    assert D.lpt_shards([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    assert D.lpt_shards([], 3) == [[], [], []]
    assert D.max_over_ranks(2.5) == 2.5  # no process group: the value itself
