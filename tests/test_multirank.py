"""The N > 1 path of bench.py on CPU: two gloo ranks run independent replicas
(no collective on the data path); the whole-job time is the slowest rank's
and the throughput counts the particle-steps of every rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: a replica that took (10 + 5 r) ms for (1000 + r) particle-steps
        ms, total = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000 + rank, dist, "cpu")
        q.put((rank, ms, total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for _, ms, total in res:
        assert ms == 15.0 and total == 2001.0


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(12.5, 7, None, "cpu") == (12.5, 7.0)


def _partition_rank(rank, world, port, q, R):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = bench.ensemble_partition(R, world, rank)
        peaks = bench.ensemble_members(R)[first:first + count]
        # the Philox keys this rank's handle uses: seed0 (= 1 + first) + local r
        keys = torch.tensor([1 + first + r for r in range(count)] + [-1] * (R - count), dtype=torch.int64)
        got = [torch.empty_like(keys) for _ in range(world)]
        dist.all_gather(got, keys)
        q.put((rank, first, count, [int(k) for k in torch.cat(got) if k >= 0], peaks))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,R", [(2, 64), (2, 7), (3, 10)])
def test_gloo_ranks_partition_the_ensemble(world, R):
    """Each rank owns a contiguous block of members; together the ranks own
    every member exactly once, each with its own Philox key 1 + r and the
    seed-blob peak of member r in the unsplit ensemble."""
    import bench
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_partition_rank, args=(r, world, port, q, R)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    all_peaks = bench.ensemble_members(R)
    nxt = 0
    for rank, first, count, keys, peaks in res:
        assert first == nxt and count in (R // world, R // world + 1)
        assert peaks == all_peaks[first:first + count]
        nxt = first + count
        assert sorted(keys) == list(range(1, R + 1))        # every member's key, once, on every rank's view
    assert nxt == R
