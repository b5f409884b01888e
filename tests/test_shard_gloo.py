"""Multi-rank path on CPU: world_size-2 gloo process group exercising the
sounding sharding and the max-over-ranks timing reduction bench.py uses."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2109_00661_gb300.shard import job_throughput, shard_range


def test_shard_range_partitions_units():
    for n in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_soundings = 1001
    start, stop = shard_range(n_soundings, rank, world)
    # each rank "processes" its own soundings: a stand-in per-sounding result
    # (its index) and a stand-in elapsed time that differs between ranks
    mine = torch.arange(start, stop, dtype=torch.float64)
    elapsed = torch.tensor([1.0 + 0.5 * rank], dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
    count = torch.tensor([float(stop - start)], dtype=torch.float64)
    dist.all_reduce(count, op=dist.ReduceOp.SUM)
    total = torch.tensor([float(mine.sum())], dtype=torch.float64)
    dist.all_reduce(total, op=dist.ReduceOp.SUM)
    q.put((rank, float(elapsed.item()), float(count.item()), float(total.item())))
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, elapsed, count, total in out:
        assert elapsed == 1.5           # the slowest rank sets the job time
        assert count == 1001            # every sounding processed once
        assert total == sum(range(1001))
    assert job_throughput([501, 500], [1.0, 1.5]) == pytest.approx(1001 / 1.5)
