"""Multi-rank path on CPU: world_size-2 gloo process groups exercising the
sounding sharding and the max-over-ranks timing reduction bench.py uses, and a
short synthetic flight line split across the ranks with shard_range, each rank
running the (serial, CPU) oracle sampler on its own block of soundings: the
gathered per-sounding model odds equal a single-process run's exactly."""
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


def _line_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, stop = shard_range(5, rank, world)
    mine = [(s, _line_sounding(s)) for s in range(start, stop)]
    out = [None] * world
    dist.all_gather_object(out, mine)
    t = torch.tensor([float(len(mine))], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    q.put((rank, [x for part in out for x in part], float(t.item())))
    dist.destroy_process_group()


def _line_sounding(s):
    """The oracle sampler on sounding s of a 5-sounding synthetic line (tiny
    settings: 24 particles, kappa, lambda <= 1, 2 sweeps per stage); the
    Philox streams are keyed by the global sounding index."""
    import oracle as O
    from oracle import rjsmc as R
    from paper_2109_00661_gb300 import inputs as I
    name = "sounding-g20-f40-k120"
    so = I.oracle_system(name)
    so["T"] = O.tmatrix(so["freqs"], so["times"])
    truth, _ = I.flight_line(5)
    y = O.forward(I.subset(truth, [s]), so, mode=O.HANKEL_RULE, nthreads=1)[0]
    data = I.noisy(y, seed=100 + s)
    st = R.SMCSettings(n_particles=24, kappa_max=1, lambda_max=1, n_sweeps=2, seed=7, sounding=s)
    res = R.run(st, R.ForwardLik(so, data, I.EPS_AN, I.EPS_MN, lmax=3, nthreads=1), max_stages=40)
    post, lb = R.model_odds(res.counts, 1, 1)
    return [float(v) for v in post], float(lb), len(res.gammas)


def test_two_rank_flight_line_matches_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_line_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = [(s, _line_sounding(s)) for s in range(5)]
    for rank, gathered, count in out:
        assert count == 5
        assert sorted(gathered) == ref
