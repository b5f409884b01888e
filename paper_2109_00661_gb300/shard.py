"""Sounding / model sharding across ranks (weak scaling, no collective on the
data path).

Soundings (and, for the forward benchmark, models) are independent units, so
each rank takes a contiguous block of them and runs the whole path on its own
GPU.  The only cross-rank traffic is the timing reduction of the benchmark:
the slowest rank's time sets the throughput of the job.
"""
from __future__ import annotations


def shard_range(n_units: int, rank: int, world: int):
    """Contiguous block [start, stop) of n_units for this rank; blocks differ in
    size by at most one unit and cover every unit exactly once."""
    if world < 1 or not (0 <= rank < world) or n_units < 0:
        raise ValueError("invalid shard request")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def job_throughput(units_per_rank, seconds_per_rank):
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return float(sum(units_per_rank)) / max(seconds_per_rank)
