"""Replica placement across ranks (one process per GPU).

The time step has no exchange between independent systems, so several GPUs only ever run
replicas side by side (weak scaling): a rank advances the replicas it was given and nothing
crosses ranks on the data path.  The only collectives are the harness's barrier and the
max-over-ranks of the timed region.
"""
from __future__ import annotations


def partition(sites, world: int):
    """Indices of the replicas each rank runs: longest-processing-time-first greedy on the
    per-replica site counts (replicas in decreasing size go to the least-loaded rank, ties to
    the lower rank), so the slowest rank carries at most the mean load plus one replica.
    Every replica is assigned exactly once; a rank may get none when world > len(sites)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sites)), key=lambda i: (-sites[i], i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += sites[i]
    return [sorted(o) for o in out]


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank's own replica of a single-system workload: distinct per rank."""
    return int(base) + int(rank)


def aggregate_rate(sites_per_rank, ms_per_rank) -> float:
    """Whole-job site-updates/s: all ranks' site updates over the slowest rank's time."""
    t = max(ms_per_rank)
    if t <= 0:
        raise ValueError("non-positive time")
    return float(sum(sites_per_rank)) / (t * 1e-3)
