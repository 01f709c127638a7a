"""Placement of independent instances on ranks (one GPU each).

An ensemble's instances share nothing, so a multi-GPU run splits them over the ranks with no
data exchange at all (only the benchmark's final aggregation of times and counts).  The
split is greedy longest-processing-time (LPT) scheduling on a per-instance cost: instances
in decreasing cost order, each to the rank with the least cost so far (ties to the lower
rank).  Its makespan is within 4/3 - 1/(3 N) of the optimum (Graham, 1969)."""
from __future__ import annotations


def lpt_shard(costs, n_ranks: int):
    """Instance indices per rank (each list ascending) for the given per-instance costs."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * n_ranks
    out = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]
