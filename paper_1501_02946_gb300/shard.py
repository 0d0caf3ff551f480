"""Host-side sharding of independent reconstructions across ranks.

Instances of a batch are independent, so a multi-GPU batch splits them over
ranks with no data-path collective.  Each instance is costed by the bytes its
stages move (the same per-kernel algorithmic bytes the benchmark reports),
and instances are dealt largest-first to the least-loaded rank (greedy
longest-processing-time scheduling), which keeps every rank within the
largest instance's cost of the mean.
"""
from __future__ import annotations

import heapq


def instance_cost(n_sensors, n_t, nx, ny, nz, sigma=2):
    """Algorithmic bytes of one forward reconstruction of this size."""
    Mx = sigma * nx
    nX1, nY1 = 2 * (nx // 2) + 1, ny // 2 + 1
    g = 4 * n_sensors * n_t
    T = 8 * Mx * nY1 * n_t
    G1 = 8 * nX1 * nY1 * n_t
    F = 8 * nx * nY1 * nz
    f = 4 * nx * ny * nz
    return (g + T) + (T + G1) + (G1 + F) + 2 * F + (F + f)


def partition(costs, world):
    """Assign instance indices to `world` ranks; returns a list of index lists
    (each sorted) covering every instance exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(x) for x in out]


def shard_for_rank(costs, rank, world):
    return partition(costs, world)[rank]
