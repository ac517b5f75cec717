"""Edge sharding of one hypergraph across ranks (multi-GPU layout of S^3TTVc).

Edges are independent units of the computation, so a hypergraph can be cut
into per-rank edge sets whose partial results y_r = B_r x^(N-1) add up to y.
The cut balances the per-edge cost model of the series kernels,
(2s - 5) w (w + 1) / 2 + s w + 60 s with w = N - s + 1, greedily (largest
edges first, each to the currently lightest rank).  Every rank keeps the full
node set (x replicated); one sum-all-reduce of y completes a call.
"""
from __future__ import annotations

import numpy as np


def edge_cost(sizes, N):
    s = np.asarray(sizes, dtype=np.float64)
    w = N - s + 1
    prod = np.where(s >= 3, (2 * s - 5) * w * (w + 1) / 2 + s * w, 2 * w)
    return prod + 60.0 * s


def partition_edges(edge_ptr, world, N):
    """Rank of every edge (int32 array of length m), greedy longest-processing-time balance."""
    sizes = np.diff(np.asarray(edge_ptr, dtype=np.int64))
    cost = edge_cost(sizes, N)
    order = np.argsort(-cost, kind="stable")
    owner = np.empty(sizes.size, dtype=np.int32)
    load = np.zeros(world)
    # chunked greedy: equal-cost runs are dealt round-robin, which keeps it O(m log m)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += cost[i]
    return owner, load


def shard(edge_ptr, members, owner, rank):
    """CSR of the edges owned by `rank`."""
    edge_ptr = np.asarray(edge_ptr, dtype=np.int64)
    sizes = np.diff(edge_ptr)
    keep = owner == rank
    new_sizes = sizes[keep]
    ptr = np.zeros(new_sizes.size + 1, dtype=np.int64)
    np.cumsum(new_sizes, out=ptr[1:])
    mask = np.repeat(keep, sizes)
    return ptr, np.asarray(members, dtype=np.int32)[mask]
