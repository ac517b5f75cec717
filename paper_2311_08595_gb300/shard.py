"""Edge sharding of one hypergraph across ranks (multi-GPU layout of S^3TTVc).

Edges are independent units of the computation, so a hypergraph can be cut
into per-rank edge sets whose partial results y_r = B_r x^(N-1) add up to y.
The cut balances the per-edge cost model of the series kernels,
(2s - 5) w (w + 1) / 2 + s w + 60 s with w = N - s + 1, greedily (largest
edges first, each to the currently lightest rank).  Every rank keeps the full
node set (x replicated); one sum-all-reduce of y completes a call.

``ShardedGraph`` is the multi-GPU path: each rank builds a library handle on
its own edges (at the global rank N), an S^3TTVc call is the local call plus
one sum-all-reduce of y (torch.distributed: NCCL between GPUs), and the
centrality iteration of Algorithm 1 runs on every rank on the summed z with
the library's update kernels (``s3_nqz_update``), so all ranks hold the same
iterate and take the same stopping decision without further communication.
The device work goes through a backend object (default: the CUDA library
binding); it only moves buffers between the library and the collective.
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


class _LibraryBackend:
    """The CUDA library through its Python binding (device tensors)."""

    def __init__(self):
        import paper_2311_08595_gb300 as s3
        self.s3 = s3

    def build(self, n, edge_ptr, members, N):
        return self.s3.s3_build_format(n, edge_ptr, members, rank=N)

    def zeros(self, n):
        import torch
        return torch.zeros(n, dtype=torch.float64, device="cuda")

    def fill(self, v, value):
        v.fill_(value)   # a start vector (the uniform 1/n of Algorithm 1, or max 1)
        return v

    def sttsvc(self, h, x, y):
        return self.s3.s3_sttsvc(h, x, y)

    def nqz_update(self, h, z, xhat, x_next, xhat_next):
        return self.s3.s3_nqz_update(h, z, xhat, x_next, xhat_next)

    def destroy(self, h):
        self.s3.s3_destroy(h)


class ShardedGraph:
    """One rank's share of an edge-sharded hypergraph (see the module docstring).

    n, edge_ptr, members: the whole hypergraph (host CSR, identical on every rank);
    N: its rank (largest edge size) unless given.  group: torch.distributed process
    group (None = default); backend: device operations (None = the CUDA library)."""

    def __init__(self, n, edge_ptr, members, N=None, group=None, backend=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        sizes = np.diff(np.asarray(edge_ptr, dtype=np.int64))
        self.N = int(N or (sizes.max() if sizes.size else 1))
        self.n = int(n)
        self.owner, self.load = partition_edges(edge_ptr, self.world, self.N)
        ptr, mem = shard(edge_ptr, members, self.owner, self.rank)
        self.backend = backend or _LibraryBackend()
        self.h = self.backend.build(self.n, ptr, mem, self.N)

    def sttsvc(self, x, y):
        """y = B x^(N-1) on every rank: the local edges' part, then one sum over ranks."""
        self.backend.sttsvc(self.h, x, y)
        self.dist.all_reduce(y, op=self.dist.ReduceOp.SUM, group=self.group)
        return y

    def hcentrality(self, tol=1e-8, max_iter=10000):
        """Algorithm 1 with the edge-sharded S^3TTVc (FP64).  Returns (x with 1-norm 1, lambda_min,
        lambda_max, iterations, converged); every rank returns the same values."""
        b = self.backend
        x, xhat, xn, xhatn, z = (b.zeros(self.n) for _ in range(5))
        # Algorithm 1's start y = 1/n, handed to S^3TTVc at max 1 (the ratio is scale-free)
        b.fill(xhat, 1.0)
        self.sttsvc(xhat, z)
        b.nqz_update(self.h, z, xhat, x, xhat)        # x_1 (the bracket of the start is not a test)
        lo = hi = float("nan")
        for it in range(1, max_iter + 1):
            self.sttsvc(xhat, z)
            lo, hi = b.nqz_update(self.h, z, xhat, xn, xhatn)
            if (hi - lo) / lo < tol:
                return x, lo, hi, it, True
            x, xn = xn, x
            xhat, xhatn = xhatn, xhat
        return x, lo, hi, max_iter, False

    def close(self):
        if self.h is not None:
            self.backend.destroy(self.h)
            self.h = None
