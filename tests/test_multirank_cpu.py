"""Multi-rank logic on CPU with gloo (world size 2): edge sharding with one sum of y,
the edge-sharded centrality driver (paper_2311_08595_gb300.shard.ShardedGraph), and
the benchmark's max-over-ranks timing.

Without a GPU the driver runs on a stand-in backend defined here (the oracle's
S^3TTVc on each rank's edges and the update step written out in numpy); the
partition, the sum of y across ranks and the iteration are the product's code.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sharded_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import s3synth
        from paper_2311_08595_gb300.shard import partition_edges, shard
        hg = s3synth.config_small(seed=4)
        x = s3synth.x_uniform(hg.n, 0.0, 1.0, 4)
        owner, load = partition_edges(hg.edge_ptr, world, hg.rank)
        ptr, mem = shard(hg.edge_ptr, hg.members, owner, rank)
        part = s3synth.Hypergraph(hg.n, ptr, mem, rank=hg.rank)
        y = torch.tensor(oracle.ttsv1(part, x, N=hg.rank))
        dist.all_reduce(y, op=dist.ReduceOp.SUM)
        # the benchmark's timing rule: the job time is the slowest rank's
        t = torch.tensor([1.0 + rank])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            full = oracle.ttsv1(hg, x)
            q.put((float(np.max(np.abs(y.numpy() - full) / np.maximum(np.abs(full), 1e-300))), float(t.item()),
                   float(load.max() / load.min())))
    finally:
        dist.destroy_process_group()


def test_edge_sharded_sum_equals_full_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    err, tmax, imbalance = q.get(timeout=10)
    assert err < 1e-13 and tmax == 2.0 and imbalance < 1.01


def test_partition_is_complete_and_balanced():
    import s3synth
    from paper_2311_08595_gb300.shard import partition_edges, shard
    hg = s3synth.config_powerlaw(n=5000, m=25000, rank=25, seed=1)
    owner, load = partition_edges(hg.edge_ptr, 4, hg.rank)
    assert set(np.unique(owner)) == {0, 1, 2, 3}
    total = sum(shard(hg.edge_ptr, hg.members, owner, r)[1].size for r in range(4))
    assert total == hg.nnz
    assert load.max() / load.min() < 1.01


class _OracleBackend:
    """CPU stand-in for the library calls the sharded driver makes (test only)."""

    def build(self, n, edge_ptr, members, N):
        import s3synth
        return s3synth.Hypergraph(n, edge_ptr, members, rank=N)

    def zeros(self, n):
        return torch.zeros(n, dtype=torch.float64)

    def fill(self, v, value):
        v.fill_(value)
        return v

    def sttsvc(self, h, x, y):
        import oracle
        y.copy_(torch.from_numpy(oracle.ttsv1(h, x.numpy(), N=h.rank)))
        return y

    def nqz_update(self, h, z, xhat, x_next, xhat_next):
        k = h.rank - 1
        zn, xn = z.numpy(), xhat.numpy()
        ratio = zn / xn ** k
        r = zn ** (1.0 / k)
        x_next.copy_(torch.from_numpy(r / r.sum()))
        xhat_next.copy_(torch.from_numpy(r / r.max()))
        return float(ratio.min()), float(ratio.max())

    def destroy(self, h):
        pass


def _nqz_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import s3synth
        from paper_2311_08595_gb300.shard import ShardedGraph
        hg = s3synth.largest_component(s3synth.config_powerlaw(n=1500, m=7500, rank=8, seed=6))[0]
        sg = ShardedGraph(hg.n, hg.edge_ptr, hg.members, backend=_OracleBackend())
        assert sg.owner.size == hg.m and set(np.unique(sg.owner)) <= set(range(world))
        x, lo, hi, it, conv = sg.hcentrality(tol=1e-10)
        if rank == 0:
            q.put((x.numpy(), lo, hi, it, conv, hg))
        else:
            q.put((x.numpy(), lo, hi, it, conv, None))
        sg.close()
    finally:
        dist.destroy_process_group()


def test_sharded_centrality_driver_matches_single_process_oracle():
    from oracle.nqz import nqz
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_nqz_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    hg = next(o[5] for o in out if o[5] is not None)
    (x0, lo0, hi0, it0, c0, _), (x1, lo1, hi1, it1, c1, _) = out
    # every rank holds the same iterate and took the same decision
    assert c0 and c1 and it0 == it1 and np.array_equal(x0, x1) and (lo0, hi0) == (lo1, hi1)
    ref = nqz(hg, tol=1e-10)
    assert abs(it0 - ref.iters) <= 1
    assert np.max(np.abs(x0 - ref.x) / ref.x) < 1e-9
