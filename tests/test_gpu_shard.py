"""The edge-sharded path on one GPU: shard handles, their sum, the NQZ update step.

Handles built on disjoint edge sets of one hypergraph (at its global rank) must add
up to the whole hypergraph's S^3TTVc; s3_nqz_update must follow Algorithm 1's step
from a complete z; and the sharded driver on a one-rank NCCL group must give the
same centrality as s3_hcentrality.  (The two-rank driver runs on CPU ranks in
test_multirank_cpu.py.)
"""
import os
import socket

import numpy as np
import pytest

import oracle
import s3synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def test_shard_handles_sum_to_the_whole():
    import torch

    import paper_2311_08595_gb300 as s3
    from paper_2311_08595_gb300.shard import partition_edges, shard
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=51)
    x = torch.tensor(s3synth.x_degree_like(hg, seed=51), device="cuda")
    owner, _ = partition_edges(hg.edge_ptr, 3, hg.rank)
    total = torch.zeros_like(x)
    for r in range(3):
        ptr, mem = shard(hg.edge_ptr, hg.members, owner, r)
        g = s3.s3_build_format(hg.n, ptr, mem, rank=hg.rank)
        y = torch.empty_like(x)
        s3.s3_sttsvc(g, x, y)
        total += y
        s3.s3_destroy(g)
    want = oracle.ttsv1(hg, x.cpu().numpy())
    assert rel_err(total.cpu().numpy(), want) <= 1e-12


def test_nqz_update_step():
    import torch

    import paper_2311_08595_gb300 as s3
    hg = s3synth.largest_component(s3synth.config_powerlaw(n=5000, m=25000, rank=12, seed=52))[0]
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    xh = np.random.default_rng(52).uniform(0.3, 1.0, hg.n)
    z = oracle.ttsv1(hg, xh)
    zd, xd = torch.tensor(z, device="cuda"), torch.tensor(xh, device="cuda")
    xn, xhn = torch.empty_like(xd), torch.empty_like(xd)
    lo, hi = s3.s3_nqz_update(g, zd, xd, xn, xhn)
    ratio = z / xh ** (hg.rank - 1)
    r = z ** (1.0 / (hg.rank - 1))
    assert abs(lo - ratio.min()) <= 1e-13 * ratio.min() and abs(hi - ratio.max()) <= 1e-13 * ratio.max()
    # the (N-1)-th root is an FP32 estimate refined by one Newton step in FP64 (~1e-13
    # relative), and the 1-norm is summed in another order than numpy's
    assert rel_err(xn.cpu().numpy(), r / r.sum()) <= 1e-12
    assert rel_err(xhn.cpu().numpy(), r / r.max()) <= 1e-12
    s3.s3_destroy(g)


def test_sharded_driver_one_rank_matches_hcentrality():
    import torch
    import torch.distributed as dist

    import paper_2311_08595_gb300 as s3
    from paper_2311_08595_gb300.shard import ShardedGraph
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        hg = s3synth.largest_component(s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=53))[0]
        sg = ShardedGraph(hg.n, hg.edge_ptr, hg.members)
        x, lo, hi, it, conv = sg.hcentrality(tol=1e-10)
        g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
        xr, res = s3.s3_hcentrality(g, tol=1e-10)
        torch.cuda.synchronize()
        assert conv and res["converged"] and abs(it - res["iters"]) <= 1
        assert rel_err(x.cpu().numpy(), xr.cpu().numpy()) <= 1e-9
        sg.close()
        s3.s3_destroy(g)
    finally:
        dist.destroy_process_group()
