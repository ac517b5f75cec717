"""Batched persistent S^3TTVc (many graphs x many vectors) against single calls and the oracle."""
import numpy as np
import pytest

import oracle
import s3synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _graphs():
    hs = [s3synth.config_powerlaw(n=3000, m=15000, rank=r, seed=40 + r) for r in (8, 13, 25, 32)]
    edges = [(0,), (1, 2), (0, 3, 4), (5,), (2, 6, 7, 8, 9)]
    hs.append(s3synth.from_edges(12, edges, rank=7))          # size-1 edges, isolated nodes
    hs.append(s3synth.config_large_rank(n=500, m=300, rank=40, seed=9))  # windows wider than 32
    return hs


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batched_equals_single_calls(dtype):
    import torch

    import paper_2311_08595_gb300 as s3
    dt = torch.float32 if dtype == "f32" else torch.float64
    hgs = _graphs()
    gs = [s3.s3_build_format(h.n, h.edge_ptr, h.members, rank=h.rank) for h in hgs]
    nvec = 3
    xs, ys = [], []
    for gi, h in enumerate(hgs):
        for v in range(nvec):
            xs.append(torch.tensor(s3synth.x_uniform(h.n, 0.3, 1.4, 100 * gi + v), dtype=dt, device="cuda"))
            ys.append(torch.full((h.n,), float("nan"), dtype=dt, device="cuda"))
    b = s3.s3_batch_create(gs, nvec)
    for _ in range(2):   # second call replays the captured graph
        s3.s3_sttsvc_batched(b, xs, ys)
        torch.cuda.synchronize()
        for j, (x, y) in enumerate(zip(xs, ys)):
            ref = torch.empty_like(x)
            s3.s3_sttsvc(gs[j // nvec], x, ref)
            torch.cuda.synchronize()
            # the single calls may evaluate large buckets in closed form, the batched kernels
            # never do: both within the parity tolerance of the exact values, so within twice
            # of each other
            e = rel_err(y.double().cpu().numpy(), ref.double().cpu().numpy(), floor=1e-30)
            assert e <= (2e-5 if dtype == "f32" else 2e-12), f"graph {j // nvec} vector {j % nvec}: {e:.2e}"
    # one graph all the way to the oracle
    want = oracle.ttsv1(hgs[2], xs[2 * nvec + 1].double().cpu().numpy())
    tol = 1e-5 if dtype == "f32" else 1e-12
    assert rel_err(ys[2 * nvec + 1].double().cpu().numpy(), want) <= tol


def test_batched_without_graph_and_autotune():
    import torch

    import paper_2311_08595_gb300 as s3
    hgs = _graphs()[:4]
    # the batched kernels evaluate every edge by the prefix/suffix series: the single calls it
    # is compared with bit for bit run the series too (no Bernoulli form)
    gs = [s3.s3_build_format(h.n, h.edge_ptr, h.members, bernoulli=-1) for h in hgs]
    nvec = 2
    xs = [torch.tensor(s3synth.x_uniform(h.n, 0.5, 1.5, 7 * gi + v), dtype=torch.float32, device="cuda")
          for gi, h in enumerate(hgs) for v in range(nvec)]
    ys = [torch.empty_like(x) for x in xs]
    refs = []
    for j, x in enumerate(xs):
        r = torch.empty_like(x)
        s3.s3_sttsvc(gs[j // nvec], x, r)
        refs.append(r)
    b = s3.s3_batch_create(gs, nvec, use_graph=0, block_threads=64, edges_per_thread=1)
    s3.s3_sttsvc_batched(b, xs, ys)
    torch.cuda.synchronize()
    assert all(torch.equal(y, r) for y, r in zip(ys, refs))
    res = s3.s3_batch_autotune(b, xs, ys)
    assert res["tried"] >= 6 and res["ms"] > 0
    assert res["block_threads"] in (64, 128, 256)
    ys2 = [torch.empty_like(x) for x in xs]
    s3.s3_sttsvc_batched(b, xs, ys2)
    torch.cuda.synchronize()
    assert all(torch.equal(y, r) for y, r in zip(ys2, refs))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batched_bernoulli_tiles(dtype):
    # Bernoulli-form buckets run as Bernoulli tiles in the batched kernel, with the same
    # per-edge arithmetic (and the same series fallback) as the single calls' launch.  FP32:
    # the other buckets run the same series kernels too, so the results are equal bit for
    # bit.  FP64: single calls run sizes 2 and 3 in kernels of their own; every vector
    # against the oracle at the FP64 bound instead
    import torch

    import paper_2311_08595_gb300 as s3
    dt = torch.float32 if dtype == "f32" else torch.float64
    hgs = _graphs()[:4]
    gs = [s3.s3_build_format(h.n, h.edge_ptr, h.members, closed_form_max_s=0) for h in hgs]
    used = [s3.s3_bernoulli_query(g)[dtype] for g in gs]
    assert sum(len(u) for u in used) > 0, used
    nvec = 2
    xs = [torch.tensor(s3synth.x_uniform(h.n, 0.5, 1.5, 11 * gi + v), dtype=dt, device="cuda")
          for gi, h in enumerate(hgs) for v in range(nvec)]
    refs = []
    for j, x in enumerate(xs):
        r = torch.empty_like(x)
        s3.s3_sttsvc(gs[j // nvec], x, r)
        refs.append(r)
    b = s3.s3_batch_create(gs, nvec)
    ys = [torch.full_like(x, float("nan")) for x in xs]
    for _ in range(2):
        s3.s3_sttsvc_batched(b, xs, ys)
        torch.cuda.synchronize()
        if dtype == "f32":
            assert all(torch.equal(y, r) for y, r in zip(ys, refs))
        else:
            for j, y in enumerate(ys):
                want = oracle.ttsv1(hgs[j // nvec], xs[j].cpu().numpy())
                assert rel_err(y.cpu().numpy(), want) <= 1e-12, j


def test_batch_rejects_atomic_graphs():
    import paper_2311_08595_gb300 as s3
    h = s3synth.config_small(seed=1)
    g = s3.s3_build_format(h.n, h.edge_ptr, h.members, reduce=1)
    with pytest.raises(s3.S3Error):
        s3.s3_batch_create([g], 2)
