"""Warm-start kernels (features, MLP forward/backward, Adam) against the FP64 oracle,
and the benefit of the trained network on a held-out hypergraph."""
import numpy as np
import pytest

import s3synth
from oracle import mlp

pytestmark = pytest.mark.gpu


def _dev(a, dt="float32"):
    import torch
    return torch.tensor(np.asarray(a), dtype=getattr(torch, dt), device="cuda").contiguous()


@pytest.mark.parametrize("which", ["small", "powerlaw", "fig1"])
def test_features_match_oracle(which):
    import paper_2311_08595_gb300 as s3
    hg = {"small": lambda: s3synth.config_small(seed=3),
          "powerlaw": lambda: s3synth.config_powerlaw(n=3000, m=15000, rank=25, seed=5),
          "fig1": s3synth.fig1_example}[which]()
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    f = s3.s3_features(g).cpu().numpy().astype(np.float64)
    want = mlp.features(hg)
    assert np.allclose(f, want, rtol=1e-6, atol=1e-6)


def test_features_every_degree_class():
    # a hub of degree 5000 (cut into pieces), nodes of degree 250 (a warp each) and 100
    # (eight lanes each), many of degree <= 32 (sliced-ELL groups) and isolated nodes
    import paper_2311_08595_gb300 as s3
    edges = []
    for i in range(5000):
        e = [0, 1 + i % 300, 301 + i % 50]
        if i % 2 == 0:
            e.append(351 + i % 10)
        e += [400 + (7 * i + j) % 3000 for j in range(i % 5)]
        edges.append(tuple(dict.fromkeys(e)))
    hg = s3synth.from_edges(3500, edges, rank=9)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, rank=hg.rank)
    f = s3.s3_features(g).cpu().numpy().astype(np.float64)
    want = mlp.features(hg)
    assert np.allclose(f, want, rtol=1e-6, atol=1e-6)
    assert f[0, 0] == pytest.approx(np.log1p(5000), rel=1e-6)
    assert np.all(f[3400:] == 0)


def test_forward_loss_gradient_and_adam_match_oracle():
    import paper_2311_08595_gb300 as s3
    rng = np.random.default_rng(1)
    init = rng.normal(0, 0.2, mlp.NP).astype(np.float32)
    m = s3.s3_mlp_create(init)
    pb = s3.s3_mlp_get_params(m, bf16=True).astype(np.float64)
    assert np.array_equal(pb, mlp.to_bf16(init))
    n = 1000
    feat = rng.uniform(0, 4, (n, mlp.F)).astype(np.float32)
    tgt = rng.normal(0, 1, n).astype(np.float32)
    fd, td = _dev(feat), _dev(tgt)
    y = s3.s3_mlp_forward(m, fd).cpu().numpy()
    yo, _ = mlp.forward(pb, feat.astype(np.float64))
    assert np.max(np.abs(y - yo)) <= 1e-4 * max(1.0, np.max(np.abs(yo)))
    # features at an address that is not 16-byte aligned (scalar loads): the same outputs
    import torch
    shifted = torch.empty(n * mlp.F + 1, dtype=torch.float32, device="cuda")[1:]
    shifted.copy_(fd.reshape(-1))
    y2 = s3.s3_mlp_forward(m, shifted.view(n, mlp.F)).cpu().numpy()
    assert np.array_equal(y, y2)
    loss, grad = s3.s3_mlp_loss_grad(m, fd, td)
    lo, go = mlp.loss_and_grad(pb, feat.astype(np.float64), tgt.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.max(np.abs(grad - go)) <= 1e-4 * np.max(np.abs(go))
    # one Adam step on the FP32 master weights
    s3.s3_mlp_adam_step(m, lr=1e-3)
    p1 = s3.s3_mlp_get_params(m).astype(np.float64)
    po, _, _ = mlp.adam_step(init.astype(np.float64), np.zeros(mlp.NP), np.zeros(mlp.NP),
                             grad.astype(np.float64), 1, lr=1e-3)
    assert np.max(np.abs(p1 - po)) <= 1e-6


def test_training_reduces_loss_and_warm_start_helps():
    import torch

    import paper_2311_08595_gb300 as s3
    from paper_2311_08595_gb300 import warmstart as ws
    rng = np.random.default_rng(7)
    train_graphs = [s3synth.largest_component(
        s3synth.config_powerlaw(n=4000, m=20000, rank=25, seed=int(rng.integers(1 << 30))))[0] for _ in range(16)]
    feat, tgt = ws.build_dataset(train_graphs)
    model, hist = ws.train(feat, tgt, epochs=30, batch=8192, lr=3e-3)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    held = s3synth.largest_component(s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=999))[0]
    r = ws.evaluate(held, model, tol=1e-8)
    print("warm start:", r)
    assert r["max_rel_diff_x"] < 1e-7
    assert r["learned"]["iters"] <= r["uniform"]["iters"]
    x0 = s3.s3_warmstart(s3.s3_build_format(held.n, held.edge_ptr, held.members), model)
    assert torch.all(x0 > 0) and abs(float(x0.sum()) - 1.0) < 1e-12


def test_shipped_network_saves_iterations_on_held_out_graph():
    # the network the package ships (500 training hypergraphs of n = 50k, power-law recipe)
    # on a held-out hypergraph of the same recipe and another size: strictly fewer NQZ
    # iterations to 1e-8 than the uniform start, and the same centrality
    import os

    import paper_2311_08595_gb300 as s3
    from paper_2311_08595_gb300 import warmstart as ws
    path = os.path.join(os.path.dirname(s3.__file__), "data", "warmstart_500x50k.npy")
    model = s3.s3_mlp_create(params=np.load(path))
    held = s3synth.largest_component(s3synth.config_powerlaw(n=200000, m=1000000, rank=25, seed=777))[0]
    for prec in (0, 3):
        r = ws.evaluate(held, model, tol=1e-8, precision=prec)
        print("shipped warm start, precision", prec, r)
        assert r["learned"]["iters"] < r["uniform"]["iters"], r
        assert r["max_rel_diff_x"] < 1e-7
