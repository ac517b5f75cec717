"""Training and evaluation driver of the learned NQZ warm start.

All arithmetic runs in the library's kernels (features, H-eigenvector
centrality, targets, MLP forward/backward, Adam); this module only moves
device buffers around (PyTorch tensors) and loops.

    python -m paper_2311_08595_gb300.warmstart --graphs 500 --n 50000 --out weights.npy
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import (s3_build_format, s3_destroy, s3_features, s3_hcentrality, s3_mlp_adam_step, s3_mlp_create,
               s3_mlp_get_params, s3_mlp_loss_grad, s3_mlp_target)


def graph_examples(hg, tol=1e-10):
    """(features, targets) of one hypergraph: targets are log x* minus its mean, x* from FP64 NQZ."""
    g = s3_build_format(hg.n, hg.edge_ptr, hg.members)
    feat = s3_features(g)
    x, res = s3_hcentrality(g, tol=tol, precision=0)
    tgt = s3_mlp_target(g, x)
    s3_destroy(g)
    return feat, tgt, res


def build_dataset(hypergraphs, tol=1e-10, seed=0):
    """Stack every node of every hypergraph and shuffle the rows (device tensors)."""
    import torch
    feats, tgts = [], []
    for hg in hypergraphs:
        f, t, _ = graph_examples(hg, tol)
        feats.append(f)
        tgts.append(t)
    feat = torch.cat(feats)
    tgt = torch.cat(tgts)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(feat.shape[0], generator=gen).to(feat.device)
    return feat.index_select(0, perm).contiguous(), tgt.index_select(0, perm).contiguous()


def train(feat, tgt, epochs=4, batch=65536, lr=2e-3, seed=0, log=None):
    """Adam on mini-batches of contiguous rows; returns (model, loss history)."""
    model = s3_mlp_create(seed=seed)
    n = feat.shape[0]
    hist = []
    step = 0
    for ep in range(epochs):
        for b0 in range(0, n, batch):
            b1 = min(n, b0 + batch)
            want = (step % 50 == 0)
            loss, _ = s3_mlp_loss_grad(model, feat[b0:b1], tgt[b0:b1], want_grad=False)
            s3_mlp_adam_step(model, lr=lr)
            if want:
                hist.append((step, loss))
                if log:
                    log(f"epoch {ep} step {step} loss {loss:.5f}")
            step += 1
    return model, hist


def evaluate(hg, model, tol=1e-8, precision=0):
    """Iterations and wall time to tol: uniform start vs learned warm start (same handle)."""
    import torch

    from . import s3_warmstart
    g = s3_build_format(hg.n, hg.edge_ptr, hg.members)
    # one untimed pass of each allocates the handle's iteration and warm-start scratch
    s3_hcentrality(g, tol=tol, precision=precision)
    s3_warmstart(g, model)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xu, ru = s3_hcentrality(g, tol=tol, precision=precision)
    torch.cuda.synchronize()
    tu = time.perf_counter() - t0
    t0 = time.perf_counter()
    x0 = s3_warmstart(g, model)
    xw, rw = s3_hcentrality(g, x0=x0, tol=tol, precision=precision)
    torch.cuda.synchronize()
    tw = time.perf_counter() - t0
    diff = float(((xw - xu).abs() / xu).max())
    s3_destroy(g)
    return {"uniform": {"iters": ru["iters"], "seconds": tu}, "learned": {"iters": rw["iters"], "seconds": tw},
            "speedup": tu / tw, "max_rel_diff_x": diff}


def start_cost(hg, model, reps=5):
    """Device time of the warm start alone (features, MLP, exponentiation and normalisation)
    on hg, in ms, against one FP32 and one FP64 S^3TTVc call on the same handle."""
    import torch

    from . import s3_sttsvc, s3_warmstart
    g = s3_build_format(hg.n, hg.edge_ptr, hg.members)
    s3_warmstart(g, model)
    x32 = torch.ones(hg.n, dtype=torch.float32, device="cuda")
    y32 = torch.empty_like(x32)
    x64, y64 = x32.double(), torch.empty(hg.n, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    out = {}
    for name, fn in (("warm_start_ms", lambda: s3_warmstart(g, model)), ("sttsvc_f32_ms", lambda: s3_sttsvc(g, x32, y32)),
                     ("sttsvc_f64_ms", lambda: s3_sttsvc(g, x64, y64))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / reps
    s3_destroy(g)
    return out


def main():
    import s3synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=500)
    ap.add_argument("--n", type=int, default=50000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--out", default="warmstart_weights.npy",
                    help="the package ships paper_2311_08595_gb300/data/warmstart_500x50k.npy, made with the defaults")
    a = ap.parse_args()
    rng = np.random.default_rng(12345)
    hgs = [s3synth.largest_component(s3synth.config_powerlaw(n=a.n, m=5 * a.n, seed=int(rng.integers(1 << 30))))[0]
           for _ in range(a.graphs)]
    feat, tgt = build_dataset(hgs)
    model, hist = train(feat, tgt, epochs=a.epochs, log=print)
    np.save(a.out, s3_mlp_get_params(model))
    print("saved", a.out)


if __name__ == "__main__":
    main()
