"""FP64 oracle of the learned warm start -- test infrastructure only.

Restates, in plain numpy, the warm-start network as its C interface documents
it: per-node features, the 12-64-64-1 ReLU MLP evaluated with
BF16-rounded weights, the mean-squared loss, its gradient, and one Adam step.
Pins (tests/test_oracle_mlp.py): the forward pass, the loss and the output
layer's gradient against values worked out by hand for a small hand-set
network; the full gradient by central finite differences of the loss; Adam
over two steps against a hand computation; the features by hand on Fig. 1.
"""
from __future__ import annotations

import math

import numpy as np

F, H = 12, 64
OW1 = 0
OB1 = OW1 + H * F
OW2 = OB1 + H
OB2 = OW2 + H * H
OW3 = OB2 + H
OB3 = OW3 + H
NP = OB3 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OW1:OB1].reshape(H, F), p[OB1:OW2], p[OW2:OB2].reshape(H, H), p[OB2:OW3], p[OW3:OB3], p[OB3])


def to_bf16(w):
    """Round float32 values to bfloat16 (nearest, ties to even) and widen back to float64."""
    a = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def size_bin(s, N):
    """Histogram bin of an edge of size s at rank N: floor(8 log(s/2)/log(N/2)), clamped to 0..7."""
    if N <= 2 or s <= 2:
        return 0
    b = int(math.floor(8.0 * math.log(s / 2.0) / math.log(N / 2.0)))
    return min(max(b, 0), 7)


def features(hg, N=None):
    """n x 12 features from the edge lists (plain loops; small inputs)."""
    N = int(N or hg.rank)
    n = hg.n
    deg = np.zeros(n)
    ssum = np.zeros(n)
    smax = np.zeros(n)
    hist = np.zeros((n, 8))
    nbr = np.zeros(n)
    edges = hg.edges()
    for e in edges:
        for v in e:
            deg[v] += 1
    for e in edges:
        s = len(e)
        D = sum(deg[u] for u in e)
        b = size_bin(s, N)
        for v in e:
            ssum[v] += s
            smax[v] = max(smax[v], s)
            hist[v, b] += 1
            nbr[v] += D - deg[v]
    out = np.zeros((n, F))
    out[:, 0] = np.log1p(deg)
    out[:, 1] = np.log1p(np.where(deg > 0, ssum / np.maximum(deg, 1), 0.0))
    out[:, 2] = np.log1p(smax)
    out[:, 3:11] = np.log1p(hist)
    out[:, 11] = np.log1p(nbr)
    return out


def forward(params_bf16, feat):
    """Network output and the activations the gradient needs (FP64)."""
    W1, b1, W2, b2, W3, b3 = unpack(params_bf16)
    z1 = feat @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (h1, h2)


def loss_and_grad(params_bf16, feat, target):
    """L = mean (y - t)^2 and dL/dparams (FP64, with respect to the weights used)."""
    W1, b1, W2, b2, W3, b3 = unpack(params_bf16)
    y, (h1, h2) = forward(params_bf16, feat)
    n = feat.shape[0]
    d = y - target
    L = float(np.mean(d * d))
    dy = 2.0 * d / n
    g = np.zeros(NP)
    g[OW3:OB3] = h2.T @ dy
    g[OB3] = dy.sum()
    d2 = (dy[:, None] * W3[None, :]) * (h2 > 0)
    g[OW2:OB2] = (d2.T @ h1).ravel()
    g[OB2:OW3] = d2.sum(axis=0)
    d1 = (d2 @ W2) * (h1 > 0)
    g[OW1:OB1] = (d1.T @ feat).ravel()
    g[OB1:OW2] = d1.sum(axis=0)
    return L, g


def loss_only(params_bf16, feat, target):
    y, _ = forward(params_bf16, feat)
    return float(np.mean((y - target) ** 2))


def adam_step(p, m1, m2, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update (returns new p, m1, m2)."""
    m1 = beta1 * m1 + (1 - beta1) * g
    m2 = beta2 * m2 + (1 - beta2) * g * g
    c1 = 1 - beta1 ** step
    c2 = 1 - beta2 ** step
    p = p - lr * (m1 / c1) / (np.sqrt(m2 / c2) + eps)
    return p, m1, m2
