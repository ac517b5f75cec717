"""Pins of the warm-start oracle: finite differences, bf16 rounding, features by hand."""
import numpy as np
import pytest

import s3synth
from oracle import mlp


def test_bf16_rounding_known_values():
    # bfloat16 keeps 8 significant bits: the spacing just above 1 is 2^-7
    x = np.array([1.0078125, 1.00390625, 1.01171875, 3.14159265, -2.5, 65504.0, 1e-3], dtype=np.float32)
    r = mlp.to_bf16(x)
    # 1 + 2^-7 is exact; 1 + 2^-8 ties between 1 and 1 + 2^-7 (to even: 1);
    # 1 + 3 2^-8 ties between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert list(r[:3]) == [1.0078125, 1.0, 1.015625]
    assert r[3] == 3.140625 and r[4] == -2.5 and r[5] == 65536.0
    assert abs(r[6] - 1e-3) <= 2 ** -8 * 1e-3


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.to_bf16(rng.normal(0, 0.3, mlp.NP).astype(np.float32))
    feat = rng.uniform(0, 3, (40, mlp.F))
    target = rng.normal(0, 1, 40)
    L, g = mlp.loss_and_grad(p, feat, target)
    assert abs(L - mlp.loss_only(p, feat, target)) < 1e-14
    idx = np.concatenate([rng.choice(mlp.NP, 60, replace=False), [mlp.OB3, mlp.OW3, mlp.OB1]])
    h = 1e-6
    for i in idx:
        a, b = p.copy(), p.copy()
        a[i] += h
        b[i] -= h
        fd = (mlp.loss_only(a, feat, target) - mlp.loss_only(b, feat, target)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_is_sign_times_lr():
    # bias correction makes the first Adam step -lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    p, m1, m2 = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-5)


def test_features_by_hand_on_fig1():
    hg = s3synth.fig1_example()   # edges (0-based): (1,2,3,6) (0,2,3,5) (0,1,2,7) (3,4,5,6) (0,3,5) (4,6)
    f = mlp.features(hg, N=4)
    deg = np.array([3, 2, 3, 4, 2, 3, 3, 1])
    assert np.allclose(f[:, 0], np.log1p(deg))
    # node 4 (1-based 5) is in (4,5,6,7) and (5,7): mean size 3, max 4
    assert np.isclose(f[4, 1], np.log1p(3.0)) and np.isclose(f[4, 2], np.log1p(4.0))
    # bins at N = 4: size 2 -> 0, size 3 -> floor(8 log1.5/log2) = 4, size 4 -> 7 (clamped)
    assert mlp.size_bin(2, 4) == 0 and mlp.size_bin(3, 4) == 4 and mlp.size_bin(4, 4) == 7
    assert np.isclose(f[4, 3], np.log1p(1)) and np.isclose(f[4, 10], np.log1p(1))
    # summed neighbour degree of node 7 (1-based 8), only in (1,2,3,8): deg 0,1,2 = 3+2+3
    assert np.isclose(f[7, 11], np.log1p(8.0))
