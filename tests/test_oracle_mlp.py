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


def _hand_network():
    """A 12-64-64-1 network with all but a handful of weights zero (every value exact
    in bfloat16), and two feature rows for which the hand computation below holds."""
    p = np.zeros(mlp.NP)
    W1 = p[mlp.OW1:mlp.OB1].reshape(mlp.H, mlp.F)
    W2 = p[mlp.OW2:mlp.OB2].reshape(mlp.H, mlp.H)
    W1[0, 0], W1[0, 1], p[mlp.OB1 + 0] = 1.0, -1.0, 0.5
    W1[1, 0], W1[1, 1], p[mlp.OB1 + 1] = -0.5, 1.0, 0.25
    W2[0, 0], W2[0, 1], p[mlp.OB2 + 0] = 2.0, 3.0, -1.0
    W2[1, 0], W2[1, 1], p[mlp.OB2 + 1] = -1.0, 0.5, 0.5
    p[mlp.OW3 + 0], p[mlp.OW3 + 1], p[mlp.OB3] = 1.5, -2.0, 0.125
    feat = np.zeros((2, mlp.F))
    feat[0, :2] = (1.0, 2.0)
    feat[1, :2] = (3.0, 0.5)
    return p, feat


def test_forward_matches_hand_computation():
    # Worked by hand, row A = (1, 2, 0, ...), row B = (3, 0.5, 0, ...):
    #   layer 1  z1 = W1 f + b1:  A: (1-2+0.5, -0.5+2+0.25) = (-0.5, 1.75) -> h1 = (0, 1.75)
    #                             B: (3-0.5+0.5, -1.5+0.5+0.25) = (3, -0.75) -> h1 = (3, 0)
    #   layer 2  z2 = W2 h1 + b2: A: (0+5.25-1, 0+0.875+0.5) = (4.25, 1.375) -> h2 = (4.25, 1.375)
    #                             B: (6+0-1, -3+0+0.5) = (5, -2.5)           -> h2 = (5, 0)
    #   output   y = W3 h2 + b3:  A: 6.375 - 2.75 + 0.125 = 3.75;  B: 7.5 + 0.125 = 7.625
    # (W2 applied transposed gives A: z2 = (-2.75, ...); dropping b1 gives z1_A[1] = 1.5; a
    # missing ReLU after layer 1 gives z2_A[0] = 4.25 - 0 ... with h1_A[0] = -0.5: 3.25.)
    p, feat = _hand_network()
    y, (h1, h2) = mlp.forward(p, feat)
    assert y.tolist() == [3.75, 7.625]
    assert h1[0, :2].tolist() == [0.0, 1.75] and h1[1, :2].tolist() == [3.0, 0.0]
    assert h2[0, :2].tolist() == [4.25, 1.375] and h2[1, :2].tolist() == [5.0, 0.0]
    assert not np.any(h1[:, 2:]) and not np.any(h2[:, 2:])


def test_loss_and_output_gradient_by_hand():
    # targets 3.25 and 7.125: residuals d = (0.5, 0.5), L = mean d^2 = 0.25;
    # dL/db3 = (2/n) sum d = 1; dL/dW3[0] = (2/n) sum d h2[:,0] = 0.5*4.25 + 0.5*5 = 4.625;
    # dL/dW3[1] = 0.5*1.375 + 0 = 0.6875; dL/db2[1] = (2/n) sum d W3[1] [z2 > 0] = 0.5*(-2) = -1
    p, feat = _hand_network()
    L, g = mlp.loss_and_grad(p, feat, np.array([3.25, 7.125]))
    assert L == 0.25
    assert g[mlp.OB3] == 1.0 and g[mlp.OW3] == 4.625 and g[mlp.OW3 + 1] == 0.6875
    assert g[mlp.OB2 + 1] == -1.0


def test_adam_two_steps_by_hand():
    # gradients 0.5 then -0.25, lr 0.01, beta1 0.9, beta2 0.999, eps 0:
    #   step 1: m = 0.05, v = 0.00025; bias-corrected 0.5 and 0.25 -> p = -0.01 * 0.5/0.5 = -0.01
    #   step 2: m = 0.045 - 0.025 = 0.02, v = 0.00024975 + 0.0000625 = 0.00031225;
    #           corrections 1 - 0.81 = 0.19 and 1 - 0.998001 = 0.001999;
    #           p = -0.01 - 0.01 * 0.1052631579 / 0.3952253838 = -0.0126633704
    p, m1, m2 = mlp.adam_step(np.zeros(1), np.zeros(1), np.zeros(1), np.array([0.5]), 1, lr=0.01, eps=0.0)
    close = lambda a, b: abs(a - b) <= 1e-14 * abs(b)
    assert close(p[0], -0.01) and close(m1[0], 0.05) and close(m2[0], 0.00025)
    p, m1, m2 = mlp.adam_step(p, m1, m2, np.array([-0.25]), 2, lr=0.01, eps=0.0)
    assert close(m1[0], 0.02) and close(m2[0], 0.00031225)
    assert abs(p[0] - (-0.0126633704)) < 1e-10
