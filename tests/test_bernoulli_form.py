"""The Bernoulli form of the leave-one-out, checked on the CPU.

The Bernoulli kernels evaluate, for an edge e of size s at rank N (W = N-s+1),
    c(e, v_i) / K(s,N) = (prod_{j != i} x_j) * sum_{k<W} G[W-1-k] beta_k x_i^k,
with G = prod_j g_{x_j} truncated to W coefficients, g_x(t) = (e^(x t) - 1)/(x t),
and beta_k = B_k^+ / k! the coefficients of z / (1 - e^(-z)).  That rests on
E(x t) / Ebar(x t) = 1 / (1 - e^(-x t)) (Sec. II-A's E and Ebar).  G itself is
formed from the power sums p_k = sum_j x_j^k: log g_x(t) has the coefficients
beta_k x^k / k (its derivative is sum_k beta_k x^k t^(k-1)), so G = exp(sum_k
beta_k p_k t^k / k), i.e. G_0 = 1, G_m = (1/m) sum_{k=1}^m beta_k p_k G_{m-k}.
These tests
  * check beta_k against the Bernoulli numbers B_k (exact rationals, from their
    defining recurrence),
  * check both identities in exact rationals -- the recurrence against the
    product, and the per-member sum against the oracle's generating-function
    value of Algorithm 2 -- for edges of every size at several ranks, zeros included,
  * replay the FP32 kernel's operation order in numpy float32 (G as a product of
    the members' series in Horner form, the x^4-Horner split of the sum into its
    positive part P and negative part Q, P / x_i) and check that every member the
    gate (P + Q <= 4 (P - Q)) accepts is within the FP32 tolerance of the exact
    value, and that the gate rejects badly conditioned edges,
  * replay the FP64 kernel's order (power sums by a binary tree of products, the
    recurrence for G in float64, its error majorant in float32, the gate
    maj <= 64 (P - Q)) and check that accepted members are within 1e-12 of the
    exact value and that a badly conditioned edge is rejected.
The GPU tests check the kernels themselves against the oracle.
"""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

from oracle import exact

F = np.float32


def bernoulli_plus(n):
    """B_0..B_n with B_1 = +1/2, from sum_{j<=m} C(m+1, j) B_j = 0 (B_1 = -1/2 convention)."""
    B = [Fraction(1)]
    for m in range(1, n + 1):
        B.append(-sum(comb(m + 1, j) * B[j] for j in range(m)) / (m + 1))
    B[1] = -B[1]
    return B


def beta_exact(n):
    return [b / factorial(k) for k, b in enumerate(bernoulli_plus(n))]


def test_beta_is_the_series_of_z_over_one_minus_exp():
    # z / (1 - e^-z) * (1 - e^-z) / z = 1: the Cauchy product of beta with
    # f_k = (-1)^k / (k+1)! is 1, 0, 0, ...
    beta = beta_exact(31)
    f = [Fraction((-1) ** k, factorial(k + 1)) for k in range(32)]
    for m in range(32):
        assert sum(beta[k] * f[m - k] for k in range(m + 1)) == (1 if m == 0 else 0)
    assert beta[:5] == [1, Fraction(1, 2), Fraction(1, 12), 0, Fraction(-1, 720)]
    assert all(beta[k] == 0 for k in range(3, 32, 2))


@pytest.mark.parametrize("N", [8, 17, 25])
def test_power_sum_recurrence_is_the_product(N):
    rng = np.random.default_rng(N + 100)
    for s in range(2, N + 1):
        W = N - s + 1
        beta = beta_exact(max(W - 1, 1))
        xs = [Fraction(int(v), 16) for v in rng.integers(1, 40, size=s)]
        G = [Fraction(1)] + [Fraction(0)] * (W - 1)
        for xj in xs:
            g = [xj ** k / factorial(k + 1) for k in range(W)]
            G = [sum(G[m - k] * g[k] for k in range(m + 1)) for m in range(W)]
        p = [sum(xj ** k for xj in xs) for k in range(W)]
        R = [Fraction(1)] + [Fraction(0)] * (W - 1)
        for m in range(1, W):
            R[m] = sum(beta[k] * p[k] * R[m - k] for k in range(1, m + 1)) / m
        assert R == G, (N, s)


def bern_exact(xs, i, N):
    s = len(xs)
    W = N - s + 1
    beta = beta_exact(max(W - 1, 1))
    G = [Fraction(1)] + [Fraction(0)] * (W - 1)
    for xj in xs:
        g = [Fraction(xj) ** k / factorial(k + 1) for k in range(W)]
        G = [sum(G[m - k] * g[k] for k in range(m + 1)) for m in range(W)]
    prod = Fraction(1)
    for j, xj in enumerate(xs):
        if j != i:
            prod *= Fraction(xj)
    return prod * sum(G[W - 1 - k] * beta[k] * Fraction(xs[i]) ** k for k in range(W))


@pytest.mark.parametrize("N", [6, 9, 13])
def test_identity_matches_algorithm2_exactly(N):
    rng = np.random.default_rng(N)
    for s in range(2, N + 1):
        for trial in range(2):
            xs = [Fraction(int(v), 8) for v in rng.integers(0, 17, size=s)]
            if trial == 1:
                xs[0] = Fraction(0)           # a zero member
            edge = tuple(range(s))
            for i in range(s):
                # Algorithm 2's per-pair value divided by its scale K(s,N)
                want = exact.contribution_gf(edge, i, {v: xs[v] for v in edge}, N) / exact.edge_scale(N, s)
                assert bern_exact(xs, i, N) == want, (N, s, i)


def bern_fp32(a, W):
    """(values, P, Q) per member in the kernels' FP32 order; a: the already scaled x."""
    s = len(a)
    beta = [F(float(b)) for b in beta_exact(max(W - 1, 1))]
    x0 = a[0]
    G = [F(1)] + [F(0)] * (W - 1)
    for k in range(1, W):
        G[k] = F(G[k - 1] * F(x0 * F(1.0 / (k + 1))))
    pre = [F(1)] * s
    prod = x0
    for i in range(1, s):
        xi = a[i]
        pre[i] = prod
        prod = F(prod * xi)
        r = [F(0)] + [F(xi * F(1.0 / (k + 1))) for k in range(1, W)]
        for m in range(W - 1, 0, -1):
            t = G[0]
            for j in range(1, m + 1):
                t = F(np.float32(np.float64(r[m - j + 1]) * np.float64(t) + np.float64(G[j])))  # one rounding
            G[m] = t
    H = [F(G[W - 1 - k] * beta[k]) for k in range(W)]
    fma = lambda a_, b_, c_: F(np.float64(a_) * np.float64(b_) + np.float64(c_))
    vals, Ps, Qs = [F(0)] * s, [F(0)] * s, [F(0)] * s
    suf = F(1)
    for i in range(s - 1, -1, -1):
        xi = a[i]
        x2 = F(xi * xi)
        x4 = F(x2 * x2)
        p2 = F(0)
        if W > 2:
            for k in range(2 + 4 * ((W - 3) // 4), 1, -4):
                p2 = fma(p2, x4, H[k])
        p = H[0]
        if W > 1:
            p = fma(H[1], xi, p)
        P = fma(p2, x2, p)
        q = F(0)
        if W > 4:
            for k in range(4 + 4 * ((W - 5) // 4), 3, -4):
                q = fma(q, x4, F(-H[k]))
            q = F(q * x4)
        vals[i] = F(F(P - q) * F(pre[i] * suf))
        Ps[i], Qs[i] = P, q
        suf = F(suf * xi)
    return vals, Ps, Qs


@pytest.mark.parametrize("N", [12, 25])
def test_fp32_replay_within_tolerance_when_the_gate_accepts(N):
    rng = np.random.default_rng(7 + N)
    accepted = rejected = 0
    for s in range(6, N + 1):
        W = N - s + 1
        for spread in (1.2, 2.0, 4.0, 16.0):
            # x near 1 / s (the kernels scale each edge by a power of two), members up to
            # `spread` times apart
            raw = rng.uniform(1.0, spread, size=s) / s
            a = [F(v) for v in raw]
            vals, P, Q = bern_fp32(a, W)
            ok = all(float(P[i] + Q[i]) <= 4.0 * float(P[i] - Q[i]) for i in range(s))
            if not ok:
                rejected += 1
                continue
            accepted += 1
            for i in range(s):
                want = bern_exact([Fraction(float(v)) for v in a], i, N)
                err = abs(Fraction(float(vals[i])) - want) / want
                assert err <= Fraction(1, 10 ** 5), (N, s, spread, i, float(err))
    assert accepted > 0


def test_gate_rejects_badly_conditioned_edges():
    # one member 40 times the others at s = 6, N = 25: the alternating sum cancels
    a = [F(0.02)] * 5 + [F(0.8)]
    vals, P, Q = bern_fp32(a, 20)
    assert any(float(P[i] + Q[i]) > 4.0 * float(P[i] - Q[i]) for i in range(6))


def bern_exact_all(xs, N):
    """Every member's exact value of the Bernoulli form (G formed once)."""
    s = len(xs)
    W = N - s + 1
    beta = beta_exact(max(W - 1, 1))
    G = [Fraction(1)] + [Fraction(0)] * (W - 1)
    for xj in xs:
        g = [Fraction(xj) ** k / factorial(k + 1) for k in range(W)]
        G = [sum(G[m - k] * g[k] for k in range(m + 1)) for m in range(W)]
    total = Fraction(1)
    for xj in xs:
        total *= Fraction(xj)
    return [total / Fraction(xs[i]) * sum(G[W - 1 - k] * beta[k] * Fraction(xs[i]) ** k for k in range(W))
            for i in range(s)]


def bern_fp64(a, W):
    """(values, accepted) per member in the FP64 kernel's order: power sums and the recurrence
    for G in float64, the error majorant A in float32, the gate maj * 1.0001 <= 64 (P - Q)."""
    D, S = np.float64, np.float32
    beta = [D(float(b)) for b in beta_exact(max(W - 1, 1))]
    q = [D(0)] * W
    prod = D(1)
    for xi in a:
        prod = D(prod * xi)
        pw = [D(1), D(xi)] + [D(0)] * max(W - 2, 0)
        for k in range(2, W):
            pw[k] = D(pw[k // 2] * pw[k - k // 2])
        for k in range(1, W):
            q[k] = D(q[k] + pw[k])
    for k in range(1, W):
        q[k] = D(q[k] * beta[k])
    qa = [S(abs(v)) for v in q]
    G, A = [D(1)] + [D(0)] * (W - 1), [S(1)] + [S(0)] * (W - 1)
    for m in range(1, W):
        acc, acca = D(0), S(0)
        for k in range(m, 0, -1):
            acc = D(q[k] * G[m - k] + acc)
            acca = S(np.float64(qa[k]) * np.float64(A[m - k]) + np.float64(acca))
        G[m] = D(acc * D(1.0 / m))
        A[m] = S(acca * S(1.0 / m))
    H = [D(G[W - 1 - k] * beta[k]) for k in range(W)]
    Ha = [S(A[W - 1 - k] * S(abs(float(beta[k])))) for k in range(W)]
    vals, ok = [], []
    for xi in a:
        x2 = D(xi * xi)
        x4 = D(x2 * x2)
        p2 = D(0)
        if W > 2:
            for k in range(2 + 4 * ((W - 3) // 4), 1, -4):
                p2 = D(p2 * x4 + H[k])
        p = H[0]
        if W > 1:
            p = D(H[1] * xi + p)
        P = D(p2 * x2 + p)
        qn = D(0)
        if W > 4:
            for k in range(4 + 4 * ((W - 5) // 4), 3, -4):
                qn = D(qn * x4 - H[k])
            qn = D(qn * x4)
        v = D(P - qn)
        xf = S(xi)
        xf2 = S(xf * xf)
        maj = S(0)
        for k in range(2 * ((W - 1) // 2), -1, -2):
            maj = S(maj * xf2 + Ha[k])
        if W > 1:
            maj = S(Ha[1] * xf + maj)
        ok.append(float(maj) * 1.0001 <= 64.0 * float(v))
        vals.append(D(v * D(prod / xi)))
    return vals, ok


@pytest.mark.parametrize("N", [12, 25])
def test_fp64_replay_within_tolerance_when_the_gate_accepts(N):
    # the FP64 kernel's power-sum recurrence with its FP32 majorant: every member the gate
    # accepts is within the FP64 tolerance of the exact value
    rng = np.random.default_rng(11 + N)
    accepted = rejected = 0
    for s in range(6, N + 1):
        W = N - s + 1
        for spread in (1.2, 2.0, 4.0, 16.0, 64.0):
            a = [np.float64(v) for v in rng.uniform(1.0, spread, size=s) / s]
            vals, ok = bern_fp64(a, W)
            if not all(ok):
                rejected += 1
                continue
            accepted += 1
            want = bern_exact_all([Fraction(float(v)) for v in a], N)
            for i in range(s):
                err = abs(Fraction(float(vals[i])) - want[i]) / want[i]
                assert err <= Fraction(1, 10 ** 12), (N, s, spread, i, float(err))
    assert accepted > 0


def test_fp64_gate_rejects_badly_conditioned_edges():
    # one member 200 times the others at s = 6, N = 25: the recurrence cancels beyond what the
    # majorant allows
    a = [np.float64(0.004)] * 5 + [np.float64(0.8)]
    _, ok = bern_fp64(a, 20)
    assert not all(ok)
