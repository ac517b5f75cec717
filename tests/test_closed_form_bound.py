"""The error bound behind the closed-form gate, checked on the CPU.

The closed-form kernels evaluate, for an edge e of size s at rank N (n = N-1),
    R_v = sum over subsets U of e containing v of (-1)^(s-|U|) sigma_U^n,
(the inclusion-exclusion form of Sec. II-A's E(x_v) prod Ebar(x_u); the oracle
pins its equality with the generating function exactly) and accept an edge only
when every R_v > (C u / tau) A, relying on |computed R_v - R_v| <= C u A with
A = sum_U sigma_U^n, C = n + 2^(s-1) + 4 for FP32 with compensated subset sums.

This test replays that FP32 arithmetic step by step in numpy float32 (IEEE
round-to-nearest, the same operation order: subsets by increasing mask, each sum
built from the mask without its lowest member, left-to-right binary powering,
first-order correction n lo / hi) and checks the bound against exact rationals,
on well-conditioned edges and on edges the gate is meant to reject.  The GPU
tests check the kernels themselves against the oracle.
"""
from fractions import Fraction

import numpy as np
import pytest

F = np.float32


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def fp32_power(h, n):
    r = h
    for bit in bin(n)[3:]:
        r = F(r * r)
        if bit == "1":
            r = F(r * h)
    return r


def closed_form_fp32(a, n):
    """(R_v for every member, A) in the kernels' FP32 operation order; a already scaled."""
    s = len(a)
    hi = [F(0)] * (1 << s)
    lo = [F(0)] * (1 << s)
    R = [F(0)] * s
    A = F(0)
    for mask in range(1, 1 << s):
        low = mask & -mask
        i = low.bit_length() - 1
        par = mask ^ low
        if par == 0:
            hi[mask], lo[mask] = a[i], F(0)
        else:
            sm, err = two_sum(hi[par], a[i])
            hi[mask], lo[mask] = sm, F(lo[par] + err)
        pw = fp32_power(hi[mask], n)
        if par != 0:
            corr = F(F(F(n) * lo[mask]) / max(hi[mask], F(np.finfo(F).tiny)))
            pw = F(np.float64(pw) * np.float64(corr) + np.float64(pw))  # one rounding, as an FMA
        A = F(A + pw)
        neg = (s - bin(mask).count("1")) % 2 == 1
        for v in range(s):
            if mask >> v & 1:
                R[v] = F(R[v] - pw) if neg else F(R[v] + pw)
    return R, A


def exact_R(a, n):
    s = len(a)
    q = [Fraction(float(v)) for v in a]
    out = []
    for v in range(s):
        tot = Fraction(0)
        for mask in range(1, 1 << s):
            if mask >> v & 1:
                sign = -1 if (s - bin(mask).count("1")) % 2 else 1
                tot += sign * sum(q[i] for i in range(s) if mask >> i & 1) ** n
        out.append(tot)
    return out


def scaled(x):
    """x times the power of two that puts its sum in [1, 2), as the kernels scale it."""
    e = np.frexp(np.float32(x.sum(dtype=np.float32)))[1]
    return (x * np.float32(2.0 ** (1 - int(e)))).astype(F)


@pytest.mark.parametrize("N", [8, 25, 33])
@pytest.mark.parametrize("s", [2, 3, 4, 5, 6])
def test_fp32_bound_holds(s, N):
    n = N - 1
    C = n + 2 ** (s - 1) + 4
    u = 2.0 ** -24
    rng = np.random.default_rng(1000 * s + N)
    worst = 0.0
    for trial in range(40):
        kind = trial % 4
        if kind == 0:
            x = rng.uniform(0.9, 1.1, s)                  # near-uniform: accepted
        elif kind == 1:
            x = rng.uniform(0.5, 1.5, s)
        elif kind == 2:
            x = rng.uniform(0.0, 1.0, s)                  # occasionally ill-conditioned
        else:
            x = rng.uniform(0.0, 1.0, s) * 10.0 ** rng.integers(-6, 1, s)   # very different sizes
        a = scaled(x.astype(F))
        R, A = closed_form_fp32(a, n)
        ex = exact_R(a, n)
        for v in range(s):
            err = abs(Fraction(float(R[v])) - ex[v])
            bound = Fraction(C) * Fraction(u) * Fraction(float(A))
            assert err <= bound, f"s={s} N={N} x={x} v={v}: error {float(err):.3e} > bound {float(bound):.3e}"
            if float(A) > 0:
                worst = max(worst, float(err) / (C * u * float(A)))
    assert worst < 1.0


def test_gate_accepts_uniform_and_rejects_cancellation():
    # equal x pass with a wide margin; a member 1e-4 times the others makes the signed sum cancel
    n, s = 24, 4
    C = n + 2 ** (s - 1) + 4
    gate = C * 2.0 ** -24 / 2.0 ** -17
    R, A = closed_form_fp32(scaled(np.full(s, 0.7, dtype=F)), n)
    assert all(float(r) > gate * float(A) for r in R)
    R, A = closed_form_fp32(scaled(np.array([1.0, 0.9, 1.1, 1e-4], dtype=F)), n)
    assert any(float(r) <= gate * float(A) for r in R)
