"""Exact rational S^3TTVc on the blowup tensor (test infrastructure only).

Everything here is plain Python integers and ``fractions.Fraction``; it is
slow and meant for hypergraphs with a handful of nodes.  Three independent
evaluations of the same operation live here so that each can pin the others:

* ``ttsv1_bruteforce`` -- Eq. (2) applied to every entry of the blowup tensor
  B, which is enumerated from its definition in Sec. II (the set beta(e) of
  N-tuples over e that use every node of e, each entry w(e)/|beta(e)|,
  w(e) = |e|).
* ``ttsv1_generating_function`` -- Algorithm 2 (AAY): for every node v and
  edge e containing v, the coefficient of t^(N-1) in
  E_N(b_v) * conv_{u in e minus v} Ebar_N(b_u), scaled by
  w(e)/|beta(e)| * (N-1)!  (Sec. II-A).
* ``contribution_inclusion_exclusion`` -- the same per-(e, v) value written
  as an alternating sum over subsets (a finite difference of z^(N-1)).

Readings of the paper used here (see the design notes): N is the rank
(largest edge size) unless given; w(e) = |e| (Sec. II, so that B 1^(N-1) is
the degree vector); a hypergraph may list the same edge twice and the
contributions then add.
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from math import comb, factorial

__all__ = [
    "stirling2", "blowup_count", "blowup_tuples", "blowup_tensor",
    "ttsv1_bruteforce", "ttsv1_generating_function", "contribution_gf",
    "contribution_inclusion_exclusion", "edge_scale", "energy_bruteforce",
    "energy_inclusion_exclusion",
]


def stirling2(n: int, k: int) -> int:
    """Stirling number of the second kind S(n, k) by its explicit sum."""
    if n < 0 or k < 0:
        raise ValueError
    if k == 0:
        return 1 if n == 0 else 0
    total = sum((-1) ** j * comb(k, j) * (k - j) ** n for j in range(k + 1))
    assert total % factorial(k) == 0
    return total // factorial(k)


def blowup_count(N: int, s: int) -> int:
    """|beta(e)| = |e|! S(N, |e|)  (footnote to the definition of beta in Sec. II)."""
    return factorial(s) * stirling2(N, s)


def blowup_tuples(edge, N):
    """beta(e): all N-tuples over the nodes of e in which every node of e occurs."""
    es = set(edge)
    for t in itertools.product(sorted(es), repeat=N):
        if set(t) == es:
            yield t


def edge_scale(N: int, s: int) -> Fraction:
    """w(e)/|beta(e)| * (N-1)! with w(e) = |e| (the scaling in Algorithm 2)."""
    return Fraction(s * factorial(N - 1), blowup_count(N, s))


def blowup_tensor(edges, N):
    """Sparse dict {index tuple: value} of the order-N blowup tensor (Sec. II)."""
    B = {}
    for e in edges:
        s = len(e)
        if len(set(e)) != s:
            raise ValueError("repeated node inside an edge")
        val = Fraction(s, blowup_count(N, s))
        for t in blowup_tuples(e, N):
            B[t] = B.get(t, Fraction(0)) + val
    return B


def ttsv1_bruteforce(n, edges, x, N):
    """Eq. (2): s_{i1} = sum over i2..iN of B[i1..iN] * prod_k x[i_k]."""
    B = blowup_tensor(edges, N)
    y = [Fraction(0)] * n
    for t, val in B.items():
        p = Fraction(1)
        for i in t[1:]:
            p *= x[i]
        y[t[0]] += val * p
    return y


def _egf(c, N, bar):
    """E_N(c) = [1, c, c^2/2!, ..., c^(N-1)/(N-1)!]; Ebar_N(c) has 0 in slot 0."""
    out = [Fraction(c) ** k / factorial(k) for k in range(N)]
    if bar:
        out[0] = Fraction(0)
    return out


def _conv(a, b, N):
    """(a * b)[k] = sum_{i<=k} a_i b_{k-i}, kept for k < N."""
    return [sum(a[i] * b[k - i] for i in range(k + 1)) for k in range(N)]


def contribution_gf(e, v, x, N):
    """Contribution of edge e to node v by the generating function (Algorithm 2)."""
    coefs = _egf(x[v], N, bar=False)
    for u in e:
        if u != v:
            coefs = _conv(coefs, _egf(x[u], N, bar=True), N)
    return edge_scale(N, len(e)) * coefs[N - 1]


def ttsv1_generating_function(n, edges, x, N):
    """Algorithm 2 (AAY) in exact arithmetic, node by node."""
    y = [Fraction(0)] * n
    for e in edges:
        for v in e:
            y[v] += contribution_gf(e, v, x, N)
    return y


def contribution_inclusion_exclusion(e, v, x, N):
    """Same contribution as a signed subset sum.

    The number-weighted count of (N-1)-sequences over e that cover e minus v is
    sum_{T subset of e minus v} (-1)^(|e|-1-|T|) (x_v + sum_T x)^(N-1).
    """
    rest = [u for u in e if u != v]
    s = len(e)
    total = Fraction(0)
    for r in range(len(rest) + 1):
        for T in itertools.combinations(rest, r):
            z = Fraction(x[v]) + sum((Fraction(x[u]) for u in T), Fraction(0))
            total += (-1) ** (len(rest) - r) * z ** (N - 1)
    return Fraction(s, blowup_count(N, s)) * total


def energy_bruteforce(n, edges, x, N):
    """B x^N = sum over all tensor entries of B[i] prod x[i_k]."""
    B = blowup_tensor(edges, N)
    tot = Fraction(0)
    for t, val in B.items():
        p = Fraction(1)
        for i in t:
            p *= x[i]
        tot += val * p
    return tot


def energy_inclusion_exclusion(edges, x, N):
    """B x^N edge by edge: |e|/|beta(e)| * sum_{T subset e} (-1)^(|e|-|T|) (sum_T x)^N."""
    tot = Fraction(0)
    for e in edges:
        s = len(e)
        acc = Fraction(0)
        for r in range(s + 1):
            for T in itertools.combinations(e, r):
                acc += (-1) ** (s - r) * sum((Fraction(x[u]) for u in T), Fraction(0)) ** N
        tot += Fraction(s, blowup_count(N, s)) * acc
    return tot
