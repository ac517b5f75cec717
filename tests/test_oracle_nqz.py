"""Pins of the FP64 NQZ oracle (Algorithm 1)."""
import numpy as np
import pytest

import oracle
import s3synth
from oracle.nqz import nqz


def regular_hypergraph(n, d, lo, hi, seed):
    """d independent random partitions of the node set into blocks of size lo..hi."""
    rng = np.random.default_rng(seed)
    edges = []
    for _ in range(d):
        perm = rng.permutation(n)
        pos = 0
        while pos < n:
            s = int(rng.integers(lo, hi + 1))
            if n - pos - s < lo:
                s = n - pos
            edges.append(tuple(int(v) for v in perm[pos:pos + s]))
            pos += s
    return s3synth.from_edges(n, edges)


def test_regular_hypergraph_uniform_vector():
    # H1: in a d-regular hypergraph B x^(N-1) = d x^[N-1] for uniform x (B 1 = d, homogeneity)
    hg = regular_hypergraph(200, 5, 2, 6, 1)
    assert np.all(hg.degrees() == 5)
    res = nqz(hg, tol=1e-12)
    assert res.converged and res.iters == 1
    assert np.allclose(res.x, 1.0 / hg.n, rtol=1e-13)
    assert abs(res.lam - 5.0) < 1e-12


def test_graph_case_is_perron_vector():
    # H2: N=2 on a connected non-bipartite graph: NQZ is the power method and
    # converges to the Perron vector of the adjacency matrix
    rng = np.random.default_rng(3)
    n = 120
    edges = {(0, 1), (1, 2), (0, 2)}
    for v in range(3, n):                      # a random tree keeps it connected
        edges.add((int(rng.integers(0, v)), v))
    while len(edges) < 500:
        a, b = rng.choice(n, size=2, replace=False)
        edges.add((int(min(a, b)), int(max(a, b))))
    hg = s3synth.from_edges(n, sorted(edges))
    A = np.zeros((n, n))
    for a, b in edges:
        A[a, b] = A[b, a] = 1.0
    w, V = np.linalg.eigh(A)
    p = np.abs(V[:, -1])
    p /= p.sum()
    res = nqz(hg, tol=1e-11, max_iter=100000)
    assert res.converged
    assert abs(res.lam - w[-1]) < 1e-9 * w[-1]
    assert np.max(np.abs(res.x - p) / p) < 1e-7


def test_bracket_contains_eigenvalue():
    # H3: min and max of z ./ x^[N-1] bracket the H-eigenvalue at every step
    hg, _ = s3synth.largest_component(s3synth.config_small(seed=1))
    res = nqz(hg, tol=1e-12)
    assert res.converged
    lam = res.lam
    for lo, hi in res.history:
        assert lo <= lam * (1 + 1e-12) and hi >= lam * (1 - 1e-12)
    # the converged pair satisfies the eigen-equation
    y = oracle.ttsv1(hg, res.x)
    assert np.max(np.abs(y / res.x ** (hg.rank - 1) - lam)) < 1e-11 * lam


def test_start_vector_does_not_change_limit():
    hg, _ = s3synth.largest_component(s3synth.config_small(seed=4))
    a = nqz(hg, tol=1e-12)
    b = nqz(hg, tol=1e-12, x0=s3synth.x_uniform(hg.n, 0.5, 2.0, 9))
    assert a.converged and b.converged
    assert np.max(np.abs(a.x - b.x) / a.x) < 1e-9
