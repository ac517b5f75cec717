"""Pins of the shifted power method (Z-eigenpairs) and greedy symmetric CP oracle.

* Order 2 (a graph: every edge of size 2, B = the adjacency matrix): SS-HOPM is the
  shifted power method, so it must find the largest eigenvalue of A and its Perron
  vector (numpy's dense symmetric eigensolver); greedy symmetric CP with a shift
  larger than |lambda_min| finds the R largest eigenpairs.
* A d-regular N-uniform hypergraph: B 1^(N-1) = d 1, so the uniform unit vector is
  a Z-eigenvector with lambda = d n^(-(N-2)/2), reached in the first step.
* Non-uniform hypergraphs: at convergence the Z-eigen equation holds,
  ||B x^(N-1) - lambda x|| small, and lambda = x . B x^(N-1) is the largest value
  seen (SS-HOPM with alpha >= 0 increases lambda on this nonnegative tensor).
"""
import numpy as np

import oracle
import s3synth
from oracle.sshopm import sshopm, symmetric_cp


def _graph(n=60, m=240, seed=3):
    rng = np.random.default_rng(seed)
    edges = set()
    for i in range(n):                          # a cycle plus chords: connected
        edges.add((i, (i + 1) % n))
    edges.add((0, 2))                            # a triangle: not bipartite
    while len(edges) < m:
        a, b = rng.choice(n, 2, replace=False)
        edges.add((int(min(a, b)), int(max(a, b))))
    hg = s3synth.from_edges(n, sorted(edges))
    A = np.zeros((n, n))
    for a, b in hg.edges():
        A[a, b] = A[b, a] = 1.0
    return hg, A


def test_order_two_is_the_power_method():
    hg, A = _graph()
    w, V = np.linalg.eigh(A)
    r = sshopm(hg, alpha=0.0, tol=1e-15, max_iter=20000)
    assert r.converged
    assert abs(r.lam - w[-1]) <= 1e-10 * w[-1]
    v = V[:, -1] * np.sign(V[:, -1].sum())
    assert np.max(np.abs(r.x - v)) <= 1e-5


def test_order_two_cp_is_the_top_eigenpairs():
    hg, A = _graph(seed=4)
    w, V = np.linalg.eigh(A)
    rng = np.random.default_rng(0)
    starts = [rng.uniform(0.5, 1.5, hg.n) for _ in range(3)]
    comps = symmetric_cp(hg, 3, alpha=float(-w[0]) + 1.0, tol=1e-15, max_iter=200000, starts=starts)
    for r, (lam, x) in enumerate(comps):
        assert abs(lam - w[-1 - r]) <= 1e-8 * w[-1], (r, lam, w[-1 - r])
        assert abs(abs(np.dot(x, V[:, -1 - r])) - 1.0) <= 1e-6


def test_regular_uniform_hypergraph_closed_form():
    n, N = 40, 4
    edges = [tuple((i + k) % n for k in range(N)) for i in range(n)]   # every node in N edges
    hg = s3synth.from_edges(n, edges)
    r = sshopm(hg, tol=1e-14)
    assert abs(r.history[0] - N * n ** (-(N - 2) / 2)) <= 1e-14 * r.history[0]
    assert np.allclose(r.x, 1 / np.sqrt(n), rtol=1e-14) and r.iters == 1


def test_nonuniform_eigen_equation_and_monotone_lambda():
    for seed, (n, m, rank) in enumerate([(200, 600, 4), (300, 1200, 6)]):
        hg = s3synth.config_powerlaw(n=n, m=m, rank=rank, seed=seed + 5)
        lcc, _ = s3synth.largest_component(hg)
        r = sshopm(lcc, alpha=1.0, tol=1e-15, max_iter=50000)
        assert r.converged
        z = oracle.ttsv1(lcc, r.x)
        assert np.linalg.norm(z - r.lam * r.x) <= 1e-6 * r.lam
        assert all(b >= a - 1e-12 * abs(b) for a, b in zip(r.history, r.history[1:]))


def test_deflation_applies_the_rank_one_terms():
    hg, A = _graph(seed=5)
    x = np.random.default_rng(1).uniform(0, 1, hg.n)
    x /= np.linalg.norm(x)
    comps = symmetric_cp(hg, 1, tol=1e-14, max_iter=100000)
    lam1, x1 = comps[0]
    r = sshopm(hg, tol=1e-14, max_iter=1, x0=x, deflate=comps)
    # one step from x on A - lam1 x1 x1^T
    z = A @ x - lam1 * np.dot(x1, x) * x1
    want = np.dot(z / np.linalg.norm(z), (A - lam1 * np.outer(x1, x1)) @ (z / np.linalg.norm(z)))
    assert abs(r.history[1] - want) <= 1e-12 * max(1.0, abs(want))
