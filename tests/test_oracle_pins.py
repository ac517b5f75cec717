"""Pins of the CPU oracle against facts the paper and mathematics fix.

Each test checks the oracle against something other than itself: brute force
over every blowup-tensor entry, closed forms, a library routine, the paper's
worked example, or exact identities.
"""
import itertools
import json
import os
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import oracle
import s3synth
from oracle import ccss, exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))) if a.size else 0.0


# --------------------------------------------------------- combinatorics ---

def test_stirling_textbook_values():
    # S(n,k) table values (OEIS A008277)
    assert [exact.stirling2(4, k) for k in range(5)] == [0, 1, 7, 6, 1]
    assert exact.stirling2(5, 3) == 25
    assert exact.stirling2(10, 5) == 42525
    assert exact.stirling2(0, 0) == 1


@pytest.mark.parametrize("N", range(1, 7))
def test_blowup_count_matches_enumeration(N):
    # footnote of Sec. II: |beta(e)| = |e|! S(N,|e|); count the tuples directly
    for s in range(1, N + 1):
        e = tuple(range(10, 10 + s))
        brute = sum(1 for t in itertools.product(e, repeat=N) if set(t) == set(e))
        assert brute == exact.blowup_count(N, s)


def test_fig1_tensor_values():
    # Sec. II: every entry generated by e has value w(e)/|beta(e)|, w(e)=|e|;
    # at N=4 that is 4/24=1/6 (size 4), 3/36=1/12 (size 3), 2/14=1/7 (size 2).
    g = json.load(open(os.path.join(GOLD, "fig1_fig2.json")))
    N = g["rank"]
    expect = {4: Fraction(1, 6), 3: Fraction(1, 12), 2: Fraction(1, 7)}
    B = exact.blowup_tensor([tuple(e) for e in g["edges"]], N)
    per_edge = {}
    for t, val in B.items():
        key = tuple(sorted(set(t)))
        per_edge.setdefault(key, set()).add(val)
    for e in g["edges"]:
        vals = per_edge[tuple(sorted(e))]
        assert vals == {expect[len(e)]}
    # number of nonzeros = sum of |beta(e)|
    assert len(B) == sum(exact.blowup_count(N, len(e)) for e in g["edges"])


def test_fig2_ccss_structure():
    g = json.load(open(os.path.join(GOLD, "fig1_fig2.json")))
    edges = [tuple(e) for e in g["edges"]]
    lv = ccss.untrimmed_levels(edges)
    for l, paths in g["fig2_levels"].items():
        assert lv[int(l)] == {tuple(p) for p in paths}
    leaves = ccss.special_leaves(edges)
    names = g["edge_value_names"]
    got = {(path, v, names[i]) for path, L in leaves.items() for (v, i) in L}
    want = {(tuple(d["path"]), d["dropped"], d["value"]) for d in g["fig2_special_leaves"]}
    assert got == want
    assert ccss.level_counts(lv) == [8, 19, 16]
    assert ccss.level_counts(ccss.trimmed_levels(edges)) == [6, 10, 16]


# ----------------------------------------------------- exact formulations ---

@pytest.mark.parametrize("seed,N", [(0, 4), (1, 4), (2, 5), (5, 4)])
def test_bruteforce_equals_generating_function(seed, N):
    hg = s3synth.tiny_case(seed=seed, rank=4)
    rng = np.random.default_rng(seed)
    x = [Fraction(int(a), int(b)) for a, b in zip(rng.integers(1, 20, hg.n), rng.integers(1, 9, hg.n))]
    assert exact.ttsv1_bruteforce(hg.n, hg.edges(), x, N) == \
        exact.ttsv1_generating_function(hg.n, hg.edges(), x, N)


@pytest.mark.parametrize("s,N", [(1, 3), (2, 2), (2, 6), (3, 5), (4, 7), (5, 8), (6, 8)])
def test_inclusion_exclusion_equals_generating_function(s, N):
    rng = np.random.default_rng(100 * s + N)
    e = tuple(range(s))
    x = [Fraction(int(a), int(b)) for a, b in zip(rng.integers(1, 30, s), rng.integers(1, 7, s))]
    for v in e:
        assert exact.contribution_gf(e, v, x, N) == exact.contribution_inclusion_exclusion(e, v, x, N)


def test_energy_identity_exact():
    # x . (B x^(N-1)) = B x^N, the latter by an independent degree-N subset sum
    hg = s3synth.tiny_case(seed=3, rank=4)
    x = [Fraction(i + 2, 3) for i in range(hg.n)]
    for N in (4, 5):
        y = exact.ttsv1_bruteforce(hg.n, hg.edges(), x, N)
        lhs = sum(a * b for a, b in zip(x, y))
        assert lhs == exact.energy_bruteforce(hg.n, hg.edges(), x, N)
        assert lhs == exact.energy_inclusion_exclusion(hg.edges(), x, N)


def test_uniform_reduces_to_adjacency_tensor():
    # Sec. II: for an N-uniform hypergraph B is the adjacency tensor with entries w/N!
    # (w = N), so y_v = sum_{e containing v} prod_{u in e, u != v} x_u.
    N = 3
    rng = np.random.default_rng(9)
    edges = [tuple(rng.choice(7, size=N, replace=False)) for _ in range(9)]
    x = [Fraction(i + 1, 4) for i in range(7)]
    y = exact.ttsv1_bruteforce(7, edges, x, N)
    want = [Fraction(0)] * 7
    for e in edges:
        for v in e:
            p = Fraction(1)
            for u in e:
                if u != v:
                    p *= x[u]
            want[v] += p
    assert y == want


# ------------------------------------------------------------- FP64 oracle ---

def test_c_oracle_matches_golden_exact():
    g = json.load(open(os.path.join(GOLD, "tiny_exact.json")))
    for case in g["cases"]:
        hg = s3synth.from_edges(case["n"], [tuple(e) for e in case["edges"]])
        x = np.array([float(Fraction(v)) for v in case["x"]])
        y = oracle.ttsv1(hg, x, N=case["N"])
        want = np.array([float(Fraction(v)) for v in case["y"]])
        assert rel_err(y, want) < 1e-14
        # and the exact routines still reproduce the stored values
        xf = [Fraction(v) for v in case["x"]]
        assert [str(v) for v in exact.ttsv1_generating_function(case["n"], hg.edges(), xf, case["N"])] == case["y"]


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_c_oracle_matches_bruteforce(seed):
    hg = s3synth.tiny_case(seed=seed, rank=4)
    x = s3synth.x_uniform(hg.n, 0.1, 2.0, seed)
    want = exact.ttsv1_bruteforce(hg.n, hg.edges(), [Fraction(float(v)) for v in x], 4)
    assert rel_err(oracle.ttsv1(hg, x, N=4), [float(v) for v in want]) < 1e-14


def test_fig1_oracle_matches_bruteforce():
    hg = s3synth.fig1_example()
    x = s3synth.x_uniform(hg.n, 0.0, 1.0, 11)
    want = exact.ttsv1_bruteforce(hg.n, hg.edges(), [Fraction(float(v)) for v in x], 4)
    assert rel_err(oracle.ttsv1(hg, x, N=4), [float(v) for v in want]) < 1e-14


def test_ones_give_degrees_and_homogeneity():
    # Sec. II: with w(e)=|e|, B 1^(N-1) = d; homogeneity: B (c x)^(N-1) = c^(N-1) B x^(N-1)
    hg = s3synth.config_small(seed=1)
    d = hg.degrees().astype(np.float64)
    y = oracle.ttsv1(hg, np.ones(hg.n))
    assert rel_err(y[d > 0], d[d > 0]) < 1e-13
    c = 0.37
    y2 = oracle.ttsv1(hg, np.full(hg.n, c))
    assert rel_err(y2[d > 0], (c ** (hg.rank - 1)) * d[d > 0]) < 1e-13
    x = s3synth.x_uniform(hg.n, 0, 1, 3)
    assert rel_err(oracle.ttsv1(hg, 2.0 * x)[d > 0], 2.0 ** (hg.rank - 1) * oracle.ttsv1(hg, x)[d > 0]) < 1e-13


def test_graph_case_is_sparse_matvec():
    # N = 2 and all edges of size 2: B is the adjacency matrix, y = A x
    import scipy.sparse as sp
    rng = np.random.default_rng(4)
    n = 300
    edges = set()
    while len(edges) < 1500:
        a, b = rng.choice(n, size=2, replace=False)
        edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    hg = s3synth.from_edges(n, edges)
    r = [a for a, b in edges] + [b for a, b in edges]
    c = [b for a, b in edges] + [a for a, b in edges]
    A = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))
    x = rng.random(n)
    assert rel_err(oracle.ttsv1(hg, x, N=2), A @ x) < 1e-14


@pytest.mark.parametrize("N", [3, 4, 7])
def test_uniform_hypergraph_products(N):
    rng = np.random.default_rng(N)
    n = 60
    edges = [tuple(rng.choice(n, size=N, replace=False)) for _ in range(200)]
    hg = s3synth.from_edges(n, edges)
    x = rng.uniform(0.2, 1.5, n)
    want = np.zeros(n)
    for e in edges:
        for v in e:
            want[v] += np.prod([x[u] for u in e if u != v])
    assert rel_err(oracle.ttsv1(hg, x, N=N), want) < 1e-13


@pytest.mark.parametrize("N", [2, 3, 5, 10, 25, 40])
def test_size_two_closed_form(N):
    # one edge {a,b}: contribution to a is 2/(2^N-2) ((x_a+x_b)^(N-1) - x_a^(N-1)),
    # expanded into its positive binomial terms so no cancellation occurs
    hg = s3synth.from_edges(2, [(0, 1)])
    x = np.array([0.7, 1.3])
    y = oracle.ttsv1(hg, x, N=N)
    for v, u in ((0, 1), (1, 0)):
        a, b = Fraction(float(x[v])), Fraction(float(x[u]))
        exact_val = Fraction(2, 2 ** N - 2) * sum(comb(N - 1, k) * b ** k * a ** (N - 1 - k) for k in range(1, N))
        assert abs(y[v] - float(exact_val)) <= 1e-14 * float(exact_val)


def test_single_edge_bounds_and_inclusion_exclusion():
    # each contribution is an average of products of N-1 entries of x over e,
    # so it lies in [min x^(N-1), max x^(N-1)]; also equals the subset sum
    rng = np.random.default_rng(12)
    for trial in range(20):
        s = int(rng.integers(1, 7))
        N = int(rng.integers(max(s, 2), 10))
        x = rng.uniform(0.1, 2.0, s)
        hg = s3synth.from_edges(s, [tuple(range(s))])
        y = oracle.ttsv1(hg, x, N=N)
        lo, hi = x.min() ** (N - 1), x.max() ** (N - 1)
        assert np.all(y >= lo * (1 - 1e-13)) and np.all(y <= hi * (1 + 1e-13))
        xf = [Fraction(float(v)) for v in x]
        for v in range(s):
            ie = exact.contribution_inclusion_exclusion(tuple(range(s)), v, xf, N)
            assert abs(y[v] - float(ie)) <= 1e-13 * float(ie)


def test_energy_identity_fp64():
    hg = s3synth.tiny_case(seed=7, rank=4)
    x = s3synth.x_uniform(hg.n, 0.2, 1.5, 7)
    for N in (4, 6):
        y = oracle.ttsv1(hg, x, N=N)
        want = exact.energy_inclusion_exclusion(hg.edges(), [Fraction(float(v)) for v in x], N)
        assert abs(float(np.dot(x, y)) - float(want)) <= 1e-13 * float(want)


def test_invariances():
    hg = s3synth.config_small(seed=5)
    x = s3synth.x_uniform(hg.n, 0, 1, 5)
    y = oracle.ttsv1(hg, x)
    rng = np.random.default_rng(1)
    # node relabelling
    perm = rng.permutation(hg.n)
    hg2 = s3synth.Hypergraph(hg.n, hg.edge_ptr, perm[hg.members].astype(np.int32), rank=hg.rank)
    x2 = np.empty_like(x)
    x2[perm] = x
    assert rel_err(oracle.ttsv1(hg2, x2)[perm], y) < 1e-13
    # member order inside edges and edge order
    edges = hg.edges()
    rng.shuffle(edges)
    edges = [tuple(rng.permutation(list(e))) for e in edges]
    hg3 = s3synth.from_edges(hg.n, edges, rank=hg.rank)
    assert rel_err(oracle.ttsv1(hg3, x), y) < 1e-13


def test_sampled_nodes_equal_full():
    hg = s3synth.config_small(seed=2)
    x = s3synth.x_uniform(hg.n, 0, 1, 2)
    y = oracle.ttsv1(hg, x)
    nodes = np.array([0, 5, 999, 17, 17])
    assert np.array_equal(oracle.ttsv1(hg, x, nodes=nodes), y[nodes])


def test_threads_do_not_change_results():
    hg = s3synth.config_small(seed=3)
    x = s3synth.x_uniform(hg.n, 0, 1, 3)
    assert np.array_equal(oracle.ttsv1(hg, x, nthreads=1), oracle.ttsv1(hg, x, nthreads=4))


def test_oracle_rejects_bad_input():
    hg = s3synth.from_edges(3, [(0, 5)])
    with pytest.raises(ValueError):
        oracle.ttsv1(hg, np.ones(3), N=2)
    hg = s3synth.from_edges(3, [(0, 1, 2)])
    with pytest.raises(ValueError):
        oracle.ttsv1(hg, np.ones(3), N=2)
