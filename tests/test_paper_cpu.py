"""The paper's CPU algorithms (the bench's comparators) against the oracle.

Algorithm 3 (leaf-to-root products on the CCSS forest) and Algorithm 4 (the
memoised depth-first traversal) must give the oracle's y = B x^(N-1), and their
product counts must be the ones Sec. IV-C states: |e|^2 - |e| per edge for
Algorithm 3, one per forest edge for Algorithm 4 (the forest being the trimmed
CCSS of Sec. III, compared level by level with the oracle's enumeration).
"""
import numpy as np
import pytest

import oracle
import s3synth
from gpu_util import rel_err
from oracle import ccss

baseline = pytest.importorskip("baseline")


def cases():
    yield s3synth.fig1_example(), None
    for seed in range(3):
        yield s3synth.tiny_case(seed=seed, rank=4), 5
    yield s3synth.config_small(seed=1), None
    yield s3synth.config_powerlaw(n=3000, m=15000, rank=12, seed=3), None
    yield s3synth.sunflower(petals=40, k=8, core=3, n=300), None
    yield s3synth.nested(chains=20, length=4, start=3, step=2, n=400), None
    yield s3synth.from_edges(12, [(0,), (1, 2), (1, 2), (0, 3, 4), (5,), (2, 6, 7, 8, 9)]), 6


@pytest.mark.parametrize("k", range(9))
def test_algorithms_3_and_4_match_oracle(k):
    hg, N = list(cases())[k]
    x = s3synth.x_uniform(hg.n, 0.1, 1.3, k)
    want = oracle.ttsv1(hg, x, N=N)
    f = baseline.Forest(hg, N)
    for alg in (f.alg3, f.alg4):
        for threads in (1, 4):
            y = alg(x, nthreads=threads)
            assert rel_err(y, want, floor=1e-300) <= 1e-12, (hg.name, alg.__name__, threads)


def test_product_counts_follow_sec_iv():
    for hg, N in cases():
        f = baseline.Forest(hg, N)
        edges = hg.edges()
        sizes = [len(e) for e in edges]
        assert f.products3 == sum(s * s - s for s in sizes if s >= 2)
        lv = ccss.trimmed_levels([e for e in edges if len(e) >= 2])
        assert f.nodes == sum(ccss.level_counts(lv))
        assert f.products4 == f.nodes - len(lv.get(1, ()))
        assert f.leaves == hg.nnz


def test_memoisation_saves_products_on_nested_and_sunflower():
    # Fig. 3: nested families and sunflowers share prefixes, so Algorithm 4 needs fewer
    # products than Algorithm 3.  A single edge of size k already needs k^2 - k products
    # in Algorithm 3 and (k^2 + k - 6)/2 in the trimmed forest (a direct count; Sec. IV-C's
    # (k^2 - k)/2 does not match it), a ratio just under 2 that sharing then raises.
    for k in (4, 7, 12):
        f = baseline.Forest(s3synth.from_edges(k, [tuple(range(k))]))
        assert (f.products3, f.products4) == (k * k - k, (k * k + k - 6) // 2)
    for hg in (s3synth.nested(chains=50, length=5, start=4, step=3, n=2000),
               s3synth.sunflower(petals=100, k=10, core=6, n=1000)):
        f = baseline.Forest(hg)
        single = sum((len(e) ** 2 + len(e) - 6) // 2 for e in hg.edges())
        assert f.products4 < single < f.products3, (hg.name, f.products3, single, f.products4)


def test_root_ranges_partition_the_work():
    hg = s3synth.config_powerlaw(n=3000, m=15000, rank=12, seed=4)
    x = s3synth.x_uniform(hg.n, 0.2, 1.2, 4)
    f = baseline.Forest(hg)
    full = f.alg4(x)
    half = f.roots // 2
    parts = f.alg4(x, roots=(0, half)) + f.alg4(x, roots=(half, f.roots))
    single = np.zeros(hg.n)
    for e in hg.edges():
        if len(e) == 1:
            single[e[0]] += x[e[0]] ** (hg.rank - 1)
    assert rel_err(parts + single, full, floor=1e-300) <= 1e-13
    assert f.leaves_in_roots(0, half) + f.leaves_in_roots(half, f.roots) + int((hg.sizes() == 1).sum()) == hg.nnz
    p3 = f.alg3(x, roots=(0, half))
    assert rel_err(p3, f.alg4(x, roots=(0, half)), floor=1e-300) <= 1e-12
