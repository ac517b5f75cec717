"""Bernoulli-form evaluation (s3_bern.cuh) against the FP64 oracle.

Buckets of edges of size >= 6 whose window is at most 32 are evaluated from the
product G of all members' series and a Bernoulli-number polynomial per member;
every edge whose alternating sum could amplify rounding more than the gate
allows (or that holds x < 0) is recomputed by the warp-per-edge series.  These
tests check both halves against the oracle: inputs that all pass, inputs that
send many edges back (x spread over three decades, negative x, zeros), both
reduce modes, repeated calls, the biased output of the centrality iteration,
and that switching the form off gives the same results.
"""
import numpy as np
import pytest

import oracle
import s3synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def run(hg, x, dtype, calls=1, **opts):
    import torch

    import paper_2311_08595_gb300 as s3
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, **opts)
    dt = torch.float32 if dtype == "f32" else torch.float64
    xd = torch.tensor(np.asarray(x), dtype=dt, device="cuda")
    outs = []
    for _ in range(calls):
        yd = torch.full_like(xd, float("nan"))
        s3.s3_sttsvc(g, xd, yd)
        torch.cuda.synchronize()
        outs.append(yd.double().cpu().numpy())
    q = s3.s3_bernoulli_query(g)
    s3.s3_destroy(g)
    return outs, q


@pytest.fixture(scope="module")
def powerlaw():
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=31)
    return hg, s3synth.x_degree_like(hg, seed=31)


def test_bernoulli_matches_oracle(powerlaw):
    hg, x = powerlaw
    want = oracle.ttsv1(hg, x)
    for dt, tol in (("f64", F64_TOL), ("f32", F32_TOL)):
        for red in (0, 1):
            (y,), q = run(hg, x, dt, reduce=red)
            sizes = q["f32"] if dt == "f32" else q["f64"]
            # FP32 and FP64: sizes 6..25 (the closed form takes 3..5 in FP32, 2..5 in FP64)
            assert sizes == list(range(6, 26)), sizes
            assert q["rejected"] == 0, q
            e = rel_err(y, want)
            assert e <= tol, f"{dt} reduce={red}: {e:.3e}"


def test_bernoulli_off_is_the_series(powerlaw):
    hg, x = powerlaw
    for dt, tol in (("f64", F64_TOL), ("f32", F32_TOL)):
        (a,), qa = run(hg, x, dt)
        (b,), qb = run(hg, x, dt, bernoulli=-1)
        assert qb["f32"] == [] and qb["f64"] == []
        assert rel_err(a, b) <= 2 * tol


@pytest.mark.parametrize("dt,tol", [("f64", F64_TOL), ("f32", F32_TOL)])
def test_rejected_edges_go_back_to_the_series(dt, tol):
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=32)
    rng = np.random.default_rng(32)
    # x spread over three decades: many edges fail the amplification gate
    x = 10.0 ** rng.uniform(-3, 0, hg.n)
    want = oracle.ttsv1(hg, x)
    (y1, y2), q = run(hg, x, dt, calls=2)
    assert q["rejected"] > 0, q
    # FP32 cannot hold values below its normal range (products of many members near 1e-3)
    big = want > (1e-30 if dt == "f32" else 0.0)
    assert rel_err(y1[big], want[big]) <= tol and rel_err(y2[big], want[big]) <= tol
    assert np.array_equal(y1, y2)        # segmented reduce: bit-identical with rejections in play
    # negative x (every edge holding one is rejected) and zeros (accepted: exact zero products)
    x2 = s3synth.x_uniform(hg.n, 0.2, 1.2, 33)
    x2[rng.choice(hg.n, 200, replace=False)] = -0.5
    x2[rng.choice(hg.n, 200, replace=False)] = 0.0
    want2 = oracle.ttsv1(hg, x2)
    (y,), q2 = run(hg, x2, dt, reduce=1)
    assert q2["rejected"] > 0
    # mixed signs cancel inside y: compare on the scale of the largest value
    assert np.max(np.abs(y - want2)) <= tol * np.max(np.abs(want2))


def test_bernoulli_large_rank_and_small_tiles():
    # rank 40: the Bernoulli form covers sizes 9..40 (windows <= 32); a few edges of each size,
    # so every bucket ends in a partial warp
    rng = np.random.default_rng(34)
    edges = [tuple(rng.choice(3000, size=s, replace=False)) for s in range(6, 41) for _ in range(int(rng.integers(1, 40)))]
    hg = s3synth.from_edges(3000, edges)
    x = s3synth.x_uniform(hg.n, 0.5, 1.5, 34)
    want = oracle.ttsv1(hg, x, N=40)
    for dt, tol in (("f64", F64_TOL), ("f32", 1e-4)):
        (y,), q = run(hg, x, dt, rank=40)
        sizes = q["f32"] if dt == "f32" else q["f64"]
        assert sizes and min(sizes) == 9 and max(sizes) == 40, sizes
        assert rel_err(y, want) <= tol


def test_nqz_with_bernoulli_matches_oracle():
    # the centrality iteration runs S^3TTVc in its biased output mode through this path
    import paper_2311_08595_gb300 as s3
    from oracle.nqz import nqz
    hg = s3synth.config_powerlaw(n=3000, m=15000, rank=12, seed=36)
    lcc, _ = s3synth.largest_component(hg)
    g = s3.s3_build_format(lcc.n, lcc.edge_ptr, lcc.members)
    assert s3.s3_bernoulli_query(g)["f64"], "expected Bernoulli buckets at rank 12"
    xc, res = s3.s3_hcentrality(g, tol=1e-10)
    ref = nqz(lcc, tol=1e-10)
    assert res["converged"] and abs(res["iters"] - ref.iters) <= 1
    assert np.max(np.abs(xc.cpu().numpy() - ref.x) / ref.x) < 1e-9
    s3.s3_destroy(g)
