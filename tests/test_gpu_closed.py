"""Closed-form (inclusion-exclusion) evaluation of small edges against the FP64 oracle.

Buckets of edges of size 2..6 are evaluated from the signed sum over subsets
(Sec. II-A expanded term by term); every edge whose error bound fails goes back
to the series kernels.  These tests check both halves: results within the
path's tolerance for inputs that all pass, inputs that send many edges back
(zeros, x of very different sizes, negative x), both reduce modes, repeated
calls (the rejected-edge lists are reset by the series launch), and the
bit-for-bit determinism of the segmented reduce with rejections in play.
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
    q = s3.s3_closed_form_query(g)
    s3.s3_destroy(g)
    return outs, (q["f32"], q["f64"], q["rejected"])


@pytest.fixture(scope="module")
def powerlaw():
    # rank 25, Zipf sizes: buckets s = 2..6 hold most edges; every bucket gets its own launch
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=21)
    d = np.maximum(hg.degrees(), 1).astype(np.float64)
    rng = np.random.default_rng(21)
    x = d ** (1.0 / 24) * rng.uniform(0.9, 1.1, hg.n)
    return hg, x / x.max()


def test_closed_form_matches_oracle(powerlaw):
    hg, x = powerlaw
    want = oracle.ttsv1(hg, x)
    for dt, tol in (("f64", F64_TOL), ("f32", F32_TOL)):
        for red in (0, 1):
            (y,), (b32, b64, rej) = run(hg, x, dt, reduce=red, small_bucket_edges=-1)
            # FP32: sizes 3..5 (size 2 keeps its lean series kernel, size 6 is cheaper as series);
            # FP64: sizes 2..5 (size 6 goes to the Bernoulli form, with fewer FP64 operations)
            assert (b32, b64) == ([3, 4, 5], [2, 3, 4, 5]), (b32, b64)
            assert rej == 0, f"{dt}: {rej} edges rejected for a near-uniform vector"
            e = rel_err(y, want)
            assert e <= tol, f"{dt} reduce={red}: {e:.3e}"
    # the series path alone agrees to within both paths' error
    (y_off,), (b32, b64, _) = run(hg, x, "f64", small_bucket_edges=-1, closed_form_max_s=-1)
    assert b32 == [] and b64 == []
    assert rel_err(y_off, want) <= F64_TOL


def test_closed_form_sizes_limited(powerlaw):
    hg, x = powerlaw
    (y,), (b32, b64, _) = run(hg, x, "f32", small_bucket_edges=-1, closed_form_max_s=3)
    assert (b32, b64) == ([3], [2, 3])
    assert rel_err(y, oracle.ttsv1(hg, x)) <= F32_TOL


def test_rejected_edges_recomputed(powerlaw):
    hg, _ = powerlaw
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 1.0, hg.n)
    x[rng.random(hg.n) < 0.05] = 0.0          # zero members: c(e,u) = 0 for the others
    x[rng.random(hg.n) < 0.05] *= 1e-6        # members far smaller than the rest of their edge
    want = oracle.ttsv1(hg, x)
    for dt, tol in (("f64", F64_TOL), ("f32", F32_TOL)):
        ys, (_, _, rej) = run(hg, x, dt, calls=3, small_bucket_edges=-1)
        assert rej > 0
        assert rej % 3 == 0, "every call rejects the same edges"
        # FP32 cannot hold values below its normal range (products of several 1e-6 members)
        big = want > (1e-30 if dt == "f32" else 0.0)
        for y in ys:
            e = rel_err(y[big], want[big])
            assert e <= tol, f"{dt}: {e:.3e}"
            assert np.all(y[want == 0] == 0.0)
        # deterministic reduce: the lists' order varies, the sums do not
        assert all(np.array_equal(ys[0], y) for y in ys[1:])


def test_negative_members_use_series(powerlaw):
    hg, x = powerlaw
    rng = np.random.default_rng(8)
    xs = x * np.where(rng.random(hg.n) < 0.3, -1.0, 1.0)
    want = oracle.ttsv1(hg, xs)
    (y,), (_, _, rej) = run(hg, xs, "f64", small_bucket_edges=-1)
    assert rej > 0
    # mixed signs cancel inside y: compare on the scale of the largest contribution
    assert np.max(np.abs(y - want)) <= 1e-12 * np.max(np.abs(want))


def test_default_launch_plan_uses_closed_form():
    # with the default fused small-bucket launch only buckets with a launch of their own
    # qualify: the size-2 bucket (> 40000 edges); the size-6 bucket goes to the Bernoulli form
    # (FP32: its own cost rule; FP64: fewer FP64 operations than the closed form)
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=11)
    x = s3synth.x_uniform(hg.n, 0.5, 1.5, 11)
    (y,), (b32, b64, rej) = run(hg, x, "f32")
    assert (b32, b64) == ([], [2]) and rej == 0
    assert rel_err(y, oracle.ttsv1(hg, x)) <= F32_TOL


def test_low_rank_keeps_series():
    # at rank 5 the series is cheaper than 2^s subsets: no bucket uses the closed form
    hg = s3synth.config_small(seed=1)
    (_,), (b32, b64, _) = run(hg, s3synth.x_uniform(hg.n, 0.0, 1.0, 1), "f32", small_bucket_edges=-1)
    assert b32 == [] and b64 == []
