"""GPU NQZ (Algorithm 1) against the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle
import s3synth
from oracle.nqz import nqz
from test_oracle_nqz import regular_hypergraph

pytestmark = pytest.mark.gpu


def _run(hg, **kw):
    import paper_2311_08595_gb300 as s3
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    x, res = s3.s3_hcentrality(g, **kw)
    return x.cpu().numpy(), res


@pytest.fixture(scope="module")
def medium():
    hg, _ = s3synth.largest_component(s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=7))
    ref = nqz(hg, tol=1e-8, nthreads=oracle.max_threads())
    return hg, ref


def test_fp64_matches_oracle(medium):
    hg, ref = medium
    x, res = _run(hg, tol=1e-8, precision=0)
    assert res["converged"]
    assert abs(res["iters"] - ref.iters) <= 1
    assert np.max(np.abs(x - ref.x) / ref.x) < 1e-10
    lam = 0.5 * (res["lambda_min"] + res["lambda_max"])
    assert abs(lam - ref.lam) < 1e-8 * ref.lam


def test_fp32_mixed_reaches_same_vector(medium):
    hg, ref = medium
    x, res = _run(hg, tol=1e-8, precision=1)
    assert res["converged"] and res["iters_fp32"] > 0
    assert np.max(np.abs(x - ref.x) / ref.x) < 1e-7
    print(f"mixed: {res['iters']} iterations ({res['iters_fp32']} FP32), oracle {ref.iters}")


@pytest.mark.parametrize("precision", [2, 3])
def test_double_float_phases_reach_same_vector(medium, precision):
    # 2: FP32 then double-float series; 3: double-float series throughout
    hg, ref = medium
    x, res = _run(hg, tol=1e-8, precision=precision)
    assert res["converged"]
    assert (res["iters_fp32"] > 0) == (precision == 2)
    assert np.max(np.abs(x - ref.x) / ref.x) < 1e-7
    if precision == 3:
        assert abs(res["iters"] - ref.iters) <= 1


def test_repeated_calls_reuse_graphs(medium):
    # the captured passes stay on the handle: same settings -> same result; other settings recapture
    import paper_2311_08595_gb300 as s3
    hg, ref = medium
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    x1, r1 = s3.s3_hcentrality(g, tol=1e-8, precision=2)
    x2, r2 = s3.s3_hcentrality(g, tol=1e-8, precision=2)
    assert r1["iters"] == r2["iters"] and bool((x1 == x2).all())
    x3, r3 = s3.s3_hcentrality(g, tol=1e-6, precision=2, check_every=4)
    assert r3["converged"] and r3["iters"] < r1["iters"]
    x4, r4 = s3.s3_hcentrality(g, tol=1e-8, precision=2)
    assert r4["iters"] == r1["iters"] and bool((x4 == x1).all())
    assert np.max(np.abs(x4.cpu().numpy() - ref.x) / ref.x) < 1e-7


def test_regular_hypergraph_one_iteration():
    hg = regular_hypergraph(300, 4, 2, 7, 2)
    x, res = _run(hg, tol=1e-12)
    assert res["converged"] and res["iters"] == 1
    assert np.allclose(x, 1.0 / hg.n, rtol=1e-13)
    assert abs(res["lambda_max"] - 4.0) < 1e-12


def test_warm_start_same_limit(medium):
    import torch
    hg, ref = medium
    x0 = torch.tensor(s3synth.x_uniform(hg.n, 0.5, 2.0, 3), dtype=torch.float64, device="cuda")
    x, res = _run(hg, tol=1e-8, x0=x0)
    assert res["converged"] and np.max(np.abs(x - ref.x) / ref.x) < 1e-7


def test_isolated_node_rejected():
    import paper_2311_08595_gb300 as s3
    hg = s3synth.from_edges(4, [(0, 1), (1, 2)])
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    with pytest.raises(s3.S3Error) as ei:
        s3.s3_hcentrality(g)
    assert ei.value.status == 1


def test_iteration_cap_reports_noconv(medium):
    hg, _ = medium
    x, res = _run(hg, tol=1e-14, max_iter=5, raise_on_noconv=False)
    assert res["status"] == "S3_ENOCONV" and res["iters"] == 5 and not res["converged"]


@pytest.mark.parametrize("precision", [0, 1])
def test_high_rank_matches_oracle(precision):
    # order 64: the per-node pass takes 63rd roots and 63rd powers of mantissas in [0.5, 1)
    # (the FP64 oracle itself needs x^(N-1) above the FP64 range's bottom, so N stays below ~100 here)
    import paper_2311_08595_gb300 as s3
    hg, _ = s3synth.largest_component(s3synth.config_large_rank(n=300, m=300, rank=64, prob=0.08, seed=11))
    ref = nqz(hg, tol=1e-8, nthreads=oracle.max_threads())
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, rank=hg.rank)
    x, res = s3.s3_hcentrality(g, tol=1e-8, precision=precision)
    x = x.cpu().numpy()
    assert res["converged"]
    assert abs(res["iters"] - ref.iters) <= 1
    assert np.max(np.abs(x - ref.x) / ref.x) < 1e-10
