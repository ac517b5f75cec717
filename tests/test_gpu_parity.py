"""GPU S^3TTVc vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (per node, relative): every FP64-accurate path (FP64 series and the
double-float series) 1e-12 at every rank up to 128, FP32 path 1e-5 for ranks
up to 25 (the bounds stated for the method); FP32 results at ranks 100 and 128
are checked against looser 1e-4 / 2e-4 bounds (the series there are 75-127
coefficients long) and their error is printed.
"""
import numpy as np
import pytest

import oracle
import s3synth
from gpu_util import gpu_sttsvc, rel_err

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def check(hg, x, N=None, layouts=(None,), reduces=(0, 1), f32_tol=F32_TOL, f64_tol=F64_TOL, dtypes=None, **opts):
    want = oracle.ttsv1(hg, x, N=N)
    errs = {}
    for layout in layouts:
        for red in reduces:
            for dt, tol in (dtypes or (("f64", f64_tol), ("f32", f32_tol))):
                y = gpu_sttsvc(hg, x, dt, layout=layout, rank=N, reduce=red, **opts)
                e = rel_err(y, want)
                errs[(layout, red, dt)] = e
                assert e <= tol, f"{hg.name} layout={layout} reduce={red} {dt}: {e:.3e} > {tol}"
    return errs


@pytest.mark.parametrize("seed,N", [(0, 4), (1, 4), (2, 5), (3, 6), (4, 4), (5, 7)])
def test_tiny_cases(seed, N):
    hg = s3synth.tiny_case(seed=seed, rank=4)
    check(hg, s3synth.x_uniform(hg.n, 0.05, 1.5, seed), N=N, layouts=(None, "ccss"))


def test_fig1_example():
    hg = s3synth.fig1_example()
    check(hg, s3synth.x_uniform(hg.n, 0.0, 1.0, 3), layouts=(None, "ccss"))


def test_small_config_all_paths():
    # n=1000, m=5000, sizes U{2..5}, x ~ U(0,1)
    hg = s3synth.config_small(seed=1)
    x = s3synth.x_uniform(hg.n, 0.0, 1.0, 1)
    check(hg, x, layouts=(None, "ccss"))
    # every window through the warp-per-edge kernel, and small thread blocks
    check(hg, x, reduces=(0,), thread_max_w=1)
    check(hg, x, reduces=(0,), block_threads=32)
    # index order (no degree sort) and a single stream
    check(hg, x, reduces=(0, 1), order=1, streams=1, layouts=(None, "ccss"))


def test_powerlaw_medium_rank25():
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=11)
    x = s3synth.x_uniform(hg.n, 0.5, 1.5, 11)
    check(hg, x, layouts=(None, "ccss"))
    check(hg, x, reduces=(0,), thread_max_w=8)


@pytest.mark.parametrize("small", [-1, 0, 1 << 30])
def test_small_bucket_fusion(small):
    # -1: one launch per bucket (pipelined kernels, size-2 kernel); 0: default
    # threshold; 2^30: every thread-per-edge bucket of size >= 2 in the fused launch
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=13)
    x = s3synth.x_uniform(hg.n, 0.5, 1.5, 13)
    check(hg, x, small_bucket_edges=small)
    check(hg, x, reduces=(0,), small_bucket_edges=small, block_threads=64, streams=1)
    hg = s3synth.config_small(seed=2)
    check(hg, s3synth.x_uniform(hg.n, 0.0, 1.0, 2), small_bucket_edges=small)


def test_size_two_edges_all_ranks():
    # the size-2 kernel for every window W = N - 1 = 1..32 (and the warp path beyond)
    rng = np.random.default_rng(4)
    edges = [tuple(rng.choice(400, size=2, replace=False)) for _ in range(3000)]
    hg = s3synth.from_edges(400, edges)
    x = s3synth.x_uniform(hg.n, 0.1, 1.4, 4)
    for N in (2, 3, 9, 25, 33, 34, 40):
        check(hg, x, N=N, reduces=(0, 1), small_bucket_edges=-1)


DF_TOL = 1e-12   # double-float series: ~44-bit significands, ~1e-13 per node in practice


def test_double_float_series():
    # S3_DF64: FP64 x and y, series in pairs of FP32 numbers; windows wider than 24 and
    # size-1 edges fall back to FP64 kernels, CCSS runs FP64
    for hg, x, N in ((s3synth.config_small(seed=4), None, None),
                     (s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=14), None, None),
                     (s3synth.tiny_case(seed=3, rank=4), None, 6),
                     (s3synth.config_large_rank(n=3000, m=4000, rank=100, seed=15), None, None)):
        x = s3synth.x_uniform(hg.n, 0.05, 1.5, 21)
        errs = check(hg, x, N=N, dtypes=(("df", DF_TOL),), layouts=(None, "ccss"))
        print(hg.name, {k: f"{v:.1e}" for k, v in errs.items()})
    # every window 1..32 through the size-2 and thread kernels, blocks of 64 threads
    rng = np.random.default_rng(8)
    edges = [tuple(rng.choice(300, size=s, replace=False)) for s in (2, 3, 5, 9) for _ in range(400)]
    hg = s3synth.from_edges(300, edges)
    x = s3synth.x_uniform(hg.n, 0.2, 1.1, 22)
    for N in (9, 17, 25, 33):
        check(hg, x, N=N, dtypes=(("df", DF_TOL),), block_threads=64, small_bucket_edges=-1)


def test_double_float_matches_fp64_closely():
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=16)
    x = s3synth.x_uniform(hg.n, 0.3, 1.2, 23)
    a = gpu_sttsvc(hg, x, "df")
    b = gpu_sttsvc(hg, x, "f64")
    m = b != 0
    assert np.max(np.abs(a[m] - b[m]) / np.abs(b[m])) < 1e-12


def test_large_rank_100():
    hg = s3synth.config_large_rank(n=3000, m=4000, rank=100, seed=12)
    x = s3synth.x_uniform(hg.n, 0.5, 1.5, 12)
    errs = check(hg, x, reduces=(0, 1), f32_tol=1e-4, f64_tol=F64_TOL, layouts=(None, "ccss"))
    print("rank-100 errors:", {k: f"{v:.2e}" for k, v in errs.items()})


def test_edge_cases_sizes_rank_isolated_duplicates():
    edges = [(0,), (1, 2), (1, 2), (0, 3, 4), (5,), (2, 6, 7, 8, 9), (3, 4)]
    hg = s3synth.from_edges(12, edges)          # nodes 10, 11 isolated; one duplicate edge
    x = s3synth.x_uniform(hg.n, 0.2, 1.2, 5)
    x[6] = 0.0                                  # a zero entry
    for N in (5, 6, 9, 30):
        check(hg, x, N=N, layouts=(None, "ccss"))
    y = gpu_sttsvc(hg, x, "f64", rank=6)
    assert y[10] == 0.0 and y[11] == 0.0


def test_no_edges_gives_zero():
    hg = s3synth.Hypergraph(7, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), rank=3)
    for dt in ("f32", "f64"):
        assert np.all(gpu_sttsvc(hg, np.ones(7), dt, rank=3) == 0.0)


def test_maximum_rank_edges():
    # S3_MAX_RANK = 128: one edge of every width class at rank 128
    rng = np.random.default_rng(0)
    edges = [tuple(rng.choice(300, size=s, replace=False)) for s in (2, 3, 17, 64, 100, 127, 128)]
    hg = s3synth.from_edges(300, edges)
    x = s3synth.x_uniform(hg.n, 0.7, 1.3, 1)
    check(hg, x, N=128, f32_tol=2e-4, f64_tol=F64_TOL, reduces=(0,), layouts=(None, "ccss"))


def test_ones_give_degrees():
    hg = s3synth.config_powerlaw(n=5000, m=20000, rank=12, seed=3)
    d = hg.degrees().astype(np.float64)
    for dt, tol in (("f64", 1e-13), ("f32", 2e-6)):
        y = gpu_sttsvc(hg, np.ones(hg.n), dt)
        assert rel_err(y[d > 0], d[d > 0]) < tol


def test_segmented_reduce_is_deterministic():
    import torch

    import paper_2311_08595_gb300 as s3
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=5)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    for dt in (torch.float32, torch.float64):
        x = torch.tensor(s3synth.x_uniform(hg.n, 0.5, 1.5, 5), dtype=dt, device="cuda")
        ys = []
        for _ in range(3):
            y = torch.empty_like(x)
            s3.s3_sttsvc(g, x, y)
            ys.append(y.cpu())
        assert all(torch.equal(ys[0], t) for t in ys[1:])


def test_host_entry_point_matches_device():
    import torch

    import paper_2311_08595_gb300 as s3
    hg = s3synth.config_small(seed=2)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    # each type's first host call captures the call on the handle's staging buffers as a
    # graph; the later calls replay it with new inputs
    for dt, df in ((torch.float32, False), (torch.float64, False), (torch.float64, True)):
        for seed in (2, 3, 4):
            x = s3synth.x_uniform(hg.n, 0, 1, seed)
            xh = torch.tensor(x, dtype=dt).pin_memory()
            yh = torch.empty_like(xh).pin_memory()
            s3.s3_sttsvc_host(g, xh, yh, df=df)
            yd = torch.empty(hg.n, dtype=dt, device="cuda")
            s3.s3_sttsvc(g, xh.cuda(), yd, df=df)
            torch.cuda.synchronize()
            assert torch.equal(yh, yd.cpu()), (dt, df, seed)


def test_range_events_counted():
    import torch

    import paper_2311_08595_gb300 as s3
    hg = s3synth.config_small(seed=3)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    s3.s3_range_events(g, reset=True)
    y = torch.empty(hg.n, dtype=torch.float32, device="cuda")
    s3.s3_sttsvc(g, torch.full((hg.n,), 0.5, device="cuda"), y)
    assert s3.s3_range_events(g) == 0
    s3.s3_sttsvc(g, torch.full((hg.n,), 1e-12, device="cuda"), y)   # (1e-12)^4 underflows FP32
    assert s3.s3_range_events(g, reset=True) > 0
    y64 = torch.empty(hg.n, dtype=torch.float64, device="cuda")
    s3.s3_sttsvc(g, torch.full((hg.n,), 1e-12, dtype=torch.float64, device="cuda"), y64)
    assert s3.s3_range_events(g) == 0


def test_range_check_returns_erange():
    # a handle built with range_check = 1 synchronises each call and reports results that
    # left the FP32 range as S3_ERANGE (y still written); the host entry point always does
    import torch

    import paper_2311_08595_gb300 as s3
    hg = s3synth.config_small(seed=3)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, range_check=1)
    y = torch.empty(hg.n, dtype=torch.float32, device="cuda")
    s3.s3_sttsvc(g, torch.full((hg.n,), 0.5, device="cuda"), y)          # in range: no error
    with pytest.raises(s3.S3Error) as ei:
        s3.s3_sttsvc(g, torch.full((hg.n,), 1e-12, device="cuda"), y)    # (1e-12)^4 underflows
    assert ei.value.status == s3.S3_ERANGE
    assert torch.isfinite(y).all()
    s3.s3_sttsvc(g, torch.full((hg.n,), 0.5, device="cuda"), y)          # the next call is clean again
    g2 = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    xh = torch.full((hg.n,), 1e-12).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    with pytest.raises(s3.S3Error) as ei:
        s3.s3_sttsvc_host(g2, xh, yh)
    assert ei.value.status == s3.S3_ERANGE
    s3.s3_sttsvc_host(g2, torch.full((hg.n,), 0.5).pin_memory(), yh)


def test_queries_wait_for_the_handle_only():
    # s3_range_events waits for the handle's last call (an event on its stream): a kernel
    # left running on another stream does not have to finish first, and the count it
    # returns includes the handle's last call
    import torch

    import paper_2311_08595_gb300 as s3
    hg = s3synth.config_small(seed=3)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        torch.cuda._sleep(int(2e9))          # about a second of GPU time on another stream
    y = torch.empty(hg.n, dtype=torch.float32, device="cuda")
    s3.s3_sttsvc(g, torch.full((hg.n,), 1e-12, device="cuda"), y)
    assert s3.s3_range_events(g) > 0
    assert not side.query(), "the query waited for unrelated work"
    side.synchronize()


def test_invalid_calls_raise():
    import torch

    import paper_2311_08595_gb300 as s3
    hg = s3synth.config_small(seed=1)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    x = torch.ones(hg.n, device="cuda")
    with pytest.raises(s3.S3Error):
        s3.s3_sttsvc_layout(g, s3.S3_LAYOUT_CCSS, x, torch.empty_like(x))   # built without the forest
    with pytest.raises(ValueError):
        s3.s3_sttsvc(g, x[:10], torch.empty_like(x))


@pytest.mark.parametrize("dt,tol", [("f64", F64_TOL), ("f32", F32_TOL), ("df", DF_TOL)])
def test_full_size_powerlaw_sampled(dt, tol):
    # n=1M, m=5M, Zipf(2.5) sizes on {2..25}, Chung-Lu gamma=2.1: the benchmark's
    # workload, its x (degree^(1/24) jittered, max 1: the input that decides which edges
    # the closed form accepts) and its launch configuration; sampled nodes -- the 16
    # largest hubs, the lowest-x nodes and random ones -- against the oracle
    import torch

    import paper_2311_08595_gb300 as s3
    hg = _big()
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    tdt = torch.float32 if dt == "f32" else torch.float64

    def run(x):
        xd = torch.tensor(x, dtype=tdt, device="cuda")
        yd = torch.full_like(xd, float("nan"))
        s3.s3_sttsvc(g, xd, yd, df=dt == "df")
        torch.cuda.synchronize()
        return yd.double().cpu().numpy()

    deg = hg.degrees()
    x = s3synth.x_degree_like(hg, seed=5)
    rng = np.random.default_rng(0)
    nodes = np.unique(np.concatenate([np.argsort(deg)[-16:], np.argsort(x)[:16], rng.integers(0, hg.n, 200)]))
    e = rel_err(run(x)[nodes], oracle.ttsv1(hg, x, nodes=nodes, nthreads=oracle.max_threads()))
    print(f"{dt}: max rel err {e:.2e} over {nodes.size} sampled nodes")
    assert e <= tol, f"{dt}: {e:.3e}"
    # x ~ U(0.5, 1.5) on the same graph
    x2 = s3synth.x_uniform(hg.n, 0.5, 1.5, 21)
    assert rel_err(run(x2)[nodes], oracle.ttsv1(hg, x2, nodes=nodes, nthreads=oracle.max_threads())) <= tol
    # B 1 = d holds at any size
    y1 = run(np.ones(hg.n))
    assert rel_err(y1[deg > 0], deg[deg > 0]) <= (2e-6 if dt == "f32" else 1e-13)
    s3.s3_destroy(g)


_BIG = None


def _big():
    global _BIG
    if _BIG is None:
        _BIG = s3synth.config_powerlaw()
    return _BIG
