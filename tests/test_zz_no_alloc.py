"""The allocation-free FP32 entry point against the handle-based one.

s3_sttsvc_f32_noalloc serves callers that cannot allocate device memory: it
takes the hypergraph as plain device CSR arrays and keeps its only scratch in
an array compiled into the library.  Here it is called through the C ABI
several times in a row and compared with s3_sttsvc (FP32) on the same inputs,
within the FP32 tolerance of the parity tests.  The first call runs on a
vector scaled so that its results (and so the rounding residues the scratch
collects) are about 1e20 times larger than the later calls': a later call that
kept any of that scratch would be off by many orders of magnitude.  This file
is collected last on purpose.
"""
import numpy as np
import pytest

import s3synth

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _handle_path(hg, x, rank=None):
    import torch

    import paper_2311_08595_gb300 as s3
    kw = {} if rank is None else {"rank": rank}
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, **kw)
    ref = torch.empty_like(x)
    s3.s3_sttsvc(g, x, ref)
    torch.cuda.synchronize()
    N = g.rank
    s3.s3_destroy(g)
    return ref.double().cpu().numpy(), N


def _noalloc(hg, x, N, edge_ptr=None, members=None):
    import torch

    import paper_2311_08595_gb300 as s3
    ep = torch.tensor(hg.edge_ptr if edge_ptr is None else edge_ptr, dtype=torch.int64, device="cuda")
    mem = torch.tensor(hg.members if members is None else members, dtype=torch.int32, device="cuda")
    y = torch.full_like(x, float("nan"))
    s3.s3_sttsvc_f32_noalloc(hg.n, ep, mem, x, y, N)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


def _check(y, r, what):
    err = np.max(np.abs(y - r) / np.maximum(np.abs(r), 1e-30))
    assert err <= F32_TOL, f"{what}: {err:.3e}"


def _compare(hg, x_np, rank=None):
    import torch
    x = torch.tensor(x_np, dtype=torch.float32, device="cuda")
    ref, N = _handle_path(hg, x, rank)
    # first call: results ~1e20 larger (x scaled by 10^(20/(N-1))), filling the scratch
    # with residues far larger than the later calls' results
    big = x * float(10.0 ** (20.0 / max(N - 1, 1)))
    ref_big, _ = _handle_path(hg, big, rank)
    _check(_noalloc(hg, big, N), ref_big, f"{hg.name} (scaled call)")
    for k in range(2):
        _check(_noalloc(hg, x, N), ref, f"{hg.name} (call {k + 2})")


def test_noalloc_matches_handle_path_small():
    hg = s3synth.config_small(seed=1)
    _compare(hg, s3synth.x_uniform(hg.n, 0.0, 1.0, 1))


def test_noalloc_matches_handle_path_powerlaw_and_sizes():
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=11)
    _compare(hg, s3synth.x_uniform(hg.n, 0.5, 1.5, 11))
    edges = [(0,), (1, 2), (0, 3, 4), (2, 6, 7, 8, 9), (3, 4)]
    tiny = s3synth.from_edges(12, edges)
    _compare(tiny, s3synth.x_uniform(12, 0.2, 1.2, 5), rank=7)


def test_noalloc_skips_malformed_edges():
    # an edge larger than the rank and an edge holding an id outside [0, n) add
    # nothing: the result equals the handle-based call on the well-formed edges
    import torch
    good = [(0,), (1, 2), (0, 3, 4), (2, 6, 7, 8, 9), (3, 4)]
    hg = s3synth.from_edges(12, good)
    N = 5
    x = torch.tensor(s3synth.x_uniform(12, 0.2, 1.2, 6), dtype=torch.float32, device="cuda")
    ref, _ = _handle_path(hg, x, N)
    bad = [(1, 2, 3, 4, 5, 6), (5, 12), (7, -1)]       # size 6 > N; ids 12 = n and -1
    edges = good[:2] + bad[:1] + good[2:4] + bad[1:] + good[4:]
    ep = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    mem = np.array([v for e in edges for v in e], dtype=np.int32)
    for _ in range(2):
        _check(_noalloc(hg, x, N, edge_ptr=ep, members=mem), ref, "malformed edges")


def test_noalloc_rejects_too_many_nodes():
    import torch

    import paper_2311_08595_gb300 as s3
    n = (1 << 22) + 1
    ep = torch.zeros(1, dtype=torch.int64, device="cuda")
    mem = torch.zeros(1, dtype=torch.int32, device="cuda")
    x = torch.ones(n, device="cuda")
    with pytest.raises(s3.S3Error) as ei:
        s3.s3_sttsvc_f32_noalloc(n, ep, mem, x, x.clone(), 3)
    assert ei.value.status == 1 and "S3_NOALLOC_MAX_NODES" in str(ei.value)
