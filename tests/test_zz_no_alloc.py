"""The allocation-free FP32 entry point against the handle-based one.

s3_sttsvc_f32_noalloc serves callers that cannot allocate device memory: it
takes the hypergraph as plain device CSR arrays and keeps its only scratch in
an array compiled into the library.  Here it is called through the C ABI twice
in a row (the second call must not see the first call's scratch) and compared
with s3_sttsvc (FP32) on the same inputs, within the FP32 tolerance of the
parity tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import s3synth

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _compare(hg, x_np, rank=None):
    import torch

    import paper_2311_08595_gb300 as s3
    kw = {} if rank is None else {"rank": rank}
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, **kw)
    N = g.rank
    x = torch.tensor(x_np, dtype=torch.float32, device="cuda")
    ref = torch.empty_like(x)
    s3.s3_sttsvc(g, x, ref)
    ep = torch.tensor(hg.edge_ptr, dtype=torch.int64, device="cuda")
    mem = torch.tensor(hg.members, dtype=torch.int32, device="cuda")
    outs = []
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        s3.s3_sttsvc_f32_noalloc(hg.n, ep, mem, x, y, N)
        torch.cuda.synchronize()
        outs.append(y.double().cpu().numpy())
    r = ref.double().cpu().numpy()
    for y in outs:
        err = np.max(np.abs(y - r) / np.maximum(np.abs(r), 1e-30))
        assert err <= F32_TOL, f"{hg.name}: {err:.3e}"
    s3.s3_destroy(g)


def test_noalloc_matches_handle_path_small():
    hg = s3synth.config_small(seed=1)
    _compare(hg, s3synth.x_uniform(hg.n, 0.0, 1.0, 1))


def test_noalloc_matches_handle_path_powerlaw_and_sizes():
    hg = s3synth.config_powerlaw(n=20000, m=100000, rank=25, seed=11)
    _compare(hg, s3synth.x_uniform(hg.n, 0.5, 1.5, 11))
    edges = [(0,), (1, 2), (0, 3, 4), (2, 6, 7, 8, 9), (3, 4)]
    tiny = s3synth.from_edges(12, edges)
    _compare(tiny, s3synth.x_uniform(12, 0.2, 1.2, 5), rank=7)


def test_noalloc_rejects_too_many_nodes():
    import torch

    import paper_2311_08595_gb300 as s3
    n = (1 << 22) + 1
    ep = torch.zeros(1, dtype=torch.int64, device="cuda")
    mem = torch.zeros(1, dtype=torch.int32, device="cuda")
    x = torch.ones(4, device="cuda")
    with pytest.raises(s3.S3Error) as ei:
        s3.s3_sttsvc_f32_noalloc(n, ep, mem, x, x.clone(), 3)
    assert ei.value.status == 1 and "S3_NOALLOC_MAX_NODES" in str(ei.value)
