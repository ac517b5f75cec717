"""Z-eigenpairs (shifted power method) and greedy symmetric CP on the GPU vs the oracle.

The device iteration (FP64 S^3TTVc plus FP64 vector kernels) must follow the
oracle's SS-HOPM (oracle/sshopm.py, pinned against a dense eigensolver at order
2 and closed forms): same eigenvalue, same iteration count, same vector.
"""
import numpy as np
import pytest

import s3synth
from oracle.sshopm import sshopm, symmetric_cp

pytestmark = pytest.mark.gpu


def _lcc(n, m, rank, seed):
    hg = s3synth.config_powerlaw(n=n, m=m, rank=rank, seed=seed)
    return s3synth.largest_component(hg)[0]


@pytest.mark.parametrize("n,m,rank,alpha", [(400, 1600, 4, 0.0), (2000, 8000, 12, 1.0), (3000, 12000, 25, 0.5)])
def test_zeigenpair_matches_oracle(n, m, rank, alpha):
    import torch

    import paper_2311_08595_gb300 as s3
    hg = _lcc(n, m, rank, seed=rank)
    x0 = s3synth.x_uniform(hg.n, 0.5, 1.5, rank)
    ref = sshopm(hg, alpha=alpha, tol=1e-13, max_iter=20000, x0=x0)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    x, res = s3.s3_zeigenpair(g, x0=torch.tensor(x0, device="cuda"), alpha=alpha, tol=1e-13, max_iter=20000)
    assert res["converged"] and ref.converged
    assert abs(res["lambda"] - ref.lam) <= 1e-11 * abs(ref.lam)
    assert abs(res["iters"] - ref.iters) <= 2, (res["iters"], ref.iters)
    assert np.max(np.abs(x.cpu().numpy() - ref.x)) <= 1e-6
    s3.s3_destroy(g)


def test_zeigenpair_order_two_and_uniform_start():
    import paper_2311_08595_gb300 as s3
    rng = np.random.default_rng(3)
    n = 80
    edges = {(i, (i + 1) % n) for i in range(n)} | {(0, 2)}
    while len(edges) < 300:
        a, b = rng.choice(n, 2, replace=False)
        edges.add((int(min(a, b)), int(max(a, b))))
    hg = s3synth.from_edges(n, sorted(edges))
    A = np.zeros((n, n))
    for a, b in hg.edges():
        A[a, b] = A[b, a] = 1.0
    w = np.linalg.eigvalsh(A)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    _, res = s3.s3_zeigenpair(g, tol=1e-15, max_iter=50000)
    assert abs(res["lambda"] - w[-1]) <= 1e-10 * w[-1]


def test_symmetric_cp_matches_oracle():
    import torch

    import paper_2311_08595_gb300 as s3
    hg = _lcc(1500, 6000, 6, seed=40)
    rng = np.random.default_rng(41)
    starts = [rng.uniform(0.5, 1.5, hg.n) for _ in range(3)]
    ref = symmetric_cp(hg, 3, alpha=2.0, tol=1e-13, max_iter=20000, starts=starts)
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    X0 = torch.tensor(np.stack(starts), device="cuda")
    lams, X, iters = s3.s3_symmetric_cp(g, 3, X0=X0, alpha=2.0, tol=1e-13, max_iter=20000)
    for r, (lam, x) in enumerate(ref):
        assert abs(lams[r] - lam) <= 1e-9 * abs(ref[0][0]), (r, lams[r], lam)
        assert np.max(np.abs(X[r].cpu().numpy() - x)) <= 1e-5
    s3.s3_destroy(g)
