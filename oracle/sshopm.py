"""Shifted power method for Z-eigenpairs and greedy symmetric CP -- test infrastructure only.

The paper names S^3TTVc as the bottleneck of the shifted power method for
tensor eigenpairs and of symmetric CP decomposition (Sec. I).  For the order-N
blowup tensor B (Sec. II) a Z-eigenpair is (lambda, x) with
    B x^(N-1) = lambda x,   ||x||_2 = 1,
and the shifted symmetric higher-order power method (SS-HOPM) iterates
    x <- (B x^(N-1) + alpha x) / ||B x^(N-1) + alpha x||_2,   lambda = x . B x^(N-1),
from a start x0 (default: the uniform unit vector) until lambda changes by less
than tol (relative to max(1, |lambda|)); alpha >= 0 is the shift.

Greedy symmetric CP: component r is the SS-HOPM eigenpair of the deflated
tensor B - sum_{q<r} lambda_q x_q^(outer N), whose product with x^(N-1) is
    B x^(N-1) - sum_{q<r} lambda_q (x_q . x)^(N-1) x_q.

Plain numpy; S^3TTVc comes from the FP64 oracle of Algorithm 2.
"""
from __future__ import annotations

import numpy as np

from . import ttsv1 as _ttsv1


class ZEigResult:
    def __init__(self, lam, x, iters, converged, history):
        self.lam, self.x, self.iters, self.converged, self.history = lam, x, iters, converged, history


def sshopm(hg, alpha=0.0, tol=1e-12, max_iter=10000, x0=None, N=None, deflate=(), ttsv=None, nthreads=1):
    """SS-HOPM on B minus the rank-one terms in `deflate` ([(lambda_q, x_q), ...])."""
    N = int(N or hg.rank)
    f = ttsv or (lambda v: _ttsv1(hg, v, N, nthreads=nthreads))

    def apply(v):
        z = f(v)
        for lq, xq in deflate:
            z = z - lq * float(np.dot(xq, v)) ** (N - 1) * xq
        return z

    x = np.full(hg.n, 1.0) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    x = x / np.linalg.norm(x)
    z = apply(x)
    lam = float(np.dot(x, z))
    hist = [lam]
    for it in range(1, max_iter + 1):
        w = z + alpha * x
        x = w / np.linalg.norm(w)
        z = apply(x)
        new = float(np.dot(x, z))
        hist.append(new)
        if abs(new - lam) < tol * max(1.0, abs(new)):
            return ZEigResult(new, x, it, True, hist)
        lam = new
    return ZEigResult(lam, x, max_iter, False, hist)


def symmetric_cp(hg, R, alpha=0.0, tol=1e-12, max_iter=10000, starts=None, N=None, nthreads=1):
    """Greedy rank-R symmetric CP by deflated SS-HOPM: [(lambda_r, x_r), ...]."""
    comps = []
    for r in range(R):
        x0 = None if starts is None else starts[r]
        res = sshopm(hg, alpha=alpha, tol=tol, max_iter=max_iter, x0=x0, N=N, deflate=list(comps),
                     nthreads=nthreads)
        comps.append((res.lam, res.x))
    return comps
