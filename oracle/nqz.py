"""Algorithm 1 (NQZ) in FP64 -- test infrastructure only.

The H-eigenvector centrality is the positive x with B x^(N-1) = lambda x^[N-1]
(Sec. II).  Algorithm 1 finds it by a normalised power iteration: starting from
the uniform vector 1/n it applies S^3TTVc, takes the entrywise (N-1)-th root of
the result and rescales it to unit 1-norm; the ratios z_v / x_v^(N-1) of the
next S^3TTVc output z to the current iterate bracket the eigenvalue, and the
iteration stops once (largest ratio - smallest ratio) / smallest ratio falls
below the tolerance.

The iteration count returned is the number of power steps taken (each one
S^3TTVc call after the initial one).  ``x0`` replaces the uniform start when
given (the warm start of the learned model; any positive start works because
S^3TTVc is homogeneous of degree N-1 and the first step normalises).
"""
from __future__ import annotations

import numpy as np

from . import ttsv1 as _ttsv1


class NQZResult:
    def __init__(self, x, lam_min, lam_max, iters, converged, history):
        self.x, self.lam_min, self.lam_max = x, lam_min, lam_max
        self.iters, self.converged, self.history = iters, converged, history

    @property
    def lam(self):
        return 0.5 * (self.lam_min + self.lam_max)


def nqz(hg, tol=1e-8, max_iter=10000, N=None, x0=None, nthreads=1, ttsv=None):
    N = int(N or hg.rank)
    if N < 2:
        raise ValueError("NQZ needs rank >= 2")
    f = ttsv or (lambda v: _ttsv1(hg, v, N, nthreads=nthreads))
    y = np.full(hg.n, 1.0 / hg.n) if x0 is None else np.asarray(x0, dtype=np.float64)
    z = f(y)
    hist = []
    x = y
    for it in range(1, max_iter + 1):
        r = z ** (1.0 / (N - 1))
        x = r / r.sum()
        z = f(x)
        ratio = z / x ** (N - 1)
        lo, hi = float(ratio.min()), float(ratio.max())
        hist.append((lo, hi))
        if (hi - lo) / lo < tol:
            return NQZResult(x, lo, hi, it, True, hist)
    return NQZResult(x, hist[-1][0], hist[-1][1], max_iter, False, hist)
