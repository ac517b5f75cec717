"""CPU oracle for S^3TTVc and H-eigenvector centrality -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything in this package.  It shares no code
with the CUDA path and never imports it.

Contents
  exact      -- exact rational brute force (Eq. 2 over every tensor entry),
                Algorithm 2 in exact arithmetic, inclusion-exclusion.
  ttsv1      -- Algorithm 2 in FP64 (plain C, ``aay_oracle.c``), all nodes or
                a sample of nodes.
  nqz        -- Algorithm 1 (NQZ) in FP64 on top of ``ttsv1``.
  ccss       -- the CCSS forest of Sec. III (level node sets, special leaves).
  mlp        -- FP64 warm-start features and the 3-layer MLP (forward,
                backward, Adam) used to check the GPU training kernels.

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against brute force, closed forms, library routines or the paper's worked
example; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction
from math import factorial

import numpy as np

from . import exact

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aay_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile ``aay_oracle.c`` with gcc (-O2, OpenMP) into ``liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.s3o_ttsv1.restype = ctypes.c_int
        lib.s3o_ttsv1.argtypes = [
            ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
            ctypes.c_int,
        ]
        lib.s3o_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def scale_table(N):
    """scale[s] = w(e)/|beta(e)| * (N-1)! for s = 0..N, from exact integers, rounded once."""
    out = np.zeros(N + 1, dtype=np.float64)
    for s in range(1, N + 1):
        out[s] = float(Fraction(s * factorial(N - 1), exact.blowup_count(N, s)))
    return out


def max_threads():
    return int(_load().s3o_max_threads())


def ttsv1(hg, x, N=None, nodes=None, nthreads=1):
    """FP64 Algorithm 2: y = B x^(N-1) (all nodes, or y[nodes] for a sample)."""
    lib = _load()
    N = int(N or hg.rank)
    ptr = np.ascontiguousarray(hg.edge_ptr, dtype=np.int64)
    mem = np.ascontiguousarray(hg.members, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    sc = scale_table(N)
    if nodes is None:
        y = np.zeros(hg.n, dtype=np.float64)
        nd, cnt = None, 0
    else:
        nd = np.ascontiguousarray(nodes, dtype=np.int64)
        cnt = nd.size
        y = np.zeros(cnt, dtype=np.float64)
    rc = lib.s3o_ttsv1(hg.n, hg.m, ptr.ctypes.data, mem.ctypes.data, N, sc.ctypes.data,
                       x.ctypes.data, None if nd is None else nd.ctypes.data, cnt,
                       y.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle ttsv1 failed (code {rc})")
    return y


from . import ccss, nqz  # noqa: E402  (submodules that use the loader above)

__all__ = ["exact", "ccss", "nqz", "ttsv1", "scale_table", "build", "max_threads"]
