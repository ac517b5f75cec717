"""The paper's CPU algorithms (Algorithms 3 and 4 on the CCSS forest) as comparators.

ctypes binding of ``libpaper_cpu.so`` (built by ``__graft_entry__.build()`` from
``paper_cpu.cpp``): FP64, OpenMP over the host cores.  Measurement
infrastructure for ``bench.py`` and the tests; it shares no code with the CUDA
library or with the oracle.

    f = Forest(hg)            # trimmed CCSS forest of a hypergraph
    s = f.alg4(b)             # Algorithm 4 (memoised DFS), s = B b^(N-1)
    s = f.alg3(b)             # Algorithm 3 (leaf-to-root, no memoisation)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "paper_cpu.cpp")
LIB = os.path.join(HERE, "libpaper_cpu.so")

_lib = None


def build():
    """Compile libpaper_cpu.so (g++, -O3, OpenMP) if the source is newer."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        lib = ctypes.CDLL(LIB)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.pc_build.restype = P
        lib.pc_build.argtypes = [I64, I64, P, P, I32]
        lib.pc_free.argtypes = [P]
        lib.pc_info.argtypes = [P, P]
        lib.pc_leaves_in_roots.restype = I64
        lib.pc_leaves_in_roots.argtypes = [P, I64, I64]
        for nm in ("pc_alg3", "pc_alg4"):
            getattr(lib, nm).argtypes = [P, P, P, I32, I64, I64]
        _lib = lib
    return _lib


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class Forest:
    """Trimmed CCSS forest of a hypergraph (index order inside edges) at rank N."""

    def __init__(self, hg, N=None):
        lib = _load()
        self.n = hg.n
        self.N = int(N or hg.rank)
        self._ptr = np.ascontiguousarray(hg.edge_ptr, dtype=np.int64)
        self._mem = np.ascontiguousarray(hg.members, dtype=np.int32)
        self.h = lib.pc_build(hg.n, hg.m, self._ptr.ctypes.data, self._mem.ctypes.data, self.N)
        if not self.h:
            raise ValueError("bad hypergraph or rank for the CCSS forest")
        info = np.zeros(6, dtype=np.int64)
        lib.pc_info(self.h, info.ctypes.data)
        self.nodes, self.roots, self.leaves, self.levels, self.products3, self.products4 = (int(v) for v in info)

    def __del__(self):
        if getattr(self, "h", None):
            _load().pc_free(self.h)
            self.h = None

    def leaves_in_roots(self, r0, r1):
        return int(_load().pc_leaves_in_roots(self.h, int(r0), int(r1)))

    def _run(self, fn, b, nthreads, roots):
        b = np.ascontiguousarray(b, dtype=np.float64)
        s = np.zeros(self.n, dtype=np.float64)
        r0, r1 = (0, -1) if roots is None else roots
        getattr(_load(), fn)(self.h, b.ctypes.data, s.ctypes.data, int(nthreads or host_cores()), int(r0), int(r1))
        return s

    def alg3(self, b, nthreads=None, roots=None):
        """Algorithm 3: s = B b^(N-1) (roots=(r0, r1): only the leaves of those trees)."""
        return self._run("pc_alg3", b, nthreads, roots)

    def alg4(self, b, nthreads=None, roots=None):
        """Algorithm 4: s = B b^(N-1) (roots=(r0, r1): only those trees)."""
        return self._run("pc_alg4", b, nthreads, roots)
