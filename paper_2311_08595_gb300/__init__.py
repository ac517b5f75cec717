"""GB300 (sm_103a) S^3TTVc: sparse symmetric tensor times same vector on the
blowup tensor of a non-uniform hypergraph, and H-eigenvector centrality.

Thin Python binding of the C ABI in ``include/s3ttvc.h``.  Each function has
the name of the entry point it calls; arguments are marshalled (PyTorch CUDA
tensors or numpy arrays to raw pointers, streams to ``cudaStream_t``) and
every step of the computation runs in the library's CUDA kernels.  There is
no CPU fallback: without the built library the import of any entry point
raises.

    import paper_2311_08595_gb300 as s3
    g = s3.s3_build_format(n, edge_ptr, members)           # numpy CSR
    s3.s3_sttsvc(g, x, y)                                   # torch.cuda tensors
    x_c, res = s3.s3_hcentrality(g, tol=1e-8, precision=1)
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (S3_DF64, S3_EINVAL, S3_ENOCONV, S3_ENOTSUP, S3_ERANGE, S3_ETIMEOUT, S3_F32, S3_F64,  # noqa: F401
                   S3_LAYOUT_CCSS, S3_LAYOUT_EDGE, S3_REDUCE_ATOMIC, S3_REDUCE_SEGMENTED, S3Error, check, load,
                   ptr)

__all__ = [
    "Graph", "S3Error", "s3_options_init", "s3_format_inspect", "s3_build_format", "s3_graph_query",
    "s3_sttsvc", "s3_sttsvc_layout", "s3_sttsvc_host", "s3_sttsvc_profile", "s3_range_events", "s3_closed_form_query",
    "s3_bernoulli_query",
    "s3_hcentrality",
    "s3_nqz_options_init", "s3_sttsvc_f32_noalloc", "s3_destroy", "s3_version", "lib_path",
    "s3_zeig_options_init", "s3_zeigenpair", "s3_symmetric_cp", "s3_nqz_update",
    "Batch", "s3_batch_options_init", "s3_batch_create", "s3_sttsvc_batched", "s3_batch_autotune",
    "s3_batch_destroy", "MLP", "s3_features", "s3_mlp_create", "s3_mlp_get_params", "s3_mlp_forward",
    "s3_mlp_loss_grad", "s3_mlp_adam_step", "s3_warmstart", "s3_mlp_target", "s3_mlp_destroy", "s3_fma_peak",
]


def lib_path():
    return _lib.LIB_PATH


def s3_version():
    return int(load().s3_version())


def s3_options_init(**kw):
    """Default s3_options, with any field overridden by keyword."""
    o = _lib.s3_options()
    check(load().s3_options_init(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o


def _csr(edge_ptr, members):
    ep = np.ascontiguousarray(edge_ptr, dtype=np.int64)
    mem = np.ascontiguousarray(members, dtype=np.int32)
    return ep, mem


def _info_dict(info):
    d = {f: getattr(info, f) for f, _ in info._fields_}
    d["edges_per_size"] = list(info.edges_per_size)
    d["ccss_nodes_per_level"] = list(info.ccss_nodes_per_level)
    return d


def s3_format_inspect(n, edge_ptr, members, opt=None, **kw):
    """Validate/lay out on the host only (no GPU); returns the s3_format_info as a dict."""
    ep, mem = _csr(edge_ptr, members)
    o = opt or s3_options_init(**kw)
    info = _lib.s3_format_info()
    check(load().s3_format_inspect(int(n), ep.size - 1, ep.ctypes.data, mem.ctypes.data,
                                   ctypes.byref(o), ctypes.byref(info)))
    return _info_dict(info)


class Graph:
    """Owns an s3_graph_t; released by s3_destroy (or when garbage-collected)."""

    def __init__(self, handle, n, rank, opt):
        self.handle = handle
        self.n = n
        self.rank = rank
        self.opt = opt

    def __del__(self):
        try:
            s3_destroy(self)
        except Exception:
            pass


def s3_build_format(n, edge_ptr, members, opt=None, **kw):
    ep, mem = _csr(edge_ptr, members)
    o = opt or s3_options_init(**kw)
    h = ctypes.c_void_p()
    check(load().s3_build_format(int(n), ep.size - 1, ep.ctypes.data, mem.ctypes.data,
                                 ctypes.byref(o), ctypes.byref(h)))
    g = Graph(h, int(n), None, o)
    g.rank = s3_graph_query(g)["rank"]
    return g


def s3_graph_query(g):
    info = _lib.s3_format_info()
    check(load().s3_graph_query(g.handle, ctypes.byref(info)))
    return _info_dict(info)


def _dtype_code(t, df=False):
    """S3_F32 / S3_F64 from the tensor dtype; df=True: FP64 tensors, double-float series (S3_DF64)."""
    import torch
    if t.dtype == torch.float32 and not df:
        return S3_F32
    if t.dtype == torch.float64:
        return S3_DF64 if df else S3_F64
    raise TypeError("x must be float32 or float64 (float64 for df=True)")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _check_vec(g, t, name):
    if not t.is_cuda or not t.is_contiguous() or t.numel() != g.n:
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {g.n} elements")


def s3_sttsvc(g, x, y, stream=None, df=False):
    """y = B x^(N-1) on the device (x, y: CUDA tensors of the same float dtype; df=True with
    float64 tensors runs the series in double-float, S3_DF64)."""
    _check_vec(g, x, "x")
    _check_vec(g, y, "y")
    if x.dtype != y.dtype:
        raise TypeError("x and y must have the same dtype")
    check(load().s3_sttsvc(g.handle, _dtype_code(x, df), ptr(x), ptr(y), _stream(stream)))
    return y


def s3_sttsvc_layout(g, layout, x, y, stream=None, df=False):
    _check_vec(g, x, "x")
    _check_vec(g, y, "y")
    check(load().s3_sttsvc_layout(g.handle, _dtype_code(x, df), int(layout), ptr(x), ptr(y), _stream(stream)))
    return y


def s3_sttsvc_host(g, x_host, y_host, stream=None, df=False):
    """Host buffers in and out (torch CPU tensors, pinned recommended, or numpy)."""
    if isinstance(x_host, np.ndarray):
        code = S3_F32 if x_host.dtype == np.float32 else (S3_DF64 if df else S3_F64)
        xp, yp = x_host.ctypes.data, y_host.ctypes.data
    else:
        code = _dtype_code(x_host, df)
        xp, yp = x_host.data_ptr(), y_host.data_ptr()
    check(load().s3_sttsvc_host(g.handle, code, xp, yp, _stream(stream)))
    return y_host


def s3_sttsvc_profile(g, x, y, stream=None, df=False):
    """One S^3TTVc call with device timings of its phases (synchronises); returns a dict."""
    _check_vec(g, x, "x")
    _check_vec(g, y, "y")
    prof = _lib.s3_profile()
    check(load().s3_sttsvc_profile(g.handle, _dtype_code(x, df), ptr(x), ptr(y), ctypes.byref(prof),
                                   _stream(stream)))
    return {"edge_ms": prof.edge_ms, "reduce_ms": prof.reduce_ms, "total_ms": prof.total_ms,
            "launches": prof.launches, "bern_ms": prof.bern_ms}


def s3_range_events(g, reset=False):
    c = ctypes.c_int64()
    check(load().s3_range_events(g.handle, ctypes.byref(c), int(bool(reset))))
    return int(c.value)


def s3_closed_form_query(g):
    """Edge sizes evaluated in closed form for FP32 and for FP64 calls, and the edges
    rejected by its error bound so far: {"f32": [s, ...], "f64": [...], "rejected": k}."""
    a, b, r = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int64()
    check(load().s3_closed_form_query(g.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(r)))
    sizes = lambda m: [s for s in range(64) if (m >> s) & 1]
    return {"f32": sizes(a.value), "f64": sizes(b.value), "rejected": int(r.value)}


def s3_bernoulli_query(g):
    """Edge sizes evaluated in the Bernoulli form for FP32 and for FP64 calls, and the edges its
    gate sent back to the series so far: {"f32": [s, ...], "f64": [...], "rejected": k}."""
    a, b, r = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int64()
    check(load().s3_bernoulli_query(g.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(r)))
    sizes = lambda m: [s + 1 for s in range(64) if (m >> s) & 1]
    return {"f32": sizes(a.value), "f64": sizes(b.value), "rejected": int(r.value)}


def s3_nqz_options_init(**kw):
    o = _lib.s3_nqz_options()
    check(load().s3_nqz_options_init(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown NQZ option {k}")
        setattr(o, k, v)
    return o


def s3_hcentrality(g, x0=None, x_out=None, stream=None, raise_on_noconv=True, **kw):
    """Algorithm 1 (NQZ) on the device.  Returns (x_out, result dict)."""
    import torch
    o = s3_nqz_options_init(**kw)
    if x_out is None:
        x_out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    _check_vec(g, x_out, "x_out")
    if x0 is not None:
        _check_vec(g, x0, "x0")
        if x0.dtype != torch.float64:
            raise TypeError("x0 must be float64")
    res = _lib.s3_nqz_result()
    st = load().s3_hcentrality(g.handle, ctypes.byref(o), ptr(x0), ptr(x_out), ctypes.byref(res), _stream(stream))
    out = {f: getattr(res, f) for f, _ in res._fields_ if f != "reserved"}
    out["status"] = _lib.status_name(st)
    if st != _lib.S3_OK and not (st == _lib.S3_ENOCONV and not raise_on_noconv):
        check(st)
    return x_out, out


def s3_nqz_update(g, z, xhat, x_next, xhat_next, stream=None):
    """One Algorithm 1 update from a complete z (float64 CUDA tensors): returns (lambda_min, lambda_max)
    and writes the next iterate to x_next (1-norm 1) and xhat_next (max 1)."""
    for t, nm in ((z, "z"), (xhat, "xhat"), (x_next, "x_next"), (xhat_next, "xhat_next")):
        _check_vec(g, t, nm)
    lam = np.zeros(2, dtype=np.float64)
    check(load().s3_nqz_update(g.handle, ptr(z), ptr(xhat), ptr(x_next), ptr(xhat_next), lam.ctypes.data,
                               _stream(stream)))
    return float(lam[0]), float(lam[1])


def s3_zeig_options_init(**kw):
    o = _lib.s3_zeig_options()
    check(load().s3_zeig_options_init(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown Z-eigenpair option {k}")
        setattr(o, k, v)
    return o


def s3_zeigenpair(g, x0=None, x_out=None, stream=None, raise_on_noconv=True, **kw):
    """Z-eigenpair by the shifted power method on the device.  Returns (x, result dict)."""
    import torch
    o = s3_zeig_options_init(**kw)
    if x_out is None:
        x_out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    _check_vec(g, x_out, "x_out")
    if x0 is not None:
        _check_vec(g, x0, "x0")
        if x0.dtype != torch.float64:
            raise TypeError("x0 must be float64")
    res = _lib.s3_zeig_result()
    st = load().s3_zeigenpair(g.handle, ctypes.byref(o), ptr(x0), ptr(x_out), ctypes.byref(res), _stream(stream))
    if st != _lib.S3_OK and not (st == _lib.S3_ENOCONV and not raise_on_noconv):
        check(st)
    return x_out, {"lambda": res.lambda_, "iters": res.iters, "converged": res.converged, "seconds": res.seconds,
                   "status": _lib.status_name(st)}


def s3_symmetric_cp(g, R, X0=None, stream=None, **kw):
    """Greedy rank-R symmetric CP by deflated SS-HOPM.  Returns (lambdas, X (R x n CUDA tensor), iters)."""
    import torch
    o = s3_zeig_options_init(**kw)
    X = torch.empty((int(R), g.n), dtype=torch.float64, device="cuda")
    if X0 is not None:
        if (not X0.is_cuda or not X0.is_contiguous() or X0.dtype != torch.float64
                or tuple(X0.shape) != (int(R), g.n)):
            raise ValueError("X0 must be a contiguous float64 CUDA tensor of shape (R, n)")
    lams = np.zeros(int(R), dtype=np.float64)
    iters = np.zeros(int(R), dtype=np.int32)
    check(load().s3_symmetric_cp(g.handle, int(R), ctypes.byref(o), ptr(X0), ptr(X), lams.ctypes.data,
                                 iters.ctypes.data, _stream(stream)))
    return lams, X, iters


def s3_sttsvc_f32_noalloc(n, edge_ptr, members, x, y, rank, stream=None):
    """FP32 S^3TTVc that allocates no device memory (see include/s3ttvc.h).

    edge_ptr (int64, m+1), members (int32), x and y (float32, at least n each) are
    contiguous CUDA tensors on one device that the caller already owns; the
    library uses only its fixed built-in scratch.  The call runs on the tensors'
    device."""
    import torch
    n = int(n)
    for t, nm, dt in ((edge_ptr, "edge_ptr", torch.int64), (members, "members", torch.int32),
                      (x, "x", torch.float32), (y, "y", torch.float32)):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous CUDA tensor")
        if t.dtype != dt:
            raise TypeError(f"{nm} must be {dt}")
        if t.device != x.device:
            raise ValueError(f"{nm} is on {t.device}, x on {x.device}: all tensors must share one device")
    if edge_ptr.numel() < 1:
        raise ValueError("edge_ptr needs m+1 >= 1 entries")
    if x.numel() < n or y.numel() < n:
        raise ValueError(f"x and y must hold at least n = {n} floats")
    with torch.cuda.device(x.device):
        check(load().s3_sttsvc_f32_noalloc(n, edge_ptr.numel() - 1, int(rank), ptr(edge_ptr), ptr(members),
                                           ptr(x), ptr(y), _stream(stream)))
    return y


class Batch:
    """Owns an s3_batch_t (keeps its graphs alive); released by s3_batch_destroy."""

    def __init__(self, handle, graphs, nvec):
        self.handle = handle
        self.graphs = list(graphs)
        self.nvec = nvec

    def __del__(self):
        try:
            s3_batch_destroy(self)
        except Exception:
            pass


def s3_batch_options_init(**kw):
    o = _lib.s3_batch_options()
    check(load().s3_batch_options_init(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "cache_path":
            o.cache_path = v.encode()
        elif hasattr(o, k):
            setattr(o, k, int(v))
        else:
            raise TypeError(f"unknown batch option {k}")
    return o


def s3_batch_create(graphs, nvec, **kw):
    o = s3_batch_options_init(**kw)
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
    h = ctypes.c_void_p()
    check(load().s3_batch_create(len(graphs), arr, int(nvec), ctypes.byref(o), ctypes.byref(h)))
    return Batch(h, graphs, nvec)


def _ptr_arrays(b, xs, ys):
    """xs, ys: lists (graph-major, len count*nvec) of CUDA tensors -> host pointer arrays."""
    J = len(b.graphs) * b.nvec
    if len(xs) != J or len(ys) != J:
        raise ValueError(f"need {J} x and y tensors (graph-major)")
    for j, (x, y) in enumerate(zip(xs, ys)):
        g = b.graphs[j // b.nvec]
        _check_vec(g, x, "x")
        _check_vec(g, y, "y")
    code = _dtype_code(xs[0])
    xa = (ctypes.c_void_p * J)(*[t.data_ptr() for t in xs])
    ya = (ctypes.c_void_p * J)(*[t.data_ptr() for t in ys])
    return code, xa, ya


def s3_sttsvc_batched(b, xs, ys, stream=None):
    code, xa, ya = _ptr_arrays(b, xs, ys)
    check(load().s3_sttsvc_batched(b.handle, code, xa, ya, _stream(stream)))
    return ys


def s3_batch_autotune(b, xs, ys, stream=None):
    code, xa, ya = _ptr_arrays(b, xs, ys)
    r = _lib.s3_tune_result()
    check(load().s3_batch_autotune(b.handle, code, xa, ya, ctypes.byref(r), _stream(stream)))
    cands = [{"block_threads": c.block_threads, "edges_per_thread": c.edges_per_thread,
              "thread_max_w": c.thread_max_w, "ms": c.ms} for c in r.candidates[:min(r.tried, 32)]]
    return {"block_threads": r.block_threads, "edges_per_thread": r.edges_per_thread,
            "thread_max_w": r.thread_max_w, "ms": r.ms, "tried": r.tried, "candidates": cands}


def s3_batch_destroy(b):
    if b is not None and getattr(b, "handle", None):
        h, b.handle = b.handle, None
        check(load().s3_batch_destroy(h))


class MLP:
    """Owns an s3_mlp_t (warm-start network); released by s3_mlp_destroy."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        try:
            s3_mlp_destroy(self)
        except Exception:
            pass


def s3_features(g, feat=None, stream=None):
    """Per-node features (n x 12 float32 CUDA tensor)."""
    import torch
    if feat is None:
        feat = torch.empty((g.n, _lib.S3_MLP_FEATURES), dtype=torch.float32, device="cuda")
    if not feat.is_cuda or not feat.is_contiguous() or feat.numel() != g.n * _lib.S3_MLP_FEATURES:
        raise ValueError("feat must be a contiguous CUDA tensor of n x 12 floats")
    check(load().s3_features(g.handle, ptr(feat), _stream(stream)))
    return feat


def s3_mlp_create(params=None, seed=0):
    p = None
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.size != _lib.S3_MLP_PARAMS:
            raise ValueError(f"need {_lib.S3_MLP_PARAMS} parameters")
        p = params.ctypes.data
    h = ctypes.c_void_p()
    check(load().s3_mlp_create(p, int(seed), ctypes.byref(h)))
    m = MLP(h)
    m._keep = params
    return m


def s3_mlp_get_params(m, bf16=False):
    out = np.empty(_lib.S3_MLP_PARAMS, dtype=np.float32)
    check(load().s3_mlp_get_params(m.handle, out.ctypes.data, int(bool(bf16))))
    return out


def s3_mlp_forward(m, feat, out=None, stream=None):
    import torch
    n = feat.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=feat.device)
    check(load().s3_mlp_forward(m.handle, ptr(feat), int(n), ptr(out), _stream(stream)))
    return out


def s3_mlp_loss_grad(m, feat, target, want_grad=True, stream=None):
    """Loss and (optionally) its gradient as a numpy array; the gradient stays in m for the Adam step."""
    n = feat.shape[0]
    loss = ctypes.c_double()
    grad = np.empty(_lib.S3_MLP_PARAMS, dtype=np.float32) if want_grad else None
    check(load().s3_mlp_loss_grad(m.handle, ptr(feat), ptr(target), int(n), ctypes.byref(loss),
                                  None if grad is None else grad.ctypes.data, _stream(stream)))
    return float(loss.value), grad


def s3_mlp_adam_step(m, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(load().s3_mlp_adam_step(m.handle, float(lr), float(beta1), float(beta2), float(eps), _stream(stream)))


def s3_warmstart(g, m, x0=None, stream=None):
    import torch
    if x0 is None:
        x0 = torch.empty(g.n, dtype=torch.float64, device="cuda")
    _check_vec(g, x0, "x0")
    check(load().s3_warmstart(g.handle, m.handle, ptr(x0), _stream(stream)))
    return x0


def s3_mlp_target(g, x, target=None, stream=None):
    import torch
    if target is None:
        target = torch.empty(g.n, dtype=torch.float32, device="cuda")
    _check_vec(g, x, "x")
    check(load().s3_mlp_target(g.handle, ptr(x), ptr(target), _stream(stream)))
    return target


def s3_mlp_destroy(m):
    if m is not None and getattr(m, "handle", None):
        h, m.handle = m.handle, None
        check(load().s3_mlp_destroy(h))


def s3_fma_peak(fp64=False, reps=20, stream=None):
    """Measured FMA throughput of the current device (FP32, or FP64 with fp64=True)."""
    r = _lib.s3_peak_result()
    check(load().s3_fma_peak(S3_F64 if fp64 else S3_F32, int(reps), ctypes.byref(r), _stream(stream)))
    return {"tflops": r.tflops, "ms": r.ms, "flops_per_launch": r.flops_per_launch, "sm_count": r.sm_count,
            "threads_per_sm": r.threads_per_sm, "clock_mhz": r.clock_mhz}


def s3_destroy(g):
    if g is not None and getattr(g, "handle", None):
        h, g.handle = g.handle, None
        check(load().s3_destroy(h))
