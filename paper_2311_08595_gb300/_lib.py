"""ctypes binding of ``libs3ttvc.so`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: tensors are passed as raw pointers, streams as
``cudaStream_t`` handles.  A missing library raises ``ImportError`` -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libs3ttvc.so")

S3_MAX_RANK = 128
S3_MLP_FEATURES, S3_MLP_HIDDEN, S3_MLP_PARAMS = 12, 64, 5057
S3_OK, S3_EINVAL, S3_ENOMEM, S3_ECUDA, S3_ENOCONV, S3_ETIMEOUT, S3_ERANGE, S3_ENOTSUP = range(8)
S3_F32, S3_F64, S3_DF64 = 0, 1, 2
S3_REDUCE_SEGMENTED, S3_REDUCE_ATOMIC = 0, 1
S3_LAYOUT_EDGE, S3_LAYOUT_CCSS = 0, 1
S3_ORDER_DEGREE, S3_ORDER_INDEX = 0, 1


class S3Error(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


class s3_options(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("reduce", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("build_ccss", ctypes.c_int32), ("device", ctypes.c_int32), ("thread_max_w", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("order", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("small_bucket_edges", ctypes.c_int32), ("closed_form_max_s", ctypes.c_int32),
                ("range_check", ctypes.c_int32), ("bernoulli", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class s3_format_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rank", ctypes.c_int32), ("max_edge", ctypes.c_int32), ("max_degree", ctypes.c_int64),
                ("edges_per_size", ctypes.c_int64 * (S3_MAX_RANK + 1)),
                ("ccss_levels", ctypes.c_int64),
                ("ccss_nodes_per_level", ctypes.c_int64 * (S3_MAX_RANK + 1)),
                ("ccss_nodes", ctypes.c_int64), ("ccss_special_leaves", ctypes.c_int64),
                ("ccss_products", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class s3_nqz_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("switch_tol", ctypes.c_double), ("check_every", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]


class s3_nqz_result(ctypes.Structure):
    _fields_ = [("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double), ("iters", ctypes.c_int32),
                ("iters_fp32", ctypes.c_int32), ("converged", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("seconds", ctypes.c_double)]


class s3_zeig_options(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]


class s3_zeig_result(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("seconds", ctypes.c_double), ("reserved", ctypes.c_int32 * 4)]


class s3_profile(ctypes.Structure):
    _fields_ = [("edge_ms", ctypes.c_float), ("reduce_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("launches", ctypes.c_int32), ("bern_ms", ctypes.c_float), ("reserved", ctypes.c_int32 * 3)]


class s3_batch_options(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("edges_per_thread", ctypes.c_int32),
                ("thread_max_w", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("cache_path", ctypes.c_char * 256), ("reserved", ctypes.c_int32 * 8)]


class s3_tune_candidate(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("edges_per_thread", ctypes.c_int32),
                ("thread_max_w", ctypes.c_int32), ("ms", ctypes.c_float)]


class s3_tune_result(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("edges_per_thread", ctypes.c_int32),
                ("thread_max_w", ctypes.c_int32), ("tried", ctypes.c_int32), ("ms", ctypes.c_float),
                ("reserved", ctypes.c_int32), ("candidates", s3_tune_candidate * 32)]


class s3_peak_result(ctypes.Structure):
    _fields_ = [("tflops", ctypes.c_double), ("flops_per_launch", ctypes.c_double), ("ms", ctypes.c_float),
                ("sm_count", ctypes.c_int32), ("threads_per_sm", ctypes.c_int32), ("clock_mhz", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

# name -> (restype, argtypes); every symbol include/s3ttvc.h declares
SIGNATURES = {
    "s3_options_init": (_I32, [ctypes.POINTER(s3_options)]),
    "s3_format_inspect": (_I32, [_I64, _I64, _P, _P, ctypes.POINTER(s3_options), ctypes.POINTER(s3_format_info)]),
    "s3_build_format": (_I32, [_I64, _I64, _P, _P, ctypes.POINTER(s3_options), ctypes.POINTER(_P)]),
    "s3_graph_query": (_I32, [_P, ctypes.POINTER(s3_format_info)]),
    "s3_sttsvc": (_I32, [_P, _I32, _P, _P, _P]),
    "s3_sttsvc_layout": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "s3_sttsvc_host": (_I32, [_P, _I32, _P, _P, _P]),
    "s3_range_events": (_I32, [_P, ctypes.POINTER(_I64), _I32]),
    "s3_closed_form_query": (_I32, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.POINTER(_I64)]),
    "s3_bernoulli_query": (_I32, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                  ctypes.POINTER(_I64)]),
    "s3_sttsvc_profile": (_I32, [_P, _I32, _P, _P, ctypes.POINTER(s3_profile), _P]),
    "s3_nqz_options_init": (_I32, [ctypes.POINTER(s3_nqz_options)]),
    "s3_hcentrality": (_I32, [_P, ctypes.POINTER(s3_nqz_options), _P, _P, ctypes.POINTER(s3_nqz_result), _P]),
    "s3_nqz_update": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "s3_zeig_options_init": (_I32, [ctypes.POINTER(s3_zeig_options)]),
    "s3_zeigenpair": (_I32, [_P, ctypes.POINTER(s3_zeig_options), _P, _P, ctypes.POINTER(s3_zeig_result), _P]),
    "s3_symmetric_cp": (_I32, [_P, _I32, ctypes.POINTER(s3_zeig_options), _P, _P, _P, _P, _P]),
    "s3_sttsvc_f32_noalloc": (_I32, [_I64, _I64, _I32, _P, _P, _P, _P, _P]),
    "s3_batch_options_init": (_I32, [ctypes.POINTER(s3_batch_options)]),
    "s3_batch_create": (_I32, [_I32, _P, _I32, ctypes.POINTER(s3_batch_options), ctypes.POINTER(_P)]),
    "s3_sttsvc_batched": (_I32, [_P, _I32, _P, _P, _P]),
    "s3_batch_autotune": (_I32, [_P, _I32, _P, _P, ctypes.POINTER(s3_tune_result), _P]),
    "s3_batch_destroy": (_I32, [_P]),
    "s3_features": (_I32, [_P, _P, _P]),
    "s3_mlp_create": (_I32, [_P, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "s3_mlp_get_params": (_I32, [_P, _P, _I32]),
    "s3_mlp_forward": (_I32, [_P, _P, _I64, _P, _P]),
    "s3_mlp_loss_grad": (_I32, [_P, _P, _P, _I64, ctypes.POINTER(ctypes.c_double), _P, _P]),
    "s3_mlp_adam_step": (_I32, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "s3_warmstart": (_I32, [_P, _P, _P, _P]),
    "s3_mlp_target": (_I32, [_P, _P, _P, _P]),
    "s3_mlp_destroy": (_I32, [_P]),
    "s3_fma_peak": (_I32, [_I32, _I32, ctypes.POINTER(s3_peak_result), _P]),
    "s3_destroy": (_I32, [_P]),
    "s3_last_error": (ctypes.c_char_p, []),
    "s3_status_string": (ctypes.c_char_p, [_I32]),
    "s3_version": (_I32, []),
}

_lib = None


def load():
    """Load libs3ttvc.so (build it first with ``paper_2311_08595_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libs3ttvc.so is not built ({LIB_PATH}); run `python -m paper_2311_08595_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_name(st):
    try:
        return load().s3_status_string(int(st)).decode()
    except Exception:
        return str(st)


def check(st):
    if st != S3_OK:
        raise S3Error(st, load().s3_last_error().decode())


def ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()
