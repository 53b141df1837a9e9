"""ctypes binding of ``libdpvba.so`` (declared in ``include/dpvba.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Loading fails loudly if the library was not built;
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdpvba.so")

BA_OK, BA_ERR_INVALID_ARG, BA_ERR_CUDA, BA_ERR_OOM, BA_ERR_NOT_SPD, BA_ERR_TIMEOUT, BA_ERR_STATE, \
    BA_ERR_UNSUPPORTED = range(8)
BA_FP32, BA_MIXED = 0, 1
(EXPORT_S, EXPORT_Y, EXPORT_DX, EXPORT_DD, EXPORT_CT, EXPORT_W, EXPORT_PERM, EXPORT_SLOTS, EXPORT_GPTR,
 EXPORT_WIN, EXPORT_COST, EXPORT_PMPOS, EXPORT_PPTR) = range(13)
WMAX = 64


BA_DENSE_AUTO, BA_DENSE_ALWAYS, BA_DENSE_NEVER = 0, 1, 2


class BAOptions(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("lambda_pose", ctypes.c_float),
        ("lambda_depth", ctypes.c_float),
        ("z_min", ctypes.c_float),
        ("d_min", ctypes.c_float),
        ("patches_per_group", ctypes.c_int),
        ("max_refine", ctypes.c_int),
        ("timeout_cycles", ctypes.c_longlong),
        ("stream", ctypes.c_void_p),
        ("residual_pixels", ctypes.c_int),
        ("dense_policy", ctypes.c_int),
    ]


EXPORTED = [
    "ba_default_options", "ba_create", "ba_destroy", "ba_set_stream", "ba_set_graph", "ba_set_graph_batched",
    "ba_step", "ba_sync",
    "ba_last_error", "ba_status_string", "ba_linearize", "ba_debug_export", "ba_debug_info", "ba_debug_keys", "ba_debug_envelope",
    "ba_profile_enable", "ba_profile_classes", "ba_profile_read", "ba_set_record", "ba_backward", "ba_solve_pose_system_noalloc",
    "ba_set_capture", "ba_autotune", "ba_autotune_clear", "ba_proximity_edges", "ba_patch_correlation", "ba_pgo_lm",
]
KERNEL_CLASSES = ("preprocess", "init", "assemble", "solve", "backsub", "retract", "adjoint", "factor",
                  "proximity", "correlation", "pgo")


class BAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


_lib = None


def lib():
    """Load the library (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; run `python -m paper_2408_01654_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        P = ctypes.c_void_p
        i = ctypes.c_int
        L.ba_default_options.argtypes = [ctypes.POINTER(BAOptions)]
        L.ba_create.argtypes = [ctypes.POINTER(H), ctypes.POINTER(BAOptions)]
        L.ba_destroy.argtypes = [H]
        L.ba_set_stream.argtypes = [H, P]
        L.ba_set_graph.argtypes = [H, i, i, i, P, P, P, P, P, P, P, P]
        L.ba_set_graph_batched.argtypes = [H, i, P, P, P, P, P, P, P, P, P, P, P]
        L.ba_step.argtypes = [H, i, i]
        L.ba_sync.argtypes = [H]
        L.ba_last_error.argtypes = [H]
        L.ba_last_error.restype = ctypes.c_char_p
        L.ba_status_string.argtypes = [i]
        L.ba_status_string.restype = ctypes.c_char_p
        L.ba_linearize.argtypes = [H, i]
        L.ba_debug_export.argtypes = [H, i, P, ctypes.c_longlong]
        L.ba_debug_info.argtypes = [H, ctypes.POINTER(ctypes.c_longlong), i]
        L.ba_debug_keys.argtypes = [H, i, P, i, ctypes.POINTER(ctypes.c_int)]
        L.ba_debug_envelope.argtypes = [H, ctypes.POINTER(ctypes.c_int), ctypes.c_longlong,
                                        ctypes.POINTER(ctypes.c_longlong)]
        L.ba_profile_enable.argtypes = [H, i]
        L.ba_profile_classes.argtypes = [H, ctypes.c_uint]
        L.ba_profile_read.argtypes = [H, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
        L.ba_set_record.argtypes = [H, i]
        L.ba_backward.argtypes = [H, P, P, P, P, P, P]
        L.ba_solve_pose_system_noalloc.argtypes = [i, P, P, P, i, P]
        L.ba_pgo_lm.argtypes = [H, i, i, P, P, P, P, P, i, ctypes.c_double, ctypes.c_double, P, P]
        for name in EXPORTED:
            if name not in ("ba_last_error", "ba_status_string"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def check(h, status):
    if status != BA_OK:
        L = lib()
        msg = L.ba_last_error(h).decode() if h else L.ba_status_string(status).decode()
        raise BAError(status, msg or L.ba_status_string(status).decode())


def default_options(**kw) -> BAOptions:
    o = BAOptions()
    lib().ba_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o
