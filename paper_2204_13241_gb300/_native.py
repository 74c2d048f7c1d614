"""ctypes declarations of libxs.so (include/xs_api.h).

Loading fails loudly: there is no CPU fallback behind this package.  Build the
library first with ``python -c "import __graft_entry__ as g; g.build()"`` or
``python paper_2204_13241_gb300/build.py``.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

XS_OK = 0
STATUS_NAMES = {0: "XS_OK", 1: "XS_ERR_INVALID_ARG", 2: "XS_ERR_UNSUPPORTED", 3: "XS_ERR_NO_MEMORY",
                4: "XS_ERR_CUDA", 5: "XS_ERR_TIMEOUT", 6: "XS_ERR_NUMERIC", 7: "XS_ERR_BOUNDS"}
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2, "fp32f": 3}

EXPORTS = ["xs_context_create", "xs_context_destroy", "xs_intensity", "xs_intensity_batched", "xs_g2",
           "xs_xsvs_contrast", "xs_ring_index", "xs_intensity_backward", "xs_tune", "xs_last_error",
           "xs_sync_status", "xs_set_wait_timeout_ns", "xs_version", "xs_profile_enable", "xs_profile_read",
           "xs_launch_count", "xs_intensity_fp32_static", "xs_isf", "xs_contrast_from_isf", "xs_intensity_species",
           "xs_intensity_points", "xs_ewald_points", "xs_intensity_fft", "xs_xsvs_partial", "xs_xsvs_finalize",
           "xs_xpcs_batched", "xs_tuned_choice", "xs_set_table_builder"]


class XsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Box(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double * 9)]


class QGrid(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("nx0", "nx", "ny0", "ny", "nz0", "nz")]


class Traj(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("pos_on_host", ctypes.c_int32), ("f", ctypes.c_void_p),
                ("n_atoms", ctypes.c_int64), ("n_frames", ctypes.c_int64), ("box", Box)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class CorrRequest(ctypes.Structure):
    _fields_ = [("taus", ctypes.c_void_p), ("n_tau", ctypes.c_int32), ("g2_out", ctypes.c_void_p),
                ("mean_out", ctypes.c_void_p), ("Ks", ctypes.c_void_p), ("n_K", ctypes.c_int32),
                ("ring_width", ctypes.c_double), ("n_rings", ctypes.c_int32), ("beta_out", ctypes.c_void_p),
                ("ring_count_out", ctypes.c_void_p)]


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Loads libxs.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libxs.so is not built ({path}); run paper_2204_13241_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "xs_context_create": ([ctypes.POINTER(Allocator), ctypes.POINTER(P)], st),
        "xs_context_destroy": ([P], st),
        "xs_intensity": ([P, ctypes.POINTER(Traj), ctypes.POINTER(QGrid), st, P, P, P], st),
        "xs_intensity_batched": ([P, ctypes.POINTER(Traj), ctypes.POINTER(QGrid), I32, st, P, P], st),
        "xs_xpcs_batched": ([P, ctypes.POINTER(Traj), ctypes.POINTER(QGrid), I32, st, P, ctypes.POINTER(CorrRequest),
                             P], st),
        "xs_g2": ([P, P, I64, I64, P, I32, P, P, P], st),
        "xs_xsvs_contrast": ([P, P, I64, ctypes.POINTER(QGrid), ctypes.POINTER(Box), P, I32, D, I32, P, P, P], st),
        "xs_ring_index": ([ctypes.POINTER(QGrid), ctypes.POINTER(Box), D, I32, P], st),
        "xs_intensity_backward": ([P, ctypes.POINTER(Traj), ctypes.POINTER(QGrid), P, P, P, P], st),
        "xs_tune": ([P, ctypes.POINTER(Traj), ctypes.POINTER(QGrid), st, P], st),
        "xs_tuned_choice": ([P, I64, ctypes.POINTER(QGrid), st, ctypes.POINTER(I32), ctypes.POINTER(I32)], st),
        "xs_last_error": ([], ctypes.c_char_p),
        "xs_sync_status": ([P, P], st),
        "xs_set_wait_timeout_ns": ([P, I64], st),
        "xs_set_table_builder": ([P, I32], st),
        "xs_version": ([], ctypes.c_char_p),
        "xs_profile_enable": ([P, I32], st),
        "xs_profile_read": ([P, ctypes.c_char_p, ctypes.POINTER(D), ctypes.POINTER(I64)], st),
        "xs_launch_count": ([P, ctypes.POINTER(I64)], st),
        "xs_intensity_fp32_static": ([ctypes.POINTER(Traj), ctypes.POINTER(QGrid), P, P, P, P], st),
        "xs_isf": ([P, P, I64, I64, P, I32, D, P, P, P], st),
        "xs_intensity_points": ([P, ctypes.POINTER(Traj), P, I64, st, P, P, P], st),
        "xs_intensity_fft": ([P, ctypes.POINTER(Traj), I32, D, I32, ctypes.POINTER(QGrid), P, P, P], st),
        "xs_xsvs_partial": ([P, P, I64, I64, P, I32, P, I32, P, P, P], st),
        "xs_xsvs_finalize": ([P, P, I64, P, I32, I32, P], st),
        "xs_ewald_points": ([ctypes.POINTER(Box), P, I32, I32, I32, I32, P, P], st),
        "xs_intensity_species": ([P, ctypes.POINTER(Traj), P, I32, P, ctypes.POINTER(QGrid), st, P, P, P], st),
        "xs_contrast_from_isf": ([P, P, I64, ctypes.POINTER(QGrid), ctypes.POINTER(Box), P, I32, D, I32, P, P, P],
                                 st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != XS_OK:
        msg = load().xs_last_error()
        raise XsError(status, msg.decode() if msg else "")
