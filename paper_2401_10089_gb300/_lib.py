"""ctypes view of the C ABI in ``include/logm.h`` (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU or
PyTorch fallback for any step of the method.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

SUCCESS, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_CUDA = 0, -1, -2, -3, -4
INFO_OK, INFO_SINGULAR, INFO_NO_CONVERGENCE, INFO_MAX_SQRT, INFO_NONFINITE = 0, 1, 2, 3, 4
DTYPE_F64, DTYPE_F32 = 0, 1
PREC_FP64, PREC_TF32X3, PREC_BF16X3 = 0, 1, 2

_ERRORS = {ERR_INVALID_ARG: "invalid argument", ERR_UNSUPPORTED: "unsupported", ERR_WORKSPACE: "workspace",
           ERR_CUDA: "CUDA launch error"}

# Every symbol include/logm.h declares.
EXPORTS = ("logm_workspace_size", "logm_context_size", "logm_backward_workspace_size", "logm_plan", "logm_sqrt",
           "logm_graph_eval", "logm_execute", "logm_backward", "logm_execute_noalloc", "logm_set_tuning",
           "logm_get_tuning", "logm_version", "logm_probe_barrier", "logm_host_workspace_size",
           "logm_execute_host")


class LogmBatch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n_uniform", ctypes.c_int32),
                ("n_max", ctypes.c_int32), ("n", ctypes.c_void_p), ("offset", ctypes.c_void_p)]


class LogmOptions(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_sqrt", ctypes.c_int32),
                ("max_db_iter", ctypes.c_int32), ("db_form", ctypes.c_int32), ("balance", ctypes.c_int32),
                ("fp64_products", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("theta", ctypes.c_double * 5)]


class LogmTuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32 * 6)]


class LogmError(RuntimeError):
    pass


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``liblogm.so`` (building it in-tree if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and _build._stale():
            _build.build()
        if not os.path.exists(path):
            raise LogmError(f"CUDA library {path} is missing; run paper_2401_10089_gb300._build.build()")
        L = ctypes.CDLL(path)
        P, I32, SZ, V = ctypes.POINTER, ctypes.c_int32, ctypes.c_size_t, ctypes.c_void_p
        B, O = P(LogmBatch), P(LogmOptions)
        L.logm_workspace_size.restype = SZ
        L.logm_workspace_size.argtypes = [B, O]
        L.logm_context_size.restype = SZ
        L.logm_context_size.argtypes = [B, O]
        L.logm_backward_workspace_size.restype = SZ
        L.logm_backward_workspace_size.argtypes = [B, O]
        L.logm_plan.argtypes = [B, O, V, V, V, V, V, V, V, SZ, V]
        L.logm_sqrt.argtypes = [B, O, V, V, V, V, V, V, V, SZ, V]
        L.logm_graph_eval.argtypes = [B, I32, V, V, V, V, V, SZ, V]
        L.logm_execute.argtypes = [B, O, V, V, V, V, V, V, V, V, SZ, V]
        L.logm_backward.argtypes = [B, O, V, V, V, V, V, V, SZ, V]
        L.logm_execute_noalloc.argtypes = [B, O, V, V, V, V, V, V]
        L.logm_set_tuning.argtypes = [P(LogmTuning)]
        L.logm_get_tuning.argtypes = [P(LogmTuning)]
        L.logm_version.argtypes = []
        L.logm_probe_barrier.argtypes = [I32, ctypes.c_double, V, SZ, V]
        L.logm_host_workspace_size.restype = SZ
        L.logm_host_workspace_size.argtypes = [B, O]
        L.logm_execute_host.argtypes = [B, O, V, V, V, V, V, V, SZ, V]
        for name in EXPORTS:
            getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
        L.logm_workspace_size.restype = SZ
        L.logm_context_size.restype = SZ
        L.logm_backward_workspace_size.restype = SZ
        L.logm_host_workspace_size.restype = SZ
        _lib = L
        _apply_shipped_tuning(L)
        return _lib


def check(rc: int, what: str):
    if rc != SUCCESS:
        raise LogmError(f"{what} failed: {_ERRORS.get(rc, rc)}")


# Tuning table the project's autotuner picked on GB300 (see autotune.py);
# applied when the library is first loaded.
TUNING_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def _apply_shipped_tuning(L):
    import json
    if not os.path.exists(TUNING_FILE):
        return
    with open(TUNING_FILE) as f:
        table = json.load(f).get("variant")
    if table and len(table) == 6:
        t = LogmTuning()
        for i, v in enumerate(table):
            t.variant[i] = int(v)
        L.logm_set_tuning(ctypes.byref(t))
