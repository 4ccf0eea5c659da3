"""The CUDA library builds, loads and exports every symbol include/logm.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "logm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(logm_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2401_10089_gb300 import _build, _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 8
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(_lib.EXPORTS) | set(names)
    assert set(_lib.EXPORTS) == set(names)


def test_workspace_queries_without_gpu():
    from paper_2401_10089_gb300 import _lib
    L = _lib.load()
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max = 4, 0, 32, 32
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 5, 0, 40, 50
    assert L.logm_context_size(ctypes.byref(b), ctypes.byref(o)) > 4 * 32 * 32 * 8
    bad = _lib.LogmBatch()
    bad.count, bad.dtype, bad.n_uniform, bad.n_max = 4, 7, 32, 32
    assert L.logm_context_size(ctypes.byref(bad), ctypes.byref(o)) == 0


def test_invalid_arguments_rejected_before_launch():
    from paper_2401_10089_gb300 import _lib
    L = _lib.load()
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max = 1, 0, 8, 8
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 7, 0, 40, 50  # k_max = 7 has no scheme
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_INVALID_ARG
    o.k_max, o.precision = 6, 1  # k = 6 has no split-precision graph
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_INVALID_ARG
    o.precision = 0
    o.k_max, o.db_form = 5, 2  # no such Denman-Beavers form
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_INVALID_ARG
    o.db_form, o.balance = 0, 3  # no such balancing
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_INVALID_ARG
    o.balance = 0
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_INVALID_ARG


def test_execute_host_argument_checks():
    # refusals that happen before any CUDA call
    from paper_2401_10089_gb300 import _lib
    L = _lib.load()
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max = 2, 0, 0, 8  # ragged: not supported on host buffers
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 5, 0, 40, 50
    n = (ctypes.c_int32 * 2)(8, 8)
    b.n = ctypes.cast(n, ctypes.c_void_p)
    b.offset = ctypes.cast((ctypes.c_int64 * 2)(0, 64), ctypes.c_void_p)
    rc = L.logm_execute_host(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_UNSUPPORTED
    b.n_uniform = 8
    b.count = 0
    rc = L.logm_execute_host(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, 0, None)
    assert rc == _lib.SUCCESS  # empty batch: nothing to do
    o.k_max = 7
    rc = L.logm_execute_host(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_INVALID_ARG
    o.k_max, b.n_uniform, b.n_max = 6, 300, 300  # k = 6: n <= 256 only
    rc = L.logm_execute_host(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_UNSUPPORTED


def test_k6_option_limits():
    # k_max = 6 is taken by the one-block-per-matrix kernels (n <= 256), with
    # FP64 products and without the adjoint; everything else is refused
    # before any CUDA call
    from paper_2401_10089_gb300 import _lib
    L = _lib.load()
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max = 1, 0, 300, 300
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 6, 0, 40, 50
    args = (None,) * 8 + (0, None)
    assert L.logm_execute(ctypes.byref(b), ctypes.byref(o), *args) == _lib.ERR_UNSUPPORTED
    assert L.logm_plan(ctypes.byref(b), ctypes.byref(o), *((None,) * 7), 0, None) == _lib.ERR_UNSUPPORTED
    b.n_uniform = b.n_max = 64
    ctx = ctypes.c_void_p(256)  # never dereferenced: refused first
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, ctx, None, 0, None)
    assert rc == _lib.ERR_UNSUPPORTED
    rc = L.logm_backward(ctypes.byref(b), ctypes.byref(o), None, None, None, None, None, None, 0, None)
    assert rc == _lib.ERR_UNSUPPORTED
    L.logm_workspace_size.restype = ctypes.c_size_t
    assert L.logm_workspace_size(ctypes.byref(b), ctypes.byref(o)) > 0
    # the allocation-free entry point takes k_max = 6 (an empty batch returns
    # before any CUDA call) and refuses 7
    b.count = 0
    assert L.logm_execute_noalloc(ctypes.byref(b), ctypes.byref(o), *((None,) * 6)) == _lib.SUCCESS
    o.k_max = 7
    assert L.logm_execute_noalloc(ctypes.byref(b), ctypes.byref(o), *((None,) * 6)) == _lib.ERR_INVALID_ARG


def test_host_workspace_layout_size():
    # logm_execute_host's device workspace: logm_execute's own workspace first
    # (at the caller's aligned base), then the device copies of A and L and
    # the three int32 result arrays, each rounded up to 256 bytes
    from paper_2401_10089_gb300 import _lib
    L = _lib.load()
    L.logm_workspace_size.restype = ctypes.c_size_t
    L.logm_host_workspace_size.restype = ctypes.c_size_t
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 5, 0, 40, 50

    def r256(x):
        return (x + 255) // 256 * 256

    for n, count, dtype, esz in ((32, 4, 0, 8), (300, 1, 0, 8), (256, 512, 0, 8), (48, 20, 1, 4)):
        b = _lib.LogmBatch()
        b.count, b.dtype, b.n_uniform, b.n_max = count, dtype, n, n
        inner = L.logm_workspace_size(ctypes.byref(b), ctypes.byref(o))
        host = L.logm_host_workspace_size(ctypes.byref(b), ctypes.byref(o))
        assert inner > 0
        assert host == r256(inner) + 2 * r256(count * n * n * esz) + r256(12 * count)
