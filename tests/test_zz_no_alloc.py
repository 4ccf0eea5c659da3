"""logm_execute_noalloc: the entry point for callers that cannot allocate
device memory (its scratch space is a fixed device array inside the library).

Called through the C ABI with ctypes; its results must match logm_execute's,
within the FP64 path's tolerance, on two calls in a row (the second call runs
on the scratch contents the first one left behind). This file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2401_10089_gb300 import workloads

torch = pytest.importorskip("torch")

TOL = 1e-12


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _call_noalloc(lib, A):
    from paper_2401_10089_gb300 import _lib
    count, n = A.shape[0], A.shape[1]
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max, b.n, b.offset = count, _lib.DTYPE_F64, n, n, None, None
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 5, _lib.PREC_FP64, 40, 50
    for t in range(5):
        o.theta[t] = 0.0
    L = torch.empty_like(A)
    s = torch.empty(count, dtype=torch.int32, device=A.device)
    k = torch.empty_like(s)
    info = torch.empty_like(s)
    stream = ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream)
    rc = lib.logm_execute_noalloc(ctypes.byref(b), ctypes.byref(o), ctypes.c_void_p(A.data_ptr()),
                                  ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                  ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(info.data_ptr()), stream)
    assert rc == _lib.SUCCESS, rc
    return L, s, k, info


@pytest.mark.gpu
def test_noalloc_matches_execute_on_two_calls():
    import paper_2401_10089_gb300 as lg
    from paper_2401_10089_gb300 import _lib
    lib = _lib.load()
    batches = [workloads.identity_plus(40, 96, seed=501), workloads.identity_plus(12, 256, seed=502)]
    for A_np in batches:
        A = torch.tensor(A_np, device="cuda")
        L_ref, s_ref, k_ref, info_ref = lg.logm_execute(A)
        L, s, k, info = _call_noalloc(lib, A)
        torch.cuda.synchronize()
        assert torch.equal(info.cpu(), info_ref.cpu()) and (info.cpu() == 0).all()
        assert torch.equal(s.cpu(), s_ref.cpu()) and torch.equal(k.cpu(), k_ref.cpu())
        Ln, Lr = L.cpu().numpy(), L_ref.cpu().numpy()
        for i in range(A_np.shape[0]):
            assert _rel(Ln[i], Lr[i]) <= TOL


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_maximum():
    from paper_2401_10089_gb300 import _lib
    lib = _lib.load()
    A = torch.zeros((1, 300, 300), dtype=torch.float64, device="cuda")
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max = 1, _lib.DTYPE_F64, 300, 300
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 5, _lib.PREC_FP64, 40, 50
    out = torch.empty_like(A)
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = lib.logm_execute_noalloc(ctypes.byref(b), ctypes.byref(o), ctypes.c_void_p(A.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), None, None, ctypes.c_void_p(info.data_ptr()),
                                  None)
    assert rc == _lib.ERR_UNSUPPORTED
