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


def _call_noalloc(lib, A, ragged=None):
    """logm_execute_noalloc on a uniform batch A (count x n x n), or on a
    packed ragged batch when ``ragged`` = (n tensor, offset tensor, n_max)
    and A holds the packed values."""
    from paper_2401_10089_gb300 import _lib
    b = _lib.LogmBatch()
    dt = _lib.DTYPE_F64 if A.dtype == torch.float64 else _lib.DTYPE_F32
    if ragged is None:
        count, n = A.shape[0], A.shape[1]
        b.count, b.dtype, b.n_uniform, b.n_max, b.n, b.offset = count, dt, n, n, None, None
    else:
        ns, offs, n_max = ragged
        count = int(ns.numel())
        b.count, b.dtype, b.n_uniform, b.n_max = count, dt, 0, n_max
        b.n, b.offset = ctypes.c_void_p(ns.data_ptr()), ctypes.c_void_p(offs.data_ptr())
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = 5, _lib.PREC_FP64, 40, 50
    for t in range(5):
        o.theta[t] = 0.0
    L = torch.full_like(A, float("nan"))
    s = torch.empty(count, dtype=torch.int32, device=A.device)
    k = torch.empty_like(s)
    info = torch.empty_like(s)
    stream = ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream)
    rc = lib.logm_execute_noalloc(ctypes.byref(b), ctypes.byref(o), ctypes.c_void_p(A.data_ptr()),
                                  ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                  ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(info.data_ptr()), stream)
    assert rc == _lib.SUCCESS, rc
    return L, s, k, info


def _agree(A_i, L_i, s_i, k_i, L_ref_i, s_ref_i, k_ref_i, tol=TOL):
    """The two entry points may run a matrix in different block
    configurations, whose norm estimates can round differently: with the same
    plan the results must agree to tol; with another plan (only near a
    threshold) the no-allocation result is checked against the oracle at its
    own plan."""
    if (s_i, k_i) == (s_ref_i, k_ref_i):
        assert _rel(L_i, L_ref_i) <= tol
    else:
        from tests.parity import check_logm
        check_logm(A_i, L_i, s_i, k_i, 0, tol=tol)


@pytest.mark.gpu
def test_noalloc_matches_execute_on_two_calls():
    import paper_2401_10089_gb300 as lg
    from paper_2401_10089_gb300 import _lib
    lib = _lib.load()
    # 12 x 256^2: more matrices than the scratch array holds slots for (9 at n = 256)
    batches = [workloads.identity_plus(40, 96, seed=501), workloads.identity_plus(12, 256, seed=502)]
    for A_np in batches:
        A = torch.tensor(A_np, device="cuda")
        L_ref, s_ref, k_ref, info_ref = lg.logm_execute(A)
        L, s, k, info = _call_noalloc(lib, A)
        torch.cuda.synchronize()
        assert torch.equal(info.cpu(), info_ref.cpu()) and (info.cpu() == 0).all()
        Ln, Lr = L.cpu().numpy(), L_ref.cpu().numpy()
        for i in range(A_np.shape[0]):
            _agree(A_np[i], Ln[i], int(s[i]), int(k[i]), Lr[i], int(s_ref[i]), int(k_ref[i]))


@pytest.mark.gpu
def test_noalloc_ragged_batch_and_out_of_range_size():
    """A ragged batch (device n and offsets, n_max from the batch): every
    matrix agrees with logm_execute; one matrix larger than the declared
    n_max is refused with info -1 and leaves the others unaffected."""
    import paper_2401_10089_gb300 as lg
    from paper_2401_10089_gb300 import _lib
    lib = _lib.load()
    sizes = [7, 33, 64, 300, 128, 200, 256, 1]
    rng = np.random.default_rng(520)
    mats = [workloads.spd(1, n, seed=int(rng.integers(1 << 30)), lo=0.05, hi=20.0)[0] for n in sizes]
    ns = np.array(sizes, dtype=np.int32)
    offs = np.zeros(len(sizes), dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    flat = torch.tensor(np.concatenate([m.ravel() for m in mats]), device="cuda")
    ns_d, offs_d = torch.tensor(ns, device="cuda"), torch.tensor(offs, device="cuda")
    L_ref, s_ref, k_ref, info_ref = lg.logm_execute(lg.Ragged(flat, ns_d, offs_d, 256))
    for _ in range(2):
        L, s, k, info = _call_noalloc(lib, flat, ragged=(ns_d, offs_d, 256))
        torch.cuda.synchronize()
        assert info.cpu().tolist() == [0, 0, 0, -1, 0, 0, 0, 0]
        assert torch.equal(info.cpu(), info_ref.cpu())
        out, ref = L.cpu().numpy(), L_ref.values.cpu().numpy()
        for b, n in enumerate(sizes):
            if n > 256:
                continue
            sl = slice(offs[b], offs[b] + n * n)
            _agree(mats[b], out[sl].reshape(n, n), int(s[b]), int(k[b]), ref[sl].reshape(n, n), int(s_ref[b]),
                   int(k_ref[b]))


@pytest.mark.gpu
def test_noalloc_f32_storage():
    """FP32 storage of A and L (FP64 arithmetic inside): the same results as
    logm_execute on the same FP32 matrices, to FP32 rounding of L."""
    import paper_2401_10089_gb300 as lg
    from paper_2401_10089_gb300 import _lib
    lib = _lib.load()
    A = torch.tensor(workloads.spd(10, 48, seed=530, lo=0.1, hi=10.0), device="cuda").float()
    L_ref, s_ref, k_ref, info_ref = lg.logm_execute(A)
    L, s, k, info = _call_noalloc(lib, A)
    torch.cuda.synchronize()
    assert (info.cpu() == 0).all() and torch.equal(info.cpu(), info_ref.cpu())
    Ln, Lr = L.double().cpu().numpy(), L_ref.double().cpu().numpy()
    for i in range(10):
        assert _rel(Ln[i], Lr[i]) <= 1e-6


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
