"""Options in combination, each against the oracle run with the same options:
ragged batches that mix the one-block-per-matrix and the whole-GPU kernels in
split precision and with balancing, the product-form square root on the
whole-GPU kernel, and the allocation-free entry point with k_max = 3 and the
product form.

Tolerances as in the single-option tests: 1e-12 relative for FP64 results
(1e-11 with k_max = 3), SPLIT_TOL (tests/parity.py) for split precision, compared in the balanced
frame where balancing is on.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import SPLIT_TOL
from tests.parity import oracle_at_plan
from tests.test_gpu_parity import check_logm, dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def ragged_batch(sizes, seed, scale_spread=0):
    rng = np.random.default_rng(seed)
    mats = [workloads.spd(1, n, seed=int(rng.integers(1 << 30)), lo=0.1, hi=10.0)[0] for n in sizes]
    if scale_spread:
        out = []
        for A in mats:
            D = 2.0 ** rng.integers(-scale_spread, scale_spread + 1, A.shape[0])
            out.append(A * D[:, None] / D[None, :])
        mats = out
    ns = np.array(sizes, dtype=np.int32)
    offs = np.zeros(len(sizes), dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    flat = np.concatenate([m.ravel() for m in mats])
    R = lg().Ragged(dev(flat), torch.tensor(ns, device="cuda"), torch.tensor(offs, device="cuda"), max(sizes))
    return mats, offs, R


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_ragged_mixed_kernels_split_precision(precision):
    sizes = [33, 300, 64, 257, 8]
    mats, offs, R = ragged_batch(sizes, seed=600)
    L, s, k, info = lg().logm_execute(R, precision=precision)
    out = L.values.cpu().numpy()
    for b, n in enumerate(sizes):
        assert int(info[b]) == 0
        Lr, d = oracle.logm(mats[b])
        assert rel(out[offs[b]:offs[b] + n * n].reshape(n, n), Lr) <= SPLIT_TOL, (n, precision)


def test_ragged_mixed_kernels_balanced():
    sizes = [17, 280, 96]
    mats, offs, R = ragged_batch(sizes, seed=610, scale_spread=10)
    L, s, k, info = lg().logm_execute(R, balance=True)
    out = L.values.cpu().numpy()
    for b, n in enumerate(sizes):
        Lr = oracle_at_plan(mats[b], int(s[b]), int(k[b]), int(info[b]), balance=1)
        _, dv = oracle.balance(mats[b])
        Lg = out[offs[b]:offs[b] + n * n].reshape(n, n)
        assert rel(Lg / dv[:, None] * dv[None, :], Lr / dv[:, None] * dv[None, :]) <= 1e-12, n


def test_product_form_sqrt_whole_gpu():
    n = 300
    A = workloads.identity_plus(1, n, seed=620)[0]
    X, A2, AI2, it, info = lg().logm_sqrt(dev(A[None]), db_form="product")
    Xr, itr, st = oracle.sqrtm_db(A, form=1)
    assert int(info[0]) == st == 0 and abs(int(it[0]) - itr) <= 1
    assert rel(X[0].cpu().numpy(), Xr) <= 1e-12


@pytest.mark.parametrize("opts", [{"k_max": 3, "db_form": 0}, {"k_max": 5, "db_form": 1}])
def test_noalloc_entry_with_options(opts):
    from paper_2401_10089_gb300 import _lib
    L = _lib.load()
    A = workloads.identity_plus(6, 48, seed=630, lo=0.2, hi=2.0)
    Ad = dev(A)
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max, b.n, b.offset = 6, _lib.DTYPE_F64, 48, 48, None, None
    o = _lib.LogmOptions()
    o.k_max, o.precision, o.max_sqrt, o.max_db_iter = opts["k_max"], _lib.PREC_FP64, 40, 50
    o.db_form, o.balance = opts["db_form"], 0
    for t in range(5):
        o.theta[t] = 0.0
    outd = torch.empty_like(Ad)
    s = torch.zeros(6, dtype=torch.int32, device="cuda")
    k = torch.zeros_like(s)
    info = torch.zeros_like(s)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.logm_execute_noalloc(ctypes.byref(b), ctypes.byref(o), ctypes.c_void_p(Ad.data_ptr()),
                                ctypes.c_void_p(outd.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(info.data_ptr()), stream)
    assert rc == 0
    torch.cuda.synchronize()
    out = outd.cpu().numpy()
    tol = 1e-11 if opts["k_max"] == 3 else 1e-12
    for i in range(6):
        check_logm(A[i], out[i], int(s[i]), int(k[i]), int(info[i]), tol=tol, k_max=opts["k_max"],
                   db_form=opts["db_form"])
    # balancing has no fixed-size home in the static scratch: refused
    o.balance = 1
    rc = L.logm_execute_noalloc(ctypes.byref(b), ctypes.byref(o), ctypes.c_void_p(Ad.data_ptr()),
                                ctypes.c_void_p(outd.data_ptr()), None, None, ctypes.c_void_p(info.data_ptr()), stream)
    assert rc == _lib.ERR_UNSUPPORTED


def test_k3_balanced_whole_gpu():
    n = 270
    A0 = np.eye(n) + 0.008 * np.random.default_rng(640).standard_normal((n, n)) / np.sqrt(n)
    D = 2.0 ** np.random.default_rng(641).integers(-8, 9, n)
    A = A0 * D[:, None] / D[None, :]
    L, s, k, info = lg().logm_execute(dev(A[None]), balance=True)
    Lr = oracle_at_plan(A, int(s[0]), int(k[0]), int(info[0]), balance=1)
    _, dv = oracle.balance(A)
    Lg = L[0].cpu().numpy()
    assert rel(Lg / dv[:, None] * dv[None, :], Lr / dv[:, None] * dv[None, :]) <= 1e-12
