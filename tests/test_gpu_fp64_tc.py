"""The whole-GPU kernel (n > 256) with its Gauss-Jordan updates on the tensor
cores (fp64_products="tc_sliced": each update's factors split into exact BF16
digits, digit products summed exactly in FP32 on tcgen05, the integer dot
product rounded to FP64 once) against the oracle at the FP64 path's
tolerance, and against the FP64-pipe path on the same inputs."""
import functools

import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.test_gpu_parity import check_logm, dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TC = {"fp64_products": "tc_sliced"}


@functools.lru_cache(maxsize=None)
def bench_family(n):
    A = workloads.triangular_similar(n, seed=2)
    return A, oracle.logm(A)


# n = 257 and 513: one-row / one-column edges of the 128 x 64 output tiles;
# 300: a partial last Gauss-Jordan panel (300 = 9 * 32 + 12)
@pytest.mark.parametrize("n", [257, 300, 513])
def test_tc_execute_parity(n):
    A = workloads.identity_plus(2, n, seed=200 + n)
    L, s, k, info = lg().logm_execute(dev(A), **TC)
    L = L.cpu().numpy()
    for b in range(2):
        check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]))


@pytest.mark.parametrize("n", [512, 1024])
def test_tc_bench_family_parity(n):
    """The bench's 4096^2 family (A = Q T Q^T, off-diagonal std 0.1/n; cond_1
    2.3e5 at 512, 4.3e5 at 1024) through every phase at full depth (s = 5,
    27 Denman-Beavers iterations): element-wise against Algorithm 1 as written,
    and against the FP64-pipe path (same plan)."""
    A, (Lr, d) = bench_family(n)
    L, s, k, info = lg().logm_execute(dev(A[None]), **TC)
    Lp, sp, kp, infop = lg().logm_execute(dev(A[None]))
    L, Lp = L[0].cpu().numpy(), Lp[0].cpu().numpy()
    assert (int(s[0]), int(k[0])) == (int(sp[0]), int(kp[0])) == (d["s"], d["k"]) == (5, 5)
    assert int(info[0]) == 0
    err = rel(L, Lr)
    err_pipe = rel(Lp, Lr)
    print(f"n={n} tc_sliced rel_err={err:.3e} pipe rel_err={err_pipe:.3e} tc_vs_pipe={rel(L, Lp):.3e}")
    assert err <= 1e-12


def test_tc_sqrt_parity():
    n = 300
    A = workloads.identity_plus(1, n, seed=333)[0]
    X, A2, AI2, it, info = lg().logm_sqrt(dev(A[None]), **TC)
    Xr, itr, st = oracle.sqrtm_db(A)
    assert int(info[0]) == 0 and abs(int(it[0]) - itr) <= 1
    assert rel(X[0].cpu().numpy(), Xr) <= 1e-12
    assert rel(AI2[0].cpu().numpy(), A - 2 * Xr + np.eye(n)) <= 1e-11


def test_tc_ragged_mixed_with_small():
    sizes = [33, 300, 64, 257, 600]
    rng = np.random.default_rng(9)
    mats = [workloads.spd(1, n, seed=int(rng.integers(1 << 30)), lo=0.1, hi=10.0)[0] for n in sizes]
    ns = np.array(sizes, dtype=np.int32)
    offs = np.zeros(len(sizes), dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    flat = np.concatenate([m.ravel() for m in mats])
    R = lg().Ragged(dev(flat), torch.tensor(ns, device="cuda"), torch.tensor(offs, device="cuda"), 600)
    L, s, k, info = lg().logm_execute(R, **TC)
    out = L.values.cpu().numpy()
    for b, n in enumerate(sizes):
        check_logm(mats[b], out[offs[b]:offs[b] + n * n].reshape(n, n), int(s[b]), int(k[b]), int(info[b]))


def test_tc_status_codes():
    """A zero matrix (a zero pivot: info 1, NaN result) and a NaN entry (info
    4) next to a regular matrix, whose result is unaffected."""
    n = 260
    good = workloads.identity_plus(1, n, seed=700, lo=0.5, hi=1.5)[0]
    A = np.stack([good, np.zeros((n, n)), good.copy()])
    A[2, 5, 7] = np.nan
    L, s, k, info = lg().logm_execute(dev(A), **TC)
    info = info.cpu().numpy()
    assert info[0] == 0 and info[1] == 1 and info[2] == 4, info
    Lh = L.cpu().numpy()
    assert np.isnan(Lh[1]).all() and np.isnan(Lh[2]).all()
    check_logm(A[0], Lh[0], int(s[0]), int(k[0]), int(info[0]))


def test_tc_4096_triangular_similar_properties():
    """The bench's 4096 x 4096 matrix: log A = Q log(T) Q^T with log(T) upper
    triangular and diag(log T) = log diag(T) (closed form at any size)."""
    n = 4096
    rng = np.random.default_rng(2)
    T = np.triu(rng.standard_normal((n, n)) * (0.1 / n), 1)
    T[np.diag_indices(n)] = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), n))
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    Qd = dev(q * np.sign(np.diag(r))[None, :])
    A = (Qd @ dev(T) @ Qd.T).contiguous()
    L, s, k, info = lg().logm_execute(A, **TC)
    assert int(info[0]) == 0, int(info[0])
    M = (Qd.T @ L @ Qd).cpu().numpy()
    scale = np.linalg.norm(M)
    lower = np.linalg.norm(np.tril(M, -1)) / scale
    dg = np.max(np.abs(np.diag(M) - np.log(np.diag(T)))) / np.max(np.abs(np.log(np.diag(T))))
    print(f"n=4096 tc_sliced s={int(s[0])} k={int(k[0])} lower={lower:.3e} diag={dg:.3e}")
    assert lower <= 1e-12 and dg <= 1e-12
