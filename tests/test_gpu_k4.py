"""The k = 4 (14+) scheme on the GPU against the oracle: plans that pick it
(alpha_14 in (Theta_3, Theta_4] = (1.33e-2, 9.31e-2]) on the one-block and
the whole-GPU kernels, its adjoint, and its split-precision products on the
packed (uniform batch) and ragged kernels. (Each square root about halves
alpha, so after a root alpha lands in (Theta_4, Theta_5] and the scheme is
taken at s = 0.)

Tolerances: 1e-12 relative for FP64 (the FP64 path's bound), 1e-11 for the
adjoint against the oracle's Frechet adjoint, SPLIT_TOL (tests/parity.py) for split precision.
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import SPLIT_TOL
from tests.test_gpu_backward import f_and_grad
from tests.test_gpu_parity import check_logm, dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def near_identity(count, n, seed, rho=0.05):
    # I + E with E Gaussian scaled to spectral radius rho: alpha_14 lies between
    # rho and ||E||, here inside (Theta_3, Theta_4], and s = 0
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        E = rng.standard_normal((n, n))
        E *= rho / np.max(np.abs(np.linalg.eigvals(E)))
        out.append(np.eye(n) + E)
    return np.stack(out)


@pytest.mark.parametrize("n", [40, 300])
def test_execute_picks_k4(n):
    A = near_identity(3, n, seed=700 + n)
    L, s, k, info = lg().logm_execute(dev(A))
    L, k = L.cpu().numpy(), k.cpu().numpy()
    assert (k == 4).sum() >= 2, k
    for b in range(3):
        check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]))


def test_backward_k4_vs_oracle_frechet():
    A = near_identity(3, 32, seed=720)
    W = np.random.default_rng(721).standard_normal(A.shape)
    L, dA, s, k = f_and_grad(A, W)
    assert (k == 4).sum() >= 2, k
    for b in range(3):
        G, st = oracle.frechet_adjoint(A[b], W[b])
        assert st == 0
        assert rel(dA[b], G) <= 1e-11


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_k4_split_precision_packed_and_ragged(precision):
    A = near_identity(4, 64, seed=730)
    L, s, k, info = lg().logm_execute(dev(A), precision=precision)
    assert (k.cpu().numpy() == 4).sum() >= 2
    L = L.cpu().numpy()
    for b in range(4):
        Lr, d = oracle.logm(A[b])
        assert rel(L[b], Lr) <= SPLIT_TOL
    sizes = [33, 64, 17]
    mats = [near_identity(1, n, seed=740 + n)[0] for n in sizes]
    ns = np.array(sizes, dtype=np.int32)
    offs = np.zeros(3, dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    R = lg().Ragged(dev(np.concatenate([m.ravel() for m in mats])), torch.tensor(ns, device="cuda"),
                    torch.tensor(offs, device="cuda"), 64)
    Lg, s, k, info = lg().logm_execute(R, precision=precision)
    out = Lg.values.cpu().numpy()
    for b, n in enumerate(sizes):
        Lr, d = oracle.logm(mats[b])
        assert int(info[b]) == 0
        assert rel(out[offs[b]:offs[b] + n * n].reshape(n, n), Lr) <= SPLIT_TOL
