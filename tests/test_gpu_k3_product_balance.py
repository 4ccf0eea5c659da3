"""The k = 3 scheme (eq. eqP8pol), the product form of the Denman-Beavers
iteration and the diagonal balancing of Algorithm 1 on the GPU (through the
C ABI), each against the oracle run with the same option, on the
one-block-per-matrix kernels (n <= 256) and the whole-GPU kernel (n > 256).

Tolerances: FP64 paths 1e-12 relative (k_max = 3 needs more square roots:
1e-11, as in the k_max parity tests); split-precision graph SPLIT_TOL (tests/parity.py); the
adjoint with balancing against the oracle's exact Frechet adjoint 1e-11.
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import SPLIT_TOL
from tests.parity import oracle_at_plan
from tests.test_gpu_parity import check_logm, dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def near_identity(count, n, norm, seed):
    """I + E with ||E||_1 = norm exactly (a matrix the order search sends to
    k = 3 when Theta_2 < alpha <= Theta_3)."""
    rng = np.random.default_rng(seed)
    E = rng.standard_normal((count, n, n))
    E *= norm / np.abs(E).sum(axis=1).max(axis=1)[:, None, None]
    return E + np.eye(n)[None]


def badly_scaled(A0, spread, seed):
    """D A0 D^{-1} with D = diag(2^e), e uniform in [-spread, spread]."""
    rng = np.random.default_rng(seed)
    D = 2.0 ** rng.integers(-spread, spread + 1, A0.shape[:-1])
    return A0 * D[..., :, None] / D[..., None, :]


@pytest.mark.parametrize("n", [5, 40, 256, 300])
def test_order_search_takes_k3(n):
    A = near_identity(3, n, 0.006, seed=500 + n)
    L, s, k, info = lg().logm_execute(dev(A))
    L = L.cpu().numpy()
    for b in range(3):
        assert (int(s[b]), int(k[b])) == (0, 3)
        check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]))


@pytest.mark.parametrize("n", [16, 100, 300])
def test_k_max_3_parity(n):
    A = workloads.identity_plus(2, n, seed=510 + n, lo=0.3, hi=2.0)
    L, s, k, info = lg().logm_execute(dev(A), k_max=3)
    L = L.cpu().numpy()
    for b in range(2):
        assert int(k[b]) <= 3
        check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]), tol=1e-11, k_max=3)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_k3_split_precision_execute(precision):
    A = near_identity(4, 64, 0.008, seed=520)
    L, s, k, info = lg().logm_execute(dev(A), precision=precision)
    L = L.cpu().numpy()
    for b in range(4):
        assert int(info[b]) == 0 and int(k[b]) == 3
        Lr, d = oracle.logm(A[b])
        assert rel(L[b], Lr) <= SPLIT_TOL


@pytest.mark.parametrize("n", [1, 7, 32, 64, 129, 256, 300, 513])
def test_product_form_parity(n):
    A = workloads.identity_plus(2, n, seed=530 + n, hi=5.0 if n >= 16 else 0.9)
    L, s, k, info = lg().logm_execute(dev(A), db_form="product")
    L = L.cpu().numpy()
    for b in range(2):
        check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]), db_form=1)


def test_product_form_sqrt_entry_and_work_counts():
    mats = np.stack([workloads.dense_32(seed=s) for s in range(3)] + [workloads.spd(1, 32, seed=540)[0]])
    X, A2, AI2, it, info = lg().logm_sqrt(dev(mats), db_form="product")
    X = X.cpu().numpy()
    for b in range(4):
        Xr, itr, st = oracle.sqrtm_db(mats[b], form=1)
        assert int(info[b]) == st == 0 and abs(int(it[b]) - itr) <= 1
        assert rel(X[b], Xr) <= 1e-12
    # the product form takes one inversion and one product per step (none in
    # the first), eq. (ScalDB) two inversions (one in the first, none in the
    # first step of the second and later roots, which start from the
    # previous root's Y as A^{-1})
    A = workloads.identity_plus(8, 64, seed=541)
    st2 = torch.zeros((8, 4), dtype=torch.int32, device="cuda")
    stp = torch.zeros((8, 4), dtype=torch.int32, device="cuda")
    _, s2, k2, _ = lg().logm_execute(dev(A), stats=st2)
    _, sp, kp, _ = lg().logm_execute(dev(A), stats=stp, db_form="product")
    st2, stp = st2.cpu().numpy(), stp.cpu().numpy()
    s2, sp, kp = s2.cpu().numpy(), sp.cpu().numpy(), kp.cpu().numpy()
    for b in range(8):
        reused = max(0, int(s2[b]) - 1)
        assert st2[b, 1] == 2 * st2[b, 0] - s2[b] - reused  # two per step, one in a level's first, none if reused
        assert stp[b, 1] == stp[b, 0]  # one inversion per step
        graph = kp[b] - (1 if sp[b] >= 1 else 0)  # P_3 = A_I2 is free once s >= 1
        assert stp[b, 2] == stp[b, 0] - sp[b] + graph  # one product per step but a level's first


@pytest.mark.parametrize("n", [6, 48, 200, 300])
def test_balance_parity_badly_scaled(n):
    A0 = workloads.spd(2, n, seed=550 + n, lo=0.05, hi=20.0)
    A = badly_scaled(A0, 12, seed=551 + n)
    L, s, k, info = lg().logm_execute(dev(A), balance=True)
    L = L.cpu().numpy()
    for b in range(2):
        Lr = oracle_at_plan(A[b], int(s[b]), int(k[b]), int(info[b]), balance=1)
        # compare in the balanced frame: D^{-1} L D is well scaled
        B, dvec = oracle.balance(A[b])
        Lg = L[b] / dvec[:, None] * dvec[None, :]
        Lo = Lr / dvec[:, None] * dvec[None, :]
        assert rel(Lg, Lo) <= 1e-12, rel(Lg, Lo)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_balance_split_precision(precision):
    A0 = workloads.spd(3, 96, seed=560, lo=0.1, hi=10.0)
    A = badly_scaled(A0, 10, seed=561)
    L, s, k, info = lg().logm_execute(dev(A), balance=True, precision=precision)
    L = L.cpu().numpy()
    for b in range(3):
        Lr, d = oracle.logm(A[b], balance=1)
        B, dvec = oracle.balance(A[b])
        assert rel(L[b] / dvec[:, None] * dvec[None, :], Lr / dvec[:, None] * dvec[None, :]) <= SPLIT_TOL


def test_balance_backward_vs_frechet():
    A0 = workloads.spd(3, 32, seed=570, lo=0.1, hi=10.0)
    A = badly_scaled(A0, 6, seed=571)
    W = np.random.default_rng(572).standard_normal(A.shape)
    L, s, k, info, ctx = lg().logm_execute(dev(A), with_ctx=True, balance=True)
    dA, binfo = lg().logm_backward(dev(A), ctx, dev(W), balance=True)
    assert (info.cpu().numpy() == 0).all() and (binfo.cpu().numpy() == 0).all()
    dA = dA.cpu().numpy()
    for b in range(3):
        G, st = oracle.frechet_adjoint(A[b], W[b])
        assert st == 0
        # the gradient of sum(W o log(D A0 D^-1)) in the frame of D: compare
        # D G D^-1 (well scaled), exactly the similarity the adjoint carries
        _, dvec = oracle.balance(A[b])
        assert rel(dA[b] * dvec[:, None] / dvec[None, :], G * dvec[:, None] / dvec[None, :]) <= 1e-11


def test_autograd_with_product_form_and_balance():
    A = badly_scaled(workloads.spd(2, 24, seed=580, lo=0.2, hi=5.0), 4, seed=581)
    W = np.random.default_rng(582).standard_normal(A.shape)
    At = dev(A).requires_grad_(True)
    (dev(W) * lg().logm(At, db_form="product", balance=True)).sum().backward()
    for b in range(2):
        G, st = oracle.frechet_adjoint(A[b], W[b])
        _, dvec = oracle.balance(A[b])
        g = At.grad[b].cpu().numpy()
        assert rel(g * dvec[:, None] / dvec[None, :], G * dvec[:, None] / dvec[None, :]) <= 1e-11
