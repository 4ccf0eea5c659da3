"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerance: relative Frobenius error <= 1e-12 for the FP64 path on inputs with
cond(A) <= 1e4 (the target the method's FP64 path is held to). The oracle runs
Algorithm 1 with eq. (ScalDB) as written at every square-root level; the GPU
starts later levels from the previous level's Y (the same iterates in exact
arithmetic). Plan decisions (s, k) must agree unless the oracle met a
comparison within 1e-10 of its threshold where the two runs part
(``tests/parity.py``).
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import TOL, check_logm, rel  # noqa: F401  (re-exported for the other GPU tests)

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def lg():
    import paper_2401_10089_gb300 as m
    return m


def dev(a, dtype=None):
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float64, device="cuda")


def test_execute_dense_32():
    A = workloads.dense_32()
    L, s, k, info = lg().logm_execute(dev(A))  # a 2-D input gives a 2-D L
    assert L.shape == (32, 32)
    check_logm(A, L.cpu().numpy(), int(s[0]), int(k[0]), int(info[0]))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 24, 63, 64, 65, 100, 129])
def test_execute_sizes(n):
    # I + E with ||E||_1 up to 5 has eigenvalues on the negative real axis when n
    # is tiny (no real logarithm); keep ||E||_1 < 1 there.
    mats = workloads.identity_plus(6, n, seed=100 + n, hi=5.0 if n >= 16 else 0.9)
    L, s, k, info = lg().logm_execute(dev(mats))
    L = L.cpu().numpy()
    for b in range(mats.shape[0]):
        check_logm(mats[b], L[b], int(s[b]), int(k[b]), int(info[b]))


def test_execute_ragged():
    sizes = [1, 4, 7, 16, 33, 64, 65, 97, 128, 130, 256]
    rng = np.random.default_rng(7)
    mats = [workloads.spd(1, n, seed=int(rng.integers(1 << 30)), lo=0.05, hi=20.0)[0] for n in sizes]
    ns = np.array(sizes, dtype=np.int32)
    offs = np.zeros(len(sizes), dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    flat = np.concatenate([m.ravel() for m in mats])
    R = lg().Ragged(dev(flat), torch.tensor(ns, device="cuda"), torch.tensor(offs, device="cuda"), 256)
    L, s, k, info = lg().logm_execute(R)
    out = L.values.cpu().numpy()
    for b, n in enumerate(sizes):
        check_logm(mats[b], out[offs[b]:offs[b] + n * n].reshape(n, n), int(s[b]), int(k[b]), int(info[b]))


def test_execute_f32_storage():
    mats = workloads.spd(4, 48, seed=11, lo=0.1, hi=10.0).astype(np.float32)
    L, s, k, info = lg().logm_execute(dev(mats, torch.float32))
    L = L.cpu().numpy()
    for b in range(4):
        Lr, d = oracle.logm(mats[b].astype(np.float64))
        # FP64 arithmetic, FP32 rounding of the stored result
        assert rel(L[b].astype(np.float64), Lr) < 1e-6


# With k_max = 1 or 2 the loop takes roots until ||A^{1/2^s} - I|| is about
# Theta_1 = 1.83e-8 or Theta_2 = 1.53e-4, so X = I - A^{1/2^s} carries a
# relative cancellation error of about u / Theta on either side.
KMAX_TOL = {1: 1e-7, 2: 1e-10, 3: 1e-11, 4: TOL, 5: TOL}


@pytest.mark.parametrize("k_max", [1, 2, 3, 4, 5])
def test_execute_k_max(k_max):
    mats = workloads.identity_plus(4, 20, seed=21, lo=0.05, hi=0.5)
    L, s, k, info = lg().logm_execute(dev(mats), k_max=k_max)
    L = L.cpu().numpy()
    for b in range(4):
        check_logm(mats[b], L[b], int(s[b]), int(k[b]), int(info[b]), tol=KMAX_TOL[k_max], k_max=k_max)


def test_plan_parity():
    rng = np.random.default_rng(30)
    mats = [workloads.identity_plus(1, 40, seed=int(rng.integers(1 << 30)), lo=lo, hi=lo)[0]
            for lo in (0.01, 0.1, 0.2, 0.24, 0.5, 1.0, 3.0)]
    mats += [np.eye(40) + 1e-9 * rng.standard_normal((40, 40)), np.eye(40) + 1e-5 * rng.standard_normal((40, 40))]
    A = np.stack(mats)
    fin, k, alpha, info = lg().logm_plan(dev(A))
    for b in range(A.shape[0]):
        f_r, k_r, a_r = oracle.plan(A[b])
        assert int(info[b]) == 0
        assert (bool(fin[b]), int(k[b])) == (f_r, k_r), b
        assert abs(float(alpha[b]) - a_r) <= 1e-10 * a_r
    # with A_I2 (s >= 1)
    X, it, st = oracle.sqrtm_db(A[5])
    AI2 = A[5] - 2 * X + np.eye(40)
    fin, k, alpha, info = lg().logm_plan(dev(X[None]), dev(AI2[None]))
    f_r, k_r, a_r = oracle.plan(X, AI2)
    assert (bool(fin[0]), int(k[0])) == (f_r, k_r) and abs(float(alpha[0]) - a_r) <= 1e-10 * a_r


@pytest.mark.parametrize("k_max", [3, 4, 5])
def test_plan_parity_k_max(k_max):
    # the order search's choice among k in 1..k_max near
    # the identity, where every order is in play
    rng = np.random.default_rng(31)
    mats = [np.eye(30) + e * rng.standard_normal((30, 30)) / 30 for e in (1e-9, 1e-5, 3e-3, 8e-3, 0.05)]
    A = np.stack(mats)
    fin, k, alpha, info = lg().logm_plan(dev(A), k_max=k_max)
    for b in range(A.shape[0]):
        f_r, k_r, a_r = oracle.plan(A[b], k_max=k_max)
        assert int(info[b]) == 0 and (bool(fin[b]), int(k[b])) == (f_r, k_r), (b, int(k[b]), k_r)


def test_sqrt_parity():
    mats = np.stack([workloads.dense_32(seed=s) for s in range(4)])
    Ad = dev(mats)
    A, A2, AI2, it, info = lg().logm_sqrt(Ad)
    X = A.cpu().numpy()
    for b in range(4):
        Xr, itr, st = oracle.sqrtm_db(mats[b])
        assert int(info[b]) == st == 0
        assert abs(int(it[b]) - itr) <= 1
        assert rel(X[b], Xr) <= TOL
        assert np.array_equal(A2.cpu().numpy()[b], mats[b])
        assert rel(AI2.cpu().numpy()[b], mats[b] - 2 * Xr + np.eye(32)) <= 1e-11


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [1, 9, 64, 100, 256])
def test_graph_parity(k, n):
    rng = np.random.default_rng(40 + n)
    X = rng.standard_normal((3, n, n))
    X *= 0.2 / np.abs(X).sum(axis=1).max(axis=1)[:, None, None]
    Z = lg().logm_graph_eval(dev(X), k).cpu().numpy()
    Zp = lg().logm_graph_eval(dev(X), k, P3=dev(X @ X)).cpu().numpy()
    for b in range(3):
        Zr = oracle.graph_eval(X[b], k)
        assert rel(Z[b], Zr) <= 1e-14
        assert rel(Zp[b], oracle.graph_eval(X[b], k, P3=X[b] @ X[b])) <= 1e-14


def test_status_codes():
    n = 8
    A = np.stack([np.eye(n), np.zeros((n, n)), workloads.dense_32(n=n), np.eye(n)])
    A[3, 2, 2] = np.nan
    L, s, k, info = lg().logm_execute(dev(A), max_sqrt=40)
    info = info.cpu().numpy()
    assert info[0] == 0 and info[1] == 1 and info[3] == 4
    assert np.allclose(L[0].cpu().numpy(), 0.0)
    assert np.isnan(L[1].cpu().numpy()).all() and np.isnan(L[3].cpu().numpy()).all()
    L, s, k, info = lg().logm_execute(dev(A[2:3]), max_sqrt=1)
    assert int(info[0]) == 3 and int(s[0]) == 1


def test_full_size_sampled():
    """512 x 256^2, A = I + E (||E||_1 uniform in [0.2, 5]) -- the batched FP64
    configuration; the oracle checks a seeded sample of the matrices."""
    A = workloads.identity_plus(512, 256, seed=1)
    L, s, k, info = lg().logm_execute(dev(A))
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert (info == 0).all()
    s, k, L = s.cpu().numpy(), k.cpu().numpy(), L.cpu().numpy()
    pick = np.random.default_rng(0).choice(512, 6, replace=False)
    pick = np.concatenate([pick, [int(np.argmax(s))]])
    Ls, ds = oracle.logm_batch([A[b] for b in pick])
    for j, b in enumerate(pick):
        if (int(s[b]), int(k[b])) == (ds[j]["s"], ds[j]["k"]):
            assert rel(L[b], Ls[j]) <= TOL
        else:
            check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]))


def test_uniform_batch_one_round_configuration():
    # 800 matrices of 40 x 40: more than the 5-per-SM configuration holds at
    # once, fewer than its 7-per-SM twin, which then runs them in one round
    A = workloads.identity_plus(800, 40, seed=810, lo=0.2, hi=3.0)
    L, s, k, info = lg().logm_execute(dev(A))
    L, s, k, info = L.cpu().numpy(), s.cpu().numpy(), k.cpu().numpy(), info.cpu().numpy()
    for b in range(0, 800, 7):
        check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]))
