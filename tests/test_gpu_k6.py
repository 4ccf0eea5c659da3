"""The k = 6 order (k_max = 6, opt-in) on the one-block-per-matrix kernels
against the oracle:
- the graph: eq. five_mult_degopt with the fitted k = 6 coefficients, five
  products, the last two factors formed after the in-place pass;
- the plan: Theta_6 = 0.372 and m_6 = 20 of Table Table_theta;
- Algorithm 1 on every block configuration (ragged sizes 4..256) and with
  FP32 storage.

Tolerances are those of the other FP64 tests:
- 1e-14 relative for the graph alone;
- 1e-12 for Algorithm 1 (tests/parity.py);
- 1e-6 with FP32 storage of L.
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.test_gpu_parity import check_logm, dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 9, 64, 100, 256])
def test_graph_parity_k6(n):
    rng = np.random.default_rng(60 + n)
    X = rng.standard_normal((3, n, n))
    X *= np.array([0.2, 0.3, 0.37])[:, None, None] / np.abs(X).sum(axis=1).max(axis=1)[:, None, None]
    Z = lg().logm_graph_eval(dev(X), 6).cpu().numpy()
    Zp = lg().logm_graph_eval(dev(X), 6, P3=dev(X @ X)).cpu().numpy()
    for b in range(3):
        assert rel(Z[b], oracle.graph_eval(X[b], 6)) <= 1e-14
        assert rel(Zp[b], oracle.graph_eval(X[b], 6, P3=X[b] @ X[b])) <= 1e-14


def test_plan_parity_k6():
    # norms around Theta_5 = 0.246 and Theta_6 = 0.372, and a diagonal with
    # alpha = 0.3 exactly (k = 6 at s = 0)
    rng = np.random.default_rng(61)
    mats = [workloads.identity_plus(1, 40, seed=int(rng.integers(1 << 30)), lo=lo, hi=lo)[0]
            for lo in (0.1, 0.24, 0.3, 0.37, 0.45, 1.0, 3.0)]
    mats += [np.diag(np.linspace(1.3, 0.8, 40)) + 1e-3 * np.triu(rng.standard_normal((40, 40)), 1)]
    A = np.stack(mats)
    fin, k, alpha, info = lg().logm_plan(dev(A), k_max=6)
    ks = []
    for b in range(A.shape[0]):
        f_r, k_r, a_r = oracle.plan(A[b], k_max=6)
        assert int(info[b]) == 0
        assert (bool(fin[b]), int(k[b])) == (f_r, k_r), b
        assert abs(float(alpha[b]) - a_r) <= 1e-10 * a_r
        ks.append(k_r)
    assert 6 in ks
    # with A_I2 (s >= 1)
    X, it, st = oracle.sqrtm_db(A[5])
    AI2 = A[5] - 2 * X + np.eye(40)
    fin, k, alpha, info = lg().logm_plan(dev(X[None]), dev(AI2[None]), k_max=6)
    f_r, k_r, a_r = oracle.plan(X, AI2, k_max=6)
    assert (bool(fin[0]), int(k[0])) == (f_r, k_r) and abs(float(alpha[0]) - a_r) <= 1e-10 * a_r


def test_execute_k6_identity_plus_256():
    # the batched FP64 workload's distribution (||E||_1 uniform in [0.2, 5]):
    # k = 6 takes no more square roots than k = 5, and fewer on some
    A = workloads.identity_plus(8, 256, seed=62)
    L6, s6, k6, i6 = lg().logm_execute(dev(A), k_max=6)
    L5, s5, k5, i5 = lg().logm_execute(dev(A))
    s6, s5, k6 = s6.cpu().numpy(), s5.cpu().numpy(), k6.cpu().numpy()
    assert (s6 <= s5).all() and s6.sum() < s5.sum()
    assert (k6 == 6).any()
    L6 = L6.cpu().numpy()
    for b in range(8):
        check_logm(A[b], L6[b], int(s6[b]), int(k6[b]), int(i6[b]), k_max=6)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_execute_k6_configurations(variant):
    """Every configuration of the one-block-per-matrix kernel, forced on the
    buckets it can serve, with k_max = 6."""
    sizes = (4, 8, 16, 32, 64, 128, 256)
    vals, ns, offs = workloads.ragged_spd(21, sizes, seed=63, lo=0.05, hi=20.0, dtype=np.float64)
    R = lg().Ragged(torch.tensor(vals, device="cuda"), torch.tensor(ns, device="cuda"),
                    torch.tensor(offs, device="cuda"), 256)
    max_bucket = {0: 5, 1: 3, 2: 2, 3: 5, 4: 2}[variant]
    table = [variant if b <= max_bucket else 0 for b in range(6)]
    old = lg().get_tuning()
    try:
        lg().set_tuning(table)
        L, s, k, info = lg().logm_execute(R, k_max=6)
    finally:
        lg().set_tuning(old)
    out = L.values.cpu().numpy()
    assert (info.cpu().numpy() == 0).all()
    for b in range(len(ns)):
        n = int(ns[b])
        A = vals[offs[b]:offs[b] + n * n].reshape(n, n)
        check_logm(A, out[offs[b]:offs[b] + n * n].reshape(n, n), int(s[b]), int(k[b]), int(info[b]), k_max=6)


def test_execute_k6_f32_storage():
    mats = workloads.spd(4, 48, seed=64, lo=0.1, hi=10.0).astype(np.float32)
    L, s, k, info = lg().logm_execute(dev(mats, torch.float32), k_max=6)
    L = L.cpu().numpy()
    for b in range(4):
        Lr, d = oracle.logm(mats[b].astype(np.float64), k_max=6)
        assert int(info[b]) == 0
        assert rel(L[b].astype(np.float64), Lr) < 1e-6


def test_full_size_sampled_k6():
    """The batched FP64 configuration (512 x 256^2, A = I + E, ||E||_1 uniform
    in [0.2, 5]) with k_max = 6: a seeded sample, the matrix with the most
    roots and a matrix that took k = 6 against the oracle."""
    A = workloads.identity_plus(512, 256, seed=1)
    L, s, k, info = lg().logm_execute(dev(A), k_max=6)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert (info == 0).all()
    s, k, L = s.cpu().numpy(), k.cpu().numpy(), L.cpu().numpy()
    assert (k == 6).any()
    pick = np.random.default_rng(0).choice(512, 6, replace=False)
    pick = np.concatenate([pick, [int(np.argmax(s)), int(np.argmax(k == 6))]])
    for b in pick:
        check_logm(A[b], L[b], int(s[b]), int(k[b]), int(info[b]), k_max=6)
