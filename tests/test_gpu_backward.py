"""Differentiation form: logm_backward (hand-written adjoint through the graph
products and the Denman-Beavers iterations) against central finite
differences of the GPU forward (h = 1e-6, FP64) and against the oracle's
Frechet adjoint L(A^T, W), read off the block-triangular logarithm.

Tolerances: a central difference D(h) carries h^2 |f'''| / 6 of truncation
plus kappa u |f| / h of rounding noise of the forward map. For SPD inputs
with eigenvalues down to 1e-2 (kappa ~ 1e4) the noise alone reaches ~1e-6
relative at h = 1e-6, so each comparison allows 1e-6 relative plus twice
|D(h) - D(2h)|, a measured bound on both terms (the plan (s, k) is piecewise
constant; inputs are chosen away from its thresholds and the test checks that
every perturbed point keeps the plan). Against the exact Frechet
adjoint the adjoint of the computed map differs by the derivative of the
approximation error, bounded by the same backward-error analysis (u-level
relative) times the conditioning: 1e-11 relative here (measured on GB300:
1e-15 to 1e-13 for SPD inputs with cond up to 1e4).
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.test_gpu_parity import dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def f_and_grad(A, W, **kw):
    L, s, k, info, ctx = lg().logm_execute(dev(A), with_ctx=True, **kw)
    dA, binfo = lg().logm_backward(dev(A), ctx, dev(W), **kw)
    assert (info.cpu().numpy() == 0).all() and (binfo.cpu().numpy() == 0).all(), (info, binfo)
    return L.cpu().numpy(), dA.cpu().numpy(), s.cpu().numpy(), k.cpu().numpy()


def fd_dir(A, W, E, h=1e-6, **kw):
    Lp, sp, kp, _ = lg().logm_execute(dev(A + h * E), **kw)
    Lm, sm, km, _ = lg().logm_execute(dev(A - h * E), **kw)
    fp = (W * Lp.cpu().numpy()).sum(axis=(-2, -1))
    fm = (W * Lm.cpu().numpy()).sum(axis=(-2, -1))
    return (fp - fm) / (2 * h), (sp.cpu().numpy(), kp.cpu().numpy(), sm.cpu().numpy(), km.cpu().numpy())


def fd_with_error(A, W, E, h=1e-6, **kw):
    """(D(h), |D(h) - D(2h)|, plans at +-h, whether the +-2h points kept
    the same plan) from central differences at h and 2h."""
    d1, p1 = fd_dir(A, W, E, h, **kw)
    d2, p2 = fd_dir(A, W, E, 2 * h, **kw)
    same = ((p1[0] == p2[0]) & (p1[1] == p2[1]) & (p1[2] == p2[2]) & (p1[3] == p2[3]))
    return d1, np.abs(d1 - d2), p1, same


@pytest.mark.parametrize("case", ["spd64", "dense48", "near_identity", "kmax2", "kmax1"])
def test_backward_vs_central_differences(case):
    rng = np.random.default_rng(["spd64", "dense48", "near_identity", "kmax2", "kmax1"].index(case) + 90)
    kw = {}
    if case == "spd64":
        A = workloads.spd(3, 64, seed=80, lo=1e-2, hi=1e2)
    elif case == "dense48":
        A = workloads.identity_plus(3, 48, seed=81, lo=0.5, hi=3.0)
    elif case == "near_identity":
        A = workloads.identity_plus(3, 32, seed=82, lo=0.05, hi=0.2)  # s = 0
    elif case == "kmax2":  # Theta_2 = 1.53e-4: keep s within the 12 checkpointed levels
        A = workloads.identity_plus(3, 24, seed=83, lo=0.02, hi=0.05)
        kw = {"k_max": 2}
    else:  # Theta_1 = 1.83e-8
        A = workloads.identity_plus(3, 16, seed=84, lo=2e-5, hi=5e-5)
        kw = {"k_max": 1}
    W = rng.standard_normal(A.shape)
    L, dA, s, k = f_and_grad(A, W, **kw)
    if case == "near_identity":
        assert (s == 0).all()
    for t in range(3):
        E = rng.standard_normal(A.shape)
        fd, fd_err, plans, same2 = fd_with_error(A, W, E, **kw)
        same = same2 & (plans[0] == s) & (plans[1] == k) & (plans[2] == s) & (plans[3] == k)
        an = (dA * E).sum(axis=(-2, -1))
        for b in range(A.shape[0]):
            if same[b]:
                tol = 1e-5 if kw.get("k_max") == 1 else 1e-6  # k_max = 1: s ~ 28, cancellation ~u/Theta_1
                bound = tol * max(1.0, abs(fd[b])) + 2 * fd_err[b]
                assert abs(an[b] - fd[b]) <= bound, (case, b, an[b], fd[b], fd_err[b])


def test_backward_level_limit_status():
    # s above the 12 checkpointed levels (k_max = 1 needs ~20 roots here): info 6, NaN
    A = workloads.identity_plus(2, 16, seed=94, lo=0.2, hi=0.5)
    L, s, k, info, ctx = lg().logm_execute(dev(A), with_ctx=True, k_max=1)
    assert (s.cpu().numpy() > 12).all()
    dA, binfo = lg().logm_backward(dev(A), ctx, dev(np.ones_like(A)), k_max=1)
    assert (binfo.cpu().numpy() == 6).all() and torch.isnan(dA).all()


def test_backward_vs_oracle_frechet():
    A = workloads.spd(4, 32, seed=85, lo=1e-2, hi=1e2)
    A[1] = workloads.identity_plus(1, 32, seed=86, lo=1.0, hi=2.0)[0]
    W = np.random.default_rng(87).standard_normal(A.shape)
    L, dA, s, k = f_and_grad(A, W)
    for b in range(4):
        G, st = oracle.frechet_adjoint(A[b], W[b])
        assert st == 0
        err = rel(dA[b], G)
        print(f"b={b} s={s[b]} k={k[b]} rel={err:.2e}")
        assert err <= 1e-11, err


def test_autograd_function_and_gradcheck():
    A = workloads.spd(2, 40, seed=88, lo=0.1, hi=10.0)
    W = np.random.default_rng(89).standard_normal(A.shape)
    At = dev(A).requires_grad_(True)
    loss = (dev(W) * lg().logm(At)).sum()
    loss.backward()
    _, dA, _, _ = f_and_grad(A, W)
    assert np.array_equal(At.grad.cpu().numpy(), dA)
    A5 = torch.tensor(workloads.spd(1, 5, seed=90, lo=0.3, hi=3.0), dtype=torch.float64, device="cuda")
    A5.requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: lg().logm(X), (A5,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_backward_diff_configuration_sampled():
    """1024 SPD 64 x 64 (lambda log-uniform in [1e-2, 1e2]), loss = sum(W o log A):
    random-direction central differences for every matrix at once, the
    oracle's Frechet adjoint on a seeded sample."""
    A = workloads.spd(1024, 64, seed=91, lo=1e-2, hi=1e2)
    rng = np.random.default_rng(92)
    W = rng.standard_normal(A.shape)
    L, dA, s, k = f_and_grad(A, W)
    E = rng.standard_normal(A.shape)
    fd, plans = fd_dir(A, W, E)
    same = (plans[0] == s) & (plans[1] == k) & (plans[2] == s) & (plans[3] == k)
    an = (dA * E).sum(axis=(-2, -1))
    assert same.mean() > 0.95
    err = np.abs(an - fd)[same] / np.maximum(1.0, np.abs(fd[same]))
    # eigenvalues down to 1e-2 make |f'''| ~ 1e6: the h^2 truncation of the
    # central difference reaches ~1e-5 relative here (median ~1e-8)
    assert err.max() <= 1e-4 and np.median(err) <= 1e-7, (err.max(), np.median(err))
    for b in np.random.default_rng(93).choice(1024, 8, replace=False):
        G, st = oracle.frechet_adjoint(A[b], W[b])
        assert rel(dA[b], G) <= 1e-11, (b, rel(dA[b], G))
