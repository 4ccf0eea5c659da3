"""Precision form: the graph products on the tensor cores (tcgen05) in split
TF32x3 / BF16x3 with FP32 accumulation, square roots and plan in FP64.

Tolerance ``SPLIT_TOL`` = 4 * 2^-22 (derived in tests/parity.py: slice
residues of about 2^-22, FP32 roundings of X, P_3 and the lin-combs, product
norms below Theta ||X||).
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import SPLIT_TOL
from tests.test_gpu_parity import dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC_TOL = {"tf32x3": SPLIT_TOL, "bf16x3": SPLIT_TOL}


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [8, 64, 100, 256, 300])
def test_graph_eval_split_precision(precision, k, n):
    rng = np.random.default_rng(70 + n + k)
    X = rng.standard_normal((3, n, n))
    X *= 0.2 / np.abs(X).sum(axis=1).max(axis=1)[:, None, None]
    Z = lg().logm_graph_eval(dev(X), k, precision=precision).cpu().numpy()
    Zp = lg().logm_graph_eval(dev(X), k, P3=dev(X @ X), precision=precision).cpu().numpy()
    for b in range(3):
        Zr = oracle.graph_eval(X[b], k)
        assert rel(Z[b], Zr) <= PREC_TOL[precision], rel(Z[b], Zr)
        assert rel(Zp[b], Zr) <= PREC_TOL[precision]


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_execute_split_precision(precision):
    A = workloads.identity_plus(16, 128, seed=71)
    L, s, k, info = lg().logm_execute(dev(A), precision=precision)
    L64, s64, k64, info64 = lg().logm_execute(dev(A))
    assert torch.equal(s.cpu(), s64.cpu()) and torch.equal(k.cpu(), k64.cpu())
    L = L.cpu().numpy()
    for b in range(16):
        Lr, d = oracle.logm(A[b])
        assert int(info[b]) == 0
        assert rel(L[b], Lr) <= PREC_TOL[precision], rel(L[b], Lr)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("n", [8, 40, 130, 300])
def test_packed_tma_path_matches_ragged_path(precision, n):
    """A uniform batch takes the packed, TMA-fed product kernel; the same
    matrices passed as a ragged batch take the kernel that forms its operand
    tiles in shared memory. Both run the same split arithmetic (accumulation
    order aside), so they agree far below the split-precision tolerance, and
    both match the FP64 oracle."""
    rng = np.random.default_rng(700 + n)
    X = rng.standard_normal((3, n, n))
    X *= 0.2 / np.abs(X).sum(axis=1).max(axis=1)[:, None, None]
    ks = torch.tensor([5, 3, 2], dtype=torch.int32, device="cuda")
    Zu = lg().logm_graph_eval(dev(X), ks, precision=precision).cpu().numpy()
    ns = torch.full((3,), n, dtype=torch.int32, device="cuda")
    offs = torch.arange(3, dtype=torch.int64, device="cuda") * n * n
    R = lg().Ragged(dev(X.reshape(-1)), ns, offs, n)
    Zr = lg().logm_graph_eval(R, ks, precision=precision).cpu().numpy().reshape(3, n, n)
    for b, k in enumerate((5, 3, 2)):
        Zo = oracle.graph_eval(X[b], k)
        assert rel(Zu[b], Zo) <= PREC_TOL[precision], (b, rel(Zu[b], Zo))
        assert rel(Zr[b], Zo) <= PREC_TOL[precision]
        assert rel(Zu[b], Zr[b]) <= 1e-6
