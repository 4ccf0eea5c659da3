"""Batching form: thousands of matrices of uneven n in one call (a persistent
launch for the FP64 stage, one tensor-core launch per graph product), FP32
storage, split-precision products, checked against the FP64 oracle; and the
whole call captured once in a CUDA graph and replayed.

Tolerance against the oracle ``SPLIT_TOL_F32`` (tests/parity.py): the split
products' bound plus the FP32 rounding of the stored L. The oracle runs on the
same FP32 values of A (read as FP64), so the storage of A adds nothing. The
property checks (symmetry, trace = log det) keep 1e-5: they compare FP32
results with FP64 quantities of matrices whose eigenvalues span [1e-3, 1e3].
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import SPLIT_TOL_F32
from tests.test_gpu_parity import check_logm, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = (4, 8, 16, 32, 64, 128, 256)


def ragged(count, seed):
    vals, ns, offs = workloads.ragged_spd(count, SIZES, seed=seed)
    R = lg().Ragged(torch.tensor(vals, device="cuda"), torch.tensor(ns, device="cuda"),
                    torch.tensor(offs, device="cuda"), max(SIZES))
    return vals, ns, offs, R


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3", "fp64"])
def test_ragged_spd_fp32_storage(precision):
    vals, ns, offs, R = ragged(700, seed=40)
    L, s, k, info = lg().logm_execute(R, precision=precision)
    out = L.values.cpu().numpy()
    info = info.cpu().numpy()
    assert (info == 0).all()
    rng = np.random.default_rng(41)
    for n in SIZES:  # two matrices of every size
        for b in rng.choice(np.nonzero(ns == n)[0], 2, replace=False):
            A = vals[offs[b]:offs[b] + n * n].reshape(n, n).astype(np.float64)
            Lr, d = oracle.logm(A)
            Lg = out[offs[b]:offs[b] + n * n].reshape(n, n).astype(np.float64)
            assert rel(Lg, Lr) <= SPLIT_TOL_F32, (precision, n, b, rel(Lg, Lr))


def test_execute_captured_in_cuda_graph():
    vals, ns, offs, R = ragged(300, seed=42)
    L_eager, s_e, k_e, i_e = lg().logm_execute(R, precision="tf32x3")  # also sets kernel attributes
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        lg().logm_execute(R, precision="tf32x3")  # warm the workspace cache on this stream
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            L_g, s_g, k_g, i_g = lg().logm_execute(R, precision="tf32x3")
    torch.cuda.current_stream().wait_stream(stream)
    for _ in range(2):
        L_g.values.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(L_g.values, L_eager.values)
        assert torch.equal(s_g, s_e) and torch.equal(k_g, k_e) and torch.equal(i_g, i_e)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_kernel_configurations_agree_with_oracle(variant):
    """Every configuration of the one-block-per-matrix kernel, forced on the
    buckets it can serve, matches the FP64 oracle (1e-12)."""
    sizes = (4, 8, 16, 32, 64, 128, 256)
    vals, ns, offs = workloads.ragged_spd(140, sizes, seed=43, lo=0.05, hi=20.0, dtype=np.float64)
    R = lg().Ragged(torch.tensor(vals, device="cuda"), torch.tensor(ns, device="cuda"),
                    torch.tensor(offs, device="cuda"), 256)
    max_bucket = {0: 5, 1: 3, 2: 2, 3: 5, 4: 2}[variant]
    table = [variant if b <= max_bucket else 0 for b in range(6)]
    old = lg().get_tuning()
    try:
        lg().set_tuning(table)
        L, s, k, info = lg().logm_execute(R)
    finally:
        lg().set_tuning(old)
    out = L.values.cpu().numpy()
    assert (info.cpu().numpy() == 0).all()
    for b in range(len(ns)):
        n = int(ns[b])
        A = vals[offs[b]:offs[b] + n * n].reshape(n, n)
        check_logm(A, out[offs[b]:offs[b] + n * n].reshape(n, n), int(s[b]), int(k[b]), int(info[b]))


def test_autotuner_picks_a_valid_table():
    from paper_2401_10089_gb300 import autotune
    vals, ns, offs, R = ragged(600, seed=44)
    old = lg().get_tuning()
    try:
        table, times = autotune.autotune(R, precision="fp64", sample=512, reps=1)
        assert len(table) == 6
        for b, v in enumerate(table):
            assert v in autotune.CANDIDATES[b]
        assert lg().get_tuning() == table
        L, s, k, info = lg().logm_execute(R, precision="tf32x3")
        assert (info.cpu().numpy() == 0).all()
    finally:
        lg().set_tuning(old)


def test_full_size_batching_configuration():
    """The batching configuration at full size, as the benchmark runs it: 20,000
    SPD matrices, n uniform over {4, 8, ..., 256}, FP32 storage, TF32x3 graph
    products, one call. Every matrix: info 0, L symmetric (log of an SPD
    matrix) and trace(L) = log det A; two matrices of every size against the
    oracle."""
    vals, ns, offs = workloads.ragged_spd(20000, seed=4)
    R = lg().Ragged(torch.tensor(vals, device="cuda"), torch.tensor(ns, device="cuda"),
                    torch.tensor(offs, device="cuda"), 256)
    L, s, k, info = lg().logm_execute(R, precision="tf32x3")
    out = L.values.cpu().numpy()
    assert (info.cpu().numpy() == 0).all()
    for n in SIZES:
        idx = np.nonzero(ns == n)[0]
        A = np.stack([vals[offs[b]:offs[b] + n * n].reshape(n, n) for b in idx]).astype(np.float64)
        Lg = np.stack([out[offs[b]:offs[b] + n * n].reshape(n, n) for b in idx]).astype(np.float64)
        nrm = np.linalg.norm(Lg, axis=(1, 2))
        assert (np.linalg.norm(Lg - Lg.transpose(0, 2, 1), axis=(1, 2)) <= 1e-5 * nrm).all(), n
        sign, logdet = np.linalg.slogdet(A)
        assert (sign > 0).all()
        tr = np.trace(Lg, axis1=1, axis2=2)
        assert (np.abs(tr - logdet) <= 1e-5 * (np.abs(logdet) + n * nrm / np.sqrt(n))).all(), n
        for j in np.random.default_rng(44 + n).choice(len(idx), 2, replace=False):
            Lr, d = oracle.logm(A[j])
            assert rel(Lg[j], Lr) <= SPLIT_TOL_F32, (n, int(idx[j]), rel(Lg[j], Lr))
