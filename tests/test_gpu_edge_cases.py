"""Edge cases through the C ABI: empty batches on every entry point (uniform
and ragged), and ragged batches with sizes a kernel must refuse (n < 1 or
n > n_max: LOGM_INFO_BAD_SIZE = -1 for that matrix, the others unaffected). The refusals are
the kernels' own size checks (every kernel reads n before touching a
matrix); no invalid memory is addressed."""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import SPLIT_TOL
from tests.test_gpu_parity import check_logm, dev, lg, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_empty_uniform_batch_every_entry_point(precision):
    A = torch.empty((0, 16, 16), dtype=torch.float64, device="cuda")
    L, s, k, info, ctx = lg().logm_execute(A, with_ctx=True, precision=precision)
    assert L.shape == (0, 16, 16) and s.numel() == k.numel() == info.numel() == 0
    fin, kk, alpha, info = lg().logm_plan(A)
    assert fin.numel() == 0 and info.numel() == 0
    X, A2, AI2, it, info = lg().logm_sqrt(A)
    assert X.shape == (0, 16, 16) and info.numel() == 0
    Z = lg().logm_graph_eval(A, 5, precision=precision)
    assert Z.shape == (0, 16, 16)
    if precision == "fp64":
        dA, binfo = lg().logm_backward(A, ctx, torch.empty_like(A))
        assert dA.shape == (0, 16, 16) and binfo.numel() == 0


def test_empty_ragged_batch():
    R = lg().Ragged(torch.empty(0, dtype=torch.float64, device="cuda"),
                    torch.empty(0, dtype=torch.int32, device="cuda"),
                    torch.empty(0, dtype=torch.int64, device="cuda"), 32)
    L, s, k, info = lg().logm_execute(R)
    assert L.values.numel() == 0 and info.numel() == 0


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_ragged_sizes_out_of_range_are_refused(precision):
    sizes = [5, 0, 40, 100, 64]  # n_max = 64: the 0 and the 100 are refused
    valid = [n for n in sizes if 1 <= n <= 64]
    mats = {n: workloads.identity_plus(1, n, seed=950 + n, lo=0.2, hi=2.0)[0] for n in valid}
    offs, flat, pos = [], [], 0
    for n in sizes:
        offs.append(pos)
        if n in mats:
            flat.append(mats[n].ravel())
            pos += n * n
    values = np.concatenate(flat)
    R = lg().Ragged(dev(values), torch.tensor(sizes, dtype=torch.int32, device="cuda"),
                    torch.tensor(offs, dtype=torch.int64, device="cuda"), 64)
    L, s, k, info = lg().logm_execute(R, precision=precision)
    info, out = info.cpu().numpy(), L.values.cpu().numpy()
    assert info.tolist() == [0, -1, 0, -1, 0]
    tol = 1e-12 if precision == "fp64" else SPLIT_TOL
    for b, n in enumerate(sizes):
        if n in mats:
            Lr, d = oracle.logm(mats[n])
            assert rel(out[offs[b]:offs[b] + n * n].reshape(n, n), Lr) <= tol, n


@pytest.mark.parametrize("dtype,pinned", [(torch.float64, True), (torch.float64, False), (torch.float32, True)])
def test_execute_host_matches_device_call(dtype, pinned):
    # logm_execute_host (copies inside the C-ABI call) against logm_execute on
    # device copies of the same matrices: identical results
    A = torch.from_numpy(workloads.identity_plus(20, 48, seed=960, lo=0.2, hi=3.0)).to(dtype)
    if pinned:
        A = A.pin_memory()
    Lh, sh, kh, ih = lg().logm_execute_host(A)
    Ld, sd, kd, idv = lg().logm_execute(A.cuda())
    assert not Lh.is_cuda and torch.equal(Lh, Ld.cpu())
    assert torch.equal(sh, sd.cpu()) and torch.equal(kh, kd.cpu()) and torch.equal(ih, idv.cpu())
    L1, _, _, _ = lg().logm_execute_host(A[3].contiguous())  # a single (n, n) matrix
    assert torch.equal(L1, Ld[3].cpu())
