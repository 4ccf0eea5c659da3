"""Failure detection without a GPU fault: the grid barrier of the whole-GPU
kernel (the library's only spin-wait) gives up after its time limit and
reports a status instead of hanging. logm_probe_barrier runs that barrier on
two co-resident blocks expecting arrivals that never come; the test checks
the status, that the wait ended within a bound, and that the context still
runs the method afterwards."""
import ctypes
import time

import numpy as np
import pytest

from paper_2401_10089_gb300 import _lib, workloads
from tests.test_gpu_parity import check_logm, dev, lg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def probe(missing, timeout_s):
    L = _lib.load()
    ws = torch.zeros(4, dtype=torch.int32, device="cuda")  # counter (8 B) + status
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = L.logm_probe_barrier(missing, ctypes.c_double(timeout_s), ctypes.c_void_p(ws.data_ptr()), 16, stream)
    torch.cuda.synchronize()
    return rc, int(ws[2].item()), time.perf_counter() - t0


def test_barrier_wait_runs_out_and_reports():
    rc, status, dt = probe(1, 0.005)
    assert rc == _lib.SUCCESS and status == 1
    assert 0.005 <= dt < 2.0
    rc, status, dt = probe(0, 0.005)  # everyone arrives: no timeout
    assert rc == _lib.SUCCESS and status == 0


def test_barrier_probe_argument_checks():
    L = _lib.load()
    assert L.logm_probe_barrier(-1, ctypes.c_double(0.01), None, 0, None) == _lib.ERR_INVALID_ARG
    assert L.logm_probe_barrier(1, ctypes.c_double(0.0), None, 0, None) == _lib.ERR_INVALID_ARG
    assert L.logm_probe_barrier(1, ctypes.c_double(0.01), None, 16, None) == _lib.ERR_WORKSPACE


def test_context_usable_after_timeout():
    probe(2, 0.002)
    A = workloads.identity_plus(1, 300, seed=900)
    L, s, k, info = lg().logm_execute(dev(A))
    check_logm(A[0], L[0].cpu().numpy(), int(s[0]), int(k[0]), int(info[0]))
