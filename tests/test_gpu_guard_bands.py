"""Out-of-bounds writes without compute-sanitizer: every buffer a call writes
(L, s, k, info, the workspace, the context, dA) sits between guard bands of a
known bit pattern, and the bands must be intact after the call. The L payload
is pre-filled with the same pattern and must be fully overwritten. Covers the
one-block and whole-GPU kernels, uniform and ragged batches, split precision
(packed and in-place product kernels), the whole-GPU kernel with its
tensor-core updates and the adjoint."""
import ctypes

import numpy as np
import pytest

from paper_2401_10089_gb300 import _lib, api, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes on each side
CANARY = 0x5A


class Banded:
    """A device byte buffer of `nbytes` between two guard bands."""

    def __init__(self, nbytes, fill_payload=True):
        self.nbytes = int(nbytes)
        self.raw = torch.full((GUARD + max(self.nbytes, 1) + GUARD,), CANARY, dtype=torch.uint8, device="cuda")
        if not fill_payload:
            self.raw[GUARD:GUARD + self.nbytes].zero_()

    def ptr(self):
        return ctypes.c_void_p(self.raw.data_ptr() + GUARD)

    def guards_intact(self):
        return bool((self.raw[:GUARD] == CANARY).all()) and bool((self.raw[GUARD + self.nbytes:] == CANARY).all())

    def payload(self):
        return self.raw[GUARD:GUARD + self.nbytes]


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def run_execute(A, precision="fp64", with_ctx=False, fp64_products="pipe"):
    L = _lib.load()
    b, o = api._batch(A), api._options(precision=precision, fp64_products=fp64_products)
    v = api._values(A)
    esz = v.element_size()
    out = Banded(v.numel() * esz)
    s, k, info = Banded(4 * b.count), Banded(4 * b.count), Banded(4 * b.count)
    ws = Banded(L.logm_workspace_size(ctypes.byref(b), ctypes.byref(o)), fill_payload=False)
    ctx = Banded(L.logm_context_size(ctypes.byref(b), ctypes.byref(o)), fill_payload=False) if with_ctx else None
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), ctypes.c_void_p(v.data_ptr()), out.ptr(), s.ptr(),
                        k.ptr(), info.ptr(), None, ctx.ptr() if ctx else None, ws.ptr(), ws.nbytes, _stream())
    torch.cuda.synchronize()
    assert rc == _lib.SUCCESS
    return out, s, k, info, ws, ctx


def check(bufs):
    for name, buf in bufs.items():
        if buf is not None:
            assert buf.guards_intact(), name


def ragged(sizes, seed):
    # ||E||_1 <= 0.9: every eigenvalue of I + E has a positive real part
    mats = [workloads.identity_plus(1, n, seed=seed + n, lo=0.1, hi=0.9)[0] for n in sizes]
    ns = np.array(sizes, dtype=np.int32)
    offs = np.zeros(len(sizes), dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    vals = torch.tensor(np.concatenate([m.ravel() for m in mats]), device="cuda")
    return api.Ragged(vals, torch.tensor(ns, device="cuda"), torch.tensor(offs, device="cuda"), max(sizes))


@pytest.mark.parametrize("case", ["uniform48", "uniform300", "ragged_mixed", "uniform64_tf32", "ragged_tf32",
                                  "uniform300_tc", "ragged_mixed_tc"])
def test_guard_bands_intact(case):
    precision = "tf32x3" if case.endswith("tf32") else "fp64"
    fp64_products = "tc_sliced" if case.endswith("_tc") else "pipe"
    case = case[:-3] if case.endswith("_tc") else case
    if case == "uniform48":
        A = torch.tensor(workloads.identity_plus(5, 48, seed=970, lo=0.1, hi=0.9), device="cuda")
    elif case == "uniform300":
        A = torch.tensor(workloads.identity_plus(1, 300, seed=971, lo=0.1, hi=0.9), device="cuda")
    elif case == "uniform64_tf32":
        A = torch.tensor(workloads.identity_plus(6, 64, seed=972, lo=0.1, hi=0.9), device="cuda")
    else:
        A = ragged([33, 300, 7] if case == "ragged_mixed" else [33, 64, 17], seed=973)
    out, s, k, info, ws, ctx = run_execute(A, precision=precision, fp64_products=fp64_products)
    check({"L": out, "s": s, "k": k, "info": info, "workspace": ws})
    assert not bool((out.payload() == CANARY).all())
    assert (info.payload().view(torch.int32) == 0).all()
    # every element of L written: no 8-byte (or 4-byte) word of the payload left at the canary
    w = out.payload().view(torch.int64 if api._values(A).element_size() == 8 else torch.int32)
    pattern = int.from_bytes(bytes([CANARY]) * w.element_size(), "little", signed=True)
    assert not bool((w == pattern).any())


def test_guard_bands_backward():
    L = _lib.load()
    A = torch.tensor(workloads.spd(3, 40, seed=974, lo=0.1, hi=10.0), device="cuda")
    W = torch.tensor(np.random.default_rng(975).standard_normal((3, 40, 40)), device="cuda")
    out, s, k, info, ws, ctx = run_execute(A, with_ctx=True)
    check({"L": out, "ctx": ctx, "workspace": ws})
    b, o = api._batch(A), api._options()
    dA = Banded(A.numel() * 8)
    binfo = Banded(4 * b.count)
    bws = Banded(L.logm_backward_workspace_size(ctypes.byref(b), ctypes.byref(o)), fill_payload=False)
    rc = L.logm_backward(ctypes.byref(b), ctypes.byref(o), ctypes.c_void_p(A.data_ptr()), ctx.ptr(),
                         ctypes.c_void_p(W.data_ptr()), dA.ptr(), binfo.ptr(), bws.ptr(), bws.nbytes, _stream())
    torch.cuda.synchronize()
    assert rc == _lib.SUCCESS
    check({"dA": dA, "binfo": binfo, "bwd workspace": bws, "ctx after backward": ctx})
    assert (binfo.payload().view(torch.int32) == 0).all()
