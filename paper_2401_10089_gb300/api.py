"""Python binding of the C ABI: same names as ``include/logm.h``.

These functions only marshal arguments. Matrices are CUDA tensors owned by
PyTorch (its caching allocator provides device memory and workspace, its
current stream orders the work); every step of the method runs in the CUDA
library. A batch is either a (count, n, n) tensor or a :class:`Ragged`
(packed values, device sizes, device element offsets).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib

_PREC = {"fp64": _lib.PREC_FP64, "tf32x3": _lib.PREC_TF32X3, "bf16x3": _lib.PREC_BF16X3}


@dataclass
class Ragged:
    """Packed ragged batch: matrix b is values[offset[b] : offset[b] + n[b]**2] (row-major)."""
    values: torch.Tensor   # 1-D float64/float32 CUDA tensor
    n: torch.Tensor        # int32 CUDA tensor [count]
    offset: torch.Tensor   # int64 CUDA tensor [count]
    n_max: int

    @property
    def count(self) -> int:
        return int(self.n.numel())

    @property
    def device(self):
        return self.values.device

    @property
    def dtype(self):
        return self.values.dtype

    def empty_like(self):
        return Ragged(torch.empty_like(self.values), self.n, self.offset, self.n_max)


def _dtype_code(t: torch.dtype) -> int:
    if t == torch.float64:
        return _lib.DTYPE_F64
    if t == torch.float32:
        return _lib.DTYPE_F32
    raise TypeError(f"unsupported dtype {t}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _batch(A) -> _lib.LogmBatch:
    b = _lib.LogmBatch()
    if isinstance(A, Ragged):
        if not A.values.is_cuda:
            raise ValueError("Ragged.values must be a CUDA tensor")
        b.count, b.dtype, b.n_uniform, b.n_max = A.count, _dtype_code(A.values.dtype), 0, A.n_max
        b.n, b.offset = A.n.data_ptr(), A.offset.data_ptr()
        return b
    if A.dim() == 2:
        A = A.unsqueeze(0)
    if A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("expected a (count, n, n) or (n, n) tensor")
    if not A.is_cuda or not A.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    b.count, b.dtype, b.n_uniform, b.n_max = A.shape[0], _dtype_code(A.dtype), A.shape[1], A.shape[1]
    b.n = b.offset = None
    return b


def _values(A):
    return A.values if isinstance(A, Ragged) else A


_DB_FORM = {"two_inverse": 0, "product": 1}
_FP64_PRODUCTS = {"pipe": 0, "tc_sliced": 1}


def _options(k_max=5, precision="fp64", max_sqrt=40, max_db_iter=50, theta=None, db_form="two_inverse",
             balance=False, fp64_products="pipe") -> _lib.LogmOptions:
    """k_max in 1..6 (6: FP64 products, n <= 256, no adjoint); db_form
    "two_inverse" (eq. ScalDB) or "product";
    balance: diagonal balancing of Algorithm 1, Step 1; theta: Theta_{m_k} for
    k = 1..5 (0 = the paper's Table Table_theta); fp64_products: "pipe" (FP64
    FMAs) or "tc_sliced" (the whole-GPU kernel's inversion updates from exact
    BF16 digit products on the tensor cores)."""
    o = _lib.LogmOptions()
    o.k_max, o.max_sqrt, o.max_db_iter = k_max, max_sqrt, max_db_iter
    o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    o.db_form = _DB_FORM[db_form] if isinstance(db_form, str) else int(db_form)
    o.balance = 1 if balance else 0
    o.fp64_products = _FP64_PRODUCTS[fp64_products] if isinstance(fp64_products, str) else int(fp64_products)
    th = (0.0,) * 5 if theta is None else theta
    for t in range(5):
        o.theta[t] = th[t]
    return o


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class _Workspace:
    """Per-device cache of the largest workspace requested so far."""

    def __init__(self):
        self.buf = {}

    def get(self, device, nbytes: int) -> torch.Tensor:
        key = torch.device(device).index
        cur = self.buf.get(key)
        if cur is None or cur.numel() < nbytes:
            cur = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
            self.buf[key] = cur
        return cur


_ws = _Workspace()
_ws_host = _Workspace()


def logm_workspace_size(A, **opts) -> int:
    """Device workspace bytes of logm_plan / logm_sqrt / logm_graph_eval / logm_execute for batch A."""
    L = _lib.load()
    b, o = _batch(A), _options(**opts)
    return int(L.logm_workspace_size(ctypes.byref(b), ctypes.byref(o)))


def logm_context_size(A, **opts) -> int:
    """Bytes of the context logm_execute(with_ctx=True) saves for the backward: (s, k), the balancing
    diagonal and every square-root level's input per matrix."""
    L = _lib.load()
    b, o = _batch(A), _options(**opts)
    return int(L.logm_context_size(ctypes.byref(b), ctypes.byref(o)))


def _workspace(A, b, o, L):
    nbytes = int(L.logm_workspace_size(ctypes.byref(b), ctypes.byref(o)))
    if nbytes == 0:
        raise _lib.LogmError("unsupported batch (workspace size 0)")
    w = _ws.get(_values(A).device, nbytes)
    return w, nbytes


def _i32(count, device):
    return torch.empty(count, dtype=torch.int32, device=device)


def logm_plan(A, AI2=None, **opts):
    """(finish, k, alpha, info) of one pass of Algorithm 1's loop test and the order search."""
    L = _lib.load()
    b, o = _batch(A), _options(**opts)
    dev = _values(A).device
    fin, k, info = _i32(b.count, dev), _i32(b.count, dev), _i32(b.count, dev)
    alpha = torch.empty(b.count, dtype=torch.float64, device=dev)
    w, nb = _workspace(A, b, o, L)
    rc = L.logm_plan(ctypes.byref(b), ctypes.byref(o), _ptr(_values(A)),
                     _ptr(None if AI2 is None else _values(AI2)), _ptr(fin), _ptr(k), _ptr(alpha),
                     _ptr(info), _ptr(w), nb, _stream(dev))
    _lib.check(rc, "logm_plan")
    return fin, k, alpha, info


def logm_sqrt(A, active=None, **opts):
    """One square root in place: returns (A, A2, AI2, iters, info)."""
    L = _lib.load()
    b, o = _batch(A), _options(**opts)
    v = _values(A)
    dev = v.device
    A2 = torch.empty_like(v)
    AI2 = torch.empty_like(v)
    it, info = _i32(b.count, dev), _i32(b.count, dev)
    w, nb = _workspace(A, b, o, L)
    rc = L.logm_sqrt(ctypes.byref(b), ctypes.byref(o), _ptr(v), _ptr(A2), _ptr(AI2), _ptr(active), _ptr(it),
                     _ptr(info), _ptr(w), nb, _stream(dev))
    _lib.check(rc, "logm_sqrt")
    return A, A2, AI2, it, info


def logm_graph_eval(X, k, P3=None, precision="fp64"):
    """Z = z(X) with k graph products per matrix (k: int or int32 CUDA tensor)."""
    L = _lib.load()
    b = _batch(X)
    v = _values(X)
    dev = v.device
    if not torch.is_tensor(k):
        k = torch.full((b.count,), int(k), dtype=torch.int32, device=dev)
    Z = torch.empty_like(v)
    prec = _PREC[precision] if isinstance(precision, str) else int(precision)
    o = _options(precision=prec)
    w, nb = _workspace(X, b, o, L)
    rc = L.logm_graph_eval(ctypes.byref(b), prec, _ptr(v), _ptr(None if P3 is None else _values(P3)),
                           _ptr(k), _ptr(Z), _ptr(w), nb, _stream(dev))
    _lib.check(rc, "logm_graph_eval")
    return Z


def logm_execute(A, with_ctx=False, stats=None, **opts):
    """L = log(A) by Algorithm 1: returns (L, s, k, info[, ctx]).

    ``stats``: optional int32 CUDA tensor of 4 * count entries that receives,
    per matrix, the Denman-Beavers iterations, inverses, graph products and
    estimator matrix-vector products the plan executed."""
    L = _lib.load()
    b, o = _batch(A), _options(**opts)
    v = _values(A)
    dev = v.device
    out = torch.empty_like(v)
    s, k, info = _i32(b.count, dev), _i32(b.count, dev), _i32(b.count, dev)
    ctx = None
    if with_ctx:
        ctx = torch.empty(int(L.logm_context_size(ctypes.byref(b), ctypes.byref(o))), dtype=torch.uint8,
                          device=dev)
    w, nb = _workspace(A, b, o, L)
    rc = L.logm_execute(ctypes.byref(b), ctypes.byref(o), _ptr(v), _ptr(out), _ptr(s), _ptr(k), _ptr(info),
                        _ptr(stats), _ptr(ctx), _ptr(w), nb, _stream(dev))
    _lib.check(rc, "logm_execute")
    Lout = out if not isinstance(A, Ragged) else Ragged(out, A.n, A.offset, A.n_max)
    if with_ctx:
        return Lout, s, k, info, ctx
    return Lout, s, k, info


def _host_batch(A):
    if A.is_cuda:
        raise ValueError("logm_execute_host takes host (CPU) tensors")
    A3 = A.unsqueeze(0) if A.dim() == 2 else A
    if A3.dim() != 3 or A3.shape[1] != A3.shape[2] or not A3.is_contiguous():
        raise ValueError("expected a contiguous (count, n, n) or (n, n) CPU tensor")
    b = _lib.LogmBatch()
    b.count, b.dtype, b.n_uniform, b.n_max = A3.shape[0], _dtype_code(A3.dtype), A3.shape[1], A3.shape[1]
    b.n = b.offset = None
    return A3, b


def logm_host_workspace_size(A, **opts) -> int:
    """Device bytes ``logm_execute_host`` needs for the host tensor A."""
    L = _lib.load()
    _, b = _host_batch(A)
    return int(L.logm_host_workspace_size(ctypes.byref(b), ctypes.byref(_options(**opts))))


def logm_execute_host(A, out=None, device=None, workspace=None, **opts):
    """L = log(A) for host matrices through ``logm_execute_host`` (the copies to
    and from the device happen inside the call): A is a (count, n, n) or
    (n, n) CPU tensor (page-locked for asynchronous copies), ``out`` an
    optional CPU tensor of the same shape for L, ``workspace`` an optional
    uint8 CUDA tensor of at least ``logm_host_workspace_size(A)`` bytes.
    Returns (L, s, k, info) as CPU tensors once the stream has finished."""
    L = _lib.load()
    A3, b = _host_batch(A)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    o = _options(**opts)
    nb = int(L.logm_host_workspace_size(ctypes.byref(b), ctypes.byref(o)))
    if nb == 0:
        raise _lib.LogmError("logm_execute_host: unsupported batch")
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nb:
            raise ValueError("workspace too small")
        w, nb = workspace, workspace.numel() * workspace.element_size()
    else:
        w = _ws_host.get(dev, nb)
    pin = A3.is_pinned()
    Lout = out if out is not None else torch.empty(A3.shape, dtype=A3.dtype, pin_memory=pin)
    s = torch.empty(b.count, dtype=torch.int32, pin_memory=pin)
    k = torch.empty_like(s)
    info = torch.empty_like(s)
    stream = torch.cuda.current_stream(dev)
    rc = L.logm_execute_host(ctypes.byref(b), ctypes.byref(o), _ptr(A3), _ptr(Lout), _ptr(s), _ptr(k), _ptr(info),
                             _ptr(w), nb, ctypes.c_void_p(stream.cuda_stream))
    _lib.check(rc, "logm_execute_host")
    stream.synchronize()
    if A.dim() == 2 and out is None:
        Lout = Lout[0]
    return Lout, s, k, info


def logm_backward_workspace_size(A, **opts) -> int:
    """Device workspace bytes of logm_backward for batch A (0: unsupported, n_max > 256)."""
    L = _lib.load()
    b, o = _batch(A), _options(**opts)
    return int(L.logm_backward_workspace_size(ctypes.byref(b), ctypes.byref(o)))


_ws_bwd = _Workspace()


def logm_backward(A, ctx, dL, **opts):
    """dA = gradient of sum(dL * log(A)) with respect to A at the forward's plan.

    ``ctx`` is the context tensor ``logm_execute(A, with_ctx=True)`` returned."""
    L = _lib.load()
    b, o = _batch(A), _options(**opts)
    v = _values(A)
    dev = v.device
    dA = torch.empty_like(v)
    info = _i32(b.count, dev)
    nb = int(L.logm_backward_workspace_size(ctypes.byref(b), ctypes.byref(o)))
    if nb == 0:
        raise _lib.LogmError("logm_backward: unsupported batch (n_max > 256?)")
    w = _ws_bwd.get(dev, nb)
    rc = L.logm_backward(ctypes.byref(b), ctypes.byref(o), _ptr(v), _ptr(ctx), _ptr(_values(dL)), _ptr(dA),
                         _ptr(info), _ptr(w), nb, _stream(dev))
    _lib.check(rc, "logm_backward")
    return dA, info


def logm_version() -> int:
    return int(_lib.load().logm_version())


class LogmFunction(torch.autograd.Function):
    """L = log(A) with the hand-written adjoint (logm_backward) as its backward."""

    @staticmethod
    def forward(ctx, A, k_max=5, max_sqrt=40, max_db_iter=50, db_form="two_inverse", balance=False):
        opts = dict(k_max=k_max, max_sqrt=max_sqrt, max_db_iter=max_db_iter, db_form=db_form, balance=balance)
        Ac = A.contiguous()
        L, s, k, info, cbuf = logm_execute(Ac, with_ctx=True, **opts)
        ctx.save_for_backward(Ac, cbuf)
        ctx.opts = opts
        ctx.mark_non_differentiable(s, k, info)
        return L, s, k, info

    @staticmethod
    def backward(ctx, dL, ds, dk, dinfo):
        A, cbuf = ctx.saved_tensors
        dA, info = logm_backward(A, cbuf, dL.contiguous(), **ctx.opts)
        return dA, None, None, None, None, None


def logm(A, k_max=5, max_sqrt=40, max_db_iter=50, db_form="two_inverse", balance=False):
    """Differentiable matrix logarithm of a (count, n, n) or (n, n) CUDA tensor."""
    L, s, k, info = LogmFunction.apply(A, k_max, max_sqrt, max_db_iter, db_form, balance)
    return L


def set_tuning(variants):
    """Per-size-bucket kernel configuration (buckets n <= 8, 16, 32, 64, 128, 256;
    0: 256-thread blocks, 1: 128-thread blocks for n <= 64, 2: 64-thread blocks
    for n <= 32, 3: 256-thread blocks three per SM). ``None`` restores all-0."""
    L = _lib.load()
    if variants is None:
        _lib.check(L.logm_set_tuning(None), "logm_set_tuning")
        return
    t = _lib.LogmTuning()
    for i, v in enumerate(variants):
        t.variant[i] = int(v)
    _lib.check(L.logm_set_tuning(ctypes.byref(t)), "logm_set_tuning")


def get_tuning():
    L = _lib.load()
    t = _lib.LogmTuning()
    _lib.check(L.logm_get_tuning(ctypes.byref(t)), "logm_get_tuning")
    return [int(t.variant[i]) for i in range(6)]
