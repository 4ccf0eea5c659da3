"""Plain FP64 CPU oracle for the matrix logarithm of arXiv 2401.10089.

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` leg are the only callers allowed. The CUDA
library and its Python binding never import this package, and this package
never imports them: the two implementations share no code.

The arithmetic lives in ``logm_oracle.c`` (plain C, built here with gcc);
this module only marshals numpy arrays. Each function cites the part of the
paper it follows:

* ``graph_eval``   -- degree-optimal form, eq. (five_mult_degopt), Sec. 3, with
                      Table table_simple_experiment for k = 5, the exact
                      Taylor polynomials of eq. (Taylor_log) for k = 1, 2,
                      T_8 by eq. (eqP8pol) for k = 3 (``coeffs_k3``) and the
                      14+ scheme for k = 4 (``coeffs_k4``, solved here; the
                      paper does not print it) and a 20+ scheme for k = 6
                      (``coeffs_k6``, fitted by ``derive_k6.py``; opt-in).
* ``sqrtm_db``     -- scaled Denman-Beavers iteration, eq. (ScalDB), Sec. 6, or
                      its product form (``form=1``, the variant cited in Sec. 2);
                      ``logm`` runs eq. (ScalDB) as written at every level unless
                      ``reuse_root=1`` (later levels start from the previous Y).
* ``balance``      -- the diagonal balancing T of Algorithm 1, Step 1.
* ``normest_pow``  -- 1-norm power estimate (Higham 1988, cited in Sec. 6),
                      with A_I2 of eq. (AI2) for even powers.
* ``plan``         -- one pass of Algorithm 1's loop test (eqs. alphaapprox,
                      normAm9, alpha2term1, normAm9plus1) and the order search
                      (eqs. min_in, min_inp, roughmax_even).
* ``logm``         -- Algorithm 1 (T = I unless ``balance=1``).
* ``expm_taylor``, ``frechet_adjoint``, ``horner`` -- independent checks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "logm_oracle.c")
_HDR = os.path.join(_HERE, "logm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblogm_oracle.so")
_lock = threading.Lock()
_lib = None

# Theta_{m_k} of Table Table_theta (Sec. 5) for k = 1..6.
THETA_TABLE = (1.83e-8, 1.53e-4, 1.33e-2, 9.31e-2, 2.46e-1, 3.72e-1)
# Orders with coefficients: T_2, T_4 (eq. Taylor_log), T_8 (eq. eqP8pol), the
# 14+ scheme (k = 4, solved here), Table table_simple_experiment and the
# 20+ scheme (k = 6, fitted here; opt-in, the default k_max stays 5).
AVAILABLE_K = (1, 2, 3, 4, 5, 6)
M_OF_K = {1: 2, 2: 4, 3: 8, 4: 14, 5: 14, 6: 20}
# Status codes, written out on their own (same meanings as the library's).
OK, SINGULAR, NO_CONVERGENCE, MAX_SQRT, NONFINITE = 0, 1, 2, 3, 4


class Opts(ctypes.Structure):
    _fields_ = [
        ("k_max", ctypes.c_int32),
        ("max_sqrt", ctypes.c_int32),
        ("max_db_iter", ctypes.c_int32),
        ("force_s", ctypes.c_int32),
        ("force_k", ctypes.c_int32),
        ("db_form", ctypes.c_int32),
        ("balance", ctypes.c_int32),
        ("reuse_root", ctypes.c_int32),
        ("theta", ctypes.c_double * 6),
    ]


class Diag(ctypes.Structure):
    _fields_ = [
        ("s", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("info", ctypes.c_int32),
        ("db_iters", ctypes.c_int32),
        ("n_estimates", ctypes.c_int32),
        ("n_inv", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("norm_b", ctypes.c_double),
        ("norm_ai2", ctypes.c_double),
        ("margin", ctypes.c_double),
        ("margin_s", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


def build(force: bool = False) -> str:
    """Compile ``logm_oracle.c`` into ``_build/liblogm_oracle.so`` (gcc, -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            L.orc_norm1.restype = d
            L.orc_norm1.argtypes = [i, p]
            L.orc_normest_pow.restype = d
            L.orc_normest_pow.argtypes = [i, p, p, i]
            L.orc_gemm.argtypes = [i, p, p, p]
            L.orc_lu.argtypes = [i, p, p]
            L.orc_inverse.argtypes = [i, p, p, p]
            L.orc_sqrtm_db.argtypes = [i, p, p, i, p]
            L.orc_sqrtm_db_product.argtypes = [i, p, p, i, p]
            L.orc_sqrtm_db_reuse.argtypes = [i, p, p, i, p, p, d]
            L.orc_balance.argtypes = [i, p, p]
            L.orc_coeffs_k3.argtypes = [p]
            L.orc_coeffs_k4.argtypes = [p]
            L.orc_graph_eval.argtypes = [i, i, p, p, p]
            L.orc_horner.argtypes = [i, i, p, p, p]
            L.orc_plan.argtypes = [i, p, p, p, p, p, p]
            L.orc_logm.argtypes = [i, p, p, p, p]
            L.orc_logm_batch.argtypes = [i, p, p, p, p, p, p, i]
            L.orc_expm_taylor.argtypes = [i, p, p]
            L.orc_frechet_adjoint.argtypes = [i, p, p, p, p]
            L.orc_coeffs_k5.argtypes = [p, p, p]
            L.orc_coeffs_k6.argtypes = [p, p, p]
            _lib = L
    return _lib


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_opts(k_max=5, max_sqrt=40, max_db_iter=50, force_s=-1, force_k=0, theta=None,
              db_form=0, balance=0, reuse_root=0) -> Opts:
    """Options of Algorithm 1. ``reuse_root=0`` (default) runs eq. (ScalDB)
    as written at every square-root level; ``reuse_root=1`` starts later
    levels from the previous level's Y as A^{-1} (one inversion fewer per
    level, the same iterates in exact arithmetic)."""
    o = Opts()
    o.k_max, o.max_sqrt, o.max_db_iter = k_max, max_sqrt, max_db_iter
    o.force_s, o.force_k = force_s, force_k
    o.db_form, o.balance, o.reuse_root = db_form, balance, reuse_root
    th = THETA_TABLE if theta is None else theta
    for t in range(6):
        o.theta[t] = th[t] if t < len(th) else THETA_TABLE[t]
    return o


def coeffs_k3():
    """c3, c4, d1, d2, e2, e0 of eq. (eqP8pol) for T_8 (closed form)."""
    c = np.zeros(6)
    lib().orc_coeffs_k3(_ptr(c))
    return c


def coeffs_k4():
    """c3, c4, d1, d2, e2, f1, f2, f4, g1, g4, y3, y4, y5 of the k = 4 (14+)
    scheme: P_4 = P_3 (c3 X + c4 P_3), P_5 = (d1 X + d2 P_3 + P_4)(e2 P_3 +
    P_4), P_6 = (f1 X + f2 P_3 + f4 P_4 + P_5)(g1 X + g4 P_4 + P_5),
    z = X + y3 P_3 + y4 P_4 + y5 P_5 + P_6."""
    c = np.zeros(13)
    lib().orc_coeffs_k4(_ptr(c))
    return c


def balance(A):
    """(T^{-1} A T, diag(T)) by the radix-2 Parlett-Reinsch balancing."""
    B = _c(A).copy()
    d = np.empty(B.shape[0])
    lib().orc_balance(B.shape[0], _ptr(B), _ptr(d))
    return B, d


def coeffs_k5():
    h = np.zeros(14)
    g = np.zeros(14)
    y = np.zeros(7)
    lib().orc_coeffs_k5(_ptr(h), _ptr(g), _ptr(y))
    return h, g, y


def coeffs_k6():
    """h (20), g (20), y (8) of the k = 6 scheme in the order h_{2,2..3},
    h_{3,2..4}, ..., h_{6,2..7}; y = y_1..y_8 (y_1 = 0, y_2 = 1)."""
    h = np.zeros(20)
    g = np.zeros(20)
    y = np.zeros(8)
    lib().orc_coeffs_k6(_ptr(h), _ptr(g), _ptr(y))
    return h, g, y


def gemm(A, B):
    A, B = _c(A), _c(B)
    C = np.empty_like(A)
    lib().orc_gemm(A.shape[0], _ptr(A), _ptr(B), _ptr(C))
    return C


def norm1(A):
    A = _c(A)
    return lib().orc_norm1(A.shape[0], _ptr(A))


def inverse(A):
    """(A^{-1}, log|det A|, status) by LU with partial pivoting."""
    A = _c(A)
    Ai = np.empty_like(A)
    ld = ctypes.c_double()
    st = lib().orc_inverse(A.shape[0], _ptr(A), _ptr(Ai), ctypes.byref(ld))
    return Ai, ld.value, st


def sqrtm_db(A, max_iter=50, form=0):
    """(A^{1/2}, iterations, status) by eq. (ScalDB) (form 0) or its product
    form (form 1)."""
    A = _c(A)
    X = np.empty_like(A)
    it = ctypes.c_int32()
    f = lib().orc_sqrtm_db_product if form == 1 else lib().orc_sqrtm_db
    st = f(A.shape[0], _ptr(A), _ptr(X), max_iter, ctypes.byref(it))
    return X, it.value, st


def sqrtm_db_reuse(A, Ainv, logabsdet, max_iter=50):
    """(A^{1/2}, iterations, status) by eq. (ScalDB) with A^{-1} and log|det A|
    given for the first step (as Algorithm 1's later roots have them)."""
    A, Ainv = _c(A), _c(Ainv)
    X = np.empty_like(A)
    it = ctypes.c_int32()
    st = lib().orc_sqrtm_db_reuse(A.shape[0], _ptr(A), _ptr(X), max_iter, ctypes.byref(it), _ptr(Ainv),
                                   float(logabsdet))
    return X, it.value, st


def normest_pow(B, p, AI2=None):
    B = _c(B)
    AI2 = None if AI2 is None else _c(AI2)
    return lib().orc_normest_pow(B.shape[0], _ptr(B), _ptr(AI2), p)


def graph_eval(X, k, P3=None):
    X = _c(X)
    P3 = None if P3 is None else _c(P3)
    Z = np.empty_like(X)
    r = lib().orc_graph_eval(X.shape[0], k, _ptr(X), _ptr(P3), _ptr(Z))
    if r != 0:
        raise ValueError(f"unsupported k={k}")
    return Z


def horner(X, b):
    X = _c(X)
    b = _c(b)
    Z = np.empty_like(X)
    lib().orc_horner(X.shape[0], len(b) - 1, _ptr(b), _ptr(X), _ptr(Z))
    return Z


def plan(A, AI2=None, **kw):
    """(finish, k, alpha) of one loop test of Algorithm 1 and the order search."""
    A = _c(A)
    AI2 = None if AI2 is None else _c(AI2)
    fin, k, al = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    o = make_opts(**kw)
    lib().orc_plan(A.shape[0], _ptr(A), _ptr(AI2), ctypes.byref(o), ctypes.byref(fin),
                   ctypes.byref(k), ctypes.byref(al))
    return bool(fin.value), k.value, al.value


def logm(A, **kw):
    """(L, diag dict) by Algorithm 1. The diag's ``margin`` is the smallest
    relative distance of a plan quantity from the threshold it was compared
    with, ``margin_s`` the square-root level of that comparison."""
    A = _c(A)
    L = np.empty_like(A)
    o = make_opts(**kw)
    d = Diag()
    lib().orc_logm(A.shape[0], _ptr(A), _ptr(L), ctypes.byref(o), ctypes.byref(d))
    return L, d.as_dict()


def logm_batch(mats, nthreads=0, **kw):
    """Algorithm 1 on a list of square matrices (one OpenMP thread per matrix)."""
    ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    offs = np.zeros(len(mats), dtype=np.int64)
    if len(mats) > 1:
        offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    flat = np.concatenate([_c(m).ravel() for m in mats]) if mats else np.zeros(0)
    out = np.empty_like(flat)
    o = make_opts(**kw)
    diags = (Diag * max(1, len(mats)))()
    lib().orc_logm_batch(len(mats), _ptr(ns), _ptr(offs), _ptr(flat), _ptr(out), ctypes.byref(o),
                         ctypes.cast(diags, ctypes.c_void_p), nthreads)
    Ls = [out[o_:o_ + n * n].reshape(n, n) for o_, n in zip(offs, ns)]
    return Ls, [diags[b].as_dict() for b in range(len(mats))]


def expm_taylor(A):
    A = _c(A)
    E = np.empty_like(A)
    lib().orc_expm_taylor(A.shape[0], _ptr(A), _ptr(E))
    return E


def frechet_adjoint(A, W, **kw):
    """L(A^T, W): gradient of sum(W * log(A)) with respect to A."""
    A, W = _c(A), _c(W)
    G = np.empty_like(A)
    o = make_opts(**kw)
    st = lib().orc_frechet_adjoint(A.shape[0], _ptr(A), _ptr(W), _ptr(G), ctypes.byref(o))
    return G, st
