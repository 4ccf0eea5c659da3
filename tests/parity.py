"""The parity rule for one GPU result against the oracle (CPU-only helper).

Plan decisions (s, k) are integers decided in FP64 on both sides from nearly
equal quantities. The oracle reports the smallest relative distance between a
plan quantity and the threshold it was compared with (``margin``) and the
square-root level of that comparison (``margin_s``). A GPU plan that differs
from the oracle's is accepted only when that comparison lies within
``NEAR_THRESHOLD`` of its threshold at the level where the two runs part
(min of the two s); the GPU result is then compared with the oracle run at
the GPU's (s, k). Otherwise the plans must be identical.
"""
import numpy as np

import oracle

TOL = 1e-12
NEAR_THRESHOLD = 1e-10

# Split-precision graph products (TF32x3, BF16x3) against the FP64 oracle.
# Each FP32 operand is split into slices whose dropped cross terms leave
# about 2^-22 relative (TF32x3: hi + lo of 11 bits each; BF16x3: the terms
# s_a s_b with a + b > 2 of three 8-bit slices); X, P_3 and every lin-comb
# node are rounded to FP32 (2^-24 each). The products P_4.. of the graph
# have norms below Theta_k ||X|| (||X|| <= Theta_k < 1/4), so their
# accumulation errors enter z = sum y_i P_i scaled down by that factor, and
# L = -2^s z keeps z's relative error. About four such 2^-22 contributions
# bound the result: 4 * 2^-22 = 9.5e-7.
SPLIT_TOL = 4 * 2.0 ** -22
# The same with FP32 storage of L (one more rounding).
SPLIT_TOL_F32 = SPLIT_TOL + 2.0 ** -24


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_at_plan(A, s, k, info, **kw):
    """The oracle's L for A at the GPU's plan (s, k): the oracle's own run
    when the plans agree, else (only if a plan comparison was within
    ``NEAR_THRESHOLD`` of its threshold where the runs part) the oracle
    forced to (s, k). Asserts info 0 on both sides."""
    Lr, d = oracle.logm(A, **kw)
    assert info == d["info"] == 0, (info, d)
    if (s, k) == (d["s"], d["k"]):
        return Lr
    near = d["margin"] <= NEAR_THRESHOLD and d["margin_s"] == min(s, d["s"])
    assert near, ("plan differs away from every threshold", (s, k), (d["s"], d["k"]), d["margin"], d["margin_s"])
    Lf, df = oracle.logm(A, force_s=s, force_k=k, **kw)
    assert df["info"] == 0, df
    return Lf


def check_logm(A, L, s, k, info, tol=TOL, **kw):
    """Compare one GPU result (L, s, k, info) with the oracle's Algorithm 1
    (run as the paper writes it unless ``kw`` says otherwise); returns the
    relative Frobenius error."""
    err = rel(L, oracle_at_plan(A, s, k, info, **kw))
    assert err <= tol, err
    return err
