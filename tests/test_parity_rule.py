"""The parity rule of ``tests/parity.py`` with the oracle on both sides (CPU).

A GPU plan (s, k) that differs from the oracle's is accepted only where a
plan comparison sat within 1e-10 of its threshold. Here the "GPU result" is
the oracle forced to a shifted plan: away from every threshold the rule must
reject it, at a threshold it must accept it.
"""
import numpy as np
import pytest

import oracle
from paper_2401_10089_gb300 import workloads
from tests.parity import check_logm


def test_rule_accepts_the_oracles_own_result():
    A = workloads.identity_plus(1, 40, seed=880)[0]
    L, d = oracle.logm(A)
    assert check_logm(A, L, d["s"], d["k"], 0) == 0.0


@pytest.mark.parametrize("ds,dk", [(1, 0), (-1, 0), (0, -1)])
def test_rule_rejects_a_shifted_plan_away_from_thresholds(ds, dk):
    A = workloads.identity_plus(1, 40, seed=881, lo=2.0, hi=2.0)[0]
    L, d = oracle.logm(A)
    assert d["s"] >= 1 and d["k"] >= 2 and d["margin"] > 1e-6, d
    s, k = d["s"] + ds, d["k"] + dk
    Lf, df = oracle.logm(A, force_s=s, force_k=k)
    assert (df["s"], df["k"]) == (s, k) and df["info"] == 0
    with pytest.raises(AssertionError, match="plan differs"):
        check_logm(A, Lf, s, k, 0)


def test_rule_accepts_a_shifted_plan_at_a_threshold():
    # diagonal A: the norms of the powers of A - I are exact, and with
    # max |lambda - 1| a hair above Theta_5 the first pass's comparisons all
    # sit at the threshold (relative distance 1e-13)
    theta = oracle.THETA_TABLE[4]
    A = np.diag(np.linspace(1.0 - 0.5 * theta, 1.0 + theta * (1.0 + 1e-13), 12))
    L, d = oracle.logm(A)
    assert d["s"] == 1 and d["margin_s"] == 0 and 5e-14 < d["margin"] < 2e-13, d
    Lf, df = oracle.logm(A, force_s=0)  # the other side of the threshold
    assert df["s"] == 0
    assert check_logm(A, Lf, 0, df["k"], 0) == 0.0
    # the two sides agree to rounding: the approximation error at Theta is below u
    assert np.linalg.norm(Lf - L) <= 1e-14 * np.linalg.norm(L)
