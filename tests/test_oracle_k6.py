"""The oracle's k = 6 order (opt-in, k_max = 6): its table, its graph
evaluation, its plan and Algorithm 1 with it.

The coefficients are the fitted ones of tests/golden/k6_coefficients.txt
(pinned against the paper's criteria in test_k6_scheme.py); here the oracle
is pinned to them and to what Algorithm 1 must do with Theta_6 = 0.372 and
m_6 = 20 of Table Table_theta:

  * the C table is the golden file, value for value;
  * graph_eval(X, 6) is the exact-rational expansion of eq. five_mult_degopt
    with those coefficients, evaluated by Horner (a wrong index or a dropped
    term in the C scheme changes a monomial);
  * on diagonal inputs alpha is known exactly, so (s, k) follow by hand;
  * log A from closed forms, and fewer square roots than with k_max = 5 where
    ||A - I|| lies between Theta_5 and Theta_6.
"""
import math

import numpy as np
import pytest

import oracle
from tests.test_k6_scheme import exact_monomials, load

U = 2.0 ** -53


def rel(a, b):
    return np.linalg.norm(a - b, 1) / np.linalg.norm(b, 1)


def test_c_table_is_the_golden_file():
    h, g, y = oracle.coeffs_k6()
    gh, gg, gy = load()
    assert np.array_equal(h, np.concatenate([gh[j] for j in range(2, 7)]))
    assert np.array_equal(g, np.concatenate([gg[j] for j in range(2, 7)]))
    assert np.array_equal(y, np.array([0.0, 1.0] + gy))


def test_graph_eval_k6_is_the_expanded_polynomial():
    b = [float(c) for c in exact_monomials(*load())]
    assert len(b) == 65 and b[0] == 0.0
    rng = np.random.default_rng(61)
    for n, r in ((1, 0.37), (5, 0.3), (12, 0.2)):
        X = rng.standard_normal((n, n))
        X *= r / np.linalg.norm(X, 1)
        Z = oracle.graph_eval(X, 6)
        H = oracle.horner(X, np.array(b))
        assert rel(Z, H) < 64 * U, n
        # through P3 = X^2 given by the caller (Algorithm 1 with s >= 1)
        Z3 = oracle.graph_eval(X, 6, P3=X @ X)
        assert rel(Z3, H) < 64 * U, n
    # the comparison sees a swapped pair of coefficients (h_{6,6}, h_{6,7})
    h, g, y = load()
    h[6][4], h[6][5] = h[6][5], h[6][4]
    b_bad = [float(c) for c in exact_monomials(h, g, y)]
    assert rel(Z, oracle.horner(X, np.array(b_bad))) > 1e-6


def test_graph_eval_k6_scalar_log():
    # on the disk |x| <= Theta_6 the scheme is -log(1 - x) to a few u
    for x in (-0.372, -0.2, 1e-3, 0.1, 0.3, 0.372):
        z = oracle.graph_eval(np.array([[x]]), 6)[0, 0]
        assert abs(z + math.log1p(-x)) <= 8 * U * abs(math.log1p(-x)), x


def _expected_plan_diagonal(lam, k_max):
    th = oracle.THETA_TABLE
    s, mu = 0, np.array(lam, dtype=float)
    while np.max(np.abs(mu - 1)) > th[k_max - 1]:
        mu = np.sqrt(mu)
        s += 1
    a = np.max(np.abs(mu - 1))
    return s, next(k for k in oracle.AVAILABLE_K if a <= th[k - 1])


@pytest.mark.parametrize("lam", [
    [1.3, 0.8],          # alpha in (Theta_5, Theta_6]: k = 6 at s = 0
    [1.2, 0.95, 1.0],    # alpha <= Theta_5: k = 5 even with k_max = 6
    [0.64, 1.1],         # alpha = 0.36
    [3.0, 0.2, 1.0],
    [100.0, 0.01],
    [1.0 + 1e-5, 0.99999],
])
def test_plan_diagonal_k6(lam):
    s_exp, k_exp = _expected_plan_diagonal(lam, 6)
    L, d = oracle.logm(np.diag(lam), k_max=6)
    assert (d["s"], d["k"], d["info"]) == (s_exp, k_exp, oracle.OK)
    assert np.allclose(np.diag(L), np.log(lam), rtol=1e-13, atol=1e-15)


def test_plan_call_k6():
    A = np.diag([1.3, 0.8, 1.0])
    fin, k, a = oracle.plan(A, k_max=6)
    assert fin and k == 6 and a == pytest.approx(0.3, rel=1e-12)
    fin, k, a = oracle.plan(A)  # k_max = 5: alpha = 0.3 > Theta_5, one more root
    assert not fin and k == 5


def test_logm_k6_closed_forms_and_fewer_roots():
    for r, t in ((1.0, 0.3), (1.2, 0.25), (2.0, 1.5), (0.3, -2.5)):
        A = r * np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
        L6, d6 = oracle.logm(A, k_max=6)
        L5, d5 = oracle.logm(A)
        ref = np.array([[math.log(r), -t], [t, math.log(r)]])
        assert d6["info"] == oracle.OK and np.allclose(L6, ref, rtol=0, atol=2e-14 * max(1, abs(t)))
        assert d6["s"] <= d5["s"]
    # eigenvalues 1.3 .. 0.8 with a small non-normal part: alpha_m stays near
    # 0.3 for every m, between Theta_5 and Theta_6, so no square root with
    # k_max = 6 and one with k_max = 5
    rng = np.random.default_rng(62)
    E = np.triu(rng.standard_normal((8, 8)), 1)
    A = np.diag(np.linspace(1.3, 0.8, 8)) + 1e-3 * E
    L6, d6 = oracle.logm(A, k_max=6)
    L5, d5 = oracle.logm(A)
    assert (d6["s"], d6["k"]) == (0, 6) and d5["s"] == 1
    assert rel(L6, L5) < 1e-14
    assert rel(oracle.expm_taylor(L6), A) < 1e-14


def test_logm_k6_random_matches_k5():
    # the two orders give the same logarithm to rounding on general inputs,
    # the k = 6 one with no more square roots
    rng = np.random.default_rng(63)
    for n in (3, 16, 40):
        A = np.eye(n) + rng.standard_normal((n, n)) / math.sqrt(n)
        L6, d6 = oracle.logm(A, k_max=6)
        L5, d5 = oracle.logm(A)
        assert d6["info"] == d5["info"] == oracle.OK
        assert d6["s"] <= d5["s"]
        assert rel(L6, L5) < 1e-12


def test_plan_with_ai2_k6():
    # s >= 1: the plan takes A_I2 = A_2 - 2A + I (eq. AI2) with A = A_2^{1/2};
    # on a diagonal, alpha = max |mu - 1| exactly
    lam = np.array([1.69, 0.64, 1.0])
    X = np.diag(np.sqrt(lam))
    AI2 = np.diag(lam) - 2 * X + np.eye(3)
    fin, k, a = oracle.plan(X, AI2, k_max=6)
    assert fin and k == 6 and a == pytest.approx(0.3, rel=1e-12)
    fin, k, a = oracle.plan(X, AI2)  # k_max = 5: not finished at this level
    assert not fin and k == 5
