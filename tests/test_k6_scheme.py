"""Pins of the derived k = 6 degree-optimal scheme (tests/golden/k6_coefficients.txt,
written by oracle/derive_k6.py): the paper prints no k >= 6 coefficients, so
the table is checked against what the paper requires of such a scheme.

  * eq. Taylor_log: its monomials b_i equal 1/i to rounding for i <= 34
    (exact rational arithmetic on the stored doubles);
  * eqs. Eb, theta_Eb: the backward-error Theta, recomputed at 60 digits, is
    at least Table Table_theta's Theta_6 = 0.372, with the sum taken from
    m_6 = 20 as in the table and also over every term;
  * Sec. 4, eqs. aj and stability_error: the monomials computed with FP64
    rounding are within O(u) of the exact ones, and |(1/i - b_i) i| <= 1 for
    i > 34;
  * the scheme evaluated directly (50 digits) approximates -log(1 - x) to
    within a few u on the disk |x| <= 0.372.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from tests.oracle_helpers import _add, _mul, theta_from_monomials

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "k6_coefficients.txt")
K, DEG, M = 6, 64, 34
U = 2.0 ** -53


def load():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, v = line.split()
            vals[name] = float(v)
    h = {j: [vals[f"h_{j}_{i}"] for i in range(2, j + 2)] for j in range(2, K + 1)}
    g = {j: [vals[f"g_{j}_{i}"] for i in range(2, j + 2)] for j in range(2, K + 1)}
    y = [vals[f"y_{i}"] for i in range(3, K + 3)]
    return h, g, y


def exact_monomials(h, g, y):
    def sc(w, a):
        return [Fraction(w) * t for t in a]

    P = {2: [Fraction(0), Fraction(1)], 3: [Fraction(0), Fraction(0), Fraction(1)]}
    for j in range(2, K + 1):
        a, b = [Fraction(0)], [Fraction(0)]
        for i in range(2, j + 2):
            a = _add(a, sc(h[j][i - 2], P[i]))
            b = _add(b, sc(g[j][i - 2], P[i]))
        P[j + 2] = _mul(a, b)
    z = P[2][:]
    for i in range(3, K + 3):
        z = _add(z, sc(y[i - 3], P[i]))
    return z + [Fraction(0)] * (DEG + 1 - len(z))


def fp64_monomials(h, g, y):
    P = {2: np.zeros(DEG + 1), 3: np.zeros(DEG + 1)}
    P[2][1] = 1.0
    P[3][2] = 1.0
    for j in range(2, K + 1):
        a, b = np.zeros(DEG + 1), np.zeros(DEG + 1)
        for i in range(2, j + 2):
            a = a + h[j][i - 2] * P[i]
            b = b + g[j][i - 2] * P[i]
        P[j + 2] = np.convolve(a, b)[:DEG + 1]
    z = P[2].copy()
    for i in range(3, K + 3):
        z = z + y[i - 3] * P[i]
    return z


@pytest.fixture(scope="module")
def scheme():
    h, g, y = load()
    return h, g, y, exact_monomials(h, g, y)


def test_taylor_terms_matched_to_order_34(scheme):
    h, g, y, b = scheme
    assert b[0] == 0 and b[1] == 1
    worst = max(abs(float((b[i] - Fraction(1, i)) * i)) for i in range(2, M + 1))
    assert worst <= 4 * U, worst
    # and not beyond: the scheme is not the exact Taylor polynomial of degree 64
    assert abs(float((b[M + 1] - Fraction(1, M + 1)) * (M + 1))) > 1e-8


def test_theta_at_least_the_papers_theta_6(scheme):
    pytest.importorskip("mpmath")
    b = scheme[3]
    assert float(theta_from_monomials(b, 20, N=200)) >= 0.372
    assert float(theta_from_monomials(b, 1, N=200)) >= 0.372  # every term counted


def test_stability_indicator_of_sec_4(scheme):
    h, g, y, b = scheme
    bt = fp64_monomials(h, g, y)
    rel = max(abs(float((Fraction(bt[i]) - b[i]) / b[i])) for i in range(1, DEG + 1) if b[i] != 0)
    assert rel <= 16 * U, rel / U
    assert max(abs((1.0 / i - bt[i]) * i) for i in range(M + 1, DEG + 1)) <= 1.0


def test_direct_evaluation_on_the_disk(scheme):
    mp = pytest.importorskip("mpmath")
    h, g, y, _ = scheme
    mp.mp.dps = 50

    def z(x):
        P = {2: x, 3: x * x}
        for j in range(2, K + 1):
            a = sum(mp.mpf(h[j][i - 2]) * P[i] for i in range(2, j + 2))
            b = sum(mp.mpf(g[j][i - 2]) * P[i] for i in range(2, j + 2))
            P[j + 2] = a * b
        return P[2] + sum(mp.mpf(y[i - 3]) * P[i] for i in range(3, K + 3))

    for r in (0.05, 0.2, 0.372):
        for t in range(12):
            x = mp.mpf(r) * mp.expjpi(mp.mpf(t) / 6)
            f = -mp.log(1 - x)
            assert abs(z(x) - f) / abs(f) <= 4 * U, (r, t)


def test_a_planted_mistake_is_caught(scheme):
    # one coefficient off by one part in 10^10: the Taylor pin fails
    h, g, y, _ = scheme
    h2 = {j: list(v) for j, v in h.items()}
    h2[4][1] *= 1.0 + 1e-10
    b = exact_monomials(h2, g, y)
    worst = max(abs(float((b[i] - Fraction(1, i)) * i)) for i in range(2, M + 1))
    assert worst > 1e3 * U
