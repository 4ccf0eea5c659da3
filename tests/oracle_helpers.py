"""Exact polynomial helpers for the oracle pins (test-side arithmetic only)."""
from fractions import Fraction

import numpy as np


def _mul(a, b):
    r = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, z in enumerate(b):
                r[i + j] += x * z
    return r


def _add(a, b):
    n = max(len(a), len(b))
    a = a + [Fraction(0)] * (n - len(a))
    b = b + [Fraction(0)] * (n - len(b))
    return [u + v for u, v in zip(a, b)]


def k5_monomials(h, g, y):
    """Monomial coefficients b_0..b_32 of the k = 5 degree-optimal form with the
    given doubles, expanded in exact rational arithmetic (eq. five_mult_degopt
    written as polynomials in x instead of matrices)."""
    P = {1: [Fraction(1)], 2: [Fraction(0), Fraction(1)]}
    P[3] = _mul(P[2], P[2])
    t = 0
    for j in range(2, 6):
        lf, rf = [Fraction(0)], [Fraction(0)]
        for i in range(2, j + 2):
            lf = _add(lf, [Fraction(float(h[t])) * c for c in P[i]])
            rf = _add(rf, [Fraction(float(g[t])) * c for c in P[i]])
            t += 1
        P[j + 2] = _mul(lf, rf)
    z = [Fraction(0)]
    for i in range(1, 8):
        z = _add(z, [Fraction(float(y[i - 1])) * c for c in P[i]])
    return z


def k3_monomials(c):
    """Monomials b_0..b_8 of eq. (eqP8pol) with c = (c3, c4, d1, d2, e2, e0)
    given as doubles, in exact rational arithmetic:
    y02 = x^2 (c4 x^2 + c3 x), z = (y02 + d2 x^2 + d1 x)(y02 + e2 x^2)
    + e0 y02 + x^2/2 + x."""
    c3, c4, d1, d2, e2, e0 = (Fraction(float(v)) for v in c)
    x = [Fraction(0), Fraction(1)]
    x2 = _mul(x, x)
    y02 = _mul(x2, _add([c4 * t for t in x2], [c3 * t for t in x]))
    left = _add(_add(y02, [d2 * t for t in x2]), [d1 * t for t in x])
    right = _add(y02, [e2 * t for t in x2])
    z = _mul(left, right)
    z = _add(z, [e0 * t for t in y02])
    z = _add(z, [Fraction(1, 2) * t for t in x2])
    return _add(z, x)


def k4_monomials(c):
    """Monomials b_0..b_16 of the k = 4 (14+) scheme with
    c = (c3, c4, d1, d2, e2, f1, f2, f4, g1, g4, y3, y4, y5) given as doubles,
    in exact rational arithmetic: p4 = x^2 (c3 x + c4 x^2),
    p5 = (d1 x + d2 x^2 + p4)(e2 x^2 + p4),
    p6 = (f1 x + f2 x^2 + f4 p4 + p5)(g1 x + g4 p4 + p5),
    z = x + y3 x^2 + y4 p4 + y5 p5 + p6."""
    c3, c4, d1, d2, e2, f1, f2, f4, g1, g4, y3, y4, y5 = (Fraction(float(v)) for v in c)

    def sc(w, a):
        return [w * t for t in a]

    x = [Fraction(0), Fraction(1)]
    x2 = _mul(x, x)
    p4 = _mul(x2, _add(sc(c3, x), sc(c4, x2)))
    p5 = _mul(_add(_add(sc(d1, x), sc(d2, x2)), p4), _add(sc(e2, x2), p4))
    p6 = _mul(_add(_add(_add(sc(f1, x), sc(f2, x2)), sc(f4, p4)), p5), _add(_add(sc(g1, x), sc(g4, p4)), p5))
    z = _add(_add(_add(_add(x, sc(y3, x2)), sc(y4, p4)), sc(y5, p5)), p6)
    return z


def backward_error_coeffs(b, N=60, dps=60):
    """c_k of exp(-p(-x)) - 1 - x = sum c_k x^k (eq. DeltaAseries) for the
    polynomial p with monomial coefficients b (rationals), k = 0..N."""
    import mpmath as mp
    mp.mp.dps = dps
    S = [mp.mpf(0)] * (N + 1)
    for i, bi in enumerate(b):
        if i <= N:
            S[i] = -mp.mpf(bi.numerator) / bi.denominator * (-1) ** i
    E = [mp.mpf(0)] * (N + 1)
    E[0] = mp.mpf(1)
    for k in range(1, N + 1):
        E[k] = sum(j * S[j] * E[k - j] for j in range(1, k + 1)) / k
    E[0] -= 1
    E[1] -= 1
    return E


def read_golden_coeffs(path):
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, v = line.split()
            vals[name] = float(v)
    h = [vals[f"h_{j}_{i}"] for j in range(2, 6) for i in range(2, j + 2)]
    g = [vals[f"g_{j}_{i}"] for j in range(2, 6) for i in range(2, j + 2)]
    y = [vals[f"y_{i}"] for i in range(1, 8)]
    return np.array(h), np.array(g), np.array(y)


def theta_from_monomials(b, m, dps=60, N=160):
    """Theta_m = max{theta: sum_{k>=m} |c_{k+1}| theta^k <= u} (eqs. Eb,
    theta_Eb) where exp(-p(-x)) - 1 - x = sum c_k x^k and p has monomial
    coefficients b (rationals). Needs mpmath."""
    import mpmath as mp
    mp.mp.dps = dps
    S = [mp.mpf(0)] * (N + 1)
    for i, bi in enumerate(b):
        if i <= N:
            S[i] = -mp.mpf(bi.numerator) / bi.denominator * (-1) ** i
    E = [mp.mpf(0)] * (N + 1)
    E[0] = mp.mpf(1)
    for k in range(1, N + 1):
        E[k] = sum(j * S[j] * E[k - j] for j in range(1, k + 1)) / k
    c = E[:]
    c[0] -= 1
    c[1] -= 1

    def hbar(th):
        return sum(abs(c[k + 1]) * th ** k for k in range(m, N))

    lo, hi = mp.mpf("1e-12"), mp.mpf(1)
    u = mp.mpf(2) ** -53
    for _ in range(200):
        mid = (lo + hi) / 2
        if hbar(mid) <= u:
            lo = mid
        else:
            hi = mid
    return float(lo)
