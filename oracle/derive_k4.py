"""Solve for the coefficients of the k = 4 (14+) scheme of Sec. 3.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests call
``derive()`` to check that the table compiled into ``logm_oracle.c`` is the
correctly rounded solution of its defining equations.

The scheme, in the degree-optimal form of eq. (five_mult_degopt):

    P_3 = X X
    P_4 = P_3 (c3 X + c4 P_3)
    P_5 = (d1 X + d2 P_3 + P_4)(e2 P_3 + P_4)
    P_6 = (f1 X + f2 P_3 + f4 P_4 + P_5)(g1 X + g4 P_4 + P_5)
    z   = X + y3 P_3 + y4 P_4 + y5 P_5 + P_6

is a polynomial of degree 16 in X with no constant term and x^1 coefficient
1. Its 13 unknowns are set by the 13 equations "coefficient of x^i = 1/i",
i = 2..14: the Taylor polynomial T_14 of -log(1 - x) (eq. Taylor_log)
matched exactly, with x^15, x^16 left over (the "+" of Table Table_theta's
m = 14+). The system has
several real roots; a search from random starting points found them, and the
one with the smallest largest coefficient (with c4 > 0) is the one kept. The
rounded values in ``START`` lie in its basin: Newton's method from them, at
50 digits, converges to it.

    python -m oracle.derive_k4      # prints the 13 doubles
"""
from __future__ import annotations

NAMES = ("c3", "c4", "d1", "d2", "e2", "f1", "f2", "f4", "g1", "g4", "y3", "y4", "y5")
START = (0.360275, 0.301844, 0.341229, -0.180471, 0.189073, -0.014079, 0.244007, -0.852563,
         0.146354, 0.978752, 0.502061, 0.609561, 1.209175)
DEGREE = 16


def monomials(c, zero, one):
    """Coefficients of z(x) (degree <= 16) for coefficient values c, in the
    number type of ``zero`` / ``one``."""
    c3, c4, d1, d2, e2, f1, f2, f4, g1, g4, y3, y4, y5 = c
    D = DEGREE + 1

    def mul(a, b):
        r = [zero] * D
        for i in range(D):
            if a[i] != 0:
                for j in range(D - i):
                    r[i + j] += a[i] * b[j]
        return r

    def comb(*terms):
        return [sum((w * v[i] for w, v in terms), zero) for i in range(D)]

    X = [zero] * D
    X[1] = one
    P3 = mul(X, X)
    P4 = mul(P3, comb((c3, X), (c4, P3)))
    P5 = mul(comb((d1, X), (d2, P3), (one, P4)), comb((e2, P3), (one, P4)))
    P6 = mul(comb((f1, X), (f2, P3), (f4, P4), (one, P5)), comb((g1, X), (g4, P4), (one, P5)))
    return comb((one, X), (y3, P3), (y4, P4), (y5, P5), (one, P6))


def derive(dps: int = 50):
    """The 13 coefficients as Python floats (correctly rounded from a
    ``dps``-digit solution) and the largest residual of the equations."""
    import mpmath as mp

    mp.mp.dps = dps
    zero, one = mp.mpf(0), mp.mpf(1)

    def equations(*c):
        z = monomials(c, zero, one)
        return [z[i] - one / i for i in range(2, 15)]

    root = mp.findroot(equations, [mp.mpf(v) for v in START], tol=mp.mpf(10) ** (-dps + 5), maxsteps=200)
    root = [root[i] for i in range(len(NAMES))]
    resid = max(abs(v) for v in equations(*root))
    return [float(v) for v in root], float(resid)


if __name__ == "__main__":
    vals, resid = derive()
    for name, v in zip(NAMES, vals):
        print(f"{name} {v!r}")
    print(f"# largest residual {resid:.1e}")
