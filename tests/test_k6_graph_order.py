"""The evaluation order of the k = 6 graph in the one-block-per-matrix kernels,
replayed on the CPU with numpy in float64. This is a design check of the data
flow that fits P_2 .. P_8 of eq. five_mult_degopt into seven n x n matrices;
it is independent of the CUDA code and of the oracle's evaluation.

The kernels' order:
 1. P_4 .. P_6 as for any k.
 2. The factors of P_7 into T1, T2.
 3. One elementwise pass overwriting P_2, P_3, P_4 by
      C_L = sum_{i<=6} h_{6,i} P_i,  C_R = sum_{i<=6} g_{6,i} P_i,
      C_Y = sum_{i<=6} y_i P_i.
 4. P_7 into the freed P_5 matrix.
 5. L_6 = C_L + h_{6,7} P_7 and R_6 = C_R + g_{6,7} P_7.
 6. z = y_8 L_6 R_6 + C_Y + y_7 P_7.
The replay keeps the seven matrices by name and every step reads them as they
are at that point. A value read after it was overwritten would change the
result, which must equal the oracle's straightforward evaluation.
"""
import numpy as np

import oracle


def replay(X, h, g, y, swap_bug=False):
    """The kernels' sequence on seven named matrices; returns z(X)."""
    slot = {"Acur": X.copy(), "A2": X @ X, "Y": None, "W1": None, "W2": None, "T1": None, "T2": None}
    live = {2: "Acur", 3: "A2", 4: "Y", 5: "W1", 6: "W2"}  # P_i -> matrix holding it
    t = 0
    for j in range(2, 6):
        hj, gj = h[t:t + j], g[t:t + j]
        slot["T1"] = sum(hj[i - 2] * slot[live[i]] for i in range(2, j + 2))
        slot["T2"] = sum(gj[i - 2] * slot[live[i]] for i in range(2, j + 2))
        if j < 5:
            slot[live[j + 2]] = slot["T1"] @ slot["T2"]
        t += j
    h6, g6 = h[t:t + 6], g[t:t + 6]
    P = [slot[live[i]] for i in range(2, 7)]  # read every element before writing any
    cl = sum(h6[i] * P[i] for i in range(5))
    cr = sum((h6 if swap_bug else g6)[i] * P[i] for i in range(5))
    cy = P[0] + sum(y[i + 1] * P[i] for i in range(1, 5))  # y = y_1 .. y_8, y_2 = 1
    slot["Acur"], slot["A2"], slot["Y"] = cl, cr, cy
    slot["W1"] = slot["T1"] @ slot["T2"]  # P_7
    slot["W2"] = slot["Acur"] + h6[5] * slot["W1"]
    slot["T1"] = slot["A2"] + g6[5] * slot["W1"]
    return y[7] * (slot["W2"] @ slot["T1"]) + slot["Y"] + y[6] * slot["W1"]


def test_k6_order_reproduces_the_graph():
    h, g, y = oracle.coeffs_k6()
    rng = np.random.default_rng(65)
    for n, r in ((1, 0.37), (6, 0.3), (40, 0.2)):
        X = rng.standard_normal((n, n))
        X *= r / np.abs(X).sum(axis=0).max()
        Z = oracle.graph_eval(X, 6)
        assert np.linalg.norm(replay(X, h, g, y) - Z) <= 1e-14 * np.linalg.norm(Z)
        # a mistake in the in-place pass (h where g belongs) is seen
        assert np.linalg.norm(replay(X, h, g, y, swap_bug=True) - Z) > 1e-6 * np.linalg.norm(Z)
