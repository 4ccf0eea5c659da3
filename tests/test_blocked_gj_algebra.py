"""The algebra of the whole-GPU kernel's blocked Gauss-Jordan inversion, on
the CPU in float64 with numpy (a design check of the data flow, independent of
the CUDA code and of the oracle).

The tensor-core form groups 32-column panels into super-panels of four. Inside
a super-panel each panel's rank-32 update reaches only the super-panel's other
columns at once. For the columns outside, only the row swaps are applied at
once; the factors U_q = P_q - I_{J_q} are kept with rows permuted by the later
swaps, and the pivot-row blocks follow the recurrence
    v_q = W[J_q, :] + sum_{p < q} U_p[J_q, :] v_p.
One K = 128 product then updates the outside columns. These tests replay that
flow, with partial pivoting inside each panel, and check that it reproduces
the inverse and log|det| of the unblocked elimination.
"""
import numpy as np
import pytest

PW, SC = 32, 128


def _panel(W, kb, jb, piv, pivval):
    """Gauss-Jordan on the panel columns [kb, kb + jb) of all rows, with
    partial pivoting: returns the finished panel (in-place inverse form)."""
    P = W[:, kb:kb + jb].copy()
    for c in range(jb):
        k = kb + c
        p = k + int(np.argmax(np.abs(P[k:, c])))
        piv[k] = p
        P[[k, p]] = P[[p, k]]
        d = P[k, c]
        pivval[k] = d
        prow = P[k] / d
        prow[c] = 1.0 / d
        f = P[:, c].copy()
        Q = P - np.outer(f, prow)
        Q[:, c] = -f / d
        Q[k] = prow
        P = Q
    return P


def _trace(s, kb, jb, piv):
    """Original position of what the panel's swaps leave at position s."""
    for t in range(jb - 1, -1, -1):
        k, p = kb + t, piv[kb + t]
        s = p if s == k else (k if s == p else s)
    return s


def blocked_inverse(A, sc=SC, correction=True):
    """The inverse and log|det A| by the blocked flow: super-panels of sc
    columns; correction=False drops the recurrence's sum (a planted mistake)."""
    n = A.shape[0]
    W = A.copy()
    piv = np.zeros(n, dtype=int)
    pivval = np.zeros(n)
    ucat = np.zeros((n, sc))
    vcat = np.zeros((n, sc))
    for K0 in range(0, n, sc):
        B = min(sc, n - K0)
        m = (B + PW - 1) // PW
        outside = np.ones(n, dtype=bool)
        outside[K0:K0 + B] = False
        for q in range(m):
            kb = K0 + q * PW
            jb = min(PW, n - kb)
            Pn = _panel(W, kb, jb, piv, pivval)
            W[:, kb:kb + jb] = Pn
            U = Pn.copy()
            U[kb:kb + jb, :] -= np.eye(jb)
            ucat[:, q * PW:q * PW + jb] = U
            ucat[:, q * PW + jb:(q + 1) * PW] = 0.0
            UsT = ucat[[_trace(kb + c, kb, jb, piv) for c in range(jb)], :q * PW]
            # the swaps as one permutation of the rows they touch, every column but J_q
            pos = list(range(kb, kb + jb)) + [int(piv[kb + t]) for t in range(jb)]
            src = [_trace(x, kb, jb, piv) for x in pos]
            cols = np.r_[0:kb, kb + jb:n]
            W[np.ix_(pos, cols)] = W[np.ix_(src, cols)]
            R = W[kb:kb + jb, :].copy()
            corr = UsT @ vcat[outside, :q * PW].T if correction else 0.0
            vcat[outside, q * PW:q * PW + jb] = (R[:, outside] + corr).T
            vcat[outside, q * PW + jb:(q + 1) * PW] = 0.0
            if m > 1:  # the narrow update: the super-panel's other columns
                inner = [j for j in range(K0, K0 + B) if not kb <= j < kb + jb]
                W[:, inner] += U @ R[:, inner]
            if q > 0:  # the later swaps reach the earlier factors' rows
                ucat[pos, :q * PW] = ucat[src, :q * PW]
        W[:, outside] += ucat[:, :m * PW] @ vcat[outside, :m * PW].T
    perm = list(range(n))
    for k in range(n - 1, -1, -1):
        p = piv[k]
        perm[k], perm[p] = perm[p], perm[k]
    return W[:, perm], float(np.sum(np.log(np.abs(pivval))))


@pytest.mark.parametrize("n", [40, 129, 257, 300])
def test_blocked_gauss_jordan_reproduces_the_inverse(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 0.5 * n ** 0.5 * np.eye(n)
    X, ld = blocked_inverse(A)
    Ai = np.linalg.inv(A)
    assert np.linalg.norm(X - Ai) / np.linalg.norm(Ai) < 1e-12
    assert abs(ld - np.linalg.slogdet(A)[1]) < 1e-9 * n


def test_blocked_and_unblocked_agree_and_the_recurrence_matters():
    rng = np.random.default_rng(5)
    n = 257
    A = rng.standard_normal((n, n)) + 8.0 * np.eye(n)
    Ai = np.linalg.inv(A)
    X, _ = blocked_inverse(A)
    X1, _ = blocked_inverse(A, sc=PW)  # super-panels of one panel: the unblocked form
    assert np.linalg.norm(X - X1) / np.linalg.norm(Ai) < 1e-12
    # a planted mistake (pivot rows without the earlier panels' terms) is caught
    Xbad, _ = blocked_inverse(A, correction=False)
    assert np.linalg.norm(Xbad - Ai) / np.linalg.norm(Ai) > 1e-6
