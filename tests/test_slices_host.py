"""Digit split and level combination of the tensor-core FP64 products, on the
CPU: the __host__ __device__ helpers of csrc/fp64_slices.cuh compiled for the
host (g++), against exact rational arithmetic.

What the GPU path relies on:
  * the digits reconstruct the fixed-point integer exactly and stay within
    [-128, 128] (exact in BF16; products of two digits <= 2^14);
  * every level sum over 32 terms fits the FP32 accumulator exactly (<= 2^22);
  * the combined product is the exact dot product to within one FP64
    rounding of the result plus the split error, 2 K 2^(e_u + e_v - F)
    (F = 63 fractional bits), i.e. below FP64's own dot-product error bound
    K u sum |u_k v_k| whenever the row and column scales are within 2^9 of
    the magnitudes that meet in the sum.
"""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "slices_harness.cpp")
HDR = os.path.join(os.path.dirname(HERE), "paper_2401_10089_gb300", "csrc", "fp64_slices.cuh")
BUILD = os.path.join(HERE, "native", "_build")
LIB = os.path.join(BUILD, "libslices.so")
K = 32
F = 63


@pytest.fixture(scope="module")
def h():
    os.makedirs(BUILD, exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC],
                       check=True)
        os.replace(tmp, LIB)
    L = ctypes.CDLL(LIB)
    p = ctypes.c_void_p
    L.h_split.restype = ctypes.c_int32
    L.h_split.argtypes = [p, ctypes.c_int, p]
    L.h_sliced_dot.restype = ctypes.c_double
    L.h_sliced_dot.argtypes = [p, p, ctypes.c_int]
    L.h_level_int.restype = ctypes.c_int32
    L.h_level_int.argtypes = [ctypes.c_float]
    L.h_small_int_to_double.restype = ctypes.c_double
    L.h_small_int_to_double.argtypes = [ctypes.c_int64]
    L.h_slice_exponent.restype = ctypes.c_int32
    L.h_slice_exponent.argtypes = [ctypes.c_double]
    L.h_levels_to_double.restype = ctypes.c_int
    L.h_levels_to_double.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, p]
    L.h_combine_both.argtypes = [p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, p]
    L.h_level_int_wide.restype = ctypes.c_int32
    L.h_level_int_wide.argtypes = [ctypes.c_float]
    L.h_combine_fast.restype = ctypes.c_double
    L.h_combine_fast.argtypes = [p, ctypes.c_int32, ctypes.c_int32, p]
    L.h_combine_fp.restype = ctypes.c_double
    L.h_combine_fp.argtypes = [p, ctypes.c_int32, ctypes.c_int32]
    L.h_exact_int_to_double.restype = ctypes.c_double
    L.h_exact_int_to_double.argtypes = [ctypes.c_int64]
    L.h_levels32_agree.restype = ctypes.c_int
    L.h_levels32_agree.argtypes = [p, ctypes.c_int]
    L.h_split_routes_agree.restype = ctypes.c_int
    L.h_split_routes_agree.argtypes = [ctypes.c_double, ctypes.c_int32]
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def split(h, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    d = np.zeros(8 * len(u), dtype=np.int32)
    e = h.h_split(_ptr(u), len(u), _ptr(d))
    return e, d.reshape(8, len(u))


def rows(rng):
    yield rng.standard_normal(K)
    yield rng.standard_normal(K) * np.exp(rng.uniform(-30, 30, K))  # wide dynamic range in one row
    yield np.concatenate([np.zeros(K - 3), [1e-300, -5e-310, 3e-320]])  # subnormals
    yield -np.full(K, 1.0 - 2.0 ** -53)  # digits at the edge (-128)
    yield np.full(K, 2.0 ** 600 * (1 - 2.0 ** -52))
    yield np.zeros(K)
    u = rng.standard_normal(K)
    u[5:] = 0.0  # a short panel (K < 32): zero tail
    yield u


def test_digits_reconstruct_the_fixed_point_integer(h):
    rng = np.random.default_rng(1)
    for u in rows(rng):
        e, d = split(h, u)
        m = np.max(np.abs(u))
        if m == 0:
            assert e == 0 and not d.any()
            continue
        assert Fraction(m) < Fraction(2) ** e <= 2 * Fraction(m)  # the smallest e with m < 2^e
        assert d[0].min() >= -128 and d[0].max() <= 128 and d[1:].min() >= -128 and d[1:].max() <= 127
        for t in range(K):
            X = sum(int(d[i, t]) * 256 ** (7 - i) for i in range(8))
            exact = Fraction(u[t]) * Fraction(2) ** (F - e)
            assert abs(Fraction(X) - exact) <= Fraction(1, 2)  # X = round(u 2^(F - e))


def test_level_sums_fit_fp32_exactly(h):
    # worst case: every digit at its extreme; level 9 has 8 pairs of 32 terms
    assert 8 * 32 * 128 * 128 == 2 ** 22
    for v in list(range(-4096, 4097)) + [2 ** 22, -2 ** 22, 2 ** 22 - 1, -(2 ** 22 - 1), 3 * 2 ** 20 + 7]:
        assert h.h_level_int(float(v)) == v
    for x in (0, 1, -1, 2 ** 50 + 12345, -(2 ** 50) - 7, 2 ** 47 - 1):
        assert h.h_small_int_to_double(x) == float(x)


def test_sliced_dot_against_exact(h):
    rng = np.random.default_rng(2)
    us = list(rows(rng))
    vs = list(rows(np.random.default_rng(3)))
    for u in us:
        for v in vs:
            for k in (K, 7):
                uu, vv = np.ascontiguousarray(u[:k]), np.ascontiguousarray(v[:k])
                got = h.h_sliced_dot(_ptr(uu), _ptr(vv), k)
                eu = h.h_slice_exponent(float(np.max(np.abs(uu))))
                ev = h.h_slice_exponent(float(np.max(np.abs(vv))))
                exact = sum(Fraction(a) * Fraction(b) for a, b in zip(uu, vv))
                if abs(exact) > Fraction(np.finfo(np.float64).max):
                    continue  # beyond the double range
                # (+ k 2^-1074: products below the double range underflow, in any FP64 dot as well)
                bound = abs(exact) * Fraction(2) ** -53 + 2 * k * Fraction(2) ** (eu + ev - F) + k * Fraction(2) ** -1074
                assert abs(Fraction(got) - exact) <= bound, (got, float(exact))


def test_sliced_dot_matches_fp64_on_gaussian_data(h):
    # on data like a Gauss-Jordan update (Gaussian rows and columns) the
    # sliced product is at least as close to the exact value as an FP64 dot
    rng = np.random.default_rng(4)
    worse = 0
    for _ in range(300):
        u = rng.standard_normal(K)
        v = rng.standard_normal(K) * 10.0 ** rng.uniform(-3, 3)
        got = h.h_sliced_dot(_ptr(u), _ptr(v), K)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(u, v))
        fp64 = float(np.dot(u, v))
        worse += abs(Fraction(got) - exact) > abs(Fraction(fp64) - exact)
    assert worse <= 30  # one correctly rounded result against a sum of 32 rounded products


def test_non_finite_rows_propagate(h):
    u = np.ones(K)
    u[3] = np.inf
    v = np.ones(K)
    assert h.h_slice_exponent(np.inf) == h.h_slice_exponent(np.nan)
    assert np.isnan(h.h_sliced_dot(_ptr(u), _ptr(v), K))


def _round_exact(x: Fraction) -> float:
    """The nearest double to a rational (ties to even), for normal results."""
    return float(x)  # Python rounds Fraction -> float correctly (round-half-even)


def test_integer_conversion_rounds_correctly(h):
    # the epilogue's integer route: (hi 2^32 + lo) 2^E to the nearest double, no FP64 instruction
    rng = np.random.default_rng(5)
    out = ctypes.c_double()
    cases = [(0, 0, 0), (1, 0, -32), (0, 1, 0), (-1, 0, 0), (0, -1, 5), (2 ** 47 - 1, 2 ** 47 - 1, -70),
             (-(2 ** 47) + 1, 2 ** 47 - 1, -70), (1, -(2 ** 32), 0), (3, 2 ** 31, -3), (2 ** 40, 1, -70)]
    for _ in range(3000):
        hi = int(rng.integers(-(2 ** 47), 2 ** 47))
        lo = int(rng.integers(-(2 ** 47), 2 ** 47))
        if rng.random() < 0.3:  # near-ties: low bits with a single one
            lo = (lo & ~((1 << 24) - 1)) | (1 << int(rng.integers(0, 24)))
        cases.append((hi, lo, int(rng.integers(-200, 200))))
    for hi, lo, E in cases:
        ok = h.h_levels_to_double(hi, lo, E, ctypes.byref(out))
        exact = (Fraction(hi) * 2 ** 32 + lo) * Fraction(2) ** E
        assert ok == 1
        assert out.value == _round_exact(exact), (hi, lo, E, out.value, float(exact))


def test_integer_conversion_declines_out_of_range(h):
    out = ctypes.c_double(7.0)
    assert h.h_levels_to_double(1, 0, -1100, ctypes.byref(out)) == 0 and out.value == 7.0
    assert h.h_levels_to_double(2 ** 46, 0, 960, ctypes.byref(out)) == 0


def test_epilogue_routes_agree(h):
    # combine_levels_add (FP64 ops) and combine_levels_add_int (integer route + one add)
    # round T the same way: identical results on level sums within the FP32-exact range
    rng = np.random.default_rng(6)
    res = np.zeros(2)
    for _ in range(2000):
        c = rng.integers(-(2 ** 22), 2 ** 22 + 1, 8).astype(np.int32)
        eu, ev = (int(x) for x in rng.integers(-40, 40, 2))
        w = float(rng.standard_normal() * 2.0 ** rng.integers(-20, 20))
        h.h_combine_both(_ptr(c), eu, ev, w, _ptr(res))
        assert res[0] == res[1], (c, eu, ev, w, res)


def test_integer_split_matches_scaled_split(h):
    # the device split runs on integer operations only (fixed point from the
    # mantissa and exponent bits, digits from one biased integer): the same
    # integers and digits as the FP64-scaled split with its carry chain
    rng = np.random.default_rng(7)
    vals = [0.0, -0.0, 1.0, -1.0, 0.5, 1.5 * 2 ** -60, 5e-324, -3e-310, 1.0 - 2 ** -53, -(1.0 - 2 ** -53)]
    vals += list(rng.standard_normal(2000) * np.exp(rng.uniform(-80, 80, 2000)))
    # exact ties of the rounding: a mantissa whose dropped bits are 10...0
    vals += [float(Fraction(2 ** 52 + 2 * t + 1, 2 ** 52)) * 2.0 ** -70 for t in range(50)]
    for u in vals:
        m = abs(u)
        e0 = h.h_slice_exponent(m) if m > 0 else 0
        for e in (e0, e0 + 1, e0 + 9, e0 + 70):
            assert h.h_split_routes_agree(u, e) == 1, (u, e)


def test_32bit_conversion_matches_the_exact_one(h):
    # the epilogue's branch-free 32-bit conversion of the eight level sums
    # against the 128-bit one (itself pinned to exact rationals above)
    rng = np.random.default_rng(8)
    lim = 2 ** 22
    cases = [np.zeros(8), np.full(8, lim), np.full(8, -lim), np.array([0] * 7 + [1]), np.array([0] * 7 + [-1]),
             np.array([1] + [0] * 7), np.array([-1] + [0] * 7), np.array([lim, -lim, lim, -lim, lim, -lim, lim, -lim]),
             np.array([0, 0, 0, 0, 0, 0, 1, -256]), np.array([0, 0, 1, 0, 0, 0, 0, 0])]
    for _ in range(20000):
        c = rng.integers(-lim, lim + 1, 8)
        z = rng.random(8) < rng.random()  # leading levels zero: small T, every normalisation case
        c[np.cumsum(~z) == 0] = 0
        if rng.random() < 0.2:  # near ties of the rounding
            c[-3:] = rng.integers(-2, 3, 3)
        cases.append(c)
    for c in cases:
        c = np.ascontiguousarray(c, dtype=np.int32)
        for E in (-70, -200, 0, 37):
            assert h.h_levels32_agree(_ptr(c), E) == 1, (c.tolist(), E)
    for E in (-1100, -1030, 990, 1000):  # results out of the normal range: both refuse alike
        c = np.full(8, 3, dtype=np.int32)
        assert h.h_levels32_agree(_ptr(c), E) == 1


def test_exact_int_to_double(h):
    rng = np.random.default_rng(9)
    xs = [0, 1, -1, 2 ** 52, -(2 ** 52), 2 ** 53 - 1, -(2 ** 53 - 1), 3, 2 ** 47 + 5]
    xs += [int(v) for v in rng.integers(-(2 ** 53) + 1, 2 ** 53, 5000)]
    xs += [int(v) >> int(s) for v, s in zip(rng.integers(-(2 ** 53) + 1, 2 ** 53, 2000), rng.integers(0, 53, 2000))]
    for x in xs:
        assert h.h_exact_int_to_double(x) == float(x), x


def test_level_sums_over_four_chunks(h):
    # a K = 128 update accumulates four chunks of 32 terms per level: sums up
    # to 4 * 2^22 = 2^24, still exact in FP32, converted by the two-part route
    rng = np.random.default_rng(10)
    vals = [0, 1, -1, 2 ** 24, -(2 ** 24), 2 ** 24 - 1, -(2 ** 24 - 1), 2 ** 23 + 1, 4095, 4096, 4097, -2049, 2048]
    vals += [int(v) for v in rng.integers(-(2 ** 24), 2 ** 24 + 1, 20000)]
    for v in vals:
        assert h.h_level_int_wide(float(v)) == v, v


def test_branch_free_combination_matches_or_defers(h):
    # the epilogue's branch-free route gives combine_levels_fp's value bit for
    # bit, or flags the element for it: exactly when a scale is non-finite or
    # the result would be subnormal or overflow (zero stays zero)
    rng = np.random.default_rng(11)
    nonfin = -0x40000000
    cases = []
    for _ in range(4000):
        c = rng.integers(-(2 ** 24), 2 ** 24 + 1, 8).astype(np.int32)
        if rng.random() < 0.1:
            c[:] = 0
        eu, ev = (int(x) for x in rng.integers(-1100, 1100, 2))
        cases.append((c, eu, ev))
    for eu, ev in ((nonfin, 3), (5, nonfin), (-1022, -60), (1023, 200), (0, 0)):
        cases.append((rng.integers(-1000, 1000, 8).astype(np.int32), eu, ev))
    n_slow = 0
    for c, eu, ev in cases:
        slow = np.zeros(1, dtype=np.int32)
        r = h.h_combine_fast(_ptr(c), eu, ev, _ptr(slow))
        ref = h.h_combine_fp(_ptr(c), eu, ev)
        if slow[0]:
            n_slow += 1
            finite = eu != nonfin and ev != nonfin
            a = abs(ref)
            assert (not finite) or a == float("inf") or a < 2.2250738585072014e-308, (c, eu, ev, ref)
        else:
            assert np.float64(r).tobytes() == np.float64(ref).tobytes(), (c, eu, ev, r, ref)
    assert 0 < n_slow < len(cases)
