"""The coefficient tables compiled into the CUDA library, read from its
sources, against the paper's values (tests/golden, Table
table_simple_experiment) and the oracle's k = 4 table: a typo in a device
table is caught on the CPU, before any GPU run. The FP32 copies of the
split-precision kernels must be the FP64 values rounded to float."""
import os
import re

import numpy as np

import oracle
from tests.oracle_helpers import read_golden_coeffs

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2401_10089_gb300", "csrc")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table(fname, name):
    src = open(os.path.join(CSRC, fname)).read()
    m = re.search(r"__constant__\s+(?:double|float)\s+" + re.escape(name) + r"\[\d+\]\s*=\s*\{([^}]*)\}", src)
    assert m, (fname, name)
    return np.array([float(t.rstrip("f")) for t in re.findall(r"[-+]?\d+\.\d*(?:e[-+]?\d+)?f?", m.group(1))])


def test_fp64_device_tables():
    h, g, y = read_golden_coeffs(os.path.join(GOLDEN, "k5_coefficients.txt"))
    assert np.array_equal(table("logm_algo.cuh", "c_h5"), h)
    assert np.array_equal(table("logm_algo.cuh", "c_g5"), g)
    assert np.array_equal(table("logm_algo.cuh", "c_y5"), y)
    assert np.array_equal(table("logm_algo.cuh", "c_k4"), oracle.coeffs_k4())


def test_fp32_device_tables_are_the_rounded_values():
    h, g, y = read_golden_coeffs(os.path.join(GOLDEN, "k5_coefficients.txt"))
    f32 = lambda a: np.asarray(a, dtype=np.float32)  # noqa: E731
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_h5")), f32(h))
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_g5")), f32(g))
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_y5")), f32(y))
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_k4")), f32(oracle.coeffs_k4()))
