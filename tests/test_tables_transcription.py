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
    # k = 6 (fitted; the golden file is the fit's output)
    h6, g6, y6 = oracle.coeffs_k6()
    assert np.array_equal(table("logm_algo.cuh", "c_h6"), h6)
    assert np.array_equal(table("logm_algo.cuh", "c_g6"), g6)
    assert np.array_equal(table("logm_algo.cuh", "c_y6"), y6[2:])


def test_fp32_device_tables_are_the_rounded_values():
    h, g, y = read_golden_coeffs(os.path.join(GOLDEN, "k5_coefficients.txt"))
    f32 = lambda a: np.asarray(a, dtype=np.float32)  # noqa: E731
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_h5")), f32(h))
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_g5")), f32(g))
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_y5")), f32(y))
    assert np.array_equal(f32(table("scheme_f32.cuh", "c_tc_k4")), f32(oracle.coeffs_k4()))


def test_theta_table_of_the_library():
    """The library's default Theta_{m_k} (one table, logm_internal.h, used by
    every entry point) against the paper's backward-error table (golden) and
    the oracle's copy."""
    src = open(os.path.join(CSRC, "logm_internal.h")).read()
    m = re.search(r"constexpr\s+double\s+kThetaPaper\[6\]\s*=\s*\{([^}]*)\}", src)
    assert m
    dev = np.array([float(t) for t in re.findall(r"[-+]?\d+\.\d*(?:e[-+]?\d+)?", m.group(1))])
    gold = np.array([float(line.split()[3]) for line in open(os.path.join(GOLDEN, "theta_table.txt"))
                     if line.strip() and not line.startswith("#")])
    assert np.array_equal(dev, gold)
    assert np.array_equal(np.array(oracle.THETA_TABLE), gold)
    # no second copy of the table elsewhere in the library's sources
    for f in os.listdir(CSRC):
        if f != "logm_internal.h":
            code = re.sub(r"//[^\n]*|/\*.*?\*/", "", open(os.path.join(CSRC, f)).read(), flags=re.S)
            assert "9.31e-2" not in code and "2.46e-1" not in code and "3.72e-1" not in code, f
