"""The table-driven FP64 power x^p (Tang's table-driven log2 and exp2, used
for the dissipation potential's q^(a-1)) against a 40-digit decimal
reference: within 2 ulp wherever x^p is a normal double; special inputs
follow pow().  The double-float power of the FP32-bulk correction against the
same reference."""
import ctypes
import decimal
import math
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_dp = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def plib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("fpow") / "fpow.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                    os.path.join(ROOT, "tests", "native", "fpow_check.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    return lib


def run(lib, x, p):
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty_like(x)
    lib.host_pow(len(x), x.ctypes.data_as(_dp), p.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out


def test_within_two_ulp(plib):
    D = decimal.Decimal
    decimal.getcontext().prec = 40
    rng = np.random.default_rng(11)
    x = 10.0 ** rng.uniform(-300, 300, 6000)
    x[:40] = 1.0 + rng.uniform(-1e-9, 1e-9, 40)   # log2 x near 0
    x[40:80] = 2.0 ** rng.integers(-1000, 1000, 40)  # mantissa exactly 1
    p = rng.uniform(-1.0, 1.0, len(x))
    p[80:120] = -0.4                                # Norton n = 5: q^(a - 1)
    keep = np.abs(np.log2(x) * p) < 1000
    x, p = x[keep], p[keep]
    out = run(plib, x, p)
    worst = 0.0
    for xi, pi, oi in zip(x, p, out):
        ref = (D(float(xi)).ln() * D(float(pi))).exp()
        worst = max(worst, float(abs(D(float(oi)) - ref) / ref) / 2.0 ** -52)
    assert worst < 2.0, worst


def test_special_inputs(plib):
    x = np.array([1.0, 4.0, 0.0, 0.0, 5e-324, -2.0, np.inf, np.nan, 2.0, 1e-300])
    p = np.array([0.37, 0.0, 0.5, -0.5, 0.5, 0.5, 0.5, 0.5, 1100.0, -5.0])
    out = run(plib, x, p)
    assert out[0] == 1.0 and out[1] == 1.0
    assert out[2] == 0.0 and out[3] == math.inf
    assert out[4] == pytest.approx(math.pow(5e-324, 0.5), rel=1e-15)
    assert math.isnan(out[5]) and out[6] == math.inf and math.isnan(out[7])
    assert out[8] == math.inf and out[9] == math.inf  # beyond the double range


@pytest.fixture(scope="module")
def hlib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("dpow") / "hsc.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I/usr/local/cuda/include", os.path.join(ROOT, "tests", "native", "host_solver_check.cpp"),
                    "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.host_dpow.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              ctypes.POINTER(ctypes.c_float)]
    return lib


def test_double_float_power_within_2_pow_minus_45(hlib):
    """The correction's double-float power F = ac (x 2^e)^a (Tang's table
    method in FP32 pairs, a (e + E2) in FP64) against a 40-digit reference of
    the pair it was given: relative error below 2^-45 over x in [e^-8, e^8],
    scalings 2^-60..2^20, a in (-1, 1) and the Norton exponents a_phi - 1 =
    (1 - n)/(2n), ac over e^+-20; special inputs (zero, negative, out of
    range) leave the fast path."""
    D = decimal.Decimal
    decimal.getcontext().prec = 40
    rng = np.random.default_rng(5)
    out = (ctypes.c_float * 4)()
    worst = 0.0
    for it in range(4000):
        x = float(np.exp(rng.uniform(-8, 8)))
        if it < 40:
            x = 1.0 + float(rng.uniform(-1e-9, 1e-9))   # log2 x near 0
        e = int(rng.integers(-60, 20))
        n = float(rng.uniform(1, 20))
        a = (1 - n) / (2 * n) if it % 2 else float(rng.uniform(-1, 1))
        ac = float(np.exp(rng.uniform(-20, 20)))
        assert hlib.host_dpow(x, e, a, ac, out) == 1
        xe = (D(float(out[0])) + D(float(out[1]))) * D(2) ** e
        ref = D(ac) * (xe.ln() * D(a)).exp()
        got = D(float(out[2])) + D(float(out[3]))
        worst = max(worst, float(abs((got - ref) / ref)))
    assert worst < 2.0 ** -45, worst
    # a pair that is zero, negative or whose result leaves [2^-100, 2^100] takes the FP64 power
    for x, e, a in ((0.0, 0, -0.4), (-1.0, 0, -0.4), (1.5, -400, 0.9), (1e-300, 0, -0.4)):
        assert hlib.host_dpow(x, e, a, 1.0, out) == 0
