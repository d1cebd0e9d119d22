"""The double-float power of the FP32-bulk correction (dpow.cuh) on the GPU:
the device build gives the same pairs as the host build bit for bit (every
step is an exact or explicitly rounded FP32 operation, or one of the three
rounded FP64 ones), takes the same fast-path decisions, and is within 2^-45
of a 40-digit reference of F = ac (x 2^e)^a."""
import ctypes
import decimal
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = tmp_path_factory.mktemp("dpow")
    dev = str(d / "dpow_dev.so")
    host = str(d / "hsc.so")
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-diag-suppress", "177",
                    os.path.join(ROOT, "tests", "native", "dpow_check.cu"), "-o", dev], check=True)
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I/usr/local/cuda/include", os.path.join(ROOT, "tests", "native", "host_solver_check.cpp"),
                    "-o", host], check=True)
    dl, hl = ctypes.CDLL(dev), ctypes.CDLL(host)
    dl.dpow_many.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_int]
    hl.host_dpow.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.POINTER(ctypes.c_float)]
    return dl, hl


def test_device_power_equals_host_build_and_reference(libs):
    dl, hl = libs
    rng = np.random.default_rng(23)
    n = 1 << 14
    x = np.exp(rng.uniform(-8, 8, n))
    e = rng.integers(-60, 20, n).astype(np.int32)
    nn = rng.uniform(1, 20, n)
    a = np.where(np.arange(n) % 2 == 1, (1 - nn) / (2 * nn), rng.uniform(-1, 1, n))
    ac = np.exp(rng.uniform(-20, 20, n))
    # edges: 1 + tiny, zero, negative, results beyond 2^+-100
    x[:4], e[:4], a[:4] = [1.0 + 1e-12, 0.0, -1.0, 1.5], [0, 0, 0, -400], [-0.4, -0.4, -0.4, 0.9]
    ac[:4] = 1.0
    out = np.zeros(4 * n, dtype=np.float32)
    ok = np.zeros(n, dtype=np.int32)
    assert dl.dpow_many(x.ctypes.data, e.ctypes.data, a.ctypes.data, ac.ctypes.data, out.ctypes.data,
                        ok.ctypes.data, n) == 0
    hout = (ctypes.c_float * 4)()
    href = np.zeros(4 * n, dtype=np.float32)
    hok = np.zeros(n, dtype=np.int32)
    for i in range(n):
        hok[i] = hl.host_dpow(float(x[i]), int(e[i]), float(a[i]), float(ac[i]), hout)
        href[4 * i:4 * i + 4] = np.frombuffer(hout, dtype=np.float32)
    assert np.array_equal(ok, hok)
    assert list(ok[:4]) == [1, 0, 0, 0] and ok[4:].all()
    fast = np.repeat(ok.astype(bool), 4)
    assert np.array_equal(out[fast].view(np.uint32), href[fast].view(np.uint32))
    D = decimal.Decimal
    decimal.getcontext().prec = 40
    worst = 0.0
    for i in range(4, n, 37):
        xe = (D(float(out[4 * i])) + D(float(out[4 * i + 1]))) * D(2) ** int(e[i])
        ref = D(float(ac[i])) * (xe.ln() * D(float(a[i]))).exp()
        got = D(float(out[4 * i + 2])) + D(float(out[4 * i + 3]))
        worst = max(worst, float(abs((got - ref) / ref)))
    assert worst < 2.0 ** -45, worst
