"""recip_pos (solver.cuh) on the GPU: the reciprocal from an FP32 seed and two
Newton steps r <- r + r (1 - x r) that scales the ode23 error measure.  Each
step squares the relative error, so from the seed's < 2^-22 the result is
within rounding of 1/x: at most one unit in the last place of the correctly
rounded FP64 reciprocal, over the normal range."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rlib(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("recip") / "recip.so")
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-diag-suppress", "177",
                    os.path.join(ROOT, "tests", "native", "recip_check.cu"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.recip_many.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return lib


def test_recip_pos_within_one_ulp(rlib):
    rng = np.random.default_rng(0)
    x = np.exp2(rng.uniform(-1020.0, 1020.0, 1 << 20))
    edges = np.array([1.0, np.nextafter(2.0, 0.0), 2.0, np.nextafter(1.0, 2.0), 3.0, 0.1, 1e-300, 1e300,
                      np.ldexp(1.0, -1021), np.ldexp(1.0, 1021), 1.5, 1.25, 1.75])
    x = np.concatenate([x, edges, rng.uniform(1.0, 2.0, 1 << 16)])
    r = np.empty_like(x)
    assert rlib.recip_many(x.ctypes.data, r.ctypes.data, x.size) == 0
    exact = 1.0 / x
    ulps = np.abs(r - exact) / np.spacing(exact)
    assert np.all(np.isfinite(r))
    assert ulps.max() <= 1.0, (ulps.max(), x[np.argmax(ulps)])
