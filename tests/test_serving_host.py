"""Host-side logic of the serving driver (no GPU)."""
import numpy as np

from paper_2006_04391_gb300 import serving


def test_fifo_completion_recursion():
    a = np.array([0.0, 1.0, 1.5, 10.0])
    s = np.array([2.0, 1.0, 1.0, 0.5])
    c = serving.fifo_completion(a, s)
    assert np.allclose(c, [2.0, 3.0, 4.0, 10.5])
    # arrival order need not be sorted
    perm = [2, 0, 3, 1]
    c2 = serving.fifo_completion(a[perm], s[perm])
    assert np.allclose(c2, c[perm])


def test_poisson_arrivals_rate_and_determinism():
    t = serving.poisson_arrivals(20000, rate=4.0, seed=1)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert abs(np.mean(np.diff(t)) - 0.25) < 0.01
    assert np.array_equal(t, serving.poisson_arrivals(20000, rate=4.0, seed=1))


def test_percentiles():
    p = serving.percentiles(np.arange(101))
    assert p["p50"] == 50.0 and p["p99"] == 99.0
