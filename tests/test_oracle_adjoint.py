"""Pin of the oracle's discrete adjoint of the load history: central finite
differences (step 1e-6 relative) of J = w . Sigma_K through tightly converged
forward solves."""
import numpy as np

import oracle as O
import oracle.ms as MS
import synth


def J_of(ph, prm, w, loads, hs):
    laws = [(O.KIND_NORTON, prm), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    r = MS.solve(ph, laws, loads, hs, tol=1e-13, max_iter=20000)
    return float(w @ r["Sigma"][-1])


def test_adjoint_matches_central_differences():
    N = 6
    ph = synth.sphere_phase(N, 0.2)
    prm = (70.0, 0.3, 0.1, 1.0, 5.0)
    laws = [(O.KIND_NORTON, prm), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    loads = synth.ramp(2, [0.004, -0.001, 0.0, 0.0, 0.0, 0.003])
    hs = [0.1, 0.1]
    w = np.array([1.0, -0.3, 0.2, 0.1, 0.4, -0.5])
    r = MS.solve_taped(ph, laws, loads, hs, tol=1e-13)
    grad, _ = MS.adjoint(ph, laws, loads, hs, r["tape"], w, 0, tol=1e-13)
    fd = np.zeros(3)
    for i, pos in enumerate([0, 2, 4]):          # E, sigma0, n
        d = 1e-6 * prm[pos]
        pp, pm = list(prm), list(prm)
        pp[pos] += d
        pm[pos] -= d
        fd[i] = (J_of(ph, tuple(pp), w, loads, hs) - J_of(ph, tuple(pm), w, loads, hs)) / (2 * d)
    assert np.all(np.abs(grad - fd) <= 1e-5 * np.abs(fd) + 1e-9), (grad, fd)
