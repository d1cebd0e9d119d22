"""Pins of the oracle's ode23s update (Sec. 4.3: the Rosenbrock triple of
Shampine and Reichelt behind MATLAB's ode23s, with the paper's step control,
stress-driven error measure and the tangent by differentiating the stage
equations, Corollary 1 / Eq. rosenbrock_combined_update).

The third derivative of the force potential (the hand partial that the
Rosenbrock tangent needs) is pinned against central differences of the
already pinned Hessian; one substep against the Rosenbrock formulas applied by
hand to the linear (n = 1) ODE; the adaptive result against the exact
solution, DOP853 and central differences of the ODE solution; L-stability
through the substep count on a stiff step."""
import numpy as np
import pytest

import oracle as O
import synth
from test_oracle_ode12 import _linear_rhs
from test_oracle_ode23 import P5, Z6, _linear_exact, _ms_reference, _reference

PRM = synth.MATRIX_16
MS = synth.ALUMINIUM_MS


@pytest.mark.parametrize("n_exp", [1.0, 2.0, 5.0, 10.0])
def test_norton_third_derivative_matches_differences(n_exp):
    prm = PRM[:4] + (n_exp,)
    rng = np.random.default_rng(int(n_exp) + 3)
    for _ in range(10):
        A, u, v = rng.normal(size=(3, 5)) * 0.1
        out = O.psi_force_aaa(prm, A, u, v)
        d = 1e-6
        Hp = O.psi_force_a(prm, A + d * u)[1]
        Hm = O.psi_force_a(prm, A - d * u)[1]
        fd = (Hp - Hm) @ v / (2 * d)
        # (rounding of the differences: ~1e-10 |H v|; n = 1 has Psi_AAA = 0)
        noise = 1e-8 * np.abs(O.psi_force_a(prm, A)[1] @ v).max()
        assert np.allclose(out, fd, rtol=1e-6, atol=noise + 1e-7 * np.abs(fd).max())
        # symmetric in its two directions
        assert np.allclose(out, O.psi_force_aaa(prm, A, v, u), rtol=1e-12, atol=1e-6 * noise)


def test_michel_suquet_third_derivative_matches_differences():
    rng = np.random.default_rng(11)
    k = 0
    while k < 12:
        A = rng.normal(size=6) * 0.08
        A[5] = -MS[2]
        u, v = rng.normal(size=(2, 6)) * 0.05
        g, H = O.psi_force_ms(MS, A)[1:]
        if g[5] <= 0.0:   # inside the elastic domain: everything vanishes
            assert np.all(O.psi_force_aaa(MS, A, u, v, kind=O.KIND_MICHEL_SUQUET) == 0.0)
            continue
        d = 1e-7
        fd = (O.psi_force_ms(MS, A + d * u)[2] - O.psi_force_ms(MS, A - d * u)[2]) @ v / (2 * d)
        out = O.psi_force_aaa(MS, A, u, v, kind=O.KIND_MICHEL_SUQUET)
        assert np.allclose(out, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
        k += 1


def test_one_substep_is_the_rosenbrock_triple():
    """Tolerances no error can exceed: one substep over the whole step, equal to
    W = I - h d J, k1 = W^-1 (f0 + h d T), k2 = W^-1 (f(h/2, y0 + h/2 k1) - k1)
    + k1, y1 = y0 + h k2 applied by hand to ydot = -M y + b0 + b1 t."""
    prm = PRM[:4] + (1.0,)
    eps_n, eps, zn = synth.ode23_batch(12, seed=41)
    h = 0.1
    sig, z, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e30, atol=1e30, info=True, method="ode23s")
    assert np.all(inf[:, 0] == 1) and np.all(inf[:, 1] == 0)
    d = 1.0 / (2.0 + np.sqrt(2.0))
    for i in range(12):
        f, C = _linear_rhs(prm, eps_n[i], eps[i], h)
        y0 = P5(zn[i])
        Jm = np.stack([f(0.0, y0 + e) - f(0.0, y0) for e in np.eye(5)], axis=1)  # affine: exact
        T = f(1.0, y0) - f(0.0, y0)
        W = np.eye(5) - h * d * Jm
        k1 = np.linalg.solve(W, f(0.0, y0) + h * d * T)
        k2 = np.linalg.solve(W, f(h / 2, y0 + h / 2 * k1) - k1) + k1
        y1 = y0 + h * k2
        assert np.allclose(z[i], Z6(y1), rtol=1e-11, atol=1e-16)
        assert np.allclose(sig[i], C @ (eps[i] - Z6(y1)), rtol=1e-10, atol=1e-14)


def test_linear_case_matches_the_exact_solution():
    prm = PRM[:4] + (1.0,)
    eps_n, eps, zn = synth.ode23_batch(16, seed=43)
    h = 0.1
    sig, z, C, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-9, atol=1e-13, tangent=True, info=True,
                                    method="ode23s")
    assert np.all(inf[:, 2] == 1)
    for i in range(16):
        ze = _linear_exact(prm, eps_n[i], eps[i], zn[i], h)
        assert np.max(np.abs(z[i] - ze)) <= 1e-7 * np.max(np.abs(ze - zn[i])) + 1e-15
        _, Cel = _linear_rhs(prm, eps_n[i], eps[i], h)
        dz = np.zeros((6, 6))
        for k in range(6):
            e1 = eps[i].copy()
            e1[k] += 1.0
            dz[:, k] = _linear_exact(prm, eps_n[i], e1, zn[i], h) - ze
        Ct = Cel @ (np.eye(6) - dz)
        assert np.max(np.abs(C[i] - Ct)) <= 1e-6 * np.max(np.abs(Ct))


@pytest.mark.parametrize("n_exp", [3.0, 5.0, 10.0])
def test_nonlinear_case_matches_dop853(n_exp):
    prm = PRM[:4] + (n_exp,)
    eps_n, eps, zn = synth.ode23_batch(8, seed=int(n_exp) + 90)
    h = 0.1
    sig_t, z_t, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-9, atol=1e-13, info=True, method="ode23s")
    sig_d, z_d, inf_d = O.update_ode23(prm, eps_n, eps, zn, h, info=True, method="ode23s")
    assert np.all(inf[:, 2] == 1) and np.all(inf_d[:, 2] == 1)
    for i in range(8):
        zr = _reference(prm, eps_n[i], eps[i], zn[i], h)
        sr = O.stress(prm, eps[i], P5(zr))
        # (the triple continues with its order-2 solution: the controlled error is its own)
        assert np.max(np.abs(z_t[i] - zr)) <= 1e-6 * np.max(np.abs(zr - zn[i])) + 1e-14
        assert np.max(np.abs(sig_d[i] - sr)) <= 20 * (1e-3 * np.max(np.abs(sr)) + 1e-6)


@pytest.mark.parametrize("kind", [O.KIND_NORTON, O.KIND_MICHEL_SUQUET])
def test_tangent_matches_differences_of_the_ode_solution(kind):
    """Corollary 1 for the Rosenbrock stages (with the hand third derivative):
    the integrated tangent against central differences of the ODE solution."""
    prm = PRM if kind == O.KIND_NORTON else MS
    eps_n, eps, zn = synth.ode23_batch(3, seed=47)
    h = 0.1
    out = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-9, atol=1e-13, tangent=True, info=True, kind=kind,
                         method="ode23s")
    C, inf = out[-2], out[-1]
    assert np.all(inf[:, 2] == 1)
    pe = prm if kind == O.KIND_NORTON else MS[:2] + (1.0, 1.0, 1.0)
    for i in range(3):
        Cfd = np.zeros((6, 6))
        for k in range(6):
            ep, em = eps[i].copy(), eps[i].copy()
            ep[k] += 1e-6
            em[k] -= 1e-6
            if kind == O.KIND_NORTON:
                zp, zm = _reference(prm, eps_n[i], ep, zn[i], h), _reference(prm, eps_n[i], em, zn[i], h)
            else:
                zp, zm = _ms_reference(prm, eps_n[i], ep, zn[i], h)[0], _ms_reference(prm, eps_n[i], em, zn[i], h)[0]
            Cfd[:, k] = (O.stress(pe, ep, P5(zp)) - O.stress(pe, em, P5(zm))) / 2e-6
        assert np.max(np.abs(C[i] - Cfd)) <= 1e-6 * np.max(np.abs(Cfd))


def test_michel_suquet_matches_dop853():
    eps_n, eps, zn = synth.ode23_batch(4, seed=53)
    sig, z, a, inf = O.update_ode23(MS, eps_n, eps, zn, 0.1, rtol=1e-9, atol=1e-13, info=True,
                                    kind=O.KIND_MICHEL_SUQUET, method="ode23s")
    assert np.all(inf[:, 2] == 1)
    for i in range(4):
        zr, ar = _ms_reference(MS, eps_n[i], eps[i], zn[i], 0.1)
        assert np.max(np.abs(z[i] - zr)) <= 1e-6 * np.max(np.abs(zr - zn[i])) + 1e-14
        assert abs(a[i] - ar) <= 1e-6 * ar + 1e-14


def test_stiff_step_needs_few_substeps():
    """A deviatoric strain ramp of amplitude 0.05 over h = 10 from the virgin
    state: after the initial transient the flow is quasi-steady and the
    evolution ODE stiff (|lambda| h >> 1); the explicit pair is held back by
    stability, the linearly implicit Rosenbrock triple is not; both meet the
    tolerance."""
    rng = np.random.default_rng(0)
    n = 16
    d = rng.normal(size=(n, 6))
    d[:, :3] -= d[:, :3].mean(1, keepdims=True)
    eps = 0.05 * d / np.abs(d).max(1, keepdims=True)
    zero = np.zeros((n, 6))
    s23, z23, i23 = O.update_ode23(PRM, zero, eps, zero, 10.0, info=True)
    s3s, z3s, i3s = O.update_ode23(PRM, zero, eps, zero, 10.0, info=True, method="ode23s")
    assert np.all(i23[:, 2] == 1) and np.all(i3s[:, 2] == 1)
    assert (i3s[:, 0] + i3s[:, 1]).sum() * 5 < (i23[:, 0] + i23[:, 1]).sum()
    assert np.all(np.abs(s3s - s23) <= 20 * (1e-3 * np.abs(s23).max(1, keepdims=True) + 1e-6))
