"""Pins of the oracle's ode12 update (Sec. 4.3: the explicit Euler / Heun pair,
with the same step-size control, stress-driven error measure and tangent ODE
of Corollary 1 as ode23).

None of these re-types the oracle's arithmetic: one substep is checked
against Heun's method applied by hand to the linear (n = 1) ODE, whose
right-hand side is assembled here from the elastic constants; the adaptive
integration against the exact solution of that ODE (matrix exponential) and
against scipy's DOP853 for n > 1 and for the Michel-Suquet law; the tangent
against central differences of the ODE solution; the control exponent 1/2
through the growth of the substep count with the tolerance."""
import numpy as np
import pytest
import scipy.linalg

import oracle as O
import synth
from test_oracle_ode23 import P5, Z6, _linear_exact, _ms_reference, _reference

PRM = synth.MATRIX_16
MS = synth.ALUMINIUM_MS


def _linear_rhs(prm, eps_n, eps, h):
    """n = 1: ydot = -M y + b0 + b1 t (the Maxwell case of the force-potential
    form, M = (edot0/sigma0) G^-1 P^T C P)."""
    E, nu, s0, e0 = prm[:4]
    lam, mu = O.lame(E, nu)
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[:3, :3] += 2 * mu * np.eye(3)
    C[3:, 3:] = mu * np.eye(3)
    Pm, Gi = O.P_MATRIX, np.linalg.inv(O.G_MATRIX)
    M = e0 / s0 * Gi @ Pm.T @ C @ Pm
    B = e0 / s0 * Gi @ Pm.T @ C
    b0, b1 = B @ eps_n, B @ (eps - eps_n) / h
    return lambda t, y: -M @ y + b0 + b1 * t, C


def test_one_substep_is_heun():
    """With tolerances no error can exceed, the whole load step is one accepted
    substep: y_1 = y_0 + h/2 (f(0, y_0) + f(h, y_0 + h f(0, y_0))), sigma =
    C (eps - P y_1)."""
    prm = PRM[:4] + (1.0,)
    eps_n, eps, zn = synth.ode23_batch(20, seed=31)
    h = 0.1
    sig, z, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e30, atol=1e30, info=True, method="ode12")
    assert np.all(inf[:, 0] == 1) and np.all(inf[:, 1] == 0) and np.all(inf[:, 2] == 1)
    for i in range(20):
        f, C = _linear_rhs(prm, eps_n[i], eps[i], h)
        y0 = P5(zn[i])
        k1 = f(0.0, y0)
        y1 = y0 + 0.5 * h * (k1 + f(h, y0 + h * k1))
        assert np.allclose(z[i], Z6(y1), rtol=1e-12, atol=1e-16)
        assert np.allclose(sig[i], C @ (eps[i] - Z6(y1)), rtol=1e-11, atol=1e-14)


def test_linear_case_matches_the_exact_solution():
    """n = 1: ode12 at rtol 1e-8 equals the exact ODE solution to 1e-6 of the
    flow (its Heun solution is one order better than the Euler error it
    controls); its tangent the exact (affine) derivative to 1e-5."""
    prm = PRM[:4] + (1.0,)
    eps_n, eps, zn = synth.ode23_batch(16, seed=5)
    h = 0.1
    sig, z, C, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-8, atol=1e-12, tangent=True, info=True,
                                    method="ode12")
    assert np.all(inf[:, 2] == 1)
    for i in range(16):
        ze = _linear_exact(prm, eps_n[i], eps[i], zn[i], h)
        assert np.max(np.abs(z[i] - ze)) <= 1e-6 * np.max(np.abs(ze - zn[i])) + 1e-15
        _, Cel = _linear_rhs(prm, eps_n[i], eps[i], h)
        dz = np.zeros((6, 6))
        for k in range(6):
            e1 = eps[i].copy()
            e1[k] += 1.0
            dz[:, k] = _linear_exact(prm, eps_n[i], e1, zn[i], h) - ze
        Ct = Cel @ (np.eye(6) - dz)
        assert np.max(np.abs(C[i] - Ct)) <= 1e-5 * np.max(np.abs(Ct))


@pytest.mark.parametrize("n_exp", [3.0, 5.0, 10.0])
def test_nonlinear_case_matches_dop853(n_exp):
    """n > 1: ode12 at rtol 1e-8 against DOP853 at 1e-13; at MATLAB's default
    tolerances the stress stays within a small multiple of the tolerance."""
    prm = PRM[:4] + (n_exp,)
    eps_n, eps, zn = synth.ode23_batch(8, seed=int(n_exp) + 50)
    h = 0.1
    sig_t, z_t, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-8, atol=1e-12, info=True, method="ode12")
    sig_d, z_d, inf_d = O.update_ode23(prm, eps_n, eps, zn, h, info=True, method="ode12")
    assert np.all(inf[:, 2] == 1) and np.all(inf_d[:, 2] == 1)
    for i in range(8):
        zr = _reference(prm, eps_n[i], eps[i], zn[i], h)
        sr = O.stress(prm, eps[i], P5(zr))
        assert np.max(np.abs(z_t[i] - zr)) <= 1e-6 * np.max(np.abs(zr - zn[i])) + 1e-14
        assert np.max(np.abs(sig_d[i] - sr)) <= 20 * (1e-3 * np.max(np.abs(sr)) + 1e-6)


def test_tangent_matches_differences_of_the_ode_solution():
    """Corollary 1 for the Euler/Heun pair: the integrated tangent against central
    differences of the ODE solution."""
    eps_n, eps, zn = synth.ode23_batch(3, seed=19)
    h = 0.1
    # (rtol 1e-6: the pair's O(dt^2) estimate needs ~10^4 substeps here already)
    sig, z, C, inf = O.update_ode23(PRM, eps_n, eps, zn, h, rtol=1e-6, atol=1e-10, tangent=True, info=True,
                                    method="ode12")
    assert np.all(inf[:, 2] == 1)
    for i in range(3):
        Cfd = np.zeros((6, 6))
        for k in range(6):
            ep, em = eps[i].copy(), eps[i].copy()
            ep[k] += 1e-6
            em[k] -= 1e-6
            sp = O.stress(PRM, ep, P5(_reference(PRM, eps_n[i], ep, zn[i], h)))
            sm = O.stress(PRM, em, P5(_reference(PRM, eps_n[i], em, zn[i], h)))
            Cfd[:, k] = (sp - sm) / 2e-6
        assert np.max(np.abs(C[i] - Cfd)) <= 1e-5 * np.max(np.abs(Cfd))


def test_control_exponent_is_one_half():
    """The local error estimate of the pair is O(dt^2): a hundredfold smaller
    tolerance takes about tenfold the substeps (ode23's O(dt^3) estimate: about
    4.6-fold)."""
    eps_n, eps, zn = synth.ode23_batch(64, seed=23)
    n12 = [O.update_ode23(PRM, eps_n, eps, zn, 0.1, rtol=r, atol=r * 1e-3, info=True, method="ode12")[-1][:, 0].sum()
           for r in (1e-5, 1e-7)]
    n23 = [O.update_ode23(PRM, eps_n, eps, zn, 0.1, rtol=r, atol=r * 1e-3, info=True)[-1][:, 0].sum()
           for r in (1e-5, 1e-7)]
    assert 7.0 < n12[1] / n12[0] < 13.0
    assert 3.0 < n23[1] / n23[0] < 6.5


def test_michel_suquet_matches_dop853():
    eps_n, eps, zn = synth.ode23_batch(4, seed=29)
    h = 0.1
    sig, z, a, inf = O.update_ode23(MS, eps_n, eps, zn, h, rtol=1e-8, atol=1e-12, info=True,
                                    kind=O.KIND_MICHEL_SUQUET, method="ode12")
    assert np.all(inf[:, 2] == 1)
    for i in range(4):
        zr, ar = _ms_reference(MS, eps_n[i], eps[i], zn[i], h)
        assert np.max(np.abs(z[i] - zr)) <= 1e-6 * np.max(np.abs(zr - zn[i])) + 1e-14
        assert abs(a[i] - ar) <= 1e-6 * ar + 1e-14


def test_no_flow_and_stress_free_state():
    prm = (70.0, 0.3, 1e30, 1.0, 5.0)
    eps_n, eps, zn = synth.ode23_batch(6, seed=2)
    sig, z = O.update_ode23(prm, eps_n, eps, zn, 0.1, method="ode12")
    assert np.array_equal(z, zn)
    z0 = np.zeros((1, 6))
    sig, z, inf = O.update_ode23(PRM, z0, z0, z0, 0.1, info=True, method="ode12")
    assert np.all(sig == 0.0) and np.all(z == 0.0) and inf[0, 0] == 1 and inf[0, 1] == 0
