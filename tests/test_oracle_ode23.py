"""Pins of the oracle's ode23 update (force-potential form of Eq. gsm_internal
integrated by the Bogacki-Shampine pair with step-size control, Sec. 4.3;
tangent ODE of Corollary 1; stress-driven error measure, Sec. 4.5).

None of these re-types the oracle's formulas: the force potential is pinned
through duality with the (already pinned) dissipation potential phi; the
integrator against the exact solution of the linear case (n = 1, matrix
exponential from scipy) and against scipy's DOP853 at tight tolerance, with
the right-hand side assembled from oracle functions."""
import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle as O
import synth

PRM = synth.MATRIX_16  # (E, nu, sigma0, edot0, n)


def P5(z):
    return np.array([z[0], z[1], z[3], z[4], z[5]])


def Z6(y):
    return np.array([y[0], y[1], -y[0] - y[1], y[2], y[3], y[4]])


@pytest.mark.parametrize("n_exp", [1.0, 3.0, 5.0, 10.0])
def test_force_potential_is_the_dual_of_phi(n_exp):
    """phi_v(Psi_A(A)) = A and Psi_AA(A) = phi_vv(Psi_A(A))^-1 (Legendre duality);
    Psi_AA against central differences of Psi_A."""
    prm = PRM[:4] + (n_exp,)
    rng = np.random.default_rng(int(n_exp))
    for _ in range(20):
        A = rng.normal(size=5) * 0.1
        g, H = O.psi_force_a(prm, A)
        assert np.allclose(O.phi_v(prm, g), A, rtol=1e-12, atol=1e-14)
        assert np.allclose(H, np.linalg.inv(O.phi_vv(prm, g)), rtol=1e-9, atol=1e-14 * np.abs(H).max())
        for a in range(5):
            d = 1e-6 * max(1.0, abs(A[a]))
            Ap, Am = A.copy(), A.copy()
            Ap[a] += d
            Am[a] -= d
            fd = (O.psi_force_a(prm, Ap)[0] - O.psi_force_a(prm, Am)[0]) / (2 * d)
            assert np.allclose(fd, H[:, a], rtol=1e-6, atol=1e-8 * np.abs(H).max())
    g, H = O.psi_force_a(prm, np.zeros(5))
    assert np.all(g == 0.0)


def _linear_exact(prm, eps_n, eps, zn, h):
    """n = 1: ydot = -M y + b0 + b1 t with M = (edot0/sigma0) G^-1 P^T C P and
    b(t) = (edot0/sigma0) G^-1 P^T C eps(t); exact y(h) by the exponential of
    the augmented matrix [[-M, b1, b0], [0, 0, 1], [0, 0, 0]]."""
    E, nu, s0, e0 = prm[:4]
    lam, mu = O.lame(E, nu)
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[:3, :3] += 2 * mu * np.eye(3)
    C[3:, 3:] = mu * np.eye(3)
    Pm, Gi = O.P_MATRIX, np.linalg.inv(O.G_MATRIX)
    M = e0 / s0 * Gi @ Pm.T @ C @ Pm
    B = e0 / s0 * Gi @ Pm.T @ C
    b0 = B @ eps_n
    b1 = B @ (eps - eps_n) / h
    Aug = np.zeros((7, 7))
    Aug[:5, :5] = -M
    Aug[:5, 5] = b1
    Aug[:5, 6] = b0
    Aug[5, 6] = 1.0
    x = scipy.linalg.expm(Aug * h) @ np.concatenate([P5(zn), [0.0, 1.0]])
    return Z6(x[:5])


def test_linear_case_matches_the_exact_solution():
    """n = 1 (Maxwell): ode23 at tight tolerance equals the exact solution of the
    ODE (not of a time discretization) to 1e-9; its tangent equals the exact
    derivative (the exact map is affine in eps_{n+1})."""
    prm = PRM[:4] + (1.0,)
    eps_n, eps, zn = synth.ode23_batch(40, seed=3)
    h = 0.1
    sig, z, C, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-11, atol=1e-15, tangent=True, info=True)
    assert np.all(inf[:, 2] == 1)
    for i in range(40):
        ze = _linear_exact(prm, eps_n[i], eps[i], zn[i], h)
        assert np.max(np.abs(z[i] - ze)) <= 1e-9 * np.max(np.abs(ze - zn[i])) + 1e-15
        # tangent: d sigma/d eps = C (I - dz/deps), dz/deps from the affine exact map
        E, nu = prm[:2]
        Cel = np.linalg.inv(np.diag([1 / E] * 3 + [2 * (1 + nu) / E] * 3) + np.pad(
            np.full((3, 3), -nu / E) - np.diag([-nu / E] * 3), ((0, 3), (0, 3))))
        dz = np.zeros((6, 6))
        for k in range(6):
            e1 = eps[i].copy()
            e1[k] += 1.0
            dz[:, k] = _linear_exact(prm, eps_n[i], e1, zn[i], h) - ze
        Ct = Cel @ (np.eye(6) - dz)
        assert np.max(np.abs(C[i] - Ct)) <= 1e-8 * np.max(np.abs(Ct))


def _reference(prm, eps_n, eps, zn, h):
    """y(h) of the same ODE by scipy's DOP853 at rtol 1e-13, right-hand side from
    oracle functions: A = -psi_y(eps(t), y), f = Psi_A(A)."""
    def f(t, y):
        et = eps_n + (t / h) * (eps - eps_n)
        return O.psi_force_a(prm, -O.psi_y(prm, et, y))[0]
    r = scipy.integrate.solve_ivp(f, (0.0, h), P5(zn), method="DOP853", rtol=1e-13, atol=1e-16)
    assert r.success
    return Z6(r.y[:, -1])


@pytest.mark.parametrize("n_exp", [3.0, 5.0, 10.0])
def test_nonlinear_case_matches_dop853(n_exp):
    """n > 1: ode23 at rtol 1e-10 against DOP853 at 1e-13 (the ODE solution);
    at the default tolerances (rtol 1e-3, atol 1e-6) the stress error stays
    within a small multiple of the tolerance (stress-driven error control)."""
    prm = PRM[:4] + (n_exp,)
    eps_n, eps, zn = synth.ode23_batch(12, seed=int(n_exp))
    h = 0.1
    sig_t, z_t, inf = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-10, atol=1e-13, info=True)
    sig_d, z_d, inf_d = O.update_ode23(prm, eps_n, eps, zn, h, info=True)
    assert np.all(inf[:, 2] == 1) and np.all(inf_d[:, 2] == 1)
    for i in range(12):
        zr = _reference(prm, eps_n[i], eps[i], zn[i], h)
        sr = O.stress(prm, eps[i], P5(zr))
        assert np.max(np.abs(z_t[i] - zr)) <= 1e-8 * np.max(np.abs(zr - zn[i])) + 1e-14
        assert np.max(np.abs(sig_d[i] - sr)) <= 20 * (1e-3 * np.max(np.abs(sr)) + 1e-6)


def test_tangent_matches_differences_of_the_ode_solution():
    """Corollary 1: the tangent integrated with the primal (tight tolerance)
    equals central differences of the ODE solution y(h; eps_{n+1})."""
    prm = PRM
    eps_n, eps, zn = synth.ode23_batch(4, seed=9)
    h = 0.1
    sig, z, C = O.update_ode23(prm, eps_n, eps, zn, h, rtol=1e-10, atol=1e-13, tangent=True)
    for i in range(4):
        Cfd = np.zeros((6, 6))
        for k in range(6):
            d = 1e-6
            ep, em = eps[i].copy(), eps[i].copy()
            ep[k] += d
            em[k] -= d
            sp = O.stress(prm, ep, P5(_reference(prm, eps_n[i], ep, zn[i], h)))
            sm = O.stress(prm, em, P5(_reference(prm, eps_n[i], em, zn[i], h)))
            Cfd[:, k] = (sp - sm) / (2 * d)
        assert np.max(np.abs(C[i] - Cfd)) <= 1e-6 * np.max(np.abs(Cfd))


def test_no_flow_limits():
    """sigma0 -> large: no flow, z = z_n, sigma = C (eps - z_n), tangent = C.
    A stress-free state (eps = z_n = eps_n) stays stress free in one substep."""
    prm = (70.0, 0.3, 1e30, 1.0, 5.0)
    eps_n, eps, zn = synth.ode23_batch(10, seed=1)
    sig, z, C = O.update_ode23(prm, eps_n, eps, zn, 0.1, tangent=True)
    assert np.array_equal(z, zn)
    for i in range(10):
        assert np.allclose(sig[i], O.stress(prm, eps[i], P5(zn[i])), rtol=1e-15, atol=1e-18)
    lam, mu = O.lame(70.0, 0.3)
    Cel = np.zeros((6, 6))
    Cel[:3, :3] = lam
    Cel[:3, :3] += 2 * mu * np.eye(3)
    Cel[3:, 3:] = mu * np.eye(3)
    assert np.allclose(C, Cel[None], rtol=1e-14, atol=1e-12)
    z0 = np.zeros((1, 6))
    sig, z, inf = O.update_ode23(PRM, z0, z0, z0, 0.1, info=True)
    assert np.all(sig == 0.0) and np.all(z == 0.0) and inf[0, 0] == 1 and inf[0, 1] == 0


# ------------------------------------------------- Michel-Suquet law (kind 2)
MS = synth.ALUMINIUM_MS  # (E, nu, sigma_Y, H, edot0, sigma_d, n)


def _A_samples(rng, k):
    A = rng.normal(size=(k, 6)) * 0.05
    A[:, 5] = -MS[2]
    return A


def test_ms_force_potential_derivatives():
    """Psi_A and Psi_AA against central differences of Psi, outside and inside the
    elastic domain (there Psi and all its derivatives vanish)."""
    rng = np.random.default_rng(4)
    for A in _A_samples(rng, 30):
        v, g, H = O.psi_force_ms(MS, A)
        for a in range(6):
            d = 1e-7
            Ap, Am = A.copy(), A.copy()
            Ap[a] += d
            Am[a] -= d
            vp, gp, _ = O.psi_force_ms(MS, Ap)
            vm, gm, _ = O.psi_force_ms(MS, Am)
            assert abs((vp - vm) / (2 * d) - g[a]) <= 1e-6 * max(np.abs(g).max(), 1e-12)
            assert np.allclose((gp - gm) / (2 * d), H[:, a], rtol=1e-5, atol=1e-6 * max(np.abs(H).max(), 1e-12))
    inside = np.array([0.001, -0.002, 0.001, 0.0, 0.002, -MS[2]])  # von Mises well below sigma_Y
    v, g, H = O.psi_force_ms(MS, inside)
    assert v == 0.0 and np.all(g == 0.0) and np.all(H == 0.0)


def test_ms_reduces_to_norton_without_yield_and_hardening():
    """sigma_Y = 0, H = 0: the Michel-Suquet ODE is the Norton ODE with sigma0 = sigma_d."""
    ms = (70.0, 0.3, 0.0, 0.0, 1.0, 0.1, 5.0)
    en, e, zn = synth.ode23_batch(50, seed=2)
    sig1, z1, a1, C1, i1 = O.update_ode23(ms, en, e, zn, 0.1, tangent=True, info=True, kind=O.KIND_MICHEL_SUQUET)
    sig2, z2, C2, i2 = O.update_ode23(synth.MATRIX_16, en, e, zn, 0.1, tangent=True, info=True)
    assert np.array_equal(i1, i2)
    assert np.allclose(sig1, sig2, rtol=1e-13, atol=0) and np.allclose(z1, z2, rtol=1e-13, atol=1e-18)
    assert np.allclose(C1, C2, rtol=1e-12, atol=1e-10)


def test_ms_elastic_domain_and_accumulated_plastic_strain():
    """Inside the yield surface nothing flows; under radial loading of a virgin
    state alpha equals the equivalent viscoplastic strain sqrt(2/3 e_vp:e_vp)."""
    en = np.zeros((1, 6))
    e_small = np.array([[1e-4, -5e-5, -5e-5, 0, 0, 0]])
    sig, z, a = O.update_ode23(MS, en, e_small, np.zeros((1, 6)), 0.1, kind=O.KIND_MICHEL_SUQUET)
    assert np.all(z == 0.0) and a[0] == 0.0
    d = np.array([1.0, -0.5, -0.5, 0.0, 0.0, 0.0])  # deviatoric uniaxial-type direction
    sig, z, a = O.update_ode23(MS, en, 0.004 * d[None], np.zeros((1, 6)), 0.1, rtol=1e-11, atol=1e-14,
                               kind=O.KIND_MICHEL_SUQUET)
    T = np.array([[z[0, 0], z[0, 5] / 2, z[0, 4] / 2], [z[0, 5] / 2, z[0, 1], z[0, 3] / 2],
                  [z[0, 4] / 2, z[0, 3] / 2, z[0, 2]]])
    eq = np.sqrt(2.0 / 3.0 * np.sum(T * T))
    assert a[0] > 0 and abs(a[0] - eq) <= 1e-8 * eq


def _ms_reference(prm, eps_n, eps, zn, h):
    """The Michel-Suquet ODE by scipy's DOP853 at rtol 1e-13, right-hand side from
    oracle functions: A = gen_stress_ms(eps(t), y, alpha), f = Psi_A(A)."""
    def f(t, y):
        et = eps_n + (t / h) * (eps - eps_n)
        return O.psi_force_ms(prm, O.gen_stress_ms(prm, et, y))[1]
    y0 = np.concatenate([P5(zn), [0.0]])
    r = scipy.integrate.solve_ivp(f, (0.0, h), y0, method="DOP853", rtol=1e-13, atol=1e-16)
    assert r.success
    return Z6(r.y[:5, -1]), r.y[5, -1]


def test_ms_matches_dop853_and_its_tangent():
    eps_n, eps, zn = synth.ode23_batch(6, seed=13)
    h = 0.1
    sig, z, a, C = O.update_ode23(MS, eps_n, eps, zn, h, rtol=1e-10, atol=1e-13, tangent=True,
                                  kind=O.KIND_MICHEL_SUQUET)
    for i in range(6):
        zr, ar = _ms_reference(MS, eps_n[i], eps[i], zn[i], h)
        assert np.max(np.abs(z[i] - zr)) <= 1e-8 * np.max(np.abs(zr - zn[i])) + 1e-14
        assert abs(a[i] - ar) <= 1e-8 * ar + 1e-14
    Cfd = np.zeros((6, 6))
    for k in range(6):
        ep, em = eps[0].copy(), eps[0].copy()
        ep[k] += 1e-6
        em[k] -= 1e-6
        sp = O.stress(MS[:2] + (1.0, 1.0, 1.0), ep, P5(_ms_reference(MS, eps_n[0], ep, zn[0], h)[0]))
        sm = O.stress(MS[:2] + (1.0, 1.0, 1.0), em, P5(_ms_reference(MS, eps_n[0], em, zn[0], h)[0]))
        Cfd[:, k] = (sp - sm) / 2e-6
    assert np.max(np.abs(C[0] - Cfd)) <= 1e-6 * np.max(np.abs(Cfd))
