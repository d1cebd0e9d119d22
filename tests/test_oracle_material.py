"""Pins of the FP64 oracle's material law against things other than itself.

Every expected value here comes from a closed form, a finite difference, the
paper's own force-potential form of the evolution law, or an invariant --
never from re-typing the oracle's formula.  Paper: AutoMat, arXiv 2006.04391.
"""
import numpy as np
import pytest

import oracle as O
import synth

PRM = synth.MATRIX_16          # (E, nu, sigma0, edot0, n) = (70, 0.3, 0.1, 1, 5)
H = 0.01


def compliance_stiffness(E, nu):
    """C = S^-1 from the engineering compliance (1/E, -nu/E, 2(1+nu)/E)."""
    S = np.zeros((6, 6))
    S[:3, :3] = -nu / E
    np.fill_diagonal(S[:3, :3], 1.0 / E)
    S[3:, 3:] = np.eye(3) * 2.0 * (1.0 + nu) / E
    return np.linalg.inv(S)


def to_tensor(v, engineering):
    f = 0.5 if engineering else 1.0
    return np.array([[v[0], f * v[5], f * v[4]],
                     [f * v[5], v[1], f * v[3]],
                     [f * v[4], f * v[3], v[2]]])


def to_voigt(T, engineering):
    f = 2.0 if engineering else 1.0
    return np.array([T[0, 0], T[1, 1], T[2, 2], f * T[1, 2], f * T[0, 2], f * T[0, 1]])


def y_of(z):
    return np.array([z[0], z[1], z[3], z[4], z[5]])


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module")
def batch():
    eps, zn = synth.material_batch(4000, seed=11)
    return eps, zn


def test_elastic_law_is_hooke_from_compliance():
    """Elastic phase: sigma = C eps with C the inverse of the textbook compliance."""
    eps, zn = synth.material_batch(50, seed=1)
    sig, z, Ct = O.update(O.KIND_ELASTIC, (400.0, 0.2), eps, zn, 0.1, tangent=True)
    C = compliance_stiffness(400.0, 0.2)
    assert rel(sig, eps @ C.T) < 1e-14
    assert rel(Ct, np.broadcast_to(C, Ct.shape)) < 1e-14
    assert np.array_equal(z, zn)


def test_stress_is_gradient_of_free_energy():
    """Eq. gsm_sigma: sigma = d psi/d eps, central differences on psi."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        eps = rng.uniform(-0.02, 0.02, 6)
        y = rng.uniform(-0.005, 0.005, 5)
        sig = O.stress(PRM, eps, y)
        fd = np.zeros(6)
        for i in range(6):
            d = 1e-6 * max(1.0, abs(eps[i]))
            ep, em = eps.copy(), eps.copy()
            ep[i] += d
            em[i] -= d
            fd[i] = (O.psi(PRM, ep, y) - O.psi(PRM, em, y)) / (2 * d)
        assert rel(fd, sig) < 1e-7


def test_potential_derivatives_by_finite_differences():
    """psi_y, psi_yy, phi_v, phi_vv against central differences (step 1e-6 relative)."""
    rng = np.random.default_rng(4)
    for n in (1.0, 3.0, 5.0, 10.0):
        prm = PRM[:4] + (n,)
        eps = rng.uniform(-0.02, 0.02, 6)
        y = rng.uniform(-0.005, 0.005, 5)
        v = rng.uniform(-1.0, 1.0, 5)
        g = O.psi_y(prm, eps, y)
        Hy = O.psi_yy(prm)
        gv = O.phi_v(prm, v)
        Hv = O.phi_vv(prm, v)
        fd_g, fd_H, fd_gv, fd_Hv = np.zeros(5), np.zeros((5, 5)), np.zeros(5), np.zeros((5, 5))
        for a in range(5):
            dy = 1e-6
            yp, ym = y.copy(), y.copy()
            yp[a] += dy
            ym[a] -= dy
            fd_g[a] = (O.psi(prm, eps, yp) - O.psi(prm, eps, ym)) / (2 * dy)
            fd_H[:, a] = (O.psi_y(prm, eps, yp) - O.psi_y(prm, eps, ym)) / (2 * dy)
            dv = 1e-6 * max(1.0, abs(v[a]))
            vp, vm = v.copy(), v.copy()
            vp[a] += dv
            vm[a] -= dv
            fd_gv[a] = (O.phi(prm, vp) - O.phi(prm, vm)) / (2 * dv)
            fd_Hv[:, a] = (O.phi_v(prm, vp) - O.phi_v(prm, vm)) / (2 * dv)
        assert rel(fd_g, g) < 1e-7
        assert rel(fd_H, Hy) < 1e-7
        assert rel(fd_gv, gv) < 1e-7
        assert rel(fd_Hv, Hv) < 1e-7


def test_equivalent_rate_norm_is_von_mises_rate():
    """phi uses s = sqrt(2/3 zdot:zdot) (engineering shears halved in the tensor)."""
    rng = np.random.default_rng(5)
    prm = PRM[:4] + (1.0,)     # n = 1: phi = sigma0/edot0 * s^2 / 2
    for _ in range(5):
        v = rng.uniform(-1, 1, 5)
        zd = np.array([v[0], v[1], -v[0] - v[1], v[2], v[3], v[4]])
        T = to_tensor(zd, engineering=True)
        s = np.sqrt(2.0 / 3.0 * np.sum(T * T))
        assert abs(O.phi(prm, v) - 0.1 * s * s / 2.0) < 1e-14 * max(1.0, s * s)


def test_generic_newton_equals_radial_return(batch):
    """Sec. 4.1: all strategies agree to machine precision -- the generic
    5-unknown Newton equals the conventional scalar radial return."""
    eps, zn = batch
    for n in (1.0, 3.0, 5.0, 10.0):
        prm = PRM[:4] + (n,)
        for h in (1e-3, 1e-2, 1e-1):
            s1, z1, inf = O.update(O.KIND_NORTON, prm, eps, zn, h, info=True)
            s2, z2 = O.radial_return(prm, eps, zn, h)
            assert np.all(inf[:, 2] & 1), "all voxels converged"
            # per-voxel normwise relative error
            es = np.max(np.abs(s1 - s2), axis=1) / np.max(np.abs(s2), axis=1)
            ez = np.max(np.abs(z1 - z2), axis=1) / np.max(np.abs(z2), axis=1)
            assert es.max() < 1e-12, (n, h, es.max())
            assert ez.max() < 1e-12, (n, h, ez.max())


def test_maxwell_closed_form(batch):
    """n = 1 (linear Norton): z = (z_n + beta dev eps)/(1 + beta), beta = 3 mu h edot0/sigma0."""
    eps, zn = batch
    prm = PRM[:4] + (1.0,)
    E, nu = prm[0], prm[1]
    mu = E / (2 * (1 + nu))
    for h in (1e-3, 0.1, 3.0):
        beta = 3 * mu * h * prm[3] / prm[2]
        dev = eps.copy()
        dev[:, :3] -= eps[:, :3].sum(axis=1, keepdims=True) / 3.0
        z_exact = (zn + beta * dev) / (1 + beta)
        sig, z = O.update(O.KIND_NORTON, prm, eps, zn, h)
        assert rel(z, z_exact) < 1e-13
        C = compliance_stiffness(E, nu)
        assert rel(sig, (eps - z_exact) @ C.T) < 1e-12


def test_update_satisfies_the_papers_force_potential_form(batch):
    """Eq. gsm_internal + Eq. implicit_euler in the paper's own variables:
    (z - z_n)/h = dPsi/dA(A) at A = -d omega/d eps_vp = sigma, with Psi of
    Eq. michel_suquet_psi at sigma_Y = 0, H = 0 (written here in tensor form)."""
    eps, zn = batch
    for n in (3.0, 5.0, 10.0):
        prm = PRM[:4] + (n,)
        sigma_d, edot0 = prm[2], prm[3]
        sig, z = O.update(O.KIND_NORTON, prm, eps[:500], zn[:500], H)
        for i in range(500):
            A = to_tensor(sig[i], engineering=False)
            devA = A - np.trace(A) / 3.0 * np.eye(3)
            seq = np.sqrt(1.5 * np.sum(devA * devA))
            dPsi = edot0 * (seq / sigma_d) ** n * 1.5 * devA / seq
            lhs = to_tensor((z[i] - zn[i]) / H, engineering=True)
            assert np.max(np.abs(lhs - dPsi)) <= 1e-10 * np.max(np.abs(dPsi))


def test_linear_elastic_limits():
    """sigma0 -> infinity or h -> 0: no viscoplastic flow, sigma = C (eps - z_n)."""
    eps, zn = synth.material_batch(200, seed=7)
    C = compliance_stiffness(70.0, 0.3)
    s, z = O.update(O.KIND_NORTON, (70.0, 0.3, 1e12, 1.0, 5.0), eps, zn, 0.01)
    assert rel(s, (eps - zn) @ C.T) < 1e-12
    s, z = O.update(O.KIND_NORTON, PRM, eps, zn, 1e-30)
    assert rel(s, (eps - zn) @ C.T) < 1e-12


def test_newton_matrix_spd_and_tangent_symmetric_positive(batch):
    """Theorem 1 (Sec. 2): with convex potentials the Newton matrix K is SPD;
    the consistent tangent is symmetric positive definite."""
    eps, zn = batch
    sig, z, Ct = O.update(O.KIND_NORTON, PRM, eps[:300], zn[:300], H, tangent=True)
    for i in range(300):
        y, yn = y_of(z[i]), y_of(zn[i])
        K = O.newton_matrix(PRM, y, yn, H)
        assert np.all(np.linalg.eigvalsh(K) > 0)
        assert np.max(np.abs(Ct[i] - Ct[i].T)) <= 1e-12 * np.max(np.abs(Ct[i]))
        assert np.all(np.linalg.eigvalsh(0.5 * (Ct[i] + Ct[i].T)) > 0)


def test_tangent_by_finite_differences_and_identity(batch):
    """Eq. tangent_formula vs central differences of the whole update, and the
    paper's identity C_t = C^el (I - d eps_vp / d eps) (Sec. 4.3)."""
    eps, zn = batch
    C = compliance_stiffness(70.0, 0.3)
    for i in range(20):
        e0, z0 = eps[i], zn[i]
        _, _, Ct = O.update(O.KIND_NORTON, PRM, e0, z0, H, tangent=True)
        fd_s, fd_z = np.zeros((6, 6)), np.zeros((6, 6))
        for j in range(6):
            d = 1e-7
            ep, em = e0.copy(), e0.copy()
            ep[j] += d
            em[j] -= d
            sp, zp = O.update(O.KIND_NORTON, PRM, ep, z0, H)
            sm, zm = O.update(O.KIND_NORTON, PRM, em, z0, H)
            fd_s[:, j] = (sp[0] - sm[0]) / (2 * d)
            fd_z[:, j] = (zp[0] - zm[0]) / (2 * d)
        assert rel(fd_s, Ct[0]) < 1e-6
        assert rel(C @ (np.eye(6) - fd_z), Ct[0]) < 1e-6


def test_solution_minimises_incremental_potential(batch):
    """The converged y is the minimiser of Pi(y) = psi + h phi((y - y_n)/h)."""
    eps, zn = batch
    rng = np.random.default_rng(9)
    _, z = O.update(O.KIND_NORTON, PRM, eps[:50], zn[:50], H)
    for i in range(50):
        y, yn = y_of(z[i]), y_of(zn[i])
        R = O.residual(PRM, eps[i], y, yn, H)
        scale = np.max(np.abs(O.psi_y(PRM, eps[i], yn)))
        assert np.max(np.abs(R)) < 1e-11 * scale
        P0 = O.incremental_potential(PRM, eps[i], y, yn, H)
        for _ in range(5):
            dy = rng.normal(size=5) * 1e-5
            assert O.incremental_potential(PRM, eps[i], y + dy, yn, H) >= P0


def test_deviatoric_and_flags(batch):
    eps, zn = batch
    _, z, inf = O.update(O.KIND_NORTON, PRM, eps, zn, H, info=True)
    assert np.max(np.abs(z[:, 0] + z[:, 1] + z[:, 2])) < 1e-17
    assert np.all(inf[:, 2] == 1)


def test_stress_free_state_needs_no_iteration():
    """psi_y(eps, y_n) = 0 exactly (eps = z_n = 0): y = y_n, no iteration, C_t = C."""
    sig, z, Ct, inf = O.update(O.KIND_NORTON, PRM, np.zeros((1, 6)), np.zeros((1, 6)), H,
                               tangent=True, info=True)
    assert np.array_equal(z, np.zeros((1, 6))) and np.array_equal(sig, np.zeros((1, 6)))
    assert rel(Ct[0], compliance_stiffness(70.0, 0.3)) < 1e-14
    assert inf[0, 0] == 0 and inf[0, 1] == 0


def test_hydrostatic_strain_stays_elastic():
    """A hydrostatic strain has no deviatoric stress: no viscoplastic flow."""
    eps = np.array([[0.01, 0.01, 0.01, 0, 0, 0]])
    zn = np.zeros((1, 6))
    sig, z = O.update(O.KIND_NORTON, PRM, eps, zn, H)
    C = compliance_stiffness(70.0, 0.3)
    assert np.max(np.abs(z)) < 1e-30
    assert rel(sig[0], C @ eps[0]) < 1e-15


def test_nonfinite_input_is_flagged():
    eps = np.array([[np.nan, 0, 0, 0, 0, 0]])
    _, _, inf = O.update(O.KIND_NORTON, PRM, eps, np.zeros((1, 6)), H, info=True)
    assert inf[0, 2] & 2
