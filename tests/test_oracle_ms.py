"""Pins of the FP64 basic-scheme oracle (Moulinec-Suquet, cited in Sec. 1/3).

Expected values come from the closed-form laminate, the defining properties
of the Green operator (projection onto compatible fields), symmetry, and the
single-voxel law -- never from the oracle itself.
"""
import numpy as np
import pytest

import oracle as O
import oracle.ms as MS
import synth

VOIGT = MS.VOIGT


def stiffness(E, nu):
    S = np.zeros((6, 6))
    S[:3, :3] = -nu / E
    np.fill_diagonal(S[:3, :3], 1.0 / E)
    S[3:, 3:] = np.eye(3) * 2.0 * (1.0 + nu) / E
    return np.linalg.inv(S)


def sym_grad_voigt(xi, u):
    """Engineering-Voigt components of sym(xi (x) u) (complex)."""
    e = 0.5 * (np.outer(xi, u) + np.outer(u, xi))
    return np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[0, 2], 2 * e[0, 1]])


def test_green_operator_reproduces_compatible_fields():
    """Gamma0 : (C0 : sym(xi (x) u)) = sym(xi (x) u) for every admissible mode."""
    N = 5
    lam0, mu0 = 80.0, 60.0
    C0 = np.zeros((6, 6))
    C0[:3, :3] = lam0
    C0[:3, :3] += np.eye(3) * 2 * mu0
    C0[3:, 3:] = np.eye(3) * mu0
    rng = np.random.default_rng(0)
    k, excl = MS.wavevectors(N)
    xi = 2 * np.pi * k
    eps_hat = np.zeros((N, N, N, 6), dtype=complex)
    for idx in np.ndindex(N, N, N):
        u = rng.normal(size=3) + 1j * rng.normal(size=3)
        eps_hat[idx] = sym_grad_voigt(xi[(slice(None),) + idx], u)
    eps_hat[0, 0, 0] = 0
    sig_hat = eps_hat @ C0.T
    tau = MS.voigt_to_tensor_field(sig_hat, engineering=False)
    back = MS.gamma0_apply(tau, lam0, mu0, N)
    assert np.max(np.abs(back - eps_hat)) < 1e-13 * np.max(np.abs(eps_hat))


def test_green_operator_output_is_compatible_and_equilibrating():
    """For any tau: Gamma0 tau is a symmetric gradient, and xi.(C0 Gamma0 tau) = xi.tau."""
    N = 4
    lam0, mu0 = 50.0, 30.0
    C0 = np.zeros((6, 6))
    C0[:3, :3] = lam0
    C0[:3, :3] += np.eye(3) * 2 * mu0
    C0[3:, 3:] = np.eye(3) * mu0
    rng = np.random.default_rng(1)
    t = rng.normal(size=(N, N, N, 6)) + 1j * rng.normal(size=(N, N, N, 6))
    tau = MS.voigt_to_tensor_field(t, engineering=False)
    d = MS.gamma0_apply(tau, lam0, mu0, N)
    k, excl = MS.wavevectors(N)
    xi = 2 * np.pi * k
    s = MS.voigt_to_tensor_field(d @ C0.T, engineering=False)
    lhs = np.einsum("ij...,j...->i...", s, xi)
    rhs = np.einsum("ij...,j...->i...", tau, xi)
    keep = ~excl
    keep[0, 0, 0] = False
    assert np.max(np.abs((lhs - rhs)[:, keep])) < 1e-12 * np.max(np.abs(rhs))
    # compatibility: the strain of a mode is sym(xi (x) u) with u = (d xi)/|xi|^2-style;
    # check the 2-D compatibility minors e_ij xi_k xi_l - ... via rank: eps = sym(xi u)
    # implies eps_ij xi_k xi_l + eps_kl xi_i xi_j - eps_ik xi_j xi_l - eps_jl xi_i xi_k = 0.
    E = MS.voigt_to_tensor_field(d, engineering=True)
    for (i, j, kk, l) in [(0, 0, 1, 1), (0, 1, 1, 2), (0, 0, 2, 2), (1, 2, 0, 2)]:
        c = (E[i, j] * xi[kk] * xi[l] + E[kk, l] * xi[i] * xi[j]
             - E[i, kk] * xi[j] * xi[l] - E[j, l] * xi[i] * xi[kk])
        assert np.max(np.abs(c[keep])) < 1e-9 * np.max(np.abs(E))


def test_even_grid_excludes_mixed_nyquist_modes():
    k, excl = MS.wavevectors(4)
    # modes with an index -2 and at least one other nonzero index
    expected = 0
    for a in np.ndindex(4, 4, 4):
        kk = [x if x < 2 else x - 4 for x in a]
        if any(abs(x) == 2 for x in kk) and sum(x != 0 for x in kk) >= 2:
            expected += 1
    # hand count: 64 - 27 modes contain the index -2; 3 of them are pure-axis
    assert excl.sum() == expected == 34
    assert not MS.wavevectors(5)[1].any()


def test_homogeneous_grid_converges_after_one_update():
    """C0 = C, compatible non-uniform start: one strain update gives the exact
    uniform solution, so the second evaluation has e < 1e-14."""
    N = 6
    E = np.array([0.01, -0.002, 0.003, 0.001, -0.004, 0.002])
    k, excl = MS.wavevectors(N)
    xi = 2 * np.pi * k
    rng = np.random.default_rng(2)
    eps_hat = np.zeros((N, N, N, 6), dtype=complex)
    u = rng.normal(size=(3, N, N, N))
    u_hat = np.stack([np.fft.fftn(u[c]) for c in range(3)])
    for idx in np.ndindex(N, N, N):
        if excl[idx]:
            continue
        eps_hat[idx] = sym_grad_voigt(1j * xi[(slice(None),) + idx], u_hat[(slice(None),) + idx])
    eps0 = np.stack([np.fft.ifftn(eps_hat[..., c]).real for c in range(6)], axis=-1).reshape(-1, 6) * 1e-3
    eps0 += E  # mean E after the (zero-increment) first load application below
    ph = np.zeros((N, N, N), dtype=np.uint8)
    laws = [(O.KIND_ELASTIC, (70.0, 0.3))]
    r = MS.solve(ph, laws, E[None], [0.1], tol=1e-14, max_iter=5, eps0=eps0, E_prev0=E)
    assert r["errors"][0][0] > 1e-3
    assert r["errors"][0][1] < 1e-14
    assert r["iters"][0] == 2
    C = stiffness(70.0, 0.3)
    assert np.max(np.abs(r["Sigma"][0] - C @ E)) < 1e-13 * np.max(np.abs(C @ E))


def laminate_exact(Ca, Cb, f, E):
    """Layers normal to x with fractions f (phase a) and 1-f.  Continuity of
    (e22, e33, g23) and of (s11, s13, s12); averages of (e11, g13, g12) = E."""
    jump = [0, 4, 5]          # components free to jump: e11, g13, g12
    cont = [1, 2, 3]
    # unknowns: the jump components in phase a (3) and b (3)
    A = np.zeros((6, 6))
    rhs = np.zeros(6)
    for r, c in enumerate(jump):
        A[r, r] = f
        A[r, 3 + r] = 1 - f
        rhs[r] = E[c]
    traction = [0, 4, 5]      # s11, s13, s12 equal in both layers
    for r, s in enumerate(traction):
        for m, c in enumerate(jump):
            A[3 + r, m] = Ca[s, c]
            A[3 + r, 3 + m] = -Cb[s, c]
        rhs[3 + r] = -sum((Ca[s, c] - Cb[s, c]) * E[c] for c in cont)
    x = np.linalg.solve(A, rhs)
    ea, eb = E.copy(), E.copy()
    ea[jump] = x[:3]
    eb[jump] = x[3:]
    return f * Ca @ ea + (1 - f) * Cb @ eb


@pytest.mark.parametrize("N,n_first", [(8, 3), (9, 4), (10, 5)])
def test_laminate_matches_closed_form(N, n_first):
    E = np.array([0.01, 0.002, -0.003, 0.004, 0.001, 0.005])
    ph = synth.laminate_phase(N, n_first)
    laws = [(O.KIND_ELASTIC, (70.0, 0.3)), (O.KIND_ELASTIC, (400.0, 0.2))]
    r = MS.solve(ph, laws, E[None], [0.1], tol=1e-13, max_iter=3000)
    exact = laminate_exact(stiffness(400.0, 0.2), stiffness(70.0, 0.3), n_first / N, E)
    assert np.max(np.abs(r["Sigma"][0] - exact)) < 1e-12 * np.max(np.abs(exact))


def test_centred_sphere_has_cubic_response():
    """Uniaxial macro strain on a centred sphere: transverse stresses equal, shears zero."""
    N = 9
    ph = synth.sphere_phase(N, 0.1)
    laws = [(O.KIND_ELASTIC, (70.0, 0.3)), (O.KIND_ELASTIC, (400.0, 0.2))]
    r = MS.solve(ph, laws, np.array([[0.01, 0, 0, 0, 0, 0]]), [0.1], tol=1e-12)
    S = r["Sigma"][0]
    assert abs(S[1] - S[2]) < 1e-12 * abs(S[0])
    assert np.max(np.abs(S[3:])) < 1e-12 * abs(S[0])
    # stiffer than the matrix, softer than the inclusion
    assert stiffness(70.0, 0.3)[0, 0] * 0.01 < S[0] < stiffness(400.0, 0.2)[0, 0] * 0.01


def test_homogeneous_viscoplastic_grid_follows_single_voxel_history():
    """One Norton phase: fields stay uniform, each step converges at the first
    evaluation, and Sigma_k follows the single-voxel law with z_n carried over."""
    N = 4
    prm = synth.MATRIX_16
    ph = np.zeros((N, N, N), dtype=np.uint8)
    loads = synth.ramp(4, [0.01, 0, 0, 0, 0, 0.004])
    r = MS.solve(ph, [(O.KIND_NORTON, prm)], loads, [0.1] * 4, tol=1e-10)
    assert list(r["iters"]) == [1, 1, 1, 1]
    zn = np.zeros((1, 6))
    for k in range(4):
        s, zn = O.update(O.KIND_NORTON, prm, loads[k][None], zn, 0.1)
        assert np.max(np.abs(r["Sigma"][k] - s[0])) < 1e-14


def _single_mode_stress(N, kvec, A, mean):
    """sigma(x) = mean + A cos(2 pi k . x) on the voxel centres x = (i, j, l)/N
    of the unit cell, stress-like Voigt (N^3, 6)."""
    i, j, l = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    ph = 2.0 * np.pi * (kvec[0] * i + kvec[1] * j + kvec[2] * l) / N
    return (np.asarray(mean)[None, :] + np.cos(ph).reshape(-1, 1) * np.asarray(A)[None, :])


def _tensor(v):
    s = np.asarray(v, dtype=float)
    return np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])


@pytest.mark.parametrize("N,kvec", [(8, (1, 2, -3)), (9, (2, -1, 4)), (6, (0, 1, 1))])
def test_equilibrium_error_of_a_single_mode_field(N, kvec):
    """Closed form of the stopping measure (Sec. 3 iterates until equilibrium; the
    measure is reading 8): for sigma = S + A cos(2 pi k.x) the normalised DFT
    holds A/2 at the two modes +-k, whose wave vectors are +-2 pi k, so
        sum_xi |xi . c(xi)|^2 = 2 |2 pi (A k)/2|^2 = 2 pi^2 |A k|^2
    and e = sqrt(2) pi |A k| / |S|_F, with |S|_F counting each shear twice.
    A dropped 2 pi, a missing 1/N^3 or an engineering-shear weight on the
    stress changes the value."""
    A = np.array([0.3, -0.1, 0.2, 0.05, -0.07, 0.11])
    S = np.array([1.0, 0.4, -0.2, 0.3, 0.1, -0.5])
    sig = _single_mode_stress(N, kvec, A, S)
    sig_hat = np.stack([np.fft.fftn(sig[:, c].reshape(N, N, N)) for c in range(6)])
    e = MS.equilibrium_error(sig_hat, sig.mean(axis=0), N, floor=0.0)
    Ak = _tensor(A) @ np.asarray(kvec, dtype=float)
    S_F = np.sqrt(np.sum(S[:3] ** 2) + 2.0 * np.sum(S[3:] ** 2))
    expect = np.sqrt(2.0) * np.pi * np.linalg.norm(Ak) / S_F
    assert abs(e - expect) < 1e-12 * expect


def test_equilibrium_error_nyquist_modes_and_floor():
    """Even N: the pure-axis Nyquist mode k = (N/2, 0, 0) is a single real mode,
    cos(pi i) = (-1)^i, with c = A and |xi| = pi N, so e = pi N |A e_1| / |S|_F;
    a mixed Nyquist mode (N/2, 1, 0) is excluded (reading 6) and contributes
    nothing; with zero mean stress the floor is the denominator."""
    N = 8
    A = np.array([0.3, -0.1, 0.2, 0.05, -0.07, 0.11])
    S = np.array([1.0, 0.4, -0.2, 0.3, 0.1, -0.5])
    S_F = np.sqrt(np.sum(S[:3] ** 2) + 2.0 * np.sum(S[3:] ** 2))
    sig = _single_mode_stress(N, (N // 2, 0, 0), A, S)
    sig_hat = np.stack([np.fft.fftn(sig[:, c].reshape(N, N, N)) for c in range(6)])
    e = MS.equilibrium_error(sig_hat, sig.mean(axis=0), N, floor=0.0)
    expect = np.pi * N * np.linalg.norm(_tensor(A)[:, 0]) / S_F
    assert abs(e - expect) < 1e-12 * expect
    mixed = _single_mode_stress(N, (N // 2, 1, 0), A, S)
    mixed_hat = np.stack([np.fft.fftn(mixed[:, c].reshape(N, N, N)) for c in range(6)])
    # (FFT rounding only: the same field on a non-excluded mode gives e of order 10)
    assert MS.equilibrium_error(mixed_hat, mixed.mean(axis=0), N, floor=0.0) < 1e-12 * expect
    # zero mean: e = sqrt(2) pi |A k| / floor
    k = (1, 0, 2)
    z = _single_mode_stress(N, k, A, np.zeros(6))
    z_hat = np.stack([np.fft.fftn(z[:, c].reshape(N, N, N)) for c in range(6)])
    e0 = MS.equilibrium_error(z_hat, np.zeros(6), N, floor=0.25)
    expect0 = np.sqrt(2.0) * np.pi * np.linalg.norm(_tensor(A) @ np.array(k, float)) / 0.25
    assert abs(e0 - expect0) < 1e-12 * expect0
