"""Host (g++) build of the device headers: expression-template AD derivatives
against finite differences, and the AD-driven per-voxel solve against the
FP64 oracle.  Checks the algorithm without a GPU; the GPU parity tests are in
tests/test_gpu_*.py."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "host_solver_check.cpp")
_dp = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def hlib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("hsc") / "hsc.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I/usr/local/cuda/include", SRC, "-o", out], check=True)
    return ctypes.CDLL(out)


def P(a):
    return a.ctypes.data_as(_dp)


def test_ad_derivatives_match_finite_differences(hlib):
    rng = np.random.default_rng(0)
    for n in (1.0, 5.0, 10.0):
        prm = np.array(synth.MATRIX_16[:4] + (n,))
        eps = rng.uniform(-0.02, 0.02, 6)
        y = rng.uniform(-0.005, 0.005, 5)
        v = rng.uniform(-1, 1, 5)
        g, H = np.empty(5), np.empty((5, 5))
        hlib.host_psi_derivs(P(prm), P(eps), P(y), P(g), P(H))
        # psi is quadratic: its gradient is linear in y, so differences are exact up to rounding
        for a in range(5):
            yp, ym = y.copy(), y.copy()
            yp[a] += 1e-6
            ym[a] -= 1e-6
            gp, gm, Hd = np.empty(5), np.empty(5), np.empty((5, 5))
            hlib.host_psi_derivs(P(prm), P(eps), P(yp), P(gp), P(Hd))
            hlib.host_psi_derivs(P(prm), P(eps), P(ym), P(gm), P(Hd))
            assert np.max(np.abs((gp - gm) / 2e-6 - H[:, a])) < 1e-6 * np.max(np.abs(H))
            # the gradient itself against differences of the oracle's psi
            fd = (O.psi(tuple(prm), eps, yp) - O.psi(tuple(prm), eps, ym)) / 2e-6
            assert abs(fd - g[a]) < 1e-7 * max(1.0, np.max(np.abs(g)))
        gv, Hv = np.empty(5), np.empty((5, 5))
        hlib.host_phi_derivs(P(prm), P(v), P(gv), P(Hv))
        for a in range(5):
            vp, vm = v.copy(), v.copy()
            vp[a] += 1e-6
            vm[a] -= 1e-6
            gp, gm, Hd = np.empty(5), np.empty(5), np.empty((5, 5))
            hlib.host_phi_derivs(P(prm), P(vp), P(gp), P(Hd))
            hlib.host_phi_derivs(P(prm), P(vm), P(gm), P(Hd))
            assert np.max(np.abs((gp - gm) / 2e-6 - Hv[:, a])) < 1e-6 * np.max(np.abs(Hv))
            fd = (O.phi(tuple(prm), vp) - O.phi(tuple(prm), vm)) / 2e-6
            assert abs(fd - gv[a]) < 1e-7 * max(1.0, np.max(np.abs(gv)))


def test_ad_second_order_blocks(hlib):
    """sigma = psi_eps and its second-order blocks: psi_ee = C, psi_ey = -C P."""
    prm = np.array(synth.MATRIX_16)
    eps = np.array([0.01, -0.004, 0.002, 0.003, -0.001, 0.005])
    y = np.array([0.001, -0.002, 0.0005, 0.0, 0.0007])
    sig, Cee, Cey = np.empty(6), np.empty((6, 6)), np.empty((6, 5))
    hlib.host_psi_blocks(P(prm), P(eps), P(y), P(sig), P(Cee), P(Cey))
    assert np.max(np.abs(sig - O.stress(tuple(prm), eps, y))) < 1e-14
    lam, mu = O.lame(70.0, 0.3)
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[:3, :3] += 2 * mu * np.eye(3)
    C[3:, 3:] = mu * np.eye(3)
    assert np.max(np.abs(Cee - C)) < 1e-12
    assert np.max(np.abs(Cey + C @ O.P_MATRIX)) < 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_host_solver_matches_oracle(hlib, mode):
    prm = np.array(synth.MATRIX_16)
    eps, zn = synth.material_batch(3000, seed=5)
    n = eps.shape[0]
    for h in (1e-3, 1e-2, 1e-1):
        sig, z, tan = np.empty((n, 6)), np.empty((n, 6)), np.empty((n, 21))
        st = np.empty(n, dtype=np.int32)
        hlib.host_update(mode, P(prm), ctypes.c_int64(n), P(eps), P(zn), ctypes.c_double(h), P(sig), P(z), P(tan),
                         st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        s2, z2, C2 = O.update(O.KIND_NORTON, tuple(prm), eps, zn, h, tangent=True)
        iu = np.triu_indices(6)
        assert np.all((st >> 16) & 1)
        assert (np.abs(sig - s2).max(1) / np.abs(s2).max(1)).max() < 1e-11
        assert (np.abs(z - z2).max(1) / np.abs(z2).max(1)).max() < 1e-11
        assert (np.abs(tan - C2[:, iu[0], iu[1]]).max(1) / np.abs(C2).max((1, 2))).max() < 1e-11


def _trial_cases(case, n, rng):
    mag = 10.0 ** rng.uniform(-25, -1, (n, 1))
    dev = rng.normal(size=(n, 6)) * mag
    hyd = np.array([[1, 1, 1, 0, 0, 0]])
    if case == "hydrostatic":
        return rng.uniform(-0.01, 0.01, (n, 1)) * hyd + dev * 0.01, np.zeros((n, 6))
    if case == "tiny_deviatoric":
        return dev - dev[:, :3].mean(1, keepdims=True) * hyd, np.zeros((n, 6))
    # unloading onto the accumulated viscous strain: eps - z_n nearly hydrostatic
    y = rng.normal(size=(n, 5)) * 0.01
    zn = np.stack([y[:, 0], y[:, 1], -y[:, 0] - y[:, 1], y[:, 2], y[:, 3], y[:, 4]], 1)
    return zn + dev + rng.uniform(-0.01, 0.01, (n, 1)) * hyd, zn


@pytest.mark.parametrize("case", ["hydrostatic", "tiny_deviatoric", "unloading"])
@pytest.mark.parametrize("mode", [0, 1])
def test_host_solver_small_trial_states(hlib, case, mode):
    """Deviatoric trial strains from 1e-25 to 1e-1, alone, on a hydrostatic
    strain, or on an accumulated viscous strain, n from 1 to 20: every voxel
    converges and sigma matches the oracle to 1e-10; z matches it up to the
    rounding of the inputs (where the flow is below the resolution of y the
    two sides may differ by that rounding)."""
    rng = np.random.default_rng(["hydrostatic", "tiny_deviatoric", "unloading"].index(case) * 2 + mode)
    n = 600
    eps, zn = _trial_cases(case, n, rng)
    for n_exp in (1.0, 2.0, 5.0, 10.0, 20.0):
        prm = np.array(synth.MATRIX_16[:4] + (n_exp,))
        for h in (1e-4, 1e-2, 1.0):
            sig, z = np.empty((n, 6)), np.empty((n, 6))
            st = np.empty(n, dtype=np.int32)
            hlib.host_update(mode, P(prm), ctypes.c_int64(n), P(eps), P(zn), ctypes.c_double(h), P(sig), P(z), None,
                             st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
            s2, z2 = O.update(O.KIND_NORTON, tuple(prm), eps, zn, h)
            assert np.all((st >> 16) & 1), "converged"
            assert np.all((st >> 17) & 7 == 0), "no non-finite, cap or non-SPD flag"
            assert (np.abs(sig - s2).max(1) / np.abs(s2).max(1)).max() < 1e-10
            bound = 1e-10 * np.abs(z2 - zn).max(1) + 2e-15 * (np.abs(eps).max(1) + np.abs(zn).max(1))
            assert np.all(np.abs(z - z2).max(1) <= bound)


def _ode23_host(hlib, prm, en, e, zn, h, rtol, atol, tangent, kind=1, method="ode23"):
    n = e.shape[0]
    nz = zn.shape[1]
    sig, z = np.empty((n, 6)), np.empty((n, nz))
    st = np.empty(n, dtype=np.int32)
    C = np.empty((n, 36)) if tangent else None
    prm = np.asarray(list(prm) + [0.0] * (7 - len(prm)), dtype=float)
    fn = {"ode23": hlib.host_update_ode23, "ode12": hlib.host_update_ode12, "ode23s": hlib.host_update_ode23s}[method]
    fn(kind, P(prm), ctypes.c_int64(n), P(en), P(e), P(np.ascontiguousarray(zn)),
       ctypes.c_double(h), ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_int(100000),
       P(sig), P(z), P(C) if tangent else None, st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return sig, z, C, st


@pytest.mark.parametrize("tangent", [False, True])
@pytest.mark.parametrize("n_exp,rtol,atol", [(1.0, 1e-3, 1e-6), (5.0, 1e-3, 1e-6), (10.0, 1e-3, 1e-6),
                                             (5.0, 1e-8, 1e-11)])
def test_host_ode23_matches_oracle(hlib, tangent, n_exp, rtol, atol):
    """The AD-driven ode23 update (host build of the device header) against the
    oracle's hand-derived one.  Where both take the same substeps the results
    agree to rounding (1e-10); a borderline accept/reject decision can flip
    between the two roundings, after which both remain within the error
    control's tolerance of each other: at most 2 % of voxels, and every voxel
    within 10 (rtol |sigma| + atol)."""
    prm = synth.MATRIX_16[:4] + (n_exp,)
    en, e, zn = synth.ode23_batch(400, seed=int(n_exp) + int(tangent))
    sig, z, C, st = _ode23_host(hlib, prm, en, e, zn, 0.1, rtol, atol, tangent)
    out = O.update_ode23(prm, en, e, zn, 0.1, rtol=rtol, atol=atol, tangent=tangent, info=True)
    assert np.all((st >> 16) & 1) and np.all(out[-1][:, 2] == 1)
    rel = np.abs(sig - out[0]).max(1) / np.abs(out[0]).max(1)
    relz = np.abs(z - out[1]).max(1) / np.maximum(np.abs(out[1] - zn).max(1), 1e-300)
    tight = (rel < 1e-10) & (relz < 1e-10)
    if tangent:
        C2 = out[2].reshape(-1, 36)
        tight &= np.abs(C - C2).max(1) / np.abs(C2).max(1) < 1e-9
    assert tight.mean() >= 0.98
    assert np.all(np.abs(sig - out[0]) <= 10 * (rtol * np.abs(out[0]).max(1, keepdims=True) + atol))


@pytest.mark.parametrize("tangent", [False, True])
def test_host_ode23_michel_suquet_matches_oracle(hlib, tangent):
    """The paper's Michel-Suquet law (kinematic hardening, yield) through the AD
    ode23 update against the oracle's hand-derived one; z and alpha stored as
    7 components."""
    prm = synth.ALUMINIUM_MS
    en, e, zn6 = synth.ode23_batch(400, seed=21 + int(tangent))
    alpha_n = np.random.default_rng(3).uniform(0.0, 0.01, 400)
    zn = np.concatenate([zn6, alpha_n[:, None]], axis=1)
    sig, z, C, st = _ode23_host(hlib, prm, en, e, zn, 0.1, 1e-3, 1e-6, tangent, kind=2)
    out = O.update_ode23(prm, en, e, zn6, 0.1, tangent=tangent, info=True, kind=O.KIND_MICHEL_SUQUET,
                         alpha_n=alpha_n)
    assert np.all((st >> 16) & 1) and np.all(out[-1][:, 2] == 1)
    rel = np.abs(sig - out[0]).max(1) / np.abs(out[0]).max(1)
    relz = np.abs(z[:, :6] - out[1]).max(1) / np.maximum(np.abs(out[1] - zn6).max(1), 1e-300)
    rela = np.abs(z[:, 6] - out[2]) / np.maximum(np.abs(out[2] - alpha_n), 1e-300)
    tight = (rel < 1e-10) & (relz < 1e-10) & ((rela < 1e-10) | (np.abs(z[:, 6] - out[2]) < 1e-18))
    if tangent:
        C2 = out[3].reshape(-1, 36)
        tight &= np.abs(C - C2).max(1) / np.abs(C2).max(1) < 1e-9
    assert tight.mean() >= 0.98
    assert np.all(np.abs(sig - out[0]) <= 10 * (1e-3 * np.abs(out[0]).max(1, keepdims=True) + 1e-6))
    assert np.all(z[:, 6] >= alpha_n)  # alpha never decreases


def test_host_ode23_michel_suquet_tangent_from_the_virgin_state(hlib):
    """The first load step of a basic-scheme run starts the Michel-Suquet law
    at eps = z = alpha = 0, where the force norm is 0 inside the elastic domain:
    the tangent ODE must stay finite there and give the oracle's stress and
    tangent, from uniaxial and shear strains, below and beyond yield."""
    prm = synth.ALUMINIUM_MS
    e = np.array([[0.0015, 0, 0, 0, 0, 0], [0.0002, 0, 0, 0, 0, 0], [0, 0, 0, 0.002, 0, 0],
                  [0.001, -0.0004, -0.0004, 0, 0.0008, 0]])
    n = e.shape[0]
    en, zn = np.zeros((n, 6)), np.zeros((n, 7))
    sig, z, C, st = _ode23_host(hlib, prm, en, e, zn, 0.5, 1e-8, 1e-11, True, kind=2)
    out = O.update_ode23(prm, en, e, zn[:, :6], 0.5, rtol=1e-8, atol=1e-11, tangent=True, info=True,
                         kind=O.KIND_MICHEL_SUQUET, alpha_n=np.zeros(n))
    assert np.all((st >> 16) & 1) and np.all(np.isfinite(C))
    assert np.allclose(sig, out[0], rtol=1e-10, atol=1e-16)
    C2 = out[3].reshape(-1, 36)
    assert np.all(np.abs(C - C2).max(1) / np.abs(C2).max(1) < 1e-9)


@pytest.mark.parametrize("tangent", [False, True])
@pytest.mark.parametrize("kind", [1, 2])
def test_host_ode12_matches_oracle(hlib, tangent, kind):
    """The AD-driven ode12 (Euler/Heun pair) against the oracle's hand-derived
    one, Norton and Michel-Suquet, under the same flip-tolerant criterion as
    ode23."""
    prm = synth.MATRIX_16 if kind == 1 else synth.ALUMINIUM_MS
    en, e, zn6 = synth.ode23_batch(300, seed=61 + kind + int(tangent))
    alpha_n = np.random.default_rng(7).uniform(0.0, 0.01, 300) if kind == 2 else None
    zn = zn6 if kind == 1 else np.concatenate([zn6, alpha_n[:, None]], axis=1)
    sig, z, C, st = _ode23_host(hlib, prm, en, e, zn, 0.1, 1e-3, 1e-6, tangent, kind=kind, method="ode12")
    kw = {"alpha_n": alpha_n} if kind == 2 else {}
    out = O.update_ode23(prm, en, e, zn6, 0.1, tangent=tangent, info=True, kind=kind, method="ode12", **kw)
    assert np.all((st >> 16) & 1) and np.all(out[-1][:, 2] == 1)
    rel = np.abs(sig - out[0]).max(1) / np.abs(out[0]).max(1)
    relz = np.abs(z[:, :6] - out[1]).max(1) / np.maximum(np.abs(out[1] - zn6).max(1), 1e-300)
    tight = (rel < 1e-10) & (relz < 1e-10)
    same = ((st & 0xFFFF) == out[-1][:, 0]) & (((st >> 20) & 0x7FF) == out[-1][:, 1])
    if tangent:
        C2 = out[3 if kind == 2 else 2].reshape(-1, 36)
        tight &= np.abs(C - C2).max(1) / np.abs(C2).max(1) < 1e-9
    assert tight.mean() >= 0.98 and same.mean() >= 0.98
    assert np.all(np.abs(sig - out[0]) <= 10 * (1e-3 * np.abs(out[0]).max(1, keepdims=True) + 1e-6))


def test_host_stage_lu_solves_with_pivoting(hlib):
    """The register LU of the Rosenbrock stages against numpy's solve, on
    matrices that need row exchanges (small or zero leading pivots) and on
    I - c J with J like the law Jacobians; a singular matrix is reported."""
    rng = np.random.default_rng(17)
    for n in (5, 6):
        for trial in range(40):
            W = rng.normal(size=(n, n))
            if trial % 3 == 0:
                W[0, 0] = 0.0                     # forces a swap at the first column
            if trial % 3 == 1:
                W[:, :2] = W[:, :2] * 1e-3        # small pivots in the first columns
            b = rng.normal(size=n)
            x = np.zeros(n)
            assert hlib.host_stage_solve(n, P(np.ascontiguousarray(W)), P(b), P(x)) == 0
            assert np.allclose(x, np.linalg.solve(W, b), rtol=1e-9, atol=1e-12 * np.abs(x).max())
        S = np.zeros((n, n))
        S[:, 0] = 1.0
        x = np.zeros(n)
        assert hlib.host_stage_solve(n, P(S), P(np.ones(n)), P(x)) == -1


def test_host_force_aaa_matches_oracle(hlib):
    """The hand third derivative of the GPU laws (the ode23s tangent's partial)
    against the oracle's, Norton and Michel-Suquet, active states."""
    rng = np.random.default_rng(5)
    for kind, prm, k in ((1, synth.MATRIX_16, 5), (2, synth.ALUMINIUM_MS, 6)):
        pv = np.asarray(list(prm) + [0.0] * (7 - len(prm)), dtype=float)
        for _ in range(20):
            A = rng.normal(size=k) * 0.2
            if k == 6:
                A[5] = -prm[2]
            u, v = rng.normal(size=(2, k))
            out = np.zeros(k)
            hlib.host_force_aaa(kind, P(pv), P(A), P(u), P(v), P(out))
            ref = O.psi_force_aaa(prm, A, u, v, kind=kind)
            assert np.allclose(out, ref, rtol=1e-11, atol=1e-13 * max(np.abs(ref).max(), 1e-300))


@pytest.mark.parametrize("tangent", [False, True])
@pytest.mark.parametrize("kind", [1, 2])
def test_host_ode23s_matches_oracle(hlib, tangent, kind):
    """The Rosenbrock update built from the AD second derivatives and the hand
    third derivative against the oracle's hand-derived one."""
    prm = synth.MATRIX_16 if kind == 1 else synth.ALUMINIUM_MS
    n = 300 if not tangent else 120
    en, e, zn6 = synth.ode23_batch(n, seed=81 + kind + int(tangent))
    alpha_n = np.random.default_rng(8).uniform(0.0, 0.01, n) if kind == 2 else None
    zn = zn6 if kind == 1 else np.concatenate([zn6, alpha_n[:, None]], axis=1)
    sig, z, C, st = _ode23_host(hlib, prm, en, e, zn, 0.1, 1e-3, 1e-6, tangent, kind=kind, method="ode23s")
    kw = {"alpha_n": alpha_n} if kind == 2 else {}
    out = O.update_ode23(prm, en, e, zn6, 0.1, tangent=tangent, info=True, kind=kind, method="ode23s", **kw)
    assert np.all((st >> 16) & 1) and np.all(out[-1][:, 2] == 1)
    rel = np.abs(sig - out[0]).max(1) / np.abs(out[0]).max(1)
    relz = np.abs(z[:, :6] - out[1]).max(1) / np.maximum(np.abs(out[1] - zn6).max(1), 1e-300)
    tight = (rel < 1e-10) & (relz < 1e-10)
    if tangent:
        C2 = out[3 if kind == 2 else 2].reshape(-1, 36)
        tight &= np.abs(C - C2).max(1) / np.abs(C2).max(1) < 1e-9
    assert tight.mean() >= 0.98
    assert np.all(np.abs(sig - out[0]) <= 10 * (1e-3 * np.abs(out[0]).max(1, keepdims=True) + 1e-6))


@pytest.mark.parametrize("kind", [1, 2])
def test_constant_psi_blocks_and_their_pattern(hlib, kind):
    """The ODE tangents use psi's second-derivative blocks as constants of the
    law: psi is quadratic in (eps, y) for both laws, so a sweep at any point
    gives the blocks of the sweep at the origin bit for bit.  The structural
    pattern read off the expression type must cover every non-zero entry, and
    the blocks take the closed forms of the isotropic elastic energy
    (psi_yy = P^T C P with z = (y0, y1, -y0-y1, y2, y3, y4), psi_ee = C)."""
    prm = np.array(synth.MATRIX_16[:4] + (5.0,)) if kind == 1 else np.array(synth.ALUMINIUM_MS)
    NY = 5 if kind == 1 else 6
    assert hlib.host_psi_degree(kind) == 2  # the compile-time certificate of a quadratic psi
    E, nu = prm[0], prm[1]
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    m = NY * 6 + NY * NY + 36 + 6 * NY
    rng = np.random.default_rng(kind)
    for trial in range(3):
        out = np.empty(2 * m)
        rows = np.empty(6 + NY, dtype=np.uint32)
        eps = rng.uniform(-0.02, 0.02, 6)
        y = rng.uniform(-0.005, 0.005, NY)
        hlib.host_const_blocks(kind, P(prm), P(eps), P(y), P(out), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        B, B0 = out[:m], out[m:]
        assert np.array_equal(B, B0)
        o = 0
        Hye = B[o:o + 6 * NY].reshape(NY, 6); o += 6 * NY
        Hyy = B[o:o + NY * NY].reshape(NY, NY); o += NY * NY
        Cee = B[o:o + 36].reshape(6, 6); o += 36
        Cey = B[o:o + 6 * NY].reshape(6, NY)
        full = np.zeros((6 + NY, 6 + NY))
        full[:6, :6], full[:6, 6:], full[6:, :6], full[6:, 6:] = Cee, Cey, Hye, Hyy
        pat = np.array([[(int(r) >> j) & 1 for j in range(6 + NY)] for r in rows])
        assert np.all(pat[full != 0] == 1)
        # structure: 9 / 7 / 12 / 9 marked entries (the lambda terms of psi_ye cancel numerically)
        assert (pat[6:, :6].sum(), pat[6:, 6:].sum(), pat[:6, :6].sum(), pat[:6, 6:].sum()) == (9, 7, 12, 9)
        Pm = np.zeros((6, NY))
        Pm[0, 0] = Pm[1, 1] = 1.0
        Pm[2, 0] = Pm[2, 1] = -1.0
        Pm[3, 2] = Pm[4, 3] = Pm[5, 4] = 1.0
        C = np.zeros((6, 6))
        C[:3, :3] = lam
        C[:3, :3] += 2 * mu * np.eye(3)
        C[3:, 3:] = mu * np.eye(3)
        Hyy_ref = Pm.T @ C @ Pm
        if kind == 2:
            Hyy_ref[:5, :5] += prm[3] * (2.0 / 3.0) * np.array(
                [[2, 1, 0, 0, 0], [1, 2, 0, 0, 0], [0, 0, 0.5, 0, 0], [0, 0, 0, 0.5, 0], [0, 0, 0, 0, 0.5]])
        assert np.allclose(Cee, C, rtol=1e-14, atol=0)
        assert np.allclose(Cey, -C @ Pm, rtol=1e-14, atol=1e-12 * mu)
        assert np.allclose(Hye, -(C @ Pm).T, rtol=1e-14, atol=1e-12 * mu)
        assert np.allclose(Hyy, Hyy_ref, rtol=1e-14, atol=1e-12 * mu)
