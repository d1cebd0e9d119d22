"""GPU parity of gsm_update_ode23 (C ABI) against the oracle's ode23 update
(force-potential form, Bogacki-Shampine pair with stress-driven step-size
control, tangent ODE of Corollary 1).

Where GPU and oracle take the same substeps their results agree to rounding
(1e-10 for sigma and z, 1e-9 for the tangent); a borderline accept/reject
decision can flip between the two roundings, after which both stay within
the error control's tolerance of each other.  Criterion: at least 98 % of
voxels tight, every voxel within 10 (rtol |sigma| + atol)."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def soa(a, ld):
    import torch
    out = np.zeros((a.shape[1], ld))
    out[:, :a.shape[0]] = a.T
    return torch.from_numpy(out).cuda()


def run(G, mat, en, e, zn, h, rtol=1e-3, atol=1e-6, tangent=False, ld=None, max_substeps=100000, method="ode23"):
    import torch
    n = e.shape[0]
    ld = ld or n
    E0, E1, Z0 = soa(en, ld), soa(e, ld), soa(zn, ld)
    sig = torch.full_like(E1, float("nan"))
    z = torch.full_like(E1, float("nan"))
    tan = torch.full((36, ld), float("nan"), dtype=torch.float64, device="cuda") if tangent else None
    st = torch.zeros(ld, dtype=torch.int32, device="cuda")
    G.gsm_update_ode23(mat, E0, E1, Z0, h, sig, z, tan, st, rtol=rtol, atol=atol, max_substeps=max_substeps, n_vox=n,
                       method=method)
    torch.cuda.synchronize()
    out = [sig.cpu().numpy()[:, :n].T, z.cpu().numpy()[:, :n].T, st.cpu().numpy()[:n]]
    if tangent:
        out.append(tan.cpu().numpy()[:, :n].T)
    return out


def check(res, ref, zn, rtol, atol, tangent):
    sig, z, st = res[:3]
    assert np.all((st >> 16) & 1), "every voxel converged"
    rel = np.abs(sig - ref[0]).max(1) / np.abs(ref[0]).max(1)
    relz = np.abs(z - ref[1]).max(1) / np.maximum(np.abs(ref[1] - zn).max(1), 1e-300)
    tight = (rel < 1e-10) & (relz < 1e-10)
    if tangent:
        C2 = ref[2].reshape(-1, 36)
        tight &= np.abs(res[3] - C2).max(1) / np.abs(C2).max(1) < 1e-9
    assert tight.mean() >= 0.98, tight.mean()
    assert np.all(np.abs(sig - ref[0]) <= 10 * (rtol * np.abs(ref[0]).max(1, keepdims=True) + atol))
    acc = st & 0xFFFF
    assert np.mean(acc[tight] == ref[-1][tight, 0]) == 1.0


@pytest.mark.parametrize("tangent", [False, True])
@pytest.mark.parametrize("n_exp,rtol,atol", [(1.0, 1e-3, 1e-6), (5.0, 1e-3, 1e-6), (10.0, 1e-3, 1e-6),
                                             (5.0, 1e-8, 1e-11)])
def test_ode23_matches_oracle(gsm, tangent, n_exp, rtol, atol):
    prm = synth.MATRIX_16[:4] + (n_exp,)
    n = 2 * 4096 + 37 if not tangent else 4096 + 37   # several blocks and a ragged tail
    en, e, zn = synth.ode23_batch(n, seed=int(n_exp * 7) + int(tangent))
    mat = gsm.norton(*prm)
    res = run(gsm, mat, en, e, zn, 0.1, rtol, atol, tangent, ld=n + 5)
    ref = O.update_ode23(prm, en, e, zn, 0.1, rtol=rtol, atol=atol, tangent=tangent, info=True)
    check(res, ref, zn, rtol, atol, tangent)


def test_ode23_full_size_sampled(gsm):
    """2^22 voxels, the benchmark's launch; 2000 sampled voxels against the oracle."""
    n = 1 << 22
    en, e, zn = synth.ode23_batch(n, seed=2024)
    mat = gsm.norton(*synth.MATRIX_16)
    sig, z, st = run(gsm, mat, en, e, zn, 0.1)
    idx = np.random.default_rng(3).choice(n, 2000, replace=False)
    ref = O.update_ode23(synth.MATRIX_16, en[idx], e[idx], zn[idx], 0.1, info=True)
    check((sig[idx], z[idx], st[idx]), ref, zn[idx], 1e-3, 1e-6, False)
    assert np.all((st >> 16) & 1)


def test_ode23_degenerate_and_invalid(gsm):
    import torch
    mat = gsm.norton(*synth.MATRIX_16)
    zero = np.zeros((3, 6))
    sig, z, st, C = run(gsm, mat, zero, zero, zero, 0.1, tangent=True)
    assert np.all(sig == 0) and np.all(z == 0)
    assert np.all((st & 0xFFFF) == 1) and np.all(((st >> 20) & 0x7FF) == 0)
    lam, mu = 70.0 * 0.3 / (1.3 * 0.4), 70.0 / 2.6
    Cel = np.zeros((6, 6))
    Cel[:3, :3] = lam
    Cel[:3, :3] += 2 * mu * np.eye(3)
    Cel[3:, 3:] = mu * np.eye(3)
    assert np.allclose(C.reshape(-1, 6, 6), Cel[None], rtol=1e-13, atol=1e-12)
    # the substep cap ends the loop with the cap flag and without convergence
    en, e, zn = synth.ode23_batch(64, seed=5)
    sig, z, st = run(gsm, mat, en, e, zn, 0.1, max_substeps=2)
    steps = (st & 0xFFFF) + ((st >> 20) & 0x7FF)
    capped = (st & gsm.ST_CAP) != 0
    conv = ((st >> 16) & 1) == 1
    assert capped.sum() > 32 and np.all(capped != conv) and np.all(steps <= 2)
    t = torch.zeros(6, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(gsm.GsmError):
        gsm.gsm_update_ode23(mat, t, t, t, 0.0, t.clone(), t.clone())
    with pytest.raises(gsm.GsmError):
        gsm.gsm_update_ode23(mat, t, t, t, 0.1, t.clone(), t.clone(), rtol=0.0)
    with pytest.raises(gsm.GsmError):
        gsm.gsm_update_ode23(gsm.elastic(70.0, 0.3), t, t, t, 0.1, t.clone(), t.clone())


def run_ms(G, mat, en, e, zn7, h, tangent=False, ld=None):
    import torch
    n = e.shape[0]
    ld = ld or n
    E0, E1, Z0 = soa(en, ld), soa(e, ld), soa(zn7, ld)
    sig = torch.full_like(E1, float("nan"))
    z = torch.full((7, ld), float("nan"), dtype=torch.float64, device="cuda")
    tan = torch.full((36, ld), float("nan"), dtype=torch.float64, device="cuda") if tangent else None
    st = torch.zeros(ld, dtype=torch.int32, device="cuda")
    G.gsm_update_ode23(mat, E0, E1, Z0, h, sig, z, tan, st, n_vox=n)
    torch.cuda.synchronize()
    out = [sig.cpu().numpy()[:, :n].T, z.cpu().numpy()[:, :n].T, st.cpu().numpy()[:n]]
    if tangent:
        out.append(tan.cpu().numpy()[:, :n].T)
    return out


@pytest.mark.parametrize("tangent", [False, True])
def test_michel_suquet_matches_oracle(gsm, tangent):
    """The paper's Michel-Suquet law (aluminium of the metal-matrix composite:
    kinematic hardening, yield, n = 3.6) against the oracle's hand-derived ode23."""
    prm = synth.ALUMINIUM_MS
    n = 4096 + 37
    en, e, zn6 = synth.ode23_batch(n, seed=40 + int(tangent))
    alpha_n = np.random.default_rng(5).uniform(0.0, 0.01, n)
    zn7 = np.concatenate([zn6, alpha_n[:, None]], axis=1)
    res = run_ms(gsm, gsm.michel_suquet(*prm), en, e, zn7, 0.1, tangent, ld=n + 3)
    ref = O.update_ode23(prm, en, e, zn6, 0.1, tangent=tangent, info=True, kind=O.KIND_MICHEL_SUQUET,
                         alpha_n=alpha_n)
    sig, z, st = res[:3]
    assert np.all((st >> 16) & 1)
    rel = np.abs(sig - ref[0]).max(1) / np.abs(ref[0]).max(1)
    relz = np.abs(z[:, :6] - ref[1]).max(1) / np.maximum(np.abs(ref[1] - zn6).max(1), 1e-300)
    da = np.abs(z[:, 6] - ref[2])
    tight = (rel < 1e-10) & (relz < 1e-10) & (da <= 1e-10 * np.maximum(ref[2] - alpha_n, 1e-300) + 1e-18)
    if tangent:
        C2 = ref[3].reshape(-1, 36)
        tight &= np.abs(res[3] - C2).max(1) / np.abs(C2).max(1) < 1e-9
    assert tight.mean() >= 0.98
    assert np.all(np.abs(sig - ref[0]) <= 10 * (1e-3 * np.abs(ref[0]).max(1, keepdims=True) + 1e-6))
    assert np.all(z[:, 6] >= alpha_n)


def test_michel_suquet_tangent_from_the_virgin_state(gsm):
    """eps_n = z_n = alpha_n = 0 (the first step of a scheme run): the force
    norm starts at 0 inside the elastic domain; stress and tangent are finite
    and the oracle's, below and beyond yield."""
    prm = synth.ALUMINIUM_MS
    e = np.array([[0.0015, 0, 0, 0, 0, 0], [0.0002, 0, 0, 0, 0, 0], [0, 0, 0, 0.002, 0, 0],
                  [0.001, -0.0004, -0.0004, 0, 0.0008, 0]])
    n = e.shape[0]
    sig, z, st, C = run_ms(gsm, gsm.michel_suquet(*prm), np.zeros((n, 6)), e, np.zeros((n, 7)), 0.5, True)
    ref = O.update_ode23(prm, np.zeros((n, 6)), e, np.zeros((n, 6)), 0.5, tangent=True, kind=O.KIND_MICHEL_SUQUET,
                         alpha_n=np.zeros(n))
    assert np.all((st >> 16) & 1) and np.all(np.isfinite(C))
    assert np.allclose(sig, ref[0], rtol=1e-10, atol=1e-16)
    C2 = ref[3].reshape(-1, 36)
    assert np.all(np.abs(C - C2).max(1) / np.abs(C2).max(1) < 1e-9)


def test_michel_suquet_without_yield_and_hardening_is_norton(gsm):
    en, e, zn = synth.ode23_batch(2048, seed=8)
    s1, z1, st1 = run(gsm, gsm.norton(70.0, 0.3, 0.1, 1.0, 5.0), en, e, zn, 0.1)
    zn7 = np.concatenate([zn, np.zeros((2048, 1))], axis=1)
    s2, z2, st2 = run_ms(gsm, gsm.michel_suquet(70.0, 0.3, 0.0, 0.0, 1.0, 0.1, 5.0), en, e, zn7, 0.1)
    same = (st1 & 0xFFFF) == (st2 & 0xFFFF)
    assert same.mean() > 0.98
    assert np.max(np.abs(s1 - s2)[same] / np.abs(s1[same]).max(1, keepdims=True)) < 1e-10


def test_michel_suquet_is_refused_by_the_implicit_paths(gsm):
    import torch
    mat = gsm.michel_suquet(*synth.ALUMINIUM_MS)
    t = torch.zeros(6, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(gsm.GsmError):
        gsm.gsm_update(mat, t, t, 0.1, t.clone(), t.clone())
    # the basic scheme takes it with the ode23 integrator only
    ctx = gsm.ms_create(torch.zeros(4, 4, 4, dtype=torch.uint8).cuda(), [mat])
    out = gsm.ms_run(ctx, [[0.001, 0, 0, 0, 0, 0]], [0.1], check=False)
    gsm.ms_destroy(ctx)
    assert out["rc"] == gsm.GSM_ENOTSUP


# ------------------------------------------------------------ ode12 (Sec. 4.3)

@pytest.mark.parametrize("tangent", [False, True])
@pytest.mark.parametrize("n_exp", [1.0, 5.0])
def test_ode12_matches_oracle(gsm, tangent, n_exp):
    """The explicit Euler / Heun pair (gsm_update_ode, GSM_ODE12) against the
    oracle's ode12, several blocks and a ragged tail."""
    prm = synth.MATRIX_16[:4] + (n_exp,)
    n = 2 * 4096 + 37 if not tangent else 2048 + 37
    en, e, zn = synth.ode23_batch(n, seed=int(n_exp * 3) + 70 + int(tangent))
    res = run(gsm, gsm.norton(*prm), en, e, zn, 0.1, tangent=tangent, ld=n + 3, method="ode12")
    ref = O.update_ode23(prm, en, e, zn, 0.1, tangent=tangent, info=True, method="ode12")
    check(res, ref, zn, 1e-3, 1e-6, tangent)


def test_ode12_michel_suquet_matches_oracle(gsm):
    prm = synth.ALUMINIUM_MS
    n = 4096 + 11
    en, e, zn6 = synth.ode23_batch(n, seed=77)
    alpha_n = np.random.default_rng(9).uniform(0.0, 0.01, n)
    zn7 = np.concatenate([zn6, alpha_n[:, None]], axis=1)
    import torch
    E0, E1, Z0 = soa(en, n), soa(e, n), soa(zn7, n)
    sig = torch.empty_like(E1)
    z = torch.empty(7, n, dtype=torch.float64, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    gsm.gsm_update_ode23(gsm.michel_suquet(*prm), E0, E1, Z0, 0.1, sig, z, None, st, method="ode12")
    ref = O.update_ode23(prm, en, e, zn6, 0.1, info=True, kind=O.KIND_MICHEL_SUQUET, alpha_n=alpha_n, method="ode12")
    s, zz, stt = sig.cpu().numpy().T, z.cpu().numpy().T, st.cpu().numpy()
    assert np.all((stt >> 16) & 1)
    rel = np.abs(s - ref[0]).max(1) / np.abs(ref[0]).max(1)
    da = np.abs(zz[:, 6] - ref[2])
    tight = (rel < 1e-10) & (da <= 1e-10 * np.maximum(ref[2] - alpha_n, 1e-300) + 1e-18)
    assert tight.mean() >= 0.98
    assert np.all(np.abs(s - ref[0]) <= 10 * (1e-3 * np.abs(ref[0]).max(1, keepdims=True) + 1e-6))


def test_ode_method_is_checked(gsm):
    import ctypes
    import torch
    t = torch.zeros(6, 4, dtype=torch.float64, device="cuda")
    mat = gsm.norton(*synth.MATRIX_16)
    lib = gsm.load()
    rc = lib.gsm_update_ode(mat.handle, 7, 4, t.data_ptr(), t.data_ptr(), t.data_ptr(), 4, ctypes.c_double(0.1),
                            ctypes.c_double(1e-3), ctypes.c_double(1e-6), 100, t.clone().data_ptr(),
                            t.clone().data_ptr(), None, None, None)
    assert rc == gsm.GSM_EINVAL


# ------------------------------------------------------- ode23s (Sec. 4.3)

@pytest.mark.parametrize("tangent", [False, True])
@pytest.mark.parametrize("kind", [O.KIND_NORTON, O.KIND_MICHEL_SUQUET])
def test_ode23s_matches_oracle(gsm, tangent, kind):
    """The Rosenbrock triple (gsm_update_ode, GSM_ODE23S; tangent with the hand
    third derivative) against the oracle's ode23s."""
    import torch
    prm = synth.MATRIX_16 if kind == O.KIND_NORTON else synth.ALUMINIUM_MS
    n = 4096 + 37 if not tangent else 1024 + 37
    en, e, zn6 = synth.ode23_batch(n, seed=90 + int(tangent) + 2 * kind)
    if kind == O.KIND_NORTON:
        mat, zn, nz, kw = gsm.norton(*prm), zn6, 6, {}
    else:
        alpha_n = np.random.default_rng(12).uniform(0.0, 0.01, n)
        mat, zn, nz = gsm.michel_suquet(*prm), np.concatenate([zn6, alpha_n[:, None]], axis=1), 7
        kw = {"alpha_n": alpha_n}
    ld = n + 3
    E0, E1, Z0 = soa(en, ld), soa(e, ld), soa(zn, ld)
    sig = torch.full_like(E1, float("nan"))
    z = torch.full((nz, ld), float("nan"), dtype=torch.float64, device="cuda")
    tan = torch.full((36, ld), float("nan"), dtype=torch.float64, device="cuda") if tangent else None
    st = torch.zeros(ld, dtype=torch.int32, device="cuda")
    gsm.gsm_update_ode23(mat, E0, E1, Z0, 0.1, sig, z, tan, st, n_vox=n, method="ode23s")
    torch.cuda.synchronize()
    ref = O.update_ode23(prm, en, e, zn6, 0.1, tangent=tangent, info=True, kind=kind, method="ode23s", **kw)
    s_, z_, st_ = sig.cpu().numpy()[:, :n].T, z.cpu().numpy()[:, :n].T, st.cpu().numpy()[:n]
    assert np.all((st_ >> 16) & 1)
    rel = np.abs(s_ - ref[0]).max(1) / np.abs(ref[0]).max(1)
    relz = np.abs(z_[:, :6] - ref[1]).max(1) / np.maximum(np.abs(ref[1] - zn6).max(1), 1e-300)
    tight = (rel < 1e-10) & (relz < 1e-10)
    if tangent:
        C2 = ref[-2].reshape(-1, 36)
        tight &= np.abs(tan.cpu().numpy()[:, :n].T - C2).max(1) / np.abs(C2).max(1) < 1e-9
    assert tight.mean() >= 0.98, tight.mean()
    assert np.all(np.abs(s_ - ref[0]) <= 10 * (1e-3 * np.abs(ref[0]).max(1, keepdims=True) + 1e-6))


def test_ode23s_stiff_step(gsm):
    """A long deviatoric ramp (amplitude 0.05 over h = 10): the Rosenbrock triple
    takes far fewer substeps than ode23 on the GPU too, and the oracle's result."""
    rng = np.random.default_rng(0)
    n = 512
    d = rng.normal(size=(n, 6))
    d[:, :3] -= d[:, :3].mean(1, keepdims=True)
    eps = 0.05 * d / np.abs(d).max(1, keepdims=True)
    zero = np.zeros((n, 6))
    r23 = run(gsm, gsm.norton(*synth.MATRIX_16), zero, eps, zero, 10.0)
    r3s = run(gsm, gsm.norton(*synth.MATRIX_16), zero, eps, zero, 10.0, method="ode23s")
    steps = lambda st: ((st & 0xFFFF) + ((st >> 20) & 0x7FF)).sum()
    assert steps(r3s[2]) * 5 < steps(r23[2])
    ref = O.update_ode23(synth.MATRIX_16, zero, eps, zero, 10.0, info=True, method="ode23s")
    rel = np.abs(r3s[0] - ref[0]).max(1) / np.abs(ref[0]).max(1)
    assert np.mean(rel < 1e-10) >= 0.98
