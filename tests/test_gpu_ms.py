"""GPU parity of the basic scheme (ms_create / ms_run / ms_solve) against the
FP64 oracle and the closed-form laminate.

Iteration-matched parity: the GPU runs exactly the oracle's number of
material evaluations per step (forced_iters); the two then differ only by FFT
rounding, which the contracting fixed-point iteration does not amplify, so
the per-step mean stress must agree to 1e-10 (relative to max |Sigma|) and
the final fields to 1e-9.  Free runs to tol agree to O(tol).
"""
import numpy as np
import pytest

import oracle as O
import oracle.ms as OMS
import synth
from test_oracle_ms import laminate_exact, stiffness

pytestmark = pytest.mark.gpu


def gpu_laws(G, laws):
    out = []
    for kind, prm in laws:
        if kind == O.KIND_NORTON:
            out.append(G.norton(*prm))
        elif kind == O.KIND_MICHEL_SUQUET:
            out.append(G.michel_suquet(*prm))
        else:
            out.append(G.elastic(*prm))
    return out


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def sphere16_ref():
    ph, loads, hs = synth.sphere_composite_16()
    laws = [(O.KIND_NORTON, synth.MATRIX_16), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    ref = OMS.solve(ph, laws, loads, hs, tol=1e-8)
    return ph, loads, hs, laws, ref


@pytest.mark.parametrize("N,nf", [(8, 3), (9, 4), (16, 5)])
def test_laminate_closed_form(gsm, N, nf):
    import torch
    E = np.array([0.01, 0.002, -0.003, 0.004, 0.001, 0.005])
    ph = synth.laminate_phase(N, nf)
    laws = [gsm.elastic(70.0, 0.3), gsm.elastic(400.0, 0.2)]
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), laws, E[None], [0.1], tol=1e-13, max_iter=3000)
    exact = laminate_exact(stiffness(400.0, 0.2), stiffness(70.0, 0.3), nf / N, E)
    assert out["rc"] == 0
    assert rel(out["Sigma"][0], exact) < 1e-11


def test_config1_iteration_matched(gsm, sphere16_ref):
    """16^3 sphere composite, 10 steps, FP64: Sigma_k and final fields."""
    import torch
    ph, loads, hs, laws, ref = sphere16_ref
    N = ph.shape[0]
    eps = torch.zeros(6, N ** 3, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(eps)
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws))
    out = gsm.ms_run(ctx, loads, hs, forced_iters=ref["iters"], eps=eps, z=z)
    assert out["rc"] == 0
    assert list(out["iters"]) == list(ref["iters"])
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-10
    assert rel(eps.cpu().numpy().T, ref["eps"]) < 1e-9
    assert rel(z.cpu().numpy().T, ref["z"]) < 1e-9
    # final errors are the oracle's last errors
    last = np.array([e[-1] for e in ref["errors"]])
    assert np.max(np.abs(out["final_error"] - last) / last) < 1e-6


def test_config1_free_run(gsm, sphere16_ref):
    import torch
    ph, loads, hs, laws, ref = sphere16_ref
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, hs, tol=1e-8)
    assert out["rc"] == 0
    assert np.all(np.abs(out["iters"] - ref["iters"]) <= 1)
    assert np.all(out["final_error"] < 1e-8)
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-7


@pytest.mark.parametrize("N", [9, 12])
def test_odd_and_even_grids(gsm, N):
    import torch
    ph = synth.sphere_phase(N, 0.15)
    laws = [(O.KIND_NORTON, synth.MATRIX_16[:4] + (3.0,)), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    loads = synth.ramp(2, [0.004, -0.001, 0.0, 0.002, 0.0, 0.003])
    ref = OMS.solve(ph, laws, loads, [0.05, 0.05], tol=1e-9)
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, [0.05, 0.05],
                       forced_iters=ref["iters"])
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-10


def test_fp32_bulk_then_fp64(gsm, sphere16_ref):
    """FP32 fields/FFTs/laws until e < 1e-5, then FP64 to tol: the mean stress
    matches the FP64 oracle to O(tol)."""
    import torch
    ph, loads, hs, laws, ref = sphere16_ref
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, hs, tol=1e-8,
                       precision=gsm.MS_PREC_FP32_BULK)
    assert out["rc"] == 0
    assert np.all(out["fp32_iters"] > 0) and np.all(out["fp32_iters"] < out["iters"])
    assert np.all(out["final_error"] < 1e-8)
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-6


def test_resume_equals_straight_run(gsm):
    import torch
    ph = synth.sphere_phase(10, 0.1)
    laws = [(O.KIND_NORTON, synth.MATRIX_16), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    loads = synth.ramp(4, [0.004, 0, 0, 0, 0, 0])
    hs = [0.1] * 4
    glaws = gpu_laws(gsm, laws)
    phase = torch.from_numpy(ph).cuda()
    ctx = gsm.ms_create(phase, glaws)
    full = gsm.ms_run(ctx, loads, hs, forced_iters=[40] * 4)
    eps = torch.zeros(6, 1000, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(eps)
    a = gsm.ms_run(ctx, loads[:2], hs[:2], forced_iters=[40] * 2, eps=eps, z=z)
    b = gsm.ms_run(ctx, loads[2:], hs[2:], forced_iters=[40] * 2, eps=eps, z=z, resume=True, E_prev=loads[1])
    both = np.vstack([a["Sigma"], b["Sigma"]])
    assert rel(both, full["Sigma"]) < 1e-12


def test_homogeneous_grid_converges_at_first_evaluation(gsm):
    import torch
    ph = np.zeros((8, 8, 8), dtype=np.uint8)
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), [gsm.elastic(70.0, 0.3)],
                       np.array([[0.01, 0, 0, 0, 0, 0.002]]), [0.1], tol=1e-14)
    assert list(out["iters"]) == [1] and out["final_error"][0] < 1e-14
    assert rel(out["Sigma"][0], stiffness(70.0, 0.3) @ np.array([0.01, 0, 0, 0, 0, 0.002])) < 1e-14


def test_iteration_cap_reports_not_converged(gsm, sphere16_ref):
    import torch
    ph, loads, hs, laws, ref = sphere16_ref
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads[:1], hs[:1], tol=1e-12,
                       max_iter=5)
    assert out["rc"] == gsm.GSM_ENOTCONV and out["iters"][0] == 5


@pytest.fixture(scope="module")
def fibre256():
    return synth.fibre_composite(256, seed=0)


@pytest.mark.parametrize("precision", [0, 1])
def test_fibre_composite_256_first_evaluation(gsm, precision, fibre256):
    """256^3 RSA fibre composite in the benchmark configuration.  With uniform
    strain E_1 the first evaluation's mean stress is the phase-weighted
    single-voxel response, which the oracle computes one voxel per phase."""
    import torch
    ph, frac, nf = fibre256
    loads, hs = synth.shear_tension_load(20, 0.02)
    laws = [(O.KIND_NORTON, synth.MATRIX_256), (O.KIND_ELASTIC, synth.FIBRE_256)]
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), precision)
    out = gsm.ms_run(ctx, loads[:1], hs[:1], forced_iters=[1], switch_tol=1e30)
    f = ph.mean(dtype=np.float64)
    s_m, _ = O.update(O.KIND_NORTON, synth.MATRIX_256, loads[:1], np.zeros((1, 6)), hs[0])
    s_f, _ = O.update(O.KIND_ELASTIC, synth.FIBRE_256, loads[:1], np.zeros((1, 6)), hs[0])
    expect = (1 - f) * s_m[0] + f * s_f[0]
    assert rel(out["Sigma"][0], expect) < 1e-12
    more = gsm.ms_run(ctx, loads[:1], hs[:1], forced_iters=[6], switch_tol=1e30)
    assert np.isfinite(more["Sigma"]).all() and more["final_error"][0] < out["final_error"][0]


UNIAXIAL = [False, True, True, True, True, True]


@pytest.mark.parametrize("mask,ref_update", [(UNIAXIAL, False), (None, True), (UNIAXIAL, True)])
def test_mixed_and_updated_reference_iteration_matched(gsm, mask, ref_update):
    """Mixed boundary conditions (uniaxial stress along 11) and/or the per-step
    reference medium from tangents (Sec. 3), 12^3 sphere composite, 3 steps
    with the matrix flowing: the GPU run with the oracle's per-step evaluation
    counts gives the oracle's Sigma_k, macroscopic strains and reference media."""
    import torch
    ph = synth.sphere_phase(12, 0.2)
    laws = [(O.KIND_NORTON, synth.MATRIX_16), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    loads = synth.ramp(3, [0.006, 0, 0, 0, 0, 0])
    hs = [0.1] * 3
    ref = OMS.solve(ph, laws, loads, hs, tol=1e-8, max_iter=20000, stress_mask=mask, ref_update=ref_update)
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws))
    out = gsm.ms_run(ctx, loads, hs, forced_iters=ref["iters"], stress_mask=mask, ref_update=ref_update)
    gsm.ms_destroy(ctx)
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-9
    assert rel(out["E"], ref["E"]) < 1e-9
    assert np.allclose(out["reference"], ref["reference"], rtol=1e-10, atol=0)
    if mask is not None:
        assert np.max(np.abs(out["Sigma"][:, 1:])) < 1e-6 * np.max(np.abs(out["Sigma"][:, 0]))


def test_uniaxial_stress_free_run_and_bulk_precision(gsm):
    """Free runs to tol with mixed boundary conditions and the updated reference,
    FP64 and FP32 bulk: the prescribed stresses vanish to tol and the response
    agrees with the oracle to O(tol); the homogeneous grid gives Young's modulus."""
    import torch
    ph = synth.sphere_phase(12, 0.2)
    laws = [(O.KIND_NORTON, synth.MATRIX_16), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    loads = synth.ramp(2, [0.004, 0, 0, 0, 0, 0])
    ref = OMS.solve(ph, laws, loads, [0.1, 0.1], tol=1e-8, max_iter=20000, stress_mask=UNIAXIAL, ref_update=True)
    for prec in (gsm.MS_PREC_FP64, gsm.MS_PREC_FP32_BULK):
        out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, [0.1, 0.1], precision=prec,
                           tol=1e-8, max_iter=20000, stress_mask=UNIAXIAL, ref_update=True)
        assert out["rc"] == 0
        assert rel(out["Sigma"], ref["Sigma"]) < 1e-6
        assert np.max(np.abs(out["Sigma"][:, 1:])) < 1e-6 * np.max(np.abs(out["Sigma"][:, 0]))
    hom = gsm.ms_solve(torch.zeros(6, 6, 6, dtype=torch.uint8).cuda(), [gsm.elastic(70.0, 0.3)],
                       [[0.003, 0, 0, 0, 0, 0]], [0.1], tol=1e-12, stress_mask=UNIAXIAL)
    assert abs(hom["Sigma"][0][0] - 70.0 * 0.003) < 1e-12 * 0.21
    assert np.allclose(hom["E"][0], [0.003, -0.0009, -0.0009, 0, 0, 0], rtol=0, atol=1e-15)


def test_taped_run_rejects_mixed_conditions(gsm):
    import torch
    ph = synth.sphere_phase(8, 0.2)
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), [gsm.norton(*synth.MATRIX_16), gsm.elastic(*synth.INCLUSION_16)])
    lib = gsm.load()
    ld, keep, n = gsm._load_struct([[0.002, 0, 0, 0, 0, 0]], [0.1], 1e-8, 100, None, 0.0, UNIAXIAL)
    res, out = gsm._result_struct(n)
    import ctypes
    th = ctypes.c_void_p()
    assert lib.ms_run_taped(ctx.handle, ctypes.byref(ld), ctypes.byref(res), ctypes.byref(th)) == -5
    gsm.ms_destroy(ctx)


# ------------------------------------------------ ode23 laws inside the scheme

ODE = (1e-8, 1e-11)


@pytest.mark.parametrize("method", ["ode23", "ode12", "ode23s"])
@pytest.mark.parametrize("kind,prm", [(O.KIND_NORTON, synth.MATRIX_16), (O.KIND_MICHEL_SUQUET, synth.ALUMINIUM_MS)])
def test_ode23_scheme_homogeneous_grid(gsm, kind, prm, method):
    """A homogeneous grid is one voxel integrated from eps_{k-1} to eps_k by
    ode23 each step: the GPU scheme gives the oracle's history."""
    import torch
    ph = np.zeros((6, 6, 6), dtype=np.uint8)
    loads = synth.ramp(3, [0.004, -0.001, 0.0, 0.0, 0.002, 0.0])
    ref = OMS.solve(ph, [(kind, prm)], loads, [0.1] * 3, tol=1e-12, ode=(1e-6, 1e-9), ode_method=method)
    z = torch.zeros(6, 216, dtype=torch.float64, device="cuda")
    eps = torch.zeros(6, 216, dtype=torch.float64, device="cuda")
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, [(kind, prm)]), loads, [0.1] * 3, tol=1e-12,
                       ode=(1e-6, 1e-9), ode_method=method, eps=eps, z=z)
    assert out["rc"] == 0 and np.all(out["iters"] == ref["iters"])
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-10
    assert np.allclose(z.cpu().numpy().T, ref["z"][:, :6], rtol=1e-9, atol=1e-14)


def test_ode23_norton_composite_iteration_matched(gsm):
    """Norton matrix integrated by ode23, 12^3 sphere composite, 3 steps, the
    oracle's evaluation counts: the GPU gives the oracle's Sigma_k and fields.
    The adaptive control may take a different accept/reject decision in a few
    voxels whose error estimate sits at the threshold (each such voxel's
    stress then differs by about rtol |sigma|), hence 1e-9 rather than the
    1e-10 of the implicit-Euler scheme."""
    import torch
    ph = synth.sphere_phase(12, 0.2)
    laws = [(O.KIND_NORTON, synth.MATRIX_16), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    loads = synth.ramp(3, [0.006, 0, 0, 0, 0, 0])
    forced = [40, 40, 40]
    ref = OMS.solve(ph, laws, loads, [0.1] * 3, forced_iters=forced, ode=ODE)
    eps = torch.zeros(6, 12 ** 3, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(eps)
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, [0.1] * 3, forced_iters=forced,
                       ode=ODE, eps=eps, z=z)
    assert np.all(out["iters"] == forced)
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-9
    assert rel(eps.cpu().numpy().T, ref["eps"]) < 1e-8
    assert rel(z.cpu().numpy().T, ref["z"][:, :6]) < 1e-7


@pytest.mark.parametrize("method", ["ode12", "ode23s"])
def test_ode12_ode23s_michel_suquet_composite_mixed_iteration_matched(gsm, method):
    """The MMC with the ode12 pair (rtol 1e-6: the pair's substep count grows as
    tol^(-1/2)) or the ode23s triple (reference medium from its Rosenbrock
    tangent), uniaxial stress, updated reference, the oracle's evaluation
    counts."""
    import torch
    ph = synth.sphere_phase(8, 0.2)
    laws = [(O.KIND_MICHEL_SUQUET, synth.ALUMINIUM_MS), (O.KIND_ELASTIC, synth.ALUMINA)]
    loads = synth.ramp(2, [0.003, 0, 0, 0, 0, 0])
    forced = [12, 12]
    kw = dict(forced_iters=forced, stress_mask=UNIAXIAL, ref_update=True, ode=(1e-6, 1e-9), ode_method=method)
    ref = OMS.solve(ph, laws, loads, [0.5, 0.5], **kw)
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, [0.5, 0.5], **kw)
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-9
    assert rel(out["E"], ref["E"]) < 1e-9
    assert np.allclose(out["reference"], ref["reference"], rtol=1e-9, atol=0)


def test_ode23_michel_suquet_composite_mixed_iteration_matched(gsm):
    """The paper's metal-matrix composite (Michel-Suquet aluminium, elastic
    alumina) under uniaxial stress with the per-step reference medium from the
    ode23 tangents, the oracle's evaluation counts."""
    import torch
    ph = synth.sphere_phase(10, 0.2)
    laws = [(O.KIND_MICHEL_SUQUET, synth.ALUMINIUM_MS), (O.KIND_ELASTIC, synth.ALUMINA)]
    loads = synth.ramp(2, [0.003, 0, 0, 0, 0, 0])
    forced = [30, 30]
    ref = OMS.solve(ph, laws, loads, [0.5, 0.5], forced_iters=forced, stress_mask=UNIAXIAL, ref_update=True, ode=ODE)
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, [0.5, 0.5], forced_iters=forced,
                       stress_mask=UNIAXIAL, ref_update=True, ode=ODE)
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-9
    assert rel(out["E"], ref["E"]) < 1e-9
    assert np.allclose(out["reference"], ref["reference"], rtol=1e-9, atol=0)


def test_ode23_michel_suquet_free_run(gsm):
    """Free run to tol of the same composite (8^3): converges, the lateral
    stresses vanish, and Sigma agrees with the oracle's free run to O(tol)."""
    import torch
    ph = synth.sphere_phase(8, 0.2)
    laws = [(O.KIND_MICHEL_SUQUET, synth.ALUMINIUM_MS), (O.KIND_ELASTIC, synth.ALUMINA)]
    loads = synth.ramp(2, [0.003, 0, 0, 0, 0, 0])
    ref = OMS.solve(ph, laws, loads, [0.5, 0.5], tol=1e-8, max_iter=5000, stress_mask=UNIAXIAL, ode=ODE)
    out = gsm.ms_solve(torch.from_numpy(ph).cuda(), gpu_laws(gsm, laws), loads, [0.5, 0.5], tol=1e-8, max_iter=5000,
                       stress_mask=UNIAXIAL, ode=ODE)
    assert out["rc"] == 0
    assert rel(out["Sigma"], ref["Sigma"]) < 1e-6
    assert np.max(np.abs(out["Sigma"][:, 1:])) < 1e-7 * np.max(np.abs(out["Sigma"][:, 0]))


def test_ode23_scheme_rejections(gsm):
    """ode23 runs in FP64 only; the Michel-Suquet law needs it, starts fresh
    only, and the taped run takes the implicit-Euler update only."""
    import ctypes
    import torch
    ph = torch.from_numpy(synth.sphere_phase(8, 0.2)).cuda()
    loads, hs = [[0.002, 0, 0, 0, 0, 0]], [0.1]
    nor = [gsm.norton(*synth.MATRIX_16), gsm.elastic(*synth.INCLUSION_16)]
    kin = [gsm.michel_suquet(*synth.ALUMINIUM_MS), gsm.elastic(*synth.ALUMINA)]
    out = gsm.ms_solve(ph, nor, loads, hs, precision=gsm.MS_PREC_FP32_BULK, ode=ODE, check=False)
    assert out["rc"] == gsm.GSM_ENOTSUP
    out = gsm.ms_solve(ph, kin, loads, hs, check=False)
    assert out["rc"] == gsm.GSM_ENOTSUP
    eps = torch.zeros(6, 512, dtype=torch.float64, device="cuda")
    out = gsm.ms_solve(ph, kin, loads, hs, ode=ODE, eps=eps, z=torch.zeros_like(eps), resume=True, check=False)
    assert out["rc"] == gsm.GSM_ENOTSUP
    ctx = gsm.ms_create(ph, nor)
    ld, keep, n = gsm._load_struct(loads, hs, 1e-8, 100, None, 0.0, ode=ODE)
    res, _ = gsm._result_struct(n)
    th = ctypes.c_void_p()
    assert gsm.load().ms_run_taped(ctx.handle, ctypes.byref(ld), ctypes.byref(res), ctypes.byref(th)) == -5
    # the same context then runs ode23 twice (work arrays allocated once)
    a = gsm.ms_run(ctx, loads, hs, ode=ODE)
    b = gsm.ms_run(ctx, loads, hs, ode=ODE)
    assert a["rc"] == 0 and np.array_equal(a["Sigma"], b["Sigma"])
    gsm.ms_destroy(ctx)
