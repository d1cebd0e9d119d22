"""GPU adjoint of the load history (ms_run_taped / ms_adjoint) against the
oracle adjoint and central finite differences, and the autograd wrapper."""
import numpy as np
import pytest

import oracle as O
import oracle.ms as OMS
import synth

pytestmark = pytest.mark.gpu

PRM = (70.0, 0.3, 0.1, 1.0, 5.0)
W = np.array([1.0, -0.3, 0.2, 0.1, 0.4, -0.5])


def setup(N=16, steps=3):
    ph = synth.sphere_phase(N, 0.2)
    loads = synth.ramp(steps, [0.004, -0.001, 0.0, 0.0, 0.0, 0.003])
    return ph, loads, [0.1] * steps


def gpu_J(G, ph, prm, loads, hs, tol=1e-13):
    import torch
    laws = [G.norton(*prm), G.elastic(*synth.INCLUSION_16)]
    out = G.ms_solve(torch.from_numpy(ph).cuda(), laws, loads, hs, tol=tol, max_iter=50000)
    return float(W @ out["Sigma"][-1])


def test_adjoint_matches_oracle_adjoint(gsm):
    import torch
    ph, loads, hs = setup()
    laws = [(O.KIND_NORTON, PRM), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    r = OMS.solve_taped(ph, laws, loads, hs, tol=1e-12)
    g_ref, _ = OMS.adjoint(ph, laws, loads, hs, r["tape"], W, 0, tol=1e-12)
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), [gsm.norton(*PRM), gsm.elastic(*synth.INCLUSION_16)])
    res, tape = gsm.ms_run_taped(ctx, loads, hs, tol=1e-12)
    g, its = gsm.ms_adjoint(tape, W, 0, tol=1e-12)
    assert np.all(np.abs(g - g_ref) <= 1e-7 * np.abs(g_ref) + 1e-12), (g, g_ref)


def test_adjoint_after_a_forward_run_with_the_per_step_reference(gsm):
    """The forward run with the per-step reference medium from tangents (Sec.
    3) converges to the same states, so its adjoint (whose equilibrium solves
    take each step's tangent-field reference) gives the oracle adjoint."""
    import torch
    ph, loads, hs = setup()
    laws = [(O.KIND_NORTON, PRM), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    r = OMS.solve_taped(ph, laws, loads, hs, tol=1e-12)
    g_ref, _ = OMS.adjoint(ph, laws, loads, hs, r["tape"], W, 0, tol=1e-12)
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), [gsm.norton(*PRM), gsm.elastic(*synth.INCLUSION_16)])
    res, tape = gsm.ms_run_taped(ctx, loads, hs, tol=1e-12, ref_update=True)
    assert np.all(res["reference"][1:, 1] < res["reference"][0, 1])  # the matrix flows: a softer reference
    g, its = gsm.ms_adjoint(tape, W, 0, tol=1e-12)
    assert np.all(np.abs(g - g_ref) <= 1e-7 * np.abs(g_ref) + 1e-12), (g, g_ref)


def test_adjoint_matches_central_differences(gsm):
    import torch
    ph, loads, hs = setup()
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), [gsm.norton(*PRM), gsm.elastic(*synth.INCLUSION_16)])
    res, tape = gsm.ms_run_taped(ctx, loads, hs, tol=1e-13, max_iter=50000)
    g, _ = gsm.ms_adjoint(tape, W, 0, tol=1e-13, max_iter=50000)
    for i, pos in enumerate([0, 2, 4]):
        d = 1e-6 * PRM[pos]
        pp, pm = list(PRM), list(PRM)
        pp[pos] += d
        pm[pos] -= d
        fd = (gpu_J(gsm, ph, tuple(pp), loads, hs) - gpu_J(gsm, ph, tuple(pm), loads, hs)) / (2 * d)
        assert abs(g[i] - fd) <= 1e-5 * abs(fd) + 1e-10, (i, g[i], fd)


def test_autograd_function(gsm):
    import torch
    ph, loads, hs = setup(N=12, steps=2)
    theta = torch.tensor([70.0, 0.1, 5.0], dtype=torch.float64, requires_grad=True)
    S = gsm.effective_stress(theta, torch.from_numpy(ph).cuda(), loads, hs, tol=1e-12, adj_tol=1e-12)
    J = (torch.from_numpy(W) * S).sum()
    J.backward()
    ctx = gsm.ms_create(torch.from_numpy(ph).cuda(), [gsm.norton(*PRM), gsm.elastic(*synth.INCLUSION_16)])
    res, tape = gsm.ms_run_taped(ctx, loads, hs, tol=1e-12)
    g, _ = gsm.ms_adjoint(tape, W, 0, tol=1e-12)
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0)
    assert np.allclose(S.detach().numpy(), res["Sigma"][-1], rtol=1e-14, atol=0)


def test_adjoint_at_full_grid_matches_central_differences(gsm):
    """128^3 centred sphere (20 %), 3 ramp steps to 0.1 % of h = 0.01 (the
    matrix flows, moderately, so that the basic scheme needs ~700 iterations
    to 1e-12 rather than thousands): dSigma11/d(E, n) from the adjoint against
    central differences (relative step 1e-6) of GPU forward solves; the
    property holds at any grid size and load."""
    import torch
    N, steps = 128, 3
    ph = synth.sphere_phase(N, 0.2)
    loads = synth.ramp(steps, [0.001, 0.0, 0.0, 0.0, 0.0, 0.0])
    hs = [0.01] * steps
    w = np.array([1.0, 0, 0, 0, 0, 0])
    phase = torch.from_numpy(ph).cuda()
    ctx = gsm.ms_create(phase, [gsm.norton(*PRM), gsm.elastic(*synth.INCLUSION_16)])
    res, tape = gsm.ms_run_taped(ctx, loads, hs, tol=1e-12, max_iter=50000)
    g, _ = gsm.ms_adjoint(tape, w, 0, tol=1e-12, max_iter=50000)
    del tape
    gsm.ms_destroy(ctx)

    def J(prm):
        c = gsm.ms_create(phase, [gsm.norton(*prm), gsm.elastic(*synth.INCLUSION_16)])
        out = gsm.ms_run(c, loads, hs, tol=1e-12, max_iter=50000)
        gsm.ms_destroy(c)
        return float(w @ out["Sigma"][-1])

    for i, pos in ((0, 0), (2, 4)):
        d = 1e-6 * PRM[pos]
        pp, pm = list(PRM), list(PRM)
        pp[pos] += d
        pm[pos] -= d
        fd = (J(tuple(pp)) - J(tuple(pm))) / (2 * d)
        assert abs(g[i] - fd) <= 1e-5 * abs(fd) + 1e-10, (i, g[i], fd)
