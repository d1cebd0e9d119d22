"""Serving engine (serve_* C ABI): a job's result is the same alone and in a
mixed batch, equals the single-solve path, and admission respects the HBM
budget."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

LAWS = [(O.KIND_NORTON, synth.MATRIX_16), (O.KIND_ELASTIC, synth.INCLUSION_16)]


def job(N, frac, n_exp, E_dir, steps, seed):
    ph = synth.sphere_phase(N, frac) if seed % 2 == 0 else synth.rsa_spheres(N, max(2.0, N / 8), frac, seed=seed)[0]
    laws = [(O.KIND_NORTON, synth.MATRIX_16[:4] + (n_exp,)), (O.KIND_ELASTIC, synth.INCLUSION_16)]
    return {"N": N, "phase": ph, "laws": laws, "E": synth.ramp(steps, E_dir), "h": [0.1] * steps}


def glaws(G, spec, precision=0):
    return [G.norton(*p, precision=precision) if k == O.KIND_NORTON else G.elastic(*p) for k, p in spec]


def serve_all(G, jobs, budget=8 << 30, max_active=16, precision=1, stagger=False, tol=1e-7):
    sv = G.Server(budget, max_active)
    ids = []
    done = {}
    pending = list(range(len(jobs)))
    ticks = 0
    peak = 0
    while len(done) < len(jobs):
        if pending and (not stagger or ticks % 7 == 0):
            i = pending.pop(0)
            j = jobs[i]
            ids.append((sv.submit(j["phase"], glaws(G, j["laws"], G.GSM_FP32_FP64FIX), j["E"], j["h"], tol=tol,
                                  precision=precision), i))
        a, q, f = sv.tick()
        ticks += 1
        peak = max(peak, a)
        for jid, i in ids:
            if i not in done and sv.state(jid)[0] in (G.SERVE_DONE, G.SERVE_DONE_NOTCONV):
                done[i] = sv.fetch(jid)
    sv.close()
    return done, peak


def test_alone_equals_mixed_and_single_path(gsm):
    import torch
    jobs = [job(16, 0.1, 5.0, [0.004, 0, 0, 0, 0, 0], 3, 0),
            job(24, 0.15, 3.0, [0.0, 0.003, 0, 0.002, 0, 0], 4, 2),
            job(12, 0.2, 10.0, [0.002, -0.001, 0, 0, 0, 0.003], 2, 4),
            job(20, 0.1, 5.0, [0.003, 0.003, -0.002, 0, 0, 0], 3, 1)]
    for prec in (gsm.MS_PREC_FP64, gsm.MS_PREC_FP32_BULK):
        mixed, peak = serve_all(gsm, jobs, precision=prec, stagger=True)
        assert peak >= 2
        for i, j in enumerate(jobs):
            alone, _ = serve_all(gsm, [j], precision=prec)
            assert np.array_equal(mixed[i]["Sigma"], alone[0]["Sigma"]), (prec, i)
            assert np.array_equal(mixed[i]["iters"], alone[0]["iters"])
            single = gsm.ms_solve(torch.from_numpy(j["phase"]).cuda(), glaws(gsm, j["laws"], gsm.GSM_FP32_FP64FIX),
                                  j["E"], j["h"], tol=1e-7, precision=prec)
            assert np.array_equal(single["Sigma"], alone[0]["Sigma"])


def test_served_results_match_oracle(gsm):
    """A served job (FP32 bulk, FP64 finish with FP32-Newton + FP64-fix laws)
    agrees with the FP64 oracle to the tolerance's order."""
    import oracle.ms as OMS
    j = job(12, 0.15, 5.0, [0.004, 0, 0, 0, 0, 0.002], 2, 0)
    ref = OMS.solve(j["phase"], j["laws"], j["E"], j["h"], tol=1e-10)
    out, _ = serve_all(gsm, [j])
    Sig = out[0]["Sigma"]
    assert np.max(np.abs(Sig - ref["Sigma"])) / np.max(np.abs(ref["Sigma"])) < 1e-6


def test_admission_respects_budget(gsm):
    jobs = [job(16, 0.1, 5.0, [0.002, 0, 0, 0, 0, 0], 2, 2 * k) for k in range(5)]
    one = gsm.serve_job_bytes(16, gsm.MS_PREC_FP32_BULK)
    out, peak = serve_all(gsm, jobs, budget=int(2.5 * one), max_active=8)
    assert len(out) == 5 and peak <= 2


def test_oversized_job_is_rejected(gsm):
    sv = gsm.Server(1 << 20, 4)
    j = job(64, 0.1, 5.0, [0.002, 0, 0, 0, 0, 0], 1, 0)
    with pytest.raises(gsm.GsmError) as ei:
        sv.submit(j["phase"], glaws(gsm, j["laws"]), j["E"], j["h"])
    assert ei.value.code == gsm.GSM_ENOMEM
    sv.close()


def test_stream_driver_poisson(gsm):
    from paper_2006_04391_gb300 import serving
    jobs = [job(N, 0.1, 5.0, [0.002, 0, 0, 0, 0, 0.001], 2, k) for k, N in enumerate([12, 16, 20, 16, 12, 24])]
    arr = serving.poisson_arrivals(len(jobs), rate=50.0, seed=3)
    res = serving.run_stream(gsm, jobs, arr, hbm_budget=4 << 30, max_active=8, tol=1e-7)
    lat = [r["latency"] for r in res["jobs"]]
    assert all(x > 0 for x in lat) and res["latency_p99"] >= res["latency_p50"] > 0
    assert all(r["rc"] == 0 for r in res["jobs"])


def test_ode_law_jobs_served_with_implicit_jobs(gsm):
    """Jobs whose laws integrate over each step by ode23 / ode23s (the paper's
    Michel-Suquet metal-matrix composite; ODE tolerance below the equilibrium
    tolerance) are served in the same ticks as an implicit-Euler Norton job:
    each result equals its solo serve and the single-solve path bit for bit."""
    import torch
    ms_laws = [gsm.michel_suquet(*synth.ALUMINIUM_MS), gsm.elastic(*synth.ALUMINA)]
    nor_laws = [gsm.norton(*synth.MATRIX_16), gsm.elastic(*synth.INCLUSION_16)]
    specs = [  # (phase, laws, E, h, ode, method)
        (synth.sphere_phase(10, 0.2), ms_laws, synth.ramp(2, [0.003, -0.001, -0.001, 0, 0, 0]), [0.5, 0.5],
         (1e-8, 1e-11), "ode23"),
        (synth.sphere_phase(12, 0.15), nor_laws, synth.ramp(2, [0.004, 0, 0, 0, 0.002, 0]), [0.1, 0.1],
         None, "ode23"),
        (synth.sphere_phase(8, 0.2), ms_laws, synth.ramp(2, [0.002, 0, 0, 0.002, 0, 0]), [0.5, 0.5],
         (1e-8, 1e-11), "ode23s"),
    ]

    def serve(idx):
        sv = gsm.Server(4 << 30, 8)
        ids = {}
        for k, i in enumerate(idx):
            ph, laws, E, h, ode, meth = specs[i]
            ids[i] = sv.submit(ph, laws, E, h, tol=1e-6, precision=gsm.MS_PREC_FP64, ode=ode, ode_method=meth)
        out = {}
        while len(out) < len(idx):
            sv.tick()
            for i, jid in ids.items():
                if i not in out and sv.state(jid)[0] in (gsm.SERVE_DONE, gsm.SERVE_DONE_NOTCONV):
                    out[i] = sv.fetch(jid)
        sv.close()
        return out

    mixed = serve([0, 1, 2])
    for i, (ph, laws, E, h, ode, meth) in enumerate(specs):
        alone = serve([i])[i]
        assert np.array_equal(mixed[i]["Sigma"], alone["Sigma"]) and np.array_equal(mixed[i]["iters"], alone["iters"])
        single = gsm.ms_solve(torch.from_numpy(ph).cuda(), laws, E, h, tol=1e-6, max_iter=20000, ode=ode,
                              ode_method=meth)
        assert np.array_equal(single["Sigma"], alone["Sigma"])
    # the Michel-Suquet law still needs an ODE integrator when served
    sv = gsm.Server(1 << 30, 2)
    with pytest.raises(gsm.GsmError):
        sv.submit(specs[0][0], ms_laws, specs[0][2], specs[0][3], precision=gsm.MS_PREC_FP64)
    sv.close()


def test_serving_tolerance_holds_the_effective_stress(gsm):
    """Jobs of the serving stream (32^3, 5-6 steps, n in {3, 5, 10}) served at
    the benchmark's equilibrium tolerance 1e-4: the effective stresses are
    within 1e-6 (relative to the largest) of the FP64 path converged to 1e-9,
    which the parity tests hold to the oracle."""
    import torch
    jobs = synth.serving_stream(3, seed=21, grids=(32,), steps=(5, 6))
    out, _ = serve_all(gsm, jobs, precision=gsm.MS_PREC_FP32_BULK, tol=1e-4)
    for i, j in enumerate(jobs):
        ref = gsm.ms_solve(torch.from_numpy(j["phase"]).cuda(), glaws(gsm, j["laws"]), j["E"], j["h"], tol=1e-9,
                           max_iter=50000)
        assert ref["rc"] == 0
        err = np.max(np.abs(out[i]["Sigma"] - ref["Sigma"])) / np.max(np.abs(ref["Sigma"]))
        assert err < 1e-6, (i, err)


def test_fair_share_lets_small_jobs_pass_a_large_one(gsm):
    """A 48^3 job submitted first and three 12^3 jobs after it: with fair-share
    ticks the small jobs run many iterations per iteration of the large one
    and finish first, with results bit-identical to their solo runs."""
    big = job(48, 0.15, 5.0, [0.004, 0, 0, 0, 0, 0.002], 3, 0)
    small = [job(12, 0.1 + 0.05 * k, 5.0, [0.002, 0.001, 0, 0, 0, 0], 2, 2 * k) for k in range(3)]
    sv = gsm.Server(8 << 30, 8)
    ids = [sv.submit(j["phase"], glaws(gsm, j["laws"], gsm.GSM_FP32_FP64FIX), j["E"], j["h"], tol=1e-7)
           for j in [big] + small]
    finished = []
    res = {}
    while len(finished) < 4:
        sv.tick()
        for jid in ids:
            if jid not in finished and sv.state(jid)[0] in (gsm.SERVE_DONE, gsm.SERVE_DONE_NOTCONV):
                finished.append(jid)
                res[jid] = sv.fetch(jid)
    sv.close()
    assert finished[-1] == ids[0]
    for jid, j in zip(ids[1:], small):
        alone, _ = serve_all(gsm, [j], tol=1e-7)
        assert np.array_equal(res[jid]["Sigma"], alone[0]["Sigma"])
