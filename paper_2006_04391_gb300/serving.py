"""Serving driver: a stream of homogenization jobs on one GPU.

Jobs arrive over wall-clock time; each arrival is submitted to the native
serving engine (``serve_submit``), which admits it when a slot and the HBM
budget allow and advances every active job by one batched basic-scheme
iteration per ``serve_tick``.  The driver records, per job, arrival,
admission and completion times, and reports latency percentiles and
throughput.  The baselines are one-job-at-a-time paths (``ms_solve`` per
job, in arrival order: the plain FP64 path, and the same FP32-bulk path the
server runs); their latencies under the same arrivals follow from their
service times by the single-server queue recursion c_i = max(a_i, c_{i-1}) +
s_i.

This module is host-side orchestration only; all arithmetic runs in the
library's kernels.
"""
import time

import numpy as np


def percentiles(x, ps=(50, 99)):
    """Percentiles with linear interpolation (numpy's default)."""
    x = np.asarray(x, dtype=np.float64)
    return {f"p{p}": float(np.percentile(x, p)) for p in ps}


def fifo_completion(arrivals, service):
    """Completion times of a single FIFO server: c_i = max(a_i, c_{i-1}) + s_i."""
    order = np.argsort(arrivals, kind="stable")
    c = np.zeros(len(arrivals))
    t = -np.inf
    for i in order:
        t = max(arrivals[i], t) + service[i]
        c[i] = t
    return c


def poisson_arrivals(n, rate, seed):
    """Arrival times of a Poisson process with the given rate (first at 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    gaps[0] = 0.0
    return np.cumsum(gaps)


def make_laws(G, laws_spec, precision):
    from . import GSM_FP64  # noqa: F401
    out = []
    for kind, prm in laws_spec:
        out.append(G.norton(*prm, precision=precision) if kind == 1 else G.elastic(*prm))
    return out


def run_stream(G, jobs, arrivals, hbm_budget, max_active=64, ms_precision=None, law_precision=None,
               tol=1e-6, max_iter=20000, poll=1e-4):
    """Serve ``jobs`` (dicts with N, phase, laws, E, h) arriving at ``arrivals`` seconds.

    Returns per-job records and totals.  All times are wall-clock seconds
    measured on the host around the synchronous ticks.
    """
    ms_precision = G.MS_PREC_FP32_BULK if ms_precision is None else ms_precision
    law_precision = G.GSM_FP32_FP64FIX if law_precision is None else law_precision
    server = G.Server(hbm_budget, max_active)
    laws = [make_laws(G, j["laws"], law_precision) for j in jobs]
    order = list(np.argsort(arrivals, kind="stable"))
    n = len(jobs)
    rec = [dict() for _ in range(n)]
    outstanding = {}
    n_done = 0
    ticks = 0
    max_seen_active = 0
    t0 = time.perf_counter()
    while n_done < n:
        now = time.perf_counter() - t0
        while order and arrivals[order[0]] <= now:
            i = order.pop(0)
            j = jobs[i]
            jid = server.submit(j["phase"], laws[i], j["E"], j["h"], tol=tol, max_iter=max_iter,
                                precision=ms_precision)
            outstanding[jid] = i
            rec[i]["arrival"] = float(arrivals[i])
            rec[i]["submitted"] = now
        if not outstanding:
            time.sleep(max(0.0, min(poll, arrivals[order[0]] - now)) if order else poll)
            continue
        a, q, f = server.tick()
        ticks += 1
        max_seen_active = max(max_seen_active, a)
        now = time.perf_counter() - t0
        for jid in list(outstanding):
            st, step, it = server.state(jid)
            i = outstanding[jid]
            if st == G.SERVE_ACTIVE and "admitted" not in rec[i]:
                rec[i]["admitted"] = now
            if st in (G.SERVE_DONE, G.SERVE_DONE_NOTCONV):
                res = server.fetch(jid)
                rec[i].update(finished=now, latency=now - rec[i]["arrival"], Sigma=res["Sigma"],
                              iters=res["iters"], final_error=res["final_error"], rc=res["rc"])
                del outstanding[jid]
                n_done += 1
    makespan = max(r["finished"] for r in rec) - min(r["arrival"] for r in rec)
    server.close()
    evals = sum(int(np.sum(r["iters"])) * jobs[i]["N"] ** 3 for i, r in enumerate(rec))
    return {"jobs": rec, "makespan_s": makespan, "ticks": ticks, "max_active": max_seen_active,
            "jobs_per_s": n / makespan, "voxel_updates_per_s": evals / makespan,
            **{f"latency_{k}": v for k, v in percentiles([r["latency"] for r in rec]).items()}}


def iteration_times(G, jobs, ms_precision=None, law_precision=None, k0=10, k1=30, warm=2):
    """Seconds per basic-scheme iteration of each job run alone through ms_run
    (default: the plain FP64 path), in the steady state of a load step: the
    difference of forced runs of k1 and k0 iterations of the first load step
    (after ``warm`` untimed ones), divided by k1 - k0, so that the step start
    and the first (cold-started) evaluation drop out."""
    import torch
    ms_precision = G.MS_PREC_FP64 if ms_precision is None else ms_precision
    law_precision = G.GSM_FP64 if law_precision is None else law_precision
    out = []
    for j in jobs:
        laws = make_laws(G, j["laws"], law_precision)
        phase = torch.from_numpy(np.ascontiguousarray(j["phase"])).cuda()
        ctx = G.ms_create(phase, laws, ms_precision)
        G.ms_run(ctx, j["E"][:1], j["h"][:1], forced_iters=[warm], switch_tol=1e30)
        t = {}
        for k in (k0, k1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.ms_run(ctx, j["E"][:1], j["h"][:1], forced_iters=[k], switch_tol=1e30)
            torch.cuda.synchronize()
            t[k] = time.perf_counter() - t0
        out.append((t[k1] - t[k0]) / (k1 - k0))
        G.ms_destroy(ctx)
    return np.array(out)


def run_sequential(G, jobs, tol=1e-6, max_iter=20000, ms_precision=None, law_precision=None):
    """Service time of each job run alone through ms_solve (default: the plain FP64 path)."""
    import torch
    ms_precision = G.MS_PREC_FP64 if ms_precision is None else ms_precision
    law_precision = G.GSM_FP64 if law_precision is None else law_precision
    out = []
    for j in jobs:
        laws = make_laws(G, j["laws"], law_precision)
        phase = torch.from_numpy(np.ascontiguousarray(j["phase"])).cuda()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = G.ms_solve(phase, laws, j["E"], j["h"], precision=ms_precision, tol=tol, max_iter=max_iter)
        torch.cuda.synchronize()
        out.append({"service_s": time.perf_counter() - t, "Sigma": r["Sigma"], "iters": r["iters"],
                    "rc": r["rc"]})
    return out
