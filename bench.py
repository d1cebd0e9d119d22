#!/usr/bin/env python
"""Benchmark of the GSM material update (and the basic scheme) on GB300.

Step = one implicit-Euler material update (AutoMat, arXiv 2006.04391,
Sec. 4.1) of the 2^24-voxel material-law batch: Norton matrix law
(E=70, nu=0.3, sigma0=0.1, edot0=1, n=5), eps ~ U[-0.02,0.02]^6, deviatoric
z_n ~ U[-0.005,0.005], h = 0.01.  Inputs (1.6 GB) and outputs (1.6 GB) are
larger than L2 (129 MB), so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank processes its own 2^24-voxel batch (voxels are
independent: weak scaling, no collective on the data path); the timed region
is bracketed by a barrier and a device synchronize, and rank 0 prints one
JSON line with the maximum time over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC_FULL = "material voxel-updates/s; basic-scheme iters/s @256^3; serve p50/p99 latency"
N_VOX = 1 << 24
H_STEP = 0.01
PARAMS = (70.0, 0.3, 0.1, 1.0, 5.0)

# The material kernels are bound by FP64 issue (FP64 pipe 81-86 % busy,
# DRAM below 12 %; ncu), so their roofline is FP64 operations per second:
# each DADD, DMUL or DFMA takes one FP64 issue slot, and GB300 issues two FP64
# operations per SM per cycle (ncu peak_sustained), i.e. 2 x 152 x 2.07 GHz
# = 629.4 G/s at the maximum clock.  Operations per voxel are the FP64
# additions, multiplications and FMAs the algorithm executes, counted by ncu
# (smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on) on this
# workload at three step sizes:
#   FP32 bulk + FP64 correction: 124.3 per voxel with one correction; each
#     further correction repeats the residual sweep (~95);
#   FP64: 425.5 + 164.0 per line-search iteration (one Newton step), which
#     reproduces the three counts within 0.1 %.
FP64_OPS_PEAK_G = 2 * 152 * 2.07
OPS_FIX_FIRST = 124.3
OPS_FIX_EXTRA = 95.0
OPS_FP64_BASE = 425.5
OPS_FP64_LINE = 164.0
BYTES_PER_VOXEL_FP64 = 4 * 6 * 8          # eps, z_n in; sigma, z out
# DRAM bytes of one full-size FP32-bulk launch (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, one capture of launch 6 of this workload: the
# inputs are read once, less what the 129 MB L2 still holds)
TRAFFIC_FP32FIX = 1476729344 + 1631010816


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-ms", action="store_true", help="skip the basic-scheme measurement")
    ap.add_argument("--voxels", type=int, default=N_VOX, help="batch size (profiling runs use a small batch)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-ode23", action="store_true", help="skip the ODE material-update measurements")
    ap.add_argument("--ode-voxels", type=int, default=1 << 22,
                    help="voxels of the ODE measurements (profiling runs use a small batch)")
    ap.add_argument("--no-mmc", action="store_true", help="skip the MMC scheme run of the ODE measurements")
    ap.add_argument("--ms-n", type=int, default=256, help="grid of the basic-scheme measurement (profiling: 128)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the homogenization-setting scheme runs")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-jobs", type=int, default=16, help="jobs in the serving sample")
    ap.add_argument("--serve-full", action="store_true",
                    help="serve the full stream distribution (grids up to 192^3, 5-20 steps): long")
    return ap.parse_args()


_BACKEND = None


def dist_setup(args=None):
    """One process per GPU under torchrun (NCCL); gloo where CUDA is absent
    (the multi-rank tests run this path on CPU).  Returns (world, rank)."""
    global _BACKEND
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cuda = torch.cuda.is_available()
    if world > 1:
        import torch.distributed as dist
        if cuda:
            torch.cuda.set_device(local)
            _BACKEND = "nccl"
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            _BACKEND = "gloo"
            dist.init_process_group("gloo")
    elif cuda:
        torch.cuda.set_device(0)
    return world, rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Maximum of a host scalar over all ranks (the timing rule: the slowest
    rank's time is the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _BACKEND == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, max_ms):
    """value = units all ranks processed / the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (max_ms * 1e-3)


def bench_config(world, voxels):
    return {"workload": f"material-law batch: {voxels} independent voxels per GPU, Norton E=70, nu=0.3, "
                        "sigma0=0.1, edot0=1, n=5, h=0.01; value: FP32 Newton + one FP64 correction per voxel, "
                        "fp64 block: full FP64",
            "voxels_per_gpu": voxels, "l2": "inputs 1.6 GB > L2 at 2^24 voxels, no flush",
            "parallelism": f"replicas x{world}"}


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def ops_per_voxel(status, mode):
    """Mean FP64 operations per voxel from the kernel's status words."""
    import numpy as np
    line = (status & 0xFF).astype(np.float64)
    newton = ((status >> 8) & 0xFF).astype(np.float64)
    fix = ((status >> 20) & 0xF).astype(np.float64)
    if mode == "fp64":
        f = OPS_FP64_BASE + OPS_FP64_LINE * line
        return float(f.mean()), float(line.mean()), float(newton.mean())
    f = (OPS_FIX_FIRST + OPS_FIX_EXTRA * np.maximum(fix - 1, 0)) * (fix > 0)
    return float(f.mean()), float(line.mean()), float((newton - fix).mean()), float(fix.mean())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def run_ours(args):
    global N_VOX
    N_VOX = args.voxels
    import numpy as np
    import torch

    import paper_2006_04391_gb300 as G
    import synth

    world, rank = dist_setup(args)
    G.load()
    dev = torch.cuda.current_device()
    eps, zn = synth.material_batch(N_VOX, seed=2024 + rank)
    e = torch.from_numpy(np.ascontiguousarray(eps.T)).cuda()
    z0 = torch.from_numpy(np.ascontiguousarray(zn.T)).cuda()
    sig = torch.empty_like(e)
    z = torch.empty_like(e)
    st = torch.empty(N_VOX, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    results = {}
    # clocks sampled over both timed material regions (the FP32-bulk region
    # alone is shorter than the 200 ms sampling period)
    clocks = Clocks(dev) if rank == 0 else None
    if clocks:
        clocks.start()
    for mode, prec in (("fp64", G.GSM_FP64), ("fp32fix", G.GSM_FP32_FP64FIX)):
        mat = G.norton(*PARAMS, precision=prec)
        for _ in range(args.warmup):
            G.gsm_update(mat, e, z0, H_STEP, sig, z, None, st)
        torch.cuda.synchronize()
        status = st.cpu().numpy()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        barrier(world)
        torch.cuda.synchronize()
        l0 = G.kernel_launches()
        ev[0].record(stream)
        for k in range(args.steps):
            G.gsm_update(mat, e, z0, H_STEP, sig, z, None, st)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        launches = G.kernel_launches() - l0
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), world)
        results[mode] = {"ms": total_ms / args.steps, "per_launch_ms": statistics.mean(per),
                         "status": status, "launches": launches}
    results["clocks"] = clocks.stop() if clocks else None

    e2e_ms = None
    if not args.no_e2e:
        e2e_ms = bench_e2e(G, torch, np, eps, zn, e, z0, sig, z, st, stream, world, args)

    ms_block = None
    if not args.no_ms and rank == 0:
        ms_block = bench_ms(G, torch, args)
    serve_block = None
    if not args.no_serve and rank == 0:
        serve_block = bench_serve(G, args)
    adj_block = None
    if not args.no_adjoint and rank == 0:
        adj_block = bench_adjoint(G, torch)
    ode_block = None
    if not args.no_ode23 and rank == 0:
        ode_block = bench_ode23(G, torch, args)
    report(args, world, rank, results, e2e_ms, ms_block, serve_block, adj_block, ode_block)


def bench_e2e(G, torch, np, eps, zn, e, z0, sig, z, st, stream, world, args):
    """End to end through the public API from pinned host buffers (FP32 bulk + FP64 fix).

    Three ways of the same update, each step from inputs in pinned host memory
    to results in pinned host memory:
      zero-copy: gsm_update reads eps, z_n from and writes sigma, z to the
                 pinned host arrays directly (over NVLink-C2C on GB300);
      staged:    copies host -> device, gsm_update on device arrays, copies
                 device -> host, all on one stream;
      streamed:  gsm_update_host: chunks of 2^20 voxels, copies in both
                 directions overlapping the updates.
    Returns {name: ms per step}.
    """
    mat = G.norton(*PARAMS, precision=G.GSM_FP32_FP64FIX)
    h_eps = torch.from_numpy(np.ascontiguousarray(eps.T)).pin_memory()
    h_zn = torch.from_numpy(np.ascontiguousarray(zn.T)).pin_memory()
    h_sig = torch.empty_like(h_eps).pin_memory()
    h_z = torch.empty_like(h_eps).pin_memory()

    def zero_copy():
        G.gsm_update(mat, h_eps, h_zn, H_STEP, h_sig, h_z, None, None)

    def streamed():
        G.gsm_update_host(mat, h_eps, h_zn, H_STEP, h_sig, h_z, None, None)

    def staged():
        e.copy_(h_eps, non_blocking=True)
        z0.copy_(h_zn, non_blocking=True)
        G.gsm_update(mat, e, z0, H_STEP, sig, z, None, st)
        h_sig.copy_(sig, non_blocking=True)
        h_z.copy_(z, non_blocking=True)

    out = {}
    for name, step in (("zero_copy", zero_copy), ("staged", staged), ("streamed", streamed)):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier(world)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        out[name] = max_over_ranks(a.elapsed_time(b), world) / args.steps
    # the zero-copy and streamed results are the device results
    ref = torch.empty_like(h_sig)
    G.gsm_update(mat, e, z0, H_STEP, sig, z, None, st)
    zero_copy()
    torch.cuda.synchronize()
    ref.copy_(sig)
    out["zero_copy_matches_device"] = bool(torch.equal(ref, h_sig))
    h_sig.fill_(float("nan"))
    streamed()
    torch.cuda.synchronize()
    out["streamed_matches_device"] = bool(torch.equal(ref, h_sig))
    return out


def e2e_block(world, e2e):
    nan = float("nan")
    if not e2e:
        return {"value": nan, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    best = min(("zero_copy", "staged", "streamed"), key=lambda k: e2e[k])
    return {"value": world * N_VOX / (e2e[best] * 1e-3), "unit": "voxel-updates/s",
            "h2d_bytes_per_step": 2 * 6 * 8 * N_VOX, "d2h_bytes_per_step": 2 * 6 * 8 * N_VOX,
            "path": best, "zero_copy": world * N_VOX / (e2e["zero_copy"] * 1e-3),
            "staged": world * N_VOX / (e2e["staged"] * 1e-3),
            "streamed": world * N_VOX / (e2e["streamed"] * 1e-3),
            "zero_copy_matches_device": e2e["zero_copy_matches_device"],
            "streamed_matches_device": e2e["streamed_matches_device"],
            "note": "inputs start and results end in pinned host memory; zero_copy: the kernel reads and "
                    "writes them over NVLink-C2C; staged: H2D copies, kernel, D2H copies on one stream; "
                    "streamed: gsm_update_host, 2^20-voxel chunks, copies overlapping the updates"}


def report(args, world, rank, results, e2e_ms, ms_block, serve_block=None, adj_block=None, ode_block=None):
    if rank != 0:
        return
    peaks = measured_peaks()
    r64, r32 = results["fp64"], results["fp32fix"]
    fpv, line64, newton64 = ops_per_voxel(r64["status"], "fp64")
    fpv32, line32, newton32, fix32 = ops_per_voxel(r32["status"], "fp32fix")
    achieved = fpv * N_VOX / (r64["per_launch_ms"] * 1e-3) / 1e9
    achieved32 = fpv32 * N_VOX / (r32["per_launch_ms"] * 1e-3) / 1e9
    value = whole_job_rate(N_VOX, world, r32["ms"])
    out = {
        "metric": "material voxel-updates/s",
        "metric_full": METRIC_FULL,
        "value": value,
        "unit": "voxel-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r32["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64fix",
        "data": "synthetic",
        "config": bench_config(world, N_VOX),
        "fp64": {"value": whole_job_rate(N_VOX, world, r64["ms"]), "ms_per_step": r64["ms"],
                 "mean_line_iters": line64, "mean_newton_iters": newton64},
        "fp32fix": {"mean_line_iters": line32, "mean_fp32_newton_iters": newton32, "mean_fp64_corrections": fix32},
        "roofline": {"kernel": "norton_kernel<MODE_FP32_FIX>", "bound": "alu", "achieved": achieved32,
                     "peak": FP64_OPS_PEAK_G, "unit": "G FP64 ops/s", "frac": achieved32 / FP64_OPS_PEAK_G,
                     "traffic": TRAFFIC_FP32FIX, "fp64_ops_per_voxel": fpv32,
                     "peak_source": "FP64 issue rate of GB300: 2 per SM per cycle (ncu peak_sustained) x 152 SMs "
                                    "x 2.07 GHz; MEASURED_PEAKS.json has no FP64 entry",
                     "note": "FP64 operations of the trial strain and the FP64 correction; the FP32 bulk runs on the "
                             "FP32 pipe",
                     "hbm_frac": BYTES_PER_VOXEL_FP64 * N_VOX / (r32["per_launch_ms"] * 1e-3) / 1e9
                     / peaks.get("hbm_gbs", 6783.1)},
        "roofline_fp64_mode": {"kernel": "norton_kernel<MODE_FP64>", "bound": "alu", "achieved": achieved,
                               "peak": FP64_OPS_PEAK_G, "unit": "G FP64 ops/s",
                               "frac": achieved / FP64_OPS_PEAK_G, "fp64_ops_per_voxel": fpv},
        "e2e": e2e_block(world, e2e_ms),
        "gpu_launches": r32["launches"],
        "clocks": results["clocks"],
    }
    if ms_block is not None:
        out["basic_scheme"] = ms_block
    if serve_block is not None:
        out["serve"] = serve_block
    if adj_block is not None:
        out["adjoint"] = adj_block
    if ode_block is not None:
        out["ode23"] = ode_block
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out))


def bench_ms(G, torch, args):
    """Basic-scheme iterations/s at 256^3 (--ms-n) (fibre composite), FP64 and FP32 bulk."""
    if not hasattr(G.load(), "ms_create"):
        return None
    import numpy as np
    import synth
    N = args.ms_n
    ph, frac, nf = synth.fibre_composite(N, seed=0)
    phase = torch.from_numpy(ph).cuda()
    res = {"workload": f"{N}^3 RSA cylinders r=6 L={min(180.0, 0.7 * N):g}, 15 percent (achieved {frac:.4f}, "
                       f"{nf} fibres), n=10, shear+tension"}
    loads, hs = synth.shear_tension_load(20, 0.02)
    # FP64: FP64 fields, FFTs and laws.  FP32 bulk: FP32 fields, FFTs and law
    # iterations, FP64 reductions; its FP64 iterations evaluate the law as FP32
    # Newton + one FP64 correction per voxel.
    for name, prec, law_prec in (("fp64", G.MS_PREC_FP64, G.GSM_FP64),
                                 ("fp32_bulk", G.MS_PREC_FP32_BULK, G.GSM_FP32_FP64FIX)):
        laws = [G.norton(*synth.MATRIX_256, precision=law_prec), G.elastic(*synth.FIBRE_256)]
        ctx = G.ms_create(phase, laws, prec)
        n_it = 30
        # FP32 bulk: FP32 iterations until e < 1e-5 (not reached in 30 iterations), then one FP64
        G.ms_run(ctx, loads[:1], hs[:1], forced_iters=[3])  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = G.ms_run(ctx, loads[:1], hs[:1], forced_iters=[n_it])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"iters_per_s": n_it / dt, "iters": n_it, "fp32_iters": int(out["fp32_iters"][0]),
                     "final_error": float(out["final_error"][0]),
                     "law": "FP64" if law_prec == G.GSM_FP64 else "FP32 Newton + FP64 correction"}
        G.ms_destroy(ctx)
    if not args.no_mixed:
        res["homogenization_setting"] = bench_mixed(G, torch)
    return res


def bench_mixed(G, torch):
    """The paper's homogenization setting (Sec. 3) on a smaller grid: uniaxial
    tension (eps_11 prescribed, all other mean stresses zero) to 1 % in 5 steps
    of h = 0.1 on a 64^3 centred sphere (20 %), Norton matrix n = 5, FP32 bulk
    with FP64-correction laws, free runs to e < 1e-6: fixed elastic reference
    vs the reference adjusted per step to the tangents."""
    import synth
    N = 64
    ph = torch.from_numpy(synth.sphere_phase(N, 0.2)).cuda()
    loads = synth.ramp(5, [0.01, 0, 0, 0, 0, 0])
    out = {"workload": f"{N}^3 centred sphere 20 %, uniaxial tension to 1 % in 5 steps (mixed boundary "
                       "conditions), Norton n=5, FP32 bulk, tol 1e-6"}
    for name, ref in (("fixed_reference", False), ("updated_reference", True)):
        laws = [G.norton(*synth.MATRIX_16, precision=G.GSM_FP32_FP64FIX), G.elastic(*synth.INCLUSION_16)]
        ctx = G.ms_create(ph, laws, G.MS_PREC_FP32_BULK)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = G.ms_run(ctx, loads, [0.1] * 5, tol=1e-6, max_iter=20000,
                     stress_mask=[False, True, True, True, True, True], ref_update=ref)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        G.ms_destroy(ctx)
        out[name] = {"s": dt, "iters": int(r["iters"].sum()), "iters_per_s": float(r["iters"].sum()) / dt,
                     "Sigma11_final": float(r["Sigma"][-1][0]), "E22_final": float(r["E"][-1][1]),
                     "mu0_last": float(r["reference"][-1][1]), "rc": int(r["rc"])}
    return out


def bench_ode23(G, torch, args):
    """Adaptive ode23 material update (force-potential form, stress-driven error
    control, MATLAB's default tolerances rtol 1e-3, atol 1e-6) on 2^22 (--ode-voxels) voxels of
    load-step-like inputs (synth.ode23_batch, Norton n = 5, h = 0.1), without and
    with the tangent ODE; FP64."""
    import numpy as np
    import synth
    n = args.ode_voxels
    en, e, zn = synth.ode23_batch(n, seed=2024)
    E0 = torch.from_numpy(np.ascontiguousarray(en.T)).cuda()
    E1 = torch.from_numpy(np.ascontiguousarray(e.T)).cuda()
    Z0 = torch.from_numpy(np.ascontiguousarray(zn.T)).cuda()
    sig = torch.empty_like(E1)
    z = torch.empty_like(E1)
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    mat = G.norton(*PARAMS)
    out = {"workload": f"{n} voxels, synth.ode23_batch (z_n as the material batch, eps_n = z_n + U[-0.002,0.002]^6, "
                       "eps = eps_n + U[-0.001,0.001]^6), Norton n=5, h=0.1, rtol 1e-3, atol 1e-6, FP64"}
    stream = torch.cuda.current_stream()
    for name, tan in (("no_tangent", None), ("tangent", torch.empty(36, n, dtype=torch.float64, device="cuda"))):
        for _ in range(max(1, args.warmup // 2)):
            G.gsm_update_ode23(mat, E0, E1, Z0, 0.1, sig, z, tan, st)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 3
        a.record(stream)
        for _ in range(k):
            G.gsm_update_ode23(mat, E0, E1, Z0, 0.1, sig, z, tan, st)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / k
        s = st.cpu().numpy()
        out[name] = {"voxel_updates_per_s": n / (ms * 1e-3), "ms_per_launch": ms,
                     "mean_accepted_substeps": float((s & 0xFFFF).mean()),
                     "mean_rejected_substeps": float(((s >> 20) & 0x7FF).mean()),
                     "converged_fraction": float(((s >> 16) & 1).mean())}
        del tan
    # the paper's Michel-Suquet law (kinematic hardening, yield), same inputs, alpha_n = 0
    import synth as S
    Z7 = torch.cat([Z0, torch.zeros(1, n, dtype=torch.float64, device="cuda")])
    z7 = torch.empty_like(Z7)
    ms = G.michel_suquet(*S.ALUMINIUM_MS)
    G.gsm_update_ode23(ms, E0, E1, Z7, 0.1, sig, z7, None, st)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(3):
        G.gsm_update_ode23(ms, E0, E1, Z7, 0.1, sig, z7, None, st)
    b.record(stream)
    torch.cuda.synchronize()
    ms_t = a.elapsed_time(b) / 3
    s = st.cpu().numpy()
    out["michel_suquet_no_tangent"] = {"law": "aluminium of the paper's MMC (E=55, nu=0.33, sigma_Y=0.025, "
                                              "H=1.8, edot0=1, sigma_d=0.13, n=3.6)",
                                       "voxel_updates_per_s": n / (ms_t * 1e-3), "ms_per_launch": ms_t,
                                       "mean_accepted_substeps": float((s & 0xFFFF).mean()),
                                       "mean_rejected_substeps": float(((s >> 20) & 0x7FF).mean()),
                                       "converged_fraction": float(((s >> 16) & 1).mean())}
    # ode12 (explicit Euler / Heun pair) and ode23s (Rosenbrock triple), same inputs; with
    # the tangent on the first 2^20 (ode12) or 2^18 (ode23s) voxels
    for name, meth, m, tan in (
            ("ode12_no_tangent", "ode12", n, None),
            ("ode12_tangent", "ode12", min(n, 1 << 20),
             torch.empty(36, min(n, 1 << 20), dtype=torch.float64, device="cuda")),
            ("ode23s_no_tangent", "ode23s", n, None),
            ("ode23s_tangent", "ode23s", min(n, 1 << 18),
             torch.empty(36, min(n, 1 << 18), dtype=torch.float64, device="cuda"))):
        views = [t[:, :m].contiguous() for t in (E0, E1, Z0)]
        sg, zz = torch.empty_like(views[1]), torch.empty_like(views[1])
        st2 = torch.empty(m, dtype=torch.int32, device="cuda")
        G.gsm_update_ode23(mat, *views, 0.1, sg, zz, tan, st2, method=meth)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            G.gsm_update_ode23(mat, *views, 0.1, sg, zz, tan, st2, method=meth)
        b.record(stream)
        torch.cuda.synchronize()
        t_ms = a.elapsed_time(b) / 3
        s2 = st2.cpu().numpy()
        out[name] = {"voxels": m, "voxel_updates_per_s": m / (t_ms * 1e-3), "ms_per_launch": t_ms,
                     "mean_accepted_substeps": float((s2 & 0xFFFF).mean()),
                     "mean_rejected_substeps": float(((s2 >> 20) & 0x7FF).mean()),
                     "converged_fraction": float(((s2 >> 16) & 1).mean())}
        del tan
    if not args.no_mmc:
        out["mmc_scheme"] = bench_mmc_scheme(G, torch)
    return out


def bench_mmc_scheme(G, torch):
    """The paper's metal-matrix composite inside the basic scheme: Michel-Suquet
    aluminium with a centred alumina sphere (20 %) on 64^3, uniaxial tension
    (mixed boundary conditions) in 2 steps of h = 0.5, the per-step reference
    from the ode23 tangents, the laws integrated by ode23 (rtol 1e-6, atol
    1e-9); 12 material evaluations per step (bounded; a free run needs a few
    hundred)."""
    import synth
    N = 64
    ph = torch.from_numpy(synth.sphere_phase(N, 0.2)).cuda()
    loads = synth.ramp(2, [0.003, 0, 0, 0, 0, 0])
    laws = [G.michel_suquet(*synth.ALUMINIUM_MS), G.elastic(*synth.ALUMINA)]
    ctx = G.ms_create(ph, laws, G.MS_PREC_FP64)
    kw = dict(stress_mask=[False, True, True, True, True, True], ref_update=True, ode=(1e-6, 1e-9))
    G.ms_run(ctx, loads[:1], [0.5], forced_iters=[2], **kw)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = G.ms_run(ctx, loads, [0.5, 0.5], forced_iters=[12, 12], **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    G.ms_destroy(ctx)
    n_eval = int(r["iters"].sum())
    return {"workload": f"{N}^3 centred alumina sphere 20 % in Michel-Suquet aluminium, uniaxial tension to 0.3 % "
                        "in 2 steps of h=0.5, per-step reference from ode23 tangents, ode23 rtol 1e-6 atol 1e-9, "
                        "12 evaluations per step, FP64",
            "s": dt, "evaluations": n_eval, "evaluations_per_s": n_eval / dt,
            "voxel_updates_per_s": n_eval * N ** 3 / dt, "Sigma11": [float(x) for x in r["Sigma"][:, 0]],
            "final_error": [float(x) for x in r["final_error"]]}


def bench_adjoint(G, torch):
    """Adjoint of the load history on the adjoint workload: 128^3 centred
    sphere (20 %), Norton matrix, uniaxial ramp to 1 % in 10 steps of h = 0.1,
    FP64, per-step checkpoints.

    Converged to 1e-8 this takes ~1340 basic-scheme iterations per step
    forward and about as many adjoint iterations per step and component
    (the matrix flows, and the fixed elastic reference medium of the basic
    scheme contracts by ~0.99 per iteration), i.e. minutes.  The benchmark
    therefore times a bounded run: 20 forced forward iterations per step,
    then the adjoint of Sigma_11 with 20 adjoint iterations per step.  The
    per-iteration rates are the measurement; the time to a converged gradient
    is those rates times the converged counts."""
    import numpy as np
    import synth
    N, steps, k_fwd, k_adj = 128, 10, 20, 20
    ph = synth.sphere_phase(N, 0.2)
    phase = torch.from_numpy(ph).cuda()
    loads = synth.ramp(steps, [0.01, 0, 0, 0, 0, 0])
    hs = [0.1] * steps
    ctx = G.ms_create(phase, [G.norton(*synth.MATRIX_16), G.elastic(*synth.INCLUSION_16)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, tape = G.ms_run_taped(ctx, loads, hs, tol=1e-30, forced_iters=[k_fwd] * steps)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    g, its = G.ms_adjoint(tape, [1, 0, 0, 0, 0, 0], 0, tol=1e-30, max_iter=k_adj, check=False)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    fwd_iters = int(np.sum(res["iters"]))
    adj_iters = int(np.sum(its))
    del tape
    G.ms_destroy(ctx)
    return {"workload": f"{N}^3 centred sphere ({100 * float(ph.mean()):.1f} % inclusion E=400, nu=0.2), Norton "
                        f"matrix n=5, uniaxial ramp to 1 % in {steps} steps of h=0.1, FP64, per-step checkpoints",
            "sample": f"bounded: {k_fwd} forward iterations and {k_adj} adjoint iterations per step (dSigma11)",
            "forward_taped_s": t_fwd, "forward_iters": fwd_iters, "forward_iters_per_s": fwd_iters / t_fwd,
            "adjoint_s": t_adj, "adjoint_iters": adj_iters, "adjoint_iters_per_s": adj_iters / t_adj,
            "tape_bytes": 12 * 8 * N ** 3 * steps}


def bench_serve(G, args):
    """Serving stream vs the plain one-job-at-a-time FP64 path, same jobs.

    Jobs follow the serving workload's distributions (RSA spheres 5-25 % or
    cylinders 10-30 %, Norton n in {3, 5, 10}, random unit load directions
    with 1-2 % amplitude); by default a bounded sample (grids 32-96^3, 2-5
    steps) so the benchmark stays within minutes.  Arrivals are Poisson with
    rate 1.5 / (mean solo FP64 service time).  Both paths solve to e < 1e-6.
    """
    import numpy as np
    import synth
    from paper_2006_04391_gb300 import serving
    tol = 1e-6
    if args.serve_full:
        jobs = synth.serving_stream(args.serve_jobs, seed=7)
    else:
        jobs = synth.serving_stream(args.serve_jobs, seed=7, grids=(32, 64, 96), steps=(2, 5))
    seq = serving.run_sequential(G, jobs, tol=tol)
    service = np.array([r["service_s"] for r in seq])
    rate = 1.5 / service.mean()
    arrivals = serving.poisson_arrivals(len(jobs), rate, seed=11)
    seq_done = serving.fifo_completion(arrivals, service)
    seq_lat = seq_done - arrivals
    budget = 64 << 30
    stream = serving.run_stream(G, jobs, arrivals, hbm_budget=budget, max_active=64, tol=tol)
    closed = serving.run_stream(G, jobs, np.zeros(len(jobs)), hbm_budget=budget, max_active=64, tol=tol)
    diff = max(float(np.max(np.abs(r["Sigma"] - q["Sigma"])) / max(float(np.max(np.abs(q["Sigma"]))), 1e-300))
               for r, q in zip(stream["jobs"], seq))
    vox_evals = sum(int(np.sum(q["iters"])) * j["N"] ** 3 for q, j in zip(seq, jobs))
    return {
        "workload": (f"{len(jobs)} jobs, grids {sorted(set(j['N'] for j in jobs))}, "
                     f"{sum(len(j['h']) for j in jobs)} load steps in total, "
                     + ("full stream distribution" if args.serve_full else "bounded sample (grids <= 96^3, 2-5 steps)")
                     + f", Poisson arrivals at {rate:.3f}/s = 1.5 x solo FP64 rate, tol {tol}"),
        "served": {"latency_p50_s": stream["latency_p50"], "latency_p99_s": stream["latency_p99"],
                   "makespan_s": stream["makespan_s"], "ticks": stream["ticks"], "max_active": stream["max_active"],
                   "path": "FP32 bulk fields/FFTs, FP64 finish with FP32-Newton + FP64-fix laws, batched ticks"},
        "sequential_fp64": {"latency_p50_s": float(np.percentile(seq_lat, 50)),
                            "latency_p99_s": float(np.percentile(seq_lat, 99)),
                            "makespan_s": float(seq_done.max() - arrivals.min()),
                            "mean_service_s": float(service.mean())},
        "throughput_jobs_per_s": {"served_all_at_once": len(jobs) / closed["makespan_s"],
                                  "sequential_fp64": len(jobs) / float(service.sum()),
                                  "ratio": (len(jobs) / closed["makespan_s"]) / (len(jobs) / float(service.sum()))},
        "voxel_updates_per_s": {"served_all_at_once": closed["voxel_updates_per_s"],
                                "sequential_fp64": vox_evals / float(service.sum())},
        "max_rel_sigma_diff_served_vs_fp64": diff,
    }


def cpu_baseline(n_sample=1 << 22):
    import oracle as O
    import synth
    eps, zn = synth.material_batch(n_sample, seed=99)
    t0 = time.perf_counter()
    O.update(O.KIND_NORTON, PARAMS, eps, zn, H_STEP)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": "voxel-updates/s", "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{n_sample} voxels of the same distribution (1/{N_VOX // n_sample} of the batch), "
                      f"{dt:.1f} s, C++ FP64 oracle with OpenMP"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    import synth
    n_sample = 1 << 20
    eps, zn = synth.material_batch(n_sample, seed=99)
    for _ in range(args.warmup):
        O.update(O.KIND_NORTON, PARAMS, eps[:4096], zn[:4096], H_STEP)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.update(O.KIND_NORTON, PARAMS, eps, zn, H_STEP)
    dt = (time.perf_counter() - t0) / args.steps
    value = n_sample / dt
    cb = {"value": value, "unit": "voxel-updates/s", "cores": O.max_threads(), "kind": "oracle",
          "sample": f"{n_sample} voxels per step of the 2^24-voxel batch distribution"}
    print(json.dumps({
        "impl": "reference", "metric": "material voxel-updates/s", "metric_full": METRIC_FULL,
        "value": value, "unit": "voxel-updates/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(int(os.environ.get("WORLD_SIZE", "1")), N_VOX),
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
