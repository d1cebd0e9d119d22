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

# Algorithmic FP64 operation counts of the update (add/sub/mul = 1, fma = 2,
# each div, sqrt, rsqrt, log, exp = 1), from a hand-derived implementation of
# the same steps (no AD): predictor, one line-search step, one Newton step,
# final stress.  The per-voxel total weights them with the iteration counts
# the kernel reports in its status words.
FLOPS_PREDICTOR = 73
FLOPS_LINE = 165
FLOPS_NEWTON = 300
FLOPS_STRESS = 30
# FP64 correction step of the FP32-bulk mode: FP64 residual (70), update (5),
# conversions and test (10).  The FP32 Newton matrix of a correction is FP32 work.
FLOPS_FIX64 = 85
BYTES_PER_VOXEL_FP64 = 4 * 6 * 8          # eps, z_n in; sigma, z out


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
    return ap.parse_args()


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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


def flops_per_voxel(status, mode):
    import numpy as np
    line = (status & 0xFF).astype(np.float64)
    newton = ((status >> 8) & 0xFF).astype(np.float64)
    if mode == "fp64":
        f = FLOPS_PREDICTOR + FLOPS_LINE * line + FLOPS_NEWTON * newton + FLOPS_STRESS
        return float(f.mean()), float(line.mean()), float(newton.mean())
    return float(line.mean()), float(newton.mean())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# FP64 FMA peak of GB300 from the unit counts and clocks: 1.25 TFLOP/s nominal
# (1.19 TFLOP/s measured with an FMA-throughput kernel at 1987 MHz).
FP64_PEAK_GFLOPS = 1250.0


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
    for mode, prec in (("fp64", G.GSM_FP64), ("fp32fix", G.GSM_FP32_FP64FIX)):
        mat = G.norton(*PARAMS, precision=prec)
        for _ in range(args.warmup):
            G.gsm_update(mat, e, z0, H_STEP, sig, z, None, st)
        torch.cuda.synchronize()
        status = st.cpu().numpy()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        clocks = Clocks(dev) if (mode == "fp64" and rank == 0) else None
        if clocks:
            clocks.start()
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
        clk = clocks.stop() if clocks else None
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), world)
        results[mode] = {"ms": total_ms / args.steps, "per_launch_ms": statistics.mean(per),
                         "status": status, "launches": launches, "clocks": clk}

    e2e_ms = float("nan")
    if not args.no_e2e:
        e2e_ms = bench_e2e(G, torch, np, eps, zn, e, z0, sig, z, st, stream, world, args)

    ms_block = None
    if not args.no_ms and rank == 0:
        ms_block = bench_ms(G, torch)
    report(args, world, rank, results, e2e_ms, ms_block)


def bench_e2e(G, torch, np, eps, zn, e, z0, sig, z, st, stream, world, args):
    """End to end through the public API with pinned host buffers (FP32 bulk + FP64 fix)."""
    mat = G.norton(*PARAMS, precision=G.GSM_FP32_FP64FIX)
    h_eps = torch.from_numpy(np.ascontiguousarray(eps.T)).pin_memory()
    h_zn = torch.from_numpy(np.ascontiguousarray(zn.T)).pin_memory()
    h_sig = torch.empty_like(h_eps).pin_memory()
    h_z = torch.empty_like(h_eps).pin_memory()

    def e2e_step():
        e.copy_(h_eps, non_blocking=True)
        z0.copy_(h_zn, non_blocking=True)
        G.gsm_update(mat, e, z0, H_STEP, sig, z, None, st)
        h_sig.copy_(sig, non_blocking=True)
        h_z.copy_(z, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(a.elapsed_time(b), world) / args.steps


def report(args, world, rank, results, e2e_ms, ms_block):
    if rank != 0:
        return
    peaks = measured_peaks()
    r64, r32 = results["fp64"], results["fp32fix"]
    fpv, line64, newton64 = flops_per_voxel(r64["status"], "fp64")
    line32, newton32 = flops_per_voxel(r32["status"], "fp32fix")
    achieved = fpv * N_VOX / (r64["per_launch_ms"] * 1e-3) / 1e9
    value = world * N_VOX / (r32["ms"] * 1e-3)
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
        "config": {"workload": "material-law batch: 2^24 independent voxels, Norton n=5, h=0.01, "
                               "FP32 Newton + FP64 correction (value) and full FP64 (fp64 block)",
                   "voxels_per_gpu": N_VOX, "l2": "inputs 1.6 GB > L2, no flush", "parallelism": f"replicas x{world}"},
        "fp64": {"value": world * N_VOX / (r64["ms"] * 1e-3), "ms_per_step": r64["ms"],
                 "mean_line_iters": line64, "mean_newton_iters": newton64},
        "fp32fix": {"mean_line_iters": line32, "mean_newton_plus_fix_iters": newton32},
        "roofline": {"kernel": "norton_kernel<MODE_FP64>", "bound": "alu", "achieved": achieved,
                     "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)", "frac": achieved / FP64_PEAK_GFLOPS,
                     "traffic": None, "algorithmic_flops_per_voxel": fpv,
                     "peak_source": "nominal FP64 of GB300 (unit counts x clock); MEASURED_PEAKS.json has no FP64 entry",
                     "hbm_frac_fp32fix": BYTES_PER_VOXEL_FP64 * N_VOX / (r32["per_launch_ms"] * 1e-3) / 1e9
                     / peaks.get("hbm_gbs", 6783.1)},
        "e2e": {"value": world * N_VOX / (e2e_ms * 1e-3), "unit": "voxel-updates/s",
                "h2d_bytes_per_step": 2 * 6 * 8 * N_VOX, "d2h_bytes_per_step": 2 * 6 * 8 * N_VOX},
        "gpu_launches": r32["launches"] + r64["launches"],
        "clocks": r64["clocks"],
    }
    if ms_block is not None:
        out["basic_scheme"] = ms_block
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out))


def bench_ms(G, torch):
    """Basic-scheme iterations/s at 256^3 (fibre composite), FP64 and FP32 bulk."""
    if not hasattr(G.load(), "ms_create"):
        return None
    import numpy as np
    import synth
    ph, frac, nf = synth.fibre_composite(256, seed=0)
    phase = torch.from_numpy(ph).cuda()
    res = {"workload": f"256^3 RSA cylinders r=6 L=180, 15 percent (achieved {frac:.4f}, {nf} fibres), "
                       "n=10, shear+tension"}
    loads, hs = synth.shear_tension_load(20, 0.02)
    for name, prec in (("fp64", G.MS_PREC_FP64), ("fp32_bulk", G.MS_PREC_FP32_BULK)):
        laws = [G.norton(*synth.MATRIX_256), G.elastic(*synth.FIBRE_256)]
        ctx = G.ms_create(phase, laws, prec)
        n_it = 30
        G.ms_run(ctx, loads[:1], hs[:1], forced_iters=[3], switch_tol=1e30)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = G.ms_run(ctx, loads[:1], hs[:1], forced_iters=[n_it], switch_tol=1e30)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"iters_per_s": n_it / dt, "iters": n_it}
        G.ms_destroy(ctx)
    return res


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
        "config": {"workload": "material-law batch, Norton n=5, h=0.01 (oracle on a 2^20-voxel sample per step)"},
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
