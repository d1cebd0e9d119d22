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

# The material kernels are bound by arithmetic issue (FP64 pipe 81-86 % busy,
# DRAM below 12 %; ncu), not by HBM or a dense contraction.  Two counts of the
# work per voxel are reported:
#
# * algorithmic flops: the flops of the method's own formulas per piece of the
#   implicit-Euler update (Sec. 4.1), counted by the oracle's counting scalar
#   (oracle.flop_pieces: add/sub, mul, div and sqrt one flop each, structural
#   zeros and law constants free, pow counted apart), times the iteration
#   counts the kernel writes into its status words.  These are the roofline's
#   numerator; the denominator is the FMA throughput measured in the same run
#   by gsm_peak_probe (2 flops per FMA).  tests/test_bench_flops.py holds these
#   constants equal to the oracle's counts.
ALG_FLOPS = {"predictor": 41, "line": 289, "newton": 304, "residual": 67, "subst": 50, "stress": 26,
             "tangent": 449}
ALG_POWS = {"predictor": 0, "line": 3, "newton": 3, "residual": 1, "subst": 0, "stress": 0, "tangent": 2}
# The GPU starts its 1-D search from the root of a scalar model of the
# segment function, which the oracle's search does not use; hand count: per
# scalar (FP32) iteration 9 flops and 2 exponentials, and in the FP64 mode one
# FP64 refinement step of 12 flops, a power and an exponential.
MODEL_FLOPS, MODEL_POWS = 9, 2
MODEL64_FLOPS, MODEL64_POWS = 12, 2
#
# * executed FP64 operations: each DADD, DMUL or DFMA takes one FP64 issue
#   slot and GB300 issues two FP64 operations per SM per cycle (ncu
#   peak_sustained).  Operations per voxel, counted by ncu
#   (smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on) on this
#   workload at three step sizes (profiles/norton_kernel_fp64_op_counts_2p20.md):
#     FP32 bulk + correction (double-float residual and power): 50.52 per
#       voxel with one correction; a further correction repeats the power's
#       FP64 exponent product and the conversions (~5, estimated; one
#       correction is the rule);
#     FP64: 806.5 per voxel at the two line-search evaluations every voxel
#       takes since the search starts from the segment model's root; 158.8 per
#       further evaluation (the earlier fit over three step sizes).
#   They explain the gap between the algorithmic rate and the peak: a power
#   (one algorithmic operation) executes as tens of FP64 operations.
FP64_ISSUE_PER_SM_CLK = 2
OPS_FIX_FIRST = 50.52
OPS_FIX_EXTRA = 5.0
OPS_FP64_BASE = 488.9
OPS_FP64_LINE = 158.8
BYTES_PER_VOXEL_FP64 = 4 * 6 * 8          # eps, z_n in; sigma, z out
# DRAM bytes of one full-size FP32-bulk launch (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, one capture of launch 6 of this workload: the
# inputs are read once, less what the 129 MB L2 still holds)
TRAFFIC_FP32FIX = 1476579840 + 1630033408


# The paper's own figures for this path (context, other hardware and workload:
# a 150^3 short-fibre metal-matrix composite, 80 load steps, 1681 elasticity
# iterations with implicit Euler, FP64, 2x Intel Xeon E5-2687Wv4 (24 cores)
# + NVIDIA Quadro GV100 over PCIe, the FFT solver on the CPU; Sec. 3 and the
# timing tables of Sec. 6).  Voxel-update rates are derived from the totals:
# 1681 x 150^3 evaluations / the material-law time (host staging included).
PAPER_FIGURES = {
    "hardware": "2x Intel Xeon E5-2687Wv4 (24 cores) + NVIDIA Quadro GV100, FP64",
    "workload": "150^3 short-fibre metal-matrix composite, 80 load steps, 1681 iterations, implicit Euler",
    "material_law_no_tangent_automatic_s": {"cpu": 4996.7, "gpu": 257.7},
    "material_law_no_tangent_conventional_s": {"cpu": 830.1, "gpu": 249.7},
    "derived_voxel_updates_per_s_automatic": {"cpu": 1681 * 150 ** 3 / 4996.7, "gpu": 1681 * 150 ** 3 / 257.7},
    "total_homogenization_automatic_with_reference_update_s": {"cpu": 6282.41, "gpu": 541.88},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-probe", action="store_true", help="skip the SIMT FMA-throughput probe")
    ap.add_argument("--no-ms", action="store_true", help="skip the basic-scheme measurement")
    ap.add_argument("--voxels", type=int, default=N_VOX, help="batch size (profiling runs use a small batch)")
    ap.add_argument("--h", type=float, default=H_STEP, help="step size of the material batch (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--adjoint-converged", action="store_true",
                    help="also run the adjoint workload to convergence (six gradients; minutes)")
    ap.add_argument("--no-ode23", action="store_true", help="skip the ODE material-update measurements")
    ap.add_argument("--ode-voxels", type=int, default=1 << 22,
                    help="voxels of the ODE measurements (profiling runs use a small batch)")
    ap.add_argument("--no-mmc", action="store_true", help="skip the MMC scheme run of the ODE measurements")
    ap.add_argument("--ms-n", type=int, default=256, help="grid of the basic-scheme measurement (profiling: 128)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the homogenization-setting scheme runs")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-jobs", type=int, default=0, help="jobs of the serving stream (default 64; sample 16)")
    ap.add_argument("--serve-sample", action="store_true",
                    help="serve a bounded sample of the stream (grids <= 96^3, 2-5 steps) instead of the full stream")
    ap.add_argument("--serve-tol", type=float, default=1e-4, help="equilibrium tolerance of every serving arm")
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


def _status_fields(status, model=False):
    import numpy as np
    line = (status & 0xFF).astype(np.float64)
    newton = ((status >> 8) & 0xFF).astype(np.float64)
    fix = ((status >> 20) & 0xF).astype(np.float64)
    if model:
        return line, newton, fix, ((status >> 24) & 0x7F).astype(np.float64)
    return line, newton, fix


def ops_per_voxel(status, mode):
    """Mean executed FP64 operations per voxel from the kernel's status words."""
    import numpy as np
    line, newton, fix = _status_fields(status)
    if mode == "fp64":
        f = OPS_FP64_BASE + OPS_FP64_LINE * line
        return float(f.mean()), float(line.mean()), float(newton.mean())
    f = (OPS_FIX_FIRST + OPS_FIX_EXTRA * np.maximum(fix - 1, 0)) * (fix > 0)
    return float(f.mean()), float(line.mean()), float((newton - fix).mean()), float(fix.mean())


def alg_flops_per_voxel(status, mode):
    """Mean algorithmic flops per voxel: (FP64 flops, FP32 flops, FP64 pows, FP32 pows).

    FP64 mode: predictor + line x (one 1-D search step) + newton x (one
    Newton step) + stress, all FP64.  FP32 bulk + FP64 correction: the
    predictor, search and Newton steps of the FP32 solve are FP32; each FP64
    correction is an FP64 residual sweep, substitutions with the FP32 factor
    (FP32) and w += dw (5 FP64 adds); the stress is FP64."""
    line, newton, fix, model = _status_fields(status, model=True)
    A, W = ALG_FLOPS, ALG_POWS
    if mode == "fp64":
        step64 = model > 0
        f64 = A["predictor"] + A["line"] * line + A["newton"] * newton + A["stress"] + MODEL64_FLOPS * step64
        p64 = W["line"] * line + W["newton"] * newton + MODEL64_POWS * step64
        return float(f64.mean()), float((MODEL_FLOPS * model).mean()), float(p64.mean()), \
            float((MODEL_POWS * model).mean())
    bulk = newton - fix
    f32 = A["predictor"] + A["line"] * line + A["newton"] * bulk + A["subst"] * fix + MODEL_FLOPS * model
    p32 = W["line"] * line + W["newton"] * bulk + MODEL_POWS * model
    f64 = (A["residual"] + 5) * fix + A["stress"]
    p64 = W["residual"] * fix
    return float(f64.mean()), float(f32.mean()), float(p64.mean()), float(p32.mean())


def bench_simt_peaks(G, torch):
    """Measured FMA throughput of the SIMT pipes (gsm_peak_probe): FP64 and
    FP32, best of three launches of ~0.1-0.2 s each, CUDA events on the
    launching stream, with the SM clock sampled during the probe."""
    stream = torch.cuda.current_stream()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    out = {}
    for name, prec, iters in (("fp64", 0, 40000), ("fp32", 1, 2000000)):
        G.peak_probe(prec, iters // 20)
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fmas = G.peak_probe(prec, iters)
            b.record(stream)
            torch.cuda.synchronize()
            best = max(best, 2.0 * fmas / (a.elapsed_time(b) * 1e-3) / 1e9)
        out[name + "_gflops"] = best
    out["clocks"] = clocks.stop()
    out["how"] = ("gsm_peak_probe: (SM count x 4) blocks x 512 threads x 8 independent FMA chains, "
                  "best of 3 launches, 2 flops per FMA")
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def run_ours(args):
    global N_VOX, H_STEP
    N_VOX = args.voxels
    H_STEP = args.h
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
    if rank == 0 and not args.no_probe:
        results["simt"] = bench_simt_peaks(G, torch)

    e2e_ms = None
    if not args.no_e2e:
        e2e_ms = bench_e2e(G, torch, np, eps, zn, e, z0, sig, z, st, stream, world, args)

    # With several ranks (the scaling run) only the headline material update
    # and its end-to-end path run: the other blocks are single-GPU measurements.
    if world > 1:
        args.no_ms = args.no_serve = args.no_adjoint = args.no_ode23 = args.no_cpu = True
    ms_block = None
    if not args.no_ms and rank == 0:
        ms_block = bench_ms(G, torch, args)
    serve_block = None
    if not args.no_serve and rank == 0:
        serve_block = bench_serve(G, args)
    adj_block = None
    if not args.no_adjoint and rank == 0:
        adj_block = bench_adjoint(G, torch)
        if args.adjoint_converged:
            adj_block["converged"] = bench_adjoint_converged(G, torch)
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
    h_st = torch.empty(N_VOX, dtype=torch.int32).pin_memory()

    # every way writes the same outputs as the device-timed arm: sigma, z and the status words
    def zero_copy():
        G.gsm_update(mat, h_eps, h_zn, H_STEP, h_sig, h_z, None, h_st)

    def streamed():
        G.gsm_update_host(mat, h_eps, h_zn, H_STEP, h_sig, h_z, None, h_st)

    def staged():
        e.copy_(h_eps, non_blocking=True)
        z0.copy_(h_zn, non_blocking=True)
        G.gsm_update(mat, e, z0, H_STEP, sig, z, None, st)
        h_sig.copy_(sig, non_blocking=True)
        h_z.copy_(z, non_blocking=True)
        h_st.copy_(st, non_blocking=True)

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
            "h2d_bytes_per_step": 2 * 6 * 8 * N_VOX, "d2h_bytes_per_step": (2 * 6 * 8 + 4) * N_VOX,
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
    simt = results.get("simt") or {}
    r64, r32 = results["fp64"], results["fp32fix"]
    fpv, line64, newton64 = ops_per_voxel(r64["status"], "fp64")
    fpv32, line32, newton32, fix32 = ops_per_voxel(r32["status"], "fp32fix")
    a64_64, _, pw64_64, _ = alg_flops_per_voxel(r64["status"], "fp64")
    a32_64, a32_32, pw32_64, pw32_32 = alg_flops_per_voxel(r32["status"], "fp32fix")
    t64 = r64["per_launch_ms"] * 1e-3
    t32 = r32["per_launch_ms"] * 1e-3
    sm_mhz = (results.get("clocks") or {}).get("sm_mhz") or 2070.0
    issue_peak = FP64_ISSUE_PER_SM_CLK * 152 * sm_mhz * 1e-3  # G FP64 ops/s at the run's median clock
    P64 = simt.get("fp64_gflops")
    P32 = simt.get("fp32_gflops")
    src = "measured in this run by gsm_peak_probe (FMA chains), 2 flops per FMA"
    if not P64:  # the probe did not run (a profiling run): nominal rates at the run's clock
        P64 = 2 * FP64_ISSUE_PER_SM_CLK * 152 * sm_mhz * 1e-3
        P32 = 2 * 128 * 152 * sm_mhz * 1e-3
        src = "not measured in this run: nominal 2 FP64 / 128 FP32 FMA per SM per cycle at the run's median clock"
    ach64 = a32_64 * N_VOX / t32 / 1e9
    ach32 = a32_32 * N_VOX / t32 / 1e9
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
        "roofline": {"kernel": "norton_kernel<MODE_FP32_FIX>", "bound": "alu", "achieved": ach64,
                     "peak": P64, "unit": "G FP64 FLOP/s", "frac": ach64 / P64,
                     "traffic": TRAFFIC_FP32FIX,
                     "peak_source": src,
                     "alg_fp64_flops_per_voxel": a32_64, "alg_fp64_pow_per_voxel": pw32_64,
                     "alg_fp32_flops_per_voxel": a32_32, "alg_fp32_pow_per_voxel": pw32_32,
                     "fp32_achieved": ach32, "fp32_peak": P32, "fp32_frac": ach32 / P32,
                     "note": "achieved = algorithmic FP64 flops of the FP64 corrections and the stress (oracle "
                             "counts x the kernel's iteration counts; pow counted apart) / mean launch time; the FP32 "
                             "solve runs on the FP32 pipe (fp32_*)",
                     "executed_fp64_ops_per_voxel": fpv32,
                     "issue_frac": fpv32 * N_VOX / t32 / 1e9 / issue_peak,
                     "hbm_frac": BYTES_PER_VOXEL_FP64 * N_VOX / t32 / 1e9 / peaks.get("hbm_gbs", 6783.1)},
        "roofline_fp64_mode": {"kernel": "norton_kernel<MODE_FP64>", "bound": "alu",
                               "achieved": a64_64 * N_VOX / t64 / 1e9, "peak": P64, "unit": "G FP64 FLOP/s",
                               "frac": a64_64 * N_VOX / t64 / 1e9 / P64,
                               "alg_fp64_flops_per_voxel": a64_64, "alg_fp64_pow_per_voxel": pw64_64,
                               "executed_fp64_ops_per_voxel": fpv,
                               "issue_frac": fpv * N_VOX / t64 / 1e9 / issue_peak},
        "simt_peaks": simt or None,
        "paper_figures": PAPER_FIGURES,
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
    """Basic-scheme iterations/s at 256^3 (--ms-n) (fibre composite), FP64 and FP32 bulk.

    iters_per_s: the steady-state rate of the first load step's iterations,
    from the difference of two forced runs (12 and 42 FP32-bulk iterations,
    4 and 10 FP64 ones), so that the step start and the FP32-bulk run's final
    FP64 iteration drop out; run_iters_per_s: a whole run of 30 forced
    iterations.  Both precisions then run 30 forced iterations from the same
    start, and the FP32-bulk result's deviation from the FP64 one (effective
    stress; sigma, eps and z fields relative to their maxima) is reported."""
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
    fields = {}
    for name, prec, law_prec, (k0, k1) in (("fp64", G.MS_PREC_FP64, G.GSM_FP64, (4, 10)),
                                           ("fp32_bulk", G.MS_PREC_FP32_BULK, G.GSM_FP32_FP64FIX, (12, 42))):
        laws = [G.norton(*synth.MATRIX_256, precision=law_prec), G.elastic(*synth.FIBRE_256)]
        ctx = G.ms_create(phase, laws, prec)
        G.ms_run(ctx, loads[:1], hs[:1], forced_iters=[3])  # warm-up
        t = {}
        for k in (k0, k1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.ms_run(ctx, loads[:1], hs[:1], forced_iters=[k])
            torch.cuda.synchronize()
            t[k] = time.perf_counter() - t0
        n_it = 30
        eps = torch.zeros(6, N ** 3, dtype=torch.float64, device="cuda")
        z = torch.zeros_like(eps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = G.ms_run(ctx, loads[:1], hs[:1], forced_iters=[n_it], eps=eps, z=z)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"iters_per_s": (k1 - k0) / (t[k1] - t[k0]), "run_iters_per_s": n_it / dt, "iters": n_it,
                     "fp32_iters": int(out["fp32_iters"][0]), "final_error": float(out["final_error"][0]),
                     "law": "FP64" if law_prec == G.GSM_FP64 else "FP32 Newton + FP64 correction"}
        fields[name] = (out["Sigma"][0], eps, z)
        G.ms_destroy(ctx)
    # FP32 bulk against FP64 after the same 30 iterations
    S64, e64, z64 = fields["fp64"]
    S32, e32, z32 = fields["fp32_bulk"]

    def stiff(E, nu):
        lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
        C = torch.zeros(6, 6, dtype=torch.float64, device="cuda")
        C[:3, :3] = lam
        C[:3, :3] += 2 * mu * torch.eye(3, dtype=torch.float64, device="cuda")
        C[3:, 3:] = mu * torch.eye(3, dtype=torch.float64, device="cuda")
        return C

    fib = phase.reshape(-1).bool()
    Cm, Cf = stiff(*synth.MATRIX_256[:2]), stiff(*synth.FIBRE_256)

    def sigma(e, zz):
        return torch.where(fib[None, :], Cf @ (e - zz), Cm @ (e - zz))

    def rel(a, b):
        return float((a - b).abs().max() / b.abs().max())

    res["fp32_bulk_vs_fp64"] = {
        "after": "30 forced iterations of the first load step (FP32 bulk: 29 FP32 + 1 FP64)",
        "Sigma": float(np.max(np.abs(S32 - S64)) / np.max(np.abs(S64))),
        "sigma": rel(sigma(e32, z32), sigma(e64, z64)), "eps": rel(e32, e64), "z": rel(z32, z64)}
    del fields, e64, z64, e32, z32
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


def bench_adjoint_converged(G, torch, tol=1e-8):
    """The adjoint workload to convergence: 128^3 centred sphere (20 %), Norton
    matrix, uniaxial ramp to 1 % in 10 steps of h = 0.1, FP64; the forward
    run to e < tol with the per-step reference medium, then the gradient of
    each of the six effective-stress components with respect to (E, sigma0, n)
    (six adjoint sweeps, each step's equilibrium to tol).  Minutes; run with
    --adjoint-converged."""
    import numpy as np
    import synth
    N, steps = 128, 10
    ph = synth.sphere_phase(N, 0.2)
    phase = torch.from_numpy(ph).cuda()
    loads = synth.ramp(steps, [0.01, 0, 0, 0, 0, 0])
    hs = [0.1] * steps
    ctx = G.ms_create(phase, [G.norton(*synth.MATRIX_16), G.elastic(*synth.INCLUSION_16)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, tape = G.ms_run_taped(ctx, loads, hs, tol=tol, max_iter=100000, ref_update=True)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    grads, adj_iters, t_adj = [], [], []
    for c in range(6):
        w = np.zeros(6)
        w[c] = 1.0
        t1 = time.perf_counter()
        g, its = G.ms_adjoint(tape, w, 0, tol=tol, max_iter=100000, check=False)
        torch.cuda.synchronize()
        t_adj.append(time.perf_counter() - t1)
        grads.append([float(x) for x in g])
        adj_iters.append(int(np.sum(its)))
    del tape
    G.ms_destroy(ctx)
    total = t_fwd + sum(t_adj)
    return {"workload": f"{N}^3 centred sphere 20 %, Norton matrix n=5, uniaxial ramp to 1 % in {steps} steps of "
                        f"h=0.1, FP64, per-step reference from tangents, forward and adjoints to tol {tol}",
            "forward_s": t_fwd, "forward_iters": int(np.sum(res["iters"])), "forward_rc": int(res["rc"]),
            "adjoint_s": t_adj, "adjoint_iters": adj_iters,
            "gradient_s": total, "gradients_per_s": 1.0 / total,
            "dSigma_dtheta": grads, "theta": "(E, sigma0, n) of the matrix"}


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
    """Serving the homogenization stream against one-job-at-a-time paths.

    Workload: the serving stream of 64 jobs (synth.serving_stream, seed 7):
    grids {32, 64, 96, 128, 192}^3, RSA spheres (5-25 %) or cylinders
    (10-30 %), Norton matrix n in {3, 5, 10}, random unit load directions
    with 1-2 % amplitude over 5-20 steps (--serve-sample: a bounded 16-job
    sample with grids <= 96^3 and 2-5 steps).  Every path solves each job to
    e < tol (default 1e-4, which holds the effective stress within 1e-6 of
    the converged FP64 result; tests/test_gpu_serve.py).

    * sequential FP32 bulk: ms_solve per job, the server's own precision
      path one job at a time (run);
    * served: Poisson arrivals at 1.5 / (mean sequential FP32-bulk service
      time), the serving engine with continuous batching and fair-share ticks
      (run, wall clock on the host);
    * sequential FP64: the plain FP64 path.  Running it on the whole stream
      takes about two hours (an FP64 iteration costs ~20 FP32-bulk ones on
      GB300), so its service times are modelled: each job's FP64 time per
      iteration (the steady-state rate of forced runs of 10 and 30
      iterations, measured) x the job's iteration count in the FP32-bulk run.
      One job per grid size (the one with the fewest load steps) runs in
      full in FP64; the ratio of its measured to its modelled time scales
      the model of the other jobs of that size (the forced runs sit early in
      a load step, where the warm-started Newton needs more steps, and the
      FP32-bulk counts exceed FP64's by ~10 %: the raw model overstates the
      FP64 time by 30-60 %).  Raw and calibrated totals, the ratios and the
      effective-stress agreement of those jobs are reported.
    Latencies of the sequential arms: FIFO queue over the same arrivals.
    """
    import numpy as np
    import synth
    from paper_2006_04391_gb300 import serving
    tol = args.serve_tol
    workers = max(1, min(16, os.cpu_count() or 1))
    if args.serve_sample:
        jobs = synth.serving_stream(args.serve_jobs or 16, seed=7, grids=(32, 64, 96), steps=(2, 5),
                                    workers=workers)
    else:
        jobs = synth.serving_stream(args.serve_jobs or 64, seed=7, workers=workers)
    n = len(jobs)
    t0 = time.perf_counter()
    seq32 = serving.run_sequential(G, jobs, tol=tol, ms_precision=G.MS_PREC_FP32_BULK,
                                   law_precision=G.GSM_FP32_FP64FIX)
    t_seq32 = time.perf_counter() - t0
    s32 = np.array([r["service_s"] for r in seq32])
    rate = 1.5 / s32.mean()
    arrivals = serving.poisson_arrivals(n, rate, seed=11)
    budget = 200 << 30
    stream = serving.run_stream(G, jobs, arrivals, hbm_budget=budget, max_active=64, tol=tol)
    # served = sequential FP32 bulk, bit for bit (a job's arithmetic does not depend on the mix)
    same = all(np.array_equal(r["Sigma"], q["Sigma"]) for r, q in zip(stream["jobs"], seq32))
    # sequential FP64, modelled from measured per-iteration times
    t_it64 = serving.iteration_times(G, jobs)
    iters = np.array([int(np.sum(q["iters"])) for q in seq32])
    s64_raw = t_it64 * iters
    # calibration and check: a full FP64 run of the job with the fewest load steps of every grid
    # size; each grid's measured / modelled ratio scales the model of its other jobs
    grids = sorted(set(j["N"] for j in jobs))
    small = [min((i for i, j in enumerate(jobs) if j["N"] == N), key=lambda i: len(jobs[i]["h"])) for N in grids]
    val = serving.run_sequential(G, [jobs[i] for i in small], tol=tol)
    val_s = np.array([r["service_s"] for r in val])
    factor = {jobs[i]["N"]: float(ms_ / s64_raw[i]) for i, ms_ in zip(small, val_s)}
    s64 = np.array([s64_raw[i] * factor[j["N"]] for i, j in enumerate(jobs)])
    for i, ms_ in zip(small, val_s):
        s64[i] = ms_  # the calibration jobs keep their measured service times
    val_sigma = max((float(np.max(np.abs(stream["jobs"][i]["Sigma"] - r["Sigma"])))
                     / max(float(np.max(np.abs(r["Sigma"]))), 1e-300) for i, r in zip(small, val)), default=0.0)
    lat32 = serving.fifo_completion(arrivals, s32) - arrivals
    lat64 = serving.fifo_completion(arrivals, s64) - arrivals
    vox = float(sum(int(np.sum(q["iters"])) * j["N"] ** 3 for q, j in zip(seq32, jobs)))
    served_jps = n / stream["makespan_s"]
    return {
        "workload": (f"{n} jobs, grids {sorted(set(j['N'] for j in jobs))}, "
                     f"{sum(len(j['h']) for j in jobs)} load steps in total, "
                     + ("bounded sample (grids <= 96^3, 2-5 steps)" if args.serve_sample
                        else "the full serving stream (grids 32-192^3, 5-20 steps)")
                     + f", Poisson arrivals at {rate:.4f}/s = 1.5 x the sequential FP32-bulk rate, tol {tol}"),
        "served": {"latency_p50_s": stream["latency_p50"], "latency_p99_s": stream["latency_p99"],
                   "makespan_s": stream["makespan_s"], "jobs_per_s": served_jps,
                   "voxel_updates_per_s": vox / stream["makespan_s"], "ticks": stream["ticks"],
                   "max_active": stream["max_active"], "bit_identical_to_sequential_fp32": same,
                   "path": "FP32 bulk fields/FFTs, FP64 finish with FP32-Newton + FP64-fix laws, batched fair-share "
                           "ticks"},
        "sequential_fp32_bulk": {"latency_p50_s": float(np.percentile(lat32, 50)),
                                 "latency_p99_s": float(np.percentile(lat32, 99)),
                                 "jobs_per_s": n / float(s32.sum()), "busy_s": float(s32.sum()),
                                 "voxel_updates_per_s": vox / float(s32.sum()), "measured": "run, all jobs"},
        "sequential_fp64": {"latency_p50_s": float(np.percentile(lat64, 50)),
                            "latency_p99_s": float(np.percentile(lat64, 99)),
                            "jobs_per_s": n / float(s64.sum()), "busy_s": float(s64.sum()),
                            "busy_s_uncalibrated": float(s64_raw.sum()),
                            "measured": "modelled: per-job FP64 s/iteration (measured) x the FP32-bulk iteration "
                                        "count, scaled per grid size by a full FP64 run of one job of that size",
                            "model_check": {"jobs": len(small), "grids": [int(jobs[i]["N"]) for i in small],
                                            "measured_s": [float(x) for x in val_s],
                                            "modelled_s": [float(s64_raw[i]) for i in small],
                                            "factor": {str(k): v for k, v in factor.items()},
                                            "fp64_iters": int(sum(int(np.sum(r["iters"])) for r in val)),
                                            "fp32_bulk_iters": int(iters[small].sum()),
                                            "max_rel_sigma_served_vs_fp64": val_sigma}},
        "throughput_ratio": {"served_vs_sequential_fp32_bulk": served_jps / (n / float(s32.sum())),
                             "sequential_fp32_bulk_vs_fp64": float(s64.sum()) / float(s32.sum()),
                             "served_vs_sequential_fp64": served_jps / (n / float(s64.sum()))},
        "bench_s": time.perf_counter() - t0,
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
