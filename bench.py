"""Benchmark of the FFT phase-field-fracture hot path on GB300.

A step is one dissipation increment (the whole staggered solve: equilibrium CG, damage PCG,
control root search, Anderson mixing, history and load-curve update) of the 512^2 fibre
composite RVE (30% discs of radius 20, E_f/E_m = 5, Gc_f/Gc_m = 2, l = 3, central enriched
crack of 64 voxels). Metric: voxel-updates/s = sum over (equilibrium-CG + damage-PCG iterations)
x voxels, per second. The headline runs the plain FP64 path; the FP32 path with iterative
refinement runs beside it on the same RVE and the same number of increments.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32r] [--impl reference]

N > 1 runs one independent RVE replica per rank (the solve of one RVE does not shard; replicas
only). Timing: W untimed increments, then K increments each bracketed by CUDA events on the
library's stream; between timed increments L2 is flushed by writing 256 MiB; barrier +
synchronize around the timed region, max over ranks. The same K increments are then replayed
from a checkpoint of the warm-up state twice: once with per-kernel CUDA events (the kernel
breakdown and the roofline of the dominant kernel class) and once end to end through the C ABI
from pinned host memory (rve_load of the state, the increment, rve_save of the new state).
One JSON line on rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
WORKLOAD = "fibre_composite_512"
METRIC = "FFT-PFF voxel-updates/s"

# DRAM bytes per launch of a kernel, from ncu captures of the current kernel code (dram__bytes_
# read.sum + dram__bytes_write.sum of the captured launch), keyed by (workload, precision, kernel
# class). A kernel without a capture of its current code reports null; an entry is removed when
# the kernel it describes changes.
TRAFFIC = {
    ("fibre_composite_512", "fp64", "projection_pass"): 6432256 + 0,
    ("polycrystal_3d_128", "fp32r", "projection_pass"): 56673536 + 2820608,
}
TRAFFIC_SOURCE = {
    ("fibre_composite_512", "fp64", "projection_pass"):
        "ncu --set full, one launch of k_axis<double,3,3,FWD_OP_INV,OpProj> in `bench.py --steps 1 --warmup 3` "
        "(cold caches: the read half comes from DRAM, the writes stay in L2)",
    ("polycrystal_3d_128", "fp32r", "projection_pass"):
        "ncu --set full, one launch of k_axis<float,6,6,FWD_OP_INV,OpProj> in "
        "`bench.py --workload polycrystal_3d_128 --precision fp32r --steps 1 --warmup 3` (cold caches)",
}


def workload_desc(name=WORKLOAD):
    return WORKLOADS[name]


def peaks():
    try:
        with open(MEASURED) as f:
            m = json.load(f)
        return m, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WORKLOADS = {
    "fibre_composite_512": "512x512 plane-strain fibre composite, RSA discs r=20 at 30% voxel fraction, E_f/E_m=5, "
                           "Gc_f/Gc_m=2, nu=0.3, l=3, k=1e-6, central CTE crack 64 voxels (phi_M=0.8), "
                           "dtau=1.5*Gc*A_g/300, f=e_y(x)e_y",
    "homogeneous_plate_64": "64x64 plane-strain homogeneous plate, E=1, nu=0.3, Gc=1, l=2, spectral split, CTE crack "
                            "16 voxels at mid-height, dtau=1.5*Gc*A_g/100",
    "polycrystal_1024": "1024x1024 periodic Voronoi polycrystal, 200 grains, cubic C11=1 C12=0.6 C44=0.5 (Zener 2.5), "
                        "uniform in-plane orientations, cleavage beta=2, l=2, CTE crack 102 voxels, dtau=1.5*A_g/400",
    "polycrystal_plate_256": "256x128x1 polycrystal plate (six strain components), 60 Laguerre grains with lognormal "
                             "size spread 0.25, SO(3)-uniform orientations, cubic C1111:C1122=24:8 with Zener 4, "
                             "cleavage beta=2, l=2, CTE crack 26 voxels, dtau=1.5*A_g/200",
    "polycrystal_3d_128": "128^3 periodic Voronoi polycrystal, 150 grains, cubic C11=1 C12=0.6 C44=0.5 with "
                          "SO(3)-uniform orientations, lognormal Gc (sigma 0.3), l=2, through CTE crack 13 voxels, "
                          "dtau=1.5*<Gc>*A_g/100 (the largest RVE of the batched 3D mix, alone)",
    "batched_3d_polycrystals": "16 periodic Voronoi 3D polycrystals, grids drawn from {32,64,128}^3, 50-200 grains, "
                               "cubic C11=1 C12=0.6 C44=0.5 with SO(3)-uniform orientations, lognormal Gc (sigma 0.3), "
                               "l=2, through CTE crack 0.1 n, dtau=1.5*<Gc>*A_g/100; lockstep batches per grid class",
}


def make_workload(rank, precision, name=WORKLOAD):
    import synth
    if name == "homogeneous_plate_64":
        w = synth.homogeneous_plate_64()
    elif name == "polycrystal_1024":
        w = synth.polycrystal_1024(seed=2 + rank)
    elif name == "polycrystal_plate_256":
        w = synth.polycrystal_plate_256(seed=5 + rank)
    elif name == "polycrystal_3d_128":
        w = synth.polycrystal_3d(128, 150, 9 + rank)
    else:
        w = synth.fibre_composite_512(seed=1 + rank)
    w.precision = precision
    return w


def solver_tols(precision):
    """Solver tolerances of the benchmark runs. FP32R: the equilibrium is refined on its FP64
    residual to 1e-7, the FP32 damage solve, the control root and the staggered loop stop at
    1e-6 / 1e-7 / 1e-6 (the settings
    whose accuracy the FP32R parity tests check against the FP64 oracle)."""
    if precision == "fp64":
        return dict(tol_stag=1e-8)
    return dict(tol_mech=1e-7, tol_dmg=1e-6, tol_root=1e-7, tol_stag=1e-6)


def _finite(obj):
    """JSON has no NaN / Infinity: report such values as null."""
    import math
    if isinstance(obj, float):
        return obj if math.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: _finite(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [_finite(v) for v in obj]
    return obj


def aggregate_over_ranks(ms, vu, world, device):
    """Job-wide timing of replicas: the slowest rank's time (MAX) and all ranks' voxel-updates
    (SUM). No data-path collective: each rank solves its own RVE."""
    if world <= 1:
        return ms, vu
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms), float(vu)], device=device, dtype=torch.float64)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0].item()), float(t[1].item())


def cufft_reference(torch, stream, g, w, precision):
    """cuFFT (through torch.fft) timed beside the library's own transforms, as a reference only.

    Ours: one equilibrium CG iteration, i.e. three fused passes (CG update + stress + x FFT; y FFT +
    projection + inverse y FFT; inverse x FFT + CG vector + dot products), timed over a whole
    solve from a zero fluctuation and divided by its iterations. cuFFT: the forward and inverse
    real 2D FFT of the same three-component field alone, without the projection, the stress or
    the CG arithmetic."""
    import numpy as np
    from paper_2508_07424_gb300 import capi
    nx, ny = w.micro.n[0], w.micro.n[1]
    g.set(capi.RVE_FIELD_FLUCT1, np.zeros((3, ny, nx)))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = g.mech_solve()
    e1.record(stream)
    torch.cuda.synchronize()
    ours_us = e0.elapsed_time(e1) * 1e3 / max(iters, 1)
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = torch.randn(3, ny, nx, dtype=dt, device="cuda")
    for _ in range(3):
        torch.fft.irfft2(torch.fft.rfft2(x), s=(ny, nx))
    reps = 50
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        y = torch.fft.irfft2(torch.fft.rfft2(x), s=(ny, nx))
    e1.record(stream)
    torch.cuda.synchronize()
    del y
    return {"what": f"cuFFT rfft2 + irfft2 of a 3 x {ny} x {nx} {dt} field (torch.fft), no operator",
            "cufft_us": e0.elapsed_time(e1) * 1e3 / reps,
            "ours_us_per_mech_iteration": ours_us, "ours_iterations": iters,
            "ours_what": "one equilibrium CG iteration: 3 fused passes incl. both FFTs, the projection, "
                         "the stress, the CG updates and dot products (solve from zero / iterations)"}


class PinnedState:
    """A checkpoint of one RVE in pinned host memory (rve_save / rve_load through the C ABI)."""

    def __init__(self, torch, g, extra_curve=64):
        import ctypes as C
        from paper_2508_07424_gb300 import capi
        self.C, self.capi, self.g = C, capi, g
        n = C.c_size_t()
        capi.check(capi.lib().rve_save(g.h, None, C.byref(n)), "rve_save")
        # room for the load curve growing by extra_curve increments
        cap = n.value + extra_curve * C.sizeof(capi.rve_step_result)
        self.buf = torch.empty(cap, dtype=torch.uint8).pin_memory()
        self.n = 0

    def save(self):
        n = self.C.c_size_t(self.buf.numel())
        self.capi.check(self.capi.lib().rve_save(self.g.h, self.C.c_void_p(self.buf.data_ptr()), self.C.byref(n)),
                        "rve_save")
        self.n = n.value
        return self.n

    def load(self):
        self.capi.check(self.capi.lib().rve_load(self.g.h, self.C.c_void_p(self.buf.data_ptr()), self.n), "rve_load")

    def copy_from(self, other):
        self.buf[:other.n].copy_(other.buf[:other.n])
        self.n = other.n


def fp64_peak(torch, stream):
    """Measured FP64 FMA rate of this GPU (TFLOP/s), with the SM clock seen meanwhile."""
    import ctypes as C
    from paper_2508_07424_gb300 import capi
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    best = 0.0
    for _ in range(3):
        tf, ms = C.c_double(), C.c_double()
        capi.check(capi.lib().rve_fp64_fma_rate(20000, C.byref(tf), C.byref(ms), C.c_void_p(stream.cuda_stream)),
                   "rve_fp64_fma_rate")
        best = max(best, tf.value)
    c = clk.stop()
    return {"tflops": best, "sm_mhz": c.get("sm_mhz"), "how": "rve_fp64_fma_rate: 8 blocks/SM x 256 threads, "
            "8 independent FMA chains per thread, CUDA events; best of 3 launches of ~1.5 s"}


KERNEL_CLASSES = ("k_axis", "k_x_fwd", "k_x_inv", "k_x_mid", "k_pointwise", "fp64_residual", "cg_x_fwd", "cg_x_inv")


def same_result(a, b):
    """Bitwise equality of two step records (NaN equal to NaN: G_inst is NaN when Gamma stays)."""
    import math
    for k in a:
        x, y = a[k], b[k]
        if isinstance(x, float) and math.isnan(x) and isinstance(y, float) and math.isnan(y):
            continue
        if x != y:
            return False
    return True


def kernel_breakdown(torch, stream, g, w, state, steps):
    """Replay the timed increments from the checkpoint with CUDA events around every launch.
    Returns per kernel class: launches and ms per increment, share of the replayed increment,
    algorithmic bytes / FFT flops per launch and the rates they give; plus the mechanics
    projection pass on its own. The replay launches plainly (no CUDA graphs), so its increment
    time is longer than the timed loop's."""
    state.load()
    g.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # a profiler cannot see the kernels inside conditional graphs, so its launch list is taken
    # over this replay of the same increments (plain launches), marked by an NVTX range
    nvtx_push("kernel_breakdown")
    e0.record(stream)
    results = [g.step(w.dtau) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    nvtx_pop()
    kinds = g.timing_kinds()
    g.timing(False)
    wall = e0.elapsed_time(e1)
    out = {"replay_ms_per_step": wall / steps, "classes": {}}
    for name in KERNEL_CLASSES + ("projection_pass",):
        ms, n, b, f = kinds[name]
        if not n:
            continue
        out["classes"][name] = {
            "launches_per_step": n / steps, "ms_per_step": ms / steps, "share": ms / wall,
            "avg_launch_us": ms * 1e3 / n, "bytes_per_launch": b, "flops_per_launch": f,
            "GB_s": b * n / (ms * 1e-3) / 1e9, "TFLOP_s": f * n / (ms * 1e-3) / 1e12 if f else None}
    out["timed_kernel_share"] = kinds["all"][0] / wall
    return out, results


def roofline_of(bd, precision, workload, hbm_peak, hbm_src, f64):
    """Roofline of the dominant kernel: the one with the largest time per increment in the replay.
    The library times each kernel template as a class (k_axis, k_x_fwd, k_x_inv, ...) and, on
    their own, three single kernels whose every launch does the same work: the mechanics
    projection pass (inside k_axis) and the two x passes of the equilibrium CG iteration (inside
    k_x_fwd / k_x_inv). Those stand for their templates; the FP64 residual class of the FP32 path
    mixes x and column passes and is not a candidate."""
    single = {"projection_pass": "k_axis", "cg_x_fwd": "k_x_fwd", "cg_x_inv": "k_x_inv"}
    have = bd["classes"]
    drop = {"fp64_residual"} | {tmpl for sub, tmpl in single.items() if sub in have}
    cls = {k: v for k, v in have.items() if k not in drop}
    dom = max(cls, key=lambda k: cls[k]["ms_per_step"])
    c = cls[dom]
    traffic = TRAFFIC.get((workload, precision, dom))
    if precision == "fp64":
        # The FP64 FFTs are bound by the FP64 FMA rate of this part (measured live), not by HBM.
        ach, peak = c["TFLOP_s"], f64["tflops"]
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": "measured in this run (rve_fp64_fma_rate)",
                "per_launch": "5 L log2 L flops per transformed line (FFT work only)",
                "hbm_GB_s": c["GB_s"], "hbm_frac": c["GB_s"] / hbm_peak}
    else:
        ach, peak = c["GB_s"], hbm_peak
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": hbm_src,
                "per_launch": "half-spectrum components read + written over nx/2+1 columns, plus the field words "
                              "of the fused prologue / epilogue"}
    name = {"projection_pass": "k_axis<OpProj> (mechanics projection pass)",
            "cg_x_fwd": "k_x_fwd<ProCGCG> (forward x pass of the equilibrium CG)",
            "cg_x_inv": "k_x_inv<EpiCGCG> (inverse x pass of the equilibrium CG)"}.get(dom, dom)
    roof.update({"kernel": name, "traffic": traffic, "traffic_source": TRAFFIC_SOURCE.get((workload, precision, dom)), "algorithmic_bytes": c["bytes_per_launch"],
                 "avg_launch_us": c["avg_launch_us"], "launches_per_step": c["launches_per_step"],
                 "share": c["share"],
                 "timing": "CUDA events around every launch on the library stream, the timed increments replayed "
                           "from a checkpoint without graphs"})
    return roof


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:  # an NVTX-less build: the range is only a profiling aid
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def timed_leg(torch, stream, w, precision, args, world, flush, e2e=True):
    """Warm-up, K device-timed increments, the kernel breakdown and the end-to-end replay of the
    same increments for one RVE in one precision."""
    from paper_2508_07424_gb300 import capi
    from paper_2508_07424_gb300.rve import Rve
    tol = solver_tols(precision)
    solver = capi.RVE_SOLVER_NEWTON if args.solver == "newton" else capi.RVE_SOLVER_STAGGERED
    w.precision = precision
    g = Rve.from_workload(w, stream=stream.cuda_stream, solver=solver, **tol)
    N = g.nvox
    for _ in range(args.warmup):
        g.step(w.dtau)
    torch.cuda.synchronize()
    state = PinnedState(torch, g, extra_curve=args.steps + 4)
    state.save()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    launches0 = g.launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    torch.cuda.synchronize()
    nvtx_push("timed_increments")  # lets a profiler select exactly the timed launches
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        results.append(g.step(w.dtau))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    nvtx_pop()
    if world > 1:
        torch.distributed.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    launches = g.launches() - launches0
    clk = clocks.stop()
    vu = sum((r["mech_iters"] + r["dmg_iters"]) * N for r in results)
    bd, replay = kernel_breakdown(torch, stream, g, w, state, args.steps)
    leg = {"ms": ms, "vu": vu, "results": results, "launches": launches, "clocks": clk, "breakdown": bd,
           "replay_same": [same_result(a, b) for a, b in zip(results, replay)], "N": N, "g": g}
    if e2e:
        # end to end through the public C ABI from pinned host memory: every step uploads the
        # committed state (fields, scalars, load curve) with rve_load, runs the increment and
        # reads the new state back with rve_save; the chain repeats the device-timed increments.
        work = PinnedState(torch, g, extra_curve=args.steps + 4)
        work.copy_from(state)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        e_res = []
        for _ in range(args.steps):
            h2d += work.n
            work.load()
            e_res.append(g.step(w.dtau))
            d2h += work.save()
        torch.cuda.synchronize()
        et = time.perf_counter() - t0
        evu = sum((r["mech_iters"] + r["dmg_iters"]) * N for r in e_res)
        leg["e2e"] = {"value": evu / et * world, "unit": "voxel-updates/s", "h2d_bytes_per_step": h2d // args.steps,
                      "d2h_bytes_per_step": d2h // args.steps, "steps": args.steps,
                      "same_increments_as_timed": all(same_result(a, b) for a, b in zip(results, e_res)),
                      "what": "per step: rve_load of the committed state from pinned host memory, step_dissipation, "
                              "rve_save of the new state (fields, scalars, load curve) to pinned host memory; host "
                              "wall clock, the same increments as the device-timed loop"}
    return leg


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2508_07424_gb300 import build
    build.build()
    stream = torch.cuda.current_stream()
    if args.workload == "batched_3d_polycrystals":
        return run_batched_3d(args, torch, stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    f64 = fp64_peak(torch, stream)
    w = make_workload(rank, args.precision, args.workload)
    legs = {}
    t_leg = time.perf_counter()
    leg = timed_leg(torch, stream, w, args.precision, args, world, flush, e2e=not args.no_e2e)
    legs["main"] = time.perf_counter() - t_leg
    tot_ms, tot_vu = aggregate_over_ranks(leg["ms"], leg["vu"], world, "cuda")
    if rank != 0:
        leg["g"].close()
        return None
    pk, src = peaks()
    roof = roofline_of(leg["breakdown"], args.precision, args.workload, pk["hbm_gbs"], src, f64)
    out = {
        "metric": METRIC,
        "value": tot_vu / (tot_ms * 1e-3),
        "unit": "voxel-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps,
        "voxel_increments_per_s": leg["N"] * args.steps * world / (tot_ms * 1e-3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": workload_config(args.workload, args.precision, args.solver, world),
        "increments": [{k: r[k] for k in ("n", "mech_iters", "dmg_iters", "stag_iters", "root_evals", "flags")}
                       for r in leg["results"]],
        "gpu_launches": int(leg["launches"]),
        "clocks": leg["clocks"],
        "roofline": roof,
        "kernels": leg["breakdown"],
        "replay_bit_identical": all(leg["replay_same"]),
        "fp64_fma_peak": f64,
        "e2e": leg.get("e2e"),
    }
    g = leg["g"]
    if world == 1 and w.micro.dim == 2:
        out["cufft_reference"] = cufft_reference(torch, stream, g, w, args.precision)
    g.close()
    if world == 1 and args.workload == WORKLOAD and args.precision == "fp64" and not args.no_side:
        t_leg = time.perf_counter()
        side = timed_leg(torch, stream, make_workload(rank, "fp32r", args.workload), "fp32r", args, 1, flush,
                         e2e=False)
        legs["fp32r_side"] = time.perf_counter() - t_leg
        out["fp32r_side_by_side"] = {
            "value": side["vu"] / (side["ms"] * 1e-3), "unit": "voxel-updates/s", "ms_per_step": side["ms"] / args.steps,
            "dtype": "f32", "steps": args.steps, "warmup": args.warmup, "clocks": side["clocks"],
            "increments": [{k: r[k] for k in ("n", "mech_iters", "dmg_iters", "stag_iters", "root_evals", "flags")}
                           for r in side["results"]],
            "roofline": roofline_of(side["breakdown"], "fp32r", args.workload, pk["hbm_gbs"], src, f64),
            "kernels": side["breakdown"]}
        side["g"].close()
    if not args.no_batch and world == 1 and args.workload == WORKLOAD:
        import synth
        ws = [make_workload(r, "fp32r", WORKLOAD) for r in range(8)]
        t_leg = time.perf_counter()
        out["batched_2d_fibre512_fp32r"] = batched_leg(torch, ws, "fp32r", 2, min(args.steps, 10),
                                                       solver_tols("fp32r"))
        legs["batched_2d"] = time.perf_counter() - t_leg
        out["batched_2d_fibre512_fp32r"]["what"] = ("8 fibre composites 512^2 (seeds 1-8), FP32R, one lockstep batch "
                                                    "(one launch per pass for all 8)")
        ws3 = synth.batched_3d_polycrystals()
        t_leg = time.perf_counter()
        out["batched_3d_polycrystals"] = batched_leg(torch, ws3, "fp32r", 1, min(args.steps, 3),
                                                     solver_tols("fp32r"))
        legs["batched_3d"] = time.perf_counter() - t_leg
        out["batched_3d_polycrystals"]["what"] = WORKLOADS["batched_3d_polycrystals"]
    if not args.no_cpu_baseline and world == 1 and args.workload == WORKLOAD:
        t_leg = time.perf_counter()
        out["cpu_baseline"] = cpu_baseline(args)
        legs["cpu_baseline"] = time.perf_counter() - t_leg
    if args.workload == "homogeneous_plate_64" and world == 1:
        out["toughness_run"] = toughness_run(args, stream)
    if not args.no_serve and world == 1 and args.workload == WORKLOAD:
        t_leg = time.perf_counter()
        out["serving"] = serving(args)
        legs["serving"] = time.perf_counter() - t_leg
    out["leg_wall_s"] = {k: round(v, 1) for k, v in legs.items()}
    return out


def workload_config(name, precision, solver, world):
    """The config object both arms print for a workload (no model keys)."""
    return {"workload": name, "desc": workload_desc(name), "precision": precision, "solver": solver,
            "step": "one dissipation increment", "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas{world}"}


def toughness_run(args, stream):
    """The 64^2 plate broken through: increments until the fracture point, G of Eq. (JaviGc)."""
    from paper_2508_07424_gb300.rve import Rve
    w = make_workload(0, args.precision, "homogeneous_plate_64")
    g = Rve.from_workload(w, stream=stream.cuda_stream, **solver_tols(args.precision))
    t0 = time.perf_counter()
    n = 0
    for _ in range(300):
        r = g.step(w.dtau)
        n = r["n"]
        if r["fractured"]:
            break
    dt = time.perf_counter() - t0
    out = {"increments": n, "fractured": bool(r["fractured"]), "wall_s": dt}
    if r["fractured"]:
        out["G_eff"] = g.toughness()
        out["G_eff_over_Gc"] = out["G_eff"] / 1.0
    g.close()
    return out


def batched_leg(torch, ws, precision, warmup, steps, tol):
    """Lockstep batching (rve_step_batch) against one-by-one stepping on the same RVEs and the
    same increments. The RVEs are grouped by grid; each group steps in lockstep from a thread of
    its own (groups of different grids run concurrently). After the warm-up every RVE is
    checkpointed; the batched run and the one-by-one run both start from the checkpoints, and
    every step record of the two runs must agree bit for bit."""
    import threading

    from paper_2508_07424_gb300.rve import Rve, step_batch
    t_setup = time.perf_counter()
    gs = []
    for w in ws:
        w.precision = precision
        gs.append(Rve.from_workload(w, **tol))
    classes = {}
    for i, w in enumerate(ws):
        classes.setdefault(tuple(w.micro.n), []).append(i)

    def run_classes(n_inc, out):
        def one(idx):
            for _ in range(n_inc):
                rs = step_batch([gs[i] for i in idx], [ws[i].dtau for i in idx])
                for i, r in zip(idx, rs):
                    out[i].append(r)
        th = [threading.Thread(target=one, args=(idx,)) for idx in classes.values()]
        for t in th:
            t.start()
        for t in th:
            t.join()

    run_classes(warmup, [[] for _ in ws])
    torch.cuda.synchronize()
    blobs = [g.save() for g in gs]
    setup_s = time.perf_counter() - t_setup
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    rb = [[] for _ in ws]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_classes(steps, rb)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    clk = clocks.stop()
    for g, b in zip(gs, blobs):
        g.load(b)
    ra = [[] for _ in ws]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, g in enumerate(gs):
        for _ in range(steps):
            ra[i].append(g.step(ws[i].dtau))
    torch.cuda.synchronize()
    t_alone = time.perf_counter() - t0
    # the same RVEs stepped concurrently without batching: one host thread per RVE, each on its
    # own stream with its own graph launches (the GPU overlaps their kernels)
    for g, b in zip(gs, blobs):
        g.load(b)
    rc = [[] for _ in ws]

    def solo(i):
        for _ in range(steps):
            rc[i].append(gs[i].step(ws[i].dtau))
    th = [threading.Thread(target=solo, args=(i,)) for i in range(len(gs))]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    t_conc = time.perf_counter() - t0
    same = all(same_result(a, b) for x, y in zip(ra, rb) for a, b in zip(x, y))
    same_c = all(same_result(a, b) for x, y in zip(ra, rc) for a, b in zip(x, y))
    vu = sum((r["mech_iters"] + r["dmg_iters"]) * g.nvox for g, rs in zip(gs, rb) for r in rs)
    for g in gs:
        g.close()
    return {"value": vu / t_batch, "unit": "voxel-updates/s", "wall_s": t_batch, "clocks": clk,
            "one_by_one": {"value": vu / t_alone, "wall_s": t_alone}, "speedup": t_alone / t_batch,
            "concurrent_unbatched": {"value": vu / t_conc, "wall_s": t_conc, "bit_identical": same_c,
                                     "what": "one host thread and stream per RVE, graph launches, no batching"},
            "speedup_vs_concurrent": t_conc / t_batch,
            "bit_identical_to_one_by_one": same, "rves": len(ws),
            "classes": {"x".join(map(str, k)): len(v) for k, v in sorted(classes.items())},
            "setup_s": setup_s, "increments_per_rve": steps, "warmup": warmup,
            "timing": "host wall clock around the timed increments, device synchronised on both sides"}


def run_batched_3d(args, torch, stream):
    """16 3D polycrystal RVEs (grids 32^3..128^3, seeded mix), stepped in lockstep per grid class
    (rve_step_batch), against the same RVEs one by one on the same increments."""
    import synth
    ws = synth.batched_3d_polycrystals()
    leg = batched_leg(torch, ws, args.precision, args.warmup, args.steps, solver_tols(args.precision))
    return {"metric": METRIC, "value": leg["value"], "unit": "voxel-updates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": leg["wall_s"] * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32r" else "f64",
            "data": "synthetic", "config": {"workload": "batched_3d_polycrystals",
                                            "desc": WORKLOADS["batched_3d_polycrystals"],
                                            "precision": args.precision, "step": "one increment of every RVE",
                                            "l2": "inputs larger than L2 (the 128^3 RVEs alone hold > 1 GB)"},
            "clocks": leg["clocks"], "batched": leg, "roofline": None, "e2e": None}


def serving(args):
    """Continuous batching, separated from precision: a seeded request mix (a bounded subset of the
    serving stream: 2D 64^2-512^2 and 3D 32^3-64^3 fibre composites and polycrystals, a fixed
    number of increments each) runs (1) one by one on the plain FP64 path, (2) one by one on the
    FP32R path, (3) through the native request server on FP32R with lockstep batching per grid
    class, and (4) through the same server without batching. Arrivals are Poisson at 1.25 x the
    FP32R one-by-one rate; the one-by-one arms are put on the same trace as a single FIFO server."""
    import numpy as np
    import torch

    import synth
    from paper_2508_07424_gb300 import serve
    from paper_2508_07424_gb300.rve import Rve
    sizes2d, sizes3d = ((64, 128, 256, 512, 1024), (32, 64, 128)) if args.serve_sizes == "full" else \
        ((64, 128, 256), (32,))
    ws = synth.serving_mix(count=args.serve_requests, n_inc=args.serve_inc, sizes2d=sizes2d, sizes3d=sizes3d)

    def one_by_one(precision):
        times, failed = [], []
        for i, w in enumerate(ws):
            t0 = time.perf_counter()
            g = Rve.from_workload(synth.replace(w, precision=precision), **solver_tols(precision))
            try:
                for _ in range(w.n_inc):
                    if g.step(w.dtau)["fractured"]:
                        break
            except Exception as e:  # a request that fails is retired, as in the server
                failed.append({"request": i, "grid": list(w.micro.n), "name": w.name, "error": str(e)})
            g.close()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        return times, failed

    serial64, failed64 = one_by_one("fp64")
    serial32, failed32 = one_by_one("fp32r")
    lam = 1.25 * len(ws) / sum(serial32)
    arrivals = np.cumsum(np.random.default_rng(40).exponential(1.0 / lam, len(ws)))
    arrivals -= arrivals[0]

    def fifo(serial):
        fin, lat = 0.0, []
        for ta, sv in zip(arrivals, serial):
            fin = max(fin, ta) + sv
            lat.append(fin - ta)
        return {"solves_per_s": len(ws) / sum(serial), "p50_s": serve.percentile(lat, 0.5),
                "p99_s": serve.percentile(lat, 0.99), "service_p50_s": serve.percentile(serial, 0.5)}

    free, _ = torch.cuda.mem_get_info()
    reqs = [(float(ta), synth.replace(w, precision="fp32r"), w.n_inc) for ta, w in zip(arrivals, ws)]

    def server_arm(batching, trace):
        srv = serve.Server(max_inflight=8, hbm_budget_bytes=int(0.5 * free), batching=batching)
        out, wall = serve.replay(srv, trace, **solver_tols("fp32r"))
        st = srv.stats()
        srv.close()
        ok = [r for r in out.values() if r["status"] == 0]
        lat = [r["t_end"] - r["t_submit"] for r in ok]
        return {"solves_per_s": len(ok) / wall, "wall_s": wall, "p50_s": serve.percentile(lat, 0.5),
                "p99_s": serve.percentile(lat, 0.99), "peak_inflight": st["peak_inflight"],
                "voxel_updates_per_s": sum(r["voxel_updates"] for r in ok) / wall,
                "failed": [{"request": r["id"], "status": r["status"]} for r in out.values() if r["status"] != 0]}

    batched = server_arm(True, reqs)
    unbatched = server_arm(False, reqs)
    saturated = server_arm(True, [(0.0, w2, n) for (_, w2, n) in reqs])
    sizes = {}
    for w in ws:
        k = "x".join(map(str, w.micro.n))
        sizes[k] = sizes.get(k, 0) + 1
    return {"requests": len(ws), "increments_per_request": args.serve_inc, "grids": sizes,
            "mix": ("the serving stream's grids: 2D {64..1024}^2 and 3D {32..128}^3" if args.serve_sizes == "full"
                    else "bounded subset of the serving stream: 2D {64,128,256}^2 and 3D 32^3") +
                   ", fibre composites and polycrystals (synth.serving_mix, seed 4)",
            "arrivals": f"Poisson, rate 1.25 x FP32R one-by-one ({lam:.3f}/s), seed 40", "slots": 8,
            "server_fp32r_batched": batched, "server_fp32r_unbatched": unbatched,
            "server_fp32r_batched_saturated": dict(saturated, what="all requests submitted at t=0 (capacity)"),
            "one_by_one_fp64": dict(fifo(serial64), failed=failed64),
            "one_by_one_fp32r": dict(fifo(serial32), failed=failed32)}


def oracle_sample(rank=0, iters=60):
    """A bounded sample of the same work in the FP64 NumPy oracle: ``iters`` equilibrium-CG
    iterations at the initial state plus ``iters`` damage-PCG iterations at the first increment's
    scale of E (each capped run stops at its iteration limit). Returns (voxel-updates, seconds)."""
    import dataclasses

    import numpy as np

    from oracle import solver as S
    w = make_workload(rank, "fp64")
    p = S.params_from_workload(w)
    model = S.Model(w.micro, dataclasses.replace(p, max_mech=iters, max_dmg=iters, tol_mech=1e-300, tol_dmg=1e-300))
    st = S.init_state(model)
    t0 = time.perf_counter()
    try:
        S.mech_solve(model, st.phi, st.F1)
    except RuntimeError:
        pass
    t1 = time.perf_counter()
    psi1 = np.full(model.grid, 0.5)
    H = S.history_field(model, 0.05, psi1, st.psi_ini, st.H)
    t2 = time.perf_counter()
    try:
        S.damage_solve(model, H, st.phi)
    except RuntimeError:
        pass
    dt = (t1 - t0) + (time.perf_counter() - t2)
    return 2 * iters * model.V, dt


def cpu_baseline(args):
    """The FP64 oracle on this host's cores: numpy.fft on one thread, and scipy.fft with one worker
    per core (the FFTs are threaded; the oracle's pointwise numpy work is not)."""
    from oracle import spectral
    cores = os.cpu_count() or 1
    a, b = oracle_sample()
    single = {"value": a / b, "cores": 1, "fft": "numpy.fft"}
    try:
        import scipy.fft  # noqa: F401
        spectral.set_fft_workers(cores)
        a, b = oracle_sample()
        multi = {"value": a / b, "cores": cores, "fft": f"scipy.fft, workers={cores}"}
    except ImportError:
        multi = None
    finally:
        spectral.set_fft_workers(None)
    best = multi if multi and multi["value"] > single["value"] else single
    return {"value": best["value"], "unit": "voxel-updates/s", "cores": best["cores"], "kind": "oracle",
            "sample": "FP64 NumPy oracle on the same 512^2 RVE: 60 equilibrium-CG + 60 damage-PCG iterations from "
                      "the enriched initial state (" + best["fft"] + ")",
            "single_core": single, "all_cores": multi}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from oracle import spectral
    cores = os.cpu_count() or 1
    try:
        import scipy.fft  # noqa: F401
        spectral.set_fft_workers(cores)
        fft = f"scipy.fft, workers={cores}"
    except ImportError:
        cores, fft = 1, "numpy.fft"
    for _ in range(args.warmup):
        oracle_sample()
    vu, dt = 0.0, 0.0
    for _ in range(args.steps):
        a, b = oracle_sample()
        vu += a
        dt += b
    spectral.set_fft_workers(None)
    val = vu / dt
    sample = f"60 equilibrium-CG + 60 damage-PCG oracle iterations per step on the same RVE ({fft})"
    return {"impl": "reference", "metric": METRIC,
            "value": val, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(WORKLOAD, "fp64", "staggered", world),
            "cpu_baseline": {"value": val, "unit": "voxel-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32r"],
                    help="default: fp64 for the 512^2 fibre composite (headline, FP32R beside it) and the 64^2 "
                         "plate; fp32r for the other workloads")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the lockstep batching legs")
    ap.add_argument("--no-side", action="store_true", help="skip the FP32R leg beside the FP64 headline")
    ap.add_argument("--workload", default=WORKLOAD, choices=list(WORKLOADS))
    ap.add_argument("--solver", default="staggered", choices=["staggered", "newton"],
                    help="increment solver: staggered fixed point (default) or the monolithic Newton of Sec. 4.1")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-inc", type=int, default=10)
    ap.add_argument("--serve-sizes", default="subset", choices=["subset", "full"],
                    help="grids of the serving mix: a bounded subset (default run) or the full range of the stream")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.precision is None:
        args.precision = "fp64" if args.workload in ("homogeneous_plate_64", WORKLOAD) else "fp32r"
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(_finite(out)))


if __name__ == "__main__":
    main()
