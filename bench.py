"""Benchmark of the FFT phase-field-fracture hot path on GB300.

A step is one dissipation increment (the whole staggered solve: equilibrium CG, damage PCG,
control root search, Anderson mixing, history and load-curve update) of the 512^2 fibre
composite RVE (30% discs of radius 20, E_f/E_m = 5, Gc_f/Gc_m = 2, l = 3, central enriched
crack of 64 voxels). Metric: voxel-updates/s = sum over (equilibrium-CG + damage-PCG iterations)
x voxels, per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32r] [--impl reference]

N > 1 runs one independent RVE replica per rank (the solve of one RVE does not shard; replicas
only). Timing: W untimed increments, then K increments each bracketed by CUDA events on the
library's stream; between timed increments L2 is flushed by writing 256 MiB; barrier +
synchronize around the timed region, max over ranks. One JSON line on rank 0.
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
                               "l=2, through CTE crack 0.1 n, dtau=1.5*<Gc>*A_g/100; run as 16 concurrent streams",
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
    if precision == "fp64":
        return dict(tol_stag=1e-8)
    return dict(tol_mech=1e-6, tol_dmg=1e-6, tol_root=1e-7, tol_stag=1e-5)


# ---- algorithmic work of the dominant kernel ----------------------------------------------------
# DRAM bytes per k_axis launch, averaged over the column passes of one 512^2 FP32 increment (ncu)
K_AXIS_TRAFFIC = 1861371


def axis_kernel_model(nx, ny, ns, word, nz=1):
    """One launch of the mechanics column pass: bytes = read + write of ns complex values per
    half-spectrum point. 2D (and plates one voxel thick): y FFT, projection, inverse y FFT in one
    launch; flops = 2 transforms x 5 log2(ny) per complex point and component + ~40 per point.
    3D: three launches per projection (y, z with the projection, y), each moving the same bytes;
    flops are not modelled there (NaN)."""
    import math
    npts = (nx // 2 + 1) * ny * nz
    bytes_ = 2.0 * ns * npts * 2 * word
    flops = npts * ns * 2 * 5 * math.log2(ny) + 40.0 * npts if nz == 1 else float("nan")
    return bytes_, flops


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


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2508_07424_gb300 import build, capi
    from paper_2508_07424_gb300.rve import Rve
    build.build()
    stream = torch.cuda.current_stream()
    if args.workload == "batched_3d_polycrystals":
        return run_batched_3d(args, torch, stream)
    w = make_workload(rank, args.precision, args.workload)
    tol = solver_tols(args.precision)
    solver = capi.RVE_SOLVER_NEWTON if args.solver == "newton" else capi.RVE_SOLVER_STAGGERED
    g = Rve.from_workload(w, stream=stream.cuda_stream, solver=solver, **tol)
    N = g.nvox
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        g.step(w.dtau)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = g.launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    vu = 0
    results = []
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        r = g.step(w.dtau)
        ev[i][1].record(stream)
        results.append(r)
        vu += (r["mech_iters"] + r["dmg_iters"]) * N
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    launches = g.launches() - launches0
    clk = clocks.stop()
    # dominant-kernel timing: CUDA events around every launch of the mechanics spectral pass on
    # the library stream, over 3 increments that follow the timed region (event records cannot sit
    # inside the replayed CUDA graphs, so these increments launch plainly).
    g.timing(True)
    for _ in range(3):
        g.step(w.dtau)
    ax_ms, ax_n, ax_bytes = g.timing(kind=0)      # the mechanics projection pass
    all_ms, all_n, all_bytes = g.timing(kind=1)   # every column pass (k_axis)
    g.timing(False)
    tot_ms, tot_vu = aggregate_over_ranks(ms, vu, world, "cuda")

    # e2e: the public C ABI from host buffers; every step uploads the microstructure, builds the
    # enriched crack, runs one increment and reads back the result and the damage field.
    e2e = None
    if not args.no_e2e:
        import numpy as np
        e_steps = max(2, min(args.steps, 5))
        m = w.micro
        gid_host = torch.from_numpy(np.ascontiguousarray(m.grain_id)).pin_memory()
        phi_host = torch.empty(N, dtype=torch.float64).pin_memory()
        h2d = gid_host.numel() * 4 + m.C_cubic.nbytes + m.R.nbytes + m.Gc.nbytes + m.cleave_n.nbytes + m.beta.nbytes
        d2h = N * 8 + 96
        ge = Rve.from_workload(w, stream=stream.cuda_stream, **tol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        evu = 0
        for _ in range(e_steps):
            m.grain_id = gid_host.numpy().reshape(m.grain_id.shape)
            ge.set_microstructure(m)
            r = ge.step(w.dtau)
            phi_host.numpy()[:] = ge.get(capi.RVE_FIELD_PHI).reshape(-1)
            evu += (r["mech_iters"] + r["dmg_iters"]) * N
        torch.cuda.synchronize()
        et = time.perf_counter() - t0
        e2e = {"value": evu / et * world, "unit": "voxel-updates/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e_steps,
               "what": "set_microstructure from host arrays + enriched-crack setup + one increment + D2H of "
                       "result and damage field, per step; the increment is the first of a fresh RVE, whose "
                       "iteration mix differs from increments 4.. of the device-timed run"}
        ge.close()

    if rank != 0:
        return None
    pk, src = peaks()
    word = 8 if args.precision == "fp64" else 4
    bytes_l, flops_l = axis_kernel_model(w.micro.n[0], w.micro.n[1], 3 if w.micro.dim == 2 else 6, word,
                                         w.micro.n[2])
    avg_s = ax_ms * 1e-3 / max(ax_n, 1)
    if ax_n == 0:
        # the Newton solver applies the projection inside its Jacobian, not in the timed CG pass
        roof = {"kernel": "k_axis (mechanics: FFT_y + projection + inverse FFT_y)", "bound": None,
                "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "note": "not timed: no equilibrium CG pass runs with this solver", "launches": 0}
    elif args.precision == "fp64":
        peak = 152 * 2 * 2 * 2.07e9 / 1e12   # FP64: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz = 1.26 TFLOP/s
        roof = {"kernel": "k_axis (mechanics: FFT_y + projection + inverse FFT_y)", "bound": "alu",
                "timing": "CUDA events per launch over 3 instrumented increments after the timed region",
                "achieved": flops_l / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops_l / avg_s / 1e12 / peak, "peak_source": "FP64 unit count x max SM clock",
                "traffic": None, "avg_launch_us": avg_s * 1e6, "launches": ax_n}
    else:
        peak = pk["hbm_gbs"]
        # The dominant kernel is k_axis, the column-pass template behind the mechanics projection
        # and the damage gradient / divergence / preconditioner passes (together the largest share
        # of the launch list). Bytes per launch: the half-spectrum components it reads and writes,
        # as the library counts them per launch; traffic: DRAM bytes per launch averaged over the
        # column passes of one increment in an ncu capture of this workload
        # (profiles/k_axis_column_passes_fibre512_fp32.md); other workloads have no capture.
        avg_all = all_ms * 1e-3 / max(all_n, 1)
        traffic = K_AXIS_TRAFFIC if (args.workload == WORKLOAD and w.micro.n[0] == 512) else None
        roof = {"kernel": "k_axis (every column pass: y FFT (and z in 3D), per-frequency operator, inverse)",
                "bound": "hbm",
                "timing": "CUDA events around every launch over 3 instrumented increments after the timed region",
                "achieved": all_bytes / avg_all / 1e9, "peak": peak, "unit": "GB/s",
                "frac": all_bytes / avg_all / 1e9 / peak, "peak_source": src, "traffic": traffic,
                "algorithmic_bytes": all_bytes, "avg_launch_us": avg_all * 1e6, "launches": all_n,
                "projection_pass": {"achieved": bytes_l / avg_s / 1e9, "algorithmic_bytes": bytes_l,
                                    "avg_launch_us": avg_s * 1e6, "launches": ax_n}}
    out = {
        "metric": f"FFT-PFF voxel-updates/s ({args.workload} increments)",
        "value": tot_vu / (tot_ms * 1e-3),
        "unit": "voxel-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps,
        "voxel_increments_per_s": N * args.steps * world / (tot_ms * 1e-3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": workload_desc(args.workload), "precision": args.precision,
                   "solver": args.solver,
                   "step": "one dissipation increment", "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas{world}"},
        "increments": [{k: r[k] for k in ("n", "mech_iters", "dmg_iters", "stag_iters", "root_evals")} for r in results],
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
        "e2e": e2e,
    }
    if world == 1 and w.micro.dim == 2:
        out["cufft_reference"] = cufft_reference(torch, stream, g, w, args.precision)
    if not args.no_cpu_baseline and world == 1 and args.workload == WORKLOAD:
        out["cpu_baseline"] = cpu_baseline(args, timed_steps=1)
    if args.precision == "fp32r" and world == 1 and args.workload == WORKLOAD:
        out["fp64_side_by_side"] = side_by_side_fp64(args, stream)
    if args.workload == "homogeneous_plate_64" and world == 1:
        out["toughness_run"] = toughness_run(args, stream)
    if not args.no_serve and world == 1 and args.workload == WORKLOAD:
        out["serving"] = serving(args)
    return out


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


def run_batched_3d(args, torch, stream):
    """16 3D polycrystal RVEs (grids 32^3..128^3) submitted at once to the native request server
    with 16 slots (one handle, stream and worker thread each); every request uploads its
    microstructure, builds its enriched crack and runs W + K increments. Value = voxel-updates of
    all requests / wall time; per-request latency p50/p99."""
    import synth
    from paper_2508_07424_gb300 import serve
    ws = synth.batched_3d_polycrystals()
    for w in ws:
        w.precision = args.precision
    n_inc = args.warmup + args.steps
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(max_inflight=len(ws), hbm_budget_bytes=int(0.8 * free))
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    out, wall = serve.replay(srv, [(0.0, w, n_inc) for w in ws])
    torch.cuda.synchronize()
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    ok = [r for r in out.values() if r["status"] == 0]
    vu = sum(r["voxel_updates"] for r in ok)
    lat = [r["t_end"] - r["t_start"] for r in ok]
    sizes = {}
    for w in ws:
        sizes[w.micro.n[0]] = sizes.get(w.micro.n[0], 0) + 1
    return {"metric": "FFT-PFF voxel-updates/s (batched_3d_polycrystals increments)", "value": vu / wall,
            "unit": "voxel-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall * 1e3 / n_inc, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32r" else "f64", "data": "synthetic",
            "config": {"workload": "batched_3d_polycrystals", "desc": WORKLOADS["batched_3d_polycrystals"],
                       "precision": args.precision, "grids": {f"{k}^3": v for k, v in sorted(sizes.items())},
                       "step": "one dissipation increment of each of the 16 RVEs (W + K per request, all timed, "
                               "including microstructure upload and crack enrichment)",
                       "l2": "inputs larger than L2 (the 128^3 RVEs alone hold > 1 GB)"},
            "requests_ok": len(ok), "failed": [r["id"] for r in out.values() if r["status"] != 0],
            "latency_p50_s": serve.percentile(lat, 0.5), "latency_p99_s": serve.percentile(lat, 0.99),
            "peak_inflight": st["peak_inflight"], "clocks": clk,
            "timing": "host wall clock around the server run, device synchronised", "roofline": None, "e2e": None}


def side_by_side_fp64(args, stream):
    """The plain FP64 path on the same RVE and increments (3 warm-up, then 3 timed increments)."""
    import torch

    from paper_2508_07424_gb300.rve import Rve
    w = make_workload(0, "fp64")
    g = Rve.from_workload(w, stream=stream.cuda_stream, **solver_tols("fp64"))
    for _ in range(3):
        g.step(w.dtau)
    torch.cuda.synchronize()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    vu = 0
    for _ in range(3):
        r = g.step(w.dtau)
        vu += (r["mech_iters"] + r["dmg_iters"]) * g.nvox
    b_.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b_)
    g.close()
    return {"value": vu / (ms * 1e-3), "unit": "voxel-updates/s", "ms_per_step": ms / 3, "dtype": "f64",
            "steps": 3, "warmup": 3}


def serving(args):
    """Continuous batching vs one-by-one: the same seeded request mix (2D 64^2-256^2 and 3D 32^3,
    fibre composites and polycrystals, a fixed number of increments each) is first run one by
    one on the plain FP64 path; its measured rate r sets Poisson arrivals at 1.25 r, replayed
    through the native request server (FP32 with refinement, 8 slots, admission by footprint)."""
    import numpy as np
    import torch

    import synth
    from paper_2508_07424_gb300 import serve
    from paper_2508_07424_gb300.rve import Rve
    ws = synth.serving_mix(count=args.serve_requests, n_inc=args.serve_inc)
    # plain FP64, one by one
    serial, plain_failed = [], []
    for i, w in enumerate(ws):
        t0 = time.perf_counter()
        g = Rve.from_workload(synth.replace(w, precision="fp64"), tol_stag=1e-8)
        try:
            for _ in range(w.n_inc):
                if g.step(w.dtau)["fractured"]:
                    break
        except Exception as e:  # a request that fails is retired, as in the server
            plain_failed.append({"request": i, "grid": list(w.micro.n), "name": w.name, "error": str(e)})
        g.close()
        serial.append(time.perf_counter() - t0)
    rate_plain = len(ws) / sum(serial)
    lam = 1.25 * rate_plain
    arrivals = np.cumsum(np.random.default_rng(40).exponential(1.0 / lam, len(ws)))
    arrivals -= arrivals[0]
    # the plain path on the same arrival trace (a single FIFO server)
    fin, lat_plain = 0.0, []
    for ta, sv in zip(arrivals, serial):
        fin = max(fin, ta) + sv
        lat_plain.append(fin - ta)
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(max_inflight=8, hbm_budget_bytes=int(0.5 * free))
    reqs = [(float(ta), synth.replace(w, precision="fp32r"), w.n_inc) for ta, w in zip(arrivals, ws)]
    out, wall = serve.replay(srv, reqs)
    st = srv.stats()
    srv.close()
    # capacity: the same requests all submitted at t = 0
    srv = serve.Server(max_inflight=8, hbm_budget_bytes=int(0.5 * free))
    out_sat, wall_sat = serve.replay(srv, [(0.0, w2, n) for (_, w2, n) in reqs])
    st_sat = srv.stats()
    srv.close()
    ok_sat = [r for r in out_sat.values() if r["status"] == 0]
    ok = [r for r in out.values() if r["status"] == 0]
    lat = [r["t_end"] - r["t_submit"] for r in ok]
    return {"requests": len(ws), "increments_per_request": args.serve_inc,
            "mix": "2D {64,128,256}^2 fibre/polycrystal + 3D 32^3 polycrystal, seeded (synth.serving_mix)",
            "arrivals": f"Poisson, rate 1.25 x plain FP64 one-by-one rate ({lam:.3f}/s)",
            "solves_per_s": len(ok) / wall, "p50_s": serve.percentile(lat, 0.5), "p99_s": serve.percentile(lat, 0.99),
            "failed": [{"request": r["id"], "status": r["status"], "grid": list(ws[r["id"]].micro.n),
                        "name": ws[r["id"]].name} for r in out.values() if r["status"] != 0],
            "voxel_updates_per_s": sum(r["voxel_updates"] for r in ok) / wall,
            "peak_inflight": st["peak_inflight"], "slots": 8, "precision": "fp32r",
            "saturated": {"solves_per_s": len(ok_sat) / wall_sat, "wall_s": wall_sat,
                          "p50_s": serve.percentile([r["t_end"] - r["t_submit"] for r in ok_sat], 0.5),
                          "p99_s": serve.percentile([r["t_end"] - r["t_submit"] for r in ok_sat], 0.99),
                          "peak_inflight": st_sat["peak_inflight"],
                          "what": "all requests submitted at t=0 (server capacity)"},
            "plain_fp64_one_by_one": {"solves_per_s": rate_plain, "p50_s": serve.percentile(lat_plain, 0.5),
                                      "p99_s": serve.percentile(lat_plain, 0.99),
                                      "service_p50_s": serve.percentile(serial, 0.5), "failed": plain_failed}}


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


def cpu_baseline(args, timed_steps=1):
    vu, dt = 0.0, 0.0
    for _ in range(timed_steps):
        a, b = oracle_sample()
        vu += a
        dt += b
    return {"value": vu / dt, "unit": "voxel-updates/s", "cores": 1, "kind": "oracle",
            "sample": "FP64 NumPy oracle on the same 512^2 RVE: 60 equilibrium-CG + 60 damage-PCG iterations; "
                      "numpy.fft and einsum run single-threaded"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    for _ in range(args.warmup):
        oracle_sample()
    vu, dt = 0.0, 0.0
    for _ in range(args.steps):
        a, b = oracle_sample()
        vu += a
        dt += b
    val = vu / dt
    return {"impl": "reference", "metric": "FFT-PFF voxel-updates/s (fibre composite 512^2 increments)",
            "value": val, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "desc": workload_desc(), "precision": "fp64",
                       "step": "60 equilibrium-CG + 60 damage-PCG iterations of the oracle on the same RVE"},
            "cpu_baseline": {"value": val, "unit": "voxel-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "60 equilibrium-CG + 60 damage-PCG oracle iterations per step"},
            "e2e": {"value": val, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32r"],
                    help="default: fp64 for homogeneous_plate_64 (the parity configuration), fp32r otherwise")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=list(WORKLOADS))
    ap.add_argument("--solver", default="staggered", choices=["staggered", "newton"],
                    help="increment solver: staggered fixed point (default) or the monolithic Newton of Sec. 4.1")
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serve-inc", type=int, default=10)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.precision is None:
        args.precision = "fp64" if args.workload == "homogeneous_plate_64" else "fp32r"
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(_finite(out)))


if __name__ == "__main__":
    main()
