"""Benchmark: adaptive BDDC setup + solve time at relative residual 1e-8.

Default workload (the timed step): Q1 linear elasticity on 48 x 48 x 24 elements
(h = 1/48, nu = 0.3), 64 irregular substructures grown from 64 seeded seed
elements (722..943 elements each, rough interfaces, 424 face pairs), E = 1e3 in
the odd z-layers of height 4 elements and 1 elsewhere, clamped at z = 0, body load
(0, 0, -1); corners (with augmentation) as initial constraints, adaptive face
constraints for lambda > tau = 10, PCG to ||r|| <= 1e-8 ||r_0||.  One step =
classification + assembly + interior elimination + pair condensations + face
eigenproblems + coarse setup + condensed rhs + PCG + recovery, with the mesh
arrays resident in HBM.  --workload picks the 24^3 Poisson, 32^3 elasticity or
256-problem workloads instead.

value = seconds per step of the mixed path; the FP64 path is timed beside it.
The roofline, kernel and tensor entries come from CUDA events the library
records around its launches (bddc_set_kernel_timing) during the timed steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the reference arm of this paper-only build) on the host cores instead.
Under torchrun every rank solves its own replica on its own GPU (the path
needs no collective); value = max over ranks of the per-step time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BDDC setup+solve s at rel.res 1e-8, mixed vs FP64 GPU; % tensor-core peak"
WORKLOADS = {
    # 24^3 Poisson, 27 substructures, 20% of elements at k = 1e4
    "poisson24": ("poisson24_3x3x3_jump1e4_adaptive_tau10", "24x24x24 Q1 hex", "config_adaptive_poisson"),
    # 32^3 elasticity, 64 substructures, 8 stiff channels E = 1e6, clamped z = 0
    "elast32": ("elast32_4x4x4_channels1e6_adaptive_tau10", "32x32x32 Q1 hex, 3 dofs/node",
                "config_elasticity_channels"),
    # the default workload: 48x48x24 elasticity, 64 region-grown irregular substructures,
    # E in {1, 1e3} by z-layers of 4
    "irregular48": ("elast48x48x24_irregular64_layers1e3_adaptive_tau10", "48x48x24 Q1 hex, 3 dofs/node",
                    "config_irregular_elasticity"),
    # 256 independent Poisson problems (2^3 or 3^3 substructures of 6^3..10^3 elements,
    # lognormal coefficients sigma = 2), solved by concurrent handles on separate streams
    "batch256": ("batch256_poisson_lognormal_adaptive_tau10", "256 problems, 12^3..30^3 Q1 hex",
                 "config_batch_poisson"),
}
BATCH_WORKERS = 8
DEFAULT_WORKLOAD = "irregular48"
TAU = 10.0
FP64_STEPS = 5        # the FP64 comparison arm times min(steps, FP64_STEPS) steps


def _peaks():
    """(bf16 TFLOP/s burst, HBM GB/s, "measured" | "fallback")."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops", 1900.0), d.get("hbm_gbs", 6800.0), "measured"
    return 1900.0, 6800.0, "fallback"


def _config(prob, seed, workload=DEFAULT_WORKLOAD):
    name, mesh, _ = WORKLOADS[workload]
    return {"workload": name, "mesh": mesh, "substructures": prob.nsub,
            "free_dofs": int((~prob.dirichlet).sum()) * prob.ncomp, "tau": TAU, "tol": 1e-8, "seed": seed,
            "precision": "fp64", "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bddc_bench_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return parse_clocks(f)


def parse_clocks(lines):
    """Summary of nvidia-smi samples (CSV without header or units, the columns of Clocks.start):
    the median SM clock, the largest maximum clock, and every throttle reason seen active in any
    sample.  Lines that are short or whose clocks are not numbers ("[N/A]") are skipped; None when
    no sample is left."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


def max_over_ranks(value, world):
    """The slowest rank's value (replicas run concurrently; the job takes the max)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _arm(args, precision, prob, dev_arrays, f_host, world, local_rank, steps=None, warmup=None):
    """Times `steps` steps of one precision arm; returns (solver, seconds per step, phase stats, adapt
    info, solve info, launches, clocks, kernel timers {class: (ms, work, launches)} summed over the
    timed steps)."""
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    import torch
    from paper_0910_5863_gb300 import bddc as B

    dev = torch.device("cuda", local_rank)
    d_xyz, d_el, d_coef, d_sub, d_dir = dev_arrays
    d_f = torch.from_numpy(f_host).to(dev)
    d_u = torch.zeros_like(d_f)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    solver = B.Solver(precision=precision, tol=1e-8, stream=stream.cuda_stream)
    if args.edge_rows:
        solver.set_edge_rows(True)

    def step():
        solver.set_mesh(prob.ncomp, d_xyz, d_el, d_coef, prob.nu, d_sub, prob.nsub, d_dir)
        solver.setup()
        ad = solver.adapt(TAU)
        _, info = solver.solve(d_f, d_u)
        return ad, info

    for _ in range(warmup):
        ad, info = step()
    torch.cuda.synchronize()
    solver.set_kernel_timing(True)
    launches0 = solver.launch_count()
    clocks = Clocks(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    phases = {k: [] for k in B.PHASES}
    kt = {}
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ad, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        for k, (ms, fl) in solver.phase_times().items():
            phases[k].append((ms, fl))
        kt = solver.kernel_times()   # collects this step's events (outside the timed region)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = solver.launch_count() - launches0
    solver.set_kernel_timing(False)
    t_step = max_over_ranks(sum(times) / len(times), world)
    return solver, t_step, phases, ad, info, launches, clk, kt


def _phase_summary(phases):
    return {k: round(sum(m for m, _ in v) / len(v), 4) for k, v in phases.items()}


# Derived ALU peaks (152 SMs at the 2.07 GHz maximum clock):
#   FP32 pipe: 128 lanes x 2 flop per clock and SM;
#   FP64 pipe: 2 multiply-adds (4 flop) per clock and SM;
#   double-float (two FP32 words): 12 FP32 instructions per multiply-add (1 mul + 3 fma
#   + 6 add of the two-sum + 2 add), 2 FP64-equivalent flop each.
FF_INSTR_PER_FMA = 12
FP32_LANE_RATE = 152 * 128 * 2.07e9
PEAK_FP32_TFLOPS = FP32_LANE_RATE * 2 / 1e12
PEAK_FF_TFLOPS = FP32_LANE_RATE / FF_INSTR_PER_FMA * 2 / 1e12
PEAK_FP64_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# TF32 dense tensor rate: the measured bf16 rate x the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25

# DRAM bytes (read + write) per launch from committed ncu captures: {(workload, kernel class): bytes}.
# The digit products on the 48x48x24 irregular mixed step: 318 launches, 137.5 GB read + 93.8 GB
# written (profiles/oz_syrk_elast32.md gives the command): the trailing blocks are read and written
# once per 128-wide block column.
TRAFFIC = {("irregular48", "oz_syrk_bf16"): (137.53e9 + 93.79e9) / 318}


def _kernel_table(kt, steps, solver, info, workload):
    """Per kernel class (the library's event timers over the timed steps): time per step and
    launch, algorithmic work per launch, achieved rate against its roofline peak."""
    bf16, hbm, src = _peaks()
    out = {}
    for name, (ms, work, n) in kt.items():
        if n == 0:
            continue
        e = {"kernel": name, "launches_per_step": n / steps, "ms_per_step": ms / steps, "ms_per_launch": ms / n,
             "traffic": TRAFFIC.get((workload, name))}
        if name in ("oz_split", "pchol_panel"):   # latency-bound helpers: time only
            e.update(bound="latency", unit="ms", work_per_launch=0.0, achieved=0.0, peak=1.0, peak_source="time only")
        elif name == "oz_syrk_bf16":
            w = 28.0 * work / n   # 28 bf16 digit products per effective multiply-add
            e.update(bound="tensor", unit="TFLOP/s", work_per_launch=w, achieved=w / (ms / n / 1e3) / 1e12, peak=bf16,
                     effective_tflops=work / n / (ms / n / 1e3) / 1e12,
                     peak_source=f"{src} bf16 {bf16} TFLOP/s (of {src}); executed bf16 flop of the 28 digit products")
        elif name == "pcg_kernel":
            # per launch (one whole PCG solve): every iteration reads every S_i and P~_i once, one
            # FP64 multiply-add per 8-byte entry, so the FP64 pipe caps the stream at
            # PEAK_FP64 / 2 x 8 bytes per second, below the HBM copy rate
            gemv = sum(2 * 8 * solver.interface_dofs(i).size ** 2 for i in range(solver.nsub))
            b = gemv * info["iters"]
            fp64_gbs = PEAK_FP64_TFLOPS * 1e12 / 2 * 8 / 1e9
            if fp64_gbs < hbm:
                bound, peak, ps = "alu", fp64_gbs, ("derived FP64 pipe rate as GEMV bytes (one multiply-add per "
                                                     f"8-byte entry), below the {src} HBM copy bandwidth {hbm} GB/s")
            else:
                bound, peak, ps = "hbm", hbm, f"{src} HBM copy bandwidth (of {src})"
            e.update(bound=bound, unit="GB/s", work_per_launch=b, achieved=b / (ms / n / 1e3) / 1e9, peak=peak,
                     peak_source=ps)
        elif name == "tc_gemm_3xtf32":
            w = 3.0 * work / n   # three TF32 products per effective product
            e.update(bound="tensor", unit="TFLOP/s", work_per_launch=w, achieved=w / (ms / n / 1e3) / 1e12,
                     peak=bf16 * NOMINAL_TF32_OVER_BF16, effective_tflops=work / n / (ms / n / 1e3) / 1e12,
                     peak_source=f"{src} bf16 {bf16} TFLOP/s x nominal TF32/BF16 1.1/2.25 (of {src}); executed TF32 flop")
        else:
            if name == "pchol_update_ff" or (name == "face_reduction" and solver.precision != 0):
                peak, ps = PEAK_FF_TFLOPS, "derived double-float rate (FP64-equivalent flop)"
            elif name == "pchol_update_fp32":
                peak, ps = PEAK_FP32_TFLOPS, "derived FP32 pipe rate"
            else:
                peak, ps = PEAK_FP64_TFLOPS, "derived FP64 pipe rate"
            w = work / n
            e.update(bound="alu", unit="TFLOP/s", work_per_launch=w, achieved=w / (ms / n / 1e3) / 1e12, peak=peak,
                     peak_source=ps)
        e["frac"] = e["achieved"] / e["peak"]
        out[name] = e
    return out


def _roofline_entry(e):
    keys = ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel", "peak_source", "work_per_launch",
            "ms_per_launch", "launches_per_step", "ms_per_step")
    return {k: e[k] for k in keys if k in e}


def run_batch_gpu(args, world, local_rank):
    """The 256-problem workload: every step solves all problems once (setup + adapt +
    solve) with BATCH_WORKERS concurrent handles; value = seconds per problem."""
    import torch
    from paper_0910_5863_gb300 import problems as P
    from paper_0910_5863_gb300 import bddc as B
    from paper_0910_5863_gb300 import batch as BT

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    probs = P.config_batch_poisson(seed=args.seed)
    arrays = BT.upload(probs, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    arms = {}
    pools = {}
    for prec in (B.MIXED, B.FP64):
        pools[prec] = pool = BT.Pool(prec, workers=BATCH_WORKERS, device=dev)
        for _ in range(args.warmup):
            BT.run(probs, arrays, pool, tau=TAU)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        clocks = Clocks(local_rank)
        clocks.start()
        walls, recs = [], None
        l0 = sum(sv.launch_count() for sv in pool.solvers)
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize(dev)
            wall, recs = BT.run(probs, arrays, pool, tau=TAU)
            walls.append(wall)
        clk = clocks.stop()
        launches = sum(sv.launch_count() for sv in pool.solvers) - l0
        wall = max_over_ranks(statistics.median(walls), world)
        lat = sorted(r["latency_s"] for r in recs)
        arms[prec] = {"s_per_problem": wall / len(probs), "problems_per_s": len(probs) / wall, "wall_s": wall,
                      "latency_median_s": lat[len(lat) // 2], "latency_max_s": lat[-1],
                      "iters_max": max(r["iters"] for r in recs), "n_added_total": sum(r["n_added"] for r in recs),
                      "all_converged": all(r["converged"] for r in recs), "clocks": clk,
                      "gpu_launches": int(launches)}
    # end to end: host arrays in, solutions out, through the same runner (mixed arm)
    h2d = sum(sum(t.numel() * t.element_size() for t in a) for a in arrays)
    d2h = sum(a[5].numel() * 8 for a in arrays)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    arrays_e2e = BT.upload(probs, dev)
    _, recs = BT.run(probs, arrays_e2e, pools[B.MIXED], tau=TAU, keep_solutions=True)
    sols = [r["u"].cpu() for r in recs]
    e2e = (time.perf_counter() - t0) / len(probs)
    del sols
    m, f = arms[B.MIXED], arms[B.FP64]
    cfg = {"workload": WORKLOADS["batch256"][0], "mesh": WORKLOADS["batch256"][1], "problems": len(probs),
           "free_dofs_total": int(sum(int((~p.dirichlet).sum()) for p in probs)), "tau": TAU, "tol": 1e-8,
           "seed": args.seed, "workers": BATCH_WORKERS, "precision": "mixed",
           "l2": "flushed before every step (256 MiB write)", "parallelism": "replicas"}
    line = {"metric": METRIC, "value": m["s_per_problem"], "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["wall_s"] * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": cfg,
            "roofline": None, "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(h2d),
                                      "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": m["gpu_launches"], "clocks": m["clocks"], "problems_per_s": m["problems_per_s"],
            "latency_median_s": m["latency_median_s"], "latency_max_s": m["latency_max_s"],
            "iters_max": m["iters_max"], "n_added_total": m["n_added_total"], "all_converged": m["all_converged"],
            "fp64": f, "mixed_over_fp64_speedup": f["s_per_problem"] / m["s_per_problem"]}
    return line


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_0910_5863_gb300 import problems as P
    from paper_0910_5863_gb300 import bddc as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = getattr(P, WORKLOADS[args.workload][2])(seed=args.seed)
    # inputs resident in HBM
    dev_arrays = (torch.from_numpy(np.ascontiguousarray(prob.xyz)).to(dev),
                  torch.from_numpy(np.ascontiguousarray(prob.elems, dtype=np.int64)).to(dev),
                  torch.from_numpy(np.ascontiguousarray(prob.coef)).to(dev),
                  torch.from_numpy(np.ascontiguousarray(prob.elem_sub, dtype=np.int32)).to(dev),
                  torch.from_numpy(np.ascontiguousarray(prob.dirichlet, dtype=np.uint8)).to(dev))
    f_host = B.free_load_vector(prob)
    if args.arm != "both":   # one arm alone (profiling runs): its step time, phases and kernels
        prec = B.MIXED if args.arm == "mixed" else B.FP64
        solver, t, ph, ad, info, launches, clk, kt = _arm(args, prec, prob, dev_arrays, f_host, world, local_rank)
        return {"metric": METRIC, "value": t, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if args.arm == "mixed" else "f64", "data": "synthetic",
                "config": dict(_config(prob, args.seed, args.workload), precision=args.arm), "arm": args.arm,
                "gpu_launches": int(launches), "clocks": clk, "phase_ms": _phase_summary(ph),
                "kernels": _kernel_table(kt, args.steps, solver, info, args.workload),
                "iters": info["iters"], "kappa": info["kappa"], "relres": info.get("relres"),
                "n_added": ad["n_added"], "omega": ad["omega"]}
    solver, t_mixed, ph_mixed, ad, info, launches, clk, kt = _arm(args, B.MIXED, prob, dev_arrays, f_host, world,
                                                                  local_rank)
    steps64, warm64 = min(args.steps, FP64_STEPS), min(args.warmup, 3)
    _, t_fp64, ph_fp64, ad64, info64, launches64, clk64, kt64 = _arm(args, B.FP64, prob, dev_arrays, f_host, world,
                                                                     local_rank, steps64, warm64)

    # end-to-end through the C ABI with host buffers (mesh and f from host, u back to host), mixed arm
    mesh_host = [np.ascontiguousarray(prob.xyz), np.ascontiguousarray(prob.elems, dtype=np.int64),
                 np.ascontiguousarray(prob.coef), np.ascontiguousarray(prob.elem_sub, dtype=np.int32),
                 np.ascontiguousarray(prob.dirichlet, dtype=np.uint8)]
    u_host = np.zeros_like(f_host)
    e2e_times = []
    for it in range(min(max(2, args.steps // 2), 5) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.set_mesh(prob.ncomp, mesh_host[0], mesh_host[1], mesh_host[2], prob.nu, mesh_host[3], prob.nsub,
                        mesh_host[4])
        solver.setup()
        solver.adapt(TAU)
        solver.solve(f_host, u_host)
        t1 = time.perf_counter()
        if it > 0:
            e2e_times.append(t1 - t0)
    h2d = sum(a.nbytes for a in mesh_host) + f_host.nbytes
    d2h = u_host.nbytes

    pm, pf = _phase_summary(ph_mixed), _phase_summary(ph_fp64)
    kmix = _kernel_table(kt, args.steps, solver, info, args.workload)
    k64 = _kernel_table(kt64, steps64, solver, info64, args.workload)
    dominant = max(kmix, key=lambda c: kmix[c]["ms_per_step"])
    line = {
        "metric": METRIC, "value": t_mixed, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mixed * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": _config(prob, args.seed, args.workload),
        "roofline": _roofline_entry(kmix[dominant]),
        "tensor": _roofline_entry(kmix["tc_gemm_3xtf32"]),
        "kernels": kmix,
        "e2e": {"value": statistics.median(e2e_times), "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "phase_ms": pm, "dominant_phase": max(pm, key=pm.get),
        "iters": info["iters"], "kappa": info["kappa"], "relres": info["relres"], "n_added": ad["n_added"],
        "omega": ad["omega"],
        "fp64": {"value": t_fp64, "unit": "s", "ms_per_step": t_fp64 * 1e3, "steps": steps64, "warmup": warm64,
                 "phase_ms": pf, "iters": info64["iters"], "kappa": info64["kappa"], "relres": info64["relres"],
                 "n_added": ad64["n_added"], "gpu_launches": int(launches64), "clocks": clk64,
                 "roofline": _roofline_entry(k64[max(k64, key=lambda c: k64[c]["ms_per_step"])]),
                 "kernels": k64},
        "mixed_over_fp64_speedup": t_fp64 / t_mixed,
    }
    line["config"]["precision"] = ("mixed (interior: FP32 tensor-core factorization + FP64 refinement; pair "
                                   "condensations, face reductions and local saddle: double-float; coarse inverse, "
                                   "Sturm counts, PCG: FP64)")
    line["config"]["edge_rows"] = bool(args.edge_rows)
    if args.edge_rows:
        line["n_edge_rows"] = solver.edge_rows()[0]
    return line


def run_oracle(args, sample_note):
    """The FP64 CPU oracle on the same workload (host cores).  Returns (seconds, cores,
    iterations, added constraints, sample description)."""
    from paper_0910_5863_gb300 import problems as P
    import oracle
    from oracle.adaptive import pair_problem

    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.environ.get("OMP_NUM_THREADS", os.cpu_count())))
    if args.workload == "batch256":
        # bounded sample: the first 4 of the 256 problems, whole runs, scaled per problem
        probs = P.config_batch_poisson(seed=args.seed)[:4]
        t0 = time.perf_counter()
        for prob in probs:
            m = oracle.Model(prob)
            m.schur()
            oracle.adapt(m, TAU)
            m.solve(tol=1e-8)
        t = (time.perf_counter() - t0) / len(probs)
        return t, cores, None, None, "4 of the 256 problems, each a full run (setup + adapt + solve); value = s per problem"
    if args.workload == "poisson24":
        prob = getattr(P, WORKLOADS[args.workload][2])(seed=args.seed)
        t0 = time.perf_counter()
        m = oracle.Model(prob)
        m.schur()
        ad = oracle.adapt(m, TAU)
        res = m.solve(tol=1e-8)
        t1 = time.perf_counter()
        return t1 - t0, cores, res.iters, ad.n_added, "one full run of the workload (setup + adapt + solve)"
    # Bounded sample.  The model (assembly and globs) and the face pair problem of the smallest
    # pair are measured on the first call; every call measures the Schur complement of one more
    # substructure (in turn).  Each part is extrapolated to the whole workload by the cubic cost
    # of its dense eliminations; PCG is not included.
    c = _ORACLE_SAMPLE
    if c.get("workload") != args.workload:
        prob = getattr(P, WORKLOADS[args.workload][2])(seed=args.seed)
        t0 = time.perf_counter()
        m = oracle.Model(prob)
        t1 = time.perf_counter()
        subs = m.subs
        keys = sorted(m.globs.faces)
        pair_n = [subs[i].G.size + subs[j].G.size for (i, j) in keys]
        f0 = int(np.argmin(pair_n))
        i, j = keys[f0]
        m.subs = [subs[i], subs[j]]
        m.schur()
        m.subs = subs
        t2 = time.perf_counter()
        pair_problem(m, i, j, TAU)
        t3 = time.perf_counter()
        cost = [s.I.size ** 3 / 3 + s.I.size ** 2 * s.G.size + s.I.size * s.G.size ** 2 for s in subs]
        c.clear()
        c.update(workload=args.workload, m=m, subs=subs, cost=cost, t_model=t1 - t0, t_pair=t3 - t2,
                 p_scale=sum(float(n) ** 3 for n in pair_n) / float(pair_n[f0]) ** 3, npairs=len(keys), next=0)
    m, subs, cost = c["m"], c["subs"], c["cost"]
    k = c["next"] % len(subs)
    c["next"] += 1
    t0 = time.perf_counter()
    m.subs = [subs[k]]
    m.schur()
    m.subs = subs
    t_s = time.perf_counter() - t0
    s_scale = sum(cost) / cost[k]
    est = c["t_model"] + t_s * s_scale + c["t_pair"] * c["p_scale"]
    return est, cores, None, None, (
        f"measured: the Schur complement of substructure {k} of {len(subs)} ({t_s:.2f} s, x {s_scale:.1f}); "
        f"once: the model ({c['t_model']:.1f} s) and the pair problem of the smallest of {c['npairs']} face "
        f"pairs ({c['t_pair']:.1f} s, x {c['p_scale']:.0f}); the factors scale by the substructures' "
        f"n_I^3/3 + n_I^2 n_G + n_I n_G^2 and the pairs' (n_G,i + n_G,j)^3; PCG not included")


_ORACLE_SAMPLE = {}


def measure_peaks(local_rank=0):
    """Library (cuBLAS) GEMM throughput per dtype at 8192^3 and the device copy bandwidth
    (CUDA events, best of several runs): the denominators quoted beside the derived ALU peaks."""
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    out = {}
    n = 8192
    for name, dt, tf32 in (("fp64", torch.float64, False), ("fp32_simt", torch.float32, False),
                           ("tf32", torch.float32, True), ("bf16", torch.bfloat16, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device=dev, dtype=torch.float32).to(dt)
        b = torch.randn(n, n, device=dev, dtype=torch.float32).to(dt)
        reps = 2 if dt == torch.float64 else 10
        best = 1e30
        for _ in range(3):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3 / reps)
        out[name + "_tflops"] = 2.0 * n ** 3 / best / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    x = torch.empty(1 << 28, dtype=torch.float64, device=dev)   # 2 GiB
    y = torch.empty_like(x)
    best = 1e30
    for _ in range(5):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        y.copy_(x)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    out["copy_gbs"] = 2 * x.numel() * 8 / best / 1e9
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--peaks", action="store_true",
                    help="print the cuBLAS GEMM rates (FP64, FP32, TF32, BF16) and the copy bandwidth and exit")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--arm", default="both", choices=["both", "mixed", "fp64"],
                    help="precision arms to time (the fp64 sub-object needs both)")
    ap.add_argument("--edge-rows", action="store_true",
                    help="also keep the adaptive edge rows (Section 3's split rows, one basis per edge); "
                         "poisson24 and elast32 workloads")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.peaks:
        print(json.dumps(measure_peaks(local_rank)), flush=True)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        for _ in range(args.warmup):
            run_oracle(args, "")
        times = []
        for _ in range(args.steps):
            t, cores, iters, added, sample = run_oracle(args, "")
            times.append(t)
        v = statistics.median(times)
        P = __import__("paper_0910_5863_gb300.problems", fromlist=["x"])
        if args.workload == "batch256":
            cfg = {"workload": WORKLOADS["batch256"][0], "mesh": WORKLOADS["batch256"][1], "problems": 256,
                   "tau": TAU, "tol": 1e-8, "seed": args.seed, "precision": "fp64", "parallelism": "replicas"}
        else:
            cfg = _config(getattr(P, WORKLOADS[args.workload][2])(args.seed), args.seed, args.workload)
            cfg["edge_rows"] = bool(args.edge_rows)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
                "steps": len(times), "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                                 "sample": sample + "; median of steps"},
                "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "iters": iters, "n_added": added}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.workload == "batch256":
        line = run_batch_gpu(args, world, local_rank)
    else:
        line = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline:
            t, cores, iters, added, sample = run_oracle(args, "")
            line["cpu_baseline"] = {"value": t, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample,
                                    "iters": iters, "n_added": added}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
