#!/usr/bin/env python
"""Benchmark of the generalized-Poisson hot path on GB300.

One step = the whole hot path over one synthetic slab configuration:
  eps(R) and the multigrid hierarchy / wet band  (gp_set_dielectric)
  the Gaussian charge density                    (gp_build_rho)
  the solve to the relative-residual tolerance   (gp_solve, cold start)
  energy and forces                              (gp_energy_forces)
Inputs (atom positions, Gaussian widths) are resident in HBM before the timed
region; every step uses a new frame of a seeded ballistic trajectory.

Prints ONE JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
instead, on bounded samples of the same workload, and prints its own line.
Multi-GPU (torchrun, N > 1): independent replicas, one per GPU, no collective
on the data path ("scaling": "weak"); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "generalized-Poisson solves/s at 1e-8 rel. residual, mixed vs FP64; smoother HBM GB/s"
UNIT = "solves/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


FP64_PEAK_GFLOPS = 1250.0   # nominal GB300 FP64 (non-tensor), the profiling recipe's table


def dtype_label(precision, tol):
    """The arithmetic types the step computes in (not a precision claim)."""
    if precision == 0:
        return "f64+df64"          # FP64 solve; the field kernels' pair terms in df64
    return "f32+df64" if tol >= 1e-10 else "f32+f64+df64"


def precision_detail(precision, tol):
    fields = "eps, rho and both force terms: per-pair arithmetic in df64 (pairs of FP32, ~2^-48 relative)"
    red = "energy, reductions, dot products: FP64 accumulation"
    if precision == 0:
        return {"solve": "FP64 multigrid-preconditioned CG", "fields": fields, "reductions": red}
    outer = ("df64 (FP32 pairs): outer residual and phi update" if tol >= 1e-10
             else "FP64: outer residual and phi update")
    return {"solve": "FP32 multigrid-preconditioned CG inside defect correction", "outer": outer,
            "fields": fields, "reductions": red}

SWEEP_PROFILE = os.path.join(ROOT, "profiles", "k_rb_sweep_mixed_192x192x384.txt")
SWEEP_SOURCE = os.path.join(ROOT, "paper_0904_4887_gb300", "csrc", "k_smooth.cu")


def source_digest(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def sweep_traffic(kernel_name, workload):
    """DRAM bytes per launch of the smoother from the committed ncu summary, or
    None when the summary is for another kernel, workload or kernel source."""
    try:
        fields = {}
        with open(SWEEP_PROFILE) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("workload") != workload or fields.get("source_digest") != source_digest(SWEEP_SOURCE):
            return None
        if kernel_name not in fields.get("kernel", ""):
            return None
        return float(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over the ranks (x itself on one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job units per second: every rank processes units_per_rank, the job
    takes the slowest rank's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- inputs
def make_inputs(w, frames, seed=0):
    at = W.workload_atoms(w, seed=seed)
    traj = W.md_frames(at, w.cell, frames, dt_fs=w.dt_fs, temperature=w.temperature, seed=seed)
    gauss = np.stack([at.Z, at.sigma_core, at.sigma_cloud], axis=1)
    return at, traj, gauss


# ----------------------------------------------------------------------------- GPU arm
def roofline_for(kind, prof, n0, hbm, hbm_src, prec_bytes):
    """Achieved vs peak for the kernel group `kind` from the live CUDA-event profile."""
    p = prof[kind]
    if p["launches"] == 0 or p["ms"] <= 0:
        return None
    per_launch_s = p["ms"] / 1e3 / p["launches"]
    if kind == "smooth0":
        # FP32: one launch = one fused red-black sweep, 16 B/pt (read u, f, eps; write u);
        # FP64: one launch = one colour of a sweep, half of 32 B/pt
        bytes_per_launch = 16.0 * n0
        achieved = bytes_per_launch / per_launch_s / 1e9
        out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
               "peak_source": hbm_src,
               "kernel": "k_rb_sweep (finest level, fused red-black sweep)" if prec_bytes == 4
               else "k_rbgs (finest level, one colour)",
               "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": per_launch_s * 1e3}
        if prec_bytes == 8:
            # the FP64 colour sweep is bound by the FP64 pipe, not HBM: 30 FP64 flops per
            # updated point (six face means, the weighted sum, the diagonal, the update)
            gf = 30.0 * (n0 / 2) / per_launch_s / 1e9
            out["fp64"] = {"achieved": gf, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                           "frac": gf / FP64_PEAK_GFLOPS, "peak_source": "nominal FP64 (recipe table)",
                           "flops_per_updated_point": 30}
        return out
    if kind == "res64":
        # read phi, rho, eps (FP64), write r in the working precision; 30 FP64 flops per point
        bytes_per_launch = (24 + prec_bytes) * n0
        flops = 30.0 * n0
        ach_f = flops / per_launch_s / 1e9
        return {"bound": "alu", "achieved": ach_f, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": ach_f / FP64_PEAK_GFLOPS, "peak_source": "nominal FP64 (recipe table)",
                "kernel": "k_residual64", "hbm_gbs": bytes_per_launch / per_launch_s / 1e9,
                "avg_launch_ms": per_launch_s * 1e3}
    return {"bound": "alu", "achieved": None, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": None,
            "kernel": kind, "avg_launch_ms": per_launch_s * 1e3,
            "note": "FP64 special-function kernel; no algorithmic flop count is defined for it"}


def gpu_arm(args, rank, world):
    import torch
    import paper_0904_4887_gb300 as P
    from paper_0904_4887_gb300 import gp as G

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.WORKLOADS[args.workload]
    nfr = args.warmup + args.steps
    at, traj, gauss_np = make_inputs(w, max(nfr, 2), seed=rank)
    gauss = torch.tensor(gauss_np, dtype=torch.float64, device=dev)
    frames = [torch.tensor(traj[i % len(traj)], dtype=torch.float64, device=dev) for i in range(nfr)]
    hbm, hbm_src = load_peaks()

    zlim = W.lower_layer_zlim(at, w) if args.kind == 2 else 0.0
    n_dir = args.n_dirichlet if args.n_dirichlet >= 0 else (0 if args.kind == 2 else 1)

    def make_solver(precision, split):
        extra = {"kind": args.kind, "gamma_tail": args.gamma_tail, "zlim": zlim} if args.kind else {}
        for key in ("nu_coarse", "nu1", "nu2", "inner"):
            if getattr(args, key) is not None:
                extra[key] = getattr(args, key)
        return P.GPSolver(w.grid, w.cell, precision=precision, split=split, levels=w.levels,
                          sweep_shape=args.sweep_shape, n_dirichlet=n_dir, **extra)

    radii = torch.tensor(W.vdw_radii(at.Z), dtype=torch.float64, device=dev) if args.kind else None

    solver = make_solver(args.precision, args.split)
    rho = solver.zeros()
    phi = solver.zeros()
    F = torch.zeros((len(at.Z), 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step(s, pos, phi_buf, rho_buf, tol=None):
        s.set_atoms(pos, radii=radii)
        s.build_rho(pos, gauss, out=rho_buf)
        phi_buf.zero_()
        st = s.ctx.gp_solve(rho_buf, phi_buf, args.tol if tol is None else tol, check=False)
        if st not in (0,):
            raise RuntimeError("solve failed: %s %s" % (G.STATUS_NAMES.get(st), s.ctx._lib.gp_last_error(s.ctx._h)))
        E, E2 = s.ctx.gp_energy_forces(phi_buf, rho_buf, gauss, F)
        return E

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        step(solver, frames[i], phi, rho)
    launches0 = G.gp_launch_count()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    outer, vcyc = [], []
    e0.record(stream)
    for i in range(args.steps):
        step(solver, frames[args.warmup + i], phi, rho)
        st = solver.stats()
        outer.append(st.outer_iterations)
        vcyc.append(st.vcycles)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    launches = G.gp_launch_count() - launches0
    stats = solver.stats()
    # second pass over the same frames with per-kernel-group CUDA-event timing
    # (the timing synchronises after each graph replay, so it is kept out of `value`)
    solver.ctx.gp_profile(True)
    for i in range(args.steps):
        step(solver, frames[args.warmup + i], phi, rho)
    torch.cuda.synchronize()
    prof = solver.ctx.gp_get_profile()
    solver.ctx.gp_profile(False)

    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    value = job_throughput(args.steps, world, ms_total / 1e3)

    if rank != 0:
        return None

    # level-0 size of the multigrid in use (band or full box)
    n_full = w.n_points
    n0 = int(round(n_full * (stats.wet_fraction if stats.split_active else 1.0)))
    prec_bytes = 4 if args.precision == 1 else 8
    total_ms = sum(v["ms"] for v in prof.values())
    dominant = max(prof, key=lambda k: prof[k]["ms"])
    roof = roofline_for(dominant, prof, n0, hbm, hbm_src, prec_bytes) or {}
    npx = w.grid[0] // 2
    shape_kernel = {0: "k_rb_sweep<float, 64, 8>", 1: "k_rb_sweep<float, 32, 16>", 2: "k_rb_sweep<float, 128, 4>",
                    3: "k_rb_sweep<float, 32, 8>", 4: "k_rb_sweep_rows<%d, 4>" % npx,
                    5: "k_rb_sweep_rows<%d, 6>" % npx, 6: "k_rb_sweep_rows<%d, 8>" % npx,
                    7: "k_rb_sweep_ws<%d, 6, 2>" % npx, 8: "k_rb_sweep_ws<%d, 4, 2>" % npx,
                    9: "k_rb_sweep_ws<%d, 6, 4>" % npx, 10: "k_rb_sweep_ws<%d, 4, 3>" % npx,
                    11: "k_rb_sweep_ws<%d, 16, 2>" % npx, 12: "k_rb_sweep_ws<%d, 14, 4>" % npx,
                    13: "k_rb_sweep_ws<%d, 14, 2>" % npx, 14: "k_rb_sweep_ws<%d, 12, 2>" % npx,
                    }.get(stats.sweep_shape, "k_rb_sweep")
    # the smoother's roofline covers its ordinary sweeps (16 B/pt); the first sweep of each
    # V-cycle starts from u = 0, reads no u (12 B/pt) and is timed in a group of its own
    smooth = roofline_for("smooth0", prof, n0, hbm, hbm_src, prec_bytes)
    if smooth is not None and args.precision == 1 and prof.get("smooth0_zero", {}).get("launches"):
        z = prof["smooth0_zero"]
        z_s = z["ms"] / 1e3 / z["launches"]
        smooth["from_zero"] = {"avg_launch_ms": z_s * 1e3, "algorithmic_bytes_per_launch": 12.0 * n0,
                               "achieved": 12.0 * n0 / z_s / 1e9, "unit": "GB/s"}
        smooth["kernel"] = shape_kernel + " (finest level, fused red-black sweep)"
        smooth["traffic"] = sweep_traffic(shape_kernel, w.name) if args.precision == 1 else None
    # the roofline object is the finest-level smoother's: the kernel with the largest share of the
    # step's device time in the launch list (a kernel group such as the coarse levels, made of many
    # short kernels, can outweigh it as a group)
    if smooth is not None:
        roof = dict(smooth)
    phases = {k: {"ms_per_step": v["ms"] / args.steps, "share": (v["ms"] / total_ms if total_ms else 0.0),
                  "launches_per_step": v["launches"] / args.steps} for k, v in prof.items() if v["launches"]}

    # comparators on the same frames: the plain FP64 full-box multigrid, and the
    # mixed-precision dry/wet split (FFT dry region + band multigrid, coupled)
    def time_variant(precision, split, label, tol=None, profile=False):
        sv = solver if (precision, split) == (args.precision, args.split) else make_solver(precision, split)
        step(sv, frames[0], phi, rho, tol)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        ncmp = max(1, min(args.steps, 3))
        c0.record(stream)
        for i in range(ncmp):
            step(sv, frames[args.warmup + i], phi, rho, tol)
        c1.record(stream)
        torch.cuda.synchronize()
        sst = sv.stats()
        # the solve alone (cold start, the last frame's eps and rho in place)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(ncmp):
            phi.zero_()
            sv.ctx.gp_solve(rho, phi, args.tol if tol is None else tol, check=True)
        s1.record(stream)
        torch.cuda.synchronize()
        out = {"solver": label, "value": ncmp / (c0.elapsed_time(c1) / 1e3), "unit": UNIT, "steps": ncmp,
               "solve_only_ms": s0.elapsed_time(s1) / ncmp,
               "tol": args.tol if tol is None else tol,
               "outer_iterations": sst.outer_iterations, "vcycles": sst.vcycles,
               "split_active": bool(sst.split_active), "wet_fraction": sst.wet_fraction}
        if profile:
            # a second, profiled pass: what bounds each kernel group of this solver
            sv.ctx.gp_profile(True)
            for i in range(ncmp):
                step(sv, frames[args.warmup + i], phi, rho, tol)
            torch.cuda.synchronize()
            pv = sv.ctx.gp_get_profile()
            sv.ctx.gp_profile(False)
            pb = 4 if precision == 1 else 8
            tot = sum(v["ms"] for v in pv.values())
            out["phases"] = {k: {"ms_per_step": v["ms"] / ncmp, "share": v["ms"] / tot if tot else 0.0}
                             for k, v in pv.items() if v["launches"]}
            out["smoother"] = roofline_for("smooth0", pv, n0 if not sst.split_active else
                                           int(round(n_full * sst.wet_fraction)), hbm, hbm_src, pb)
            out["residual64"] = roofline_for("res64", pv, n_full, hbm, hbm_src, pb)
        if sv is not solver:
            del sv
        return out

    comparator = None
    split_variant = None
    tight = None
    if not args.no_comparator:
        if not (args.precision == 0 and args.split == 0):
            comparator = time_variant(0, 0, "FP64 full-box multigrid (precision=0, split=0)", profile=True)
        if args.split == 0:
            split_variant = time_variant(args.precision, 1, "dry/wet split, %s (split=1)"
                                         % ("mixed" if args.precision == 1 else "FP64"))
        if args.tol > 1e-10:
            # the configurations' tolerance: below 1e-10 is where the mixed solve's outer
            # residual and phi update switch from df64 (FP32 pairs) to FP64
            tight = time_variant(args.precision, args.split, "the headline solver at tol 1e-10", tol=1e-10)

    # the same step with the paper's own dielectrics: Eq. 9-10 (kind 1) and Eq. 19
    # (kind 2, the lowest layer excluding the solvent below it), eps from every atom
    # image within the tail-bounded radius, on the same frames and solver settings
    def time_dielectric(kind):
        zl = W.lower_layer_zlim(at, w) if kind == 2 else 0.0
        sv = P.GPSolver(w.grid, w.cell, precision=args.precision, split=0, levels=w.levels,
                        sweep_shape=args.sweep_shape, n_dirichlet=n_dir, kind=kind, gamma_tail=args.gamma_tail,
                        zlim=zl)
        rv = torch.tensor(W.vdw_radii(at.Z), dtype=torch.float64, device=dev)

        def stepk(pos):
            sv.set_atoms(pos, radii=rv)
            sv.build_rho(pos, gauss, out=rho)
            phi.zero_()
            sv.ctx.gp_solve(rho, phi, args.tol, check=True)
            sv.ctx.gp_energy_forces(phi, rho, gauss, F)

        stepk(frames[0])
        torch.cuda.synchronize()
        ncmp = max(1, min(args.steps, 3))
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for i in range(ncmp):
            stepk(frames[args.warmup + i])
        c1.record(stream)
        torch.cuda.synchronize()
        sst = sv.stats()
        sv.ctx.gp_profile(True)
        for i in range(ncmp):
            stepk(frames[args.warmup + i])
        torch.cuda.synchronize()
        pv = sv.ctx.gp_get_profile()
        sv.ctx.gp_profile(False)
        out = {"dielectric": {1: "Eq. 9-10", 2: "Eq. 19 (z_lim %.3f A)" % zl}[kind],
               "value": ncmp / (c0.elapsed_time(c1) / 1e3), "unit": "steps/s", "steps": ncmp,
               "gamma_cutoff_A": sst.gamma_cutoff, "tol": args.tol,
               "outer_iterations": sst.outer_iterations, "vcycles": sst.vcycles,
               "eps_ms": pv["eps"]["ms"] / ncmp, "forces_eps_ms": pv["forces_eps"]["ms"] / ncmp,
               "step": "set_dielectric + build_rho + solve (cold) + energy_forces"}
        del sv
        return out

    dielectrics = None
    if not args.no_dielectrics and world == 1:
        dielectrics = {"eq9_10": time_dielectric(1), "eq19": time_dielectric(2)}

    # end to end through the public API with host buffers: every step copies its
    # inputs in from pinned memory and its result (phi, forces; E comes back with
    # the call) out to pinned memory, as a serving loop would: the copy-back of
    # step i runs on a copy stream while step i+1 computes into the other phi
    # buffer, and the clock stops after the last copy has landed
    e2e = None
    if not args.no_e2e:
        pos_h = [torch.tensor(traj[i % len(traj)], dtype=torch.float64).pin_memory() for i in range(args.steps)]
        gauss_h = torch.tensor(gauss_np, dtype=torch.float64).pin_memory()
        phi_h = [torch.empty(solver.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        F_h = [torch.empty((len(at.Z), 3), dtype=torch.float64).pin_memory() for _ in range(2)]
        pos_d = torch.empty((len(at.Z), 3), dtype=torch.float64, device=dev)
        phi_d = [phi, torch.zeros_like(phi)]
        F_d = [F, torch.zeros_like(F)]
        copy_stream = torch.cuda.Stream()
        done = [torch.cuda.Event(), torch.cuda.Event()]
        for d in done:
            d.record(copy_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            b = i % 2
            done[b].synchronize()                       # the copy-back of step i-2 from these buffers landed
            pos_d.copy_(pos_h[i], non_blocking=True)
            gauss.copy_(gauss_h, non_blocking=True)
            step(solver, pos_d, phi_d[b], rho)
            F_d[b].copy_(F)
            ready = torch.cuda.Event()
            ready.record()
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ready)
                phi_h[b].copy_(phi_d[b], non_blocking=True)
                F_h[b].copy_(F_d[b], non_blocking=True)
                done[b].record(copy_stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2e = {"value": args.steps / (t1 - t0), "unit": UNIT,
               "h2d_bytes_per_step": int(pos_h[0].numel() * 8 + gauss_h.numel() * 8),
               "d2h_bytes_per_step": int(phi_h[0].numel() * 8 + F_h[0].numel() * 8 + 16)}

    # warm-started MD frames (graph-captured fixed-count outer solve + forces)
    md = None
    if args.md_frames > 0:
        md = md_frames_run(dev, args.md_frames, 5, args.precision, 0, args.graph_outer, args.tol, rank)

    cpu = None
    oracle_full = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_sample(w, at, traj[0], budget_s=args.cpu_budget, tol=args.tol)
        cpu = {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
               "sample": cpu["sample"]}
        # a COMPLETE oracle step, measured, on the small full-box workload
        # (one process, then every host core)
        wc = W.WORKLOADS["fp64_fullbox_32x32x64"]
        atc, trc, _ = make_inputs(wc, 1)
        oracle_full = [oracle_full_step(wc, atc, trc[0], args.tol, workers=k) for k in (1, os.cpu_count() or 1)]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_label(args.precision, args.tol), "data": "synthetic",
        "precision": precision_detail(args.precision, args.tol),
        "config": {"workload": w.name, "grid": list(w.grid), "cell_A": list(w.cell), "atoms": int(len(at.Z)),
                   "tol": args.tol, "precision": "mixed" if args.precision == 1 else "fp64",
                   "dielectric": {0: "erf product",
                                  1: "Eq. 9-10 (beta 2.4, image sum to %.1f A, tail < %.0e)"
                                     % (stats.gamma_cutoff, args.gamma_tail),
                                  2: "Eq. 19 (beta 2.4, image sum to %.1f A, tail < %.0e, z_lim %.3f A)"
                                     % (stats.gamma_cutoff, args.gamma_tail, zlim)}[args.kind],
                   "split": bool(args.split), "split_active": bool(stats.split_active),
                   "wet_fraction": stats.wet_fraction, "levels": stats.levels,
                   "outer_iterations_mean": float(np.mean(outer)), "vcycles_mean": float(np.mean(vcyc)),
                   "l2": "inputs larger than L2 (FP64 fields of 113 MB each)",
                   "step": "set_dielectric + build_rho + solve (cold) + energy_forces",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof, "smoother": smooth, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk, "fp64_fullbox": comparator, "split_scheme": split_variant, "tol_1e-10": tight,
        "md": md, "oracle_full_step": oracle_full, "dielectrics": dielectrics, "phases": phases,
        "dominant_kernel_group": dominant,
    }
    return line


# ----------------------------------------------------------------------------- MD frames
def md_frames_run(dev, frames, warmup, precision, split, graph_outer, tol, seed, world=1):
    """Consecutive MD frames of the 128x128x256, 144-atom workload (seeded
    300 K Maxwell velocities, dt 0.5 fs): each frame rebuilds eps and rho,
    solves warm-started from the previous phi with `graph_outer` corrections
    captured as one CUDA graph, then energy + forces. Frames/s, per-frame
    p50 / p99 latency (CUDA events) and the outer corrections and V-cycles a
    warm frame needed."""
    import torch
    import paper_0904_4887_gb300 as P

    w = W.WORKLOADS["md_128x128x256"]
    at, traj, gauss_np = make_inputs(w, frames + warmup, seed=seed)
    gauss = torch.tensor(gauss_np, dtype=torch.float64, device=dev)
    pos = [torch.tensor(traj[i], dtype=torch.float64, device=dev) for i in range(frames + warmup)]
    # two outer corrections of 4 CG iterations each in the graph: a warm start needs
    # fewer V-cycles than the cold headline solve
    s = P.GPSolver(w.grid, w.cell, precision=precision, split=split, graph_outer=graph_outer, inner=4)
    rho, phi = s.zeros(), s.zeros()
    F = torch.zeros((len(at.Z), 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def frame(p):
        s.set_atoms(p)
        s.build_rho(p, gauss, out=rho)
        st = s.ctx.gp_solve(rho, phi, tol, check=False)
        if st != 0:
            raise RuntimeError("frame solve failed with status %d" % st)
        s.ctx.gp_energy_forces(phi, rho, gauss, F)

    for i in range(warmup):
        frame(pos[i])
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(frames + 1)]
    outer, vcyc = [], []
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(frames):
        frame(pos[warmup + i])
        evs[i + 1].record(stream)
        st = s.stats()
        outer.append(st.outer_iterations)
        vcyc.append(st.vcycles)
    torch.cuda.synchronize()
    lat = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(frames)])
    total = evs[0].elapsed_time(evs[frames])
    return {"workload": w.name, "atoms": int(len(at.Z)), "frames": frames, "tol": tol,
            "graph_outer": graph_outer, "value": frames / (total / 1e3), "unit": "frames/s", "total_ms": total,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "outer_iterations_mean": float(np.mean(outer)), "vcycles_per_frame_mean": float(np.mean(vcyc)),
            "step": "set_dielectric + build_rho + warm-started graph-captured solve + energy_forces"}


def md_arm(args, rank, world):
    """--mode md: the MD frames above as their own JSON line."""
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    r = md_frames_run(dev, args.frames, args.warmup, args.precision, args.split, args.graph_outer, args.tol,
                      rank, world)
    total = max_over_ranks(r["total_ms"], world, dev)
    if rank != 0:
        return None
    return {"metric": "MD frames/s (warm-started graph-captured solve + forces)",
            "value": job_throughput(r["frames"], world, total / 1e3),
            "unit": "frames/s", "n_gpus": world, "steps": r["frames"], "warmup": args.warmup,
            "ms_per_step": total / r["frames"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_label(args.precision, args.tol), "data": "synthetic",
            "config": {"workload": r["workload"], "atoms": r["atoms"], "tol": args.tol,
                       "graph_outer": args.graph_outer, "split": bool(args.split),
                       "outer_iterations_mean": r["outer_iterations_mean"],
                       "vcycles_per_frame_mean": r["vcycles_per_frame_mean"]},
            "latency_ms": r["latency_ms"]}


# ----------------------------------------------------------------------------- sixth-order residual
# FP64 flops per point of k_residual6 (an FMA counts 2): per axis 8 + 8 for the
# two first-derivative sums (phi, eps), 10 for the second-derivative sum, 3 to
# combine them; 5 to weight the axes by 1/h^2; 1 + 1 + 2 for -4 pi rho, the
# subtraction and mu eps; 2 for the r^2 partial sum
FD6_FLOPS_PER_POINT = 3 * (8 + 8 + 10 + 3) + 5 + 4 + 2
FD6_BYTES_PER_POINT = 32          # read phi, eps, rho (FP64), write r (FP64)
FD6_CALLS_PER_STEP = 100


def residual6_arm(args, rank, world):
    """Time gp_residual6 (the sixth-order residual of Eq. 16-18, FP64) on the
    workload's dielectric and a solved phi: a step is 100 residual evaluations,
    each the kernel, the finalisation of its partial sums and the 8-byte
    readback of the sum of squares (no norm of b).
    Reported against the nominal FP64 rate (the kernel is FP64-ALU bound) with
    the HBM rate of its algorithmic bytes beside it."""
    import torch
    import paper_0904_4887_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.WORKLOADS[args.workload]
    at, traj, gauss_np = make_inputs(w, 1, seed=rank)
    s = P.GPSolver(w.grid, w.cell, precision=args.precision, levels=w.levels)
    pos = torch.tensor(traj[0], dtype=torch.float64, device=dev)
    gauss = torch.tensor(gauss_np, dtype=torch.float64, device=dev)
    s.set_atoms(pos)
    rho = s.build_rho(pos, gauss)
    phi = s.solve(rho, tol=1e-8)
    r = s.zeros()
    import ctypes
    from paper_0904_4887_gb300 import gp as G

    def call():
        # rel_host NULL: the kernel, the finalisation of its partial sums and the readback
        st = s.ctx._lib.gp_residual6(s.ctx._h, G._ptr(rho), G._ptr(phi), ctypes.c_double(0.0), G._ptr(r), None)
        if st != 0:
            raise RuntimeError("gp_residual6 failed with status %d" % st)

    for _ in range(args.warmup):
        call()
    stream = torch.cuda.current_stream()
    n = int(np.prod(w.grid))
    clocks = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = G.gp_launch_count()
    e0.record(stream)
    for _ in range(args.steps * FD6_CALLS_PER_STEP):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = G.gp_launch_count() - launches0
    total = max_over_ranks(e0.elapsed_time(e1), world, dev)
    if rank != 0:
        return None
    per_call_s = total / 1e3 / (args.steps * FD6_CALLS_PER_STEP)
    gflops = FD6_FLOPS_PER_POINT * n / per_call_s / 1e9
    gbs = FD6_BYTES_PER_POINT * n / per_call_s / 1e9
    hbm, hbm_src = load_peaks()
    return {"metric": "sixth-order FP64 residual evaluations/s (Eq. 16-18)",
            "value": job_throughput(args.steps * FD6_CALLS_PER_STEP, world, total / 1e3),
            "unit": "residuals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid), "atoms": int(len(at.Z)),
                       "calls_per_step": FD6_CALLS_PER_STEP,
                       "l2": "inputs larger than L2 (4 FP64 fields of %d MB)" % (8 * n // 10 ** 6)},
            "roofline": {"bound": "alu", "achieved": gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": gflops / FP64_PEAK_GFLOPS, "peak_source": "nominal FP64 (non-tensor)",
                         "kernel": "k_residual6", "flops_per_point": FD6_FLOPS_PER_POINT,
                         "avg_call_ms": per_call_s * 1e3, "traffic": None},
            "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "peak_source": hbm_src,
                    "bytes_per_point": FD6_BYTES_PER_POINT},
            "gpu_launches": int(launches),
            "clocks": clk}


# ----------------------------------------------------------------------------- sixth-order solve
def solve6_arm(args, rank, world):
    """--mode solve6: the sixth-order path of Sec. III (Eq. 16-18) on the
    workload: a step is eps + rho, the bordered solve to `tol`, the adjoint
    solve, energy and forces through the adjoint, on a new frame each step."""
    import torch
    import paper_0904_4887_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.WORKLOADS[args.workload]
    nfr = args.warmup + args.steps
    at, traj, gauss_np = make_inputs(w, max(nfr, 2), seed=rank)
    gauss = torch.tensor(gauss_np, dtype=torch.float64, device=dev)
    frames = [torch.tensor(traj[i % len(traj)], dtype=torch.float64, device=dev) for i in range(nfr)]
    s = P.GPSolver(w.grid, w.cell, precision=args.precision, levels=w.levels)
    rho, phi, lam = s.zeros(), s.zeros(), s.zeros()
    F = torch.zeros((len(at.Z), 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    stats = []

    def step(pos):
        s.set_atoms(pos)
        s.build_rho(pos, gauss, out=rho)
        phi.zero_()
        lam.zero_()
        mu, st = s.ctx.gp_solve6(rho, phi, args.tol, check=False)
        st1 = s.stats()
        nu, st2 = s.ctx.gp_adjoint6(rho, lam, args.tol, check=False)
        if st != 0 or st2 != 0:
            raise RuntimeError("sixth-order solve failed: %d %d" % (st, st2))
        s.ctx.gp_energy_forces6(phi, mu, lam, rho, gauss, F)
        return st1.outer_iterations, st1.inner_iterations

    for i in range(args.warmup):
        step(frames[i])
    from paper_0904_4887_gb300 import gp as G
    launches0 = G.gp_launch_count()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        stats.append(step(frames[args.warmup + i]))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = G.gp_launch_count() - launches0
    total = max_over_ranks(e0.elapsed_time(e1), world, dev)
    if rank != 0:
        return None
    return {"metric": "sixth-order solves/s (Eq. 16-18: bordered solve + adjoint + forces)",
            "value": job_throughput(args.steps, world, total / 1e3), "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (FGMRES, operator, residual)+%s (multigrid preconditioner)+df64 (fields)"
                     % ("f32" if args.precision == 1 else "f64"),
            "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid), "atoms": int(len(at.Z)), "tol": args.tol,
                       "restart": 12, "fgmres_cycles_mean": float(np.mean([a for a, _ in stats])),
                       "krylov_and_pcg_steps_mean": float(np.mean([b for _, b in stats])),
                       "step": "set_dielectric + build_rho + gp_solve6 + gp_adjoint6 + gp_energy_forces6"},
            "gpu_launches": int(launches), "clocks": clk}


# ----------------------------------------------------------------------------- oracle (CPU) timing
def _split(seq, parts):
    """`seq` in `parts` contiguous chunks of near-equal length (none empty)."""
    parts = max(1, min(parts, len(seq)))
    k, r = divmod(len(seq), parts)
    out, i = [], 0
    for p in range(parts):
        j = i + k + (1 if p < r else 0)
        out.append(seq[i:j])
        i = j
    return out


_W = {}


def _worker_init(payload):
    from oracle import gp_oracle  # noqa: F401  (imported once per worker, before the clock)
    _W.update(payload)


def _w_product(idx):
    from oracle import gp_oracle as O
    return O.dielectric_product(_W["grid"], _W["cell"], _W["pos"][idx])


def _w_rho(idx):
    from oracle import gp_oracle as O
    at = _W["at"]
    return O.charge_density_raw(_W["grid"], _W["cell"], _W["pos"][idx], at.Z[idx], at.sigma_core[idx],
                                at.sigma_cloud[idx])


def _w_grad(idx):
    from oracle import gp_oracle as O
    at = _W["at"]
    Ge, Gr = O.energy_gradient(_W["phi"], _W["grid"], _W["cell"], _W["pos"], at.Z, at.sigma_core, at.sigma_cloud,
                               atoms=list(idx))
    return Ge[idx], Gr[idx]


def oracle_full_step(w, at, pos, tol, workers=1):
    """One COMPLETE step of the FP64 oracle, timed part by part: eps, rho, the
    PCG solve to `tol`, the energy, and the forces of every atom. With
    workers > 1 the per-atom loops (the eps product and the density over atom
    chunks, the gradient of each atom) run in that many spawned processes,
    started before the clock; the solve stays one NumPy process (its FFTs and
    stencils are single-threaded)."""
    from oracle import gp_oracle as O
    grid, cell = w.grid, w.cell
    h = O.spacing(grid, cell)
    n = len(at.Z)
    chunks = _split(np.arange(n), workers)
    pool = None

    def start_pool(payload):
        # workers are started (and their imports done) before the clock runs
        import multiprocessing as mp
        pl = mp.get_context("spawn").Pool(workers, initializer=_worker_init, initargs=(payload,))
        pl.map(abs, range(workers))
        return pl

    if workers > 1:
        pool = start_pool({"grid": grid, "cell": cell, "pos": pos, "at": at})
    try:
        t0 = time.perf_counter()
        if pool:
            P = np.ones((grid[2], grid[1], grid[0]))
            for part in pool.map(_w_product, chunks):
                P *= part
        else:
            P = O.dielectric_product(grid, cell, pos)
        eps = 1.0 + (O.DielectricParams().eps0 - 1.0) * P
        t1 = time.perf_counter()
        if pool:
            rho = sum(pool.map(_w_rho, chunks))
        else:
            rho = O.charge_density_raw(grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud)
        rho = rho - rho.mean()
        t2 = time.perf_counter()
        phi, info = O.solve(rho, eps, h, tol=tol)
        t3 = time.perf_counter()
        E = O.energy(rho, phi, grid, cell)
        t_energy = time.perf_counter() - t3
        if pool:
            pool.close()
            pool.join()
            pool = start_pool({"grid": grid, "cell": cell, "pos": pos, "at": at, "phi": phi})
        t4 = time.perf_counter()
        if pool:
            parts = pool.map(_w_grad, chunks)
            F = -np.concatenate([ge + gr for ge, gr in parts])
        else:
            Ge, Gr = O.energy_gradient(phi, grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud)
            F = -(Ge + Gr)
        t5 = time.perf_counter()
    finally:
        if pool:
            pool.close()
            pool.join()
    return {"workload": w.name, "workers": workers, "tol": tol, "pcg_iterations": info.iterations,
            "residual": info.residual, "t_eps_s": t1 - t0, "t_rho_s": t2 - t1, "t_solve_s": t3 - t2,
            "t_energy_s": t_energy, "t_forces_s": t5 - t4,
            "t_step_s": (t1 - t0) + (t2 - t1) + (t3 - t2) + t_energy + (t5 - t4),
            "energy": E, "max_force": float(np.max(np.abs(F)))}


def oracle_sample(w, at, pos, budget_s=20.0, tol=1e-8):
    """The FP64 oracle's step time on a bounded sample of the workload, scaled
    to one step (an estimate): eps and rho over m of the n atoms (their cost is
    one pass per atom, so x n/m), PCG iterations on the full grid for about a
    third of the budget (the iteration count for `tol` comes from the
    contraction measured over them: the one modelled quantity), and the
    gradient of 1 and of 3 atoms (a fixed part, the dielectric product and the
    face gradients, plus n times the per-atom part)."""
    from oracle import gp_oracle as O

    grid, cell = w.grid, w.cell
    h = O.spacing(grid, cell)
    n = len(at.Z)
    m = max(2, min(n, int(n * min(1.0, budget_s / 400.0))))
    sel = np.arange(m)
    t0 = time.perf_counter()
    P = O.dielectric_product(grid, cell, pos[sel])
    t_eps = (time.perf_counter() - t0) * n / m
    t0 = time.perf_counter()
    O.charge_density_raw(grid, cell, pos[sel], at.Z[sel], at.sigma_core[sel], at.sigma_cloud[sel])
    t_rho = (time.perf_counter() - t0) * n / m
    # (the density of the sampled atoms also serves as the right-hand side below)
    eps = 1.0 + 77.36 * P
    rho = O.charge_density(grid, cell, pos[sel], at.Z[sel], at.sigma_core[sel], at.sigma_cloud[sel])
    t0 = time.perf_counter()
    O.solve(rho, eps, h, tol=1e-300, maxiter=1)
    t_one = time.perf_counter() - t0
    # k iterations for about a third of the budget; their mean contraction sets the count
    k = int(max(2, min(40, 0.33 * budget_s / max(t_one, 1e-3))))
    t0 = time.perf_counter()
    phi, info = O.solve(rho, eps, h, tol=1e-300, maxiter=k)
    t_it = (time.perf_counter() - t0) / k
    rate = max(min(info.residual ** (1.0 / k), 0.95), 0.05)
    iters = math.ceil(math.log(tol) / math.log(rate))
    t_solve = t_it * iters
    # the gradient has a fixed part (the dielectric product, the face gradients) and a
    # part per atom: time 1 and 3 atoms
    t0 = time.perf_counter()
    O.energy_gradient(phi, grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud, atoms=[0])
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.energy_gradient(phi, grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud, atoms=[0, 1, 2])
    t3 = time.perf_counter() - t0
    per_atom = max((t3 - t1) / 2.0, 0.0)
    t_force = max(t1 - per_atom, 0.0) + n * per_atom
    t_step = t_eps + t_rho + t_solve + t_force
    return {"value": 1.0 / t_step, "cores": 1, "t_step_s": t_step,
            "sample": ("%s: eps and rho over %d of %d atoms (x%.0f), %d PCG iterations on the full grid x %d "
                       "needed for %.0e (their mean contraction %.3f: the modelled part), gradient of 1 and 3 "
                       "atoms (fixed part + %d x the per-atom part); one NumPy process; an estimate of one "
                       "complete step"
                       % (w.name, m, n, n / m, k, iters, tol, rate, n))}


def reference_arm(args, rank, world):
    """The oracle as the reference: each step is one bounded sample of the
    workload (oracle_sample), timed as it runs; `value` is the complete step
    that sample estimates, in solves/s, and ms_per_step the sample's own wall
    time, so the timed region is what this process actually spent."""
    if rank != 0:
        return None
    w = W.WORKLOADS[args.workload]
    at, traj, _ = make_inputs(w, 2)
    budget = max(2.0, min(args.cpu_budget, 150.0 / max(1, args.steps + args.warmup)))
    est, wall = [], []
    last = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle_sample(w, at, traj[i % len(traj)], budget_s=budget, tol=args.tol)
        if i >= args.warmup:
            wall.append(time.perf_counter() - t0)
            est.append(r["t_step_s"])
            last = r
    value = 1.0 / float(np.mean(est))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(wall)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid), "cell_A": list(w.cell), "atoms": int(len(at.Z)),
                       "tol": args.tol, "solver": "FP64 CPU oracle (FFT-preconditioned CG)",
                       "step": "one bounded sample of a complete oracle step; value = 1 / the step it estimates"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def oracle_arm(args, rank, world):
    """--mode oracle: one complete oracle step on the workload, timed single-
    process and with every host core; prints its own JSON line (not a bench
    line: the reference figures of the CPU baseline)."""
    if rank != 0:
        return None
    w = W.WORKLOADS[args.workload]
    at, traj, _ = make_inputs(w, 1)
    out = {"mode": "oracle", "workload": w.name, "grid": list(w.grid), "atoms": int(len(at.Z)), "tol": args.tol,
           "host_cores": os.cpu_count(), "runs": []}
    for workers in sorted(set(args.oracle_workers)):
        workers = os.cpu_count() if workers <= 0 else workers
        r = oracle_full_step(w, at, traj[0], args.tol, workers=workers)
        r["solves_per_s"] = 1.0 / r["t_step_s"]
        out["runs"].append(r)
        print(json.dumps(r), file=sys.stderr, flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gp", choices=["gp", "reference"])
    ap.add_argument("--workload", default="mixed_192x192x384", choices=sorted(W.WORKLOADS))
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-dielectrics", action="store_true",
                    help="skip the steps with the paper's Eq. 9-10 and Eq. 19 dielectrics")
    ap.add_argument("--mode", default="step", choices=["step", "md", "residual6", "solve6", "oracle"])
    ap.add_argument("--oracle-workers", type=int, nargs="+", default=[1, 0],
                    help="--mode oracle: process counts to time the complete step with (0 = every host core)")
    ap.add_argument("--frames", type=int, default=100)
    ap.add_argument("--graph-outer", type=int, default=2)
    ap.add_argument("--md-frames", type=int, default=40,
                    help="step mode: warm-started MD frames timed after the headline (0 = none)")
    ap.add_argument("--kind", type=int, default=0, choices=[0, 1, 2],
                    help="dielectric: 0 erf product (the workloads), 1 Eq. 9-10 dummy density, "
                         "2 Eq. 19 (solvent excluded below the lowest layer)")
    ap.add_argument("--n-dirichlet", type=int, default=-1,
                    help="split: Dirichlet planes (-1: 0 = the whole dry run for --kind 2, else 1)")
    ap.add_argument("--gamma-tail", type=float, default=1e-13,
                    help="--kind 1, 2: bound on the part of gamma's image sum left out")
    ap.add_argument("--nu-coarse", type=int, default=None,
                    help="smoothing sweeps on the levels below the finest (default: the library's)")
    ap.add_argument("--nu1", type=int, default=None, help="pre-smoothing sweeps (default: the library's)")
    ap.add_argument("--nu2", type=int, default=None, help="post-smoothing sweeps (default: the library's)")
    ap.add_argument("--inner", type=int, default=None,
                    help="CG iterations of the first outer correction (default: the library's)")
    ap.add_argument("--sweep-shape", type=int, default=-1,
                    help="finest-level smoother tile (-1: autotuned; fixed shapes keep profiles comparable)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gp":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "gp":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        line = reference_arm(args, rank, world)
    elif args.mode == "oracle":
        line = oracle_arm(args, rank, world)
    elif args.mode == "md":
        line = md_arm(args, rank, world)
    elif args.mode == "residual6":
        line = residual6_arm(args, rank, world)
    elif args.mode == "solve6":
        line = solve6_arm(args, rank, world)
    else:
        line = gpu_arm(args, rank, world)
    if line is not None:
        print(json.dumps(line))
    if world > 1 and args.impl == "gp":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
