#!/usr/bin/env python3
"""Benchmark of the multigrid CGKS hot path on one GB300 (or N replicas).

A step is one 3-level V-cycle (Sec. 4.2 of the paper: a CGKS pre-smoothing step, the defect at the
new state, KFVS forward-Euler smoothing with FAS forcing on the two agglomerated levels, injection
correction) on the laminar boundary-layer box: 96 x 64 x 69 grid, wall-normal grading 1e-4 x 1.1
(capped at 2 dx), 42 wall layers of prisms and Kuhn tetrahedra above (1,511,424 cells), no-slip wall,
Mach 0.5, Re 1e4, Pr 0.72, seeded synthetic mesh and free-stream start.  The metric is fine cells x
V-cycles per second, for the FP64 V-cycle (value) and the mixed-precision one (mixed), with a
roofline entry for every kernel of the cycle; `converge` reports wall times to a 1e-10 residual drop
of single-grid FP64, FP64 V-cycle and mixed V-cycle (compression factor on) on small ramps and
boundary layers, a ramp that is not launch-bound and the 96 x 4 x 69 slab of the workload's layout,
with each final state's error against the oracle's own steady state where one is stored.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-converge-slab]

Multi-GPU: one process per GPU (torchrun); each rank runs an independent replica (the method is
not partitioned in this build), the step time is the maximum over ranks and the value counts the
cells of all replicas.  --impl reference times the CPU oracle (the plain C implementation used by
the tests) on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-iters/s; wall time to 1e-10 residual drop: FP64 vs mixed V-cycle"
UNIT = "Mcell-iters/s"
# the x-out side is the extrapolation outflow (boundary kind 5): a Riemann-invariant farfield there cuts
# through the boundary layer, and measured, admits distinct discrete steady states and holds the
# V-cycle at a 3e-5 drop with the compression factor on
WORKLOAD = dict(nx=96, ny=64, nz=69, outflow=5)
PARAMS = dict(mach=0.5, reynolds=1e4, prandtl=0.72, gamma=1.4, viscous=1, n_levels=3, cfl_fine=0.5,
              cfl_coarse=0.9, coarse_steps=2, agglo_seed=0)
# bounded sample of the same workload for the CPU oracle: 4 of its 64 periodic columns in y, i.e. the
# same x-z layout and physics (82,944 cells)
SAMPLE = dict(nx=96, ny=4, nz=69, outflow=5)
# FP64 floating-point operations per Gauss point of the gas-kinetic flux kernel (2 per DFMA, 1 per
# DADD/DMUL), from the ncu instruction counts of a full capture of the kernel on the 48x32x32 box;
# the kernel's own arithmetic, all of which the method needs
FLOP_PER_GP = 3249.5
# DRAM bytes (read + write) per Gauss point of the same kernel from the same capture (None when the
# kernel has changed since)
DRAM_BYTES_PER_GP = 172.3
# FP64 operations per unit of the other kernels bound by the FP64 pipe, from ncu instruction counts
# on the same box (2 per DFMA, 1 per DMUL or DADD; averages over the launches of a V-cycle):
# reconstruction per cell (DFMA 1,464.3, DMUL 318.1, DADD 155.6), gather with the gradient update per
# Gauss point seen from a cell (DFMA 16.06, DMUL 2.17, DADD 5.11), the flux alone of the V-cycle's
# defect per Gauss point (DFMA 1,179.1, DMUL 490.4, DADD 230.0), coarse KFVS face flux per face (DFMA
# 183.8, DMUL 66.5, DADD 30.9: the launches of a V-cycle weighted by their faces).  The residual-only gather of the defect (5.6 FLOP per point seen), the
# coarse time step and the KFVS gather are latency-bound gathers, reported against HBM.
FLOP_PER_CELL_RECON = 3402.2
FLOP_PER_GP_SIDE_GATHER = 39.39
FLOP_PER_GP_FLUX = 3078.6
FLOP_PER_FACE_KFVS = 464.8
ALU_KERNELS = {"k_gks_points": FLOP_PER_GP, "k_reconstruct": FLOP_PER_CELL_RECON,
               "k_gather": FLOP_PER_GP_SIDE_GATHER, "k_kfvs_faces": FLOP_PER_FACE_KFVS,
               "k_gks_points_flux": FLOP_PER_GP_FLUX}


def workload_name(w):
    import meshgen as mg
    _, npz = mg.wall_layout(w["nx"], w["nz"])
    cells = w["nx"] * w["ny"] * (2 * npz + 6 * (w["nz"] - npz))
    return (f"3-level FP64 V-cycle, laminar boundary-layer box {w['nx']}x{w['ny']}x{w['nz']} "
            f"({cells:,} cells: {npz} prism layers + Kuhn tetrahedra), no-slip wall, farfield inflow and top, "
            f"extrapolation outflow, M 0.5, Re 1e4, Pr 0.72")


def launches_per_vcycle(P, history=False):
    """Kernels launched by one V-cycle (fine step, defect, restriction, coarse levels, corrections).
    FP64 (FAS): a coarse level evaluates its KFVS residual at W^0 for the forcing and the first step
    (faces + gather) plus the forcing kernel; mixed (defect correction): the first step needs no
    residual (the defect is the restricted one) and later residuals are FP32 directional derivatives
    (faces + gather)."""
    dtm = 2 if P["dt_mode"] == 1 else 0
    fine_step = 3 + dtm + (2 if history else 0)
    n = fine_step * max(P["pre"], 1)
    nl = P["n_levels"]
    C = P["coarse_steps"]
    if nl > 1:
        n += 3 + dtm + 1  # defect (reconstruct, points, gather) + restriction

        def coarse(l):
            k = (0 if P["precision"] == 1 else 3) + C * (1 + dtm + 1) + (C - 1) * 2
            if l + 1 < nl:
                k += 2 + 1 + coarse(l + 1) + 1 + P["post"] * (2 + 1 + dtm + 1)
            return k
        n += coarse(1) + 1 + P["post"] * fine_step
    return n


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return None
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x, world, device):
    """Largest x over the ranks of the process group (x itself on one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells_per_replica, steps, ms_max, world):
    """Whole-job Mcell-iters/s: every replica advanced its cells `steps` times, and the job took
    the slowest rank's time."""
    return world * cells_per_replica * steps / (ms_max * 1e-3) / 1e6


def host_cores():
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample(sample, cycles):
    """The oracle (as it stands) on a bounded sample of the workload: fine cells x V-cycles per
    second after one warm-up cycle, with the threads OpenMP was given (OMP_NUM_THREADS)."""
    import meshgen as mg
    import oracle
    oracle.build()
    mesh = mg.wall_box(**sample)
    M = oracle.Mesh(mesh)
    S = oracle.Solver(M, oracle.params(**PARAMS))
    W, G = mg.uniform_state(M.nc, mach=PARAMS["mach"])
    S.set_state(W, G)
    S.run(1, multigrid=True)  # warm-up (first touch of the work arrays)
    t0 = time.perf_counter()
    S.run(cycles, multigrid=True)
    dt = time.perf_counter() - t0
    return {"value": M.nc * cycles / dt / 1e6, "cells": M.nc, "cycles": cycles, "seconds": dt,
            "threads": int(os.environ.get("OMP_NUM_THREADS", host_cores()))}


def cpu_baseline():
    """The oracle timed on the host cores at one thread and at all cores, each in a child process
    (OpenMP fixes its thread count at start-up): V-cycles of the workload's layout and physics on
    bounded samples of 4 (all cores) and 2 (one thread) of its 64 periodic columns in y."""
    cores = host_cores()
    runs = {}
    for key, threads, sample, cycles in (("all_cores", cores, SAMPLE, 6),
                                         ("one_thread", 1, dict(SAMPLE, ny=2), 2)):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample",
                            json.dumps({"sample": sample, "cycles": cycles})],
                           env=env, capture_output=True, text=True, timeout=900)
        if r.returncode:
            raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
        runs[key] = json.loads(r.stdout.strip().splitlines()[-1])
    a, o = runs["all_cores"], runs["one_thread"]
    return {"value": a["value"], "unit": UNIT, "cores": a["threads"], "kind": "oracle",
            "sample": f"{a['cycles']} V-cycles of the same layout and physics at {SAMPLE['nx']}x{SAMPLE['ny']}x"
                      f"{SAMPLE['nz']} ({a['cells']:,} cells), after 1 warm-up cycle",
            "seconds": a["seconds"],
            "one_thread": {"value": o["value"], "unit": UNIT, "cores": 1,
                           "sample": f"{o['cycles']} V-cycles at {SAMPLE['nx']}x2x{SAMPLE['nz']} ({o['cells']:,} "
                                     f"cells), after 1 warm-up cycle", "seconds": o["seconds"]},
            "parallel_speedup": a["value"] / o["value"]}


def measured_hbm_peak():
    """The measured HBM copy bandwidth of this GPU (GB/s), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        return None


def kernel_rooflines(stats, steps, fp64_peak, hbm_peak):
    """Per-kernel roofline of the timed region: stats maps a kernel name to (ms, launches, units,
    algorithmic bytes) summed over the timed V-cycles.  FP64-pipe kernels: achieved TFLOP/s = FLOP
    per unit x units / time against the measured FMA-chain peak; the rest: algorithmic bytes / time
    against the measured HBM copy bandwidth."""
    out = {}
    for name, (ms, n, units, by) in stats.items():
        if n == 0 or ms <= 0:
            continue
        row = {"launches_per_step": n / steps, "ms_per_launch": ms / n, "ms_per_step": ms / steps,
               "units_per_launch": units / n}
        if name in ALU_KERNELS:
            ach = ALU_KERNELS[name] * units / (ms * 1e-3) / 1e12
            row.update(bound="alu", unit="TFLOP/s", achieved=ach, peak=fp64_peak,
                       frac=ach / fp64_peak if fp64_peak else None, flop_per_unit=ALU_KERNELS[name])
            # the memory side of the same launches, for comparison
            row["hbm_GBps"] = by / (ms * 1e-3) / 1e9
            row["hbm_frac"] = row["hbm_GBps"] / hbm_peak if hbm_peak else None
            row["algorithmic_bytes_per_launch"] = by / n
        else:
            ach = by / (ms * 1e-3) / 1e9
            row.update(bound="hbm", unit="GB/s", achieved=ach, peak=hbm_peak,
                       frac=ach / hbm_peak if hbm_peak else None, algorithmic_bytes_per_launch=by / n)
        out[name] = row
    return out


def _state_diff(Wa, Wb):
    """max |Wa - Wb| over each variable's largest |Wb| (momentum components share one scale)."""
    import numpy as np
    sw = np.abs(Wb).max(axis=1)
    sw[1:4] = sw[1:4].max()
    return float((np.abs(Wa - Wb).max(axis=1) / sw).max())


def converge_cases(slab):
    """Cases driven to a 1e-10 residual drop: (name, mesh factory, physics, max iterations, golden)
    with golden the name of the oracle's stored steady state of the same case (or None)."""
    import meshgen as mg
    vis = dict(mach=0.5, reynolds=1e4, prandtl=0.72, viscous=1)
    out = mg.BC_SUPER_OUT
    cases = [("Mach 3 compression ramp 32x16x2, 2 prism layers + hexahedra, inviscid",
              lambda: mg.ramp_box(32, 16, 2, n_prism=2), dict(mach=3.0), 20000, "ramp_32x16x2"),
             ("Mach 3 compression ramp 64x32x8, 4 prism layers + hexahedra, inviscid",
              lambda: mg.ramp_box(64, 32, 8, n_prism=4), dict(mach=3.0), 20000, "ramp_64x32x8"),
             ("Mach 3 compression ramp 128x64x16, 8 prism layers + hexahedra, inviscid (not launch-bound)",
              lambda: mg.ramp_box(128, 64, 16, n_prism=8), dict(mach=3.0), 20000, None),
             ("boundary layer 12x2x12 (first 2e-3, ratio 1.3), 12 prism layers, extrapolation outflow, M 0.5, Re 1e4",
              lambda: mg.wall_box(12, 2, 12, first=2e-3, ratio=1.3, outflow=out), vis, 100000, "wall_12x2x12"),
             ("boundary layer 24x4x24 (first 1e-3, ratio 1.2), 17 prism layers + Kuhn tetrahedra, extrapolation "
              "outflow, M 0.5, Re 1e4", lambda: mg.wall_box(24, 4, 24, first=1e-3, ratio=1.2, outflow=out), vis, 100000,
              None)]
    if slab:
        cases.append(("the workload's layout on a 96x4x69 slab (4 periodic columns), extrapolation outflow, M 0.5, Re 1e4",
                      lambda: mg.wall_box(96, 4, 69, outflow=out), vis, 60000, None))
    return cases


def _load_golden(name, it):
    """The oracle's steady state of a converge case for iteration `it` ("sg" or "vc"), written by
    tests/golden/make_steady_states.py (which runs only the oracle), or None."""
    import numpy as np
    if name is None:
        return None
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_steady_states as golden
    p = golden.reference(name, it)
    return np.load(p) if os.path.exists(p) else None


def run_converge(cg, torch, slab, budget_s=1200.0):
    """Wall time (host clock around the library's own steady-solve loop) to a 1e-10 drop of the
    density residual for single-grid FP64 CGKS, the FP64 V-cycle, the mixed V-cycle and (small
    cases) the FP64 V-cycle with the LU-SGS coarse smoother (Sec. 4.3), all with the compression
    factor of Sec. 3.3 on.  Each final state is compared with the oracle's own steady state where one
    is stored, and with the other runs.  Cases are skipped once `budget_s` seconds have passed."""
    import math
    import meshgen as mg
    t_start = time.perf_counter()
    out = []
    for name, mk, phys, max_it, gold in converge_cases(slab):
        if time.perf_counter() - t_start > budget_s:
            out.append({"case": name, "skipped": "time budget of the converge section spent"})
            continue
        mesh = mk()
        row = {"case": name, "cells": len(mesh["cell_type"])}
        states = {}
        runs = [("single_grid_fp64", False, 0, 0), ("vcycle_fp64", True, 0, 0), ("vcycle_mixed", True, 1, 0)]
        if len(mesh["cell_type"]) < 20000:  # LU-SGS sweeps are one launch per colour: small cases only
            runs.append(("vcycle_fp64_lusgs", True, 0, 1))
        for key, mgrid, prec, sm in runs:
            P = cg.default_params(n_levels=3, precision=prec, coarse_smoother=sm, **phys)
            ctx = cg.upload_mesh(mesh, P)
            W, G = mg.uniform_state(ctx.nc, mach=phys["mach"])
            ctx.state_init(torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda())
            torch.cuda.synchronize()
            r = ctx.steady_solve(multigrid=mgrid, drop=1e-10, max_iters=max_it, raise_on_notconv=False)
            states[key] = ctx.state_get()[0].cpu().numpy()
            row[key] = {"iters": r["iters"], "seconds": r["seconds"], "drop": r["drop"], "converged": r["converged"]}
            ref = _load_golden(gold, "vc" if mgrid else "sg")
            if ref is not None:
                row[key]["state_err_vs_oracle"] = _state_diff(states[key], ref["W"])
                row[key]["oracle_iteration"] = ("V-cycle" if bool(ref["multigrid"]) else "single grid") + \
                    f", {int(ref['iters'])} iterations, drop {float(ref['drop']):.1e}"
            ctx.close()
        row["state_diff_mixed_vs_fp64_vcycle"] = _state_diff(states["vcycle_mixed"], states["vcycle_fp64"])
        row["state_diff_vcycle_vs_single_grid"] = _state_diff(states["vcycle_fp64"], states["single_grid_fp64"])
        sg = row["single_grid_fp64"]
        if not sg["converged"] and 0 < sg["drop"] < 1:
            # the single grid's mean rate, extended to 1e-10 (labelled as an extrapolation)
            sg["extrapolated_seconds_to_1e-10"] = sg["seconds"] * math.log(1e-10) / math.log(sg["drop"])
        out.append(row)
    return {"target_drop": 1e-10, "compression_factor": "on (Sec. 3.3)",
            "clock": "host wall time around cgks_steady_solve (checks the drop every 10 iterations)",
            "state_err_vs_oracle": "max over variables of |W - W_oracle| / max |W_oracle| (momentum components "
                                   "share one scale); W_oracle the oracle's own steady state of the same case from "
                                   "the same free stream (tests/golden), to a 1e-12 drop, by the same iteration "
                                   "where the steady state is not unique (the boundary layers)",
            "seconds": time.perf_counter() - t_start, "cases": out}


def run_scale(args):
    """Scale sweep: quadrant-layout boxes of 1.0 M, 5.0 M and 20.0 M cells (hex / prism / tet
    quadrants, no-slip wall, M 0.8, Re 1e5), single-grid FP64 steps, FP64 V-cycles and mixed
    V-cycles, Mcell-iters/s from CUDA events over `steps` iterations after `warmup`."""
    import torch
    import meshgen as mg
    import paper_2402_02075_gb300 as cg
    phys = dict(mach=0.8, reynolds=1e5, prandtl=0.72, viscous=1, n_levels=3)
    rows = []
    for n in (84, 144, 228):
        t0 = time.perf_counter()
        mesh = mg.scale_box(n)
        ctx = cg.upload_mesh(mesh, cg.default_params(**phys))
        setup = time.perf_counter() - t0
        W, G = mg.uniform_state(ctx.nc, mach=0.8)
        Wd, Gd = torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda()
        row = {"n": n, "cells": ctx.nc, "setup_s": setup}
        for key, mgrid, prec in (("single_grid_fp64", False, 0), ("vcycle_fp64", True, 0), ("vcycle_mixed", True, 1)):
            ctx.set_params(cg.default_params(precision=prec, **phys))
            ctx.state_init(Wd, Gd)
            run = ctx.vcycle if mgrid else ctx.step
            run(args.warmup, history=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(ctx.stream)
            run(args.steps, history=False)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            row[key] = {"ms_per_iter": ms, "Mcell_iters_per_s": ctx.nc / (ms * 1e-3) / 1e6}
        rows.append(row)
        ctx.close()
        del mesh, Wd, Gd
        torch.cuda.empty_cache()
    print(json.dumps({"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "data": "synthetic (seeded quadrant-layout boxes, free-stream start)", "dtype": "f64",
                      "scale": rows}))


RAMP_WORKLOAD = dict(nx=256, ny=128, nz=128, n_prism=8)


def run_ramp_throughput(cg, torch, steps, warmup):
    """The supersonic compression ramp at size: Mach 3 over 15 degrees, 256 x 128 x 128 grid with 8
    prism layers at the slip wall and hexahedra above (4,456,448 cells), inviscid, compression factor on
    (Sec. 3.3).  FP64 and mixed-precision V-cycles timed with CUDA events on the library stream after
    max(warmup, 20) V-cycles from the free stream (by then the shock stands at the corner and the
    compression factor is active there)."""
    import meshgen as mg
    t0 = time.perf_counter()
    mesh = mg.ramp_box(**RAMP_WORKLOAD)
    phys = dict(mach=3.0, n_levels=3)
    ctx = cg.upload_mesh(mesh, cg.default_params(**phys))
    setup = time.perf_counter() - t0
    W, G = mg.uniform_state(ctx.nc, mach=3.0)
    ctx.state_init(torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda())
    ctx.vcycle(max(warmup, 20), history=False)
    out = {"workload": f"Mach 3 compression ramp {RAMP_WORKLOAD['nx']}x{RAMP_WORKLOAD['ny']}x{RAMP_WORKLOAD['nz']}, "
                       f"{RAMP_WORKLOAD['n_prism']} prism layers + hexahedra, inviscid, compression factor on",
           "cells": ctx.nc, "setup_s": setup, "unit": UNIT}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for key, prec in (("vcycle_fp64", 0), ("vcycle_mixed", 1)):
        ctx.set_params(cg.default_params(precision=prec, **phys))
        ctx.vcycle(2, history=False)
        torch.cuda.synchronize()
        ev0.record(ctx.stream)
        ctx.vcycle(steps, history=False)
        ev1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        out[key] = {"ms_per_cycle": ms, "value": ctx.nc / (ms * 1e-3) / 1e6}
    a = ctx.state_get()[2]
    out["alpha_min"] = float(a.min())
    out["cells_alpha_below_0.99"] = int((a < 0.99).sum())
    ctx.close()
    return out


ADJ_WORKLOAD = dict(nx=160, ny=80, nz=80, n_prism=8)
ADJ_SMALL = dict(nx=64, ny=32, nz=8, n_prism=4)


def _steady(ctx, chunk=200, max_steps=200000):
    """Single-grid steps until the density-residual norm stops falling at round-off."""
    steps, last = 0, float("inf")
    while steps < max_steps:
        h = ctx.step(chunk)
        steps += chunk
        if h[-1] < 1e-10 and h.min() > 0.9 * last:
            break
        last = min(last, h.min())
    return steps, float(h[-1])


def run_adjoint(args):
    """The discrete adjoint (an extension of the method): (1) on the Mach-3 compression ramp at
    160 x 80 x 80 with 8 prism layers (1,126,400 cells) the time of forming the stored linearisation
    and of one transposed product (the three kernels of each adjoint iteration) with its HBM bytes;
    (2) on the same ramp at 64 x 32 x 8 the whole gradient of the wall force in the Mach number and 64
    wall modes at the steady state, with the phases timed and dJ/dMach checked against central
    differences of the converged functional."""
    import numpy as np
    import torch
    import meshgen as mg
    import paper_2402_02075_gb300 as cg
    prm = dict(mach=3.0, n_levels=1, compression_factor=0)
    out = {"metric": "adjoint: transposed-product HBM GB/s; gradient wall time", "n_gpus": 1, "dtype": "f64",
           "data": "synthetic (seeded ramp meshes, free-stream start)"}
    # (1) full size
    w = ADJ_WORKLOAD
    mesh = mg.ramp_box(w["nx"], w["ny"], w["nz"], n_prism=w["n_prism"])
    ctx = cg.upload_mesh(mesh, cg.default_params(**prm))
    nc = ctx.nc
    W, G = mg.uniform_state(nc, mach=3.0)
    ctx.state_init(torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda(), torch.ones(nc, dtype=torch.float64, device="cuda"))
    ctx.step(20, history=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.linearize()
    torch.cuda.synchronize()
    t_lin = time.perf_counter() - t0
    nf = ctx.level_info(0)[1]
    ngp = mg_gauss_points(mesh)
    rb = torch.randn(5, nc, dtype=torch.float64, device="cuda")
    gb = torch.randn(15, nc, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.residual_vjp(rb, gb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for _ in range(args.steps):
        ctx.residual_vjp(rb, gb)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # bytes of one product: the stored matrices (41 x 10 per point; per cell 20 x 51 for its own
    # slot and 6 x 200 for the neighbour slots), the point cotangents written and read, the point
    # geometry, the neighbour records written and read, the cell vectors in and out
    by = 8 * (410 * ngp + 2220 * nc + 2 * 41 * ngp + 3 * ngp + 2 * 40 * nf + 2 * 20 * nc + 3 * 20 * nc)
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    out["full"] = {"workload": f"ramp {w['nx']}x{w['ny']}x{w['nz']}, {w['n_prism']} prism layers", "cells": nc,
                   "faces": nf, "gauss_points": ngp, "linearize_s": t_lin, "vjp_ms": ms,
                   "stored_linearisation_GB": 8 * (410 * ngp + 2220 * nc) / 1e9,
                   "vjp_bytes_GB": by / 1e9, "vjp_GBps": by / (ms * 1e-3) / 1e9, "hbm_peak_GBps": peak,
                   "frac": (by / (ms * 1e-3) / 1e9) / peak if peak else None}
    # the same products with the reconstruction's part recomputed (adjoint_recompute 1): only the
    # point-flux linearisation is stored
    ctx.set_params(cg.default_params(adjoint_recompute=1, **prm))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.linearize()
    torch.cuda.synchronize()
    t_lin_r = time.perf_counter() - t0
    Wb0, Gb0 = ctx.residual_vjp(rb, gb)
    for _ in range(args.warmup):
        ctx.residual_vjp(rb, gb)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for _ in range(args.steps):
        ctx.residual_vjp(rb, gb)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms_r = e0.elapsed_time(e1) / args.steps
    out["full"]["recompute"] = {"linearize_s": t_lin_r, "vjp_ms": ms_r,
                                "stored_linearisation_GB": 8 * 410 * ngp / 1e9,
                                "what": "reconstruction's transposed product recomputed per cell in every product "
                                        "(reverse mode), the point-flux linearisation stored"}
    ctx.close()
    del mesh
    torch.cuda.empty_cache()
    # (2) whole gradient at a steady state: the 64 x 32 x 8 ramp and the full 160 x 80 x 80 ramp
    out["gradient"] = []
    for w in (ADJ_SMALL, ADJ_WORKLOAD):
        out["gradient"].append(_adjoint_gradient(cg, torch, mg, w, prm))
    print(json.dumps(out))


def _adjoint_gradient(cg, torch, mg, w, prm):
    """Steady state from the free stream by single-grid steps, then the gradient of the wall force
    in the Mach number and 64 wall modes (cgks_adjoint: linearisation, transposed pseudo-time solve,
    parameter partials), each phase timed; dJ/dMach checked against central differences of the
    converged functional."""
    mesh = mg.ramp_box(w["nx"], w["ny"], w["nz"], n_prism=w["n_prism"])
    ctx = cg.upload_mesh(mesh, cg.default_params(**prm))
    nc = ctx.nc
    W, G = mg.uniform_state(nc, mach=3.0)
    Wd, Gd, ad = torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda(), torch.ones(nc, dtype=torch.float64, device="cuda")
    ctx.state_init(Wd, Gd, ad)
    t0 = time.perf_counter()
    steps, res = _steady(ctx)
    t_primal = time.perf_counter() - t0
    modes = mg.ramp_wall_modes(mesh, 64)
    t0 = time.perf_counter()
    g = ctx.adjoint(1, modes, tol=1e-10)
    t_adj = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.adjoint(1, None, tol=1e-10)
    t_adj_mach = time.perf_counter() - t0
    Ws, Gs, _ = ctx.state_get()
    ctx.close()
    J = []
    for sgn in (1.0, -1.0):
        c = cg.upload_mesh(mesh, cg.default_params(**dict(prm, mach=3.0 + sgn * 1e-6)))
        c.state_init(Ws, Gs, ad)
        _steady(c)
        J.append(c.wall_force(1))
        c.close()
    fd = (J[0] - J[1]) / 2e-6
    return {"workload": f"ramp {w['nx']}x{w['ny']}x{w['nz']}, {w['n_prism']} prism layers", "cells": nc,
            "primal_steps": steps, "primal_final_norm": res, "primal_s": t_primal,
            "adjoint_iters": g["iters"], "adjoint_rel_res": g["rel_res"],
            "gradient_64_modes_and_mach_s": t_adj, "gradient_mach_only_s": t_adj_mach,
            "adjoint_solver": "transposed pseudo-time iteration", "dJ_dmach": g["dJ_dmach"], "dJ_dmach_fd": fd,
            "dJ_dmach_rel_err": abs(g["dJ_dmach"] - fd) / abs(fd),
            "dJ_dmodes_first4": [float(x) for x in g["dJ_dmodes"][:4]]}


def mg_gauss_points(mesh):
    """Gauss points of a mesh dict (3 per triangular face, 4 per quadrilateral, each face once): the
    cells' face slots count interior and periodic faces twice and the other boundary faces once."""
    import numpy as np
    pts = {4: 4 * 3, 5: 2 * 3 + 3 * 4, 6: 6 * 4, 7: 4 + 4 * 3}
    t = np.asarray(mesh["cell_type"])
    slots = sum(int((t == k).sum()) * v for k, v in pts.items())
    bn = np.diff(np.asarray(mesh["bface_ptr"]))
    bnd = np.asarray(mesh["bface_tag"]) < 100
    return (slots + int(np.where(bn[bnd] == 3, 3, 4).sum())) // 2


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import meshgen as mg
    import oracle
    oracle.build()
    mesh = mg.wall_box(**SAMPLE)
    M = oracle.Mesh(mesh)
    S = oracle.Solver(M, oracle.params(**PARAMS))
    W, G = mg.uniform_state(M.nc, mach=PARAMS["mach"])
    S.set_state(W, G)
    S.run(args.warmup, multigrid=True)
    t0 = time.perf_counter()
    S.run(args.steps, multigrid=True)
    dt = time.perf_counter() - t0
    value = M.nc * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", host_cores()))
    sample = (f"each step one V-cycle of the same layout and physics at {SAMPLE['nx']}x{SAMPLE['ny']}x{SAMPLE['nz']} "
              f"({M.nc:,} cells: {SAMPLE['ny']} of the workload's {WORKLOAD['ny']} periodic columns) instead of the "
              f"full {WORKLOAD['nx']}x{WORKLOAD['ny']}x{WORKLOAD['nz']} box; the metric is a per-cell rate")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": {"workload": workload_name(WORKLOAD), "params": {k: v for k, v in PARAMS.items()}},
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-converge-slab", action="store_true",
                    help="leave out the 96x4x69 slab of the workload's layout from the converge cases")
    ap.add_argument("--no-converge", action="store_true")
    ap.add_argument("--no-ramp", action="store_true", help="leave out the 4.46M-cell supersonic ramp throughput")
    ap.add_argument("--size", default="full", choices=["full", "small"],
                    help="small: the same layout at 48x32x32 (profiling captures only)")
    ap.add_argument("--adjoint", action="store_true",
                    help="adjoint measurements (stored linearisation, transposed product, gradient) instead")
    ap.add_argument("--scale", action="store_true",
                    help="scale sweep at 1.0M / 5.0M / 20.0M cells instead of the benchmark line")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        spec = json.loads(args.oracle_sample)
        print(json.dumps(oracle_sample(spec["sample"], spec["cycles"])))
        return
    global WORKLOAD
    if args.scale:
        run_scale(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    if args.size == "small":
        WORKLOAD = dict(nx=48, ny=32, nz=32, outflow=5)
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import numpy as np
    import torch
    import torch.distributed as dist

    import meshgen as mg
    import paper_2402_02075_gb300 as cg

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, world, "cuda")

    mesh = mg.wall_box(**WORKLOAD)
    P = cg.default_params(**PARAMS)
    t0 = time.perf_counter()
    ctx = cg.Context(P)
    ctx.mesh_upload(mesh)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    levels = [ctx.level_info(l) for l in range(P.n_levels)]
    nc = levels[0][0]
    # Gauss points: every cell face counted from its cells (12 per tet, 18 per prism, 24 per hex),
    # plus the non-periodic boundary faces once more, halved
    per_cell = np.array([0, 0, 0, 0, 12, 18, 24])[mesh["cell_type"]].sum()
    bnv = np.diff(mesh["bface_ptr"])[mesh["bface_tag"] < 100]
    ngp = int(per_cell + bnv.sum()) // 2
    W, G = mg.uniform_state(nc, mach=PARAMS["mach"])
    Wd, Gd = torch.from_numpy(W).cuda(), torch.from_numpy(G).cuda()
    ctx.state_init(Wd, Gd)
    ctx.vcycle(args.warmup, history=False)
    stream = ctx.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        ctx.vcycle(args.steps, history=False)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    stats = {k: ctx.kernel_stats(k) for k in ctx.KERNELS}
    ctx.profile(False)
    k_ms, k_n = stats["k_gks_points"][:2]
    ms_max = max_over_ranks(ms)
    value = job_rate(nc, args.steps, ms_max, world)
    # end to end through the public API with host buffers: per step, the state is copied in from
    # pinned host memory (cgks_state_init) and the residual norm is read back (cgks_vcycle)
    Wo, Go, ao = ctx.state_get()
    Wh, Gh, ah = Wo.cpu().pin_memory(), Go.cpu().pin_memory(), ao.cpu().pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.state_init(Wh, Gh, ah)
        ctx.vcycle(1, history=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": job_rate(nc, args.steps, e2e_s * 1e3, world), "unit": UNIT,
           "h2d_bytes_per_step": int(Wh.numel() + Gh.numel() + ah.numel()) * 8, "d2h_bytes_per_step": 8}
    # single-grid FP64 steps on the same workload: their rate, and a V-cycle's cost in steps
    ctx.state_init(Wd, Gd)
    ctx.step(args.warmup, history=False)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    ctx.step(args.steps, history=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_sg = max_over_ranks(ev0.elapsed_time(ev1))
    single_grid = {"value": job_rate(nc, args.steps, ms_sg, world), "unit": UNIT, "ms_per_step": ms_sg / args.steps,
                   "vcycle_cost_in_steps": ms_max / ms_sg,
                   "what": "explicit single-grid FP64 CGKS steps (Eq. smo with local time steps)"}
    # the mixed-precision V-cycle on the same workload: coarse levels in FP32 defect-correction form
    ctx.set_params(cg.default_params(precision=1, **PARAMS))
    ctx.state_init(Wd, Gd)
    ctx.vcycle(args.warmup, history=False)
    barrier()
    torch.cuda.synchronize()
    ctx.profile(True)
    ev0.record(stream)
    ctx.vcycle(args.steps, history=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_mixed = max_over_ranks(ev0.elapsed_time(ev1))
    stats_mixed = {k: ctx.kernel_stats(k) for k in ctx.KERNELS}
    ctx.profile(False)
    Pm = ctx.params
    mixed = {"value": job_rate(nc, args.steps, ms_mixed, world), "unit": UNIT,
             "ms_per_step": ms_mixed / args.steps,
             "gpu_launches": launches_per_vcycle({f: getattr(Pm, f) for f in (
                 "dt_mode", "pre", "post", "n_levels", "coarse_steps", "precision")}) * args.steps,
             "what": "3-level V-cycle, FP64 fine CGKS, coarse levels smoothing the correction with the "
                     "FP32 linearised KFVS operator (precision 1)"}
    peak = cg.cgks_fp64_peak()
    hbm = measured_hbm_peak()
    k_avg = k_ms / max(k_n, 1)
    roofline = {"bound": "alu", "kernel": "k_gks_points (FP64 gas-kinetic flux per Gauss point)",
                "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
                "peak_source": "measured FP64 FMA-chain rate of this GPU (cgks_fp64_peak)",
                "traffic": None, "kernel_ms": k_avg, "launches": k_n}
    if FLOP_PER_GP:
        ach = FLOP_PER_GP * ngp / (k_avg * 1e-3) / 1e12
        roofline.update(achieved=ach, frac=ach / peak, flop_per_gauss_point=FLOP_PER_GP)
    if DRAM_BYTES_PER_GP:
        roofline["traffic"] = DRAM_BYTES_PER_GP * ngp
    kernels = kernel_rooflines(stats, args.steps, peak, hbm)
    jvp = kernel_rooflines({"k_kfvs_jvp_faces": stats_mixed["k_kfvs_jvp_faces"],
                            "k_kfvs_gather": stats_mixed["k_kfvs_gather"]}, args.steps, peak, hbm)
    kernels["k_kfvs_jvp_faces"] = dict(jvp.get("k_kfvs_jvp_faces", {}), cycle="mixed")
    kernels["k_kfvs_gather (mixed: FP64 and FP32 face fluxes)"] = dict(jvp.get("k_kfvs_gather", {}), cycle="mixed")
    roofline["kernels"] = kernels
    roofline["hbm_peak_source"] = "MEASURED_PEAKS.json hbm_gbs (copy bandwidth of this GPU pool)"
    launches = launches_per_vcycle({f: getattr(P, f) for f in ("dt_mode", "pre", "post", "n_levels", "coarse_steps",
                                                               "precision")})
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded mesh, free-stream start)",
           "config": {"workload": workload_name(WORKLOAD), "cells_per_level": [l[0] for l in levels],
                      "faces_per_level": [l[1] for l in levels], "gauss_points": ngp,
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "working set (about 7 GB) far above L2 (129 MB); no flush needed",
                      "setup_s": setup_s, "params": {k: v for k, v in PARAMS.items()}},
           "e2e": e2e, "gpu_launches": launches * args.steps, "roofline": roofline, "clocks": clk.summary(),
           "mixed": mixed, "single_grid": single_grid}
    ctx.close()
    if rank == 0 and world == 1 and not args.no_ramp:
        out["ramp"] = run_ramp_throughput(cg, torch, args.steps, args.warmup)
    if rank == 0 and world == 1 and not args.no_converge:
        out["converge"] = run_converge(cg, torch, not args.no_converge_slab)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
