#!/usr/bin/env python
"""Throughput of the cRKDG hot path on one GB300 (or one mesh split over N GPUs).

Metric: cell-DOF updates per second per RK stage = cells * m(k+1)^d * s / time,
counting every accepted time step (s stages + limiters + the final stage + the
dt control).  One bench step = one cRKDG time step of the workload.

Default workload (N=1): the largest single-GPU configuration, the 2D Euler
(gamma 1.4) Sedov-type blast on [0,1.1]^2, 2048 x 2048 cells, Q^3, four-stage
fourth-order cRKDG (CFL 0.103), split precision: FP64 cell averages, limiter
decisions, conservation sums and time step; FP32-level operators, the inner stages'
maps as three-product TF32 tensor-core GEMMs.  Other configurations: --workload
(e.g. sedov_shell_2048_q3_mixed times the same configuration on a developed blast).

Arms:
  --impl gb300      (default) the CUDA library through its C ABI.
  --impl reference  the CPU oracle on the host cores (rank 0 only).
Under torchrun (N > 1) the workload's one mesh is split into N blocks, one per
rank (strong scaling): one halo exchange per step plus the global trial step
and restart decision (paper_2412_16002_gb300.decomp); the ensemble and the
indicator workloads run N independent replicas instead (weak scaling).  The
reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 peak of the GB300 derived from the unit count and clock: 152 SMs x 4 FP64
# flop per clock (two DFMA per clock per SM, the 1.25 TFLOP/s class rate) x 2070 MHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# FP32 (non-tensor) peak from the same unit count: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12

WORKLOADS = {
    "euler1d_blast_tube_4096_p2": dict(kind="euler1d", nx=4096, k=2),
    "burgers_sine_200_p2": dict(kind="burgers", nx=200, k=2),
    "sedov_2048_q3_mixed": dict(kind="sedov", nx=2048, k=3, precision="mixed"),
    "sedov_2048_q3_fp64": dict(kind="sedov", nx=2048, k=3),
    "sedov_512_q3": dict(kind="sedov", nx=512, k=3),
    "sedov_512_q3_mixed": dict(kind="sedov", nx=512, k=3, precision="mixed"),
    "riemann_1024_q2": dict(kind="riemann", nx=1024, k=2),
    "riemann_1024_q2_mixed": dict(kind="riemann", nx=1024, k=2, precision="mixed"),
    "riemann_1024_q2_tvb": dict(kind="riemann", nx=1024, k=2, indicator="tvb"),
    "riemann_1024_q2_mlp": dict(kind="riemann", nx=1024, k=2, indicator="mlp"),
    "riemann_1024_q2_mixed_tvb": dict(kind="riemann", nx=1024, k=2, precision="mixed", indicator="tvb"),
    "riemann_1024_q2_mixed_mlp": dict(kind="riemann", nx=1024, k=2, precision="mixed", indicator="mlp"),
    "ensemble_64_riemann_mlp": dict(kind="ensemble", count=64, indicator="mlp"),
    # the standard RKDG (F in every stage), for comparison with the compact scheme
    "sedov_2048_q3_standard": dict(kind="sedov", nx=2048, k=3, scheme="standard"),
    # the same configuration timed on a developed blast (dense shell of radius 0.3 around the
    # corner, hot low-density interior, flowing radially) instead of the initial data
    "sedov_shell_2048_q3_mixed": dict(kind="sedov_shell", nx=2048, k=3, precision="mixed"),
    "sedov_shell_2048_q3_fp64": dict(kind="sedov_shell", nx=2048, k=3),
    "riemann_1024_q2_standard": dict(kind="riemann", nx=1024, k=2, scheme="standard"),
    # the non-rectangular benchmarks at the paper's resolutions: the double Mach reflection
    # (Example 4.9, Q^3, cells of side 1/360) and the shock diffraction (Example 4.8, Q^2, 1/64)
    "double_mach_360_q3": dict(kind="double_mach", per_unit=360, k=3),
    "shock_diffraction_64_q2": dict(kind="shock_diffraction", per_unit=64, k=2),
}
DEFAULT = "sedov_2048_q3_mixed"
# timed steps when --steps is not given
DEFAULT_STEPS = {"euler1d": 2000, "burgers": 2000, "sedov": 50, "sedov_shell": 50, "riemann": 100, "ensemble": 5,
                 "double_mach": 50, "shock_diffraction": 50}


def launches_per_attempt(precision, indicator):
    """Kernels one step attempt launches: the inner and final stages; the indicator: the
    troubled-cell pass, after (learned) the feature kernel and the network's forward pass, on
    the split path also the merge to FP64 nodal values the feature kernel reads; then the
    component totals of the new state for the step's conservation drift (two reduction
    kernels, after the FP64 path's cell-average kernel)."""
    n = 2 + (2 if precision == "mixed" else 3)
    if indicator == "tvb":
        n += 1
    elif indicator == "mlp":
        n += 3 + (1 if precision == "mixed" else 0)
    return n


def make_workload(name, seed=0, nx=None):
    from paper_2412_16002_gb300 import inputs

    w = dict(WORKLOADS[name])
    if w["kind"] == "ensemble":  # sampled as one of its problems (Q^2 Riemann)
        w = dict(kind="riemann", nx=nx or 256, k=2)
    if nx is not None:
        w["nx"] = nx
    if w["kind"] == "euler1d":
        return inputs.euler_blast_tube(w["nx"], w["k"])
    if w["kind"] == "burgers":
        return inputs.burgers_sine(w["nx"], w["k"])
    if w["kind"] == "sedov":
        return inputs.sedov(w["nx"], w["k"])
    if w["kind"] == "sedov_shell":
        return inputs.sedov_shell(w["nx"], w["k"])
    if w["kind"] in ("double_mach", "shock_diffraction"):
        # a sample of width nx holds about nx^2 cells: the bounding rectangle's area (4 x 2 or
        # 13 x 12) in cells of side 1 / per_unit
        area = 8.0 if w["kind"] == "double_mach" else 156.0
        per_unit = max(2, int(round(nx / math.sqrt(area)))) if nx is not None else w["per_unit"]
        make = inputs.double_mach if w["kind"] == "double_mach" else inputs.shock_diffraction
        return make(cells_per_unit=per_unit, k=w["k"])
    return inputs.riemann_quadrants(seed, w["nx"], w["k"])


def active_cells(wl):
    """Cells of the domain: every cell of a rectangular mesh, the fluid cells of a
    non-rectangular one (the solid cells carry no unknowns of the problem)."""
    if getattr(wl, "geo", None) is None:
        return wl.cells
    from paper_2412_16002_gb300.inputs import GEO_SOLID

    return int(((wl.geo & GEO_SOLID) == 0).sum())


INITIAL_STATE = {"sedov_shell": "a developed Sedov-type blast: dense shell of radius 0.3 around the corner, "
                                "hot low-density interior, radial flow, cold ambient state (p = 1e-13) outside"}

TAB_S = {"midpoint2": 2, "heun3": 3, "rk4": 4}
TAB_NSLOT = {"midpoint2": 1, "heun3": 2, "rk4": 4}
TAB_NA = {"midpoint2": 1, "heun3": 2, "rk4": 3}  # nonzero a_ij


def flux_flops(flux, dim):
    """FP64 operations of one flux evaluation f(u).e_dir (divisions and roots count 1)."""
    if flux == "euler":
        return 10 if dim == 1 else 14
    return 1 if flux == "advection" else 2


def algorithmic_flops(wl):
    """FP64 flops per cell per time step of the method as written (Scheme 1L), split into
    the inner-stage kernel and the final-stage kernel.  Counts: flux at every node and
    trace point; volume term 2n per node per component per direction; trace interpolation
    2n per trace point per component; lift 5 per node per component per direction; stage
    combination 2 per node per component per nonzero a_ij; limiter: average 2 per node per
    component, S_K interpolation 2n per point per component, rho*e 6 per point and 10 per
    theta; the spectral radius (10) of every trace point of a stage with b_i != 0 (computed
    with the trace flux that G needs anyway); LF flux per face point per such stage: 8 per
    component (the two trace fluxes and radii are those of G's traces); u* accumulation 2
    per node per component per nonzero b_i; a0 10 per S_K point."""
    d, n, m = wl.dim, wl.k + 1, wl.m
    nn = n ** d
    ntr = 2 * d * (n if d == 2 else 1)
    L = (n + 3) // 2
    nsk = 2 * n * L if d == 2 else L
    s, nslot, na = TAB_S[wl.tableau], TAB_NSLOT[wl.tableau], TAB_NA[wl.tableau]
    ff = flux_flops(wl.flux, d)
    g = nn * (ff * (2 if d == 2 else 1) * (1 if d == 2 else 1) + 2 * n * m * d + 5 * m * d) + ntr * (2 * n * m + ff)
    lim = 2 * nn * m + nsk * (2 * n * m) + (nsk * 6 + 20 if wl.flux == "euler" else 10)
    inner = s * g + na * 2 * nn * m + (s - 1) * lim + nslot * 2 * nn * m + nslot * ntr * 10
    lf = ntr * nslot * 8 * m
    final = lf + nn * m * 5 * d + lim + nsk * 10
    return inner, final


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_rate(local_ms, units_per_rank, world, device=None):
    """Whole-job throughput of N independent replicas: every rank advanced units_per_rank
    units in local_ms; the job's time is the maximum over ranks (all_reduce MAX when
    world > 1).  Returns (units/s of the whole job, the maximum ms)."""
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return units_per_rank * world / (ms / 1e3), ms


def read_traffic(kernel, workload):
    """DRAM bytes per launch recorded by the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("dram_bytes_per_launch:"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample(name, nx=None):
    """The workload the oracle steps: the full mesh when it has at most 16384 cells, else
    the same workload on an nx-cell-wide mesh (64 by default; a bounded sample)."""
    wl = make_workload(name)
    if wl.cells > 16384:
        wl = make_workload(name, nx=nx or 64)
    return wl


def reference_sample_width(name, total_steps, budget_s=150.0):
    """Width of the reference arm's sample mesh, chosen so that total_steps oracle steps take
    about budget_s: one calibration step on a 16-wide mesh, then the cost scaled by the cell
    count (64 at most, 4 at least).  None for workloads small enough to run in full."""
    if make_workload(name).cells <= 16384:
        return None
    n, el, _ = _oracle_worker(name, 1, 1, 0.0, 16)
    per_cell = el / max(n, 1) / (16 * 16)
    cells = budget_s / max(total_steps, 1) / max(per_cell, 1e-12)
    return int(max(4, min(64, cells ** 0.5)))


def _oracle_worker(name, warmup, steps, budget_s, nx=None):
    """One host process: the oracle (plain C, one thread) steps the sample of `name`; returns
    (accepted timed steps, seconds, units per step).  With steps None it runs until budget_s."""
    sys.path.insert(0, ROOT)
    from oracle import HEUN3, MIDPOINT2, RK4, Oracle

    tabs = {"midpoint2": MIDPOINT2, "heun3": HEUN3, "rk4": RK4}
    wl = oracle_sample(name, nx)
    o = Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, velocity=wl.velocity,
               bounds=wl.bounds, eps=wl.eps, bc=wl.bc, bc_state=wl.bc_state,
               scheme=WORKLOADS[name].get("scheme", "compact"))
    if getattr(wl, "geo", None) is not None:
        o.set_geometry(wl.geo, wl.geo_states[0], wl.geo_states[1], *wl.shock)
    o.set_state(wl.state)
    t = 0.0
    for _ in range(warmup):
        rc, info = o.step(o.max_dt(wl.cfl), tabs[wl.tableau], t)
        t += info["dt_taken"]
    n = 0
    t0 = time.perf_counter()
    while (n < steps) if steps is not None else (time.perf_counter() - t0 < budget_s):
        rc, info = o.step(o.max_dt(wl.cfl), tabs[wl.tableau], t)
        if rc != 0:
            break
        t += info["dt_taken"]
        n += 1
    el = time.perf_counter() - t0
    return n, el, active_cells(wl) * wl.dofs_per_cell * TAB_S[wl.tableau]


def oracle_throughput(name, procs, warmup=0, steps=None, budget_s=10.0, nx=None):
    """Oracle throughput on `procs` host cores: procs independent processes (spawned, so no
    CUDA state is inherited) each step their own copy of the sample; the job's time is the
    slowest process's.  Returns (cell-DOF-stage/s, steps per process, seconds)."""
    if procs == 1:
        n, el, u = _oracle_worker(name, warmup, steps, budget_s, nx)
        return n * u / el, n, el
    import multiprocessing as mp

    from oracle.oracle import build_oracle

    build_oracle()  # once, before the workers load it
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.starmap(_oracle_worker, [(name, warmup, steps, budget_s, nx)] * procs)
    el = max(r[1] for r in res)
    units = sum(r[0] * r[2] for r in res)
    return units / el, min(r[0] for r in res), el


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline_record(name, budget_s):
    """The oracle timed on one host core and on every host core (independent processes)."""
    swl = oracle_sample(name)
    mesh = f"{swl.nx}x{swl.ny}" if swl.dim == 2 else f"{swl.nx}"
    cores = host_cores()
    v1, n1, el1 = oracle_throughput(name, 1, budget_s=budget_s)
    vp, np_, elp = oracle_throughput(name, cores, budget_s=budget_s) if cores > 1 else (v1, n1, el1)
    return {"value": vp, "unit": "cell-DOF-stage/s", "cores": cores, "kind": "oracle",
            "single_core_value": v1, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"{name} on a {mesh}-cell mesh from its initial state: {n1} steps on one core "
                      f"({el1:.1f} s); then {cores} independent oracle processes, one per core, "
                      f"at least {np_} steps each ({elp:.1f} s)"}


def workload_config(name, wl, world):
    """The config dict both arms print for a workload."""
    return {"workload": name, "precision": WORKLOADS[name].get("precision", "fp64"),
            "scheme": WORKLOADS[name].get("scheme", "compact"),
            "indicator": WORKLOADS[name].get("indicator", "off"), "cells": active_cells(wl), "k": wl.k, "m": wl.m,
            "dofs_per_cell": wl.dofs_per_cell, "tableau": wl.tableau, "stages": TAB_S[wl.tableau],
            "cfl": wl.cfl, "initial_state": INITIAL_STATE.get(WORKLOADS[name]["kind"], "the workload's initial data at t = 0"),
            "l2": "GPU arm: L2 flushed (256 MB write) between timed steps" if wl.dim == 2 else
                  "GPU arm: state L2-resident by design in the device-resident loop; L2 flushed before the timed launch",
            "parallelism": f"replicas{world}"}


def run_reference(args, wl, name):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    cores = host_cores()
    nx = reference_sample_width(name, args.steps + args.warmup)
    swl = oracle_sample(name, nx)
    v, n, el = oracle_throughput(name, cores, warmup=args.warmup, steps=args.steps, nx=nx)
    mesh = f"{swl.nx}x{swl.ny}" if swl.dim == 2 else f"{swl.nx}"
    line = {
        "impl": "reference", "metric": "cell-DOF updates/s per RK stage", "value": v,
        "unit": "cell-DOF-stage/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(name, wl, world),
        "cpu_baseline": {"value": v, "unit": "cell-DOF-stage/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                         "sample": f"{cores} independent oracle processes, one per host core, each "
                                   f"{args.steps} time steps of {name} on a {mesh} mesh (full mesh "
                                   f"{wl.nx}x{wl.ny}) after {args.warmup} warm-up steps"},
        "e2e": {"value": v, "unit": "cell-DOF-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def proc_grid(world, dim):
    """px x py blocks for `world` ranks: 1D a row; 2D the most square factorisation, the longer
    side along x."""
    if dim == 1:
        return world, 1
    py = int(world ** 0.5)
    while world % py:
        py -= 1
    return world // py, py


def run_decomposed(args, wl, name):
    """N > 1: the workload's one mesh split into N blocks, one per GPU (strong scaling): each
    step one halo exchange of u^n's boundary layer (NCCL with device buffers, or gloo with
    host-staged buffers), the global trial step (all-reduce MIN) and the global restart
    decision (all-reduce of the flags).  Time: CUDA events on each rank's stream around the
    K steps (host-side collectives included), maximum over ranks."""
    import torch
    import torch.distributed as dist

    from paper_2412_16002_gb300.decomp import DomainSolver, Layout, TorchTransport

    world, rank, local = dist_setup()
    torch.cuda.set_device(local % torch.cuda.device_count())  # ranks share a GPU only on a smaller box
    dist.init_process_group(args.dist_backend)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        from paper_2412_16002_gb300 import build

        build()
    dist.barrier()
    from paper_2412_16002_gb300.solver import Solver

    precision = WORKLOADS[name].get("precision", "fp64")
    if WORKLOADS[name].get("indicator", "off") != "off":
        raise SystemExit("the troubled-cell indicators are not available on subdomains")
    px, py = proc_grid(world, wl.dim)
    lay = Layout(wl.dim, wl.nx, wl.ny, px, py, rank, (wl.bc[0] == "periodic", wl.bc[2] == "periodic"))
    ldom, lbc = lay.local_mesh(wl.domain, wl.bc)
    stream = torch.cuda.current_stream()
    g = Solver(wl.dim, lay.nxl, lay.nyl, wl.k, ldom, wl.flux, gamma=wl.gamma, velocity=wl.velocity,
               bounds=wl.bounds, eps=wl.eps, bc=lbc, bc_state=wl.bc_state, stream=stream, precision=precision)
    nccl = args.dist_backend == "nccl"
    tr = TorchTransport(device=dev if nccl else None)
    ds = DomainSolver(lay, g, tr, wl.domain, device_buffers=nccl, device=dev)
    local_state = ds.local_block(wl.state)
    g.set_state(torch.from_numpy(local_state).to(dev))
    for _ in range(args.warmup):
        ds.step(ds.max_dt(wl.cfl), wl.tableau)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    g.set_profiling(True)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    restarts = 0
    ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = ds.step(ds.max_dt(wl.cfl), wl.tableau)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        restarts += info["restarts"]
    dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    kt, kn = g.kernel_times()
    g.set_profiling(False)
    units = active_cells(wl) * wl.dofs_per_cell * TAB_S[wl.tableau] * args.steps
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = units / (ms_max / 1e3)

    # end to end: each rank's local block host -> device, the steps, its state device -> host
    host_in = torch.from_numpy(local_state.reshape(-1).copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    import ctypes as C

    e2e_steps = max(3, min(args.steps, 10))
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g._chk(g.lib.crkdg_set_state(g.h, C.c_void_p(host_in.data_ptr()), host_in.numel(), 0))
        ds.step(ds.max_dt(wl.cfl), wl.tableau)
        g._chk(g.lib.crkdg_get_state(g.h, C.c_void_p(host_out.data_ptr()), host_out.numel(), 0))
    torch.cuda.synchronize()
    t = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = active_cells(wl) * wl.dofs_per_cell * TAB_S[wl.tableau] * e2e_steps / float(t.item())
    nbytes = host_in.numel() * 8 * world  # every rank's local block (owned cells and halo ring)
    if rank == 0:
        inner_f, final_f = algorithmic_flops(wl)
        avg_inner = kt["inner"] / max(kn["inner"], 1)
        avg_final = kt["final"] / max(kn["final"], 1)
        sfx = "_x" if precision == "mixed" else ""
        isfx = "_tc" if (precision == "mixed" and wl.dim == 2 and wl.k == 3 and wl.flux == "euler") else sfx
        dom_k, avg_ms, fl = ("k_inner" + isfx, avg_inner, inner_f) if avg_inner >= avg_final else \
            ("k_final" + sfx, avg_final, final_f)
        achieved = fl * lay.nxl * lay.nyl / (avg_ms / 1e3) / 1e12
        peak = FP32_PEAK_TFLOPS if precision == "mixed" else FP64_PEAK_TFLOPS
        cfg = workload_config(name, wl, world)
        cfg["parallelism"] = f"domain{px}x{py}"
        line = {
            "metric": "cell-DOF updates/s per RK stage", "value": value, "unit": "cell-DOF-stage/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f32+f64", "data": "synthetic", "config": cfg,
            "run": {"backend": args.dist_backend, "halo_bytes_per_rank_step": ds.halo_bytes,
                    "restarts_in_timed_steps": restarts, "rank0_local_cells": lay.nxl * lay.nyl},
            "roofline": {"bound": "alu", "kernel": dom_k, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "note": "rank 0's dominant kernel over its local cells (owned block and halo ring)"},
            "e2e": {"value": e2e_value, "unit": "cell-DOF-stage/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": int(kn["inner"]) * launches_per_attempt(precision, "off") * world,
            "clocks": clocks,
        }
        print(json.dumps(line))
    g.close()
    dist.destroy_process_group()


def run_gb300(args, wl, name):
    import torch

    world, rank, local = dist_setup()
    if world > 1 and WORKLOADS[name]["kind"] != "ensemble" and WORKLOADS[name].get("indicator", "off") == "off":
        return run_decomposed(args, wl, name)
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        from paper_2412_16002_gb300 import build

        build()
    if world > 1:
        dist.barrier()
    from paper_2412_16002_gb300.solver import Solver

    stream = torch.cuda.current_stream()
    precision = WORKLOADS[name].get("precision", "fp64")
    indicator = WORKLOADS[name].get("indicator", "off")
    train = None
    if indicator == "mlp":
        theta, train = trained_indicator()
    g = Solver.from_workload(wl, stream=stream, precision=precision, indicator=indicator,
                             scheme=WORKLOADS[name].get("scheme", "compact"))
    if indicator == "mlp":
        g.set_mlp(theta)
    u0 = torch.from_numpy(wl.state).to(dev)
    g.set_state(u0)
    t = 0.0
    if wl.dim == 1:
        t, _, _ = g.advance(args.warmup, wl.cfl, 1e30, wl.tableau, t)
    else:
        for _ in range(args.warmup):
            info = g.step(g.max_dt(wl.cfl), wl.tableau)
            t += info["dt_taken"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    g.set_profiling(True)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    restarts = 0
    if wl.dim == 1:
        # device-resident step loop: the K timed steps are one persistent launch; the
        # whole state stays L2-resident by design, L2 is flushed before the launch
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t, done, restarts = g.advance(args.steps, wl.cfl, 1e30, wl.tableau, t)
        e1.record(stream)
        torch.cuda.synchronize()
        assert done == args.steps, (done, args.steps)
        ms = e0.elapsed_time(e1)
        l2_note = "state L2-resident by design in the device-resident loop; L2 flushed (256 MB write) before the timed launch"
    else:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            info = g.step(g.max_dt(wl.cfl), wl.tableau)
            ev[i][1].record(stream)
            restarts += info["restarts"]
            t += info["dt_taken"]
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        l2_note = "flushed between timed steps (256 MB write)"
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    kt, kn = g.kernel_times()
    g.set_profiling(False)
    value, ms_max = job_rate(ms, active_cells(wl) * wl.dofs_per_cell * TAB_S[wl.tableau] * args.steps, world, dev)

    # end to end through the C ABI with host buffers: H2D of the state, one step, D2H
    host_in = torch.from_numpy(g.get_state().reshape(-1).copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    import ctypes as C

    lib, h = g.lib, g.h
    nbytes = host_in.numel() * 8
    e2e_steps = max(3, args.steps if wl.dim == 1 else min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g._chk(lib.crkdg_set_state(h, C.c_void_p(host_in.data_ptr()), host_in.numel(), 0))
        g.step(g.max_dt(wl.cfl), wl.tableau)
        g._chk(lib.crkdg_get_state(h, C.c_void_p(host_out.data_ptr()), host_out.numel(), 0))
        host_in, host_out = host_out, host_in  # the result is the next step's input
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = job_rate(1e3 * e2e_s, active_cells(wl) * wl.dofs_per_cell * TAB_S[wl.tableau] * e2e_steps, world, dev)

    if rank == 0:
        inner_f, final_f = algorithmic_flops(wl)
        avg_inner = kt["inner"] / max(kn["inner"], 1)
        avg_final = kt["final"] / max(kn["final"], 1)
        sfx = "_x" if precision == "mixed" else ""
        # the split path's 2D Euler Q^3 inner stages run on the tensor cores (k_inner_tc)
        isfx = "_tc" if (precision == "mixed" and wl.dim == 2 and wl.k == 3 and wl.flux == "euler") else sfx
        if kn["run"] > 0:
            avg_run = kt["run"] / kn["run"]
            dom, avg_ms, fl = "k_run1d", avg_run, (inner_f + final_f) * args.steps
        elif avg_inner >= avg_final or indicator != "off":
            # with an indicator the final window also holds the indicator's kernels; the
            # inner window is one kernel
            dom, avg_ms, fl = "k_inner" + isfx, avg_inner, inner_f
        else:
            dom, avg_ms, fl = "k_final" + sfx, avg_final, final_f
        achieved = fl * active_cells(wl) / (avg_ms / 1e3) / 1e12
        # the split path runs its operators in FP32: its roofline is the FP32 peak
        peak = FP32_PEAK_TFLOPS if precision == "mixed" else FP64_PEAK_TFLOPS
        peak_src = ("FP32 derived from unit count and clock (152 SMs x 128 lanes x 2 x 2070 MHz)" if precision == "mixed"
                    else "FP64 derived from unit count and clock (152 SMs x 4 flop/clk x 2070 MHz)")
        line = {
            "metric": "cell-DOF updates/s per RK stage",
            "value": value,
            "unit": "cell-DOF-stage/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": workload_config(name, wl, world),
            "run": {"training": train, "restarts_in_timed_steps": restarts, "t_after": t, "l2": l2_note},
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": read_traffic(dom, name),
                         "peak_source": peak_src,
                         "avg_launch_ms": {"k_inner": avg_inner, "k_final": avg_final,
                                           "k_run1d": kt["run"] / max(kn["run"], 1)},
                         "flops_per_cell": {"k_inner": inner_f, "k_final": final_f}},
            "e2e": {"value": e2e_value, "unit": "cell-DOF-stage/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": int(kn["run"]) if kn["run"] else int(kn["inner"]) * launches_per_attempt(precision, indicator),
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_record(name, args.cpu_seconds)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def trained_indicator(seeds=range(1000, 1004), n=256, steps=800, every=200, epochs=8):
    """The learned indicator's network, trained on the GPU by the library's kernels on about
    1e6 cells labelled by the plain indicator in one ensemble run of seeded 256^2 Q^2 Riemann
    problems (4 snapshots per problem at t ~ 0.05, 0.1, 0.15, 0.2).  Returns (params, summary)."""
    from paper_2412_16002_gb300 import indicator as ind

    t0 = time.perf_counter()
    X, Y = ind.harvest_ensemble(list(seeds), n=n, k=2, steps=steps, every=every)
    theta, hist = ind.train(X, Y, epochs=epochs)
    conf = ind.confusion(theta, X, Y)
    summary = {"cells": int(Y.numel()), "troubled_fraction": float(Y.mean().item()), "epochs": epochs,
               "loss": hist[-1], "train_agreement": conf["accuracy"], "undecided": conf["undecided"],
               "seconds": time.perf_counter() - t0}
    del X, Y
    return theta, summary


def run_ensemble(args, name):
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        from paper_2412_16002_gb300 import build

        build()
    if world > 1:
        dist.barrier()
    from paper_2412_16002_gb300 import inputs
    from paper_2412_16002_gb300.ensemble import Ensemble, riemann_ensemble_specs, riemann_problem

    spec = WORKLOADS[name]
    specs = riemann_ensemble_specs(spec["count"], seed=0)
    theta, train = trained_indicator()
    probs = [riemann_problem(s, n, k) for s, n, k in specs]
    for p in probs:
        p["t_end"] = 1e30
    ens = Ensemble(probs, indicator=spec["indicator"])
    ens.set_mlp(theta)
    for i, (s, n, k) in enumerate(specs):
        x = inputs.riemann_quadrants_device(s, n, k, device=dev)
        ens.set_state(i, x)
        del x
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tiles = ens.autotune(reps=1)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        ens.step()
    cells = sum(n * n for _, n, _ in specs)
    units_step = sum(n * n * 4 * (k + 1) ** 2 * (4 if k == 3 else 3) for _, n, k in specs)
    flops_step = 0
    for _, n, k in specs:
        wl = inputs.Workload("x", 2, 1, 1, k, (0, 1, 0, 1), "euler", ("outflow",) * 4, None,
                             tableau="rk4" if k == 3 else "heun3")
        fi, ff = algorithmic_flops(wl)
        flops_step += (fi + ff) * n * n
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ens.set_profiling(True)
    for _ in range(args.steps):
        ens.step()
    ms, nst = ens.times()
    ens.set_profiling(False)
    clocks = sampler.stop() if sampler else None
    value, ms_max = job_rate(ms, units_step * args.steps, world, dev)
    troubled = sum(ens.info(i)["troubled"] for i in range(len(specs)))
    restarts = sum(ens.info(i)["restarts"] for i in range(len(specs)))

    # end to end through the C ABI with host buffers: every problem's state host -> device,
    # K steps, every state device -> host (pinned host memory)
    hosts = [torch.empty(ens.state_size(i), dtype=torch.float64).pin_memory() for i in range(len(specs))]
    for i in range(len(specs)):
        ens.get_state(i, hosts[i].numpy())
    nbytes = sum(h.numel() * 8 for h in hosts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(len(specs)):
        ens.set_state(i, hosts[i].numpy())
    for _ in range(args.steps):
        ens.step()
    for i in range(len(specs)):
        ens.get_state(i, hosts[i].numpy())
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = job_rate(1e3 * e2e_s, units_step * args.steps, world, dev)
    del hosts
    if rank == 0:
        achieved = flops_step * args.steps / (ms_max / 1e3) / 1e12
        line = {
            "metric": "cell-DOF updates/s per RK stage",
            "value": value,
            "unit": "cell-DOF-stage/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": name, "problems": len(specs), "cells": cells,
                       "dofs": sum(n * n * 4 * (k + 1) ** 2 for _, n, k in specs),
                       "q3_problems": sum(k == 3 for _, _, k in specs), "sizes": "256^2..1536^2 (seeded)",
                       "indicator": spec["indicator"], "tiles": tiles, "autotune_s": tune_s,
                       "training": train, "troubled_cells_last_step": troubled,
                       "restarts_total": restarts, "graph_steps_timed": nst,
                       "l2": "inputs larger than L2 (state 26 GB)", "parallelism": f"replicas{world}"},
            "roofline": {"bound": "alu", "kernel": "k_ens (ensemble step graph)", "achieved": achieved,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": None,
                         "peak_source": "FP64 derived from unit count and clock (152 SMs x 4 flop/clk x 2070 MHz)",
                         "note": "FP64 flops of the method per step (the network's FP32 work not counted)"},
            "e2e": {"value": e2e_value, "unit": "cell-DOF-stage/s", "h2d_bytes_per_step": nbytes // args.steps,
                    "d2h_bytes_per_step": nbytes // args.steps},
            "gpu_launches": int(nst) * 14,
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_record(name, args.cpu_seconds)
            line["cpu_baseline"]["sample"] += " (one Q^2 Riemann problem of the ensemble, no indicator)"
        print(json.dumps(line))
    ens.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="N > 1: halo exchange over NCCL (device buffers) or gloo (host-staged)")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    if args.steps is None:
        args.steps = DEFAULT_STEPS[WORKLOADS[args.workload]["kind"]]
    wl = make_workload(args.workload)
    if args.impl == "reference":
        run_reference(args, wl, args.workload)
    elif WORKLOADS[args.workload]["kind"] == "ensemble":
        run_ensemble(args, args.workload)
    else:
        run_gb300(args, wl, args.workload)


if __name__ == "__main__":
    main()
