#!/usr/bin/env python
"""Benchmark of the SSLBM hot path on GB300 (one JSON line on stdout).

Workload: the 8192 x 8192 no-flux multi-seed SEIRD grid (64 Gaussian infected seeds,
d^S = d^E = d^R = 0.05, d^I = 0.01, beta = 0.5, sigma = 0.2, gamma = 0.1, mu = 0.01), FP32
fields.  One benchmark step = 100 SSLBM lattice steps (temporal-blocked launches) followed
by the FP64 diagnostics reduction (total population, peak infected); with the default
103 steps the run covers the workload's 10,000 lattice steps.  The 1.34 GB state is far
larger than the 129 MB L2, so no flush is needed between steps.

value: GLUPS (billion lattice-cell updates per second) over all ranks, device-timed
with CUDA events on the solver's stream.  e2e: the same metric through the public API
with pinned host buffers (initial state in, final state out) inside the timed region.
roofline: the blocked SSLBM kernel's algorithmic bytes per launch (40 B per cell: read
and write five FP32 planes) over its event-timed average launch duration, against the
measured HBM copy bandwidth.  cpu_baseline: the FP64 CPU oracle on the host cores, on a
bounded sample of the same grid.  Multi-GPU runs are independent replicas (weak scaling).

--impl reference times the FP64 CPU oracle (the reference arm of this method) on the
same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SSLBM GLUPS & % HBM roofline; ensemble scenario-steps/s vs FP64 at fixed L2 err"
UNIT = "GLUPS"
NX = NY = 8192
LATTICE_STEPS_PER_STEP = 100
BYTES_PER_CELL_FP32 = 40  # read + write of five FP32 planes per launch
BYTES_PER_CELL_FP64 = 80
FP64_FLOPS_PER_CELL = 46  # the SSLBM update per cell-step: four laplacians, sources, update
BGK_BYTES_PER_CELL_FP32 = 168  # 20 populations + D, read and write
FD4_PLANES_PER_CELL = 85  # RK4 stage kernels: 15 + 25 + 25 + 20 plane reads and writes per step


PIPE_SOURCES = ("paper_2603_19789_gb300/csrc/sslbm_pipe.cuh", "paper_2603_19789_gb300/csrc/sslbm_internal.cuh",
                "paper_2603_19789_gb300/csrc/sslbm_kernels.cu", "paper_2603_19789_gb300/csrc/pipe_launch.cuh")


def captured_traffic(depth: int, cells: int):
    """DRAM bytes per launch of the fused kernel at this depth, from the ncu capture summarised
    in profiles/ (bytes per cell x cells), or None when no capture matches the current sources."""
    import glob
    import hashlib
    import re
    h = hashlib.sha256()
    for p in PIPE_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
    pat = re.compile(r"^TRAFFIC kernel=pipe_kernel K=(\d+) bytes_per_cell_per_launch=([0-9.]+) sources=(\w+)")
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as fh:
            for line in fh:
                m = pat.match(line.strip())
                if m and int(m.group(1)) == depth and m.group(3) == digest:
                    return float(m.group(2)) * cells
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if n_gpus > 1 and world != n_gpus:
        raise SystemExit(f"--gpus {n_gpus} must be launched with torchrun (WORLD_SIZE={world})")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    from paper_2603_19789_gb300.decomp import max_over_ranks as _max
    return _max(x, world, device="cuda")


def cpu_oracle_glups(state64, wl, budget_s: float = 12.0, rows: int | None = None):
    """GLUPS of the FP64 oracle on a band of the grid (rows x 8192, no-flux band edges)."""
    import oracle
    tau = [oracle.tau_from_d(v) for v in wl["d"][:4]]
    band = np.ascontiguousarray(state64[:, : (rows or state64.shape[1]), :])
    scratch = np.empty_like(band)
    t0 = time.perf_counter()
    oracle.sslbm_run_inplace(band, scratch, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], 1)
    one = time.perf_counter() - t0
    steps = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.sslbm_run_inplace(band, scratch, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], steps)
    el = time.perf_counter() - t0
    cells = band.shape[1] * band.shape[2]
    return cells * steps / el / 1e9, steps, band.shape, el


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2603_19789_gb300 import inputs
    oracle.build()
    wl = inputs.roofline_workload(NX, NY)
    tau = [oracle.tau_from_d(v) for v in wl["d"][:4]]
    rows = 1024
    band = np.ascontiguousarray(wl["state"][:, :rows, :])
    scratch = np.empty_like(band)
    for _ in range(args.warmup):
        oracle.sslbm_run_inplace(band, scratch, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sslbm_run_inplace(band, scratch, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], 1)
    el = time.perf_counter() - t0
    cells = rows * NX
    value = cells * args.steps / el / 1e9
    sample = (f"one FP64 oracle lattice step per benchmark step on a {NX}x{rows} band of the "
              f"{NX}x{NY} grid (no-flux band edges)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl["name"], "nx": NX, "ny": NY, "band_rows": rows,
                       "lattice_steps_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def pass_split(n, depth):
    """The passes sslbm_step makes for n steps at this depth (ceil(n / depth) passes whose
    depths differ by at most one), as text, e.g. '10 x 7 + 5 x 6'."""
    ks = []
    while n > 0:
        if depth > 1 and n > 1:
            p = (n + depth - 1) // depth
            k = (n + p - 1) // p
        else:
            k = 1
        ks.append(k)
        n -= k
    return " + ".join(f"{ks.count(k)} x {k}" for k in sorted(set(ks), reverse=True))


def timed_steps(solver, n_lat, steps, stream, diag=True):
    """Run `steps` benchmark steps; returns (total ms, kernel ms) from CUDA events."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        starts[i].record(stream)
        solver.step(n_lat)
        ends[i].record(stream)
        if diag:
            solver.diagnostics()
    t1.record(stream)
    t1.synchronize()
    total = t0.elapsed_time(t1)
    kern = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    return total, kern


def main():
    global NX, NY
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=103)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--depth", type=int, default=0, help="temporal-blocking depth (0 = default)")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary variant timings")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-inflight", type=int, default=4, help="end-to-end jobs in flight (solvers and threads)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the ensemble measurement")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate kernel timing")
    ap.add_argument("--ens-scenarios", type=int, default=512, help="ensemble size (profiling cases)")
    ap.add_argument("--ens-steps", type=int, default=5000, help="ensemble steps (profiling cases)")
    ap.add_argument("--ens-tiling", default="", help="depth,seg_rows instead of the autotuner")
    ap.add_argument("--fused-diagnostics", action="store_true",
                    help="take the diagnostics in the last pass of each step (sslbm_set_fused_diagnostics)")
    ap.add_argument("--nx", type=int, default=NX, help="grid width (profiling cases; default 8192)")
    ap.add_argument("--ny", type=int, default=NY, help="grid height (profiling cases; default 8192)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2603_19789_gb300 import build as libbuild
    from paper_2603_19789_gb300 import inputs
    from paper_2603_19789_gb300 import sslbm as L

    NX, NY = args.nx, args.ny
    rank, world, local = dist_setup(args.gpus)
    libbuild.build()
    L.load()
    stream = torch.cuda.current_stream()
    wl = inputs.roofline_workload(NX, NY)
    state64 = wl["state"]
    state32 = np.ascontiguousarray(state64.astype(np.float32))
    rates = wl["rates"].as_tuple()

    s = L.Solver(NX, NY, rates, d=wl["d"], bc=wl["bc"], precision=L.FP32)
    s.write(state32)
    if args.fused_diagnostics:
        s.set_fused_diagnostics(True)
    tuned = None
    if args.depth:
        s.set_blocking(args.depth)
    else:
        tuned = s.autotune(300.0)  # (depth, seg_rows, ms per lattice step) from the library's autotuner
    depth, seg = s.get_blocking()
    for _ in range(args.warmup):
        s.step(LATTICE_STEPS_PER_STEP)
        s.diagnostics()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, kern_ms = timed_steps(s, LATTICE_STEPS_PER_STEP, args.steps, stream)
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(world)
    total_ms = max_over_ranks(total_ms, world)
    cells = NX * NY
    value = world * cells * LATTICE_STEPS_PER_STEP * args.steps / (total_ms * 1e-3) / 1e9
    fused_diag = s.get_fused_diagnostics()[1]  # the last pass took the diagnostics
    # step launches, then the diagnostics: one kernel adding the fused pass's partials, or two
    launches_per_step = math.ceil(LATTICE_STEPS_PER_STEP / depth) + (1 if fused_diag else 2)
    launch_ms = kern_ms / (args.steps * math.ceil(LATTICE_STEPS_PER_STEP / depth))
    hbm, peak_kind = load_peaks()
    achieved = BYTES_PER_CELL_FP32 * cells / (launch_ms * 1e-3) / 1e9
    tot, peak_I = s.diagnostics()

    extras = {}
    if not args.no_extras:
        extras = secondary_timings(L, wl, state64, state32, stream, hbm)

    ens = None
    if not args.no_ensemble and rank == 0:
        tiling = tuple(int(v) for v in args.ens_tiling.split(",")) if args.ens_tiling else None
        ens = ensemble_timing(L, torch, stream, n_scen=args.ens_scenarios, steps=args.ens_steps,
                              tiling=tiling)

    sur = None
    if not args.no_surrogate and rank == 0:
        sur = surrogate_timing(L, torch, stream, hbm)

    e2e = None
    if not args.no_e2e:
        e2e = e2e_timing(L, torch, s, state32, stream, world, wl, jobs=8 * args.e2e_inflight,
                         inflight=args.e2e_inflight)

    cpu = None
    if rank == 0 and not args.no_cpu:
        g, steps_cpu, shape, el = cpu_oracle_glups(state64, wl, budget_s=10.0, rows=2048)
        import oracle
        cpu = {"value": g, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{steps_cpu} FP64 oracle lattice steps on a {shape[2]}x{shape[1]} band of the "
                         f"{NX}x{NY} grid ({el:.1f} s)"}
    s.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "nx": NX, "ny": NY, "bc": "no-flux",
                       "precision": "fp32", "lattice_steps_per_step": LATTICE_STEPS_PER_STEP,
                       "temporal_block_depth": depth, "seg_rows": seg or "auto",
                       "passes_per_step": pass_split(LATTICE_STEPS_PER_STEP, depth),
                       "blocking_chosen_by": "autotuner" if tuned else "--depth",
                       "diagnostics": "fused into the last pass of each step" if fused_diag
                                      else "separate reduction after each step",
                       "l2": f"state {20 * cells / 1e9:.2f} GB vs 129 MB L2"
                             + (" (no flush needed)" if 20 * cells > 129e6 else " (fits in L2)"),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": captured_traffic(depth, cells),
                         "traffic_source": "ncu capture in profiles/ scaled by cells (null if the "
                                           "kernel sources changed since)",
                         "peak_kind": peak_kind,
                         "kernel": f"pipe_kernel<fp32, K={depth}>" if depth > 1 else "step1_kernel<fp32>",
                         "bytes_per_launch": BYTES_PER_CELL_FP32 * cells,
                         "launch_ms": launch_ms,
                         # the lattice steps of a bench step spread over its passes (depths differ
                         # by at most one), so a launch averages cells * steps / passes updates
                         "cell_updates_per_launch": cells * LATTICE_STEPS_PER_STEP
                                                    / math.ceil(LATTICE_STEPS_PER_STEP / depth),
                         # what one-step kernels would have to move for the same cell-steps: above
                         # the HBM peak because the K steps of a launch share one pass over HBM
                         "per_step_equivalent": {
                             "achieved": BYTES_PER_CELL_FP32 * value * 1e9 / world / 1e9,
                             "frac": BYTES_PER_CELL_FP32 * value / world / hbm,
                             "unit": "GB/s",
                             "note": "40 B per cell-step x cell-steps per second (whole step, diagnostics "
                                     "included) / measured HBM peak"}},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "diagnostics": {"total_population": float(tot.sum()), "peak_I": peak_I},
            "extras": extras,
            "ensemble": ens,
            "surrogate": sur,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def e2e_timing(L, torch, s, state32, stream, world, wl, steps=3, jobs=8, inflight=2):
    """Jobs through the public API with host buffers: IC in from pinned host memory, 100
    lattice steps, diagnostics, final state out.  Serial: one job after another on one
    solver.  Pipelined (the reported value): `inflight` solvers, each with its own stream
    and host thread, so that one job's copies overlap another's compute; every job still
    does all its copies inside the timed region."""
    import threading
    host_in = torch.from_numpy(state32).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    L.sslbm_write(s.h, L.SCHEME_SSLBM, L.ALL, host_in)
    s.step(LATTICE_STEPS_PER_STEP)
    L.sslbm_read(s.h, L.SCHEME_SSLBM, L.ALL, host_out)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        L.sslbm_write(s.h, L.SCHEME_SSLBM, L.ALL, host_in)
        s.step(LATTICE_STEPS_PER_STEP)
        s.diagnostics()
        L.sslbm_read(s.h, L.SCHEME_SSLBM, L.ALL, host_out)
    torch.cuda.synchronize()
    el_serial = max_over_ranks(time.perf_counter() - t0, world)
    serial = world * NX * NY * LATTICE_STEPS_PER_STEP * steps / el_serial / 1e9

    depth, seg = s.get_blocking()
    solvers = []
    for _ in range(inflight):
        sv = L.Solver(NX, NY, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=L.FP32,
                      stream=torch.cuda.Stream())
        sv.set_blocking(depth, seg)
        solvers.append(sv)
    outs = [torch.empty_like(host_in).pin_memory() for _ in range(inflight)]
    errors = []

    def run(i, n):
        try:
            sv = solvers[i]
            for _ in range(n):
                L.sslbm_write(sv.h, L.SCHEME_SSLBM, L.ALL, host_in)
                sv.step(LATTICE_STEPS_PER_STEP)
                sv.diagnostics()
                L.sslbm_read(sv.h, L.SCHEME_SSLBM, L.ALL, outs[i])
        except Exception as e:  # surfaced after the join
            errors.append(e)

    for i in range(inflight):
        run(i, 1)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    threads = [threading.Thread(target=run, args=(i, jobs // inflight)) for i in range(inflight)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, world)
    if errors:
        raise errors[0]
    for sv in solvers:
        sv.close()
    njobs = inflight * (jobs // inflight)
    v = world * NX * NY * LATTICE_STEPS_PER_STEP * njobs / el / 1e9
    nbytes = host_in.numel() * host_in.element_size()
    return {"value": v, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 48,
            "steps": njobs, "ms_per_step": el / njobs * 1e3,
            "pipeline": f"{inflight} jobs in flight: {inflight} solvers, each on its own stream and host thread",
            "serial": {"value": serial, "steps": steps, "ms_per_step": el_serial / steps * 1e3}}


def fused_diagnostics_timing(L, wl, state32, stream, reps=20):
    """One blocked FP32 pass (1024-row segments) with and without the diagnostics fused into
    it, and the separate diagnostics reduction, in ms per call at depths 2, 4 and 8."""
    import torch
    s = L.Solver(NX, NY, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=L.FP32)
    s.write(state32)

    def per_call(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    out = {}
    for k in (2, 4, 8):
        s.set_blocking(k, 1024)
        s.set_fused_diagnostics(False)
        plain = per_call(lambda: s.step(k))
        separate = per_call(lambda: s.diagnostics())
        s.set_fused_diagnostics(True)
        fused = per_call(lambda: s.step(k))
        if not s.get_fused_diagnostics()[1]:
            raise RuntimeError("the fused diagnostics were not taken")
        out[f"K{k}"] = {"plain_pass_ms": plain, "fused_pass_ms": fused, "separate_reduction_ms": separate}
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


def secondary_timings(L, wl, state64, state32, stream, hbm):
    """Other variants on the same grid: FP64, deviation-S, split-S, Kahan, depth sweep, BGK,
    D2Q9, two-pass SLBM, varying diffusivity, FD4."""
    import torch
    from paper_2603_19789_gb300 import inputs
    out = {}
    rates = wl["rates"].as_tuple()
    cells = NX * NY

    def glups_of(precision, n_lat, reps, depth=None, schemes=L.WANT_SSLBM, bgk=False):
        s = L.Solver(NX, NY, rates, d=wl["d"], bc=wl["bc"], precision=precision, schemes=schemes)
        if bgk:
            s.write(state64, scheme=L.SCHEME_BGK)
        else:
            s.write(state64 if precision in (L.FP64, L.FP64_DW) else state32)
        if depth == "auto":
            s.autotune()
        elif depth:
            s.set_blocking(depth)
        run = s.bgk_step if bgk else s.step
        run(n_lat)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            run(n_lat)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        s.close()
        del s
        torch.cuda.empty_cache()
        return cells * n_lat * reps / (ms * 1e-3) / 1e9, ms / (n_lat * reps)

    for k in (1, 2, 3, 4, 6, 8):
        g, ms = glups_of(L.FP32, 48, 4, depth=k)
        out[f"fp32_depth{k}_glups"] = g
        if k == 1:
            out["fp32_depth1_hbm_frac"] = BYTES_PER_CELL_FP32 * cells / (ms * 1e-3) / 1e9 / hbm
    out["fused_diagnostics"] = fused_diagnostics_timing(L, wl, state32, stream)
    # the other storages at the autotuned blocking, and one step per launch against HBM
    g, _ = glups_of(L.FP32_DEV, 48, 4, depth="auto")
    out["fp32_dev_glups"] = g
    g, _ = glups_of(L.FP32_SPLIT, 48, 4, depth="auto")
    out["fp32_split_glups"] = g
    g, ms = glups_of(L.FP32_SPLIT, 20, 2, depth=1)
    out["fp32_split_depth1_glups"] = g
    out["fp32_split_depth1_hbm_frac"] = 48 * cells / (ms * 1e-3) / 1e9 / hbm
    g, ms = glups_of(L.FP32_KAHAN, 20, 2, depth=1)
    out["fp32_kahan_glups"] = g
    out["fp32_kahan_hbm_frac"] = 80 * cells / (ms * 1e-3) / 1e9 / hbm
    g, _ = glups_of(L.FP32_KAHAN, 48, 2, depth="auto")
    out["fp32_kahan_blocked_glups"] = g
    g, ms = glups_of(L.FP64, 20, 2)
    out["fp64_glups"] = g
    out["fp64_hbm_frac"] = BYTES_PER_CELL_FP64 * cells / (ms * 1e-3) / 1e9 / hbm
    # the FP64 kernels are bound by the FP64 arithmetic rate, not by HBM: their roofline is a
    # measured FP64 rate (cuBLAS DGEMM, 4096^3, best of 5), against the update's 46 FP64
    # flops per cell-step (an FMA counts 2)
    A = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    Bm = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(A, Bm)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(A, Bm)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    del A, Bm
    torch.cuda.empty_cache()
    out["fp64_measured_peak_tflops"] = 2 * 4096 ** 3 / (best * 1e-3) / 1e12
    out["fp64_tflops"] = FP64_FLOPS_PER_CELL * g / 1e3
    out["fp64_frac_of_measured_fp64"] = out["fp64_tflops"] / out["fp64_measured_peak_tflops"]
    # FP64 accuracy in FP32 arithmetic: the double-word storage (hi + lo float pairs, 80 B per
    # cell-step), one step per launch
    g, ms = glups_of(L.FP64_DW, 20, 2)
    out["fp64_dw_glups"] = g
    out["fp64_dw_hbm_frac"] = 80 * cells / (ms * 1e-3) / 1e9 / hbm
    out["fp64_dw_vs_fp64"] = g / out["fp64_glups"]
    g, ms = glups_of(L.FP32, 20, 2, schemes=L.WANT_BGK, bgk=True)
    out["bgk_fp32_glups"] = g
    out["bgk_fp32_hbm_frac"] = BGK_BYTES_PER_CELL_FP32 * cells / (ms * 1e-3) / 1e9 / hbm
    # the D2Q9 lattice, one step per launch: 40 / 80 B per cell-step
    for prec, name, nbytes in ((L.FP32, "fp32", BYTES_PER_CELL_FP32), (L.FP64, "fp64", BYTES_PER_CELL_FP64)):
        s9 = L.Solver(NX, NY, rates, d=wl["d"], bc=wl["bc"], precision=prec, lattice=L.LATTICE_D2Q9)
        s9.write(state32 if prec == L.FP32 else state64)
        s9.set_blocking(1)
        s9.step(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20 if prec == L.FP32 else 6
        a.record(stream)
        s9.step(reps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        out[f"d2q9_{name}_glups"] = cells / (ms * 1e-3) / 1e9
        out[f"d2q9_{name}_hbm_frac"] = nbytes * cells / (ms * 1e-3) / 1e9 / hbm
        if prec == L.FP32:
            # the temporal-blocked D2Q9 kernel at the autotuned depth, 48 steps per measurement
            depth, seg, _ = s9.autotune()
            s9.step(depth)
            torch.cuda.synchronize()
            a.record(stream)
            s9.step(48)
            b.record(stream)
            b.synchronize()
            out["d2q9_fp32_blocked_glups"] = cells * 48 / (a.elapsed_time(b) * 1e-3) / 1e9
            out["d2q9_fp32_blocked_depth"] = depth
        s9.close()
        del s9
        torch.cuda.empty_cache()
    # the two-pass SLBM: predictor (4 planes in, 4 out) + corrector (4 predictor + 5 state
    # planes in, 5 out) = 22 planes per cell-step
    for prec, name, esz in ((L.FP32, "fp32", 4), (L.FP64, "fp64", 8)):
        s2 = L.Solver(NX, NY, rates, d=wl["d"], bc=wl["bc"], precision=prec, lattice=L.LATTICE_D2Q5_SLBM)
        s2.write(state32 if prec == L.FP32 else state64)
        s2.step(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20 if prec == L.FP32 else 6
        a.record(stream)
        s2.step(reps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        out[f"slbm_{name}_glups"] = cells / (ms * 1e-3) / 1e9
        out[f"slbm_{name}_hbm_frac"] = 22 * esz * cells / (ms * 1e-3) / 1e9 / hbm
        s2.close()
        del s2
        torch.cuda.empty_cache()
    # spatially varying, anisotropic diffusion: 5 state planes and the 2 scale planes read,
    # 5 planes written = 12 planes per cell-step; a mobility map of a few 'cities'
    kx, ky = inputs.mobility_fields(NX, NY, 7)
    for prec, name, esz in ((L.FP32, "fp32", 4), (L.FP64, "fp64", 8)):
        sv = L.Solver(NX, NY, rates, d=wl["d"], bc=wl["bc"], precision=prec, lattice=L.LATTICE_D2Q5_VARD)
        sv.set_diffusivity_scale(kx, ky)
        sv.write(state32 if prec == L.FP32 else state64)
        sv.set_blocking(1)
        sv.step(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20 if prec == L.FP32 else 6
        a.record(stream)
        sv.step(reps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        out[f"vard_{name}_glups"] = cells / (ms * 1e-3) / 1e9
        out[f"vard_{name}_hbm_frac"] = 12 * esz * cells / (ms * 1e-3) / 1e9 / hbm
        if prec == L.FP32:
            # the temporal-blocked kernel at the autotuned depth, 48 steps per measurement
            depth, seg, _ = sv.autotune()
            sv.step(depth)
            torch.cuda.synchronize()
            a.record(stream)
            sv.step(48)
            b.record(stream)
            b.synchronize()
            out["vard_fp32_blocked_glups"] = cells * 48 / (a.elapsed_time(b) * 1e-3) / 1e9
            out["vard_fp32_blocked_depth"] = depth
        sv.close()
        del sv
        torch.cuda.empty_cache()
    # the fourth-order finite-difference reference (RK4): four stage kernels per step that
    # move 85 planes per cell (stage states, slope sum and u, read and written)
    for prec, name, esz, reps in ((L.FP64, "fp64", 8, 3), (L.FP32, "fp32", 4, 6)):
        f = L.Fd4(NX, NY, rates, wl["d"][:4], bc=wl["bc"], precision=prec)
        f.write(state64 if prec == L.FP64 else state32)
        f.step(1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f.step(reps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        out[f"fd4_{name}_glups"] = cells / (ms * 1e-3) / 1e9
        out[f"fd4_{name}_hbm_frac"] = FD4_PLANES_PER_CELL * esz * cells / (ms * 1e-3) / 1e9 / hbm
        f.close()
        del f
        torch.cuda.empty_cache()
    return out


def surrogate_timing(L, torch, stream, hbm, batch=64, n=256, reps=10):
    """The learned surrogate's kernels at the rollout's batch (64 scenarios, 256 x 256): one
    surrogate step = make_input + inference + residual check/projection, with seeded initial
    parameters (the time does not depend on their values); then the library's rollout call
    on the same scenarios under the workload's fallback rule, against the plain FP64 SSLBM
    batched over the scenarios and the FP32 ensemble.  A surrogate step advances every
    scenario by 20 lattice steps."""
    from paper_2603_19789_gb300 import inputs
    from paper_2603_19789_gb300 import surrogate as S
    sur = L.Surrogate(n=n, max_batch=batch)
    sur.set_params(S.initial_params())
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    u = torch.rand((batch, 5, n, n), device="cuda", generator=g)
    r0 = torch.full((batch,), 2.6, device="cuda")
    ld = torch.full((batch,), -2.0, device="cuda")
    x = sur.make_input(u, r0, ld)
    y = sur.infer(x)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    infer_ms = timed(lambda: sur.infer(x, y))
    step_ms = timed(lambda: (sur.make_input(u, r0, ld), sur.infer(x, y), sur.check_project(y, u)))
    flops = batch * S.forward_flops(n)
    nbytes = batch * S.forward_bytes(n)
    # the library's rollout call on the workload's scenarios, under the workload's rule
    # (conservation residual <= 1e-4, no negative density), 10 surrogate steps per call
    sc, specs, sr0, slogd = S.scenario_specs(batch, n, 11)
    us = torch.stack([torch.from_numpy(inputs.ensemble_state(c).astype(np.float32)) for c in sc]).cuda()
    tr0, tld = torch.from_numpy(sr0).cuda(), torch.from_numpy(slogd).cuda()
    xs = torch.empty((batch, 8, n, n), dtype=torch.float32, device="cuda")
    ys = torch.empty_like(us)
    fb = L.Ensemble(specs)
    fb.set_tiling(4, 64)
    L.sslbm_surrogate_rollout(sur.f, fb.e, batch, 2, S.K_STEPS, us, tr0, tld, xs, ys, 1e-4, 0.0, 0, False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, _, _ = L.sslbm_surrogate_rollout(sur.f, fb.e, batch, 10, S.K_STEPS, us, tr0, tld, xs, ys, 1e-4, 0.0, 0,
                                         False)
    torch.cuda.synchronize()
    roll_s = time.perf_counter() - t0
    fb.close()
    sur.close()
    roll = batch * 10 * S.K_STEPS / roll_s
    fp64_b = S.fp64_batched_scenario_steps_per_s(n, batch)
    fp32_e = S.fp32_ensemble_scenario_steps_per_s(n, batch, steps=400)
    return {"batch": batch, "n": n, "params": S.initial_params().size, "fused": True,
            "infer_ms": infer_ms, "gflop_per_inference": flops / 1e9, "tflops": flops / (infer_ms * 1e-3) / 1e12,
            "hbm_bytes_per_inference": nbytes, "hbm_frac": nbytes / (infer_ms * 1e-3) / 1e9 / hbm,
            "surrogate_step_ms": step_ms,
            "rollout_scenario_steps_per_s": roll, "rollout_fallbacks": st["fallbacks"],
            "rollout_rule": "conservation residual <= 1e-4 and no negative density",
            "fp64_batched_scenario_steps_per_s": fp64_b, "rollout_vs_fp64_batched": roll / fp64_b,
            "fp32_ensemble_scenario_steps_per_s": fp32_e, "rollout_vs_fp32_ensemble": roll / fp32_e,
            "note": "seeded initial parameters (the time does not depend on them); the trained network's "
                    "fallback rate and error against the SSLBM: studies.py surrogate"}


def ensemble_timing(L, torch, stream, n_scen=512, steps=5000, err_scen=6, fp64_steps=40, tiling=None):
    """The 512-scenario ensemble (grids 256..1024 squared, periodic, FP32) for 5000 steps in
    one persistent graph-captured launch, against the plain FP64 SSLBM run scenario by
    scenario on the same GPU.  The FP64 time is measured on one scenario of each grid size
    for fp64_steps steps and weighted by the ensemble's size mix; the FP32 error is the
    root-mean-square difference from FP64 per compartment (density units, total ~1) on the
    first err_scen scenarios after all steps.  The same run with S stored as a hi/lo pair
    (FP32_SPLIT, autotuned on its own) is reported under "split": its throughput and error."""
    from paper_2603_19789_gb300 import inputs
    scen = inputs.ensemble_scenarios(n_scen)
    specs = [dict(nx=s["nx"], ny=s["ny"], rates=s["rates"].as_tuple(), d=s["d"]) for s in scen]
    cells = sum(s["nx"] * s["ny"] for s in scen)
    # plain FP64 SSLBM, one scenario per grid size
    per_size = {}
    for s in scen:
        if s["nx"] in per_size:
            continue
        f = L.Solver(s["nx"], s["ny"], s["rates"].as_tuple(), d=s["d"], bc=L.BC_PERIODIC, precision=L.FP64)
        f.write(inputs.ensemble_state(s))
        f.step(4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f.step(fp64_steps)
        e1.record(stream)
        e1.synchronize()
        per_size[s["nx"]] = e0.elapsed_time(e1) / fp64_steps
        f.close()
    fp64_ms = sum(per_size[s["nx"]] * steps for s in scen)
    # FP64 references of the first err_scen scenarios
    refs = []
    for i in range(min(err_scen, n_scen)):
        s = scen[i]
        f = L.Solver(s["nx"], s["ny"], s["rates"].as_tuple(), d=s["d"], bc=L.BC_PERIODIC, precision=L.FP64)
        f.write(inputs.ensemble_state(s))
        f.step(steps)
        refs.append(f.read())
        f.close()

    def run(precision, tile):
        ens = L.Ensemble(specs, precision=precision)
        if tile:
            ens.set_tiling(*tile)
            depth, seg = tile
        else:
            depth, seg, _ = ens.autotune(trial_blocks=2)
        for i, s in enumerate(scen):
            ens.write(i, inputs.ensemble_state(s).astype(np.float32))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.run(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        per = []
        for i, ref in enumerate(refs):
            got = ens.read(i)
            per.append(np.sqrt(((got - ref) ** 2).reshape(5, -1).mean(axis=1)))
        rms = (np.max(per, axis=0), np.median(per, axis=0))
        ens.close()
        del ens
        torch.cuda.empty_cache()
        return depth, seg, ms, rms

    depth, seg, ms, rms = run(L.FP32, tiling)
    sdepth, sseg, sms, srms = run(L.FP32_SPLIT, None)

    def errs(r):
        mx, md = r
        return {"S": mx[0], "E": mx[1], "I": mx[2], "R": mx[3], "D": mx[4],
                "median": {"S": md[0], "E": md[1], "I": md[2], "R": md[3], "D": md[4]},
                "scenarios": err_scen, "units": "density (total ~1); the largest and the median over the scenarios"}

    return {"scenarios": n_scen, "steps": steps, "cells": cells, "precision": "fp32",
            "tiling": {"depth": depth, "seg_rows": seg, "chosen_by": "--ens-tiling" if tiling else "autotuner"},
            "launch": "one persistent kernel per run, replayed from a CUDA graph",
            "ms": ms, "scenario_steps_per_s": n_scen * steps / (ms * 1e-3),
            "glups": cells * steps / (ms * 1e-3) / 1e9,
            "fp64_plain_scenario_steps_per_s": n_scen * steps / (fp64_ms * 1e-3),
            "fp64_plain_note": f"plain FP64 SSLBM per scenario, {fp64_steps} steps timed on one "
                               "scenario per grid size, weighted by the size mix",
            "speedup_vs_fp64": fp64_ms / ms,
            "rms_error_vs_fp64": errs(rms),
            "split": {"precision": "fp32_split", "tiling": {"depth": sdepth, "seg_rows": sseg},
                      "ms": sms, "scenario_steps_per_s": n_scen * steps / (sms * 1e-3),
                      "glups": cells * steps / (sms * 1e-3) / 1e9, "speedup_vs_fp64": fp64_ms / sms,
                      "rms_error_vs_fp64": errs(srms)}}


if __name__ == "__main__":
    main()
