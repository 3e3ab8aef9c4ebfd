"""Measurement studies built on the library (run on a GPU).

precision  -- the small-increment precision study: the multi-seed no-flux workload at
              4096 x 4096 with every infected seed at amplitude 1e-6, 50,000 steps, in six
              storage/arithmetic variants: FP64, FP32, FP32 with S stored as its deviation
              from the total density, FP32 with S stored as a hi/lo pair, FP32 with
              compensated (Kahan) accumulation of every compartment, and FP64 accuracy in
              double-word FP32 arithmetic.  Reports,
              at log-spaced checkpoints, each other variant's per-compartment root-mean-square
              and max-norm error against the FP64 run, divided by the compartment's peak so
              far (E and I decay to ~0 after the wave), the relative L2 error of the infected
              fraction 1 - S, and every variant's drift of the total population (FP64
              reductions).  The FP64 run is the reference: it matches the CPU oracle to
              1e-12 relative on the parity workloads, and the oracle itself would need tens of
              minutes of host time for 50,000 steps of this grid.

surrogate  -- the learned surrogate end to end on n x n periodic grids (default 256): 2000
              ensemble trajectories x 10 snapshot pairs (t, t + 20), Adam training with the
              library's forward/backward kernels, then a 64-scenario x 100-step rollout with
              residual checks and SSLBM fallback, judged against the SSLBM run in lock step,
              and its scenario-steps/s against the plain FP64 SSLBM on the same grid.

accuracy   -- the accuracy comparison of Sec. III at scale: FP64 SSLBM and BGK against the
              GPU fourth-order finite-difference RK4 reference under diffusive refinement
              (grids 64..512, fixed tau), relative L2 / max-norm errors and observed order.

timing     -- the cost comparison of Sec. IV (Table tab:timing): time per step of SSLBM,
              BGK, second- and fourth-order FDM (RK4) in FP64 and FP32 on grids 200..8192,
              normalised by the FP64 SSLBM at 200 x 200.

train-step -- time of one surrogate training step (B = 16, 256 x 256, default network).

variant    -- one update variant (lattice x storage, one step per launch or the default
              blocking) on the n x n multi-seed no-flux workload: GLUPS and the fraction of
              the measured HBM bandwidth its algorithmic bytes per cell-step reach; the
              profiling command of the one-step kernels.

Usage:  python -m paper_2603_19789_gb300.studies precision [--n 4096] [--steps 50000]
        [--checkpoints 5] [--out FILE]
        python -m paper_2603_19789_gb300.studies surrogate [--n 256] [--trajectories 2000]
        [--train-steps 3000] [--out FILE]
        python -m paper_2603_19789_gb300.studies accuracy [--out FILE]
        python -m paper_2603_19789_gb300.studies timing [--out FILE]
        python -m paper_2603_19789_gb300.studies train-step [--n 256] [--out FILE]
        python -m paper_2603_19789_gb300.studies variant --lattice d2q9 --precision fp32
        [--n 8192] [--steps 20] [--depth 1] [--bc periodic|noflux] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import inputs
from . import sslbm as L

VARIANTS = (("fp64", L.FP64), ("fp32", L.FP32), ("fp32_dev", L.FP32_DEV), ("fp32_split", L.FP32_SPLIT),
            ("fp32_kahan", L.FP32_KAHAN), ("fp64_dw", L.FP64_DW))


def precision_study(n: int = 4096, steps: int = 50000, checkpoints: int = 6, seed: int = inputs.DEFAULT_SEED):
    import torch
    wl = inputs.precision_workload(n, n, seed)
    st = wl["state"]
    total0 = float(st.sum())
    # log-spaced checkpoints: the take-off (smallest increments) comes first
    marks = sorted({int(round(steps ** ((i + 1) / checkpoints))) for i in range(checkpoints)} | {steps})
    solvers = {}
    for name, prec in VARIANTS:
        s = L.Solver(n, n, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=prec,
                     s_ref=1.0)
        s.write(st)
        if prec != L.FP64:
            s.autotune(200.0)
        solvers[name] = s
    out = {"workload": wl["name"], "n": n, "steps": steps, "seed_amplitude": 1e-6,
           "reference": "fp64 (GPU)", "checkpoints": []}
    done = 0
    peaks = {}
    timing = {name: 0.0 for name, _ in VARIANTS}
    for t in marks:
        rec = {"step": t, "drift": {}, "l2_over_peak": {}, "linf_over_peak": {},
               "rel_l2_one_minus_S": {}}
        states = {}
        for name, _ in VARIANTS:
            s = solvers[name]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(t - done)
            torch.cuda.synchronize()
            timing[name] += time.perf_counter() - t0
            tot, _ = s.diagnostics()
            rec["drift"][name] = (float(tot.sum()) - total0) / total0
            states[name] = s.read()
        ref = states["fp64"]
        for name, _ in VARIANTS:
            peaks[name] = np.maximum(peaks.get(name, 0.0), np.abs(ref).reshape(5, -1).max(axis=1))
        for name, _ in VARIANTS[1:]:
            diff = (states[name] - ref).reshape(5, -1)
            # each compartment's error over its peak value so far (E and I decay to ~0)
            pk = peaks["fp64"]
            rec["l2_over_peak"][name] = dict(zip("SEIRD", (np.sqrt((diff ** 2).mean(axis=1)) / pk).tolist()))
            rec["linf_over_peak"][name] = dict(zip("SEIRD", (np.abs(diff).max(axis=1) / pk).tolist()))
            dref = 1.0 - ref[0]
            da = 1.0 - states[name][0]
            rec["rel_l2_one_minus_S"][name] = float(np.linalg.norm(da - dref) / np.linalg.norm(dref))
        out["checkpoints"].append(rec)
        done = t
        del states
    out["glups"] = {name: n * n * steps / timing[name] / 1e9 for name, _ in VARIANTS}
    for s in solvers.values():
        s.close()
    return out


def accuracy_study(sizes=(64, 128, 256, 512), d_phys=1e-4, d_lattice=0.05, t_end=None, sub=4):
    """The accuracy comparison of Sec. III at scale: the SSLBM and the BGK LBM against the
    fourth-order finite-difference RK4 reference, under diffusive refinement.

    The centre-bump workload on the unit square (periodic), its bump width fixed
    physically (sigma = 1/16), no perturbation; d = d_phys for S, E, I, R; rates per unit
    time as in the workload.  Each grid n has dx = 1/n and dt = d_lattice dx^2 / d_phys,
    so tau (= 3 d_lattice + 1/2) is the same on every grid and the time error (first order
    in dt) scales like the space error (second order in dx).  The reference runs on the
    same grid with dt / sub.  Reported per compartment at the final time: relative L2 and
    max-norm errors of SSLBM and BGK against the reference, and the observed order of the
    SSLBM between successive grids."""
    out = {"d_phys": d_phys, "d_lattice": d_lattice, "tau": 3 * d_lattice + 0.5, "sub": sub, "grids": []}
    dt0 = d_lattice * (1.0 / 128) ** 2 / d_phys
    t_end = t_end if t_end is not None else 2000 * dt0
    out["t_end"] = t_end
    prev = None
    for n in sizes:
        wl = inputs.centre_bump_workload(n, n, sig=n / 16.0, noise=0.0)
        st = wl["state"]
        rates = wl["rates"].as_tuple()
        dx = 1.0 / n
        dt = d_lattice * dx * dx / d_phys
        steps = int(round(t_end / dt))
        d = (d_phys, d_phys, d_phys, d_phys, 0.0)
        t0 = time.perf_counter()
        s = L.Solver(n, n, rates, d=d, dx=dx, dt=dt, bc=L.BC_PERIODIC, precision=L.FP64,
                     schemes=L.WANT_SSLBM | L.WANT_BGK)
        s.write(st)
        s.write(st, scheme=L.SCHEME_BGK)
        s.step(steps)
        s.bgk_step(steps)
        a = s.read()
        b = s.read(scheme=L.SCHEME_BGK)
        s.close()
        f = L.Fd4(n, n, rates, d[:4], dx=dx, dt=dt / sub, bc=L.BC_PERIODIC, precision=L.FP64)
        f.write(st)
        f.step(steps * sub)
        ref = f.read()
        f.close()
        el = time.perf_counter() - t0

        def errs(x):
            l2 = [float(np.linalg.norm(x[c] - ref[c]) / np.linalg.norm(ref[c])) for c in range(5)]
            li = [float(np.abs(x[c] - ref[c]).max() / np.abs(ref[c]).max()) for c in range(5)]
            return {"rel_l2": dict(zip("SEIRD", l2)), "rel_linf": dict(zip("SEIRD", li))}

        rec = {"n": n, "dx": dx, "dt": dt, "steps": steps, "seconds": el,
               "sslbm": errs(a), "bgk": errs(b)}
        if prev is not None:
            rec["sslbm_order_l2"] = {c: float(np.log2(prev["sslbm"]["rel_l2"][c] / rec["sslbm"]["rel_l2"][c]))
                                     for c in "SEIRD"}
        out["grids"].append(rec)
        prev = rec
    return out


def timing_study(sizes=(200, 400, 600, 800, 1000, 2048, 4096, 8192), budget_ms=150.0):
    """The cost comparison of Sec. IV (Table tab:timing) on one GB300: time per step of the
    SSLBM, the BGK LBM, the second-order FDM and the fourth-order FDM (both RK4 in time)
    on n x n periodic grids, in FP64 and FP32, normalised by the FP64 SSLBM at 200 x 200
    as the paper normalises by its SSLBM at 200 x 200.  The state is the centre-bump
    workload (d = 0.05 lattice units for S, E, I, R; R0 = 3 with gamma + mu = 0.11).
    Each case: 3 warm-up steps, a trial, then enough steps for about budget_ms, timed with
    CUDA events on the solver's stream.  FP32 SSLBM uses the library's default blocking."""
    import torch
    rates = inputs.rates_from_sigma_mu(3 * 0.11, 0.2, 0.1, 0.01).as_tuple()
    d = (0.05, 0.05, 0.05, 0.05, 0.0)
    cases = [("SSLBM", L.FP64), ("BGK", L.FP64), ("FDM 2nd", L.FP64), ("FDM 4th", L.FP64),
             ("SSLBM", L.FP32), ("BGK", L.FP32), ("FDM 2nd", L.FP32), ("FDM 4th", L.FP32)]
    out = {"sizes": list(sizes), "unit": "ms per step", "cases": [], "rows": {}}
    for n in sizes:
        st = inputs.centre_bump_workload(n, n)["state"]
        row = {}
        for name, prec in cases:
            if name == "SSLBM":
                obj = L.Solver(n, n, rates, d=d, precision=prec)
                obj.write(st if prec == L.FP64 else st.astype(np.float32))
                run = obj.step
            elif name == "BGK":
                obj = L.Solver(n, n, rates, d=d, precision=prec, schemes=L.WANT_BGK)
                obj.write(st, scheme=L.SCHEME_BGK)
                run = obj.bgk_step
            else:
                obj = L.Fd4(n, n, rates, d[:4], precision=prec, order=2 if name == "FDM 2nd" else 4)
                obj.write(st)
                run = obj.step
            stream = obj.stream
            run(3)

            def timed(k):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                run(k)
                b.record(stream)
                b.synchronize()
                return a.elapsed_time(b) / k

            trial = timed(5)
            k = int(min(20000, max(5, budget_ms / max(trial, 1e-4))))
            ms = timed(k)
            obj.close()
            del obj
            torch.cuda.empty_cache()
            key = f"{name} {'fp64' if prec == L.FP64 else 'fp32'}"
            row[key] = {"ms_per_step": ms, "glups": n * n / (ms * 1e-3) / 1e9, "steps_timed": k}
        out["rows"][str(n)] = row
    base = out["rows"][str(sizes[0])]["SSLBM fp64"]["ms_per_step"]
    for n in sizes:
        for key, v in out["rows"][str(n)].items():
            v["normalised"] = v["ms_per_step"] / base
    return out


def surrogate_study(n=256, trajectories=2000, snapshots=10, horizon=2000, train_steps=20000, batch=16,
                    lr=1e-3, width=32, modes=12, layers=4, hidden=64, scenarios=64, rollout_steps=100,
                    params=None):
    """Generate trajectories with the ensemble kernel, train the surrogate on the GPU, and
    roll it out with residual checks and SSLBM fallback, judged against the SSLBM.  With
    params (a flat FP32 parameter vector) the training is skipped."""
    import torch

    from . import surrogate as S
    sur = L.Surrogate(n=n, width=width, modes=modes, layers=layers, hidden=hidden,
                      max_batch=max(batch, scenarios))
    t_data, hist = 0.0, None
    if params is None:
        t0 = time.perf_counter()
        X, Y, r0, logd = S.generate_pairs(n, trajectories, snapshots, horizon)
        t_data = time.perf_counter() - t0
        sur.set_params(S.initial_params(width, modes, layers, hidden))
        hist = S.train(sur, X, Y, r0, logd, steps=train_steps, batch=batch, lr=lr)
        del X, Y
        torch.cuda.empty_cache()
    else:
        sur.set_params(np.asarray(params, dtype=np.float32))
    theta = sur.get_params()
    # the workload's rule: conservation residual <= 1e-4 and no negative density at all
    roll = S.rollout(sur, n=n, scenarios=scenarios, steps=rollout_steps, threshold=1e-4, neg_threshold=0.0)
    # throughput alone: one rollout call for all steps, no judge between calls
    fast = S.rollout(sur, n=n, scenarios=scenarios, steps=rollout_steps, threshold=1e-4, neg_threshold=0.0,
                     reference=False, err_every=rollout_steps)
    roll.pop("state")
    roll.pop("reference_state")
    fp64 = S.fp64_scenario_steps_per_s(n)
    fp64_b = S.fp64_batched_scenario_steps_per_s(n, scenarios)
    fp32_e = S.fp32_ensemble_scenario_steps_per_s(n, scenarios)
    out = {"n": n, "trajectories": trajectories, "pairs": trajectories * snapshots,
           "params": sur.nparams, "data_seconds": t_data, "train": hist, "rollout": roll,
           "rollout_one_call": {k: fast[k] for k in ("fallbacks", "fallback_rate", "seconds", "scenario_steps_per_s")},
           "fp64_plain_scenario_steps_per_s": fp64,
           "fp64_batched_scenario_steps_per_s": fp64_b,
           "fp32_ensemble_scenario_steps_per_s": fp32_e,
           "speedup_vs_fp64": fast["scenario_steps_per_s"] / fp64,
           "speedup_vs_fp64_batched": fast["scenario_steps_per_s"] / fp64_b,
           "ratio_to_fp32_ensemble": fast["scenario_steps_per_s"] / fp32_e}
    return out, theta


def train_step_timing(n=256, batch=16, steps=50):
    """Time of one training step (forward, loss, backward through the tensor-core products,
    Adam) of the default network (W = 32, m = 12, L = 4, H = 64) on a synthetic batch, by
    CUDA events over `steps` steps after five warm-up steps."""
    import torch
    from . import sslbm as L
    from . import surrogate as S
    L.load()
    sur = L.Surrogate(n=n, max_batch=batch)
    sur.set_params(S.initial_params(32, 12, 4, 64, seed=0))
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    X = torch.rand((batch, 5, n, n), device="cuda", generator=g) * 0.2
    Y = (X * 0.99).contiguous()
    x = sur.make_input(X, torch.full((batch,), 2.0, device="cuda"), torch.full((batch,), -2.0, device="cuda"))
    for _ in range(5):
        sur.train_step(x, Y, 1e-4, want_loss=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(sur.stream)
    for _ in range(steps):
        sur.train_step(x, Y, 1e-4, want_loss=False)
    b.record(sur.stream)
    b.synchronize()
    loss = sur.train_step(x, Y, 1e-4, want_loss=True)
    return {"n": n, "batch": batch, "steps": steps, "ms_per_step": a.elapsed_time(b) / steps, "loss": loss}


# algorithmic bytes per cell-step of each (lattice, precision) at one step per launch: every
# plane the update reads, read once, and every plane it writes, written once
_ESIZE = {L.FP64: 8, L.FP32: 4, L.FP32_DEV: 4, L.FP32_SPLIT: 4, L.FP32_KAHAN: 4, L.FP64_DW: 4}
_PLANES = {L.FP32_SPLIT: 6, L.FP32_KAHAN: 10, L.FP64_DW: 10}
LATTICES = {"d2q5": L.LATTICE_D2Q5, "d2q9": L.LATTICE_D2Q9, "vard": L.LATTICE_D2Q5_VARD}
PRECISION_NAMES = {"fp64": L.FP64, "fp32": L.FP32, "fp32_dev": L.FP32_DEV, "fp32_split": L.FP32_SPLIT,
                   "fp32_kahan": L.FP32_KAHAN, "fp64_dw": L.FP64_DW}


def _measured_hbm_gbs():
    """The measured copy bandwidth of the GPU (MEASURED_PEAKS.json at the repository root), or None."""
    import os
    try:
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def variant_timing(lattice="d2q9", precision="fp32", n=8192, steps=20, depth=1, bc=None):
    """GLUPS of one update variant on the n x n multi-seed no-flux workload (inputs larger than
    L2 at the default size): 4 warm-up steps, then `steps` steps timed with CUDA events on the
    solver's stream.  depth applies where a blocked kernel exists (the D2Q5 FP32 storages, FP32
    D2Q9 and varying diffusion): 1 = one step per launch, 0 = the default blocking, k = k steps
    per launch.
    hbm_frac = algorithmic bytes per cell-step (every plane read once and written once; the
    two scale planes read once on the varying-diffusion lattice) over the step time, divided
    by the measured HBM bandwidth; it is reported for one-step launches only."""
    import torch
    lat, prec = LATTICES[lattice], PRECISION_NAMES[precision]
    wl = inputs.roofline_workload(n, n)
    st = wl["state"] if prec in (L.FP64, L.FP64_DW) else np.ascontiguousarray(wl["state"].astype(np.float32))
    bc = wl["bc"] if bc is None else bc
    s = L.Solver(n, n, wl["rates"].as_tuple(), d=wl["d"], bc=bc, precision=prec, lattice=lat)
    if lat == L.LATTICE_D2Q5_VARD:
        s.set_diffusivity_scale(*inputs.mobility_fields(n, n, 7))
    s.write(st)
    blockable = (L.LATTICE_D2Q5, L.LATTICE_D2Q9, L.LATTICE_D2Q5_VARD)
    if lat in blockable and depth and not (lat != L.LATTICE_D2Q5 and prec != L.FP32):
        s.set_blocking(depth)
    s.step(4)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    s.step(steps)
    b.record(s.stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    s.close()
    planes = _PLANES.get(prec, 5)
    nbytes = _ESIZE[prec] * (2 * planes + (2 if lat == L.LATTICE_D2Q5_VARD else 0))
    out = {"lattice": lattice, "precision": precision, "n": n, "bc": "periodic" if bc == L.BC_PERIODIC else "no-flux",
           "depth": depth, "steps": steps, "ms_per_step": ms,
           "glups": n * n / (ms * 1e-3) / 1e9, "bytes_per_cell_step": nbytes}
    one_step = lat not in blockable or depth == 1 or prec in (L.FP64, L.FP32_KAHAN)
    peak = _measured_hbm_gbs()
    if one_step and peak:
        out["hbm_frac"] = nbytes * n * n / (ms * 1e-3) / 1e9 / peak
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["precision", "surrogate", "accuracy", "timing", "train-step", "variant"])
    ap.add_argument("--lattice", default="d2q9", choices=sorted(LATTICES))
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISION_NAMES))
    ap.add_argument("--depth", type=int, default=1)
    ap.add_argument("--bc", default=None, choices=["periodic", "noflux"], help="variant: the workload's (no-flux) if unset")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--steps", type=int, default=50000)
    ap.add_argument("--checkpoints", type=int, default=6)
    ap.add_argument("--trajectories", type=int, default=2000)
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--params", default=None, help="trained parameters (.npy): skip the training")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    from . import build
    build.build()
    if args.study in ("accuracy", "timing", "train-step", "variant"):
        res = (accuracy_study() if args.study == "accuracy" else
               timing_study() if args.study == "timing" else
               variant_timing(args.lattice, args.precision, n=args.n or 8192,
                              steps=args.steps if args.steps != 50000 else 20, depth=args.depth,
                              bc=None if args.bc is None else (L.BC_PERIODIC if args.bc == "periodic" else L.BC_NOFLUX))
               if args.study == "variant" else train_step_timing(n=args.n or 256))
        text = json.dumps(res, indent=1)
        if args.out:
            with open(args.out, "w") as fh:
                fh.write(text + "\n")
        print(text)
        return
    if args.study == "surrogate":
        res, theta = surrogate_study(n=args.n or 256, trajectories=args.trajectories, train_steps=args.train_steps,
                                     params=np.load(args.params) if args.params else None)
        text = json.dumps(res, indent=1)
        if args.out:
            with open(args.out, "w") as fh:
                fh.write(text + "\n")
            np.save(args.out.rsplit(".", 1)[0] + "_params.npy", theta)
        print(text)
        return
    res = precision_study(args.n or 4096, args.steps, args.checkpoints)
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text + "\n")
    print(text)


if __name__ == "__main__":
    sys.exit(main())
