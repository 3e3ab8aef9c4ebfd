"""Training data, training and rollout of the learned surrogate (host orchestration only:
every computation runs in libsslbm's kernels; torch provides device buffers and batch
gathering).

Data: trajectories of the periodic ensemble workload's parameter ranges (R0 ~ U[1.2, 4],
d ~ logU[1e-3, 1e-1], 1..8 Gaussian seeds) on n x n grids, produced by the persistent
ensemble launch; from each trajectory, snapshots at stratified random multiples of 20 steps
over the rollout horizon (one per stratum), each paired with the state 20 steps later.

Rollout (the library's sslbm_surrogate_rollout): each surrogate step advances a batch of
scenarios by 20 SSLBM steps.  The network's output is nonnegative and holds its input's
population by construction; the prediction y is still checked against the input state u --
the conservation residual |sum y - sum u| / sum u and the negative mass sum max(-y, 0) / sum u,
infinite for a non-finite prediction -- and a scenario whose conservation residual exceeds
1e-4 or that has any negative density (neg_threshold = 0) takes the SSLBM's 20 steps instead
(the fallback, run by the ensemble kernel).  The SSLBM also judges the rollout: a reference
ensemble advanced in lock step between the rollout calls gives the error.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs
from . import sslbm as L

K_STEPS = 20


def forward_flops(n=256, width=32, modes=12, layers=4, hidden=64, cin=8):
    """Floating-point operations of one forward pass of one sample, from the layer sizes
    (multiply-adds count 2): lift, per layer the transforms along x and y and their
    inverses plus the channel map, the complex mode mixing, and the projection MLP."""
    P, W, m, H = n * n, width, modes, hidden
    lift = 2 * cin * W * P
    per_layer = (2 * W * P * 4 * m            # along x: h Fx
                 + 2 * W * 2 * m * n * 4 * m  # along y: Fy H1
                 + 8 * W * W * 2 * m * m      # complex mixing of the 2m x m modes
                 + 2 * W * n * 2 * m * 4 * m  # inverse along y: Fyi U
                 + 2 * W * (W + 4 * m) * P)   # channel map + inverse along x: [B | G1] [h ; Fxi]
    proj = 2 * H * W * P + 2 * 5 * H * P
    return lift + layers * per_layer + proj


def forward_bytes(n=256, width=32, modes=12, layers=4, cin=8):
    """HBM bytes one sample's fused inference must move: the input, each layer's BF16
    activations in and out, the transforms' BF16 rows (H1, G1) and the FP32 output; the
    spectral weights and modes (a few MB for the whole batch) stay in L2."""
    P, W, m = n * n, width, modes
    act = 2 * W * P                 # one BF16 activation field
    rows = 2 * W * n * 4 * m        # one BF16 H1 or G1 array
    lift = 4 * cin * P + act + rows
    mid = 2 * rows + act + act + rows       # along y reads H1, inverse writes G1; row kernel: h, G1 in; h, H1 out
    last = 2 * rows + act + 4 * 5 * P + 4 * 5 * P   # G1 written/read, h in, x[:5] in, y out
    return lift + (layers - 1) * mid + last


def initial_params(width=32, modes=12, layers=4, hidden=64, seed=0):
    """Seeded starting point for training, in the flat FP32 parameter order of
    sslbm_fno_set_params: dense maps uniform in +-1/sqrt(fan_in), spectral weights uniform
    in +-1/width^2, biases zero."""
    g = np.random.default_rng(seed)
    W, m, H = width, modes, hidden

    def dense(rows, cols):
        b = 1.0 / math.sqrt(cols)
        return g.uniform(-b, b, rows * cols)

    parts = [dense(W, 8), np.zeros(W)]
    for _ in range(layers):
        parts += [g.uniform(-1.0, 1.0, W * W * 2 * m * m * 2) / (W * W), dense(W, W), np.zeros(W)]
    parts += [dense(H, W), np.zeros(H), dense(5, H), np.zeros(5)]
    return np.concatenate(parts).astype(np.float32)


def scenario_specs(count, n, seed):
    sc = inputs.ensemble_scenarios(count, seed=seed, sizes=(n,))
    specs = [dict(nx=s["nx"], ny=s["ny"], rates=s["rates"].as_tuple(), d=s["d"]) for s in sc]
    r0 = np.array([s["R0"] for s in sc], dtype=np.float32)
    logd = np.array([math.log10(s["d"][0]) for s in sc], dtype=np.float32)
    return sc, specs, r0, logd


def snapshot_slots(trajectories, snapshots=10, horizon=2000, seed=7):
    """Stratified random snapshot times, in units of K_STEPS: the horizon is cut into
    `snapshots` equal strata of slots and each trajectory draws one slot from each, so
    the pairs cover the whole rollout window (the early exponential growth included)."""
    slots = horizon // K_STEPS
    per = slots // snapshots
    if per < 1:
        raise ValueError("horizon too short for this many snapshots")
    rng = inputs._rng(seed + 1)
    return np.arange(snapshots)[None, :] * per + rng.integers(0, per, (trajectories, snapshots))


def generate_pairs(n=256, trajectories=2000, snapshots=10, horizon=2000, seed=7, chunk=500):
    """Returns device tensors X, Y [pairs, 5, n, n] (float32) and per-pair r0, logd.  Pair
    (i, j) is trajectory i's state at step 20 * slot[i, j] and 20 steps later."""
    import torch
    sc, specs, r0, logd = scenario_specs(trajectories, n, seed)
    slot = snapshot_slots(trajectories, snapshots, horizon, seed)
    pairs = trajectories * snapshots
    X = torch.empty((pairs, 5, n, n), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    pr0 = torch.empty(pairs, dtype=torch.float32, device="cuda")
    plogd = torch.empty_like(pr0)
    last = int(slot.max()) + 1
    for c0 in range(0, trajectories, chunk):
        c1 = min(trajectories, c0 + chunk)
        ens = L.Ensemble(specs[c0:c1])
        ens.set_tiling(4, 64)
        for i in range(c0, c1):
            ens.write(i - c0, inputs.ensemble_state(sc[i]).astype(np.float32))
        for t in range(last + 1):
            if t:
                ens.run(K_STEPS)
            for i, j in zip(*np.nonzero(slot[c0:c1] == t)):
                L.sslbm_ensemble_read(ens.e, int(i), X[(c0 + i) * snapshots + j])
            for i, j in zip(*np.nonzero(slot[c0:c1] == t - 1)):
                L.sslbm_ensemble_read(ens.e, int(i), Y[(c0 + i) * snapshots + j])
        ens.close()
        idx = torch.arange(c0 * snapshots, c1 * snapshots, device="cuda")
        pr0[idx] = torch.from_numpy(np.repeat(r0[c0:c1], snapshots)).cuda()
        plogd[idx] = torch.from_numpy(np.repeat(logd[c0:c1], snapshots)).cuda()
    torch.cuda.synchronize()
    return X, Y, pr0, plogd


def train(sur, X, Y, r0, logd, steps=3000, batch=16, lr=1e-3, lr_min=1e-5, seed=0, val_frac=0.05,
          log_every=500, mass_weight=0.0, neg_weight=30.0, ramp=0.5):
    """Adam on random batches with a cosine learning-rate schedule; the loss is the scaled
    MSE plus the negative-mass term (and optionally the mass-residual term, which the
    network's conservation step makes redundant) of sslbm_fno_set_loss_weights, whose
    weights rise linearly from zero over the first `ramp` fraction of the steps, so the
    network learns the dynamics before it is held to the nonnegativity check; returns a
    history."""
    import torch
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    pairs = X.shape[0]
    nval = max(batch, int(pairs * val_frac))
    perm = torch.randperm(pairs, generator=g)
    val_idx, tr_idx = perm[:nval], perm[nval:]
    hist = {"loss": [], "val": []}
    t0 = time.perf_counter()
    for it in range(steps):
        sel = tr_idx[torch.randint(0, tr_idx.numel(), (batch,), generator=g)].cuda()
        x = sur.make_input(X[sel].contiguous(), r0[sel].contiguous(), logd[sel].contiguous())
        cur_lr = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * it / max(1, steps)))
        w = min(1.0, it / max(1.0, ramp * steps)) if ramp > 0 else 1.0
        sur.set_loss_weights(w * mass_weight, w * neg_weight)
        want = (it % log_every == 0) or it == steps - 1
        loss = sur.train_step(x, Y[sel].contiguous(), cur_lr, want_loss=want)
        if want:
            hist["loss"].append((it, loss))
    torch.cuda.synchronize()
    hist["train_seconds"] = time.perf_counter() - t0
    hist["val_mse"] = evaluate(sur, X, Y, r0, logd, val_idx, batch)
    # the do-nothing baseline (prediction = input) on the same validation pairs
    hist["val_mse_persistence"] = float(sum(((X[val_idx[i:i + batch]] - Y[val_idx[i:i + batch]]) ** 2).mean().item()
                                            * min(batch, nval - i) for i in range(0, nval, batch)) / nval)
    return hist


def evaluate(sur, X, Y, r0, logd, idx, batch):
    tot, cnt = 0.0, 0
    for i in range(0, idx.numel(), batch):
        sel = idx[i:i + batch].cuda()
        x = sur.make_input(X[sel].contiguous(), r0[sel].contiguous(), logd[sel].contiguous())
        y = sur.infer(x)
        tot += float(((y - Y[sel]) ** 2).mean().item()) * sel.numel()
        cnt += sel.numel()
    return tot / cnt


def rollout(sur, n=256, scenarios=64, steps=100, seed=11, threshold=1e-4, neg_threshold=0.0,
            reference=True, err_every=10, reach=0):
    """Surrogate rollout with residual checks and SSLBM fallback, run by the library's
    sslbm_surrogate_rollout in calls of err_every surrogate steps.  Returns timings, the
    fallback counts and (with reference=True) the error against an SSLBM ensemble advanced in
    lock step between the calls (the judge; not timed)."""
    import torch
    sc, specs, r0, logd = scenario_specs(scenarios, n, seed)
    u = torch.empty((scenarios, 5, n, n), dtype=torch.float32, device="cuda")
    for i, s in enumerate(sc):
        u[i].copy_(torch.from_numpy(inputs.ensemble_state(s).astype(np.float32)))
    tr0, tlogd = torch.from_numpy(r0).cuda(), torch.from_numpy(logd).cuda()
    xs = torch.empty((scenarios, 8, n, n), dtype=torch.float32, device="cuda")
    ys = torch.empty_like(u)
    fb = L.Ensemble(specs)          # runs the fallback steps
    fb.set_tiling(4, 64)
    ref = L.Ensemble(specs) if reference else None
    if ref is not None:
        ref.set_tiling(4, 64)
        for i in range(scenarios):
            L.sslbm_ensemble_write(ref.e, i, u[i])
    total0 = u.double().sum(dim=(1, 2, 3))
    tot = {"surrogate_steps": 0, "fallbacks": 0, "failed_conservation": 0, "failed_nonnegativity": 0,
           "max_mass_residual": 0.0, "max_neg_residual": 0.0}
    any_negative = 0
    t_sur = 0.0
    err_hist = []
    last_ref = None
    done = 0
    while done < steps:
        k = min(err_every, steps - done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, res, fell = L.sslbm_surrogate_rollout(sur.f, fb.e, scenarios, k, K_STEPS, u, tr0, tlogd, xs, ys,
                                                  threshold, neg_threshold, reach)
        torch.cuda.synchronize()
        t_sur += time.perf_counter() - t0
        for key in ("surrogate_steps", "fallbacks", "failed_conservation", "failed_nonnegativity"):
            tot[key] += st[key]
        for key in ("max_mass_residual", "max_neg_residual"):
            tot[key] = max(tot[key], st[key])
        any_negative += int((res[:, :, 1] > 0).sum())
        done += k
        if ref is not None:
            ref.run(K_STEPS * k)
            r = torch.empty_like(u)
            for i in range(scenarios):
                L.sslbm_ensemble_read(ref.e, i, r[i])
            d2 = ((u.double() - r.double()) ** 2).sum(dim=(0, 2, 3))
            rms = (d2 / (scenarios * n * n)).sqrt().cpu().numpy()
            rel = (d2 / (r.double() ** 2).sum(dim=(0, 2, 3))).sqrt().cpu().numpy()
            # the epidemic curves: each compartment's share of the population, per scenario
            fu = u.double().mean(dim=(2, 3)) / u.double().mean(dim=(2, 3)).sum(dim=1, keepdim=True)
            fr = r.double().mean(dim=(2, 3)) / r.double().mean(dim=(2, 3)).sum(dim=1, keepdim=True)
            frac = (fu - fr).abs()
            peak = (u[:, 2].amax(dim=(1, 2)).double() / r[:, 2].amax(dim=(1, 2)).double().clamp_min(1e-30) - 1).abs()
            err_hist.append({"step": done, "rms": rms.tolist(), "rel_l2": rel.tolist(),
                             "share_abs_err_mean": frac.mean(dim=0).cpu().numpy().tolist(),
                             "share_abs_err_max": frac.amax(dim=0).cpu().numpy().tolist(),
                             "peak_I_rel_err_median": float(peak.median())})
            last_ref = r
    drift = float(((u.double().sum(dim=(1, 2, 3)) - total0).abs() / total0).max())
    fb.close()
    if ref is not None:
        ref.close()
    return {"scenarios": scenarios, "surrogate_steps": steps, "sslbm_steps_equivalent": steps * K_STEPS,
            "seconds": t_sur, "scenario_steps_per_s": scenarios * steps * K_STEPS / t_sur,
            "fallbacks": tot["fallbacks"], "fallback_rate": tot["fallbacks"] / (scenarios * steps),
            "failed_conservation": tot["failed_conservation"], "failed_nonnegativity": tot["failed_nonnegativity"],
            "max_mass_residual": tot["max_mass_residual"], "max_neg_residual": tot["max_neg_residual"],
            "scenario_steps_with_any_negative": any_negative, "thresholds": [threshold, neg_threshold],
            "rms_error_vs_sslbm": err_hist, "max_population_drift": drift,
            "min_value": float(u.min()), "state": u, "reference_state": last_ref}


def fp64_batched_scenario_steps_per_s(n=256, scenarios=64, steps=20, seed=11):
    """Plain FP64 SSLBM on the rollout's batch: one solver per scenario (the same scenarios,
    n x n periodic), all on one stream, each advanced `steps` lattice steps per timed round."""
    import torch
    sc, specs, _, _ = scenario_specs(scenarios, n, seed)
    solvers = [L.Solver(n, n, sp["rates"], d=sp["d"], bc=L.BC_PERIODIC, precision=L.FP64) for sp in specs]
    for s, c in zip(solvers, sc):
        s.write(inputs.ensemble_state(c))
    for s in solvers:
        s.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in solvers:
        s.step(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for s in solvers:
        s.close()
    return scenarios * steps / dt


def fp32_ensemble_scenario_steps_per_s(n=256, scenarios=64, steps=2000, seed=11):
    """The FP32 SSLBM ensemble (one persistent launch per run) on the rollout's batch."""
    import torch
    sc, specs, _, _ = scenario_specs(scenarios, n, seed)
    ens = L.Ensemble(specs)
    ens.set_tiling(4, 64)
    for i, c in enumerate(sc):
        ens.write(i, inputs.ensemble_state(c).astype(np.float32))
    ens.run(K_STEPS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens.run(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ens.close()
    return scenarios * steps / dt


def fp64_scenario_steps_per_s(n=256, steps=40, seed=11):
    """Plain FP64 SSLBM on one n x n scenario (the baseline the surrogate is compared with)."""
    import torch
    sc, specs, _, _ = scenario_specs(1, n, seed)
    s = L.Solver(n, n, specs[0]["rates"], d=specs[0]["d"], bc=L.BC_PERIODIC, precision=L.FP64)
    s.write(inputs.ensemble_state(sc[0]))
    s.step(4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return steps / dt
