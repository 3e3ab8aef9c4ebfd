"""The learned surrogate end to end on small grids: trajectories generated by the ensemble
kernel, training by the library's own forward/backward/Adam kernels, and the rollout with
residual checks and SSLBM fallback (the library's sslbm_surrogate_rollout), judged by the SSLBM.

What the trained network gains over the method without it: the plain SSLBM needs 20
lattice steps where the network takes one forward pass.  These tests check the accuracy
side of that trade on a 64 x 64 configuration (the throughput side is measured at 256 x 256
by the surrogate study): the trained network predicts the 20-step map far better than the
do-nothing (persistence) predictor, and its rollout stays nonnegative, conserves the
population and tracks the SSLBM.  With every check forced to fail the rollout is the SSLBM
itself, bit for bit; a scenario whose prediction fails falls back alone.
"""
import numpy as np
import pytest

from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

N = 64
CFG = dict(width=16, modes=8, layers=2, hidden=32)


@pytest.fixture(scope="module")
def trained():
    from paper_2603_19789_gb300 import build
    from paper_2603_19789_gb300 import surrogate as S
    build.build()
    L.load()
    X, Y, r0, logd = S.generate_pairs(n=N, trajectories=64, snapshots=6, horizon=240, seed=3, chunk=64)
    sur = L.Surrogate(n=N, max_batch=16, **CFG)
    sur.set_params(S.initial_params(CFG["width"], CFG["modes"], CFG["layers"], CFG["hidden"], seed=0))
    hist0 = S.evaluate(sur, X, Y, r0, logd, _val_idx(X.shape[0]), 8)
    hist = S.train(sur, X, Y, r0, logd, steps=2000, batch=8, lr=1e-3, seed=0, neg_weight=30.0)
    return S, sur, X, Y, r0, logd, hist0, hist


def _val_idx(pairs, batch=8, val_frac=0.05, seed=0):
    import torch
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    nval = max(batch, int(pairs * val_frac))
    return torch.randperm(pairs, generator=g)[:nval]


def test_training_data_are_sslbm_trajectories():
    """Each pair (X, Y) is the single-scenario SSLBM solver's state at its snapshot time and
    20 steps later; snapshot times cover each stratum of the horizon once."""
    import torch
    from paper_2603_19789_gb300 import build, inputs
    from paper_2603_19789_gb300 import surrogate as S
    build.build()
    X, Y, r0, logd = S.generate_pairs(n=N, trajectories=3, snapshots=2, horizon=120, seed=5, chunk=3)
    slot = S.snapshot_slots(3, 2, 120, 5)
    assert ((slot[:, 0] >= 0) & (slot[:, 0] < 3) & (slot[:, 1] >= 3) & (slot[:, 1] < 6)).all()
    sc, specs, _, _ = S.scenario_specs(3, N, 5)
    for i in range(3):
        s = L.Solver(N, N, specs[i]["rates"], d=specs[i]["d"], bc=L.BC_PERIODIC, precision=L.FP32)
        s.write(inputs.ensemble_state(sc[i]).astype(np.float32))
        t = 0
        for j in range(2):
            s.step(20 * int(slot[i, j]) - t)
            np.testing.assert_array_equal(s.read(dtype=np.float32), X[2 * i + j].cpu().numpy())
            s.step(20)
            t = 20 * int(slot[i, j]) + 20
            np.testing.assert_array_equal(s.read(dtype=np.float32), Y[2 * i + j].cpu().numpy())
        s.close()
    assert torch.allclose(r0[::2], torch.from_numpy(np.array([q["R0"] for q in sc], np.float32)).cuda())


def test_trained_network_beats_persistence(trained):
    S, sur, X, Y, r0, logd, mse0, hist = trained
    # the network learned the 20-step map: its validation error is well below that of
    # predicting "no change" and below the untrained network's
    assert hist["val_mse"] < 0.7 * hist["val_mse_persistence"], hist
    assert hist["val_mse"] < mse0


def test_rollout_conserves_and_tracks_sslbm(trained):
    S, sur, *_ = trained
    out = S.rollout(sur, n=N, scenarios=8, steps=10, seed=11, err_every=5)
    u, ref = out["state"], out["reference_state"]
    assert out["min_value"] >= 0.0
    assert out["max_population_drift"] < 1e-4
    assert np.isfinite(out["rms_error_vs_sslbm"][-1]["rms"]).all()
    # the rollout tracks the SSLBM better than the initial state does (the do-nothing rollout)
    sc, _, _, _ = S.scenario_specs(8, N, 11)
    u0 = np.stack([S.inputs.ensemble_state(s) for s in sc]).astype(np.float32)
    r = ref.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(u.cpu().numpy() - r)
    err_still = np.linalg.norm(u0 - r)
    assert err < 0.5 * err_still, (err, err_still, out["fallbacks"])


def test_forced_fallback_is_the_sslbm(trained):
    """With the checks forced to fail every step, the rollout is the SSLBM bit for bit."""
    S, sur, *_ = trained
    out = S.rollout(sur, n=N, scenarios=4, steps=3, seed=13, threshold=-1.0, err_every=1)
    assert out["fallbacks"] == 4 * 3
    np.testing.assert_array_equal(out["state"].cpu().numpy(), out["reference_state"].cpu().numpy())


def _rollout_setup(S, scenarios, seed):
    import torch
    sc, specs, r0, logd = S.scenario_specs(scenarios, N, seed)
    u = torch.stack([torch.from_numpy(S.inputs.ensemble_state(s).astype(np.float32)) for s in sc]).cuda()
    xs = torch.empty((scenarios, 8, N, N), dtype=torch.float32, device="cuda")
    ys = torch.empty_like(u)
    return sc, specs, u, torch.from_numpy(r0).cuda(), torch.from_numpy(logd).cuda(), xs, ys


def test_rollout_call_falls_back_only_where_a_check_fails(trained):
    """Through the C ABI: a scenario whose network input is not finite (R0 = NaN) fails both
    checks at every step and so follows the SSLBM bit for bit, while the others keep the
    network's predictions, the same as in a rollout where no scenario failed; the
    per-step residuals and fallback flags agree with the returned totals."""
    import torch
    S, sur, *_ = trained
    steps, bad = 4, 2
    sc, specs, u0, r0, logd, xs, ys = _rollout_setup(S, 4, 17)
    ok = L.Ensemble(specs)
    ok.set_tiling(4, 16)
    u_ok = u0.clone()
    st_ok, res_ok, fb_ok = L.sslbm_surrogate_rollout(sur.f, ok.e, 4, steps, S.K_STEPS, u_ok, r0, logd, xs, ys,
                                                     1e-4, 0.0, 0)
    assert st_ok["fallbacks"] == 0 and not fb_ok.any()
    assert st_ok["surrogate_steps"] == 4 * steps
    assert (res_ok[:, :, 0] <= 1e-4).all() and (res_ok[:, :, 1] == 0.0).all()  # nonnegative by construction
    r0_bad = r0.clone()
    r0_bad[bad] = float("nan")
    fb = L.Ensemble(specs)
    fb.set_tiling(4, 16)
    u = u0.clone()
    st, res, fell = L.sslbm_surrogate_rollout(sur.f, fb.e, 4, steps, S.K_STEPS, u, r0_bad, logd, xs, ys,
                                              1e-4, 0.0, 0)
    assert fell[:, bad].all() and not np.delete(fell, bad, axis=1).any()
    assert np.isinf(res[:, bad]).all()
    assert st["fallbacks"] == steps and st["surrogate_steps"] == 3 * steps
    assert st["failed_conservation"] == steps and st["failed_nonnegativity"] == steps
    others = [i for i in range(4) if i != bad]
    # the same predictions (up to the order of the FP64 atomic sums of the conservation step)
    torch.testing.assert_close(u[others], u_ok[others], rtol=1e-6, atol=0)
    # the failing scenario is the SSLBM run alone
    ref = L.Ensemble(specs[bad:bad + 1])
    ref.set_tiling(4, 16)
    L.sslbm_ensemble_write(ref.e, 0, u0[bad])
    ref.run(S.K_STEPS * steps)
    want = torch.empty_like(u0[bad])
    L.sslbm_ensemble_read(ref.e, 0, want)
    assert torch.equal(u[bad], want)
    for e in (ok, fb, ref):
        e.close()


def test_rollout_call_rejects_a_mismatched_fallback_ensemble(trained):
    S, sur, *_ = trained
    sc, specs, u0, r0, logd, xs, ys = _rollout_setup(S, 2, 19)
    small = L.Ensemble(specs[:1])
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_surrogate_rollout(sur.f, small.e, 2, 1, S.K_STEPS, u0, r0, logd, xs, ys)
    assert ei.value.status == L.SSLBM_ERR_BAD_ARG
    other = L.Ensemble([dict(specs[0], nx=N // 2, ny=N // 2), specs[1]])
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_surrogate_rollout(sur.f, other.e, 2, 1, S.K_STEPS, u0, r0, logd, xs, ys)
    assert ei.value.status == L.SSLBM_ERR_BAD_ARG
    small.close()
    other.close()
