"""The persistent ensemble launch against the single-grid solver and the oracle.

Every scenario of an ensemble must give the same bits as a single-grid solver of the same
storage (FP32, FP32 deviation-S, FP32 split-S) with the same parameters (one-step kernel),
and agree with the FP64 oracle to FP32 accuracy.  The bounded dependency waits are exercised by a host-side fault injection:
one work item never reports completion, so the waits behind it run out and the run
returns SSLBM_ERR_TIMEOUT; the GPU stays usable afterwards.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


SIZES = [(64, 64), (128, 96), (132, 40), (256, 256), (4, 7), (520, 130), (12, 300)]


def _specs(seed=3):
    g = np.random.default_rng(seed)
    out = []
    for nx, ny in SIZES:
        R0 = g.uniform(1.2, 4.0)
        d = 10 ** g.uniform(-3, -1)
        r = inputs.rates_from_sigma_mu(R0 * 0.11, 0.2, 0.1, 0.01)
        out.append(dict(nx=nx, ny=ny, rates=r.as_tuple(), d=(d, d, d, d, 0.0)))
    return out


def _states(specs, seed=5):
    return [inputs.epidemic_state(sp["nx"], sp["ny"], seed + i) for i, sp in enumerate(specs)]


def _single(sp, st, n, precision=L.FP32):
    s = L.Solver(sp["nx"], sp["ny"], sp["rates"], d=sp["d"], bc=L.BC_PERIODIC, precision=precision)
    s.write(st)
    s.set_blocking(1)
    s.step(n)
    out = s.read(dtype=np.float32)
    s.close()
    return out


@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_SPLIT])
@pytest.mark.parametrize("depth,seg", [(4, 64), (2, 16), (3, 12), (8, 32), (6, 256)])
def test_ensemble_matches_single_grid_bits(precision, depth, seg):
    specs = _specs()
    states = _states(specs)
    ens = L.Ensemble(specs, precision=precision)
    ens.set_tiling(depth, seg)
    for i, st in enumerate(states):
        ens.write(i, st)
    nsteps = 3 * depth + 1  # full step-blocks plus a remainder step
    ens.run(nsteps - 4)
    ens.run(4)  # a second run; for depth 6 and 8 the first one ends in several one-step launches
    for i, (sp, st) in enumerate(zip(specs, states)):
        got = ens.read(i, dtype=np.float32)
        ref = _single(sp, st, nsteps, precision)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (i, sp["nx"], sp["ny"])
    ens.close()


def test_ensemble_matches_oracle_and_diagnostics():
    specs = _specs(seed=11)
    states = _states(specs, seed=2)
    ens = L.Ensemble(specs)
    for i, st in enumerate(states):
        ens.write(i, st)
    ens.run(9)
    ens.run(11)  # a second run continues from the first (graph re-captured for 11 steps)
    tot, pk = ens.diagnostics()
    for i, (sp, st) in enumerate(zip(specs, states)):
        tau = [oracle.tau_from_d(v) for v in sp["d"][:4]]
        want = oracle.sslbm_run(st, tau, sp["rates"], 1.0, 0, 20)
        got = ens.read(i)
        for c in range(5):
            scale = np.abs(want[c]).max()
            assert np.abs(got[c] - want[c]).max() <= 1e-5 * scale, (i, c)
        otot, opk = oracle.diagnostics(got)
        np.testing.assert_allclose(tot[i], otot, rtol=1e-12)
        assert pk[i] == pytest.approx(opk, rel=1e-7)
    ens.close()


def test_ensemble_autotune_then_run():
    specs = _specs(seed=4)
    states = _states(specs, seed=9)
    ens = L.Ensemble(specs)
    depth, seg, ms = ens.autotune(trial_blocks=2)
    assert depth in (2, 3, 4, 6, 8) and seg in (32, 64, 128, 256) and ms > 0
    assert ens.get_tiling() == (depth, seg)
    for i, st in enumerate(states):
        ens.write(i, st)
    ens.run(10)
    for i, (sp, st) in enumerate(zip(specs, states)):
        ref = _single(sp, st, 10)
        assert np.array_equal(ens.read(i, dtype=np.float32).view(np.uint32), ref.view(np.uint32))
    ens.close()


def test_lost_completion_times_out_instead_of_hanging():
    specs = _specs(seed=6)
    states = _states(specs)
    ens = L.Ensemble(specs)
    ens.set_tiling(4, 64)
    for i, st in enumerate(states):
        ens.write(i, st)
    # item 0 (block 0, scenario 0, tile 0) never reports completion: every tile of
    # scenario 0 in block 1 waits on it and must give up after the spin limit
    ens.set_wait_limit(20000, stall_item=0)
    with pytest.raises(L.SslbmError) as ei:
        ens.run(12)
    assert ei.value.status == -4
    # the context is still usable
    ens.set_wait_limit(1 << 24, stall_item=-1)
    for i, st in enumerate(states):
        ens.write(i, st)
    ens.run(8)
    ref = _single(specs[0], states[0], 8)
    assert np.array_equal(ens.read(0, dtype=np.float32).view(np.uint32), ref.view(np.uint32))
    ens.close()


def test_ensemble_rejects_what_it_does_not_run():
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_ensemble_workspace_bytes(L.make_scenarios([dict(nx=10, ny=8, rates=(0.3, 0.2, 0.1, 0.1),
                                                                d=(0.05,) * 4)]))
    assert ei.value.status == -1  # nx not a multiple of 4
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_ensemble_workspace_bytes(L.make_scenarios([dict(nx=8, ny=8, rates=(0.3, 0.2, 0.1, 0.1),
                                                                d=(0.3,) * 4)]))
    assert ei.value.status == -2  # tau > 5/4
    with pytest.raises(L.SslbmError):
        L.sslbm_ensemble_workspace_bytes(L.make_scenarios([dict(nx=8, ny=8, rates=(0.3, 0.2, 0.1, 0.1),
                                                                d=(0.05,) * 4)]), precision=L.FP64)


def test_split_ensemble_diagnostics_and_accuracy():
    """The split storage of S in the ensemble: totals as the single-grid split solver reports
    them (value - compensation), and S after 400 steps of a small-seed epidemic closer to the
    FP64 oracle than plain FP32's."""
    specs = _specs(seed=11)[:3]
    states = [inputs.epidemic_state(sp["nx"], sp["ny"], 70 + i) for i, sp in enumerate(specs)]
    errs = {}
    for prec in (L.FP32, L.FP32_SPLIT):
        ens = L.Ensemble(specs, precision=prec)
        ens.set_tiling(4, 32)
        for i, st in enumerate(states):
            ens.write(i, st)
        ens.run(400)
        tot, _ = ens.diagnostics()
        worst = 0.0
        for i, (sp, st) in enumerate(zip(specs, states)):
            got = ens.read(i)
            s = L.Solver(sp["nx"], sp["ny"], sp["rates"], d=sp["d"], bc=L.BC_PERIODIC, precision=prec)
            s.write(st)
            s.step(400)
            stot, _ = s.diagnostics()
            s.close()
            assert np.array_equal(tot[i], stot), (prec, i)
            taus = [oracle.tau_from_d(x) for x in sp["d"][:4]]
            ref = oracle.sslbm_run(st.astype(np.float32).astype(np.float64), taus, sp["rates"], 1.0,
                                   L.BC_PERIODIC, 400)
            worst = max(worst, float(np.abs(got[0] - ref[0]).max()))
        errs[prec] = worst
        ens.close()
    assert errs[L.FP32_SPLIT] <= errs[L.FP32], errs
