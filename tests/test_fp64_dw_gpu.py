"""The FP64-accurate double-word storage (SSLBM_FP64_DW) against the FP64 oracle.

Each value is hi + lo of two floats.  The update runs in double-word arithmetic: the
building blocks of Joldes, Muller and Popescu (ACM TOMS 2017), written in dword.cuh.

Tolerance: FP64's bar, 1e-12 relative max-norm per compartment.  A double-word operation's
relative error is of order u^2 = 2^-48 (bounds 3u^2 to 15u^2) rather than FP64's 2^-53.  So
2000 steps at a few 1e-14 per step at most stay below the bar, and in practice far below it,
since the rounding errors do not add up coherently.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def rel_max(a, b):
    out = []
    for c in range(a.shape[0]):
        den = np.abs(b[c]).max()
        num = np.abs(a[c] - b[c]).max()
        out.append(num / den if den > 0 else num)
    return np.array(out)


def taus(wl):
    return [oracle.tau_from_d(v, wl.get("dx", 1.0), wl.get("dt", 1.0)) for v in wl["d"][:4]]


def solver(wl, precision=L.FP64_DW):
    _, ny, nx = wl["state"].shape
    return L.Solver(nx, ny, wl["rates"].as_tuple(), d=wl["d"], dx=wl.get("dx", 1.0), dt=wl.get("dt", 1.0),
                    bc=wl["bc"], precision=precision)


def small_workload(nx, ny, bc, seed=1):
    st = inputs.epidemic_state(nx, ny, seed)
    return dict(state=st, rates=inputs.Rates(0.5, 0.2, 0.11, 1 / 11), d=(0.05, 0.05, 0.01, 0.05, 0.0), bc=bc)


def test_centre_bump_matches_the_oracle_2000_steps():
    """Errors are divided by each compartment's peak over the run.  After the wave, E and I
    decay below FP32's smallest normal number (1.2e-38), where a double word of floats has
    no more precision and FP64 keeps decaying, so their final maximum is no scale to
    measure against."""
    wl = inputs.centre_bump_workload()
    s = solver(wl)
    s.write(wl["state"])
    ref = wl["state"]
    tau, rates = taus(wl), wl["rates"].as_tuple()
    got, want, done = {}, {}, 0
    for t in (100, 300, 1000, wl["steps"]):
        s.step(t - done)
        ref = oracle.sslbm_run(ref, tau, rates, 1.0, wl["bc"], t - done)
        done = t
        got[t], want[t] = s.read(), ref
    peak = np.max([np.abs(w).reshape(5, -1).max(axis=1) for w in want.values()], axis=0)
    for t in got:
        err = np.abs(got[t] - want[t]).reshape(5, -1).max(axis=1) / peak
        print(f"double-word t={t}: max-norm error / peak per compartment {err}")
        assert (err <= TOL).all(), (t, err)
    tot, pk = s.diagnostics()
    otot, opk = oracle.diagnostics(want[wl["steps"]])
    t0 = oracle.diagnostics(wl["state"])[0].sum()
    np.testing.assert_allclose(tot, otot, rtol=TOL, atol=TOL * t0)
    assert abs(tot.sum() - t0) / t0 < TOL


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (9, 1), (2, 3), (37, 23), (65, 40), (130, 67), (257, 5)])
def test_ragged_grids(nx, ny, bc):
    wl = small_workload(nx, ny, bc, seed=nx * 7 + ny)
    s = solver(wl)
    s.write(wl["state"])
    s.step(40)
    want = oracle.sslbm_run(wl["state"], taus(wl), wl["rates"].as_tuple(), 1.0, bc, 40)
    err = rel_max(s.read(), want)
    assert (err <= TOL).all(), err


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_paper_case_in_physical_units(bc):
    """Sec. III's case: tau = 0.501305 and 0.500003, densities of order 100 per km^2."""
    wl = inputs.paper_test_case(bc=bc)
    s = solver(wl)
    s.write(wl["state"])
    s.step(2000)
    want = oracle.sslbm_run(wl["state"], taus(wl), wl["rates"].as_tuple(), wl["dt"], bc, 2000)
    err = rel_max(s.read(), want)
    print("double-word, physical units, rel max-norm:", err)
    assert (err <= TOL).all(), err
    tot, _ = s.diagnostics()
    assert abs(tot.sum() - 5e6) / 5e6 < TOL


def test_far_more_accurate_than_fp32_storage():
    wl = small_workload(96, 64, 1, seed=4)
    want = oracle.sslbm_run(wl["state"], taus(wl), wl["rates"].as_tuple(), 1.0, 1, 300)
    errs = {}
    for prec in (L.FP64_DW, L.FP32):
        s = solver(wl, prec)
        s.write(wl["state"])
        s.step(300)
        errs[prec] = rel_max(s.read(), want).max()
    assert errs[L.FP64_DW] < 1e-5 * errs[L.FP32], errs


def test_write_read_round_trip_keeps_double_word_precision():
    wl = small_workload(70, 33, 0, seed=9)
    s = solver(wl)
    s.write(wl["state"])
    back = s.read()
    # hi = fl32(x), lo = fl32(x - hi): |hi + lo - x| <= 2^-48 |x|
    assert (np.abs(back - wl["state"]) <= 2.0 ** -48 * np.abs(wl["state"])).all()


def test_checkpoint_resume_gives_the_same_bits():
    wl = small_workload(120, 50, 1, seed=12)
    s = solver(wl)
    s.write(wl["state"])
    s.step(30)
    ck = s.checkpoint()
    s.step(20)
    a = s.checkpoint()
    s.restore(ck)
    s.step(20)
    assert np.array_equal(a, s.checkpoint())


def test_one_step_per_launch_only():
    wl = small_workload(64, 32, 0)
    s = solver(wl)
    with pytest.raises(L.SslbmError) as ei:
        s.set_blocking(2)
    assert ei.value.status == L.SSLBM_ERR_UNSUPPORTED
    s.write(wl["state"])
    depth, seg, _ = s.autotune(20.0)
    assert depth == 1
