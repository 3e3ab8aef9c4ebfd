"""Parity in the paper's own units: the test case of Sec. III (200 x 200 km^2, N = 5e6,
dx = 1 km, dt = 0.01 day, gamma = 1/5, beta = R0 gamma with R0 = 3, alpha = 1/7, phi = 0.3,
d^{S,E,R} = 4.35e-2 km^2/day, d^I = 1e-4 km^2/day; inputs.paper_test_case).

Here the host converts d to tau with Eq. (diffusivity), tau = 3 d dt / dx^2 + 1/2, which
gives tau = 0.501305 for S, E, R and 0.500003 for I (the regime right above the stability
limit tau = 1/2), and every rate enters as rate * dt.  The lattice-unit tests (dx = dt = 1,
tau in 0.53..0.65) never exercise either.  The oracle receives tau from its own conversion
(oracle.tau_from_d) and dt; the library receives d, dx and dt.

Tolerances: FP64 relative max-norm <= 1e-12 per compartment (as in test_parity_gpu.py);
FP32 variants, errors divided by the compartment's peak over the run, <= 2e-4 (n u for
n = 2000 steps); the deviation storage holds S against s_ref = N/A.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-4
STEPS = 2000  # 20 days


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def _taus(wl):
    return [oracle.tau_from_d(v, wl["dx"], wl["dt"]) for v in wl["d"][:4]]


def _solver(wl, precision, schemes=L.WANT_SSLBM, s_ref=1.0):
    _, ny, nx = wl["state"].shape
    return L.Solver(nx, ny, wl["rates"].as_tuple(), d=wl["d"], dx=wl["dx"], dt=wl["dt"], bc=wl["bc"],
                    precision=precision, schemes=schemes, s_ref=s_ref)


def _rel_max(a, b):
    return np.array([np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() if np.abs(b[c]).max() > 0
                     else np.abs(a[c] - b[c]).max() for c in range(5)])


def test_relaxation_times_of_the_paper_case():
    wl = inputs.paper_test_case()
    tau = _taus(wl)
    np.testing.assert_allclose(tau, [0.501305, 0.501305, 0.500003, 0.501305], rtol=0, atol=1e-12)


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_sslbm_fp64_matches_oracle_in_physical_units(bc):
    wl = inputs.paper_test_case(bc=bc)
    s = _solver(wl, L.FP64)
    s.write(wl["state"])
    s.step(STEPS)
    got = s.read()
    want = oracle.sslbm_run(wl["state"], _taus(wl), wl["rates"].as_tuple(), wl["dt"], bc, STEPS)
    err = _rel_max(got, want)
    print("FP64 rel max-norm per compartment:", err)
    assert (err <= FP64_TOL).all(), err
    # the epidemic moved: I, R and D grew from zero, so the rates and dt entered
    assert want[2].max() > 1.0 and want[3].max() > 1.0 and want[4].max() > 0.1
    tot, _ = s.diagnostics()
    n_total = 5e6
    assert abs(tot.sum() - n_total) / n_total < 1e-13


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_bgk_fp64_matches_oracle_in_physical_units(bc):
    wl = inputs.paper_test_case(bc=bc)
    s = _solver(wl, L.FP64, schemes=L.WANT_BGK)
    s.write(wl["state"], scheme=L.SCHEME_BGK)
    s.bgk_step(500)
    got = s.read(scheme=L.SCHEME_BGK)
    want = oracle.bgk_run_state(wl["state"], _taus(wl), wl["rates"].as_tuple(), wl["dt"], bc, 500)
    err = _rel_max(got, want)
    print("BGK FP64 rel max-norm per compartment:", err)
    assert (err <= FP64_TOL).all(), err


@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_KAHAN, L.FP32_SPLIT])
def test_fp32_variants_in_physical_units(precision):
    wl = inputs.paper_test_case(bc=L.BC_NOFLUX)
    s = _solver(wl, precision, s_ref=wl["density"])
    s.write(wl["state"])
    tau, rates = _taus(wl), wl["rates"].as_tuple()
    ref = wl["state"]
    done = 0
    got, want = {}, {}
    for t in (200, STEPS):
        s.step(t - done)
        ref = oracle.sslbm_run(ref, tau, rates, wl["dt"], wl["bc"], t - done)
        done = t
        got[t], want[t] = s.read(), ref
    peak = np.max([np.abs(w).reshape(5, -1).max(axis=1) for w in want.values()], axis=0)
    for t in got:
        diff = (got[t] - want[t]).reshape(5, -1)
        einf = np.abs(diff).max(axis=1) / peak
        e2 = np.sqrt((diff ** 2).mean(axis=1)) / peak
        print(f"precision {precision} t={t}: rel-to-peak L2 {e2}, Linf {einf}")
        assert (e2 <= FP32_TOL).all() and (einf <= FP32_TOL).all(), (t, e2, einf)


@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_SPLIT])
def test_blocked_kernel_gives_one_step_bits_near_tau_one_half(precision):
    """With tau - 1/2 of 1e-3 and 3e-6 the update's diffusion weight is tiny; every blocking
    depth must still give the bits of the one-step kernel."""
    wl = inputs.paper_test_case(side_km=96, bc=L.BC_NOFLUX)
    ref = _solver(wl, precision, s_ref=wl["density"])
    ref.write(wl["state"])
    ref.set_blocking(1)
    ref.step(16)
    base = ref.checkpoint()[128:]  # every stored plane, as stored
    for k in (2, 4, 8):
        s = _solver(wl, precision, s_ref=wl["density"])
        s.write(wl["state"])
        s.set_blocking(k)
        s.step(16)
        assert np.array_equal(s.checkpoint()[128:], base), k
