"""The D2Q9 SSLBM step on the GPU against the FP64 oracle (oracle.sslbm9_run).

The kernel evaluates the reduced form rho_c + d (4 axes + diagonals - 20 rho_c)/6 + Psi dt;
the oracle keeps the literal rho_b + (tau - 1)(rho_f - 2 rho_c + rho_b); they differ by a
few roundings per step (FP64: 1e-12 relative max-norm over 25 steps, as for D2Q5).  FP32:
each step adds a few FP32 roundings (u = 6e-8) of a contractive update; 25 steps stay
within 1e-5 of the peak.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

RATES = inputs.rates_from_sigma_mu(0.45, 0.2, 0.1, 0.01).as_tuple()
D = (0.05, 0.04, 0.01, 0.08, 0.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def relmax(a, b):
    return max(float(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-300)) for c in range(5))


def _run(nx, ny, bc, precision, steps, state):
    s = L.Solver(nx, ny, RATES, d=D, bc=bc, precision=precision, lattice=L.LATTICE_D2Q9)
    s.write(state if precision == L.FP64 else state.astype(np.float32))
    s.step(steps)
    out = s.read()
    tot, _ = s.diagnostics()
    s.close()
    return out, tot


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(37, 29), (70, 41), (1, 5), (6, 1), (2, 3)])
def test_fp64_matches_oracle(bc, nx, ny):
    st = inputs.epidemic_state(nx, ny, 3 * nx + ny)
    got, tot = _run(nx, ny, bc, L.FP64, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.sslbm9_run(st, tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-12
    # the population is conserved (FP64 diagnostics)
    assert abs(tot.sum() - st.sum()) / st.sum() < 1e-12


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_fp32_matches_oracle(bc):
    st = inputs.epidemic_state(45, 38, 11)
    got, _ = _run(45, 38, bc, L.FP32, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.sslbm9_run(st.astype(np.float32).astype(np.float64), tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-5


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(301, 19), (513, 10), (128, 9), (1, 7), (2, 3), (5, 1)])
def test_fp32_rows_span_warps_and_ragged_tails(bc, nx, ny):
    """A warp covers 32 groups of a row: these widths put the warp's last lane, a ragged last
    group and single-group rows at every kind of edge (periodic wrap and walls)."""
    st = inputs.epidemic_state(nx, ny, 5 * nx + ny)
    got, _ = _run(nx, ny, bc, L.FP32, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.sslbm9_run(st.astype(np.float32).astype(np.float64), tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-5


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_fp64_wide_rows(bc):
    st = inputs.epidemic_state(263, 17, 9)
    got, _ = _run(263, 17, bc, L.FP64, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    assert relmax(got, oracle.sslbm9_run(st, tau, RATES, 1.0, bc, 25)) <= 1e-12


def test_stability_range_and_what_it_does_not_run():
    # tau = 1.5 (d = 1/3) is stable on D2Q9 (<= 13/8) and not on D2Q5 (<= 5/4)
    s = L.Solver(8, 8, RATES, d=(1 / 3, 0.05, 0.05, 0.05, 0.0), lattice=L.LATTICE_D2Q9)
    s.close()
    with pytest.raises(L.SslbmError) as e:
        L.Solver(8, 8, RATES, d=(1 / 3, 0.05, 0.05, 0.05, 0.0))
    assert e.value.status == L.SSLBM_ERR_UNSTABLE
    with pytest.raises(L.SslbmError) as e:
        L.Solver(8, 8, RATES, d=D, lattice=L.LATTICE_D2Q9, schemes=L.WANT_SSLBM | L.WANT_BGK)
    assert e.value.status == L.SSLBM_ERR_UNSUPPORTED
    with pytest.raises(L.SslbmError):
        L.Solver(8, 8, RATES, d=D, lattice=L.LATTICE_D2Q9, precision=L.FP32_DEV)
    s = L.Solver(64, 64, RATES, d=D, lattice=L.LATTICE_D2Q9, precision=L.FP32)
    with pytest.raises(L.SslbmError) as e:
        s.set_blocking(4)
    assert e.value.status == L.SSLBM_ERR_UNSUPPORTED
    s.close()
