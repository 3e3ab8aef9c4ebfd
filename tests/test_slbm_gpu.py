"""The two-pass SLBM (grid lattice SSLBM_LATTICE_D2Q5_SLBM) on the GPU against the FP64
oracle (oracle.slbm_run).

The kernels evaluate the predictor as rho + lap5(rho)/6 and the corrector's neighbour sum
as rho* + lap5(rho*)/6, the oracle the weighted sums of Eqs. (SLBM1, SLBM2) term by term;
the two orderings differ by a few roundings per step (FP64: 1e-12 relative max-norm over
25 steps).  FP32: a few FP32 roundings per step of a contractive update, 1e-5 of the peak.
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
    s = L.Solver(nx, ny, RATES, d=D, bc=bc, precision=precision, lattice=L.LATTICE_D2Q5_SLBM)
    s.write(state if precision == L.FP64 else state.astype(np.float32))
    s.step(steps)
    out = s.read()
    tot, _ = s.diagnostics()
    s.close()
    return out, tot


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(37, 29), (70, 41), (1, 5), (6, 1), (263, 17)])
def test_fp64_matches_oracle(bc, nx, ny):
    st = inputs.epidemic_state(nx, ny, 5 * nx + ny)
    got, tot = _run(nx, ny, bc, L.FP64, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.slbm_run(st, tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-12
    assert abs(tot.sum() - st.sum()) / st.sum() < 1e-12


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(45, 38), (301, 19), (513, 10), (128, 9), (2, 3), (5, 1)])
def test_fp32_matches_oracle(bc, nx, ny):
    """Rows of several thread groups of 4 cells and ragged last groups, at every kind of edge."""
    st = inputs.epidemic_state(nx, ny, 17 + nx)
    got, _ = _run(nx, ny, bc, L.FP32, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.slbm_run(st.astype(np.float32).astype(np.float64), tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-5


def test_stability_range():
    # tau = 1.7 (d = 0.4) is stable for the two-pass SLBM (<= 7/4) and not for the SSLBM (<= 5/4)
    s = L.Solver(8, 8, RATES, d=(0.4, 0.05, 0.05, 0.05, 0.0), lattice=L.LATTICE_D2Q5_SLBM)
    s.close()
    with pytest.raises(L.SslbmError) as e:
        L.Solver(8, 8, RATES, d=(0.4, 0.05, 0.05, 0.05, 0.0))
    assert e.value.status == L.SSLBM_ERR_UNSTABLE
