"""The fourth-order finite-difference reference on the GPU (sslbm_fd4_*) against the FP64
oracle's fd4_rk4_run, and its second-order variant against fd2_rk4_run.

The kernels evaluate every operation in the oracle's order with one rounding each (no
contraction) and IEEE division, so FP64 agrees to the last bit up to the order of nothing
at all; the test allows 1e-15 relative.  FP32 keeps the same order in single precision:
over 12 RK4 steps of a contractive stencil the error stays within a few hundred FP32
roundings of the field's peak (2e-5 relative max-norm, per compartment).
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

RATES = inputs.rates_from_sigma_mu(0.45, 0.2, 0.1, 0.01).as_tuple()
D = (0.05, 0.04, 0.01, 0.05)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def _state(nx, ny, seed):
    st = inputs.epidemic_state(nx, ny, seed)
    return st


def relmax(a, b):
    return max(float(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-300)) for c in range(5))


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(37, 29), (64, 48), (3, 5)])
def test_fp64_matches_oracle(bc, nx, ny):
    st = _state(nx, ny, nx + ny)
    dx, dt = 1.0, 1.0
    f = L.Fd4(nx, ny, RATES, D, dx=dx, dt=dt, bc=bc, precision=L.FP64)
    f.write(st)
    f.step(12)
    got = f.read()
    ref = oracle.fd4_rk4_run(st, D, RATES, dx, dt, bc, 12)
    assert relmax(got, ref) <= 1e-15
    assert f.steps_done() == 12
    f.close()


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(37, 29), (3, 5)])
def test_second_order_fp64_matches_oracle(bc, nx, ny):
    st = _state(nx, ny, 2 * nx + ny)
    f = L.Fd4(nx, ny, RATES, D, dx=0.7, dt=0.9, bc=bc, precision=L.FP64, order=2)
    f.write(st)
    f.step(12)
    ref = oracle.fd2_rk4_run(st, D, RATES, 0.7, 0.9, bc, 12)
    assert relmax(f.read(), ref) <= 1e-15
    f.close()


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_fp32_matches_oracle(bc):
    st = _state(45, 33, 3)
    f = L.Fd4(45, 33, RATES, D, dx=0.5, dt=0.8, bc=bc, precision=L.FP32)
    f.write(st.astype(np.float32))
    f.step(12)
    got = f.read().astype(np.float64)
    ref = oracle.fd4_rk4_run(st.astype(np.float32).astype(np.float64), D, RATES, 0.5, 0.8, bc, 12)
    assert relmax(got, ref) <= 2e-5
    f.close()


def test_uniform_state_follows_the_ode():
    """No gradients: the scheme is RK4 on the SEIRD system (the oracle's ODE integrator)."""
    y0 = np.array([0.97, 0.01, 0.02, 0.0, 0.0])
    st = np.broadcast_to(y0[:, None, None], (5, 16, 16)).copy()
    f = L.Fd4(16, 16, RATES, D, dt=0.5, bc=L.BC_NOFLUX, precision=L.FP64)
    f.write(st)
    f.step(40)
    got = f.read()
    y = oracle.ode_rk4(y0, RATES, 0.5, 40)
    for c in range(5):
        np.testing.assert_allclose(got[c], y[c], rtol=1e-14, atol=1e-17)
    f.close()


def test_device_and_host_transfers_and_conversions():
    import torch
    st = _state(24, 20, 9)
    f = L.Fd4(24, 20, RATES, D, precision=L.FP32)
    f.write(torch.from_numpy(st).cuda())         # FP64 device data into an FP32 state
    out = torch.empty((5, 20, 24), dtype=torch.float64, device="cuda")
    L.sslbm_fd4_read(f.f, out)
    np.testing.assert_array_equal(out.cpu().numpy(), st.astype(np.float32).astype(np.float64))
    f.write(st)                                   # FP64 host data into an FP32 state
    np.testing.assert_array_equal(f.read(np.float32), st.astype(np.float32))
    f.close()


def test_rejects_what_it_does_not_run():
    with pytest.raises(L.SslbmError) as e:
        L.Fd4(16, 16, RATES, (0.3, 0.05, 0.05, 0.05), dt=1.0)  # d dt / dx^2 = 0.3 > 0.26
    assert e.value.status == L.SSLBM_ERR_UNSTABLE
    with pytest.raises(L.SslbmError):
        L.Fd4(16, 16, RATES, D, precision=L.FP32_DEV)
    with pytest.raises(L.SslbmError):
        L.Fd4(16, 16, RATES, (0.05, 0.05, 0.05, 0.05, 0.01))  # D does not move
    with pytest.raises(L.SslbmError):
        L.Fd4(16, 16, RATES, D, order=3)
