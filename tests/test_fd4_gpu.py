"""The fourth-order finite-difference reference on the GPU (sslbm_fd4_*) against the FP64
oracle's fd4_rk4_run, and its second-order variant against fd2_rk4_run.

The kernels evaluate every operation in the oracle's order with one rounding each (no
contraction) and IEEE division, so FP64 agrees to the last bit up to the order of nothing
at all; the test allows 1e-15 relative.  FP32 keeps the same order in single precision:
over 12 RK4 steps of a contractive stencil the error stays within a few hundred FP32
roundings of the field's peak (2e-5 relative max-norm, per compartment).  Both FP32
kernels are also compared bit for bit with the same formulas evaluated in float32.
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


def _ghost(i, n, periodic):
    """Cell index along an axis of n cells for a possibly ghost index i: periodic wrap, or the
    even reflection about the boundary face (u[-1] = u[0], u[-2] = u[1]), clamped to the grid
    when it is narrower than the stencil."""
    i = np.asarray(i)
    if periodic:
        return np.mod(i, n)
    i = np.where(i < 0, -1 - i, i)
    i = np.where(i >= n, 2 * n - 1 - i, i)
    return np.clip(i, 0, n - 1)


def _fd4_float32(st, d, rates, dx, dt, bc, steps, order):
    """The RK4 stages evaluated in FP32 with one rounding per operation (numpy float32), in
    the operation order the kernels document, for a bitwise comparison."""
    f = np.float32
    beta, alpha, gamma, phi = rates
    kb, ka, kg = f(beta), f(alpha), f(gamma)
    rg, dg = f((1.0 - phi) * gamma), f(phi * gamma)
    kd = [f(x) for x in d[:4]]
    scale = f(1.0 / (12.0 * dx * dx)) if order == 4 else f(1.0 / (dx * dx))
    half_dt, fdt, dt6 = f(0.5 * dt), f(dt), f(dt / 6.0)
    ny, nx = st.shape[1:]
    periodic = bc == L.BC_PERIODIC
    gx = {o: _ghost(np.arange(nx) + o, nx, periodic) for o in (-2, -1, 1, 2)}
    gy = {o: _ghost(np.arange(ny) + o, ny, periodic) for o in (-2, -1, 1, 2)}
    c2, c16, c30 = f(2), f(16), f(30)

    def slope(v):
        S, E, I, R = v[0], v[1], v[2], v[3]
        Nc = ((S + E) + I) + R
        with np.errstate(divide="ignore", invalid="ignore"):
            F = np.where(Nc != 0, ((kb * S) * I) / Nc, f(0)).astype(f)
        aE = ka * E
        r = [-F, F - aE, aE - kg * I, rg * I, dg * I]
        for c in range(4):
            u0 = v[c]
            xm2, xm1, xp1, xp2 = (u0[:, gx[o]] for o in (-2, -1, 1, 2))
            ym2, ym1, yp1, yp2 = (u0[gy[o], :] for o in (-2, -1, 1, 2))
            if order == 4:
                lx = ((((-xm2) + c16 * xm1) - c30 * u0) + c16 * xp1) - xp2
                ly = ((((-ym2) + c16 * ym1) - c30 * u0) + c16 * yp1) - yp2
            else:
                lx = (xm1 - c2 * u0) + xp1
                ly = (ym1 - c2 * u0) + yp1
            r[c] = r[c] + (kd[c] * (lx + ly)) * scale
        return np.stack(r)

    u = st.astype(f)
    for _ in range(steps):
        k1 = slope(u)
        acc, t = k1, u + half_dt * k1
        k2 = slope(t)
        acc, t = acc + c2 * k2, u + half_dt * k2
        k3 = slope(t)
        acc, t = acc + c2 * k3, u + fdt * k3
        k4 = slope(t)
        u = u + dt6 * (acc + k4)
    return u


@pytest.mark.parametrize("order", [4, 2])
@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny,steps", [(45, 33, 6), (3, 5, 6), (128, 40, 6), (4, 6, 6), (8, 3, 6), (516, 130, 6),
                                         (1028, 1001, 2)])
def test_fp32_bitwise_against_float32_evaluation(bc, nx, ny, steps, order):
    """Both FP32 stage kernels give the bits of the same formulas evaluated in float32, one
    rounding per operation.  Grids of fewer than six 128 x 8 tiles per SM run the one-cell
    kernel (several tiles, ragged edges, grids narrower than the stencil); 1028 x 1001
    (1134 tiles, a last tile of 4 columns and a last row tile of 1 row) runs the
    four-cells-per-thread kernel on a GB300's 152 SMs."""
    st = _state(nx, ny, 5 * nx + ny)
    f = L.Fd4(nx, ny, RATES, D, dx=0.5, dt=0.8, bc=bc, precision=L.FP32, order=order)
    f.write(st.astype(np.float32))
    f.step(steps)
    got = f.read(dtype=np.float32)
    f.close()
    ref = _fd4_float32(st.astype(np.float32), D, RATES, 0.5, 0.8, bc, steps, order)
    assert got.dtype == np.float32 and ref.dtype == np.float32
    bad = np.argwhere(got.view(np.uint32) != ref.view(np.uint32))
    assert bad.size == 0, (len(bad), bad[:3], got[tuple(bad[0])], ref[tuple(bad[0])])


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_fp32_vector_tiles_match_oracle(bc):
    """The four-cells-per-thread FP32 kernel (a grid of more than six tiles per SM, ragged in
    both directions) against the FP64 oracle, with the tolerance of the one-cell kernel's test."""
    st = _state(1028, 1001, 11)
    f = L.Fd4(1028, 1001, RATES, D, dx=0.5, dt=0.8, bc=bc, precision=L.FP32)
    f.write(st.astype(np.float32))
    f.step(12)
    got = f.read().astype(np.float64)
    f.close()
    ref = oracle.fd4_rk4_run(st.astype(np.float32).astype(np.float64), D, RATES, 0.5, 0.8, bc, 12)
    assert relmax(got, ref) <= 2e-5


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
