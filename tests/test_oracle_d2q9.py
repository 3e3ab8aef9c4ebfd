"""Pins of the D2Q9 SSLBM oracle (oracle.sslbm9_run).

- A Fourier mode of the diffusion part is multiplied by G = 1 - (2 tau - 1)(1 - Lambda9(k))
  per step, with the D2Q9 symbol Lambda9 = sum_i w_i cos(k . c_i)
  = 4/9 + (2/9)(cos kx + cos ky) + (1/18)(cos(kx + ky) + cos(kx - ky)).
  The paper prints the cosine coefficients as 1/9 and 1/36 (half these), which gives
  Lambda(0) = 13/18 instead of 1. Its small-k expansion, |k|^2/6 - |k|^4/72, belongs to the
  symbol above, which is isotropic to fourth order; D2Q5 carries a kx^2 ky^2 term.
- The discrete population is conserved exactly under periodic and no-flux (bounce-back)
  boundaries.
- Brute force: a direct evaluation of the update from its definition on tiny grids.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs

NO_REACTION = (0.0, 0.0, 0.0, 0.0)
CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
W = [4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36]


def lam9(kx, ky):
    return sum(w * math.cos(kx * cx + ky * cy) for w, cx, cy in zip(W, CX, CY))


def test_symbol_closed_form_and_the_printed_slip():
    for kx, ky in [(0.0, 0.0), (0.3, 1.1), (math.pi, math.pi), (2.0, -0.7)]:
        closed = 4 / 9 + 2 / 9 * (math.cos(kx) + math.cos(ky)) + (math.cos(kx + ky) + math.cos(kx - ky)) / 18
        assert lam9(kx, ky) == pytest.approx(closed, abs=1e-15)
    printed0 = 4 / 9 + (1 + 1) / 9 + (1 + 1) / 36
    assert printed0 == pytest.approx(13 / 18) and abs(printed0 - 1) > 0.2
    assert lam9(0.0, 0.0) == pytest.approx(1.0, abs=1e-15)


def test_fourth_order_isotropy():
    """1 - Lambda9 = |k|^2/6 - |k|^4/72 + O(k^6) along every direction; D2Q5's fourth-order
    term depends on the direction."""
    r = 1e-2
    quartic9, quartic5 = [], []
    for th in (0.0, math.pi / 8, math.pi / 4, 0.3):
        kx, ky = r * math.cos(th), r * math.sin(th)
        quartic9.append((1 - lam9(kx, ky) - r * r / 6) / r ** 4)
        lam5 = 1 / 3 + (math.cos(kx) + math.cos(ky)) / 3
        quartic5.append((1 - lam5 - r * r / 6) / r ** 4)
    assert all(abs(q + 1 / 72) < 1e-4 for q in quartic9), quartic9
    assert max(quartic5) - min(quartic5) > 5e-3


@pytest.mark.parametrize("tau", [0.65, 1.2, 1.6])
def test_mode_amplification_exact(tau):
    nx, ny, n = 30, 24, 25
    m, q = 3, 2
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * q / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    shape = np.cos(kx * x + ky * y)
    st = np.zeros((5, ny, nx))
    st[:4] = 1.0 + 0.3 * shape
    out = oracle.sslbm9_run(st, [tau] * 4, NO_REACTION, 1.0, 0, n)
    G = 1 - (2 * tau - 1) * (1 - lam9(kx, ky))
    np.testing.assert_allclose(out[0], 1.0 + 0.3 * G ** n * shape, rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", [0, 1])
def test_conserves_population(bc):
    st = inputs.epidemic_state(21, 16, seed=4)
    out = oracle.sslbm9_run(st, [0.65, 0.62, 0.53, 0.65], (0.5, 0.2, 0.11, 1 / 11), 1.0, bc, 40)
    assert abs(out.sum() - st.sum()) / st.sum() < 1e-13
    assert out.min() >= 0.0


def test_uniform_state_is_the_euler_ode():
    y0 = np.array([0.9, 0.03, 0.05, 0.02, 0.0])
    st = np.broadcast_to(y0[:, None, None], (5, 6, 7)).copy()
    rates = (0.5, 0.2, 0.11, 1 / 11)
    out = oracle.sslbm9_run(st, [0.7] * 4, rates, 0.5, 1, 10)
    y = y0.copy()
    for _ in range(10):
        S, E, I, R, D = y
        F = rates[0] * S * I / (S + E + I + R)
        y = y + 0.5 * np.array([-F, F - rates[1] * E, rates[1] * E - rates[2] * I,
                                (1 - rates[3]) * rates[2] * I, rates[3] * rates[2] * I])
    for c in range(5):
        np.testing.assert_allclose(out[c], y[c], rtol=1e-14, atol=1e-17)


def _brute(state, tau, rates, dt, bc):
    """One D2Q9 SSLBM step written from its definition, cell by cell."""
    _, ny, nx = state.shape
    out = np.empty_like(state)
    beta, alpha, gamma, phi = rates

    def val(p, x0, y0, x, y):
        if bc == 0:
            return p[y % ny, x % nx]
        if 0 <= x < nx and 0 <= y < ny:
            return p[y, x]
        return p[y0, x0]

    for yy in range(ny):
        for xx in range(nx):
            S, E, I, R, D = state[:, yy, xx]
            Nc = S + E + I + R
            F = beta * S * I / Nc if Nc != 0 else 0.0
            psi = [-F, F - alpha * E, alpha * E - gamma * I, (1 - phi) * gamma * I, phi * gamma * I]
            for c in range(4):
                p = state[c]
                rf = sum(w * val(p, xx, yy, xx + cx, yy + cy) for w, cx, cy in zip(W, CX, CY))
                rb = sum(w * val(p, xx, yy, xx - cx, yy - cy) for w, cx, cy in zip(W, CX, CY))
                out[c, yy, xx] = rb + (tau[c] - 1) * (rf - 2 * p[yy, xx] + rb) + psi[c] * dt
            out[4, yy, xx] = D + psi[4] * dt
    return out


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", [(5, 4), (1, 3), (2, 2)])
def test_brute_force_tiny_grids(bc, nx, ny):
    st = inputs.epidemic_state(nx, ny, seed=nx * 7 + ny)
    tau = [0.7, 0.6, 0.55, 0.8]
    rates = (0.5, 0.2, 0.11, 0.1)
    a = st.copy()
    for _ in range(3):
        a = _brute(a, tau, rates, 0.8, bc)
    b = oracle.sslbm9_run(st, tau, rates, 0.8, bc, 3)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-15)
