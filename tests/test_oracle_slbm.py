"""Pins of the two-pass SLBM oracle (oracle.slbm_run), Eqs. (SLBM1, SLBM2).

- On a Fourier mode the predictor multiplies by the D2Q5 symbol Lambda = 1/3 + (cos kx +
  cos ky)/3, and the corrector's neighbour sum by Lambda again, so one step multiplies the
  mode by G = Lambda + (tau - 1)(Lambda^2 - 1).
- Expanding Lambda = 1 - e, G = 1 - (2 tau - 1) e + (tau - 1) e^2: the single-step SSLBM's
  factor 1 - (2 tau - 1) e to first order in e (the same diffusivity), different at O(k^4).
- The population is conserved exactly under periodic and no-flux boundaries.
- Brute force: a direct evaluation of both passes from their definition on tiny grids.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs

NO_REACTION = (0.0, 0.0, 0.0, 0.0)
CX = [0, 1, 0, -1, 0]
CY = [0, 0, 1, 0, -1]
W = [1 / 3, 1 / 6, 1 / 6, 1 / 6, 1 / 6]


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.2])
def test_mode_amplification_exact(tau):
    nx, ny, n = 28, 20, 30
    m, q = 2, 3
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * q / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    shape = np.cos(kx * x + ky * y)
    st = np.zeros((5, ny, nx))
    st[:4] = 1.0 + 0.3 * shape
    out = oracle.slbm_run(st, [tau] * 4, NO_REACTION, 1.0, 0, n)
    lam = 1 / 3 + (math.cos(kx) + math.cos(ky)) / 3
    G = lam + (tau - 1) * (lam * lam - 1)
    np.testing.assert_allclose(out[0], 1.0 + 0.3 * G ** n * shape, rtol=0, atol=1e-13)


def test_agrees_with_the_sslbm_to_first_order_in_one_minus_lambda():
    tau = 0.8
    for e in (1e-2, 5e-3, 2.5e-3):
        lam = 1 - e
        g_slbm = lam + (tau - 1) * (lam * lam - 1)
        g_sslbm = 1 - (2 * tau - 1) * (1 - lam)
        assert g_slbm - g_sslbm == pytest.approx((tau - 1) * e * e, rel=1e-9)


@pytest.mark.parametrize("bc", [0, 1])
def test_conserves_population(bc):
    st = inputs.epidemic_state(19, 14, seed=6)
    out = oracle.slbm_run(st, [0.65, 0.62, 0.53, 0.65], (0.5, 0.2, 0.11, 1 / 11), 1.0, bc, 40)
    assert abs(out.sum() - st.sum()) / st.sum() < 1e-13


def _brute(state, tau, rates, dt, bc):
    _, ny, nx = state.shape
    beta, alpha, gamma, phi = rates

    def idx(i, n):
        if 0 <= i < n:
            return i
        return i % n if bc == 0 else min(max(i, 0), n - 1)

    pred = np.empty((4, ny, nx))
    for c in range(4):
        for yy in range(ny):
            for xx in range(nx):
                pred[c, yy, xx] = sum(w * state[c, idx(yy - cy, ny), idx(xx - cx, nx)]
                                      for w, cx, cy in zip(W, CX, CY))
    out = np.empty_like(state)
    for yy in range(ny):
        for xx in range(nx):
            S, E, I, R, D = state[:, yy, xx]
            Nc = S + E + I + R
            F = beta * S * I / Nc if Nc != 0 else 0.0
            psi = [-F, F - alpha * E, alpha * E - gamma * I, (1 - phi) * gamma * I, phi * gamma * I]
            for c in range(4):
                s = sum(w * pred[c, idx(yy + cy, ny), idx(xx + cx, nx)] for w, cx, cy in zip(W, CX, CY))
                out[c, yy, xx] = pred[c, yy, xx] + (tau[c] - 1) * (s - state[c, yy, xx]) + psi[c] * dt
            out[4, yy, xx] = D + psi[4] * dt
    return out


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", [(5, 4), (1, 3), (2, 2)])
def test_brute_force_tiny_grids(bc, nx, ny):
    st = inputs.epidemic_state(nx, ny, seed=nx * 5 + ny)
    tau = [0.7, 0.6, 0.55, 0.8]
    rates = (0.5, 0.2, 0.11, 0.1)
    a = st.copy()
    for _ in range(3):
        a = _brute(a, tau, rates, 0.8, bc)
    b = oracle.slbm_run(st, tau, rates, 0.8, bc, 3)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-15)
