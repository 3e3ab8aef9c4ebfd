"""Pins of the SSLBM with spatially varying, anisotropic diffusion (oracle.sslbm_vard_run).

Sec. IV lists spatially varying and anisotropic diffusion coefficients as future work and
gives no discretisation.  The reading pinned here is the D2Q5 link (flux) form
    rho_new = rho_c + sum_i D_i (rho(x + c_i) - rho_c) + Psi dt,
    D_i = d_lattice (k_a(x) + k_a(x + c_i)) / 2   (a = x or y by the link's axis),
the conservative discretisation of div(d(x) grad rho).

- Uniform fields k = 1 give the SSLBM of Eq. (sslbm_final_clean) (up to rounding order);
  a uniform k = s gives the SSLBM with diffusivity s d.
- The population is conserved exactly (Sec. II.C) for any fields, periodic and no-flux.
- The diffusion operator is symmetric, <g, A f> = <f, A g>.  The other reading, a per-cell
  tau(x) put into Eq. (sslbm_final_clean) (d(x) times the 5-point Laplacian), is not, and
  does not conserve; the test checks both, so it tells the readings apart.
- Constant anisotropic fields: a Fourier mode is multiplied per step by exactly
  G = 1 - 2 d kx (1 - cos kx) - 2 d ky (1 - cos ky).
- Maximum principle under the stability bound d_lattice * max_x sum_i k_link <= 1.
- Brute force: a direct evaluation of the update from its definition on tiny grids.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs

NO_REACTION = (0.0, 0.0, 0.0, 0.0)
RATES = (0.5, 0.2, 0.11, 1 / 11)
TAU = [0.65, 0.62, 0.53, 0.65]


def _fields(nx, ny, seed, lo=0.2, hi=1.8):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (ny, nx)), rng.uniform(lo, hi, (ny, nx))


@pytest.mark.parametrize("bc", [0, 1])
def test_uniform_fields_give_the_sslbm(bc):
    st = inputs.epidemic_state(23, 17, seed=2)
    one = np.ones((17, 23))
    got = oracle.sslbm_vard_run(st, TAU, RATES, one, one, 1.0, bc, 30)
    want = oracle.sslbm_run(st, TAU, RATES, 1.0, bc, 30)
    for c in range(5):
        assert np.abs(got[c] - want[c]).max() <= 1e-14 * np.abs(want[c]).max()
    # a uniform scale s is the SSLBM with diffusivity s d: tau' = 3 s d + 1/2
    s = 0.6
    tau_s = [3 * s * (t - 0.5) / 3 + 0.5 for t in TAU]
    got = oracle.sslbm_vard_run(st, TAU, RATES, s * one, s * one, 1.0, bc, 30)
    want = oracle.sslbm_run(st, tau_s, RATES, 1.0, bc, 30)
    for c in range(5):
        assert np.abs(got[c] - want[c]).max() <= 1e-14 * np.abs(want[c]).max()


@pytest.mark.parametrize("bc", [0, 1])
def test_conserves_population(bc):
    st = inputs.epidemic_state(19, 14, seed=6)
    kx, ky = _fields(19, 14, 3)
    out = oracle.sslbm_vard_run(st, TAU, RATES, kx, ky, 1.0, bc, 40)
    assert abs(out.sum() - st.sum()) / st.sum() < 1e-13


def _diffuse_once(f, kx, ky, tau, bc):
    st = np.zeros((5,) + f.shape)
    st[0] = f
    return oracle.sslbm_vard_run(st, [tau] * 4, NO_REACTION, kx, ky, 1.0, bc, 1)[0]


def _percell_reading(f, kx, tau):
    """The rejected reading on a periodic grid: tau(x) put into Eq. (sslbm_final_clean) at
    each cell, i.e. d_lattice k(x) times the 5-point Laplacian."""
    lap = (np.roll(f, 1, 1) + np.roll(f, -1, 1) + np.roll(f, 1, 0) + np.roll(f, -1, 0) - 4 * f)
    return f + (tau - 0.5) / 3 * kx * lap


@pytest.mark.parametrize("bc", [0, 1])
def test_operator_is_symmetric_and_the_percell_reading_is_not(bc):
    rng = np.random.default_rng(11)
    ny, nx = 12, 15
    kx, ky = _fields(nx, ny, 4)
    f, g = rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))
    af, ag = _diffuse_once(f, kx, ky, 0.8, bc), _diffuse_once(g, kx, ky, 0.8, bc)
    scale = np.abs(f).sum() * np.abs(g).sum() / f.size
    assert abs(np.vdot(g, af) - np.vdot(f, ag)) <= 1e-13 * scale
    if bc == 0:
        bf, bg = _percell_reading(f, kx, 0.8), _percell_reading(g, kx, 0.8)
        assert abs(np.vdot(g, bf) - np.vdot(f, bg)) > 1e-3 * scale
        assert abs(bf.sum() - f.sum()) > 1e-3 * np.abs(f).sum() / f.size


@pytest.mark.parametrize("ax,ay", [(1.0, 1.0), (1.7, 0.3), (0.0, 1.2)])
def test_anisotropic_mode_factor_exact(ax, ay):
    nx, ny, n, tau = 30, 24, 25, 0.7
    m, q = 2, 3
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * q / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    shape = np.cos(kx * x + ky * y)
    st = np.zeros((5, ny, nx))
    st[:4] = 1.0 + 0.3 * shape
    out = oracle.sslbm_vard_run(st, [tau] * 4, NO_REACTION, np.full((ny, nx), ax), np.full((ny, nx), ay),
                                1.0, 0, n)
    d = (tau - 0.5) / 3
    G = 1 - 2 * d * ax * (1 - math.cos(kx)) - 2 * d * ay * (1 - math.cos(ky))
    np.testing.assert_allclose(out[0], 1.0 + 0.3 * G ** n * shape, rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", [0, 1])
def test_maximum_principle(bc):
    rng = np.random.default_rng(5)
    ny, nx = 16, 13
    kx, ky = _fields(nx, ny, 9, 0.0, 1.5)
    tau = 0.5 + 3 * (1.0 / (4 * 1.5))  # d = 1/6: d * (4 links x 1.5) = 1, the bound itself
    st = np.zeros((5, ny, nx))
    st[:4] = rng.uniform(0.0, 1.0, (4, ny, nx))
    lo, hi = st[:4].min(), st[:4].max()
    out = oracle.sslbm_vard_run(st, [tau] * 4, NO_REACTION, kx, ky, 1.0, bc, 200)
    assert out[:4].min() >= lo - 1e-15 and out[:4].max() <= hi + 1e-15
    assert out[:4].max() - out[:4].min() < 0.5 * (hi - lo)  # and it diffuses


def _brute(state, tau, rates, kx, ky, dt, bc):
    _, ny, nx = state.shape
    beta, alpha, gamma, phi = rates

    def idx(i, n):
        if 0 <= i < n:
            return i
        return i % n if bc == 0 else min(max(i, 0), n - 1)

    out = np.empty_like(state)
    for yy in range(ny):
        for xx in range(nx):
            S, E, I, R, D = state[:, yy, xx]
            Nc = S + E + I + R
            F = beta * S * I / Nc if Nc != 0 else 0.0
            psi = [-F, F - alpha * E, alpha * E - gamma * I, (1 - phi) * gamma * I, phi * gamma * I]
            for c in range(4):
                d = (tau[c] - 0.5) / 3
                total = 0.0
                for cx, cy in ((1, 0), (0, 1), (-1, 0), (0, -1)):
                    kap = kx if cx else ky
                    xn, yn = idx(xx + cx, nx), idx(yy + cy, ny)
                    link = d * (kap[yy, xx] + kap[yn, xn]) / 2
                    total += link * (state[c, yn, xn] - state[c, yy, xx])
                out[c, yy, xx] = state[c, yy, xx] + total + psi[c] * dt
            out[4, yy, xx] = D + psi[4] * dt
    return out


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", [(5, 4), (1, 3), (2, 2)])
def test_brute_force_tiny_grids(bc, nx, ny):
    st = inputs.epidemic_state(nx, ny, seed=nx * 3 + ny)
    kx, ky = _fields(nx, ny, nx + 7 * ny)
    tau = [0.7, 0.6, 0.55, 0.8]
    a = st.copy()
    for _ in range(3):
        a = _brute(a, tau, RATES, kx, ky, 0.8, bc)
    b = oracle.sslbm_vard_run(st, tau, RATES, kx, ky, 0.8, bc, 3)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-15)
