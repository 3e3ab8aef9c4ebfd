"""Brute force on tiny grids: pure-Python loops written straight from the
equations (dictionary-of-neighbours, no arrays, no shared helpers) against the C
oracle, including the degenerate 1-wide and 1x1 lattices.  A cross-check of the
C indexing; the independent pins are in test_oracle_pins.py."""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs

LINKS = [((0, 0), 1 / 3), ((1, 0), 1 / 6), ((0, 1), 1 / 6), ((-1, 0), 1 / 6), ((0, -1), 1 / 6)]


def _nb(field, x, y, nx, ny, bc):
    if bc == 0:
        return field[y % ny][x % nx]
    x = min(max(x, 0), nx - 1)
    y = min(max(y, 0), ny - 1)
    return field[y][x]


def _sources(S, E, I, R, beta, alpha, gamma, phi):
    Nc = S + E + I + R
    F = beta * S * I / Nc if Nc != 0 else 0.0
    return [-F, F - alpha * E, alpha * E - gamma * I, (1 - phi) * gamma * I, phi * gamma * I]


def _brute_sslbm(st, tau, rates, dt, bc, nsteps):
    _, ny, nx = st.shape
    cur = [[[float(st[c, y, x]) for x in range(nx)] for y in range(ny)] for c in range(5)]
    for _ in range(nsteps):
        new = [[[0.0] * nx for _ in range(ny)] for _ in range(5)]
        for y in range(ny):
            for x in range(nx):
                psi = _sources(*(cur[c][y][x] for c in range(4)), *rates)
                for c in range(4):
                    rf = sum(w * _nb(cur[c], x + dx, y + dy, nx, ny, bc) for (dx, dy), w in LINKS)
                    rb = sum(w * _nb(cur[c], x - dx, y - dy, nx, ny, bc) for (dx, dy), w in LINKS)
                    rc = cur[c][y][x]
                    new[c][y][x] = rb + (tau[c] - 1) * (rf - 2 * rc + rb) + psi[c] * dt
                new[4][y][x] = cur[4][y][x] + psi[4] * dt
        cur = new
    return np.array(cur)


def _brute_bgk(st, tau, rates, dt, bc, nsteps):
    _, ny, nx = st.shape
    w = [lw for _, lw in LINKS]
    f = [[[[w[i] * st[c, y, x] for x in range(nx)] for y in range(ny)] for i in range(5)] for c in range(4)]
    D = [[float(st[4, y, x]) for x in range(nx)] for y in range(ny)]
    opp = {0: 0, 1: 3, 2: 4, 3: 1, 4: 2}
    for _ in range(nsteps):
        post = [[[[0.0] * nx for _ in range(ny)] for _ in range(5)] for _ in range(4)]
        newD = [[0.0] * nx for _ in range(ny)]
        for y in range(ny):
            for x in range(nx):
                rho = [sum(f[c][i][y][x] for i in range(5)) for c in range(4)]
                psi = _sources(*rho, *rates)
                for c in range(4):
                    for i in range(5):
                        fi = f[c][i][y][x]
                        post[c][i][y][x] = fi + (w[i] * rho[c] - fi) / tau[c] + w[i] * psi[c] * dt
                newD[y][x] = D[y][x] + psi[4] * dt
        # push each post-collision population along its link
        nf = [[[[None] * nx for _ in range(ny)] for _ in range(5)] for _ in range(4)]
        for y in range(ny):
            for x in range(nx):
                for i, ((cx, cy), _) in enumerate(LINKS):
                    tx, ty = x + cx, y + cy
                    for c in range(4):
                        if 0 <= tx < nx and 0 <= ty < ny:
                            nf[c][i][ty][tx] = post[c][i][y][x]
                        elif bc == 0:
                            nf[c][i][ty % ny][tx % nx] = post[c][i][y][x]
                        else:
                            nf[c][opp[i]][y][x] = post[c][i][y][x]
        f, D = nf, newD
    out = np.zeros((5, ny, nx))
    for c in range(4):
        for y in range(ny):
            for x in range(nx):
                out[c, y, x] = sum(f[c][i][y][x] for i in range(5))
    out[4] = np.array(D)
    return out


SHAPES = [(1, 1), (1, 5), (6, 1), (2, 2), (4, 4), (5, 3), (3, 7)]
RATES = (0.5, 0.2, 0.11, 1 / 11)
TAU = [0.65, 0.6, 0.53, 0.7]


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_sslbm_tiny_bruteforce(nx, ny, bc):
    st = inputs.epidemic_state(nx, ny, seed=nx * 31 + ny)
    got = oracle.sslbm_run(st, TAU, RATES, 1.0, bc, 4)
    want = _brute_sslbm(st, TAU, RATES, 1.0, bc, 4)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_bgk_tiny_bruteforce(nx, ny, bc):
    st = inputs.epidemic_state(nx, ny, seed=nx * 17 + ny)
    got = oracle.bgk_run_state(st, TAU, RATES, 1.0, bc, 3)
    want = _brute_bgk(st, TAU, RATES, 1.0, bc, 3)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-16)
