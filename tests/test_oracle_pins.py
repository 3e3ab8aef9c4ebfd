"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than the oracle itself:
a closed form, an invariant, a value or matrix printed in the paper, a library
routine, or a convergence order.  Together they are chosen so that a dropped
term, a wrong sign or index, or a transposed operand anywhere in the oracle makes
at least one of them fail.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
NO_REACTION = (0.0, 0.0, 0.0, 0.0)


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------------------
# Lattice and relaxation time
# ---------------------------------------------------------------------------

def test_d2q5_golden_symmetry_relations():
    """Sec. II.C 'Consistency': sum w = 1, sum w c = 0, sum w c_a c_b = c_s^2 delta_ab."""
    g = _gold("d2q5_lattice.json")
    cx, cy, w = np.array(g["cx"]), np.array(g["cy"]), np.array(g["w"])
    cs2 = g["cs2_fraction"][0] / g["cs2_fraction"][1]
    assert math.isclose(w.sum(), 1.0, rel_tol=0, abs_tol=1e-15)
    assert abs((w * cx).sum()) < 1e-15 and abs((w * cy).sum()) < 1e-15
    assert math.isclose((w * cx * cx).sum(), cs2, abs_tol=1e-15)
    assert math.isclose((w * cy * cy).sum(), cs2, abs_tol=1e-15)
    assert abs((w * cx * cy).sum()) < 1e-15


@pytest.mark.parametrize("d,dx,dt", [(0.05, 1.0, 1.0), (0.01, 1.0, 1.0), (0.0, 1.0, 1.0),
                                     (4.35e-2, 1.0, 0.01), (1e-4, 1.0, 0.01), (0.3, 0.5, 0.2)])
def test_tau_inverts_eq_diffusivity(d, dx, dt):
    """Eq. (diffusivity): d dt/dx^2 = c_s^2 (tau - 1/2) with c_s^2 = 1/3."""
    tau = oracle.tau_from_d(d, dx, dt)
    assert math.isclose((tau - 0.5) / 3.0, d * dt / dx ** 2, rel_tol=1e-14, abs_tol=1e-16)


# ---------------------------------------------------------------------------
# Diffusion operator: exact per-mode amplification
# ---------------------------------------------------------------------------

def _g_corrected(tau, thx, thy):
    """Amplification of Eq. (sslbm_clean) for a mode with per-link phases thx, thy,
    substituting rho_f = rho_b = Lambda rho (Eq. Lambda_D2Q5):
    G = Lambda + 2 (tau - 1)(Lambda - 1) = 1 - (2 tau - 1)(1 - Lambda)."""
    lam = 1.0 / 3.0 + (math.cos(thx) + math.cos(thy)) / 3.0
    return 1.0 - (2.0 * tau - 1.0) * (1.0 - lam)


def _g_printed(tau, thx, thy):
    """The last line of Eq. (G_exact) as printed: 1 - 2 (tau - 1)(1 - Lambda)."""
    lam = 1.0 / 3.0 + (math.cos(thx) + math.cos(thy)) / 3.0
    return 1.0 - 2.0 * (tau - 1.0) * (1.0 - lam)


@pytest.mark.parametrize("bc", [0, 1])
def test_sslbm_mode_amplification_exact(bc):
    """Reactions off: each compartment carries its own mode and relaxation time;
    after n steps the mode amplitude is G^n exactly (to roundoff).  Periodic uses
    cos(kx x + ky y) with k = 2 pi m / n; no-flux uses the cell-centred cosine
    cos(pi m (x + 1/2)/nx) cos(pi q (y + 1/2)/ny), the eigenfunction of the mirror
    stencil.  Non-square grid, different m and q per compartment: a transposed
    axis, a swapped compartment, a wrong weight or a wrong tau all change G."""
    nx, ny, nsteps = 40, 28, 60
    taus = [0.65, 0.53, 0.8, 1.1]
    modes = [(1, 2), (3, 1), (2, 3), (5, 4)]
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    st = np.zeros((5, ny, nx))
    expect = np.zeros((5, ny, nx))
    for c, ((m, q), tau) in enumerate(zip(modes, taus)):
        if bc == 0:
            thx, thy = 2 * math.pi * m / nx, 2 * math.pi * q / ny
            shape = np.cos(thx * x + thy * y + 0.3 * c)
        else:
            thx, thy = math.pi * m / nx, math.pi * q / ny
            shape = np.cos(thx * (x + 0.5)) * np.cos(thy * (y + 0.5))
        st[c] = 2.0 + 0.5 * shape
        expect[c] = 2.0 + 0.5 * _g_corrected(tau, thx, thy) ** nsteps * shape
        # the printed form of Eq. (G_exact) would predict a visibly different field
        assert abs(_g_printed(tau, thx, thy) ** nsteps - _g_corrected(tau, thx, thy) ** nsteps) > 1e-3
    st[4] = 0.7
    expect[4] = 0.7
    out = oracle.sslbm_run(st, taus, NO_REACTION, 1.0, bc, nsteps)
    np.testing.assert_allclose(out, expect, rtol=0, atol=2e-13)


def test_sslbm_long_wave_decays_like_continuum():
    """Sec. III.B / consistency: with reactions off, a long-wave mode decays as
    exp(-d |k|^2 t); the discrepancy is O(k^4 t), i.e. it shrinks ~4x per halving of
    k at fixed d k^2 t."""
    d = 0.05
    tau = oracle.tau_from_d(d)
    errs = []
    for n in (64, 128):
        k = 2 * math.pi / n
        t = int(round(0.5 / (d * k * k)))  # fixed decay d k^2 t = 0.5
        x = np.arange(n)[None, :]
        st = np.zeros((5, 4, n))
        st[0] = 1.0 + 0.1 * np.cos(k * x)
        st[1:4] = 1.0
        out = oracle.sslbm_run(st, [tau] * 4, NO_REACTION, 1.0, 0, t)
        amp = (out[0, 0] - 1.0) @ np.cos(k * x[0]) / (0.1 * (n / 2))
        errs.append(abs(amp / math.exp(-d * k * k * t) - 1.0))
    assert errs[0] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0  # O(k^2) relative at fixed d k^2 t


# ---------------------------------------------------------------------------
# Reaction sources: the paper's Jacobian, growth rate, homogeneity
# ---------------------------------------------------------------------------

def _symbolic(entry, beta, alpha, gamma, phi):
    vals = dict(beta=beta, alpha=alpha, gamma=gamma, phigamma=phi * gamma)
    return sum(coef * vals[k] for k, coef in entry.items())


@pytest.mark.parametrize("rates", [(0.3, 0.2, 0.11, 1 / 11), (0.5, 1 / 7, 0.2, 0.3), (0.9, 0.35, 0.05, 0.6)])
def test_step_linearisation_matches_eq_jacobian(rates):
    """Finite-difference Jacobian of one SSLBM step of a uniform state at the
    disease-free equilibrium: (step(u + h e_j) - step(u)) / h = I + dt J e_j + O(h),
    with J printed in Eq. (jacobian) and the D row from Eq. (rhoD).  One-sided,
    because a negative E, I or R would leave the model's domain."""
    g = _gold("jacobian_dfe.json")
    beta, alpha, gamma, phi = rates
    dt, h, N = 0.25, 1e-6, 1.3
    J = np.array([[_symbolic(e, *rates) for e in row] for row in g["J"]])
    Drow = np.array([_symbolic(e, *rates) for e in g["D_row"]])
    tau = [0.6, 0.55, 0.7, 0.65]
    base = np.zeros((5, 3, 4))
    base[0] = N
    got = np.zeros((5, 4))
    for j in range(4):
        up = base.copy()
        up[j] += h
        a = oracle.sslbm_run(up, tau, rates, dt, 0, 1)[:, 1, 2]
        b = oracle.sslbm_run(base, tau, rates, dt, 0, 1)[:, 1, 2]
        got[:, j] = (a - b) / h
    want = np.zeros((5, 4))
    want[:4] = np.eye(4) + dt * J
    want[4] = dt * Drow
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6)


@pytest.mark.parametrize("rates,dt", [((0.3, 0.2, 0.11, 1 / 11), 1.0), ((0.5, 0.2, 0.11, 1 / 11), 0.5),
                                       ((0.6, 1 / 7, 0.2, 0.3), 0.1)])
def test_growth_rate_matches_eq_eigenvalues(rates, dt):
    """Near the DFE the explicit update multiplies the E-I block by I + dt J_EI
    (Eq. JEI), whose dominant eigenvalue is 1 + dt lambda_1 with lambda_1 from
    Eq. (eigenvalues); the step-to-step growth of I must approach it."""
    beta, alpha, gamma, phi = rates
    lam1 = (-(alpha + gamma) + math.sqrt((alpha - gamma) ** 2 + 4 * alpha * beta)) / 2
    st = np.zeros((5, 2, 2))
    st[0] = 1.0
    st[2] = 1e-14
    n = int(60 / dt)
    prev = oracle.sslbm_run(st, [0.6] * 4, rates, dt, 0, n)
    nxt = oracle.sslbm_run(prev, [0.6] * 4, rates, dt, 0, 1)
    ratio = nxt[2, 0, 0] / prev[2, 0, 0]
    assert abs(ratio - (1 + dt * lam1)) < 1e-6 * (1 + dt * lam1)


def test_step_is_degree_one_homogeneous():
    """The force of infection beta S I / N_c of Eq. (sources) is homogeneous of
    degree one and the stencil is linear, so step(2u) == 2 step(u) exactly (scaling
    by 2 commutes with rounding).  Dropping the 1/N_c would make it degree two."""
    u = inputs.epidemic_state(9, 7, seed=3)
    rates = (0.7, 0.2, 0.11, 0.2)
    a = oracle.sslbm_run(2.0 * u, [0.6, 0.55, 0.7, 0.65], rates, 0.5, 1, 5)
    b = oracle.sslbm_run(u, [0.6, 0.55, 0.7, 0.65], rates, 0.5, 1, 5)
    assert np.array_equal(a, 2.0 * b)


def test_zero_contact_population_gives_zero_force():
    """N_c = 0 (only D populated) is left open by the paper; the oracle takes F = 0."""
    psi = oracle.sources((0.5, 0.2, 0.1, 0.1), (0.0, 0.0, 0.0, 0.0))
    assert np.all(psi == 0.0)


def test_r_over_d_ratio_fixed_by_phi():
    """From Eqs. (EqSEIRD_R, EqSEIRD_D) with R = D = 0 initially and no R diffusion
    effect (uniform state), R / D = (1 - phi) / phi at all times -- the reason the
    paper reports R and D errors jointly (Tables tab:chi_combined, tab:combined_ratio)."""
    st = np.zeros((5, 3, 3))
    st[0], st[1], st[2] = 0.9, 0.05, 0.05
    phi = 0.3
    out = oracle.sslbm_run(st, [0.6] * 4, (0.6, 1 / 7, 0.2, phi), 0.1, 0, 500)
    np.testing.assert_allclose(out[3] / out[4], (1 - phi) / phi, rtol=1e-12)


# ---------------------------------------------------------------------------
# Invariants: conservation and nonnegativity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [0, 1])
def test_sslbm_conserves_total_population(bc):
    """Eq. (mass_conservation): sum over x and all five compartments is constant."""
    st = inputs.epidemic_state(37, 23, seed=11)
    tot0 = oracle.diagnostics(st)[0].sum()
    out = oracle.sslbm_run(st, [0.65, 0.6, 0.53, 0.7], (0.5, 0.2, 0.11, 1 / 11), 1.0, bc, 300)
    tot1 = oracle.diagnostics(out)[0].sum()
    assert abs(tot1 - tot0) / tot0 < 1e-13
    # without reactions every compartment is conserved on its own
    out = oracle.sslbm_run(st, [0.65, 0.6, 0.53, 0.7], NO_REACTION, 1.0, bc, 100)
    np.testing.assert_allclose(oracle.diagnostics(out)[0], oracle.diagnostics(st)[0], rtol=1e-13)


@pytest.mark.parametrize("bc", [0, 1])
def test_sslbm_stays_nonnegative(bc):
    """Under 4 d + (outflow rate) dt <= 1 per compartment each update is a convex
    combination plus nonnegative inflows, so densities stay >= 0 (checked here on a
    rough random state with a sharp infected spike)."""
    st = inputs.epidemic_state(31, 29, seed=5)
    st[2, 10, 10] = 0.9
    st[0, 10, 10] = 0.0
    out = st
    for _ in range(20):
        out = oracle.sslbm_run(out, [0.8, 0.8, 0.56, 0.8], (0.4, 0.2, 0.11, 1 / 11), 1.0, bc, 10)
        assert out.min() >= 0.0


# ---------------------------------------------------------------------------
# Special cases reducing to library routines / convergence orders
# ---------------------------------------------------------------------------

def _seird_rhs(beta, alpha, gamma, phi):
    """Right-hand side of Eqs. (EqSEIRD_S..EqSEIRD_D) without diffusion."""
    def f(_t, y):
        S, E, I, R, D = y
        Nc = S + E + I + R
        inf = beta * S * I / Nc
        return [-inf, inf - alpha * E, alpha * E - gamma * I, (1 - phi) * gamma * I, phi * gamma * I]
    return f


def test_uniform_state_converges_to_ode_first_order():
    """North-star check (1): a spatially uniform state has no diffusion, so the
    SSLBM integrates the SEIRD ODE; against scipy's DOP853 the error falls by ~2
    per halving of dt (explicit, first order)."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    rates = (0.6, 1 / 7, 0.2, 0.3)
    y0 = np.array([0.97, 0.02, 0.01, 0.0, 0.0])
    T = 40.0
    ref = scipy_integrate.solve_ivp(_seird_rhs(*rates), (0, T), y0, method="DOP853",
                                    rtol=1e-13, atol=1e-15).y[:, -1]
    errs = []
    for dt in (0.2, 0.1, 0.05):
        st = np.broadcast_to(y0[:, None, None], (5, 2, 3)).copy()
        out = oracle.sslbm_run(st, [0.6] * 4, rates, dt, 1, int(round(T / dt)))
        assert np.ptp(out, axis=(1, 2)).max() < 1e-15  # stays uniform
        errs.append(np.abs(out[:, 0, 0] - ref).max())
    assert errs[0] > 1e-4  # not an exact match: the scheme is explicit Euler in time
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


def test_ode_rk4_fourth_order():
    scipy_integrate = pytest.importorskip("scipy.integrate")
    rates = (0.5, 0.2, 0.11, 1 / 11)
    y0 = np.array([0.95, 0.03, 0.02, 0.0, 0.0])
    T = 50.0
    ref = scipy_integrate.solve_ivp(_seird_rhs(*rates), (0, T), y0, method="DOP853",
                                    rtol=1e-13, atol=1e-15).y[:, -1]
    errs = [np.abs(oracle.ode_rk4(y0, rates, dt, int(round(T / dt))) - ref).max() for dt in (1.0, 0.5, 0.25)]
    for a, b in zip(errs, errs[1:]):
        assert 13.0 < a / b < 19.0


def _diffusion_mode_l2(n, d_lattice, T, scheme):
    """sin(2 pi x) sin(2 pi y) exp(-kappa t), kappa = 2 D (2 pi)^2 on the periodic
    unit square (Sec. III.B), cell centres x = (i + 1/2)/n, dt = d_lattice dx^2 / D."""
    D = 0.1
    dx = 1.0 / n
    dt = d_lattice * dx * dx / D
    steps = int(round(T / dt))
    t_end = steps * dt
    c = (np.arange(n) + 0.5) / n
    shape = np.sin(2 * math.pi * c)[None, :] * np.sin(2 * math.pi * c)[:, None]
    st = np.zeros((5, n, n))
    st[:4] = 1.0 + shape
    if scheme == "sslbm":
        tau = oracle.tau_from_d(D, dx, dt)
        out = oracle.sslbm_run(st, [tau] * 4, NO_REACTION, dt, 0, steps)
    else:
        out = oracle.fd4_rk4_run(st, [D] * 4, NO_REACTION, dx, dt, 0, steps)
    exact = 1.0 + shape * math.exp(-2 * D * (2 * math.pi) ** 2 * t_end)
    return math.sqrt(np.mean((out[0] - exact) ** 2))


def test_sslbm_second_order_convergence_table():
    """Table tab:convergence: the L2 error falls ~4x per halving of dx with dt ~ dx^2.
    The table's own square-grid rows show the same order; its absolute values are not
    reproducible (the dt constant and the final time are not given)."""
    rows = [r for r in _gold("convergence_table.json")["rows"] if r["grid"][0] == r["grid"][1]]
    paper_p = [math.log2(a["l2"] / b["l2"]) for a, b in zip(rows, rows[1:])]
    assert all(abs(p - 2.0) < 0.05 for p in paper_p)
    errs = [_diffusion_mode_l2(n, 0.1, 0.05, "sslbm") for n in (16, 32, 64)]
    ours = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(abs(p - 2.0) < 0.1 for p in ours), ours


def test_fd4_fourth_order_convergence():
    """The FD4 reference of Sec. III is fourth order in space (RK4 error is O(dx^8)
    at dt ~ dx^2)."""
    errs = [_diffusion_mode_l2(n, 0.1, 0.05, "fd4") for n in (12, 24, 48)]
    ours = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(3.7 < p < 4.3 for p in ours), ours


@pytest.mark.parametrize("bc", [0, 1])
def test_fd4_mode_evolution_exact(bc):
    """Classical RK4 applied to a Fourier (or, for no-flux, cell-centred cosine)
    mode of the fourth-order centred Laplacian multiplies it by
    R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 per step, z = dt d (s_x + s_y)/dx^2 with
    s(th) = (-2 cos 2th + 32 cos th - 30)/12 -- the textbook symbol of the stencil."""
    nx, ny, nsteps = 30, 22, 40
    d, dx, dt = 0.07, 1.0, 1.0
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    m, q = 2, 3
    if bc == 0:
        thx, thy = 2 * math.pi * m / nx, 2 * math.pi * q / ny
        shape = np.cos(thx * x + thy * y)
    else:
        thx, thy = math.pi * m / nx, math.pi * q / ny
        shape = np.cos(thx * (x + 0.5)) * np.cos(thy * (y + 0.5))

    def s(th):
        return (-2 * math.cos(2 * th) + 32 * math.cos(th) - 30) / 12

    z = dt * d * (s(thx) + s(thy)) / dx ** 2
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    st = np.zeros((5, ny, nx))
    st[:4] = 1.0 + 0.3 * shape
    out = oracle.fd4_rk4_run(st, [d] * 4, NO_REACTION, dx, dt, bc, nsteps)
    np.testing.assert_allclose(out[0], 1.0 + 0.3 * R ** nsteps * shape, rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", [0, 1])
def test_fd2_mode_evolution_exact(bc):
    """RK4 on a mode of the second-order (5-point) Laplacian multiplies it by R(z) per step,
    z = dt d (s_x + s_y)/dx^2 with the textbook symbol s(th) = 2 cos th - 2."""
    nx, ny, nsteps = 26, 18, 30
    d, dx, dt = 0.09, 1.0, 1.0
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    m, q = 3, 2
    if bc == 0:
        thx, thy = 2 * math.pi * m / nx, 2 * math.pi * q / ny
        shape = np.cos(thx * x + thy * y)
    else:
        thx, thy = math.pi * m / nx, math.pi * q / ny
        shape = np.cos(thx * (x + 0.5)) * np.cos(thy * (y + 0.5))
    z = dt * d * ((2 * math.cos(thx) - 2) + (2 * math.cos(thy) - 2)) / dx ** 2
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    st = np.zeros((5, ny, nx))
    st[:4] = 1.0 + 0.3 * shape
    out = oracle.fd2_rk4_run(st, [d] * 4, NO_REACTION, dx, dt, bc, nsteps)
    np.testing.assert_allclose(out[0], 1.0 + 0.3 * R ** nsteps * shape, rtol=0, atol=1e-13)


def test_fd2_second_order_convergence():
    errs = [_diffusion_mode_l2_fd2(n, 0.1, 0.05) for n in (16, 32, 64)]
    ours = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(abs(p - 2.0) < 0.1 for p in ours), ours


def _diffusion_mode_l2_fd2(n, D, c):
    dx = 1.0 / n
    dt = c * dx * dx / D
    steps = int(round(0.05 / dt))
    t_end = steps * dt
    cc = (np.arange(n) + 0.5) / n
    shape = np.sin(2 * math.pi * cc)[None, :] * np.sin(2 * math.pi * cc)[:, None]
    st = np.zeros((5, n, n))
    st[:4] = 1.0 + shape
    out = oracle.fd2_rk4_run(st, [D] * 4, NO_REACTION, dx, dt, 0, steps)
    exact = 1.0 + shape * math.exp(-2 * D * (2 * math.pi) ** 2 * t_end)
    return math.sqrt(np.mean((out[0] - exact) ** 2))


@pytest.mark.parametrize("bc", [0, 1])
def test_fd4_conserves_population(bc):
    st = inputs.epidemic_state(20, 17, seed=2)
    out = oracle.fd4_rk4_run(st, [0.05, 0.05, 0.01, 0.05], (0.5, 0.2, 0.11, 1 / 11), 1.0, 0.5, bc, 50)
    assert abs(out.sum() - st.sum()) / st.sum() < 1e-13


# ---------------------------------------------------------------------------
# BGK comparison scheme
# ---------------------------------------------------------------------------

def _bgk_mode_matrix(tau, kx, ky):
    """Linear BGK step of Eq. (pdf) for one Fourier mode: collision
    f -> f + (w rho - f)/tau, then pull streaming f_i(x) <- f_i(x - c_i), i.e.
    multiplication by exp(-i k.c_i)."""
    g = _gold("d2q5_lattice.json")
    cx, cy, w = np.array(g["cx"]), np.array(g["cy"]), np.array(g["w"])
    omega = (1 - 1 / tau) * np.eye(5) + (1 / tau) * np.outer(w, np.ones(5))
    shift = np.diag(np.exp(-1j * (kx * cx + ky * cy)))
    return shift @ omega, w


@pytest.mark.parametrize("tau", [0.65, 0.9, 1.4])
def test_bgk_mode_evolution_matches_matrix_power(tau):
    """Reactions off: the density of a mode started at equilibrium evolves as
    1^T M(k)^n w (numpy.linalg.matrix_power)."""
    nx, ny, nsteps = 24, 18, 30
    m, q = 2, 1
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * q / ny
    M, w = _bgk_mode_matrix(tau, kx, ky)
    amp = np.ones(5) @ np.linalg.matrix_power(M, nsteps) @ w
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    st = np.zeros((5, ny, nx))
    st[:4] = 1.0 + 0.25 * np.cos(kx * x + ky * y)
    out = oracle.bgk_run_state(st, [tau] * 4, NO_REACTION, 1.0, 0, nsteps)
    expect = 1.0 + 0.25 * np.real(amp * np.exp(1j * (kx * x + ky * y)))
    np.testing.assert_allclose(out[0], expect, rtol=0, atol=1e-13)


def test_bgk_diffusivity_matches_eq_diffusivity():
    """The slow BGK mode decays at d |k|^2 with d = c_s^2 (tau - 1/2) (Eq. diffusivity)."""
    tau = 0.8
    d = (tau - 0.5) / 3
    n = 128
    k = 2 * math.pi / n
    t = int(round(0.5 / (d * k * k)))
    x = np.arange(n)[None, :]
    st = np.zeros((5, 3, n))
    st[:4] = 1.0 + 0.1 * np.cos(k * x)
    out = oracle.bgk_run_state(st, [tau] * 4, NO_REACTION, 1.0, 0, t)
    amp = (out[0, 0] - 1.0) @ np.cos(k * x[0]) / (0.1 * n / 2)
    assert abs(amp / math.exp(-d * k * k * t) - 1) < 2e-3


@pytest.mark.parametrize("bc", [0, 1])
def test_bgk_conserves_total_population(bc):
    st = inputs.epidemic_state(21, 16, seed=9)
    out = oracle.bgk_run_state(st, [0.65, 0.6, 0.53, 0.7], (0.5, 0.2, 0.11, 1 / 11), 1.0, bc, 200)
    assert abs(out.sum() - st.sum()) / st.sum() < 1e-13


def test_bgk_uniform_state_is_the_same_euler_update():
    """A uniform equilibrium stays at equilibrium (f_i = w_i (rho + Psi dt)), so BGK
    and SSLBM agree on uniform states."""
    st = np.zeros((5, 4, 5))
    st[0], st[1], st[2] = 0.9, 0.06, 0.04
    rates = (0.5, 0.2, 0.11, 1 / 11)
    a = oracle.bgk_run_state(st, [0.7] * 4, rates, 0.5, 1, 40)
    b = oracle.sslbm_run(st, [0.7] * 4, rates, 0.5, 1, 40)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-16)


# ---------------------------------------------------------------------------
# Diagnostics and the windowed evaluation used for full-size sampled parity
# ---------------------------------------------------------------------------

def test_diagnostics_exact_on_integer_fields():
    g = np.random.default_rng(1)
    st = g.integers(0, 1000, size=(5, 33, 47)).astype(np.float64)
    st[2, 5, 7] = 5000.0
    tot, pk = oracle.diagnostics(st)
    assert np.array_equal(tot, st.reshape(5, -1).sum(axis=1))
    assert pk == 5000.0


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("corner", [(0, 0), (30, 5), (44, 33), (13, 20)])
def test_window_equals_full_run(bc, corner):
    st = inputs.epidemic_state(50, 38, seed=4)
    tau, rates, n = [0.65, 0.6, 0.53, 0.7], (0.5, 0.2, 0.11, 1 / 11), 6
    full = oracle.sslbm_run(st, tau, rates, 1.0, bc, n)
    x0, y0 = corner
    w, h = min(6, 50 - x0), min(5, 38 - y0)
    win = oracle.sslbm_window(st, x0, y0, w, h, tau, rates, 1.0, bc, n)
    np.testing.assert_array_equal(win, full[:, y0:y0 + h, x0:x0 + w])


def test_diagnostics_totals_match_exactly_rounded_sum():
    """Totals must be the exact sum to a few ulp (math.fsum is exactly rounded), also
    where plain left-to-right summation loses the small terms."""
    g = np.random.default_rng(7)
    st = g.uniform(0.0, 1.0, (5, 64, 80)) * 1e-12
    st[:, 0, 0] = 1.0  # a large first term swallows 2^-53-sized increments
    st[1] = 2.0 ** -53
    st[1, 0, 0] = 1.0
    tot, _ = oracle.diagnostics(st)
    for c in range(5):
        want = math.fsum(st[c].ravel().tolist())
        assert abs(tot[c] - want) <= 4 * np.spacing(want), (c, tot[c], want)
