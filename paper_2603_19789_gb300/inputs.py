"""Seeded synthetic SEIRD workloads: initial states and parameter sets.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle.  It draws random numbers and lays out initial fields; it holds none
of the scheme's arithmetic (no relaxation times, no sources, no stencil).

States are float64 numpy arrays of shape (5, ny, nx) holding S, E, I, R, D with
x fastest.  Rates are returned in the paper's notation (Table I):
beta (contact rate), alpha (incubation rate), gamma (removal rate), phi
(infection fatality ratio).  Workloads quoted as (beta, sigma, gamma, mu) --
sigma the incubation rate, gamma the recovery rate, mu the death rate of the
infected -- are mapped with alpha = sigma, gamma_paper = gamma + mu,
phi = mu / (gamma + mu), so that I leaves at gamma + mu, R gains gamma I and
D gains mu I, and R0 = beta / (gamma + mu).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEFAULT_SEED = 20260319

BC_PERIODIC = 0
BC_NOFLUX = 1


@dataclasses.dataclass(frozen=True)
class Rates:
    beta: float
    alpha: float
    gamma: float
    phi: float

    def as_tuple(self):
        return (self.beta, self.alpha, self.gamma, self.phi)


def rates_from_sigma_mu(beta: float, sigma: float, gamma: float, mu: float) -> Rates:
    """(beta, sigma, gamma, mu) -> the paper's (beta, alpha, gamma, phi)."""
    removal = gamma + mu
    return Rates(beta=beta, alpha=sigma, gamma=removal, phi=(mu / removal) if removal > 0 else 0.0)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def add_gaussian(I: np.ndarray, cx: float, cy: float, amp: float, sig: float, periodic: bool,
                 radius_sigmas: float = 8.0) -> None:
    """I += amp * exp(-r^2 / (2 sig^2)) around (cx, cy) in cell-index coordinates,
    truncated at radius_sigmas * sig (exp(-32) ~ 1e-14 of the peak at 8 sigmas).
    Periodic domains use the minimum-image distance; no-flux domains clip."""
    ny, nx = I.shape
    r = int(math.ceil(radius_sigmas * sig))
    x_lo, x_hi = int(math.floor(cx)) - r, int(math.floor(cx)) + r + 1
    y_lo, y_hi = int(math.floor(cy)) - r, int(math.floor(cy)) + r + 1
    xs = np.arange(x_lo, x_hi)
    ys = np.arange(y_lo, y_hi)
    if periodic:
        # fold the window onto the torus; a window wider than the domain is reduced to it
        if x_hi - x_lo >= nx:
            xs = np.arange(nx)
        if y_hi - y_lo >= ny:
            ys = np.arange(ny)
        dx = xs - cx
        dy = ys - cy
        dx = dx - nx * np.round(dx / nx)
        dy = dy - ny * np.round(dy / ny)
        xi = np.mod(xs, nx)
        yi = np.mod(ys, ny)
    else:
        xs = xs[(xs >= 0) & (xs < nx)]
        ys = ys[(ys >= 0) & (ys < ny)]
        dx = xs - cx
        dy = ys - cy
        xi, yi = xs, ys
    if xs.size == 0 or ys.size == 0:
        return
    g = amp * np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * sig * sig))
    np.add.at(I, (yi[:, None], xi[None, :]), g)


def state_from_infected(I: np.ndarray, total: float = 1.0) -> np.ndarray:
    """S = total - I, E = R = D = 0."""
    ny, nx = I.shape
    st = np.zeros((5, ny, nx))
    st[2] = I
    st[0] = total - I
    return st


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def centre_bump_workload(nx: int = 128, ny: int = 128, seed: int = DEFAULT_SEED,
                         amp: float = 1e-2, sig: float = 8.0, noise: float = 1e-6):
    """Plain SSLBM workload, 128x128 periodic, lattice units (dx = dt = 1), 2000 steps:
    I0 = a Gaussian bump of amplitude 1e-2 and sigma 8 cells at the domain centre
    plus a seeded uniform [0, 1e-6) perturbation per cell; S = 1 - I0; E = R = D = 0.
    Rates beta=0.3, sigma=0.2, gamma=0.1, mu=0.01; D = 0.05 for S, E, I, R."""
    I = np.zeros((ny, nx))
    add_gaussian(I, (nx - 1) / 2.0, (ny - 1) / 2.0, amp, sig, periodic=True)
    I += noise * _rng(seed).random((ny, nx))
    rates = rates_from_sigma_mu(0.3, 0.2, 0.1, 0.01)
    d = (0.05, 0.05, 0.05, 0.05, 0.0)
    return dict(state=state_from_infected(I), rates=rates, d=d, dx=1.0, dt=1.0,
                bc=BC_PERIODIC, steps=2000, name=f"centre_bump_{nx}x{ny}_periodic")


def multi_seed_infected(nx: int, ny: int, seed: int, n_seeds: int = 64,
                        amp_range=(1e-4, 1e-2), sig_range=(4.0, 32.0), periodic=False,
                        fixed_amp: float | None = None) -> np.ndarray:
    rng = _rng(seed)
    amps = rng.uniform(amp_range[0], amp_range[1], n_seeds)
    sigs = rng.uniform(sig_range[0], sig_range[1], n_seeds)
    cxs = rng.uniform(0.0, nx, n_seeds)
    cys = rng.uniform(0.0, ny, n_seeds)
    if fixed_amp is not None:
        amps = np.full(n_seeds, fixed_amp)
    I = np.zeros((ny, nx))
    for a, s, cx, cy in zip(amps, sigs, cxs, cys):
        add_gaussian(I, cx, cy, float(a), float(s), periodic=periodic)
    return I


def roofline_workload(nx: int = 8192, ny: int = 8192, seed: int = DEFAULT_SEED):
    """Large single-grid workload, no-flux walls, lattice units, 10000 steps:
    64 Gaussian infected seeds (amplitude U[1e-4, 1e-2], sigma U[4, 32] cells) at
    uniform random positions; S = 1 - I; E = R = D = 0.
    d^S = d^E = d^R = 0.05, d^I = 0.01, d^D = 0; beta = 0.5, sigma = 0.2,
    gamma = 0.1, mu = 0.01."""
    I = multi_seed_infected(nx, ny, seed, periodic=False)
    rates = rates_from_sigma_mu(0.5, 0.2, 0.1, 0.01)
    d = (0.05, 0.05, 0.01, 0.05, 0.0)
    return dict(state=state_from_infected(I), rates=rates, d=d, dx=1.0, dt=1.0,
                bc=BC_NOFLUX, steps=10000, name=f"multi_seed_{nx}x{ny}_noflux")


def precision_workload(nx: int = 4096, ny: int = 4096, seed: int = DEFAULT_SEED):
    """Small-increment workload for the precision study: the large-grid workload's
    statistics at 4096x4096 and 50000 steps, with every infected seed at
    amplitude 1e-6."""
    I = multi_seed_infected(nx, ny, seed, periodic=False, fixed_amp=1e-6)
    rates = rates_from_sigma_mu(0.5, 0.2, 0.1, 0.01)
    d = (0.05, 0.05, 0.01, 0.05, 0.0)
    return dict(state=state_from_infected(I), rates=rates, d=d, dx=1.0, dt=1.0,
                bc=BC_NOFLUX, steps=50000, name=f"small_seed_{nx}x{ny}_noflux")


def paper_test_case(chi: float = 0.10, R0: float = 3.0, side_km: int = 200, seed: int = DEFAULT_SEED,
                    bc: int = BC_PERIODIC):
    """The paper's test case (Sec. III) in physical units: a side_km x side_km km^2 domain
    with dx = 1 km (one cell per km^2) and dt = 0.01 day; total population N = 5e6, so the
    uniform density is N/A per cell; E = chi N/A + eps(x), S = N/A - E, I = R = D = 0.
    Rates per day: gamma = 1/5, beta = R0 gamma, alpha = 1/7, phi = 0.3.  Diffusion in
    km^2/day: d^S = d^E = d^R = 4.35e-2, d^I = 1e-4, d^D = 0.  The paper does not give
    eps(x); here it is seeded U[-1e-3, 1e-3] chi N/A per cell, and the boundary is periodic
    unless bc says otherwise."""
    n = int(side_km)
    dens = 5e6 / float(n * n)
    eps = _rng(seed).uniform(-1e-3, 1e-3, (n, n)) * chi * dens
    st = np.zeros((5, n, n))
    st[1] = chi * dens + eps
    st[0] = dens - st[1]
    gamma = 1.0 / 5.0
    rates = Rates(R0 * gamma, 1.0 / 7.0, gamma, 0.3)
    d = (4.35e-2, 4.35e-2, 1e-4, 4.35e-2, 0.0)
    return dict(state=st, rates=rates, d=d, dx=1.0, dt=0.01, bc=bc, density=dens,
                name=f"paper_test_case_{n}km_chi{chi:g}_R0{R0:g}")


ENSEMBLE_SIZES = (256, 384, 512, 768, 1024)


def ensemble_scenarios(n: int = 512, seed: int = DEFAULT_SEED, sizes=ENSEMBLE_SIZES):
    """Ensemble of SEIRD scenarios on periodic square grids of uneven size.
    Per scenario: size uniform over `sizes`; R0 ~ U[1.2, 4.0] with gamma = 0.1,
    mu = 0.01, sigma = 0.2 and beta = R0 (gamma + mu); one diffusivity
    d ~ logU[1e-3, 1e-1] for S, E, I, R (d^D = 0); 1..8 Gaussian infected seeds
    (amplitude U[1e-4, 1e-2], sigma U[4, 32] cells) from the scenario's own seed.
    Returns a list of dicts with nx, ny, rates, d, bc and `seed`; the state is
    built on demand by ensemble_state()."""
    rng = _rng(seed)
    out = []
    for k in range(n):
        size = int(sizes[int(rng.integers(0, len(sizes)))])
        R0 = float(rng.uniform(1.2, 4.0))
        dval = float(10.0 ** rng.uniform(-3.0, -1.0))
        nseeds = int(rng.integers(1, 9))
        sseed = int(rng.integers(0, 2 ** 62))
        rates = rates_from_sigma_mu(R0 * 0.11, 0.2, 0.1, 0.01)
        out.append(dict(index=k, nx=size, ny=size, R0=R0, rates=rates,
                        d=(dval, dval, dval, dval, 0.0), n_seeds=nseeds, seed=sseed,
                        bc=BC_PERIODIC, dx=1.0, dt=1.0))
    return out


def ensemble_state(sc) -> np.ndarray:
    I = multi_seed_infected(sc["nx"], sc["ny"], sc["seed"], n_seeds=sc["n_seeds"], periodic=True)
    return state_from_infected(I)


def random_state(nx: int, ny: int, seed: int, lo: float = 0.05, hi: float = 1.0) -> np.ndarray:
    """Five independent U[lo, hi) fields (tests of invariants and parity)."""
    return _rng(seed).uniform(lo, hi, (5, ny, nx))


def epidemic_state(nx: int, ny: int, seed: int) -> np.ndarray:
    """A mid-epidemic-looking random state: S ~ 0.6..0.9, E, I ~ 0..0.05,
    R ~ 0..0.2, D ~ 0..0.01, smooth in no direction (worst case for stencils)."""
    g = _rng(seed)
    st = np.empty((5, ny, nx))
    st[0] = g.uniform(0.6, 0.9, (ny, nx))
    st[1] = g.uniform(0.0, 0.05, (ny, nx))
    st[2] = g.uniform(0.0, 0.05, (ny, nx))
    st[3] = g.uniform(0.0, 0.2, (ny, nx))
    st[4] = g.uniform(0.0, 0.01, (ny, nx))
    return st


def mobility_fields(nx: int, ny: int, seed: int, kind: str = "regions"):
    """Per-cell diffusivity scale fields (kx, ky), float64 (ny, nx), for the spatially
    varying, anisotropic diffusion variant.  kind="regions": a mobility map of a few
    'cities' (discs of radius U[nx/16, nx/6] with scale U[1.2, 2.0]) on a background of
    U[0.3, 0.7], piecewise constant, with ky = kx times U[0.5, 1.0] (transport faster along
    x); kind="random": every cell and axis independent, U[0.2, 1.8] (the harshest case for
    a discretisation: the coefficient jumps at every link)."""
    rng = _rng(seed)
    if kind == "random":
        return rng.uniform(0.2, 1.8, (ny, nx)), rng.uniform(0.2, 1.8, (ny, nx))
    kx = np.full((ny, nx), rng.uniform(0.3, 0.7))
    for _ in range(int(rng.integers(3, 7))):
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        r = rng.uniform(max(nx, ny) / 16, max(nx, ny) / 6)
        y0, y1 = max(0, int(cy - r)), min(ny, int(cy + r) + 1)
        x0, x1 = max(0, int(cx - r)), min(nx, int(cx + r) + 1)
        y = np.arange(y0, y1)[:, None]
        x = np.arange(x0, x1)[None, :]
        box = kx[y0:y1, x0:x1]
        box[(x - cx) ** 2 + (y - cy) ** 2 <= r * r] = rng.uniform(1.2, 2.0)
    ky = kx * rng.uniform(0.5, 1.0)
    return kx, ky
