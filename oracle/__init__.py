"""FP64 CPU oracle for the SEIRD SSLBM / BGK / FD4 schemes (arXiv 2603.19789).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The product library never imports, links
or calls anything here, and nothing here imports the product package.

The arithmetic lives in ``seird_oracle.c`` (plain loops, double precision, one
routine per equation of the paper); this module compiles it with gcc, loads it
with ctypes and converts numpy arrays.  States are float64 arrays of shape
(5, ny, nx) holding S, E, I, R, D; BGK populations have shape (4, 5, ny, nx).
Boundary codes: 0 periodic, 1 no-flux (cell-centred mirror).

Parity status of each routine (the pins live in tests/test_oracle_pins.py):
  sslbm_step/run   pinned: exact Fourier-mode amplification (periodic and
                   no-flux cosine modes), DFE Jacobian of Eq. (jacobian),
                   discrete growth rate from Eq. (eigenvalues), homogeneity,
                   exact population conservation Eq. (mass_conservation),
                   second-order convergence (Table tab:convergence),
                   first-order convergence of the uniform state to the ODE.
  bgk_step/run     pinned: Fourier-mode evolution vs the 5x5 mode matrix power,
                   diffusivity Eq. (diffusivity), conservation, uniform -> Euler.
  fd4_rk4_run      pinned: exact RK4-of-FD4-symbol mode evolution, fourth-order
                   spatial convergence against the analytic diffusion mode.
  ode_rk4          pinned: fourth-order convergence against scipy's DOP853.
  diagnostics      pinned: exact sums of integer-valued fields, known maxima.
  sslbm9_run       pinned (tests/test_oracle_d2q9.py): exact mode factor with the D2Q9
                   symbol, fourth-order isotropy, conservation, brute force.
  slbm_run         pinned (tests/test_oracle_slbm.py): exact predictor-corrector mode
                   factor, conservation, brute force.
  sslbm_vard_run   pinned (tests/test_oracle_vard.py): uniform fields give the SSLBM,
                   conservation, symmetric operator, exact anisotropic mode factor,
                   maximum principle, brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seird_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile seird_oracle.c into liboracle.so next to it (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # SEIRD_ORACLE_LIB: load a prebuilt copy instead (the mutation tests point it at
        # deliberately broken builds to show that the pins catch them)
        override = os.environ.get("SEIRD_ORACLE_LIB")
        if override:
            lib = ctypes.CDLL(override)
        else:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_tau_from_d.restype = ctypes.c_double
        lib.oracle_tau_from_d.argtypes = [ctypes.c_double] * 3
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_sslbm_step.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp]
        lib.oracle_sslbm_run.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double, _i64, _dp, _dp]
        lib.oracle_sslbm9_run.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double, _i64, _dp, _dp]
        lib.oracle_slbm_run.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double, _i64, _dp, _dp]
        lib.oracle_sslbm_vard_run.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp,
                                              _i64, _dp, _dp]
        lib.oracle_bgk_init.argtypes = [_i64, _i64, _dp, _dp]
        lib.oracle_bgk_density.argtypes = [_i64, _i64, _dp, _dp]
        lib.oracle_bgk_step.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, _dp]
        lib.oracle_bgk_run.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double, _i64, _dp, _dp]
        lib.oracle_fd4_rk4_run.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                           ctypes.c_double, _i64, _dp]
        lib.oracle_fd2_rk4_run.argtypes = [_i64, _i64, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                           ctypes.c_double, _i64, _dp]
        lib.oracle_ode_rk4.argtypes = [_dp, ctypes.c_double, _i64, _dp]
        lib.oracle_sources.argtypes = [_dp, _dp, _dp]
        lib.oracle_diagnostics.argtypes = [_i64, _i64, _dp, _dp, _dp]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _vec(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    assert a.size == n, (a.size, n)
    return a


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def tau_from_d(d: float, dx: float = 1.0, dt: float = 1.0) -> float:
    """Eq. (diffusivity): tau = 3 d dt / dx^2 + 1/2."""
    return float(_load().oracle_tau_from_d(float(d), float(dx), float(dt)))


def rates_vec(beta: float, alpha: float, gamma: float, phi: float) -> np.ndarray:
    return np.array([beta, alpha, gamma, phi], dtype=np.float64)


def sources(rates, rho4) -> np.ndarray:
    """Psi^S, Psi^E, Psi^I, Psi^R of Eq. (sources) and phi*gamma*I of Eq. (rhoD)."""
    lib = _load()
    r = _vec(rates, 4)
    x = _vec(rho4, 4)
    out = np.zeros(5)
    lib.oracle_sources(_ptr(r), _ptr(x), _ptr(out))
    return out


def _state(state) -> np.ndarray:
    s = np.array(state, dtype=np.float64, order="C", copy=True)
    assert s.ndim == 3 and s.shape[0] == 5, s.shape
    return s


def sslbm_step(state, tau, rates, dt: float = 1.0, bc: int = 0) -> np.ndarray:
    """One SSLBM step (Eq. sslbm_final_clean + Eq. rhoD) of a (5, ny, nx) state."""
    lib = _load()
    a = _state(state)
    out = np.empty_like(a)
    _, ny, nx = a.shape
    lib.oracle_sslbm_step(nx, ny, int(bc), _ptr(_vec(tau, 4)), _ptr(_vec(rates, 4)), float(dt),
                          _ptr(a), _ptr(out))
    return out


def sslbm_run(state, tau, rates, dt: float = 1.0, bc: int = 0, nsteps: int = 1) -> np.ndarray:
    """nsteps SSLBM steps; returns the new (5, ny, nx) state."""
    lib = _load()
    a = _state(state)
    scratch = np.empty_like(a)
    _, ny, nx = a.shape
    lib.oracle_sslbm_run(nx, ny, int(bc), _ptr(_vec(tau, 4)), _ptr(_vec(rates, 4)), float(dt),
                         int(nsteps), _ptr(a), _ptr(scratch))
    return a


def sslbm9_run(state, tau, rates, dt: float = 1.0, bc: int = 0, nsteps: int = 1) -> np.ndarray:
    """nsteps SSLBM steps on the D2Q9 lattice; returns the new (5, ny, nx) state."""
    lib = _load()
    a = _state(state)
    scratch = np.empty_like(a)
    _, ny, nx = a.shape
    lib.oracle_sslbm9_run(nx, ny, int(bc), _ptr(_vec(tau, 4)), _ptr(_vec(rates, 4)), float(dt),
                          int(nsteps), _ptr(a), _ptr(scratch))
    return a


def slbm_run(state, tau, rates, dt: float = 1.0, bc: int = 0, nsteps: int = 1) -> np.ndarray:
    """nsteps of the two-pass SLBM (predictor-corrector); returns the new (5, ny, nx) state."""
    lib = _load()
    a = _state(state)
    scratch = np.empty_like(a)
    _, ny, nx = a.shape
    lib.oracle_slbm_run(nx, ny, int(bc), _ptr(_vec(tau, 4)), _ptr(_vec(rates, 4)), float(dt),
                        int(nsteps), _ptr(a), _ptr(scratch))
    return a


def sslbm_vard_run(state, tau, rates, kx, ky, dt: float = 1.0, bc: int = 0, nsteps: int = 1) -> np.ndarray:
    """nsteps of the SSLBM with per-cell diffusivity scale fields kx, ky ((ny, nx) each) in
    the link form (the spatially varying, anisotropic extension of Sec. IV, as read here);
    returns the new (5, ny, nx) state."""
    lib = _load()
    a = _state(state)
    scratch = np.empty_like(a)
    _, ny, nx = a.shape
    fx = np.ascontiguousarray(kx, dtype=np.float64)
    fy = np.ascontiguousarray(ky, dtype=np.float64)
    assert fx.shape == (ny, nx) and fy.shape == (ny, nx), (fx.shape, fy.shape, (ny, nx))
    lib.oracle_sslbm_vard_run(nx, ny, int(bc), _ptr(_vec(tau, 4)), _ptr(_vec(rates, 4)), float(dt), _ptr(fx),
                              _ptr(fy), int(nsteps), _ptr(a), _ptr(scratch))
    return a


def sslbm_run_inplace(state: np.ndarray, scratch: np.ndarray, tau, rates, dt: float = 1.0,
                      bc: int = 0, nsteps: int = 1) -> None:
    """sslbm_run on caller-owned float64 (5, ny, nx) buffers, without copies (used to
    time the oracle itself)."""
    lib = _load()
    _, ny, nx = state.shape
    assert scratch.shape == state.shape
    lib.oracle_sslbm_run(nx, ny, int(bc), _ptr(_vec(tau, 4)), _ptr(_vec(rates, 4)), float(dt),
                         int(nsteps), _ptr(state), _ptr(scratch))


def bgk_init(state):
    """Equilibrium initialisation f_i = w_i rho; returns (f (4,5,ny,nx), D (ny,nx))."""
    lib = _load()
    a = _state(state)
    _, ny, nx = a.shape
    f = np.empty((4, 5, ny, nx))
    lib.oracle_bgk_init(nx, ny, _ptr(a), _ptr(f))
    return f, a[4].copy()


def bgk_density(f, D) -> np.ndarray:
    """rho^C = sum_i f_i^C plus D -> a (5, ny, nx) state."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, _, ny, nx = f.shape
    out = np.empty((5, ny, nx))
    lib.oracle_bgk_density(nx, ny, _ptr(f), _ptr(out))
    out[4] = D
    return out


def bgk_run(f, D, tau, rates, dt: float = 1.0, bc: int = 0, nsteps: int = 1):
    lib = _load()
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    D = np.array(D, dtype=np.float64, order="C", copy=True)
    _, _, ny, nx = f.shape
    lib.oracle_bgk_run(nx, ny, int(bc), _ptr(_vec(tau, 4)), _ptr(_vec(rates, 4)), float(dt),
                       int(nsteps), _ptr(f), _ptr(D))
    return f, D


def bgk_run_state(state, tau, rates, dt: float = 1.0, bc: int = 0, nsteps: int = 1) -> np.ndarray:
    """BGK from the equilibrium of `state`, returned as densities (5, ny, nx)."""
    f, D = bgk_init(state)
    f, D = bgk_run(f, D, tau, rates, dt, bc, nsteps)
    return bgk_density(f, D)


def fd4_rk4_run(state, d, rates, dx: float = 1.0, dt: float = 1.0, bc: int = 0, nsteps: int = 1):
    """Fourth-order FD + RK4 reference of Sec. III; d holds d^S, d^E, d^I, d^R (physical)."""
    lib = _load()
    a = _state(state)
    _, ny, nx = a.shape
    lib.oracle_fd4_rk4_run(nx, ny, int(bc), _ptr(_vec(d, 4)), _ptr(_vec(rates, 4)), float(dx),
                           float(dt), int(nsteps), _ptr(a))
    return a


def fd2_rk4_run(state, d, rates, dx: float = 1.0, dt: float = 1.0, bc: int = 0, nsteps: int = 1):
    """Second-order FD (5-point Laplacian) + RK4: the "FDM 2nd" of the cost comparison."""
    lib = _load()
    a = _state(state)
    _, ny, nx = a.shape
    lib.oracle_fd2_rk4_run(nx, ny, int(bc), _ptr(_vec(d, 4)), _ptr(_vec(rates, 4)), float(dx),
                           float(dt), int(nsteps), _ptr(a))
    return a


def ode_rk4(y0, rates, dt: float, nsteps: int) -> np.ndarray:
    """Homogeneous SEIRD ODE integrated by RK4 from y0 = (S, E, I, R, D)."""
    lib = _load()
    y = _vec(y0, 5).copy()
    lib.oracle_ode_rk4(_ptr(_vec(rates, 4)), float(dt), int(nsteps), _ptr(y))
    return y


def diagnostics(state):
    """(totals[5], peak_I): compensated per-compartment sums and max of I."""
    lib = _load()
    a = np.ascontiguousarray(state, dtype=np.float64)
    _, ny, nx = a.shape
    tot = np.zeros(5)
    pk = np.zeros(1)
    lib.oracle_diagnostics(nx, ny, _ptr(a), _ptr(tot), _ptr(pk))
    return tot, float(pk[0])


def sslbm_window(state_full, x0: int, y0: int, w: int, h: int, tau, rates, dt: float, bc: int,
                 nsteps: int):
    """SSLBM result on the cells [y0, y0+h) x [x0, x0+w) of a large grid after nsteps,
    computed on the window's domain of dependence only.

    The D2Q5 step reads neighbours one link away, so after nsteps a cell depends
    only on cells within nsteps links.  The window is grown by nsteps on every side
    (wrapped for a periodic domain, clipped at real walls for a no-flux one), the
    oracle runs on it with mirror edges, and only the requested cells are returned:
    the artificial edges of the grown window cannot reach them in nsteps steps.
    Returns (5, h, w).
    """
    s = np.asarray(state_full)
    _, ny, nx = s.shape
    m = int(nsteps)
    if bc == 0:
        ys = np.arange(y0 - m, y0 + h + m) % ny
        xs = np.arange(x0 - m, x0 + w + m) % nx
        if len(ys) > ny or len(xs) > nx:  # window wider than the domain: run in full
            full = sslbm_run(s, tau, rates, dt, bc, nsteps)
            return full[:, y0:y0 + h, x0:x0 + w]
        sub = s[:, ys][:, :, xs]
        res = sslbm_run(sub, tau, rates, dt, 1, nsteps)
        return res[:, m:m + h, m:m + w]
    ya, yb = max(0, y0 - m), min(ny, y0 + h + m)
    xa, xb = max(0, x0 - m), min(nx, x0 + w + m)
    sub = s[:, ya:yb, xa:xb]
    res = sslbm_run(sub, tau, rates, dt, 1, nsteps)
    return res[:, y0 - ya:y0 - ya + h, x0 - xa:x0 - xa + w]
