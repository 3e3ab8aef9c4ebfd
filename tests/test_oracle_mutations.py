"""Planted mistakes in a copy of the oracle must make the pin suite fail.

Each case edits one expression of oracle/seird_oracle.c in a temporary copy
(a dropped term, a wrong sign, a swapped rate, a transposed axis, a wrong weight
or boundary rule), builds it, and runs tests/test_oracle_pins.py against that
build in a subprocess (or the routine's own pin file, where the mutant names one).  The
pins pass on the real oracle; every mutant must be caught by at least one of them.  CPU only.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "seird_oracle.c")

MUTANTS = {
    "R_source_drops_1_minus_phi": ("psi[3] = (1.0 - phi) * gamma * I;", "psi[3] = gamma * I;"),
    "E_source_wrong_sign": ("psi[1] = F - alpha * E;", "psi[1] = F + alpha * E;"),
    "I_source_swaps_alpha_gamma": ("psi[2] = alpha * E - gamma * I;", "psi[2] = gamma * E - alpha * I;"),
    "force_without_Nc": ("(beta * S) * I / Nc", "(beta * S) * I"),
    "D_source_drops_phi": ("psi[4] = phi * gamma * I;", "psi[4] = gamma * I;"),
    "rest_weight_wrong": ("W[5] = {1.0 / 3.0,", "W[5] = {1.0 / 6.0,"),
    "y_link_uses_x": ("val(p, nx, ny, bc, x + CX[i], y + CY[i])", "val(p, nx, ny, bc, x + CX[i], y + CX[i])"),
    "tau_minus_half": ("(tau[c] - 1.0) * (rho_f", "(tau[c] - 0.5) * (rho_f"),
    "noflux_wraps": ("return (i < 0) ? 0 : n - 1;", "return (i < 0) ? i + n : i - n;"),
    "tau_from_d_factor": ("return 3.0 * d_lattice + 0.5;", "return 2.0 * d_lattice + 0.5;"),
    "bgk_bounce_back_same_dir": ("v = post[(c * 5 + OPP[i]) * M + k];", "v = post[(c * 5 + i) * M + k];"),
    "bgk_no_source_weight": ("+ W[i] * psi[c] * dt;", "+ psi[c] * dt;"),
    "fd4_coefficient": ("16.0 * p[y * nx + ghost2(x + 1, nx, bc)]", "15.0 * p[y * nx + ghost2(x + 1, nx, bc)]"),
    "rk4_weight": ("y[j] += dt / 6.0 * (k1[j] + 2.0 * k2[j]", "y[j] += dt / 6.0 * (k1[j] + 1.0 * k2[j]"),
    "diagnostics_drop_compensation": ("totals[c] = s + comp;", "totals[c] = s;"),
    # the spatially varying diffusion routine, against its own pins
    "vard_percell_coefficient": ("const double k_link = 0.5 * (kap[k] + val(kap, nx, ny, bc, x + CX[i], y + CY[i]));",
                                 "const double k_link = kap[k];", "test_oracle_vard.py"),
    "vard_axes_swapped": ("const double* kap = CX[i] != 0 ? kx : ky;", "const double* kap = CX[i] != 0 ? ky : kx;",
                          "test_oracle_vard.py"),
    "vard_d_lattice": ("const double d_lattice = (tau[c] - 0.5) / 3.0;", "const double d_lattice = (tau[c] - 0.5) / 6.0;",
                       "test_oracle_vard.py"),
    "vard_link_mean_halved_twice": ("const double k_link = 0.5 * (kap[k]", "const double k_link = 0.25 * (kap[k]",
                                    "test_oracle_vard.py"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new, *pins = MUTANTS[name]
    pins_file = pins[0] if pins else "test_oracle_pins.py"
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    mutated = tmp_path / "seird_oracle_mut.c"
    mutated.write_text(src.replace(old, new, 1))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    "-o", str(lib), str(mutated), "-lm"], check=True)
    env = dict(os.environ, SEIRD_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins_file)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
