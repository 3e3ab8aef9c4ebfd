"""The index-checked debug build (libsslbm_check.so, SSLBM_BOUNDS_CHECK).

compute-sanitizer is not available on these GPUs, so the library has a build in which the
hot-path kernels -- the fused pipeline tile (single grid and ensemble), the one-step
kernels (the streaming kernel of the FP32 storages, the D2Q9 lattice and the varying
diffusion among them), the BGK step and the diagnostics -- test every row and column index
of their global loads and stores before using it, skip and record any that is out of range.
This test compiles that build and, in a child process that loads it, drives a sweep of tiny,
odd and non-multiple-of-tile grids through every precision, every blocking depth with
default and short odd segments, both boundary conditions, BGK, the FP32 D2Q9 and
varying-diffusion steps (one-step and blocked at every depth), the diagnostics (separate, and
fused into the last pass at every depth) and a mixed-size ensemble.  The checks must record nothing.  A probe first proves the recording path: one
check of an index past its limit (no memory access behind it) is counted and reported with
its value, limit and site; one inside is not.
"""
import json
import os
import subprocess
import sys

import pytest

from paper_2603_19789_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SWEEP = r"""
import json
import numpy as np
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

L.load()
out = {}
L.sslbm_debug_bounds_probe(5, 3)
out["probe_out"] = L.sslbm_debug_bounds()
L.sslbm_debug_bounds_probe(2, 3)
out["probe_in"] = L.sslbm_debug_bounds()

rates = inputs.rates_from_sigma_mu(0.45, 0.2, 0.1, 0.01).as_tuple()
d = (0.05, 0.04, 0.01, 0.08, 0.0)
sizes = [(1, 1), (2, 3), (3, 2), (5, 7), (8, 8), (31, 33), (127, 9), (129, 130), (257, 66), (112, 45), (113, 17)]
runs = 0
for nx, ny in sizes:
    st = inputs.epidemic_state(nx, ny, 7 * nx + ny)
    for bc in (L.BC_PERIODIC, L.BC_NOFLUX):
        for prec in (L.FP64, L.FP32, L.FP32_DEV, L.FP32_KAHAN, L.FP32_SPLIT, L.FP64_DW):
            both = prec in (L.FP64, L.FP32)
            s = L.Solver(nx, ny, rates, d=d, bc=bc, precision=prec,
                         schemes=(L.WANT_SSLBM | L.WANT_BGK) if both else L.WANT_SSLBM)
            s.write(st)
            for k in range(1, 9):
                for seg in ((0, 4 * k + 1) if k > 1 else (0,)):
                    try:
                        s.set_blocking(k, seg)
                    except L.SslbmError as e:
                        assert e.status == L.SSLBM_ERR_UNSUPPORTED and k > 1
                        continue
                    s.step(2 * k + 1)
                    runs += 1
            s.diagnostics()
            if prec in (L.FP32, L.FP32_DEV):  # the pipeline with the fused diagnostics
                s.set_fused_diagnostics(True)
                for k in range(2, 9):
                    for seg in (0, 4 * k + 1):
                        s.set_blocking(k, seg)
                        s.step(2 * k)
                        s.diagnostics()
                        runs += 1
                s.set_fused_diagnostics(False)
            if both:
                s.write(st, scheme=L.SCHEME_BGK)
                s.bgk_step(3)
                s.diagnostics(L.SCHEME_BGK)
            s.close()
        for lat in (L.LATTICE_D2Q9, L.LATTICE_D2Q5_VARD):
            s = L.Solver(nx, ny, rates, d=d, bc=bc, precision=L.FP32, lattice=lat)
            if lat == L.LATTICE_D2Q5_VARD:
                s.set_diffusivity_scale(*inputs.mobility_fields(nx, ny, 3))
            s.write(st)
            s.step(3)
            runs += 1
            for k in range(1, 9):  # the blocked kernels at every depth
                for seg in ((0, 4 * k + 1) if k > 1 else (0,)):
                    s.set_blocking(k, seg)
                    s.step(2 * k + 1)
                    runs += 1
            s.close()
out["runs"] = runs

specs = []
for i, (nx, ny) in enumerate([(64, 64), (132, 40), (4, 7), (520, 130), (12, 300), (36, 9)]):
    r = inputs.rates_from_sigma_mu(0.3 + 0.05 * i, 0.2, 0.1, 0.01)
    specs.append(dict(nx=nx, ny=ny, rates=r.as_tuple(), d=(0.03, 0.03, 0.02, 0.03, 0.0)))
for depth, seg in ((2, 9), (4, 17), (8, 33)):
    ens = L.Ensemble(specs)
    ens.set_tiling(depth, seg)
    for i, sp in enumerate(specs):
        ens.write(i, inputs.epidemic_state(sp["nx"], sp["ny"], 40 + i))
    ens.run(2 * depth + 1)
    ens.diagnostics()
    ens.close()
out["sweep"] = L.sslbm_debug_bounds()
print("RESULT " + json.dumps(out))
"""


def test_checked_build_records_no_out_of_range_index():
    lib = build.build(checked=True)
    env = dict(os.environ, SSLBM_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", SWEEP], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    assert out["probe_out"] == {"count": 1, "value": 5, "limit": 3, "site": 1299}
    assert out["probe_in"] == {"count": 0, "value": 0, "limit": 0, "site": -1}
    assert out["runs"] > 1500
    assert out["sweep"]["count"] == 0, out["sweep"]
