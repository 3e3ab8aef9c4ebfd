"""Full-size checks of the other configurations bench.py times on the 8192 x 8192 no-flux
multi-seed workload.

Covered: the deviation, split and Kahan storages of D2Q5, and the FP32 D2Q9 and
varying-diffusion lattices.  Each runs at the blocking the library's autotuner picks on
this grid, the call bench.py makes.

Checks per configuration:
- A blocked run of 48 steps (the benchmark's batch for these variants) gives the bits of
  the one-step kernel over the whole grid.  The one-step kernels' own parity with the oracle
  is tested on smaller grids.
- The diagnostics of the blocked result match the oracle's totals of the read-back state to
  1e-12, and its peak of I.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

N = 8192
STEPS = 48


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


@pytest.fixture(scope="module")
def workload():
    return inputs.roofline_workload()


@pytest.mark.parametrize("precision,lattice", [(L.FP32_DEV, L.LATTICE_D2Q5), (L.FP32_SPLIT, L.LATTICE_D2Q5),
                                               (L.FP32_KAHAN, L.LATTICE_D2Q5), (L.FP32, L.LATTICE_D2Q9),
                                               (L.FP32, L.LATTICE_D2Q5_VARD)])
def test_autotuned_blocking_gives_the_one_step_bits_at_full_size(workload, precision, lattice):
    import torch
    wl = workload
    s = L.Solver(N, N, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=precision, lattice=lattice)
    if lattice == L.LATTICE_D2Q5_VARD:
        s.set_diffusivity_scale(*inputs.mobility_fields(N, N, 7))
    s.write(wl["state"])
    depth, seg, _ = s.autotune(300.0)
    print(f"precision {precision} lattice {lattice}: autotuned depth {depth}, seg_rows {seg}")
    assert depth >= 2  # the blocked kernel, as in the benchmark's figure
    start = s.checkpoint(on_device=True)
    s.step(STEPS)
    blocked = s.checkpoint(on_device=True)
    tot, pk = s.diagnostics()
    otot, opk = oracle.diagnostics(s.read())
    np.testing.assert_allclose(tot, otot, rtol=1e-12)
    assert pk == pytest.approx(opk, rel=1e-7)
    s.restore(start)
    s.set_blocking(1)
    s.step(STEPS)
    ref = s.checkpoint(on_device=True)
    assert torch.equal(blocked, ref)
    s.close()


def test_double_word_at_full_size_matches_the_oracle_on_windows(workload):
    """The FP64-accurate double word (bench.py's fp64_dw_glups), 8 steps of the 8192^2 grid:
    sampled 8 x 8 windows against the oracle, which evaluates each on its domain of dependence.
    Errors are measured against each compartment's largest value on the grid: outside the
    seeds I and E fall below FP32's exponent range, which a double word of floats shares."""
    wl = workload
    steps = 8
    s = L.Solver(N, N, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=L.FP64_DW)
    s.write(wl["state"])
    s.step(steps)
    got = s.read()
    scale = np.abs(got).reshape(5, -1).max(axis=1)
    tau = [oracle.tau_from_d(v) for v in wl["d"][:4]]
    g = np.random.default_rng(5)
    pts = [(0, 0), (N - 8, 0), (0, N - 8), (N - 8, N - 8), (N // 2, N // 3)]
    pts += [(int(g.integers(0, N - 8)), int(g.integers(0, N - 8))) for _ in range(20)]
    # on the seeds: the largest initial I in each quadrant
    I0 = wl["state"][2]
    h = N // 2
    for qy in (0, h):
        for qx in (0, h):
            y, x = np.unravel_index(np.argmax(I0[qy:qy + h, qx:qx + h]), (h, h))
            pts.append((min(max(qx + x - 4, 0), N - 8), min(max(qy + y - 4, 0), N - 8)))
    for x0, y0 in pts:
        want = oracle.sslbm_window(wl["state"], x0, y0, 8, 8, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], steps)
        part = got[:, y0:y0 + 8, x0:x0 + 8]
        for c in range(5):
            assert np.abs(part[c] - want[c]).max() <= 1e-12 * scale[c], (x0, y0, c)
    s.close()
