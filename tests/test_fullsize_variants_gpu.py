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
