"""The allocation-free diagnostics entry point against the workspace-based one.

sslbm_diagnostics_noalloc serves callers that hold device buffers but cannot allocate
device memory (for example a monitoring hook inside another framework's time loop,
whose memory pool owns the free device memory), so they cannot create a solver with
its workspace.  Its scratch is a built-in device array shared by all calls; these
tests call it twice in a row on different fields -- the second call with fewer rows,
so stale partial sums from the first call would show -- and compare each result with
sslbm_diagnostics on the same state, within the tolerance the diagnostics tests use.
This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def _reference_and_fields(nx, ny, precision, seed, steps):
    import torch
    st = inputs.epidemic_state(nx, ny, seed)
    s = L.Solver(nx, ny, (0.5, 0.2, 0.11, 1 / 11), d=(0.05, 0.05, 0.01, 0.05, 0.0), bc=L.BC_NOFLUX,
                 precision=precision)
    s.write(st)
    s.step(steps)
    tot, pk = s.diagnostics()
    dtype = torch.float64 if precision == L.FP64 else torch.float32
    fields = torch.empty((5, ny, nx), dtype=dtype, device="cuda")
    L.sslbm_read(s.h, L.SCHEME_SSLBM, L.ALL, fields)
    torch.cuda.synchronize()
    s.close()
    return tot, pk, fields


@pytest.mark.parametrize("precision", [L.FP32, L.FP64])
def test_noalloc_matches_workspace_diagnostics_twice(precision):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(700, 900, 1, 12), (333, 250, 2, 7)]  # second call: fewer rows than the first
    for nx, ny, seed, steps in cases:
        tot, pk, fields = _reference_and_fields(nx, ny, precision, seed, steps)
        got_tot, got_pk = L.sslbm_diagnostics_noalloc(fields, stream)
        np.testing.assert_allclose(got_tot, tot, rtol=RTOL)
        assert got_pk == pk


def test_noalloc_rejects_rows_beyond_its_scratch():
    import torch
    fields = torch.zeros((5, 16385, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_diagnostics_noalloc(fields)
    assert ei.value.status == -1 and "16384" in str(ei.value)
    ok = torch.ones((5, 16384, 1), dtype=torch.float32, device="cuda")
    tot, pk = L.sslbm_diagnostics_noalloc(ok)
    assert np.array_equal(tot, np.full(5, 16384.0)) and pk == 1.0
