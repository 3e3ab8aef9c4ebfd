"""Diagnostics fused into the last pass of sslbm_step (sslbm_set_fused_diagnostics).

The diagnostics are the population totals and the peak of I of Sec. II.C ('Mass
conservation').  The fused pass must write the plain pass's state (the same bits), and the
totals it leaves must agree with the separate reduction and with the oracle's totals of the
read-back state.  Its peak of I must equal theirs exactly, since it is a maximum over the
same FP32 values.

Tolerances:
- Both GPU reductions sum the same FP32 values. Each keeps FP32 TwoSum pairs whose own
  error is of order (values per pair) x u^2 with u = 6e-8, then adds the pairs in FP64. So
  the two agree to 1e-13 relative.
- Against the oracle's FP64 totals of the read-back state: 1e-12, the bound of the
  existing diagnostics tests.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

AGREE = 1e-13
ORACLE = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def workload(nx, ny, bc, seed=3):
    st = inputs.epidemic_state(nx, ny, seed)
    return dict(state=st, rates=inputs.Rates(0.5, 0.2, 0.11, 1 / 11), d=(0.05, 0.05, 0.01, 0.05, 0.0),
                bc=bc)


def solver(wl, precision, schemes=L.WANT_SSLBM):
    _, ny, nx = wl["state"].shape
    return L.Solver(nx, ny, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=precision,
                    schemes=schemes)


def run_pair(wl, precision, depth, seg, n):
    """Two solvers from the same state, fused diagnostics on and off, n steps each."""
    out = []
    for fused in (True, False):
        s = solver(wl, precision)
        s.write(wl["state"])
        s.set_blocking(depth, seg)
        s.set_fused_diagnostics(fused)
        s.step(n)
        out.append(s)
    return out


def check_against_oracle(s, tot, pk):
    otot, opk = oracle.diagnostics(s.read())
    np.testing.assert_allclose(tot, otot, rtol=ORACLE)
    assert pk == pytest.approx(opk, rel=1e-7)


@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV])
@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("depth", [2, 3, 4, 5, 6, 7, 8])
def test_fused_diagnostics_match_the_separate_reduction(precision, bc, depth):
    """A 257 x 131 grid: ragged last strip and lane, several segments.  22 steps make passes
    of unequal depth for most depths, the fused one last."""
    wl = workload(257, 131, bc)
    fu, pl = run_pair(wl, precision, depth, 4 * depth + 4, 22)
    assert fu.get_fused_diagnostics() == (True, True)
    assert pl.get_fused_diagnostics() == (False, False)
    np.testing.assert_array_equal(fu.checkpoint(), pl.checkpoint())
    tf, pf = fu.diagnostics()
    tp, pp = pl.diagnostics()
    np.testing.assert_allclose(tf, tp, rtol=AGREE)
    assert pf == pp
    check_against_oracle(fu, tf, pf)


@pytest.mark.parametrize("shape,seg", [((1000, 333), 0), ((1000, 333), 40), ((96, 40), 32), ((4099, 13), 0),
                                       ((3, 5), 0), ((1, 1), 0), ((129, 2), 0)])
@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_fused_diagnostics_on_ragged_and_tiny_grids(shape, seg, bc):
    nx, ny = shape
    wl = workload(nx, ny, bc, seed=11)
    fu, pl = run_pair(wl, L.FP32, 8, seg, 16)
    assert fu.get_fused_diagnostics() == (True, True)
    np.testing.assert_array_equal(fu.checkpoint(), pl.checkpoint())
    tf, pf = fu.diagnostics()
    tp, pp = pl.diagnostics()
    np.testing.assert_allclose(tf, tp, rtol=AGREE)
    assert pf == pp
    check_against_oracle(fu, tf, pf)


def test_fused_diagnostics_are_reproducible():
    wl = workload(517, 211, L.BC_NOFLUX, seed=5)
    res = []
    for _ in range(2):
        s = solver(wl, L.FP32)
        s.write(wl["state"])
        s.set_blocking(6, 0)
        s.set_fused_diagnostics(True)
        s.step(18)
        tot, pk = s.diagnostics()
        res.append((tot.tobytes(), pk))
    assert res[0] == res[1]


def test_a_write_or_a_checkpoint_load_discards_the_fused_result():
    wl = workload(300, 120, L.BC_PERIODIC, seed=7)
    s = solver(wl, L.FP32)
    s.write(wl["state"])
    s.set_blocking(4, 0)
    s.set_fused_diagnostics(True)
    s.step(12)
    ck = s.checkpoint()
    tot0, pk0 = s.diagnostics()
    # a new state: the diagnostics are those of the written fields
    other = inputs.epidemic_state(300, 120, 99)
    s.write(other)
    assert s.get_fused_diagnostics() == (True, False)
    tot, pk = s.diagnostics()
    otot, opk = oracle.diagnostics(s.read())
    np.testing.assert_allclose(tot, otot, rtol=ORACLE)
    assert not np.allclose(tot, tot0, rtol=1e-9)
    # steps, then a checkpoint load: the loaded state's diagnostics
    s.step(8)
    assert s.get_fused_diagnostics() == (True, True)
    s.restore(ck)
    assert s.get_fused_diagnostics() == (True, False)
    tot, pk = s.diagnostics()
    np.testing.assert_allclose(tot, tot0, rtol=AGREE)
    assert pk == pk0
    # zero steps leave the state and its fused result as they are
    s.step(12)
    tot1, pk1 = s.diagnostics()
    s.step(0)
    tot2, pk2 = s.diagnostics()
    np.testing.assert_array_equal(tot1, tot2)
    assert pk1 == pk2


def test_bgk_diagnostics_between_do_not_leak_into_the_sslbm_ones():
    wl = workload(200, 90, L.BC_NOFLUX, seed=9)
    s = solver(wl, L.FP32, schemes=L.WANT_SSLBM | L.WANT_BGK)
    s.write(wl["state"])
    s.write(wl["state"], scheme=L.SCHEME_BGK)
    s.set_blocking(5, 0)
    s.set_fused_diagnostics(True)
    s.step(20)
    s.bgk_step(3)
    tb, _ = s.diagnostics(scheme=L.SCHEME_BGK)
    ts, ps = s.diagnostics()
    check_against_oracle(s, ts, ps)
    otb, _ = oracle.diagnostics(s.read(scheme=L.SCHEME_BGK))
    np.testing.assert_allclose(tb, otb, rtol=ORACLE)


@pytest.mark.parametrize("precision,depth,seg", [(L.FP32_SPLIT, 4, 0), (L.FP32_KAHAN, 4, 0), (L.FP64, 1, 0),
                                                 (L.FP32, 1, 0), (L.FP32, 2, 0), (L.FP32, 8, 32)])
def test_steps_the_fused_pass_does_not_cover_keep_the_separate_reduction(precision, depth, seg):
    """Storages without the fused pass, one step per launch, depth 2 with an odd step count
    (its last pass is a single step), and (last case: 4096 columns in 37 strips times 32
    segments) a pass of more than 1024 tiles."""
    nx, ny = (4096, 1024) if seg == 32 else (333, 97)
    wl = workload(nx, ny, L.BC_NOFLUX, seed=13)
    s = solver(wl, precision)
    s.write(wl["state"])
    s.set_blocking(depth, seg)
    s.set_fused_diagnostics(True)
    s.step(9)
    assert s.get_fused_diagnostics() == (True, False)
    tot, pk = s.diagnostics()
    check_against_oracle(s, tot, pk)


def test_set_fused_diagnostics_rejects_other_values():
    wl = workload(16, 8, L.BC_PERIODIC)
    s = solver(wl, L.FP32)
    assert L.load().sslbm_set_fused_diagnostics(s.h, 2) == L.SSLBM_ERR_BAD_ARG
    assert L.load().sslbm_set_fused_diagnostics(None, 1) == L.SSLBM_ERR_BAD_ARG
    assert L.load().sslbm_set_fused_diagnostics(s.h, 0) == L.SSLBM_OK
    assert L.load().sslbm_get_fused_diagnostics(None, None, None) == L.SSLBM_ERR_BAD_ARG
    assert s.get_fused_diagnostics() == (False, False)
