"""The D2Q9 SSLBM step on the GPU against the FP64 oracle (oracle.sslbm9_run).

The kernel evaluates the reduced form rho_c + d (4 axes + diagonals - 20 rho_c)/6 + Psi dt;
the oracle keeps the literal rho_b + (tau - 1)(rho_f - 2 rho_c + rho_b); they differ by a
few roundings per step (FP64: 1e-12 relative max-norm over 25 steps, as for D2Q5).  FP32:
each step adds a few FP32 roundings (u = 6e-8) of a contractive update; 25 steps stay
within 1e-5 of the peak.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

RATES = inputs.rates_from_sigma_mu(0.45, 0.2, 0.1, 0.01).as_tuple()
D = (0.05, 0.04, 0.01, 0.08, 0.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def relmax(a, b):
    return max(float(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-300)) for c in range(5))


def _run(nx, ny, bc, precision, steps, state):
    s = L.Solver(nx, ny, RATES, d=D, bc=bc, precision=precision, lattice=L.LATTICE_D2Q9)
    s.write(state if precision == L.FP64 else state.astype(np.float32))
    s.step(steps)
    out = s.read()
    tot, _ = s.diagnostics()
    s.close()
    return out, tot


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(37, 29), (70, 41), (1, 5), (6, 1), (2, 3)])
def test_fp64_matches_oracle(bc, nx, ny):
    st = inputs.epidemic_state(nx, ny, 3 * nx + ny)
    got, tot = _run(nx, ny, bc, L.FP64, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.sslbm9_run(st, tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-12
    # the population is conserved (FP64 diagnostics)
    assert abs(tot.sum() - st.sum()) / st.sum() < 1e-12


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_fp32_matches_oracle(bc):
    st = inputs.epidemic_state(45, 38, 11)
    got, _ = _run(45, 38, bc, L.FP32, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.sslbm9_run(st.astype(np.float32).astype(np.float64), tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-5


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(301, 19), (513, 10), (128, 9), (1, 7), (2, 3), (5, 1)])
def test_fp32_rows_span_warps_and_ragged_tails(bc, nx, ny):
    """A warp covers 32 groups of a row: these widths put the warp's last lane, a ragged last
    group and single-group rows at every kind of edge (periodic wrap and walls)."""
    st = inputs.epidemic_state(nx, ny, 5 * nx + ny)
    got, _ = _run(nx, ny, bc, L.FP32, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.sslbm9_run(st.astype(np.float32).astype(np.float64), tau, RATES, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-5


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_fp64_wide_rows(bc):
    st = inputs.epidemic_state(263, 17, 9)
    got, _ = _run(263, 17, bc, L.FP64, 25, st)
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    assert relmax(got, oracle.sslbm9_run(st, tau, RATES, 1.0, bc, 25)) <= 1e-12


def test_stability_range_and_what_it_does_not_run():
    # tau = 1.5 (d = 1/3) is stable on D2Q9 (<= 13/8) and not on D2Q5 (<= 5/4)
    s = L.Solver(8, 8, RATES, d=(1 / 3, 0.05, 0.05, 0.05, 0.0), lattice=L.LATTICE_D2Q9)
    s.close()
    with pytest.raises(L.SslbmError) as e:
        L.Solver(8, 8, RATES, d=(1 / 3, 0.05, 0.05, 0.05, 0.0))
    assert e.value.status == L.SSLBM_ERR_UNSTABLE
    with pytest.raises(L.SslbmError) as e:
        L.Solver(8, 8, RATES, d=D, lattice=L.LATTICE_D2Q9, schemes=L.WANT_SSLBM | L.WANT_BGK)
    assert e.value.status == L.SSLBM_ERR_UNSUPPORTED
    with pytest.raises(L.SslbmError):
        L.Solver(8, 8, RATES, d=D, lattice=L.LATTICE_D2Q9, precision=L.FP32_DEV)
    # temporal blocking: FP32 only
    s = L.Solver(64, 64, RATES, d=D, lattice=L.LATTICE_D2Q9, precision=L.FP64)
    with pytest.raises(L.SslbmError) as e:
        s.set_blocking(4)
    assert e.value.status == L.SSLBM_ERR_UNSUPPORTED
    s.close()
    s = L.Solver(64, 64, RATES, d=D, lattice=L.LATTICE_D2Q9, precision=L.FP32)
    assert s.get_blocking()[0] == 4  # the default where the blocked kernel exists
    s.set_blocking(8)
    s.close()


def _checkpoint_bits(s):
    return s.checkpoint()[128:].view(np.uint32)


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(131, 77), (257, 130), (64, 300), (120, 45), (5, 7), (1, 1), (2, 9)])
def test_fp32_blocked_depths_give_identical_bits(bc, nx, ny):
    """The temporal-blocked D2Q9 kernel (the pipeline tile with the nine-point stencil and
    the bounce-back substitution at walls) against the one-step kernel, bit for bit: 2k steps
    at depth k are two passes of exactly that depth; then 11 steps, which mix depths.  The
    widths put the strip's halo columns on both sides of the domain and the walls inside a
    lane's four columns."""
    st = inputs.epidemic_state(nx, ny, 7 * nx + ny).astype(np.float32)
    ref = L.Solver(nx, ny, RATES, d=D, bc=bc, precision=L.FP32, lattice=L.LATTICE_D2Q9)
    ref.write(st)
    ref.set_blocking(1)
    refs = {}
    for n in range(1, 17):
        ref.step(1)
        refs[n] = _checkpoint_bits(ref)
    ref.close()
    for k in range(2, 9):
        s = L.Solver(nx, ny, RATES, d=D, bc=bc, precision=L.FP32, lattice=L.LATTICE_D2Q9)
        s.write(st)
        s.set_blocking(k)
        s.step(2 * k)
        assert np.array_equal(_checkpoint_bits(s), refs[2 * k]), (k, nx, ny, bc)
        s.close()
    for k in (3, 8):
        s = L.Solver(nx, ny, RATES, d=D, bc=bc, precision=L.FP32, lattice=L.LATTICE_D2Q9)
        s.write(st)
        s.set_blocking(k)
        s.step(11)
        assert np.array_equal(_checkpoint_bits(s), refs[11]), (k, 11)
        s.close()


@pytest.mark.parametrize("depth,seg_rows", [(3, 12), (3, 50), (8, 32), (8, 41), (6, 100), (7, 28), (2, 8)])
def test_fp32_blocked_segment_lengths_give_identical_bits(depth, seg_rows):
    """2 x depth steps under no-flux: two passes of this depth with this row-segment length
    (segment seams inside the grid and next to the walls)."""
    st = inputs.epidemic_state(300, 333, 5).astype(np.float32)
    ref = L.Solver(300, 333, RATES, d=D, bc=L.BC_NOFLUX, precision=L.FP32, lattice=L.LATTICE_D2Q9)
    ref.write(st)
    ref.set_blocking(1)
    ref.step(2 * depth)
    want = _checkpoint_bits(ref)
    ref.close()
    s = L.Solver(300, 333, RATES, d=D, bc=L.BC_NOFLUX, precision=L.FP32, lattice=L.LATTICE_D2Q9)
    s.write(st)
    s.set_blocking(depth, seg_rows)
    s.step(2 * depth)
    assert np.array_equal(_checkpoint_bits(s), want)
    s.close()


def test_fp32_blocked_long_run_matches_oracle_and_conserves():
    """200 steps at the autotuned blocking against the FP64 oracle (FP32 tolerance), and the
    population conserved to FP32 rounding under no-flux (bounce-back keeps it exactly in
    exact arithmetic)."""
    nx, ny = 96, 70
    st = inputs.epidemic_state(nx, ny, 21)
    s = L.Solver(nx, ny, RATES, d=D, bc=L.BC_NOFLUX, precision=L.FP32, lattice=L.LATTICE_D2Q9)
    s.write(st.astype(np.float32))
    depth, seg, _ = s.autotune(50.0)
    assert 1 <= depth <= 8 and (depth == 1 or seg >= 4 * depth)
    assert np.array_equal(s.read(dtype=np.float32), st.astype(np.float32))  # the tuner left the state
    s.step(200)
    got = s.read()
    tot, _ = s.diagnostics()
    s.close()
    tau = [oracle.tau_from_d(d) for d in D[:4]]
    ref = oracle.sslbm9_run(st.astype(np.float32).astype(np.float64), tau, RATES, 1.0, L.BC_NOFLUX, 200)
    assert relmax(got, ref) <= 1e-4
    s0 = float(st.astype(np.float32).astype(np.float64).sum())
    assert abs(float(tot.sum()) - s0) / s0 < 200 * 4 * 6e-8
