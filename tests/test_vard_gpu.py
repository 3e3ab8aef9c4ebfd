"""The SSLBM with spatially varying, anisotropic diffusion on the GPU (lattice
LATTICE_D2Q5_VARD, sslbm_set_diffusivity_scale) against the FP64 oracle
(oracle.sslbm_vard_run).

The kernel forms the four link coefficients as the oracle does and sums the flux terms as
((+x) + (-x)) + ((+y) + (-y)) (the oracle: in link order), each operation rounded once; the
update itself uses the library's fused form of
Eq. (sslbm_final_clean) (rho_c + d flux with FMA, sources with dt folded into the rates),
so FP64 agrees to a few roundings per step: 1e-12 relative max-norm over 25 steps, as for
the constant-diffusivity kernel.  FP32 evaluates the same expressions in single
precision, with the scale fields rounded to FP32 (the oracle gets the same rounded fields
and state): 25 steps of a contractive update stay within 1e-5 of the peak.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

RATES = inputs.rates_from_sigma_mu(0.45, 0.2, 0.1, 0.01).as_tuple()
D = (0.05, 0.04, 0.01, 0.08, 0.0)
TAU = [oracle.tau_from_d(d) for d in D[:4]]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def relmax(a, b):
    return max(float(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-300)) for c in range(5))


def _solver(nx, ny, bc, precision, d=D):
    return L.Solver(nx, ny, RATES, d=d, bc=bc, precision=precision, lattice=L.LATTICE_D2Q5_VARD)


@pytest.mark.parametrize("kind", ["random", "regions"])
@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(37, 29), (70, 41), (263, 17), (1, 5), (6, 1), (2, 3)])
def test_fp64_matches_oracle(bc, nx, ny, kind):
    st = inputs.epidemic_state(nx, ny, 3 * nx + ny)
    kx, ky = inputs.mobility_fields(nx, ny, nx + 5 * ny, kind)
    s = _solver(nx, ny, bc, L.FP64)
    s.set_diffusivity_scale(kx, ky)
    s.write(st)
    s.step(25)
    got = s.read()
    tot, _ = s.diagnostics()
    s.close()
    ref = oracle.sslbm_vard_run(st, TAU, RATES, kx, ky, 1.0, bc, 25)
    assert relmax(got, ref) <= 1e-12
    assert abs(tot.sum() - st.sum()) / st.sum() < 1e-12  # the population is conserved


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(45, 38), (301, 19), (513, 10), (3, 7)])
def test_fp32_matches_oracle(bc, nx, ny):
    st = inputs.epidemic_state(nx, ny, 11 + nx).astype(np.float32)
    kx, ky = (f.astype(np.float32) for f in inputs.mobility_fields(nx, ny, 4 + ny, "random"))
    s = _solver(nx, ny, bc, L.FP32)
    s.set_diffusivity_scale(kx, ky)
    s.write(st)
    s.step(25)
    got = s.read()
    s.close()
    ref = oracle.sslbm_vard_run(st.astype(np.float64), TAU, RATES, kx.astype(np.float64), ky.astype(np.float64),
                                1.0, bc, 25)
    assert relmax(got, ref) <= 1e-5


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
def test_uniform_fields_are_the_constant_diffusivity_solver(bc):
    st = inputs.epidemic_state(90, 33, 2)
    s = _solver(90, 33, bc, L.FP64)
    s.set_diffusivity_scale(np.ones((33, 90)))  # ky = kx
    s.write(st)
    s.step(30)
    a = s.read()
    s.close()
    c = L.Solver(90, 33, RATES, d=D, bc=bc, precision=L.FP64)
    c.write(st)
    c.step(30)
    b = c.read()
    c.close()
    assert relmax(a, b) <= 1e-13


def test_device_fields_and_isotropic_default():
    import torch
    nx, ny = 130, 21
    st = inputs.epidemic_state(nx, ny, 8)
    kx, _ = inputs.mobility_fields(nx, ny, 3, "random")
    s = _solver(nx, ny, L.BC_NOFLUX, L.FP64)
    s.set_diffusivity_scale(torch.from_numpy(kx.astype(np.float32)).cuda())  # FP32 device source, ky = kx
    s.write(st)
    s.step(10)
    got = s.read()
    s.close()
    k32 = kx.astype(np.float32).astype(np.float64)
    ref = oracle.sslbm_vard_run(st, TAU, RATES, k32, k32, 1.0, L.BC_NOFLUX, 10)
    assert relmax(got, ref) <= 1e-12


def test_validation_and_what_it_does_not_run():
    nx, ny = 16, 12
    s = _solver(nx, ny, L.BC_PERIODIC, L.FP64)
    s.write(inputs.epidemic_state(nx, ny, 1))
    with pytest.raises(L.SslbmError) as e:
        s.step(1)  # no fields yet
    assert e.value.status == L.SSLBM_ERR_BAD_ARG
    k = np.ones((ny, nx))
    bad = k.copy()
    bad[3, 4] = -0.1
    with pytest.raises(L.SslbmError) as e:
        s.set_diffusivity_scale(bad)
    assert e.value.status == L.SSLBM_ERR_BAD_ARG
    bad[3, 4] = np.nan
    with pytest.raises(L.SslbmError) as e:
        s.set_diffusivity_scale(k, bad)
    assert e.value.status == L.SSLBM_ERR_BAD_ARG
    # d = 0.08 (d_lattice 0.08): a link sum above 12.5 leaves the centre weight negative
    big = k.copy()
    big[5, 5] = 20.0
    with pytest.raises(L.SslbmError) as e:
        s.set_diffusivity_scale(big)
    assert e.value.status == L.SSLBM_ERR_UNSTABLE
    with pytest.raises(L.SslbmError):
        s.step(1)  # a failed call leaves the solver without fields
    s.set_diffusivity_scale(k)
    s.step(2)
    with pytest.raises(L.SslbmError) as e:
        s.set_blocking(4)  # temporal blocking: FP32 only
    assert e.value.status == L.SSLBM_ERR_UNSUPPORTED
    s.close()
    # the fields decide stability: tau = 1.4 (d = 0.3) runs with small fields
    s = _solver(nx, ny, L.BC_NOFLUX, L.FP64, d=(0.3, 0.05, 0.05, 0.05, 0.0))
    s.set_diffusivity_scale(0.5 * k)
    s.close()
    with pytest.raises(L.SslbmError) as e:
        L.Solver(nx, ny, RATES, d=(0.3, 0.05, 0.05, 0.05, 0.0))
    assert e.value.status == L.SSLBM_ERR_UNSTABLE
    c = L.Solver(nx, ny, RATES, d=D)
    with pytest.raises(L.SslbmError) as e:
        c.set_diffusivity_scale(k)
    assert e.value.status == L.SSLBM_ERR_UNSUPPORTED
    c.close()
    with pytest.raises(L.SslbmError) as e:
        L.Solver(nx, ny, RATES, d=D, precision=L.FP32_DEV, lattice=L.LATTICE_D2Q5_VARD)
    assert e.value.status == L.SSLBM_ERR_UNSUPPORTED


def _vard_fp32(nx, ny, bc, st, kx, ky):
    s = _solver(nx, ny, bc, L.FP32)
    s.set_diffusivity_scale(kx, ky)
    s.write(st)
    return s


@pytest.mark.parametrize("bc", [L.BC_PERIODIC, L.BC_NOFLUX])
@pytest.mark.parametrize("nx,ny", [(131, 77), (257, 130), (64, 300), (120, 45), (5, 7), (1, 1), (2, 9)])
def test_fp32_blocked_depths_give_identical_bits(bc, nx, ny):
    """The temporal-blocked kernel (the pipeline tile with the flux-form row update, the scale
    rows staged in shared memory) against the one-step kernel, bit for bit: 2k steps at depth k
    are two passes of exactly that depth; then 11 steps, which mix depths.  Under no-flux the
    ghost images of the state and of the scale fields evolve as the cells they mirror, since
    the flux sum ((+x) + (-x)) + ((+y) + (-y)) is unchanged by a mirror image."""
    st = inputs.epidemic_state(nx, ny, 7 * nx + ny).astype(np.float32)
    kx, ky = (f.astype(np.float32) for f in inputs.mobility_fields(nx, ny, 3 + nx, "random"))
    ref = _vard_fp32(nx, ny, bc, st, kx, ky)
    ref.set_blocking(1)
    refs = {}
    for n in range(1, 17):
        ref.step(1)
        refs[n] = ref.checkpoint()[128:].view(np.uint32)
    ref.close()
    for k in range(2, 9):
        s = _vard_fp32(nx, ny, bc, st, kx, ky)
        s.set_blocking(k)
        s.step(2 * k)
        assert np.array_equal(s.checkpoint()[128:].view(np.uint32), refs[2 * k]), (k, nx, ny, bc)
        s.close()
    for k in (3, 8):
        s = _vard_fp32(nx, ny, bc, st, kx, ky)
        s.set_blocking(k)
        s.step(11)
        assert np.array_equal(s.checkpoint()[128:].view(np.uint32), refs[11]), (k, 11)
        s.close()


@pytest.mark.parametrize("depth,seg_rows", [(3, 12), (3, 50), (8, 32), (8, 41), (6, 100), (7, 28), (2, 8)])
def test_fp32_blocked_segment_lengths_give_identical_bits(depth, seg_rows):
    """2 x depth steps under no-flux: two passes of this depth with this row-segment length."""
    nx, ny = 300, 333
    st = inputs.epidemic_state(nx, ny, 5).astype(np.float32)
    kx, ky = (f.astype(np.float32) for f in inputs.mobility_fields(nx, ny, 9, "regions"))
    ref = _vard_fp32(nx, ny, L.BC_NOFLUX, st, kx, ky)
    ref.set_blocking(1)
    ref.step(2 * depth)
    want = ref.checkpoint()[128:].view(np.uint32)
    ref.close()
    s = _vard_fp32(nx, ny, L.BC_NOFLUX, st, kx, ky)
    s.set_blocking(depth, seg_rows)
    s.step(2 * depth)
    assert np.array_equal(s.checkpoint()[128:].view(np.uint32), want)
    s.close()


def test_fp32_blocked_autotuned_long_run_matches_oracle():
    """200 steps at the autotuned blocking against the FP64 oracle (FP32 tolerance), with the
    population conserved to FP32 rounding."""
    nx, ny = 96, 70
    st = inputs.epidemic_state(nx, ny, 21).astype(np.float32)
    kx, ky = (f.astype(np.float32) for f in inputs.mobility_fields(nx, ny, 13, "regions"))
    s = _vard_fp32(nx, ny, L.BC_NOFLUX, st, kx, ky)
    depth, seg, _ = s.autotune(50.0)
    assert 1 <= depth <= 8 and (depth == 1 or seg >= 4 * depth)
    assert np.array_equal(s.read(dtype=np.float32), st)  # the tuner left the state
    s.step(200)
    got = s.read()
    tot, _ = s.diagnostics()
    s.close()
    ref = oracle.sslbm_vard_run(st.astype(np.float64), TAU, RATES, kx.astype(np.float64), ky.astype(np.float64),
                                1.0, L.BC_NOFLUX, 200)
    assert relmax(got, ref) <= 1e-4
    s0 = float(st.astype(np.float64).sum())
    assert abs(float(tot.sum()) - s0) / s0 < 200 * 4 * 6e-8
