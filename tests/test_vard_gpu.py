"""The SSLBM with spatially varying, anisotropic diffusion on the GPU (lattice
LATTICE_D2Q5_VARD, sslbm_set_diffusivity_scale) against the FP64 oracle
(oracle.sslbm_vard_run).

The kernel forms the four link coefficients and the flux sum in the oracle's order, each
operation rounded once; the update itself uses the library's fused form of
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
        s.set_blocking(4)
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
