"""Checkpoint and resume (sslbm_checkpoint_bytes / _save / _load, and the ensemble's
sslbm_ensemble_checkpoint_*).

A run resumed from a checkpoint gives the bits of the uninterrupted run, for every
precision (the deviation storage of S and the Kahan compensations included), for BGK
populations, for the other lattices, and through host and device buffers.  The
read/write route cannot promise that (FP32_DEV reads S rebuilt from the deviation,
FP32_KAHAN the compensated value, a BGK write sets equilibrium populations), which is
what the checkpoint's stored planes are for.  Ensembles resume bit for bit as well, in FP32
and with deviation storage.  Checkpoints of another configuration, short buffers and damaged
headers are rejected before anything is copied.
"""
import numpy as np
import pytest

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


def _solver(nx, ny, precision, schemes=L.WANT_SSLBM, bc=L.BC_NOFLUX, lattice=L.LATTICE_D2Q5, s_ref=1.0):
    return L.Solver(nx, ny, RATES, d=D, bc=bc, precision=precision, schemes=schemes, lattice=lattice, s_ref=s_ref)


def _same_bits(a, b):
    assert a.dtype == b.dtype == np.float64 and a.shape == b.shape
    return np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("on_device", [False, True])
@pytest.mark.parametrize("precision", [L.FP64, L.FP32, L.FP32_DEV, L.FP32_KAHAN, L.FP32_SPLIT])
def test_resume_gives_the_bits_of_the_uninterrupted_run(precision, on_device):
    nx, ny = 133, 97
    st = inputs.epidemic_state(nx, ny, 7)
    a = _solver(nx, ny, precision)
    a.write(st)
    a.step(37)
    ck = a.checkpoint(on_device=on_device)
    assert len(ck) == L.sslbm_checkpoint_bytes(a.h)
    a.step(45)
    ref = a.read()
    a.close()
    b = _solver(nx, ny, precision)
    b.restore(ck)
    assert b.steps_done() == 37
    b.step(45)
    assert b.steps_done() == 82
    assert _same_bits(b.read(), ref)
    b.close()


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_resume_of_both_schemes_keeps_the_bgk_populations(precision):
    nx, ny = 70, 41
    st = inputs.epidemic_state(nx, ny, 8)
    a = _solver(nx, ny, precision, schemes=L.WANT_SSLBM | L.WANT_BGK, bc=L.BC_PERIODIC)
    a.write(st)
    a.write(st, scheme=L.SCHEME_BGK)
    a.step(20)
    a.bgk_step(11)
    ck = a.checkpoint()
    at_ck = a.read(scheme=L.SCHEME_BGK)
    a.step(13)
    a.bgk_step(9)
    ref_s, ref_b = a.read(), a.read(scheme=L.SCHEME_BGK)
    a.close()
    b = _solver(nx, ny, precision, schemes=L.WANT_SSLBM | L.WANT_BGK, bc=L.BC_PERIODIC)
    b.restore(ck)
    assert (b.steps_done(), b.steps_done(L.SCHEME_BGK)) == (20, 11)
    b.step(13)
    b.bgk_step(9)
    assert _same_bits(b.read(), ref_s)
    assert _same_bits(b.read(scheme=L.SCHEME_BGK), ref_b)
    # restarting BGK from its densities alone (populations at equilibrium) is another run
    c = _solver(nx, ny, precision, schemes=L.WANT_BGK, bc=L.BC_PERIODIC)
    c.write(at_ck, scheme=L.SCHEME_BGK)
    c.bgk_step(9)
    assert not _same_bits(c.read(scheme=L.SCHEME_BGK), ref_b)
    b.close()
    c.close()


@pytest.mark.parametrize("lattice", [L.LATTICE_D2Q9, L.LATTICE_D2Q5_SLBM, L.LATTICE_D2Q5_VARD])
@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_resume_on_the_other_lattices(lattice, precision):
    nx, ny = 66, 35
    st = inputs.epidemic_state(nx, ny, 9)
    kx = ky = None
    if lattice == L.LATTICE_D2Q5_VARD:
        g = np.random.Generator(np.random.PCG64(5))
        kx, ky = g.uniform(0.5, 1.5, (ny, nx)), g.uniform(0.5, 1.5, (ny, nx))
    solvers = []
    for _ in range(2):
        s = _solver(nx, ny, precision, lattice=lattice)
        if kx is not None:
            s.set_diffusivity_scale(kx, ky)  # fields are the handle's own, not part of a checkpoint
        solvers.append(s)
    a, b = solvers
    a.write(st)
    a.step(9)
    ck = a.checkpoint()
    a.step(10)
    b.restore(ck)
    b.step(10)
    assert b.steps_done() == 19
    assert _same_bits(b.read(), a.read())
    a.close()
    b.close()


def test_mismatched_or_damaged_checkpoints_are_rejected():
    nx, ny = 64, 48
    st = inputs.epidemic_state(nx, ny, 10)
    a = _solver(nx, ny, L.FP32)
    a.write(st)
    a.step(3)
    ck = a.checkpoint()
    others = [_solver(nx, ny + 1, L.FP32), _solver(nx + 1, ny, L.FP32), _solver(nx, ny, L.FP64),
              _solver(nx, ny, L.FP32_DEV), _solver(nx, ny, L.FP32, bc=L.BC_PERIODIC),
              _solver(nx, ny, L.FP32, schemes=L.WANT_SSLBM | L.WANT_BGK),
              _solver(nx, ny, L.FP32, lattice=L.LATTICE_D2Q9)]
    for o in others:
        with pytest.raises(L.SslbmError) as ei:
            o.restore(ck)
        assert ei.value.status == L.SSLBM_ERR_BAD_ARG
        assert o.steps_done() == 0
        o.close()
    b = _solver(nx, ny, L.FP32)
    b.write(np.zeros_like(st))
    bad = ck.copy()
    bad[0] ^= 0xFF  # magic
    damaged = [ck[:-1], ck[:100], ck[:128], bad]  # one byte short, no full header, header only, magic
    for d in damaged:
        with pytest.raises(L.SslbmError) as ei:
            b.restore(np.ascontiguousarray(d))
        assert ei.value.status == L.SSLBM_ERR_BAD_ARG
    assert b.steps_done() == 0 and not b.read().any()  # nothing was copied
    b.restore(ck)
    assert b.steps_done() == 3
    assert _same_bits(b.read(), a.read())
    a.close()
    b.close()


def test_deviation_checkpoint_requires_the_same_reference():
    """Under FP32_DEV the stored S plane is the deviation s_ref - S, so a restore into a solver
    with another s_ref would shift S by the difference: it is rejected.  Other precisions store
    S itself, and s_ref does not enter."""
    nx, ny = 40, 24
    st = inputs.epidemic_state(nx, ny, 12)
    for precision, rejected in ((L.FP32_DEV, True), (L.FP32, False)):
        a = _solver(nx, ny, precision, s_ref=1.0)
        a.write(st)
        a.step(2)
        ck = a.checkpoint()
        o = _solver(nx, ny, precision, s_ref=1.25)
        if rejected:
            with pytest.raises(L.SslbmError) as ei:
                o.restore(ck)
            assert ei.value.status == L.SSLBM_ERR_BAD_ARG and o.steps_done() == 0
        else:
            o.restore(ck)
            assert _same_bits(o.read(), a.read())
        same = _solver(nx, ny, precision, s_ref=1.0)
        same.restore(ck)
        assert _same_bits(same.read(), a.read())
        for s in (a, o, same):
            s.close()


ENS_SIZES = [(64, 64), (132, 40), (12, 300), (4, 7)]


def _ens_specs():
    out = []
    for i, (nx, ny) in enumerate(ENS_SIZES):
        r = inputs.rates_from_sigma_mu(0.3 + 0.05 * i, 0.2, 0.1, 0.01)
        out.append(dict(nx=nx, ny=ny, rates=r.as_tuple(), d=(0.03, 0.03, 0.02, 0.03, 0.0)))
    return out


def _ensemble(specs, precision=L.FP32):
    e = L.Ensemble(specs, precision=precision)
    e.set_tiling(4, 17)
    return e


@pytest.mark.parametrize("on_device", [False, True])
@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_SPLIT])
def test_ensemble_resume_gives_the_bits_of_the_uninterrupted_run(precision, on_device):
    specs = _ens_specs()
    a = _ensemble(specs, precision)
    for i, sp in enumerate(specs):
        a.write(i, inputs.epidemic_state(sp["nx"], sp["ny"], 50 + i))
    a.run(9)
    ck = a.checkpoint(on_device=on_device)
    assert len(ck) == L.sslbm_ensemble_checkpoint_bytes(a.e)
    a.run(11)
    refs = [a.read(i) for i in range(len(specs))]
    a.close()
    b = _ensemble(specs, precision)
    b.restore(ck)
    assert L.sslbm_ensemble_steps_done(b.e) == 9
    b.run(11)
    assert L.sslbm_ensemble_steps_done(b.e) == 20
    for i in range(len(specs)):
        assert _same_bits(b.read(i), refs[i]), i
    b.close()


def test_ensemble_checkpoint_mismatches_are_rejected():
    specs = _ens_specs()
    a = _ensemble(specs)
    for i, sp in enumerate(specs):
        a.write(i, inputs.epidemic_state(sp["nx"], sp["ny"], 60 + i))
    a.run(3)
    ck = a.checkpoint()
    others = [_ensemble(specs[:-1]), _ensemble(specs, L.FP32_DEV), _ensemble(specs[:-1] + [dict(specs[-1], nx=8)])]
    # under FP32_DEV a scenario whose deviation reference differs is rejected too
    dev = _ensemble(specs, L.FP32_DEV)
    for i, sp in enumerate(specs):
        dev.write(i, inputs.epidemic_state(sp["nx"], sp["ny"], 60 + i))
    dev_ck = dev.checkpoint()
    moved = _ensemble(specs[:2] + [dict(specs[2], s_ref=1.5)] + specs[3:], L.FP32_DEV)
    with pytest.raises(L.SslbmError) as ei:
        moved.restore(dev_ck)
    assert ei.value.status == L.SSLBM_ERR_BAD_ARG and L.sslbm_ensemble_steps_done(moved.e) == 0
    moved.close()
    same = _ensemble(specs, L.FP32_DEV)
    same.restore(dev_ck)
    for i in range(len(specs)):
        assert _same_bits(same.read(i), dev.read(i)), i
    same.close()
    dev.close()
    for o in others:
        with pytest.raises(L.SslbmError) as ei:
            o.restore(ck)
        assert ei.value.status == L.SSLBM_ERR_BAD_ARG
        assert L.sslbm_ensemble_steps_done(o.e) == 0
        o.close()
    b = _ensemble(specs)
    bad = ck.copy()
    bad[0] ^= 0xFF  # magic
    for d in (ck[:-1], ck[:32], bad):
        with pytest.raises(L.SslbmError) as ei:
            b.restore(np.ascontiguousarray(d))
        assert ei.value.status == L.SSLBM_ERR_BAD_ARG
    b.restore(ck)
    assert L.sslbm_ensemble_steps_done(b.e) == 3
    for i in range(len(specs)):
        assert _same_bits(b.read(i), a.read(i)), i
    a.close()
    b.close()
