"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances, stated here and derived from the arithmetic of each variant:
  FP64   relative max-norm per compartment <= 1e-12 (the kernels use the reduced form of
         Eq. sslbm_final_clean, which differs from the oracle's literal form only in the
         rounding of each step, ~1e-16 relative).
  FP32   L2 (root mean square) and max-norm error per compartment against the FP64
         oracle, divided by the compartment's peak value over the run, <= 2e-4 over the
         2000-step centre-bump run (n u with n = 2000 steps and u = 6e-8 the unit
         roundoff bounds the accumulated rounding of a contractive update); relative
         max-norm <= 1e-5 for runs of <= 20 steps.
Blocked launches (K fused steps) must give the same bits as K one-step launches.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_LONG_TOL = 2e-4
FP32_SHORT_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def rel_max(a, b):
    """max |a - b| / max |b| per compartment (absolute where b is identically 0)."""
    out = []
    for c in range(a.shape[0]):
        den = np.abs(b[c]).max()
        num = np.abs(a[c] - b[c]).max()
        out.append(num / den if den > 0 else num)
    return np.array(out)


def rel_l2(a, b):
    out = []
    for c in range(a.shape[0]):
        den = np.linalg.norm(b[c])
        num = np.linalg.norm(a[c] - b[c])
        out.append(num / den if den > 0 else num)
    return np.array(out)


def taus(d, dx=1.0, dt=1.0):
    return [oracle.tau_from_d(v, dx, dt) for v in d[:4]]


def solver_for(wl, precision, schemes=L.WANT_SSLBM, nx=None, ny=None):
    st = wl["state"]
    _, ny0, nx0 = st.shape
    return L.Solver(nx or nx0, ny or ny0, wl["rates"].as_tuple(), d=wl["d"], dx=wl["dx"], dt=wl["dt"],
                    bc=wl["bc"], precision=precision, schemes=schemes)


def small_workload(nx, ny, bc, seed=1):
    st = inputs.epidemic_state(nx, ny, seed)
    return dict(state=st, rates=inputs.Rates(0.5, 0.2, 0.11, 1 / 11), d=(0.05, 0.05, 0.01, 0.05, 0.0),
                dx=1.0, dt=1.0, bc=bc)


# ---------------------------------------------------------------------------
# FP64
# ---------------------------------------------------------------------------

def test_centre_bump_fp64_matches_oracle_2000_steps():
    wl = inputs.centre_bump_workload()
    s = solver_for(wl, L.FP64)
    s.write(wl["state"])
    s.step(wl["steps"])
    got = s.read()
    want = oracle.sslbm_run(wl["state"], taus(wl["d"]), wl["rates"].as_tuple(), 1.0, wl["bc"], wl["steps"])
    err = rel_max(got, want)
    assert (err <= FP64_TOL).all(), err
    tot, pk = s.diagnostics()
    otot, opk = oracle.diagnostics(want)
    np.testing.assert_allclose(tot, otot, rtol=1e-13, atol=1e-13)
    assert abs(pk - opk) <= 1e-12 * opk
    # population conserved to roundoff over the run (Eq. mass_conservation)
    t0 = oracle.diagnostics(wl["state"])[0].sum()
    assert abs(tot.sum() - t0) / t0 < 1e-13


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (9, 1), (2, 3), (37, 23), (130, 67), (257, 5)])
def test_fp64_ragged_grids(nx, ny, bc):
    wl = small_workload(nx, ny, bc, seed=nx * 7 + ny)
    s = solver_for(wl, L.FP64)
    s.write(wl["state"])
    s.step(40)
    want = oracle.sslbm_run(wl["state"], taus(wl["d"]), wl["rates"].as_tuple(), 1.0, bc, 40)
    err = rel_max(s.read(), want)
    assert (err <= FP64_TOL).all(), err


def test_zero_steps_is_identity_and_roundtrip_exact():
    wl = small_workload(33, 17, 1)
    s = solver_for(wl, L.FP64)
    s.write(wl["state"])
    s.step(0)
    assert np.array_equal(s.read(), wl["state"])
    assert s.steps_done() == 0


# ---------------------------------------------------------------------------
# FP32 variants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_KAHAN, L.FP32_SPLIT])
def test_centre_bump_fp32_variants_within_tolerance(precision):
    """Errors are normalised by each compartment's peak over the run: after the epidemic
    wave E and I decay below FP32's smallest subnormal (1.4e-45) while FP64 keeps
    decaying, so a ratio to the final field's own maximum would be meaningless."""
    wl = inputs.centre_bump_workload()
    s = solver_for(wl, precision)
    s.write(wl["state"])
    ref = wl["state"]
    tau, rates = taus(wl["d"]), wl["rates"].as_tuple()
    done = 0
    got, want = {}, {}
    for t in (100, 300, wl["steps"]):
        s.step(t - done)
        ref = oracle.sslbm_run(ref, tau, rates, 1.0, wl["bc"], t - done)
        done = t
        got[t], want[t] = s.read(), ref
    peak = np.max([np.abs(w).reshape(5, -1).max(axis=1) for w in want.values()], axis=0)
    for t in got:
        diff = (got[t] - want[t]).reshape(5, -1)
        einf = np.abs(diff).max(axis=1) / peak
        e2 = np.sqrt((diff ** 2).mean(axis=1)) / peak
        print(f"precision {precision} t={t}: rel-to-peak L2 {e2}, Linf {einf}")
        assert (e2 <= FP32_LONG_TOL).all() and (einf <= FP32_LONG_TOL).all(), (t, e2, einf)


@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_SPLIT, L.FP32_KAHAN])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", [(5, 3), (130, 1), (1, 70), (37, 23), (1000, 333), (250, 260)])
def test_blocked_depths_give_identical_bits(precision, bc, nx, ny):
    """2k steps at depth k are two passes of exactly that depth (sslbm_step splits n steps
    into passes of near-equal depth), so every depth's kernel is compared with the one-step
    kernel bit for bit; then 11 steps, which mix depths."""
    wl = small_workload(nx, ny, bc, seed=nx + 3 * ny)
    ref = solver_for(wl, precision)
    ref.write(wl["state"])
    ref.set_blocking(1)
    refs = {}
    # every stored plane (the checkpoint holds them as stored: the split S's compensation too)
    for n in range(1, 17):
        ref.step(1)
        refs[n] = ref.checkpoint()[128:].view(np.uint32)
        if n == 11:
            base = ref.read()
    for k in range(2, 9):
        s = solver_for(wl, precision)
        s.write(wl["state"])
        s.set_blocking(k)
        s.step(2 * k)
        got = s.checkpoint()[128:].view(np.uint32)
        assert np.array_equal(got, refs[2 * k]), (k, nx, ny, bc)
    for k in (3, 8):
        s = solver_for(wl, precision)
        s.write(wl["state"])
        s.set_blocking(k)
        s.step(11)
        assert np.array_equal(s.checkpoint()[128:].view(np.uint32), refs[11]), (k, 11)
    # and a short run agrees with the FP64 oracle to FP32 accuracy
    want = oracle.sslbm_run(wl["state"], taus(wl["d"]), wl["rates"].as_tuple(), 1.0, bc, 11)
    assert (rel_max(base, want) <= FP32_SHORT_TOL).all()


@pytest.mark.parametrize("depth,seg_rows", [(3, 12), (3, 16), (3, 50), (3, 333), (8, 32), (8, 41), (6, 100),
                                             (7, 28), (5, 21), (2, 8)])
def test_blocked_segment_lengths_give_identical_bits(depth, seg_rows):
    """2 x depth steps: two passes of exactly this depth with this row-segment length."""
    wl = small_workload(300, 333, 1, seed=5)
    ref = solver_for(wl, L.FP32)
    ref.write(wl["state"])
    ref.set_blocking(1)
    ref.step(2 * depth)
    base = ref.read(dtype=np.float32)
    s = solver_for(wl, L.FP32)
    s.write(wl["state"])
    s.set_blocking(depth, seg_rows)
    s.step(2 * depth)
    assert np.array_equal(s.read(dtype=np.float32).view(np.uint32), base.view(np.uint32))


# ---------------------------------------------------------------------------
# BGK comparison scheme
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny", [(1, 1), (45, 31), (7, 130)])
def test_bgk_fp64_matches_oracle(nx, ny, bc):
    wl = small_workload(nx, ny, bc, seed=nx * 11 + ny)
    s = solver_for(wl, L.FP64, schemes=L.WANT_BGK)
    s.write(wl["state"], scheme=L.SCHEME_BGK)
    s.bgk_step(60)
    got = s.read(scheme=L.SCHEME_BGK)
    want = oracle.bgk_run_state(wl["state"], taus(wl["d"]), wl["rates"].as_tuple(), 1.0, bc, 60)
    assert (rel_max(got, want) <= FP64_TOL).all(), rel_max(got, want)
    tot, _ = s.diagnostics(scheme=L.SCHEME_BGK)
    np.testing.assert_allclose(tot, oracle.diagnostics(want)[0], rtol=1e-13)


def test_bgk_fp32_centre_bump_within_tolerance():
    wl = inputs.centre_bump_workload()
    s = solver_for(wl, L.FP32, schemes=L.WANT_BGK | L.WANT_SSLBM)
    s.write(wl["state"], scheme=L.SCHEME_BGK)
    tau, rates = taus(wl["d"]), wl["rates"].as_tuple()
    got, want = {}, {}
    f, D = oracle.bgk_init(wl["state"])
    done = 0
    for t in (100, 500):
        s.bgk_step(t - done)
        f, D = oracle.bgk_run(f, D, tau, rates, 1.0, wl["bc"], t - done)
        done = t
        got[t], want[t] = s.read(scheme=L.SCHEME_BGK), oracle.bgk_density(f, D)
    peak = np.max([np.abs(w).reshape(5, -1).max(axis=1) for w in want.values()], axis=0)
    for t in got:
        einf = np.abs((got[t] - want[t]).reshape(5, -1)).max(axis=1) / peak
        assert (einf <= FP32_LONG_TOL).all(), (t, einf)


# ---------------------------------------------------------------------------
# Diagnostics, I/O paths, errors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_KAHAN, L.FP32_SPLIT])
def test_diagnostics_match_oracle_on_read_back_state(precision):
    wl = small_workload(517, 211, 0, seed=8)
    s = solver_for(wl, precision)
    s.write(wl["state"])
    s.step(30)
    st = s.read()
    tot, pk = s.diagnostics()
    otot, opk = oracle.diagnostics(st)
    np.testing.assert_allclose(tot, otot, rtol=1e-12)
    assert pk == pytest.approx(opk, rel=1e-7)


@pytest.mark.parametrize("precision,scheme", [(L.FP32, L.SCHEME_SSLBM), (L.FP32_DEV, L.SCHEME_SSLBM),
                                              (L.FP32_KAHAN, L.SCHEME_SSLBM), (L.FP32_SPLIT, L.SCHEME_SSLBM),
                                              (L.FP32, L.SCHEME_BGK)])
def test_diagnostics_on_wide_rows(precision, scheme):
    """Rows of 4099 cells: a thread of the FP32 reduction adds several 4-cell groups of a row
    in its TwoSum pair, and the row's last group holds three cells."""
    wl = small_workload(4099, 13, 1, seed=21)
    bgk = scheme == L.SCHEME_BGK
    s = solver_for(wl, precision, schemes=L.WANT_BGK if bgk else L.WANT_SSLBM)
    s.write(wl["state"], scheme=scheme)
    (s.bgk_step if bgk else s.step)(7)
    st = s.read(scheme=scheme)
    tot, pk = s.diagnostics(scheme=scheme)
    otot, opk = oracle.diagnostics(st)
    np.testing.assert_allclose(tot, otot, rtol=1e-12)
    assert pk == pytest.approx(opk, rel=1e-7)


def test_nonfinite_state_is_reported_not_trapped():
    wl = small_workload(40, 30, 0)
    st = wl["state"].copy()
    st[2, 5, 5] = np.nan
    s = solver_for(wl, L.FP32)
    s.write(st)
    with pytest.raises(L.SslbmError) as ei:
        s.diagnostics()
    assert ei.value.status == -5


def test_split_storage_holds_s_to_twice_fp32_precision():
    """FP32_SPLIT keeps S as a value and a compensation plane: a written FP64 S reads back to
    about 2^-48 relative (FP32 keeps 2^-24), the other compartments as FP32 values."""
    wl = small_workload(61, 37, 1, seed=31)
    st = wl["state"].copy()
    st[0] = 0.9 + 1e-9 * np.arange(61 * 37).reshape(37, 61)  # S with increments below an FP32 ulp
    s = solver_for(wl, L.FP32_SPLIT)
    s.write(st)
    back = s.read()
    assert np.abs(back[0] - st[0]).max() <= 2.0 ** -47 * np.abs(st[0]).max()
    assert np.array_equal(back[1:], st[1:].astype(np.float32).astype(np.float64))
    p = solver_for(wl, L.FP32)
    p.write(st)
    assert np.abs(p.read()[0] - st[0]).max() > 1e3 * np.abs(back[0] - st[0]).max()


def test_device_tensor_io_and_f32_dtype():
    import torch
    wl = small_workload(64, 48, 1)
    s = solver_for(wl, L.FP32)
    src = torch.from_numpy(wl["state"].astype(np.float32)).cuda()
    s.write(src)
    dst = torch.empty_like(src)
    L.sslbm_read(s.h, L.SCHEME_SSLBM, L.ALL, dst)
    torch.cuda.synchronize()
    assert torch.equal(dst, src)
    one = torch.empty((48, 64), dtype=torch.float64, device="cuda")
    L.sslbm_read(s.h, L.SCHEME_SSLBM, L.I, one)
    torch.cuda.synchronize()
    assert np.array_equal(one.cpu().numpy(), wl["state"][2].astype(np.float32).astype(np.float64))


def test_error_statuses_on_gpu():
    wl = small_workload(16, 16, 0)
    s = solver_for(wl, L.FP64)
    with pytest.raises(L.SslbmError) as ei:
        s.step(-1)
    assert ei.value.status == -1
    with pytest.raises(L.SslbmError) as ei:
        s.set_blocking(3)
    assert ei.value.status == -7
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_write(s.h, L.SCHEME_SSLBM, 7, wl["state"])
    assert ei.value.status == -1
    with pytest.raises(L.SslbmError) as ei:
        s.bgk_step(1)  # this handle holds no BGK state
    assert ei.value.status == -1


@pytest.mark.parametrize("precision", [L.FP32, L.FP32_DEV, L.FP32_SPLIT, L.FP32_KAHAN, L.FP64])
def test_autotune_leaves_state_and_picks_a_valid_configuration(precision):
    wl = small_workload(600, 333, 1, seed=12)
    s = solver_for(wl, precision)
    s.write(wl["state"])
    before = s.read()
    depth, seg, ms = s.autotune(40.0)
    assert np.array_equal(s.read(), before)  # candidates write only the spare buffer
    assert 1 <= depth <= L.MAX_DEPTH and ms > 0
    if precision == L.FP64:
        assert depth == 1
    assert s.get_blocking() == (depth, seg)
    assert s.autotune(40.0)[:2] == (depth, seg)  # cached per grid and precision
    s.step(13)
    ref = solver_for(wl, precision)
    ref.write(wl["state"])
    ref.set_blocking(1)
    ref.step(13)
    assert np.array_equal(s.read(), ref.read())
