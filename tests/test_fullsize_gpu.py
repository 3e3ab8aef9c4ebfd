"""Full-size parity: the 8192 x 8192 no-flux multi-seed workload in the launch
configurations the benchmark times (FP32 with the autotuned depth and segment length, and
the deep blockings the autotuner picks there; FP32 defaults; FP64 one-step kernel), checked
on sampled windows that the oracle computes on their domain of dependence, plus
bit-identity of the blocked and one-step kernels over the whole grid.  And a grid of more
than 2^31 cells, to exercise 64-bit indexing."""
import numpy as np
import pytest

import oracle
from paper_2603_19789_gb300 import inputs
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

NSTEPS = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


@pytest.fixture(scope="module")
def workload():
    return inputs.roofline_workload()


def _taus(d):
    return [oracle.tau_from_d(v) for v in d[:4]]


def _windows(nx, ny, w, h, seed=3):
    g = np.random.default_rng(seed)
    pts = [(0, 0), (nx - w, 0), (0, ny - h), (nx - w, ny - h), (nx // 2, 0), (0, ny // 2),
           (nx - w, ny // 3), (nx // 3, ny - h)]
    # around warp-strip boundaries of the blocked kernel (120 written columns per strip)
    pts += [(120 * k - w // 2, int(g.integers(0, ny - h))) for k in (1, 2, 17, 68)]
    pts += [(int(g.integers(0, nx - w)), int(g.integers(0, ny - h))) for _ in range(16)]
    return pts


def _check_windows(got, wl, tol_rel, tol_abs, nsteps):
    st = wl["state"]
    _, ny, nx = st.shape
    tau = _taus(wl["d"])
    w = h = 8
    for x0, y0 in _windows(nx, ny, w, h):
        want = oracle.sslbm_window(st, x0, y0, w, h, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], nsteps)
        np.testing.assert_allclose(got[:, y0:y0 + h, x0:x0 + w], want, rtol=tol_rel, atol=tol_abs,
                                   err_msg=f"window at ({x0}, {y0})")


def test_roofline_grid_fp32_bench_config(workload):
    wl = workload
    s = L.Solver(8192, 8192, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=L.FP32)
    k, seg = s.get_blocking()
    assert k == 4 and seg == 0  # the defaults the benchmark uses
    s.write(wl["state"])
    s.step(NSTEPS)
    got = s.read(dtype=np.float32)
    _check_windows(got.astype(np.float64), wl, 1e-5, 1e-9, NSTEPS)
    # the blocked launches equal one-step launches bit for bit over the whole grid
    s.write(wl["state"])
    s.set_blocking(1)
    s.step(NSTEPS)
    ref = s.read(dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    s.close()


BENCH_STEPS = 100  # lattice steps of one benchmark step


def _check_autotuned_like_the_bench(wl, s):
    """BENCH_STEPS steps in the solver's current blocking (passes of near-equal depth): sampled
    windows against the oracle, and the whole grid against the one-step kernel bit for bit.
    Tolerance per value: 2e-5 relative plus 1e-5 of the compartment's largest value on the
    grid (n u = 100 x 6e-8 bounds the accumulated rounding; a cell far smaller than its
    neighbours carries their rounding, hence the absolute part, as in the FP32 parity tests).
    The diagnostics are fused into the last pass, as in the benchmark: their totals agree with
    the oracle's totals of the read-back state to 1e-12 and with the separate reduction of the
    same state to 1e-13, and the peak of I is the same value."""
    s.write(wl["state"])
    s.set_fused_diagnostics(True)
    s.step(BENCH_STEPS)
    tot_f, pk_f = s.diagnostics()
    got = s.read(dtype=np.float32)
    otot, opk = oracle.diagnostics(got.astype(np.float64))
    np.testing.assert_allclose(tot_f, otot, rtol=1e-12)
    assert pk_f == pytest.approx(opk, rel=1e-7)
    g64 = got.astype(np.float64)
    scale = np.abs(g64).reshape(5, -1).max(axis=1)
    st = wl["state"]
    tau = _taus(wl["d"])
    for x0, y0 in _windows(8192, 8192, 8, 8):
        want = oracle.sslbm_window(st, x0, y0, 8, 8, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], BENCH_STEPS)
        part = g64[:, y0:y0 + 8, x0:x0 + 8]
        for c in range(5):
            bound = 2e-5 * np.abs(want[c]) + 1e-5 * scale[c]
            assert (np.abs(part[c] - want[c]) <= bound).all(), (x0, y0, c, np.abs(part[c] - want[c]).max())
    s.write(wl["state"])
    s.set_fused_diagnostics(False)
    s.set_blocking(1)
    s.step(BENCH_STEPS)
    ref = s.read(dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    tot, pk = s.diagnostics()
    np.testing.assert_allclose(tot_f, tot, rtol=1e-13)
    assert pk_f == pk


def test_roofline_grid_fp32_autotuned_config(workload):
    """The configuration the benchmark's number comes from: the library's autotuner picks the
    depth and segment length (the same call and budget as the benchmark), and a benchmark
    step's 100 lattice steps run as passes of that depth and one less."""
    wl = workload
    s = L.Solver(8192, 8192, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=L.FP32)
    s.write(wl["state"])
    depth, seg, ms = s.autotune(300.0)
    print(f"autotuned depth {depth}, seg_rows {seg}, {ms:.3f} ms per lattice step")
    assert 1 <= depth <= L.MAX_DEPTH
    _check_autotuned_like_the_bench(wl, s)
    s.close()


@pytest.mark.parametrize("depth,seg_rows", [(8, 1024), (7, 1024), (8, 0)])
def test_roofline_grid_fp32_deep_blocking(workload, depth, seg_rows):
    """Depth 8 with 1024-row segments, the choice the autotuner made on the benchmark grid;
    100 steps at depth 8 are 9 passes of 8 and 4 of 7."""
    wl = workload
    s = L.Solver(8192, 8192, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=L.FP32)
    s.set_blocking(depth, seg_rows)
    assert s.get_blocking() == (depth, seg_rows)
    _check_autotuned_like_the_bench(wl, s)
    s.close()


def test_roofline_grid_fp64(workload):
    wl = workload
    s = L.Solver(8192, 8192, wl["rates"].as_tuple(), d=wl["d"], bc=wl["bc"], precision=L.FP64)
    s.write(wl["state"])
    s.step(NSTEPS)
    got = s.read()
    st = wl["state"]
    tau = _taus(wl["d"])
    for x0, y0 in _windows(8192, 8192, 8, 8):
        want = oracle.sslbm_window(st, x0, y0, 8, 8, tau, wl["rates"].as_tuple(), 1.0, wl["bc"], NSTEPS)
        part = got[:, y0:y0 + 8, x0:x0 + 8]
        for c in range(5):
            scale = np.abs(want[c]).max()
            assert np.abs(part[c] - want[c]).max() <= 1e-12 * scale, (x0, y0, c)
    s.close()


def test_more_than_2_31_cells_fp32():
    import torch
    free, total = torch.cuda.mem_get_info()
    if free < 110e9:
        pytest.skip(f"needs ~100 GB of free device memory, {free / 1e9:.0f} GB free")
    nx = ny = 46341  # 2,147,488,281 cells > 2^31
    rates = (0.5, 0.2, 0.11, 1 / 11)
    d = (0.05, 0.05, 0.01, 0.05, 0.0)
    s = L.Solver(nx, ny, rates, d=d, bc=L.BC_NOFLUX, precision=L.FP32)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(inputs.DEFAULT_SEED)
    ranges = [(0.6, 0.9), (0.0, 0.05), (0.0, 0.05), (0.0, 0.2), (0.0, 0.01)]
    m, w, h = 2, 8, 8
    pts = [(0, 0), (nx - w, ny - h), (nx - w, 0), (0, ny - h), (nx // 2, ny // 2),
           (12345, 46000), (46300, 30001)]
    inputs_win = {p: np.zeros((5, min(ny, p[1] + h + m) - max(0, p[1] - m),
                               min(nx, p[0] + w + m) - max(0, p[0] - m))) for p in pts}
    for c, (lo, hi) in enumerate(ranges):
        plane = torch.rand((ny, nx), generator=gen, device="cuda", dtype=torch.float32) * (hi - lo) + lo
        L.sslbm_write(s.h, L.SCHEME_SSLBM, c, plane)
        for (x0, y0), arr in inputs_win.items():
            ya, xa = max(0, y0 - m), max(0, x0 - m)
            arr[c] = plane[ya:ya + arr.shape[1], xa:xa + arr.shape[2]].double().cpu().numpy()
        del plane
    torch.cuda.synchronize()
    s.set_blocking(2)
    s.step(m)
    tau = _taus(d)
    for c in range(5):
        out = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
        L.sslbm_read(s.h, L.SCHEME_SSLBM, c, out)
        torch.cuda.synchronize()
        for (x0, y0), arr in inputs_win.items():
            ya, xa = max(0, y0 - m), max(0, x0 - m)
            want = oracle.sslbm_run(arr, tau, rates, 1.0, 1, m)[c, y0 - ya:y0 - ya + h, x0 - xa:x0 - xa + w]
            got = out[y0:y0 + h, x0:x0 + w].double().cpu().numpy()
            np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-9, err_msg=f"c={c} at ({x0},{y0})")
        del out
    s.close()
