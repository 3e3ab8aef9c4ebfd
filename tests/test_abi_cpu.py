"""The C-ABI library builds, loads and exports every symbol include/sslbm.h declares;
host-side validation answers with the documented status codes.  No GPU calls."""
import os
import re

import numpy as np

import pytest

from paper_2603_19789_gb300 import build as sbuild
from paper_2603_19789_gb300 import sslbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sbuild.build()
    return L.load()


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "sizeof", "defined"):
                names.append(name)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 15, declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # the binding exposes each under the same name
    for n in declared:
        assert hasattr(L, n) or n in ("sslbm_create",), n


def test_binding_export_list_matches_header(lib):
    assert set(L.EXPORTS) <= set(_declared_functions())


def test_release_library_refuses_the_debug_calls(lib):
    """Index checks exist only in the debug build; the release library says so without
    touching the device."""
    assert lib.sslbm_debug_bounds(None, None, None, None) == L.SSLBM_ERR_UNSUPPORTED
    assert lib.sslbm_debug_bounds_probe(5, 3) == L.SSLBM_ERR_UNSUPPORTED


def test_checked_library_builds_and_exports_every_symbol():
    """The index-checked debug build (SSLBM_BOUNDS_CHECK) compiles for sm_103a and exports the
    same ABI; it is loaded on its own (RTLD_LOCAL), so its symbols do not mix with the
    release library's."""
    import ctypes
    path = sbuild.build(checked=True)
    assert path.endswith("libsslbm_check.so") and os.path.exists(path)
    chk = ctypes.CDLL(path)
    missing = [n for n in _declared_functions() if not hasattr(chk, n)]
    assert not missing, missing


def test_strerror_and_version(lib):
    assert L.sslbm_strerror(0) == "SSLBM_OK"
    assert L.sslbm_strerror(-2) == "SSLBM_ERR_UNSTABLE"
    assert L.sslbm_strerror(12345) == "SSLBM_ERR_UNKNOWN"
    assert L.sslbm_version() >= 100


def test_workspace_bytes_layout(lib):
    g = L.make_grid(8192, 8192, precision=L.FP32)
    n = L.sslbm_workspace_bytes(g)
    # two buffers of five FP32 planes plus a small diagnostics scratch
    assert 2 * 5 * 8192 * 8192 * 4 <= n < 2 * 5 * 8192 * 8192 * 4 + (1 << 20)
    g = L.make_grid(100, 7, precision=L.FP64, schemes=L.WANT_SSLBM | L.WANT_BGK)
    n = L.sslbm_workspace_bytes(g)
    pitch = 128
    assert n >= (2 * 5 + 2 * 21) * pitch * 7 * 8
    g = L.make_grid(100, 7, precision=L.FP32_KAHAN)
    assert L.sslbm_workspace_bytes(g) >= 2 * 10 * 128 * 7 * 4
    # the double-word storage: ten FP32 planes (high parts and minus the low parts)
    g = L.make_grid(100, 7, precision=L.FP64_DW)
    assert L.sslbm_workspace_bytes(g) == L.sslbm_workspace_bytes(L.make_grid(100, 7, precision=L.FP32_KAHAN))


@pytest.mark.parametrize("kw", [dict(nx=0, ny=5), dict(nx=5, ny=-1), dict(nx=4, ny=4, dx=0.0),
                                dict(nx=4, ny=4, dt=float("nan")), dict(nx=4, ny=4, bc=2),
                                dict(nx=4, ny=4, precision=7), dict(nx=4, ny=4, precision=6),
                                dict(nx=4, ny=4, schemes=0),
                                dict(nx=1 << 31, ny=1)])
def test_invalid_grids_rejected(lib, kw):
    args = dict(nx=4, ny=4)
    args.update(kw)
    g = L.make_grid(**args)
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_workspace_bytes(g)
    assert ei.value.status == -1


@pytest.mark.parametrize("precision", [L.FP32_DEV, L.FP32_SPLIT, L.FP32_KAHAN, L.FP64_DW])
def test_bgk_in_the_fp32_storage_variants_unsupported(lib, precision):
    g = L.make_grid(8, 8, precision=precision, schemes=L.WANT_BGK)
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_workspace_bytes(g)
    assert ei.value.status == -7


@pytest.mark.parametrize("precision", [L.FP32_SPLIT, L.FP64_DW])
@pytest.mark.parametrize("lattice", [L.LATTICE_D2Q9, L.LATTICE_D2Q5_SLBM, L.LATTICE_D2Q5_VARD])
def test_split_and_double_word_storages_only_on_d2q5(lib, lattice, precision):
    g = L.make_grid(8, 8, precision=precision, lattice=lattice)
    with pytest.raises(L.SslbmError) as ei:
        L.sslbm_workspace_bytes(g)
    assert ei.value.status == -7


def test_split_storage_workspace_holds_six_planes(lib):
    pitch = 128
    g = L.make_grid(100, 7, precision=L.FP32_SPLIT)
    n = L.sslbm_workspace_bytes(g)
    assert n >= 2 * 6 * pitch * 7 * 4
    assert n < L.sslbm_workspace_bytes(L.make_grid(100, 7, precision=L.FP32_KAHAN))


def _create_status(grid, params, ws=0, nbytes=0):
    try:
        h = L.sslbm_create(grid, params, ws, nbytes, 0)
    except L.SslbmError as e:
        return e.status, str(e)
    L.sslbm_destroy(h)
    return 0, ""


@pytest.mark.parametrize("d,status", [((0.3, 0.05, 0.05, 0.05, 0.0), -2),    # tau = 1.4 > 5/4
                                      ((0.05, -0.01, 0.05, 0.05, 0.0), -1),  # negative d
                                      ((0.05, 0.05, 0.05, 0.05, 0.1), -1)])  # D must not diffuse
def test_parameter_validation(lib, d, status):
    g = L.make_grid(16, 16)
    p = L.make_params(0.3, 0.2, 0.11, 1 / 11, d=d)
    st, msg = _create_status(g, p)
    assert st == status, msg


def test_tau_below_half_is_unstable(lib):
    g = L.make_grid(16, 16)
    p = L.make_params(0.3, 0.2, 0.11, 1 / 11, tau=(0.6, 0.49, 0.6, 0.6))
    assert _create_status(g, p)[0] == -2


def test_strict_nonnegativity_condition(lib):
    g = L.make_grid(16, 16)
    # 4 * 0.2 + beta dt = 0.8 + 0.5 > 1 for S
    p = L.make_params(0.5, 0.2, 0.11, 1 / 11, d=(0.2, 0.05, 0.05, 0.05, 0.0), strict=True)
    assert _create_status(g, p)[0] == -2


@pytest.mark.parametrize("rates", [(-0.1, 0.2, 0.1, 0.1), (0.3, 0.2, 0.1, 1.5), (float("inf"), 0.2, 0.1, 0.1)])
def test_bad_rates(lib, rates):
    g = L.make_grid(16, 16)
    p = L.make_params(*rates, d=(0.05,) * 4)
    assert _create_status(g, p)[0] == -1


def test_missing_workspace(lib):
    g = L.make_grid(16, 16)
    p = L.make_params(0.3, 0.2, 0.11, 1 / 11, d=(0.05,) * 4)
    st, msg = _create_status(g, p, ws=0, nbytes=0)
    assert st == -6 and "NULL" in msg


def test_misaligned_workspace(lib):
    g = L.make_grid(16, 16)
    p = L.make_params(0.3, 0.2, 0.11, 1 / 11, d=(0.05,) * 4)
    st, _ = _create_status(g, p, ws=0x1000 + 8, nbytes=1 << 30)
    assert st == -6


def test_small_workspace(lib):
    g = L.make_grid(16, 16)
    p = L.make_params(0.3, 0.2, 0.11, 1 / 11, d=(0.05,) * 4)
    st, _ = _create_status(g, p, ws=0x10000, nbytes=100)
    assert st == -6


@pytest.mark.parametrize("cfg", [(32, 12, 4, 64), (16, 8, 2, 32), (8, 4, 2, 12)])
def test_surrogate_initial_params_follow_the_flat_layout(cfg):
    """The seeded starting point has one value per parameter, biases zero, spectral
    weights at the 1/width^2 scale (layout of sslbm_fno_set_params)."""
    from oracle import fno
    from paper_2603_19789_gb300 import surrogate as S
    W, m, Lr, H = cfg
    th = S.initial_params(W, m, Lr, H, seed=1)
    assert th.dtype == np.float32 and th.size == fno.n_params(W, m, Lr, H)
    p = fno.unflatten(th.astype(np.float64), W, m, Lr, H)
    for name, v in p.items():
        if name[0] in "abq":
            assert not v.any(), name
        elif name[0] == "R":
            assert 0 < np.abs(v).max() <= 1.0 / (W * W)
        else:
            assert 0 < np.abs(v).max() <= 1.0 / np.sqrt(v.shape[1])
