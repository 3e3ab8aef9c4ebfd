"""Pins of the FP64 surrogate oracle (oracle/fno.py).

The spectral convolution, as the oracle writes it (numpy's 2D FFT, the kept modes, the real
part of the inverse FFT), must equal a direct double sum of its definition on small grids,
and the real-DFT-product factorisation the GPU evaluates (written out here, as a subject
under test) must equal it; every parameter gradient of the hand-derived backward pass must
equal a central finite difference of the forward pass; the prediction is nonnegative and
conserves its input's population for any parameters.
"""
import numpy as np
import pytest

from oracle import fno


def _direct_spectral(h, R, n, m):
    """K(h) as the double sum of its definition: forward sums over every cell for each kept
    mode, then the inverse sum over the kept modes for every cell (pure loops over modes)."""
    B, Ci = h.shape[:2]
    Co = R.shape[1]
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    out = np.zeros((B, Co, n, n))
    for a, kx in enumerate(fno.kx_modes(n, m)):
        for ky in range(m):
            e = np.exp(-2j * np.pi * (kx * x + ky * y) / n)
            hat = (h * e).sum(axis=(2, 3))                        # [B, Ci]
            g = hat @ (R[:, :, a, ky, 0] + 1j * R[:, :, a, ky, 1])  # [B, Co]
            c = 1.0 if ky == 0 else 2.0
            out += c * (g[:, :, None, None] * np.conj(e)[None, None]).real
    return out / (n * n)


# ---- the GPU's factorisation of the same operator (subject under test) -------------------

def _dft_mats(n, m):
    """Real DFT factors: Fx (n x 4m: cos, -sin per kept kx), Fy (2m x n: cos, -sin per ky),
    Fyi (n x 2m: cos, sin) and Fxi (4m x n: cos, -sin)."""
    x = np.arange(n)
    thx = 2 * np.pi * np.outer(x, fno.kx_modes(n, m)) / n
    thy = 2 * np.pi * np.outer(np.arange(m), x) / n
    Fx = np.empty((n, 4 * m))
    Fx[:, 0::2], Fx[:, 1::2] = np.cos(thx), -np.sin(thx)
    Fy = np.empty((2 * m, n))
    Fy[0::2], Fy[1::2] = np.cos(thy), -np.sin(thy)
    Fyi = np.empty((n, 2 * m))
    Fyi[:, 0::2], Fyi[:, 1::2] = np.cos(thy).T, np.sin(thy).T
    Fxi = np.empty((4 * m, n))
    Fxi[0::2], Fxi[1::2] = np.cos(thx).T, -np.sin(thx).T
    return Fx, Fy, Fyi, Fxi


def _factorised_spectral(h, R, n, m):
    """H1 = h Fx, T = Fy H1, hat_h = combine(T), hat_g = mix(hat_h, R), U = expand(hat_g),
    K(h) = Fyi U Fxi / n^2: the order of the GPU's products."""
    Fx, Fy, Fyi, Fxi = _dft_mats(n, m)
    T = Fy @ (h @ Fx)                                     # [B, Ci, 2m, 4m]
    Tc, Ts = T[..., 0::2, :], T[..., 1::2, :]
    hat_h = np.swapaxes((Tc[..., 0::2] - Ts[..., 1::2]) + 1j * (Tc[..., 1::2] + Ts[..., 0::2]), -1, -2)
    hat_g = np.einsum("bikq,iokq->bokq", hat_h, R[..., 0] + 1j * R[..., 1])
    c = np.where(np.arange(m) == 0, 1.0, 2.0)
    gT = np.swapaxes(hat_g, -1, -2) * c[:, None]          # [B, Co, m, 2m]
    U = np.zeros(gT.shape[:-2] + (2 * m, 4 * m))
    U[..., 0::2, 0::2], U[..., 1::2, 0::2] = gT.real, -gT.imag
    U[..., 0::2, 1::2], U[..., 1::2, 1::2] = gT.imag, gT.real
    return (Fyi @ U) @ Fxi / (n * n), hat_h


@pytest.mark.parametrize("n,m", [(6, 2), (7, 3), (8, 2)])
def test_spectral_equals_the_direct_double_sum(n, m):
    g = np.random.default_rng(10 * n + m)
    h = g.standard_normal((2, 3, n, n))
    R = g.standard_normal((3, 4, 2 * m, m, 2))
    a, hat = fno.spectral(h, R, n, m)
    b = _direct_spectral(h, R, n, m)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())
    # hat_h is the forward sum itself
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    kx = fno.kx_modes(n, m)
    direct = (h[0, 1] * np.exp(-2j * np.pi * (kx[-1] * x + (m - 1) * y) / n)).sum()
    assert abs(hat[0, 1, -1, m - 1] - direct) <= 1e-12 * np.abs(h).sum()


@pytest.mark.parametrize("n,m", [(16, 4), (32, 6), (24, 5)])
def test_gpu_factorisation_equals_the_definition(n, m):
    g = np.random.default_rng(n + m)
    h = g.standard_normal((2, 3, n, n))
    R = g.standard_normal((3, 4, 2 * m, m, 2))
    a, ha = fno.spectral(h, R, n, m)
    b, hb = _factorised_spectral(h, R, n, m)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * np.abs(a).max())
    np.testing.assert_allclose(hb, ha, rtol=0, atol=1e-12 * np.abs(ha).max())


def test_spectral_backward_is_the_adjoint():
    """<K(h), w> = <h, K^T w> for random h, w (dh of spectral_backward), and dR equals the
    derivative of <K(h), w> with respect to R (finite differences of a linear map)."""
    n, m = 12, 3
    g = np.random.default_rng(2)
    h = g.standard_normal((2, 3, n, n))
    w = g.standard_normal((2, 4, n, n))
    R = g.standard_normal((3, 4, 2 * m, m, 2))
    out, hat = fno.spectral(h, R, n, m)
    dh, dR = fno.spectral_backward(w, hat, R, n, m)
    assert abs((out * w).sum() - (h * dh).sum()) <= 1e-11 * np.abs(out * w).sum()
    for idx in [(0, 0, 0, 0, 0), (2, 3, 2 * m - 1, m - 1, 1), (1, 2, m, 1, 0), (0, 1, m - 1, 0, 1)]:
        Rp = R.copy()
        Rp[idx] += 1.0
        delta = (fno.spectral(h, Rp, n, m)[0] * w).sum() - (out * w).sum()
        assert delta == pytest.approx(dR[idx], rel=1e-9, abs=1e-9)


def test_spectral_keeps_only_the_retained_modes():
    n, m = 16, 3
    x = np.arange(n)
    # a mode outside the kept set is annihilated, one inside passes with weight R
    R = np.zeros((1, 1, 2 * m, m, 2))
    R[..., 0] = 1.0  # identity mixing
    inside = np.cos(2 * np.pi * (2 * x[None, :] + 1 * x[:, None]) / n)[None, None]
    outside = np.cos(2 * np.pi * (5 * x[None, :] + 1 * x[:, None]) / n)[None, None]
    np.testing.assert_allclose(fno.spectral(inside, R, n, m)[0], inside, atol=1e-12)
    np.testing.assert_allclose(fno.spectral(outside, R, n, m)[0], 0.0, atol=1e-12)


def test_parameter_count_is_about_two_million():
    assert 2.0e6 < fno.n_params(32, 12, 4, 64) < 2.5e6


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    W, m, L, H, n, B = 4, 3, 2, 6, 12, 2
    g = np.random.default_rng(seed)
    params = fno.init_params(seed, W, m, L, H)
    for k in params:  # nonzero biases and larger spectral weights exercise every term
        params[k] = params[k] + 0.1 * g.standard_normal(params[k].shape)
    u = g.uniform(0, 1, (B, 5, n, n))
    x = fno.make_input(u, g.uniform(1.2, 4.0, B), g.uniform(-3, -1, B))
    target = g.uniform(0, 1, (B, 5, n, n))

    def loss_of(theta):
        y, _ = fno.forward(fno.unflatten(theta, W, m, L, H), x, W, m, L, H)
        return fno.mse(y, target)[0]

    y, cache = fno.forward(params, x, W, m, L, H)
    _, dy = fno.mse(y, target)
    grads = fno.flatten(fno.backward(params, cache, dy, W, m, L, H), W, m, L, H)
    theta = fno.flatten(params, W, m, L, H)
    idx = g.choice(theta.size, 60, replace=False)
    # every parameter tensor is represented
    offs, k = [], 0
    for name, shp in fno.param_shapes(W, m, L, H):
        offs.append(k)
        k += int(np.prod(shp))
    idx = np.unique(np.concatenate([idx, np.array(offs)]))
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (loss_of(tp) - loss_of(tm)) / (2 * eps)
        assert abs(fd - grads[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grads[i])


def test_input_scaling_recovers_the_state_and_is_scale_free():
    g = np.random.default_rng(7)
    u = g.uniform(0, 1, (3, 5, 8, 8))
    u[1, 1:3] *= 1e-5                        # an early-growth sample: E, I tiny
    u[2, 1:3] = 0.0                          # no infection at all: the scale floor
    x = fno.make_input(u, np.full(3, 2.0), np.full(3, -2.0))
    sig = fno.out_scale(x)
    np.testing.assert_allclose(x[:, :5] * sig[:, :, None, None], u, rtol=1e-13, atol=0)
    peak = np.maximum(u[:, 1].reshape(3, -1).max(1), u[:, 2].reshape(3, -1).max(1))
    np.testing.assert_allclose(sig[:2, 1], peak[:2], rtol=1e-13)
    assert sig[2, 1] == pytest.approx(fno.SCALE_FLOOR, rel=1e-12)
    assert np.abs(x[:2, 1:3]).max() <= 1.0 + 1e-12 and np.isclose(x[:2, 1:3].max(), 1.0)
    # multiplying E and I by alpha leaves their input channels unchanged and shifts the
    # scale channel by log10(alpha) / 4
    v = u[:2].copy()
    v[:, 1:3] *= 1e-3
    xv = fno.make_input(v, np.full(2, 2.0), np.full(2, -2.0))
    np.testing.assert_allclose(xv[:, 1:3], x[:2, 1:3], rtol=1e-12)
    np.testing.assert_allclose(xv[:, 7], x[:2, 7] - 0.75, atol=1e-12)


def test_zero_increment_network_is_persistence():
    W, m, L, H, n = 4, 2, 2, 6, 8
    g = np.random.default_rng(3)
    params = fno.init_params(1, W, m, L, H)
    params["Q2"][:] = 0.0
    params["q2"][:] = 0.0
    u = g.uniform(0, 1, (2, 5, n, n))
    u[0, 1:3] *= 1e-4
    x = fno.make_input(u, np.array([1.5, 3.0]), np.array([-1.5, -2.5]))
    y, _ = fno.forward(params, x, W, m, L, H)
    np.testing.assert_allclose(y, u, rtol=1e-13, atol=0)


@pytest.mark.parametrize("mass_weight,neg_weight", [(0.0, 0.0), (10.0, 0.0), (3.0, 50.0)])
def test_loss_gradient_matches_finite_differences(mass_weight, neg_weight):
    g = np.random.default_rng(11)
    B, n = 2, 6
    u = g.uniform(0, 1, (B, 5, n, n))
    u[1, 1:3] *= 1e-3
    x = fno.make_input(u, np.array([2.0, 3.0]), np.array([-2.0, -1.0]))
    t = g.uniform(0, 1, (B, 5, n, n))
    t[1, 1:3] *= 1e-3
    y = t + g.normal(0, 0.2, t.shape)        # some entries negative
    y[1, 1:3] = t[1, 1:3] + g.normal(0, 1e-4, (2, n, n))
    _, total, dy = fno.loss(y, t, x, mass_weight, neg_weight)
    idx = [(0, 0, 1, 2), (0, 2, 3, 3), (1, 1, 0, 0), (1, 4, 5, 1), (1, 2, 2, 4)]
    idx += [tuple(int(v) for v in np.argwhere(y < 0)[0])]
    for i in idx:
        h = 1e-7 * max(1e-3, abs(y[i]))
        yp, ym = y.copy(), y.copy()
        yp[i] += h
        ym[i] -= h
        fd = (fno.loss(yp, t, x, mass_weight, neg_weight)[1] - fno.loss(ym, t, x, mass_weight, neg_weight)[1]) / (2 * h)
        assert fd == pytest.approx(dy[i], rel=1e-5, abs=1e-12), (i, fd, dy[i])
    # the weighted error of E and I is measured in units of the infection scale
    sig = fno.out_scale(x)
    ref = np.mean(((y - t) / sig[:, :, None, None]) ** 2)
    assert fno.loss(y, t, x)[0] == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("spread", [0.3, 3.0])
def test_prediction_is_nonnegative_and_conserves_the_population_exactly(spread):
    """For any parameters (here random, with large ones that push many values below zero
    before the clamp) the prediction is nonnegative and holds its input's population."""
    W, m, L, H, n = 4, 2, 2, 6, 8
    g = np.random.default_rng(8)
    params = fno.init_params(2, W, m, L, H)
    for k in params:
        params[k] = params[k] + spread * g.standard_normal(params[k].shape)
    u = g.uniform(0, 1, (3, 5, n, n))
    u[2, 1:3] *= 1e-5
    x = fno.make_input(u, np.array([1.5, 3.0, 2.0]), np.array([-1.5, -2.5, -2.0]))
    y, cache = fno.forward(params, x, W, m, L, H)
    assert y.min() >= 0.0
    np.testing.assert_allclose(y.reshape(3, -1).sum(axis=1), u.reshape(3, -1).sum(axis=1), rtol=1e-13)
    # with the large parameters the clamp acts (some pre-clamp values are negative); either way
    # the raw prediction does not conserve: the rescale is doing the work
    assert (cache["a"] < 0).any() or spread < 1
    sig = fno.out_scale(x)[:, :, None, None]
    v = sig * np.maximum(cache["a"], 0.0)
    assert np.abs(v.reshape(3, -1).sum(axis=1) - u.reshape(3, -1).sum(axis=1)).max() > 1e-3
    # y = v scaled by the ratio of the populations, per sample
    ratio = u.reshape(3, -1).sum(axis=1) / v.reshape(3, -1).sum(axis=1)
    np.testing.assert_allclose(y, v * ratio[:, None, None, None], rtol=1e-13, atol=0)


def test_all_clamped_prediction_is_zero():
    """If every value of a sample is clamped (sum v = 0) the prediction is 0: its conservation
    residual is then 1, so the rollout's check sends it to the SSLBM."""
    W, m, L, H, n = 4, 2, 1, 6, 8
    params = fno.init_params(3, W, m, L, H)
    params["Q2"][:] = 0.0
    params["q2"][:] = -1e6
    u = np.random.default_rng(1).uniform(0, 1, (1, 5, n, n))
    x = fno.make_input(u, np.array([2.0]), np.array([-2.0]))
    y, _ = fno.forward(params, x, W, m, L, H)
    assert not y.any()


def test_gelu_tanh_form_against_the_erf_definition_and_its_derivative():
    """The tanh form stays within 4.8e-4 of z Phi(z): the two standard GELUs differ by at
    most 4.7e-4, near |z| = 2.7 (a wrong cubic coefficient or scale moves both the size and
    the place of that gap).  gelu_grad is the derivative (central differences)."""
    import math
    z = np.linspace(-8.0, 8.0, 20001)
    erf_form = 0.5 * z * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    gap = np.abs(fno.gelu(z) - erf_form)
    assert 4.0e-4 < gap.max() < 4.8e-4
    assert 2.4 < abs(z[gap.argmax()]) < 3.0
    h = 1e-5
    fd = (fno.gelu(z + h) - fno.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(fno.gelu_grad(z), fd, rtol=0, atol=1e-8)
