"""Pins of the FP64 surrogate oracle (oracle/fno.py).

The spectral convolution evaluated as real DFT products (the factorisation the GPU uses)
must equal the same operator through numpy's FFT; every parameter gradient of the
hand-derived backward pass must equal a central finite difference of the forward pass.
"""
import numpy as np
import pytest

from oracle import fno


@pytest.mark.parametrize("n,m", [(16, 4), (32, 6), (24, 5)])
def test_spectral_dft_products_equal_numpy_fft(n, m):
    g = np.random.default_rng(n + m)
    h = g.standard_normal((2, 3, n, n))
    R = g.standard_normal((3, 4, 2 * m, m, 2))
    a, _ = fno.spectral(h, R, n, m)
    b = fno.spectral_fft(h, R, n, m)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())


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
