"""FP64 CPU oracle of the learned surrogate (a Fourier-neural-operator-style network).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/.  The paper has no learned component;
this network is defined by this project, and this module is its plain reference: numpy,
float64, one function per operation, forward and hand-derived backward.  The tests pin it
to numpy's FFT (the spectral convolution equals irfft2 of the mixed, truncated rfft2) and
to central finite differences (every parameter gradient).  The CUDA kernels are checked
against it.

Network (all per grid cell unless spectral):
    s  = max over the grid of (E, I), at least 1e-12                the infection scale
    e  = (log10(s) + 4) / 4,  s' = 10^(4 e - 4)                     (s' = s up to rounding)
    x  = [S, E/s', I/s', R, D, (R0 - 2.6)/1.4, log10(d) + 2, e]    8 input channels
    h0 = A0 x + a0                                                  lift, width W
    z_l = K_l(h_{l-1}) + B_l h_{l-1} + b_l,  h_l = gelu(z_l) (l < L), h_L = z_L
    p  = gelu(Q1 h_L + q1)                                          width H
    delta = Q2 p + q2
    v_c = sigma_c (x_c + delta_c), sigma = (1, s', s', 1, 1)        raw prediction
    u_c = sigma_c x_c                                                the input state
    y = v - u kappa,  kappa = (sum v - sum u) / sum u               state 20 steps ahead
E and I enter and leave in units of the infection scale, so the early exponential phase
(E, I of order 1e-4 on S ~ 1) is learned as the scale-free problem it is; the loss weighs
E and I in the same units (weights 1 / sigma_c^2).  The last step removes the raw
prediction's change of the total population in proportion to the input state (sums over
all channels and cells of a sample), so y conserves the population exactly and zero
fields stay zero.
Spectral convolution K on an n x n periodic grid, kept modes kx in {0..m-1} U {n-m..n-1},
ky in {0..m-1} (2m x m modes), complex weights R[i, o, kx, ky]:
    hat_h[k] = sum_{x,y} h[y, x] exp(-2 pi i (kx x + ky y) / n)
    hat_g[o, k] = sum_i hat_h[i, k] R[i, o, k]
    K(h)[o, y, x] = 1/n^2 sum_k c_ky Re(hat_g[o, k] exp(+2 pi i (kx x + ky y) / n)),
                    c_0 = 1, c_ky = 2 (ky > 0)
It is evaluated here as real DFT products, the factorisation the GPU uses:
    H1 = h Fx (along x), T = Fy H1 (along y), hat_h = combine(T), hat_g = mix(hat_h, R),
    U = expand(hat_g), G1 = Fyi U, K(h) = G1 Fxi / n^2.
gelu(z) = 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))): GELU in its tanh form, one of the
two standard definitions of GELU (the other is z Phi(z) with the normal CDF; they differ by
at most 4.7e-4).  The surrogate's specification names GELU without its form; this is the
form the GPU evaluates with its tanh instruction.
Parameters are stored flat in the order of param_shapes() (the GPU uses the same layout).
"""
from __future__ import annotations

import math

import numpy as np

C_IN, C_OUT = 8, 5
SCALE_FLOOR = 1e-12


def param_shapes(W=32, m=12, L=4, H=64):
    shapes = [("A0", (W, C_IN)), ("a0", (W,))]
    for l in range(1, L + 1):
        shapes += [(f"R{l}", (W, W, 2 * m, m, 2)), (f"B{l}", (W, W)), (f"b{l}", (W,))]
    shapes += [("Q1", (H, W)), ("q1", (H,)), ("Q2", (C_OUT, H)), ("q2", (C_OUT,))]
    return shapes


def n_params(W=32, m=12, L=4, H=64):
    return sum(int(np.prod(s)) for _, s in param_shapes(W, m, L, H))


def unflatten(theta, W=32, m=12, L=4, H=64):
    out, off = {}, 0
    for name, shp in param_shapes(W, m, L, H):
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[off:off + k], dtype=np.float64).reshape(shp)
        off += k
    return out


def flatten(params, W=32, m=12, L=4, H=64):
    return np.concatenate([params[name].reshape(-1) for name, _ in param_shapes(W, m, L, H)])


def init_params(seed, W=32, m=12, L=4, H=64):
    """Seeded initial parameters (uniform fan-in scaling)."""
    g = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes(W, m, L, H):
        if name.startswith("R"):
            scale = 1.0 / (W * W)
            p[name] = scale * g.uniform(-1, 1, shp)
        elif len(shp) == 2:
            bound = 1.0 / math.sqrt(shp[1])
            p[name] = g.uniform(-bound, bound, shp)
        else:
            p[name] = np.zeros(shp)
    return p


def kx_modes(n, m):
    return np.array([j if j < m else n - 2 * m + j for j in range(2 * m)])


def dft_mats(n, m):
    """Real DFT factors: Fx (n x 4m), Fy (2m x n), Fyi (n x 2m), Fxi (4m x n)."""
    x = np.arange(n)
    kx = kx_modes(n, m)
    ky = np.arange(m)
    thx = 2 * np.pi * np.outer(x, kx) / n          # n x 2m
    thy = 2 * np.pi * np.outer(ky, x) / n          # m x n
    Fx = np.empty((n, 4 * m))
    Fx[:, 0::2] = np.cos(thx)
    Fx[:, 1::2] = -np.sin(thx)
    Fy = np.empty((2 * m, n))
    Fy[0::2] = np.cos(thy)
    Fy[1::2] = -np.sin(thy)
    Fyi = np.empty((n, 2 * m))
    Fyi[:, 0::2] = np.cos(thy).T
    Fyi[:, 1::2] = np.sin(thy).T
    Fxi = np.empty((4 * m, n))
    Fxi[0::2] = np.cos(thx).T
    Fxi[1::2] = -np.sin(thx).T
    return Fx, Fy, Fyi, Fxi


GELU_C = math.sqrt(2.0 / math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + 0.044715 * z ** 3))
    du = GELU_C * (1.0 + 3.0 * 0.044715 * z * z)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def combine(T):
    """T[..., 2m, 4m] (rows: cos/-sin along y, cols: Re/Im along x) -> hat_h[..., 2m(kx), m(ky)] complex."""
    Tc, Ts = T[..., 0::2, :], T[..., 1::2, :]            # [..., m(ky), 4m]
    re = Tc[..., 0::2] - Ts[..., 1::2]                   # [..., m, 2m]
    im = Tc[..., 1::2] + Ts[..., 0::2]
    return np.swapaxes(re + 1j * im, -1, -2)             # [..., 2m, m]


def combine_adjoint(dhat):
    """Adjoint of combine for real-valued derivatives: d(re), d(im) -> dT."""
    d = np.swapaxes(dhat, -1, -2)                        # [..., m, 2m]
    dre, dim = d.real, d.imag
    shp = d.shape[:-2] + (2 * d.shape[-2], 2 * d.shape[-1])
    dT = np.zeros(shp)
    dT[..., 0::2, 0::2] = dre
    dT[..., 1::2, 1::2] = -dre
    dT[..., 0::2, 1::2] = dim
    dT[..., 1::2, 0::2] = dim
    return dT


def expand(hat_g):
    """hat_g[..., 2m, m] complex -> U[..., 2m(ky rows cos/sin), 4m] with the c_ky weights."""
    m = hat_g.shape[-1]
    c = np.where(np.arange(m) == 0, 1.0, 2.0)
    gT = np.swapaxes(hat_g, -1, -2) * c[:, None]         # [..., m, 2m]
    shp = gT.shape[:-2] + (2 * m, 2 * gT.shape[-1])
    U = np.zeros(shp)
    U[..., 0::2, 0::2] = gT.real
    U[..., 1::2, 0::2] = -gT.imag
    U[..., 0::2, 1::2] = gT.imag
    U[..., 1::2, 1::2] = gT.real
    return U


def expand_adjoint(dU):
    m = dU.shape[-2] // 2
    c = np.where(np.arange(m) == 0, 1.0, 2.0)
    dre = dU[..., 0::2, 0::2] + dU[..., 1::2, 1::2]
    dim = -dU[..., 1::2, 0::2] + dU[..., 0::2, 1::2]
    d = (dre + 1j * dim) * c[:, None]                    # [..., m, 2m]
    return np.swapaxes(d, -1, -2)


def spectral(h, R, n, m):
    """K(h) for h[B, Ci, n, n]; returns (out[B, Co, n, n], hat_h) via the real DFT products."""
    Fx, Fy, Fyi, Fxi = dft_mats(n, m)
    H1 = h @ Fx                                          # [B, Ci, n, 4m]
    T = Fy @ H1                                          # [B, Ci, 2m, 4m]
    hat_h = combine(T)                                   # [B, Ci, 2m, m]
    Rc = R[..., 0] + 1j * R[..., 1]                      # [Ci, Co, 2m, m]
    hat_g = np.einsum("bikq,iokq->bokq", hat_h, Rc)
    U = expand(hat_g)                                    # [B, Co, 2m, 4m]
    G1 = Fyi @ U                                         # [B, Co, n, 4m]
    return (G1 @ Fxi) / (n * n), hat_h


def spectral_fft(h, R, n, m):
    """The same operator through numpy's FFT (the pin of the DFT factorisation)."""
    F = np.fft.fft2(h)                                   # over (y, x): F[.., ky, kx]
    kx = kx_modes(n, m)
    hat_h = np.transpose(F[..., :m, :][..., kx], (0, 1, 3, 2))  # [B, Ci, 2m(kx), m(ky)]
    Rc = R[..., 0] + 1j * R[..., 1]
    hat_g = np.einsum("bikq,iokq->bokq", hat_h, Rc)
    # numpy's irfft2 takes the half spectrum along its last axis; the half axis here is ky,
    # so build the spectrum with kx as the full (first) axis and transpose the result.
    Xt = np.zeros(h.shape[:1] + (R.shape[1], n, n // 2 + 1), dtype=complex)
    Xt[:, :, kx, :m] = hat_g                             # rows kx (full axis), cols ky (half axis)
    outT = np.fft.irfft2(Xt, s=(n, n))                   # [.., x, y]
    return np.swapaxes(outT, -1, -2)


def spectral_backward(dout, h_hat, h_shape, R, n, m):
    """Adjoint of spectral(): returns (dh, dR)."""
    Fx, Fy, Fyi, Fxi = dft_mats(n, m)
    dG1 = (dout @ Fxi.T) / (n * n)                       # [B, Co, n, 4m]
    dU = Fyi.T @ dG1                                     # [B, Co, 2m, 4m]
    dhat_g = expand_adjoint(dU)                          # [B, Co, 2m, m] complex (dRe + i dIm)
    Rc = R[..., 0] + 1j * R[..., 1]
    dRc = np.einsum("bikq,bokq->iokq", np.conj(h_hat), dhat_g)
    dhat_h = np.einsum("bokq,iokq->bikq", dhat_g, np.conj(Rc))
    dT = combine_adjoint(dhat_h)                         # [B, Ci, 2m, 4m]
    dH1 = Fy.T @ dT                                      # [B, Ci, n, 4m]
    dh = dH1 @ Fx.T
    dR = np.stack([dRc.real, dRc.imag], axis=-1)
    return dh, dR


def pointwise(Wt, h, b=None):
    """Per-cell linear map: out[b, o, y, x] = sum_i W[o, i] h[b, i, y, x] (+ b[o])."""
    out = np.einsum("oi,biyx->boyx", Wt, h)
    if b is not None:
        out = out + b[None, :, None, None]
    return out


def make_input(u, R0, logd):
    """x[B, 8, n, n] from u[B, 5, n, n], R0[B], logd[B] (see the module docstring)."""
    B, _, n, _ = u.shape
    s = np.maximum(np.maximum(u[:, 1].reshape(B, -1).max(axis=1), u[:, 2].reshape(B, -1).max(axis=1)),
                   SCALE_FLOOR)
    e = (np.log10(s) + 4.0) / 4.0
    sp = 10.0 ** (4.0 * e - 4.0)
    x = np.empty((B, C_IN, n, n))
    x[:, :5] = u
    x[:, 1] /= sp[:, None, None]
    x[:, 2] /= sp[:, None, None]
    x[:, 5] = ((np.asarray(R0) - 2.6) / 1.4)[:, None, None]
    x[:, 6] = (np.asarray(logd) + 2.0)[:, None, None]
    x[:, 7] = e[:, None, None]
    return x


def out_scale(x):
    """sigma[B, 5] = (1, s', s', 1, 1) from the scale channel of x."""
    sp = 10.0 ** (4.0 * x[:, 7, 0, 0] - 4.0)
    sig = np.ones((x.shape[0], C_OUT))
    sig[:, 1] = sp
    sig[:, 2] = sp
    return sig


def forward(params, x, W=32, m=12, L=4, H=64):
    """y[B, 5, n, n] and the cache the backward pass needs."""
    n = x.shape[-1]
    cache = {"x": x}
    h = pointwise(params["A0"], x, params["a0"])
    cache["h0"] = h
    for l in range(1, L + 1):
        ks, hat_h = spectral(h, params[f"R{l}"], n, m)
        z = ks + pointwise(params[f"B{l}"], h, params[f"b{l}"])
        cache[f"hat{l}"] = hat_h
        cache[f"z{l}"] = z
        h = gelu(z) if l < L else z
        cache[f"h{l}"] = h
    zp = pointwise(params["Q1"], h, params["q1"])
    p = gelu(zp)
    cache["zp"], cache["p"] = zp, p
    sig = out_scale(x)[:, :, None, None]
    v = sig * (x[:, :5] + pointwise(params["Q2"], p, params["q2"]))
    u = sig * x[:, :5]
    su = u.reshape(u.shape[0], -1).sum(axis=1)
    kappa = (v.reshape(v.shape[0], -1).sum(axis=1) - su) / su
    y = v - u * kappa[:, None, None, None]
    return y, cache


def backward(params, cache, dy, W=32, m=12, L=4, H=64):
    """Gradients of a scalar loss with dL/dy = dy, for every parameter."""
    n = dy.shape[-1]
    g = {}
    p = cache["p"]
    sig = out_scale(cache["x"])[:, :, None, None]
    u = sig * cache["x"][:, :5]
    B = u.shape[0]
    lam = (dy * u).reshape(B, -1).sum(axis=1) / u.reshape(B, -1).sum(axis=1)
    dy = (dy - lam[:, None, None, None]) * sig               # d/d delta through y = v - u kappa
    g["Q2"] = np.einsum("boyx,biyx->oi", dy, p)
    g["q2"] = dy.sum(axis=(0, 2, 3))
    dp = pointwise(params["Q2"].T, dy)
    dzp = dp * gelu_grad(cache["zp"])
    hL = cache[f"h{L}"]
    g["Q1"] = np.einsum("boyx,biyx->oi", dzp, hL)
    g["q1"] = dzp.sum(axis=(0, 2, 3))
    dh = pointwise(params["Q1"].T, dzp)
    for l in range(L, 0, -1):
        dz = dh if l == L else dh * gelu_grad(cache[f"z{l}"])
        hprev = cache[f"h{l - 1}"]
        g[f"b{l}"] = dz.sum(axis=(0, 2, 3))
        g[f"B{l}"] = np.einsum("boyx,biyx->oi", dz, hprev)
        dh_spec, g[f"R{l}"] = spectral_backward(dz, cache[f"hat{l}"], hprev.shape, params[f"R{l}"], n, m)
        dh = pointwise(params[f"B{l}"].T, dz) + dh_spec
    x = cache["x"]
    g["A0"] = np.einsum("boyx,biyx->oi", dh, x)
    g["a0"] = dh.sum(axis=(0, 2, 3))
    return g


def mse(y, target):
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def loss(y, target, x, mass_weight=0.0, neg_weight=0.0):
    """The training loss and dL/dy:
        mse_w = mean over (b, c, cell) of ((y - t) / sigma_c)^2
        r_b   = (sum y_b - sum t_b) / sum t_b          relative mass residual
        n_b   = sum max(-y_b, 0) / sum t_b             relative mass below zero
        L     = mse_w + mass_weight mean_b r_b^2 + neg_weight mean_b n_b^2
    Returns (mse_w, L, dL/dy)."""
    B = y.shape[0]
    sig = out_scale(x)[:, :, None, None]
    d = y - target
    mse_w = float(np.mean((d / sig) ** 2))
    st = target.reshape(B, -1).sum(axis=1)
    r = d.reshape(B, -1).sum(axis=1) / st
    neg = np.maximum(-y, 0.0)
    nb = neg.reshape(B, -1).sum(axis=1) / st
    total = mse_w + mass_weight * float(np.mean(r ** 2)) + neg_weight * float(np.mean(nb ** 2))
    dy = 2.0 * d / (sig ** 2 * d.size)
    dy = dy + (2.0 * mass_weight / B * r / st)[:, None, None, None]
    dy = dy - (y < 0) * (2.0 * neg_weight / B * nb / st)[:, None, None, None]
    return mse_w, total, dy
