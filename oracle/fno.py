"""FP64 CPU oracle of the learned surrogate (a Fourier-neural-operator-style network).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/.  The paper has no learned component;
this network is defined by this project, and this module is its plain reference: numpy,
float64, one function per operation, forward and hand-derived backward, each written as
its definition below with numpy's FFT as the only library step.  The tests pin it to a
direct double sum of the spectral convolution on small grids, to single Fourier modes
(kept modes pass with their weight, the others vanish) and to central finite differences
(every parameter gradient).  The CUDA kernels are checked against it.

Network (all per grid cell unless spectral):
    s  = max over the grid of (E, I), at least 1e-12                the infection scale
    e  = (log10(s) + 4) / 4,  s' = 10^(4 e - 4)                     (s' = s up to rounding)
    x  = [S, E/s', I/s', R, D, (R0 - 2.6)/1.4, log10(d) + 2, e]    8 input channels
    h0 = A0 x + a0                                                  lift, width W
    z_l = K_l(h_{l-1}) + B_l h_{l-1} + b_l,  h_l = gelu(z_l) (l < L), h_L = z_L
    p  = gelu(Q1 h_L + q1)                                          width H
    delta = Q2 p + q2
    v_c = sigma_c max(x_c + delta_c, 0), sigma = (1, s', s', 1, 1)  nonnegative raw prediction
                                                  (a NaN stays a NaN: numpy's maximum)
    u_c = sigma_c x_c                                                the input state
    y = v (sum u / sum v)   (y = 0 if sum v = 0)                    state 20 steps ahead
E and I enter and leave in units of the infection scale, so the early exponential phase
(E, I of order 1e-4 on S ~ 1) is learned as the scale-free problem it is; the loss weighs
E and I in the same units (weights 1 / sigma_c^2).  The clamp at zero makes every density
of the prediction nonnegative by construction, and the last step rescales the whole state
(sums over all channels and cells of a sample) to the input's population, so y conserves
the population exactly and stays nonnegative: a density can go negative, or the
population drift, only through non-finite arithmetic.
Spectral convolution K on an n x n periodic grid, kept modes kx in {0..m-1} U {n-m..n-1},
ky in {0..m-1} (2m x m modes), complex weights R[i, o, kx, ky]:
    hat_h[i, k] = sum_{x,y} h[i, y, x] exp(-2 pi i (kx x + ky y) / n)
    hat_g[o, k] = sum_i hat_h[i, k] R[i, o, k]
    K(h)[o, y, x] = 1/n^2 sum_k c_ky Re(hat_g[o, k] exp(+2 pi i (kx x + ky y) / n)),
                    c_0 = 1, c_ky = 2 (ky > 0)
evaluated here exactly so: hat_h from numpy's 2D FFT, the inverse sum as the real part of
numpy's inverse 2D FFT of the spectrum that holds c_ky hat_g on the kept modes and zero
elsewhere.  (The GPU factorises the same operator into real DFT products along x and y;
that factorisation is a subject under test, not part of this definition.)
gelu(z) = 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))): GELU in its tanh form, one of the
two standard definitions of GELU (the other is z Phi(z) with the normal CDF; they differ by
at most 4.7e-4).  The surrogate's specification names GELU without its form.
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


GELU_C = math.sqrt(2.0 / math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + 0.044715 * z ** 3))
    du = GELU_C * (1.0 + 3.0 * 0.044715 * z * z)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def _kept(n, m):
    """Index arrays (ky, kx) of the kept modes in numpy's FFT layout [.., ky, kx], each of
    shape (m, 2m), and the weights c_ky."""
    kx = kx_modes(n, m)
    ky = np.arange(m)
    c = np.where(ky == 0, 1.0, 2.0)
    return ky[:, None] * np.ones((1, 2 * m), dtype=int), np.ones((m, 1), dtype=int) * kx[None, :], c


def spectral(h, R, n, m):
    """K(h) for h[B, Ci, n, n] by the definition above; returns (out[B, Co, n, n], hat_h) with
    hat_h[B, Ci, 2m(kx), m(ky)] the kept modes of h."""
    KY, KX, c = _kept(n, m)
    F = np.fft.fft2(h)                                   # F[.., ky, kx] = sum h exp(-2 pi i (kx x + ky y)/n)
    hat_h = np.swapaxes(F[..., KY, KX], -1, -2)          # [B, Ci, 2m, m]
    Rc = R[..., 0] + 1j * R[..., 1]                      # [Ci, Co, 2m, m]
    hat_g = np.einsum("bikq,iokq->bokq", hat_h, Rc)      # [B, Co, 2m, m]
    G = np.zeros(h.shape[:1] + (R.shape[1], n, n), dtype=complex)
    G[..., KY, KX] = np.swapaxes(hat_g, -1, -2) * c[:, None]
    return np.fft.ifft2(G).real, hat_h                   # ifft2 carries the 1/n^2


def spectral_backward(dout, hat_h, R, n, m):
    """Adjoint of spectral(): returns (dh, dR) for dL/dK(h) = dout.  With hat_g = a + ib,
    K(h) = 1/n^2 sum_k c_ky (a cos t - b sin t), so dL/da + i dL/db = c_ky/n^2 (FFT of dout)[k];
    through the complex products, dL/dhat_h = sum_o dL/dhat_g conj(R) and
    dL/dR = sum_b conj(hat_h) dL/dhat_g; and with hat_h = sum_x h exp(-i t),
    dL/dh = Re(sum_k dL/dhat_h exp(+i t)) = Re(n^2 ifft2(dL/dhat_h on the kept modes))."""
    KY, KX, c = _kept(n, m)
    D = np.fft.fft2(dout)
    dg = np.swapaxes(D[..., KY, KX] * c[:, None], -1, -2) / (n * n)   # [B, Co, 2m, m]
    Rc = R[..., 0] + 1j * R[..., 1]
    dRc = np.einsum("bikq,bokq->iokq", np.conj(hat_h), dg)
    dhat = np.einsum("bokq,iokq->bikq", dg, np.conj(Rc))              # [B, Ci, 2m, m]
    G = np.zeros(dout.shape[:1] + (R.shape[0], n, n), dtype=complex)
    G[..., KY, KX] = np.swapaxes(dhat, -1, -2)
    dh = (np.fft.ifft2(G) * (n * n)).real
    return dh, np.stack([dRc.real, dRc.imag], axis=-1)


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
    a = x[:, :5] + pointwise(params["Q2"], p, params["q2"])
    v = sig * np.maximum(a, 0.0)
    u = sig * x[:, :5]
    B = x.shape[0]
    su = u.reshape(B, -1).sum(axis=1)
    sv = v.reshape(B, -1).sum(axis=1)
    r = np.where(sv > 0, su / np.where(sv > 0, sv, 1.0), 0.0)
    y = v * r[:, None, None, None]
    cache["a"], cache["r"], cache["sv"] = a, r, sv
    return y, cache


def backward(params, cache, dy, W=32, m=12, L=4, H=64):
    """Gradients of a scalar loss with dL/dy = dy, for every parameter."""
    n = dy.shape[-1]
    g = {}
    p = cache["p"]
    sig = out_scale(cache["x"])[:, :, None, None]
    B = dy.shape[0]
    a, r, sv = cache["a"], cache["r"], cache["sv"]
    v = sig * np.maximum(a, 0.0)
    # y = r v with r = sum u / sum v: dL/dv = r (dy - lam), lam = sum(dy v) / sum v; then
    # v_c = sigma_c max(a_c, 0) with a = x + delta
    lam = (dy * v).reshape(B, -1).sum(axis=1) / np.where(sv > 0, sv, 1.0)
    dv = r[:, None, None, None] * (dy - lam[:, None, None, None])
    dy = dv * sig * (a > 0)                                  # dL/d delta
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
        dh_spec, g[f"R{l}"] = spectral_backward(dz, cache[f"hat{l}"], params[f"R{l}"], n, m)
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


# ---- per-element error scale of a BF16 evaluation ----------------------------------------

U_BF16 = 2.0 ** -8      # unit roundoff of BF16 (8 significant bits)
TANH_ERR = 2.0 ** -9    # bound on the absolute error of an approximate tanh inside an evaluated GELU


def sq_spectral(v, R, n, m):
    """sum_i kappa_io^2 (*) v_i for v[B, Ci, n, n] >= 0, with kappa_io the spatial kernel of
    the spectral convolution (K(h)_o = sum_i kappa_io (*) h_i, circular convolution): the
    variance of K(e) for independent errors e of variance v, and, with v = h^2, the sum of the
    squares of the terms of K(h)."""
    KY, KX, c = _kept(n, m)
    Ci, Co = R.shape[:2]
    Fv = np.fft.fft2(v)
    out = np.zeros(v.shape[:1] + (Co, n, n))
    Rc = R[..., 0] + 1j * R[..., 1]
    for o in range(Co):
        G = np.zeros((Ci, n, n), dtype=complex)
        G[:, KY, KX] = np.swapaxes(Rc[:, o], -1, -2) * c[:, None]
        k2 = np.fft.ifft2(G).real ** 2                      # [Ci, n, n]
        out[:, o] = np.fft.ifft2((np.fft.fft2(k2)[None] * Fv).sum(axis=1)).real
    return np.maximum(out, 0.0)


def sq_spectral_adjoint(v, R, n, m):
    """sum_o kappa_io(-.)^2 (*) v_o for v[B, Co, n, n] >= 0: the variance of K^T(e) (the adjoint,
    whose kernel is kappa flipped in space) for independent errors e of variance v."""
    KY, KX, c = _kept(n, m)
    Ci, Co = R.shape[:2]
    Fv = np.fft.fft2(v)
    out = np.zeros(v.shape[:1] + (Ci, n, n))
    Rc = R[..., 0] + 1j * R[..., 1]
    for i in range(Ci):
        G = np.zeros((Co, n, n), dtype=complex)
        G[:, KY, KX] = np.swapaxes(Rc[i], -1, -2) * c[:, None]
        k2 = np.fft.ifft2(G).real ** 2                      # [Co, n, n]
        out[:, i] = np.fft.ifft2((np.conj(np.fft.fft2(k2))[None] * Fv).sum(axis=1)).real
    return np.maximum(out, 0.0)


def _row_power(f, n, m):
    """sum over rows y of |sum_x f[.., y, x] exp(-2 pi i kx x / n)|^2 for the kept kx: the
    size of the partial transforms along x that a factorised DFT rounds -> [.., 2m]."""
    P = np.fft.fft(f, axis=-1)[..., kx_modes(n, m)]
    return (np.abs(P) ** 2).sum(axis=-2)


def _mode_rounding_var(f, n, m, q):
    """Variance of a kept mode of f computed as a factorised DFT (along x, then y) whose
    operands and partial transforms are rounded with relative variance q: two roundings on
    the cells' terms, two on the partial transforms -> [.., 2m] (the same for every ky)."""
    return 2.0 * q * ((f * f).sum(axis=(-2, -1))[..., None] + _row_power(f, n, m))


def _inverse_rounding_var(spec, n, m, q):
    """Variance, per row y, of an inverse transform of the kept-mode coefficients spec[.., 2m, m]
    (the c_ky weights included) evaluated as a factorised inverse DFT (along y, then x) whose
    partial transforms and operands are rounded with relative variance q -> [.., n]."""
    G = np.zeros(spec.shape[:-2] + (n, 2 * m), dtype=complex)
    G[..., :m, :] = np.swapaxes(spec, -1, -2)
    G1 = np.fft.ifft(G, axis=-2) * n                        # [.., n(y), 2m(kx)]
    return 2.0 * q * ((np.abs(G1) ** 2).sum(axis=-1) + (np.abs(spec) ** 2).sum(axis=(-2, -1))[..., None])


def spectral_rounding_var(h, hat_h, R, n, m, q):
    """Variance, per output cell, that a factorised evaluation of K(h) adds by rounding its own
    operands and intermediates (the errors of h itself are carried by sq_spectral): the
    forward transform's mode errors mixed by R and summed back to every cell, and the inverse
    transform's roundings -> [B, Co, n, n]."""
    KY, KX, c = _kept(n, m)
    Vhat = _mode_rounding_var(h, n, m, q)                   # [B, Ci, 2m]
    R2 = R[..., 0] ** 2 + R[..., 1] ** 2                    # [Ci, Co, 2m, m]
    Vg = np.einsum("bik,iokq->bokq", Vhat, R2) * (c * c)[None, None, None, :]
    const = Vg.sum(axis=(-2, -1)) / float(n) ** 4           # [B, Co]
    Rc = R[..., 0] + 1j * R[..., 1]
    g = np.einsum("bikq,iokq->bokq", hat_h, Rc) * c[None, None, None, :]
    inv = _inverse_rounding_var(g, n, m, q) / float(n) ** 4  # [B, Co, n]
    return const[..., None, None] + inv[..., :, None] * np.ones((1, 1, 1, n))


def _gelu_grad2(z):
    """Second derivative of the tanh-form GELU (central difference of gelu_grad)."""
    e = 1e-4
    return (gelu_grad(z + e) - gelu_grad(z - e)) / (2 * e)


def rounding_variances(params, x, cache, W=32, m=12, L=4, H=64, u=U_BF16):
    """Variances, per element, of the errors of an evaluation of the network that stores its
    activations in BF16 and evaluates each spectral convolution as factorised DFT products
    (along x, then y, and back) whose operands and partial transforms are rounded to BF16,
    with FP32 accumulation (neglected) and the same parameters.  Each rounding is modelled as
    an independent relative error of variance q = u^2/3 (uniform in [-u, u]), and the tanh
    inside each GELU as one with absolute error uniform in [-TANH_ERR, TANH_ERR] (variance
    qt = TANH_ERR^2/3, entering the GELU as 0.5 z dt), carried forward to first order by a
    second pass over the definition on squares:
        V(h0) = q h0^2
        V(z_l) = Ks_l(V(h_{l-1})) + B_l^2 V(h_{l-1}) + Sr_l(h_{l-1})
        V(h_l) = gelu'(z_l)^2 V(z_l) + qt (z_l/2)^2 + q h_l^2     (h_L = z_L: no gelu)
        V(zp) = Q1^2 V(h_L),  V(p) = gelu'(zp)^2 V(zp) + qt (zp/2)^2 + q p^2,  V(delta) = Q2^2 V(p)
        V(v) = sigma^2 V(delta),   V(y) = r^2 V(v) + y^2 sum V(v) / (sum v)^2
    with Ks = sq_spectral, Sr = spectral_rounding_var (the product's own roundings) and
    squares of matrices taken elementwise (V(h_l) etc. with q for u^2/3 as above).  Returns
    a dict with these variances (keys h0..hL, z1..zL, zp, p, delta, y)."""
    n = x.shape[-1]
    q = u * u / 3.0
    qt = TANH_ERR * TANH_ERR / 3.0
    h = cache["h0"]
    out = {"h0": q * h * h}
    V = out["h0"]
    for l in range(1, L + 1):
        R, Bl = params[f"R{l}"], params[f"B{l}"]
        Vz = (sq_spectral(V, R, n, m) + pointwise(Bl * Bl, V)
              + spectral_rounding_var(h, cache[f"hat{l}"], R, n, m, q))
        h = cache[f"h{l}"]
        if l < L:
            zl = cache[f"z{l}"]
            gz = gelu_grad(zl)
            V = gz * gz * Vz + qt * (0.5 * zl) ** 2 + q * h * h
        else:
            V = Vz + q * h * h
        out[f"z{l}"], out[f"h{l}"] = Vz, V
    out["zp"] = pointwise(params["Q1"] ** 2, V)
    gp = gelu_grad(cache["zp"])
    out["p"] = gp * gp * out["zp"] + qt * (0.5 * cache["zp"]) ** 2 + q * cache["p"] ** 2
    out["delta"] = pointwise(params["Q2"] ** 2, out["p"])
    sig = out_scale(x)[:, :, None, None]
    Vv = sig * sig * out["delta"]
    B = x.shape[0]
    r, sv = cache["r"], cache["sv"]
    y = sig * np.maximum(cache["a"], 0.0) * r[:, None, None, None]
    rel_r = Vv.reshape(B, -1).sum(axis=1) / np.where(sv > 0, sv, 1.0) ** 2
    out["y"] = r[:, None, None, None] ** 2 * Vv + y * y * rel_r[:, None, None, None]
    return out


def rounding_sd(params, x, cache, W=32, m=12, L=4, H=64, u=U_BF16):
    """Standard deviation of the error of each output element (rounding_variances)."""
    return np.sqrt(rounding_variances(params, x, cache, W, m, L, H, u)["y"])


def gradient_rounding_sd(params, x, cache, dy, W=32, m=12, L=4, H=64, u=U_BF16, mask_sds=4.0):
    """Standard deviation of the error of each parameter gradient (dL/dy = dy given exactly)
    for an evaluation whose forward pass is modelled by rounding_variances and whose backward
    pass rounds both operands of every per-cell product and of every spectral adjoint product
    to BF16.  The backward signal's variance follows the adjoint on squares; a weight gradient
    sum_t d_t a_t gets sum_t [a_t^2 (V(d_t) + u^2/3 d_t^2) + d_t^2 V(a_t)]; the derivative of
    gelu at a BF16-stored pre-activation z gets gelu''(z)^2 (V(z) + u^2/3 z^2); a clamped value
    within mask_sds standard deviations of zero may flip its mask, which gives that cell's
    seed its full size as an error."""
    n = x.shape[-1]
    q = u * u / 3.0
    Vf = rounding_variances(params, x, cache, W, m, L, H, u)
    sig = out_scale(x)[:, :, None, None]
    B = x.shape[0]
    a, r, sv = cache["a"], cache["r"], cache["sv"]
    v = sig * np.maximum(a, 0.0)
    lam = (dy * v).reshape(B, -1).sum(axis=1) / np.where(sv > 0, sv, 1.0)
    full = r[:, None, None, None] * sig * (dy - lam[:, None, None, None])
    d = full * (a > 0)
    near = np.abs(a) <= mask_sds * np.sqrt(Vf["delta"])
    Vd = near * full * full + q * d * d
    sd = {}

    def wsum(dv, Vdv, act, Vact):
        """V of sum_(b,cell) d a^T with both operands rounded to BF16: [rows, cols]."""
        return (np.einsum("boyx,biyx->oi", Vdv + q * dv * dv, act * act)
                + np.einsum("boyx,biyx->oi", dv * dv, Vact + q * act * act))

    sd["q2"] = Vd.sum(axis=(0, 2, 3))
    sd["Q2"] = wsum(d, Vd, cache["p"], Vf["p"])
    Vdp = pointwise((params["Q2"] ** 2).T, Vd + q * d * d)
    dp = pointwise(params["Q2"].T, d)
    g1, g2 = gelu_grad(cache["zp"]), _gelu_grad2(cache["zp"])
    dz = dp * g1
    Vdz = g1 * g1 * Vdp + dp * dp * g2 * g2 * (Vf["zp"] + q * cache["zp"] ** 2)
    sd["q1"] = Vdz.sum(axis=(0, 2, 3))
    sd["Q1"] = wsum(dz, Vdz, cache[f"h{L}"], Vf[f"h{L}"])
    dh = pointwise(params["Q1"].T, dz)
    Vdh = pointwise((params["Q1"] ** 2).T, Vdz + q * dz * dz)
    for l in range(L, 0, -1):
        if l < L:
            zl = cache[f"z{l}"]
            g1, g2 = gelu_grad(zl), _gelu_grad2(zl)
            Vdz = g1 * g1 * Vdh + dh * dh * g2 * g2 * (Vf[f"z{l}"] + q * zl * zl)
            dz = dh * g1
        else:
            Vdz, dz = Vdh, dh
        hp, Vhp = cache[f"h{l - 1}"], Vf[f"h{l - 1}"]
        R = params[f"R{l}"]
        sd[f"b{l}"] = Vdz.sum(axis=(0, 2, 3))
        sd[f"B{l}"] = wsum(dz, Vdz, hp, Vhp)
        # spectral weights: dR[i,o,k] = sum_b conj(hat_h[b,i,k]) dg[b,o,k], dg = c/n^2 FFT(dz)[k]:
        # both factors carry their propagated errors and the factorised transforms' roundings
        KY, KX, c = _kept(n, m)
        c2 = (c * c)[None, None, None, :]
        hat = cache[f"hat{l}"]                               # [B, Ci, 2m, m]
        Vhat = (Vhp.sum(axis=(2, 3))[..., None] + _mode_rounding_var(hp, n, m, q))[..., None] * np.ones(m)
        dg = np.swapaxes(np.fft.fft2(dz)[..., KY, KX] * c[:, None], -1, -2) / (n * n)
        Vdg = ((Vdz.sum(axis=(2, 3))[..., None] + _mode_rounding_var(dz, n, m, q))[..., None] * np.ones(m)
               * c2 / float(n) ** 4)
        VdR = (np.einsum("bikq,bokq->iokq", np.abs(hat) ** 2, Vdg)
               + np.einsum("bikq,bokq->iokq", Vhat, np.abs(dg) ** 2))
        sd[f"R{l}"] = np.stack([VdR, VdR], axis=-1)
        # the adjoint: dh = Re(sum_k dhat_k exp(+i t)), dhat = sum_o dg conj(R): propagated
        # errors of dz through the flipped kernel, the transform's mode errors mixed by R, and
        # the inverse transform's roundings
        dhs, _ = spectral_backward(dz, hat, R, n, m)
        R2 = R[..., 0] ** 2 + R[..., 1] ** 2
        Vmode = np.einsum("bok,iokq->bikq", _mode_rounding_var(dz, n, m, q), R2) * c2 / float(n) ** 4
        Rc = R[..., 0] + 1j * R[..., 1]
        dhat = np.einsum("bokq,iokq->bikq", dg, np.conj(Rc))
        Vdhs = (sq_spectral_adjoint(Vdz, R, n, m) + Vmode.sum(axis=(-2, -1))[..., None, None]
                + _inverse_rounding_var(dhat, n, m, q)[..., :, None])
        dh = pointwise(params[f"B{l}"].T, dz) + dhs
        Vdh = pointwise((params[f"B{l}"] ** 2).T, Vdz + q * dz * dz) + Vdhs
    sd["a0"] = Vdh.sum(axis=(0, 2, 3))
    sd["A0"] = wsum(dh, Vdh, x, np.zeros_like(x))
    return {k: np.sqrt(v) for k, v in sd.items()}
