"""The per-element bound of the surrogate's GPU parity tests (tests/fno_cases.py), checked on
the CPU from both sides:

- it admits a BF16 evaluation: the network evaluated here in the GPU's order -- activations
  stored in BF16, each spectral convolution as real DFT products along x, then y, and back,
  with BF16 operands and BF16 partial transforms, every per-cell product of the backward
  pass on BF16 operands -- stays inside it for every output and gradient element;
- it rejects planted mistakes of the kind a kernel can make: in the forward pass (as a
  mistake in a copy of the parameters the kernel reads) two output channels swapped, a
  block of spectral modes dropped or negated, the ky > 0 modes dropped, a channel of a
  channel map zeroed; in the gradients a transposed weight gradient, the negative-kx block
  of a spectral-weight gradient dropped, its ky > 0 part halved (the c_ky weight lost), its
  imaginary part negated, two rows swapped, an input channel dropped.
"""
import numpy as np
import pytest

from oracle import fno

from fno_cases import bf16_round, case, cfg_of, excess


def _bf(a):
    return bf16_round(a).astype(np.float64)


def _dft_mats(n, m):
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


def _combine(T):
    Tc, Ts = T[..., 0::2, :], T[..., 1::2, :]
    return np.swapaxes((Tc[..., 0::2] - Ts[..., 1::2]) + 1j * (Tc[..., 1::2] + Ts[..., 0::2]), -1, -2)


def _combine_adjoint(dhat):
    d = np.swapaxes(dhat, -1, -2)
    dT = np.zeros(d.shape[:-2] + (2 * d.shape[-2], 2 * d.shape[-1]))
    dT[..., 0::2, 0::2], dT[..., 1::2, 1::2] = d.real, -d.real
    dT[..., 0::2, 1::2], dT[..., 1::2, 0::2] = d.imag, d.imag
    return dT


def _expand(hat_g, m):
    c = np.where(np.arange(m) == 0, 1.0, 2.0)
    gT = np.swapaxes(hat_g, -1, -2) * c[:, None]
    U = np.zeros(gT.shape[:-2] + (2 * m, 4 * m))
    U[..., 0::2, 0::2], U[..., 1::2, 0::2] = gT.real, -gT.imag
    U[..., 0::2, 1::2], U[..., 1::2, 1::2] = gT.imag, gT.real
    return U


def _expand_adjoint(dU, m):
    c = np.where(np.arange(m) == 0, 1.0, 2.0)
    dre = dU[..., 0::2, 0::2] + dU[..., 1::2, 1::2]
    dim = -dU[..., 1::2, 0::2] + dU[..., 0::2, 1::2]
    return np.swapaxes((dre + 1j * dim) * c[:, None], -1, -2)


def bf16_evaluation(p, x, dy, W, m, L, H):
    """y and the parameter gradients, evaluated in the GPU's order with its BF16 roundings
    (products accumulate exactly here: FP32 accumulation is neglected, as in the bound)."""
    n, B = x.shape[-1], x.shape[0]
    Fx, Fy, Fyi, Fxi = [_bf(a) for a in _dft_mats(n, m)]
    h = _bf(fno.pointwise(p["A0"], x, p["a0"]))
    c = {"h0": h}
    for l in range(1, L + 1):
        hat = _combine(Fy @ _bf(h @ Fx))
        c[f"hat{l}"] = hat
        R = p[f"R{l}"]
        hat_g = np.einsum("bikq,iokq->bokq", hat, R[..., 0] + 1j * R[..., 1])
        z = _bf(Fyi @ _expand(hat_g, m)) @ Fxi / (n * n) + fno.pointwise(p[f"B{l}"], h, p[f"b{l}"])
        c[f"z{l}"] = _bf(z)
        h = _bf(fno.gelu(z)) if l < L else _bf(z)
        c[f"h{l}"] = h
    zp = fno.pointwise(p["Q1"], h, p["q1"])
    c["zp"] = _bf(zp)
    pp = _bf(fno.gelu(zp))
    a = x[:, :5] + fno.pointwise(p["Q2"], pp, p["q2"])
    sig = fno.out_scale(x)[:, :, None, None]
    v = sig * np.maximum(a, 0)
    r = (sig * x[:, :5]).reshape(B, -1).sum(1) / v.reshape(B, -1).sum(1)
    y = v * r[:, None, None, None]
    g = {}
    lam = (dy * y).reshape(B, -1).sum(1) / y.reshape(B, -1).sum(1)
    d = sig * r[:, None, None, None] * (y > 0) * (dy - lam[:, None, None, None])
    g["q2"] = d.sum(axis=(0, 2, 3))
    g["Q2"] = np.einsum("boyx,biyx->oi", _bf(d), pp)
    dz = fno.pointwise(p["Q2"].T, _bf(d)) * fno.gelu_grad(c["zp"])
    g["q1"] = dz.sum(axis=(0, 2, 3))
    g["Q1"] = np.einsum("boyx,biyx->oi", _bf(dz), c[f"h{L}"])
    dh = fno.pointwise(p["Q1"].T, _bf(dz))
    for l in range(L, 0, -1):
        dz = dh if l == L else dh * fno.gelu_grad(c[f"z{l}"])
        g[f"b{l}"] = dz.sum(axis=(0, 2, 3))
        g[f"B{l}"] = np.einsum("boyx,biyx->oi", _bf(dz), c[f"h{l - 1}"])
        dG = _expand_adjoint(Fyi.T @ _bf(_bf(dz) @ Fxi.T / (n * n)), m)
        R = p[f"R{l}"]
        Rc = R[..., 0] + 1j * R[..., 1]
        dRc = np.einsum("bikq,bokq->iokq", np.conj(c[f"hat{l}"]), dG)
        g[f"R{l}"] = np.stack([dRc.real, dRc.imag], axis=-1)
        dT = _combine_adjoint(np.einsum("bokq,iokq->bikq", dG, np.conj(Rc)))
        dh = fno.pointwise(p[f"B{l}"].T, _bf(dz)) + _bf(Fy.T @ _bf(dT)) @ Fx.T
    g["a0"] = dh.sum(axis=(0, 2, 3))
    g["A0"] = np.einsum("boyx,biyx->oi", _bf(dh), _bf(x))
    return y, g


def _oracle_case(seed, shape):
    cfg, n = cfg_of(shape)
    theta, p64, u, r0, logd, g = case(seed, shape, early=True)
    x = fno.make_input(u.astype(np.float64), r0.astype(np.float64), logd.astype(np.float64))
    dy = g.standard_normal(u.shape).astype(np.float32).astype(np.float64) * 1e-3
    y, cache = fno.forward(p64, x, **cfg)
    return cfg, n, p64, x, dy, y, cache


@pytest.mark.parametrize("shape", ["generic", "fused16"])
@pytest.mark.parametrize("seed", [2, 3])
def test_bound_admits_a_bf16_evaluation(shape, seed):
    cfg, n, p64, x, dy, y, cache = _oracle_case(seed, shape)
    go = fno.backward(p64, cache, dy, **cfg)
    sd_y = fno.rounding_sd(p64, x, cache, **cfg)
    sd_g = fno.gradient_rounding_sd(p64, x, cache, dy, **cfg)
    ye, ge = bf16_evaluation(p64, x, dy, **cfg)
    assert np.abs(ye - y).max() > 0  # the emulation does round
    assert excess(ye, y, sd_y) <= 0.5          # at most 5 sd: a margin of two below the bound
    for name in go:
        assert excess(ge[name], go[name], sd_g[name]) <= 0.6, name


def _forward_mutants(p, m):
    out = {}
    q = dict(p)
    q["Q2"] = p["Q2"][[0, 2, 1, 3, 4]]
    out["E and I output rows of Q2 swapped"] = q
    q = dict(p)
    q["R1"] = p["R1"].copy()
    q["R1"][:, :, m:] = 0.0
    out["negative-kx mode block of R1 dropped"] = q
    q = dict(p)
    q["R2"] = p["R2"].copy()
    q["R2"][:, :, :m, :, 0] *= -1.0
    out["real part of the positive-kx block of R2 negated"] = q
    q = dict(p)
    q["R1"] = p["R1"].copy()
    q["R1"][:, :, :, 1:] = 0.0
    out["ky > 0 modes of R1 dropped"] = q
    q = dict(p)
    q["B1"] = p["B1"].copy()
    q["B1"][3] = 0.0
    out["output channel 3 of B1 zeroed"] = q
    return out


@pytest.mark.parametrize("shape", ["generic", "fused16"])
def test_bound_rejects_planted_forward_mistakes(shape):
    cfg, n, p64, x, dy, y, cache = _oracle_case(2, shape)
    sd_y = fno.rounding_sd(p64, x, cache, **cfg)
    for name, q in _forward_mutants(p64, cfg["m"]).items():
        ym, _ = fno.forward(q, x, **cfg)
        assert excess(ym, y, sd_y) > 1.0, name


@pytest.mark.parametrize("shape", ["generic", "fused16"])
def test_bound_rejects_planted_gradient_mistakes(shape):
    cfg, n, p64, x, dy, y, cache = _oracle_case(3, shape)
    m = cfg["m"]
    go = fno.backward(p64, cache, dy, **cfg)
    sd_g = fno.gradient_rounding_sd(p64, x, cache, dy, **cfg)
    mutants = {
        "transposed dB1": ("B1", lambda a: a.T.copy()),
        "negative-kx block of dR1 dropped": ("R1", lambda a: np.concatenate([a[:, :, :m], 0 * a[:, :, m:]], axis=2)),
        "ky > 0 part of dR2 halved": ("R2", lambda a: np.concatenate([a[:, :, :, :1], 0.5 * a[:, :, :, 1:]], axis=3)),
        "imaginary part of dR2 negated": ("R2", lambda a: np.stack([a[..., 0], -a[..., 1]], axis=-1)),
        "rows 0 and 1 of dQ1 swapped": ("Q1", lambda a: a[[1, 0] + list(range(2, a.shape[0]))]),
        "input channel 1 of dA0 dropped": ("A0", lambda a: a * (np.arange(a.shape[1]) != 1)),
    }
    for what, (name, f) in mutants.items():
        assert excess(f(go[name]), go[name], sd_g[name]) > 1.0, what
