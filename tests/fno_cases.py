"""Seeded surrogate test cases and the element-wise comparison shared by the GPU parity tests
(test_fno_gpu.py) and the CPU checks of their bound (test_fno_bound_cpu.py).

The bound: an element a of a BF16 evaluation (activations stored in BF16, the spectral
convolutions factorised into DFT products with BF16 operands and partial transforms, FP32
accumulation) may differ from the FP64 oracle's value b by at most
    TOL_SDS * sd + FP32_SLACK * |b| + floor,
with sd the standard deviation of that element's rounding error from the oracle's second
pass on squares (oracle.fno.rounding_sd for the network's output,
oracle.fno.gradient_rounding_sd for the gradients), FP32_SLACK a few FP32 roundings of the
value itself, and floor = 1e-7 of the tensor's largest value (FP32 accumulation of sums
near zero).  TOL_SDS = 10: an emulated BF16 evaluation reaches at most 3.4 sd on the output
and 5.0 on the gradients (the Gaussian maximum over their 1e5..6e5 elements), while a swapped
output channel, a dropped or negated block of spectral modes or a transposed weight gradient
moves elements by 15 to 2000 sd (test_fno_bound_cpu.py).
"""
import numpy as np

from oracle import fno

# (W, m, L, H, n): the generic products at 32; the fused kernels at 64 and 128
SHAPES = {"generic": (8, 4, 2, 12, 32), "fused16": (16, 8, 2, 32, 64), "fused32": (32, 12, 2, 64, 128)}
B = 2
TOL_SDS = 10.0
FP32_SLACK = 8 * 2.0 ** -24


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even) and back."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def cfg_of(shape):
    W, m, Lr, H, n = SHAPES[shape]
    return dict(W=W, m=m, L=Lr, H=H), n


def case(seed, shape, early=False):
    """(theta float32 flat, p64 oracle parameters, u float32 states, r0, logd, rng).
    The oracle's parameters are the FP32 values the GPU holds, with the channel maps B_l, Q1,
    Q2 rounded to BF16 as the GPU stores them; the spectral weights are FP32 on both sides."""
    cfg, n = cfg_of(shape)
    g = np.random.default_rng(seed)
    params = fno.init_params(seed, **cfg)
    for k in params:
        params[k] = params[k] + 0.05 * g.standard_normal(params[k].shape)
    theta = fno.flatten(params, **cfg).astype(np.float32)
    p64 = fno.unflatten(theta.astype(np.float64), **cfg)
    for name in p64:
        if name[0] in "BQ" and p64[name].ndim == 2:
            p64[name] = bf16_round(p64[name]).astype(np.float64)
    u = g.uniform(0, 1, (B, 5, n, n)).astype(np.float32)
    if early:  # an early-growth sample: E, I of order 1e-4
        u[0, 1:3] *= 1e-4
    r0 = g.uniform(1.2, 4.0, B).astype(np.float32)
    logd = g.uniform(-3, -1, B).astype(np.float32)
    return theta, p64, u, r0, logd, g


def excess(got, want, sd):
    """Largest ratio |got - want| / bound over the elements (> 1: the comparison fails)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    floor = 1e-7 * max(np.abs(want).max(), 1e-300)
    bound = TOL_SDS * sd + FP32_SLACK * np.abs(want) + floor
    return float((np.abs(got - want) / bound).max())


def assert_within(got, want, sd, what):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    floor = 1e-7 * max(np.abs(want).max(), 1e-300)
    bound = TOL_SDS * sd + FP32_SLACK * np.abs(want) + floor
    ratio = np.abs(got - want) / bound
    i = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    assert ratio[i] <= 1.0, (f"{what}: element {i} differs by {abs(got[i] - want[i]):.3e} "
                             f"(got {got[i]:.6e}, oracle {want[i]:.6e}, sd {sd[i]:.3e}); "
                             f"{int((ratio > 1).sum())} of {ratio.size} elements outside the bound")
    return float(ratio.max())
