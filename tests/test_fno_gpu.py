"""The surrogate's CUDA forward/backward passes against the FP64 oracle (oracle/fno.py).

The GPU stores activations and the DFT factors in BF16 (unit roundoff 2^-9 = 2e-3) and
the channel-map weights B_l, Q1, Q2 as BF16 copies; the oracle is given the same BF16
weights, so the differences come from BF16 rounding of the activations and DFT factors
along about ten rounding stages: relative L2 errors of a few 1e-3 up to ~2e-2.  The
tolerances below (3e-2 on the network's output increment, 6e-2 on each gradient tensor,
cosine >= 0.998) are set from that and leave a dropped term or transposed operand (an
O(1) error) far outside.
"""
import numpy as np
import pytest

from oracle import fno
from paper_2603_19789_gb300 import sslbm as L

pytestmark = pytest.mark.gpu

CFG = dict(W=8, m=4, L=2, H=12)
N, B = 32, 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even) and back."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _setup(seed):
    import torch
    g = np.random.default_rng(seed)
    params = fno.init_params(seed, **CFG)
    for k in params:
        params[k] = params[k] + 0.05 * g.standard_normal(params[k].shape)
    theta = fno.flatten(params, **CFG).astype(np.float32)
    # the oracle sees the values the GPU computes with: FP32 parameters, BF16 channel maps
    p32 = fno.unflatten(theta.astype(np.float64), **CFG)
    for name in p32:
        if name[0] in "BQ" and p32[name].ndim == 2:
            p32[name] = bf16_round(p32[name]).astype(np.float64)
    u = g.uniform(0, 1, (B, 5, N, N)).astype(np.float32)
    r0 = g.uniform(1.2, 4.0, B).astype(np.float32)
    logd = g.uniform(-3, -1, B).astype(np.float32)
    s = L.Surrogate(n=N, width=CFG["W"], modes=CFG["m"], layers=CFG["L"], hidden=CFG["H"], max_batch=B)
    s.set_params(theta)
    tu = torch.from_numpy(u).cuda()
    x = s.make_input(tu, torch.from_numpy(r0).cuda(), torch.from_numpy(logd).cuda())
    xo = fno.make_input(u.astype(np.float64), r0.astype(np.float64), logd.astype(np.float64))
    return s, p32, x, xo, g


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_parameter_layout_matches_oracle():
    s = L.Surrogate(n=N, width=CFG["W"], modes=CFG["m"], layers=CFG["L"], hidden=CFG["H"], max_batch=B)
    assert s.nparams == fno.n_params(**CFG)
    s2 = L.Surrogate(n=256, width=32, modes=12, layers=4, hidden=64, max_batch=1)
    assert s2.nparams == fno.n_params(32, 12, 4, 64)


def test_make_input_matches_oracle():
    s, p32, x, xo, _ = _setup(0)
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("seed", [0, 1])
def test_forward_matches_oracle(seed):
    s, p32, x, xo, _ = _setup(seed)
    y = s.forward(x).cpu().numpy().astype(np.float64)
    yo, _ = fno.forward(p32, xo, **CFG)
    # compare the network's contribution (the residual input is exact)
    assert rel(y - xo[:, :5], yo - xo[:, :5]) < 3e-2


@pytest.mark.parametrize("seed", [0, 2])
def test_backward_matches_oracle(seed):
    import torch
    s, p32, x, xo, g = _setup(seed)
    y = s.forward(x)
    dy = g.standard_normal((B, 5, N, N)).astype(np.float32) * 1e-3
    s.backward(x, torch.from_numpy(dy).cuda())
    torch.cuda.synchronize()
    grads = fno.unflatten(s.get_grads().astype(np.float64), **CFG)
    _, cache = fno.forward(p32, xo, **CFG)
    go = fno.backward(p32, cache, dy.astype(np.float64), **CFG)
    for name in go:
        a, b = grads[name].ravel(), go[name].ravel()
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel(a, b) < 6e-2 and cos > 0.998, (name, rel(a, b), cos)


def test_training_steps_reduce_the_loss():
    import torch
    s, p32, x, xo, g = _setup(3)
    # a learnable target: a small affine change of the input state
    target = (0.9 * x[:, :5] + 0.03).contiguous()
    losses = [s.train_step(x, target, 3e-3) for _ in range(40)]
    assert losses[5] < 0.6 * losses[0] and losses[-1] < 0.3 * losses[0], losses[::5]
    # Adam moved every parameter tensor
    theta = fno.unflatten(s.get_params().astype(np.float64), **CFG)
    for name, v in theta.items():
        assert np.abs(v - fno.unflatten(fno.flatten(p32, **CFG), **CFG)[name]).max() > 0, name


def test_check_project_residuals_and_projection():
    import torch
    s = L.Surrogate(n=N, width=CFG["W"], modes=CFG["m"], layers=CFG["L"], hidden=CFG["H"], max_batch=B)
    g = np.random.default_rng(5)
    u = g.uniform(0, 1, (B, 5, N, N)).astype(np.float32)
    y = u + g.normal(0, 0.01, u.shape).astype(np.float32)
    y[0, 2, :4, :4] = -0.3
    ty = torch.from_numpy(y).cuda()
    res = s.check_project(ty, torch.from_numpy(u).cuda())
    for b in range(B):
        su, sy = u[b].astype(np.float64).sum(), y[b].astype(np.float64).sum()
        neg = np.maximum(-y[b].astype(np.float64), 0).sum()
        assert res[b, 0] == pytest.approx(abs(sy - su) / su, rel=1e-6, abs=1e-12)
        assert res[b, 1] == pytest.approx(neg / su, rel=1e-6, abs=1e-15)
    out = ty.cpu().numpy()
    assert out.min() >= 0
    np.testing.assert_allclose(out.astype(np.float64).reshape(B, -1).sum(axis=1),
                               u.astype(np.float64).reshape(B, -1).sum(axis=1), rtol=1e-5)
