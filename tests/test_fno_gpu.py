"""The surrogate's CUDA forward/backward passes and training loss against the FP64 oracle
(oracle/fno.py), for a shape that runs the generic products and shapes that run the fused
per-row kernels.

Every output element and every gradient element is compared with the oracle's value, within
the per-element bound of tests/fno_cases.py: 10 standard deviations of that element's BF16
rounding error, as the oracle's second pass on squares gives it (the GPU stores activations
and the DFT factors in BF16; the oracle is given the GPU's parameters with the channel maps
rounded to BF16 as the GPU stores them, and the GPU's input x).  The loss and its gradient
are elementwise FP32 arithmetic on given y: they match the oracle to a few FP32 roundings.
"""
import numpy as np
import pytest

from oracle import fno
from paper_2603_19789_gb300 import sslbm as L

from fno_cases import B, SHAPES, assert_within, case, cfg_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_19789_gb300 import build
    build.build()
    L.load()


def _cfg(shape):
    return cfg_of(shape)


def _setup(seed, shape="generic", early=False):
    import torch
    cfg, n = _cfg(shape)
    theta, p64, u, r0, logd, g = case(seed, shape, early)
    s = L.Surrogate(n=n, width=cfg["W"], modes=cfg["m"], layers=cfg["L"], hidden=cfg["H"], max_batch=B)
    s.set_params(theta)
    tu = torch.from_numpy(u).cuda()
    x = s.make_input(tu, torch.from_numpy(r0).cuda(), torch.from_numpy(logd).cuda())
    xo = fno.make_input(u.astype(np.float64), r0.astype(np.float64), logd.astype(np.float64))
    return s, p64, x, xo, u, g, cfg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_parameter_layout_matches_oracle():
    for shape in SHAPES:
        cfg, n = _cfg(shape)
        s = L.Surrogate(n=n, width=cfg["W"], modes=cfg["m"], layers=cfg["L"], hidden=cfg["H"], max_batch=B)
        assert s.nparams == fno.n_params(**cfg)
        assert s.fused == shape.startswith("fused")
    s2 = L.Surrogate(n=256, width=32, modes=12, layers=4, hidden=64, max_batch=1)
    assert s2.nparams == fno.n_params(32, 12, 4, 64) and s2.fused


@pytest.mark.parametrize("early", [False, True])
def test_make_input_matches_oracle(early):
    s, p32, x, xo, u, _, _ = _setup(0, early=early)
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("seed", [0, 1])
def test_forward_matches_oracle(shape, seed):
    """Every element of y within the BF16 rounding bound of the oracle's y on the GPU's x."""
    s, p64, x, xo, u, _, cfg = _setup(seed, shape, early=seed == 1)
    y = s.forward(x).cpu().numpy().astype(np.float64)
    xg = x.cpu().numpy().astype(np.float64)
    yo, cache = fno.forward(p64, xg, **cfg)
    sd = fno.rounding_sd(p64, xg, cache, **cfg)
    worst = assert_within(y, yo, sd, f"{shape} forward")
    print(f"{shape} seed {seed}: worst element at {worst * 10:.2f} sd of its rounding error")
    # the inference call computes the same values without keeping activations (up to the
    # order of the FP64 atomic sums of the conservation step)
    yi = s.infer(x).cpu().numpy()
    assert rel(yi.astype(np.float64) - u, y - u) < 1e-5
    # the prediction is nonnegative and conserves each sample's population to FP32 rounding
    assert y.min() >= 0.0
    np.testing.assert_allclose(y.reshape(B, -1).sum(axis=1), u.astype(np.float64).reshape(B, -1).sum(axis=1),
                               rtol=2e-6)


@pytest.mark.parametrize("shape", list(SHAPES))
def test_backward_matches_oracle(shape):
    """Every element of every parameter gradient within its BF16 rounding bound."""
    import torch
    s, p64, x, xo, u, g, cfg = _setup(2, shape, early=True)
    n = SHAPES[shape][-1]
    s.forward(x)
    dy = g.standard_normal((B, 5, n, n)).astype(np.float32) * 1e-3
    s.backward(x, torch.from_numpy(dy).cuda())
    torch.cuda.synchronize()
    grads = fno.unflatten(s.get_grads().astype(np.float64), **cfg)
    xg = x.cpu().numpy().astype(np.float64)
    _, cache = fno.forward(p64, xg, **cfg)
    go = fno.backward(p64, cache, dy.astype(np.float64), **cfg)
    sd = fno.gradient_rounding_sd(p64, xg, cache, dy.astype(np.float64), **cfg)
    worst = {name: assert_within(grads[name], go[name], sd[name], f"{shape} gradient {name}") for name in go}
    print(f"{shape}: worst gradient element at {max(worst.values()) * 10:.2f} sd ({max(worst, key=worst.get)})")


def test_backward_after_infer_is_refused():
    import torch
    s, p32, x, xo, u, g, cfg = _setup(4, "fused16")
    s.infer(x)
    with pytest.raises(L.SslbmError):
        s.backward(x, torch.zeros((B, 5, 64, 64), device="cuda"))


@pytest.mark.parametrize("mass_weight,neg_weight", [(0.0, 0.0), (30.0, 30.0)])
def test_training_loss_and_gradient_match_oracle(mass_weight, neg_weight):
    """train_step's loss and dL/dy (left in the dy buffer) against the oracle's loss on the
    same prediction y (left in the y buffer)."""
    import torch
    s, p32, x, xo, u, g, cfg = _setup(5, "fused16", early=True)
    n = 64
    t = u + g.normal(0, 0.02, u.shape).astype(np.float32)
    t[0, 1:3] = u[0, 1:3] * 1.5
    s.set_loss_weights(mass_weight, neg_weight)
    loss = s.train_step(x, torch.from_numpy(t).cuda(), 0.0)
    y = s._y[:B].cpu().numpy().astype(np.float64)
    dy = s._dy[:B].cpu().numpy().astype(np.float64)
    assert y.min() >= 0.0  # the network's output is nonnegative, so the negative-mass term is 0
    # the oracle evaluates the loss with the GPU's scale channel (x holds it exactly)
    mse_w, _, dyo = fno.loss(y, t.astype(np.float64), x.cpu().numpy().astype(np.float64), mass_weight, neg_weight)
    assert loss == pytest.approx(mse_w, rel=1e-5)
    np.testing.assert_allclose(dy, dyo, rtol=1e-4, atol=1e-6 * np.abs(dyo).max())


def test_training_steps_reduce_the_loss():
    import torch
    s, p32, x, xo, u, g, cfg = _setup(3, "fused16")
    # a learnable target: a small change of the input state
    target = (torch.from_numpy(u).cuda() * 0.9 + 0.03).contiguous()
    losses = [s.train_step(x, target, 3e-3) for _ in range(40)]
    assert losses[5] < 0.6 * losses[0] and losses[-1] < 0.3 * losses[0], losses[::5]
    # Adam moved every parameter tensor
    theta = fno.unflatten(s.get_params().astype(np.float64), **cfg)
    for name, v in theta.items():
        assert np.abs(v - fno.unflatten(fno.flatten(p32, **cfg), **cfg)[name]).max() > 0, name


@pytest.mark.parametrize("want_loss", [True, False])
def test_lost_tensor_core_completion_times_out_instead_of_hanging(want_loss):
    """The tensor-core products wait for their MMAs with a bounded poll.  The test hook issues
    no MMA and no completion signal (nothing then arrives on the barrier), so every wait runs
    out: the step returns SSLBM_ERR_TIMEOUT whether or not the loss is read, skips the Adam
    update (the parameters keep their bits), and the context stays usable afterwards."""
    import torch
    s, p32, x, xo, u, g, cfg = _setup(4, "generic")
    theta = s.get_params()
    target = torch.from_numpy(u).cuda().contiguous()
    s.set_wait_limit(polls=2000, stall=True)
    with pytest.raises(L.SslbmError) as e:
        s.train_step(x, target, 1e-3, want_loss=want_loss)
    assert e.value.status == L.SSLBM_ERR_TIMEOUT
    assert np.array_equal(s.get_params().view(np.uint32), theta.view(np.uint32))
    s.set_wait_limit()  # defaults again
    y = s.forward(x)
    assert torch.isfinite(y).all()
    loss = s.train_step(x, target, 1e-3, want_loss=want_loss)  # the status was cleared
    assert loss is None or np.isfinite(loss)
    after = s.get_params()
    assert np.isfinite(after).all() and not np.array_equal(after, theta)


def test_check_project_residuals_and_projection():
    import torch
    cfg, n = _cfg("generic")
    s = L.Surrogate(n=n, width=cfg["W"], modes=cfg["m"], layers=cfg["L"], hidden=cfg["H"], max_batch=B)
    g = np.random.default_rng(5)
    u = g.uniform(0, 1, (B, 5, n, n)).astype(np.float32)
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


@pytest.mark.parametrize("shape", ["generic", "fused16"])
def test_non_finite_input_gives_a_non_finite_prediction(shape):
    """The output clamp max(a, 0) keeps a NaN a NaN (as the oracle's numpy maximum does): a
    sample with a NaN input cell predicts NaN, not zeros that the rescale would make look
    admissible, and the other sample is unaffected."""
    import torch
    s, p64, x, xo, u, g, cfg = _setup(7, shape)
    u2 = u.copy()
    u2[0, 3, 2, 5] = np.nan  # one R cell of sample 0
    xb = s.make_input(torch.from_numpy(u2).cuda(), torch.full((B,), 2.0, device="cuda"),
                      torch.full((B,), -2.0, device="cuda"))
    y = s.infer(xb).cpu().numpy()
    assert np.isnan(y[0]).all()
    assert np.isfinite(y[1]).all()
    yo, _ = fno.forward(p64, xb.cpu().numpy().astype(np.float64), **cfg)
    assert np.isnan(yo[0]).all() and np.isfinite(yo[1]).all()


def test_non_finite_prediction_fails_both_checks():
    """A NaN or Inf anywhere in a prediction (a timed-out tensor-core tile is NaN) gives
    infinite residuals, so a rollout's test `residual <= threshold` sends that scenario to the
    SSLBM fallback, although the clamp and the rescale would have turned it into finite values."""
    import torch
    cfg, n = _cfg("generic")
    s = L.Surrogate(n=n, width=cfg["W"], modes=cfg["m"], layers=cfg["L"], hidden=cfg["H"], max_batch=3)
    g = np.random.default_rng(6)
    u = g.uniform(0, 1, (3, 5, n, n)).astype(np.float32)
    y = u.copy()
    y[0, 2, 5, 7] = np.nan
    y[1, 0, 1, 1] = np.inf
    res = s.check_project(torch.from_numpy(y).cuda(), torch.from_numpy(u).cuda())
    assert np.all(np.isinf(res[:2])), res
    assert np.all(res[2] <= 1e-6), res
    threshold = 1e-4
    bad = ~((res[:, 0] <= threshold) & (res[:, 1] <= 0.0))
    assert bad.tolist() == [True, True, False]


def test_projection_zeroes_outside_the_domain_of_dependence():
    """With reach r, E, I, R, D of the prediction vanish farther than r cells (per axis,
    periodic) from the input's infected or removed cells; inside they are only rescaled."""
    import torch
    cfg, n = _cfg("generic")
    s = L.Surrogate(n=n, width=cfg["W"], modes=cfg["m"], layers=cfg["L"], hidden=cfg["H"], max_batch=B)
    g = np.random.default_rng(9)
    u = np.zeros((B, 5, n, n), np.float32)
    u[:, 0] = 1.0
    u[0, 2, 3:5, 30:32] = 1e-3          # sample 0: infection near the periodic edge
    u[1, 3, 20, 10] = 0.2               # sample 1: removed population only
    y = u + np.abs(g.normal(0, 1e-4, u.shape)).astype(np.float32)
    ty = torch.from_numpy(y).cuda()
    r = 4
    s.check_project(ty, torch.from_numpy(u).cuda(), reach=r)
    out = ty.cpu().numpy().astype(np.float64)
    for b, (ys, xs) in enumerate([(range(3, 5), range(30, 32)), ([20], [10])]):
        inside = np.zeros((n, n), bool)
        for yy in ys:
            for xx in xs:
                for dy in range(-r, r + 1):
                    inside[(yy + dy) % n, [(xx + dx) % n for dx in range(-r, r + 1)]] = True
        assert np.all(out[b, 1:, ~inside] == 0.0)
        assert np.all(out[b, 1:, inside] > 0.0)
        np.testing.assert_allclose(out[b].sum(), u[b].astype(np.float64).sum(), rtol=1e-5)
        # S is untouched by the mask (only rescaled)
        ratio = out[b, 0] / y[b, 0]
        np.testing.assert_allclose(ratio, ratio.mean(), rtol=1e-6)
