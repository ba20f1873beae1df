"""Pins of the MLP oracle: BF16 rounding against PyTorch's conversion, gradients
against central finite differences, GELU derivative, and Adam's closed form for
a constant gradient."""
import numpy as np
import pytest

import synthetic as syn
from oracle import mlp


def small_params(seed=3, width=None):
    p = [(W.astype(np.float64) * 0.5, np.random.default_rng(seed + i).normal(0, 0.1, W.shape[0]))
         for i, (W, b) in enumerate(syn.mlp_init(seed))]
    return p


def test_bf16_matches_torch_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -1.0 - 2.0 ** -8, 0.0, -0.0, 65504.0])])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_gelu_derivative():
    z = np.linspace(-6, 6, 1001)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15  # 1 * Phi(1)


def test_gradients_vs_finite_differences():
    rng = np.random.default_rng(1)
    params = small_params()
    X = rng.uniform(-1, 1, size=(64, 8))
    y = (rng.uniform(size=64) > 0.5).astype(np.float64)
    logit, cache = mlp.forward(params, X, rounding=False)
    grads = mlp.backward(params, cache, logit, y, rounding=False)

    def L(ps):
        return mlp.loss(mlp.forward(ps, X, rounding=False)[0], y)

    # h = 1e-5: truncation ~h^2 and rounding ~1e-16/h both stay below 1e-9
    h = 1e-5
    for l in range(5):
        for which in (0, 1):
            arr = params[l][which]
            for _ in range(4):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                def with_delta(d):
                    ps = [(W.copy(), b.copy()) for W, b in params]
                    ps[l][which][idx] += d
                    return ps
                fd = (L(with_delta(h)) - L(with_delta(-h))) / (2 * h)
                g = grads[l][which][idx]
                assert abs(fd - g) <= 1e-6 * max(abs(g), 1e-3), (l, which, idx, fd, g)


def test_rounded_forward_close_to_exact():
    rng = np.random.default_rng(2)
    params = small_params()
    X = rng.uniform(-1, 1, size=(256, 8))
    a, _ = mlp.forward(params, X, rounding=True)
    b, _ = mlp.forward(params, X, rounding=False)
    assert np.max(np.abs(a - b)) < 0.05 * np.max(np.abs(b)) and not np.array_equal(a, b)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2, so every step moves a weight by lr g/(|g| + eps)."""
    params = [(np.zeros((2, 3)), np.zeros(2))]
    g = np.array([[0.3, -2.0, 1e-3], [5.0, -0.25, 7.0]])
    grads = [(g, np.array([1.0, -1.0]))]
    st = mlp.adam_state(params)
    p = params
    for _ in range(7):
        p = mlp.adam_step(p, grads, st, lr=1e-3, eps=1e-8)
    assert np.allclose(p[0][0], -7 * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(p[0][1], -7 * 1e-3 * np.sign([1.0, -1.0]) * (1 / (1 + 1e-8)), rtol=1e-12, atol=0)
