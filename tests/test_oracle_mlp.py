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


def _tc_like_layer(h, W, b, chunk=16, bias_scale=1.0):
    """A float32 evaluation of one hidden layer in the manner of a tensor core:
    each 16-wide slice of the K products summed exactly and rounded to float32,
    the slices accumulated one after another in float32, the bias added in
    float32, GELU in float32, then BF16."""
    Wb = mlp.bf16(W)
    K = h.shape[1]
    acc = np.zeros((h.shape[0], W.shape[0]), np.float32)
    for k0 in range(0, K, chunk):
        part = (h[:, k0:k0 + chunk] @ Wb[:, k0:k0 + chunk].T).astype(np.float32)
        acc = (acc + part).astype(np.float32)
    z = (acc + np.float32(1.0) * (b * bias_scale).astype(np.float32)).astype(np.float32)
    c = np.float32(0.70710678118654752)
    from scipy.special import erf
    e = erf((z * c).astype(np.float32).astype(np.float64)).astype(np.float32)
    g = (np.float32(0.5) * z * (np.float32(1.0) + e)).astype(np.float32)
    return mlp.bf16(g.astype(np.float64))


def test_rounding_interval_holds_a_float32_evaluation():
    """Every activation of a float32 (tensor-core-like) evaluation lies in the
    oracle's admissible BF16 interval, and the interval is a single BF16 value
    for all but about 1 % of activations (near-zero activations, whose BF16
    spacing is below the float32 sum's absolute error, span a few values)."""
    rng = np.random.default_rng(11)
    p = [(W.astype(np.float64), rng.normal(0, 0.05, W.shape[0])) for W, _ in syn.mlp_init(7)]
    X = rng.uniform(-1, 1, size=(3000, 8))
    h = mlp.bf16(X)
    for l in range(4):
        W, b = p[l]
        ex, lo, hi = mlp.hidden_layer_check(h, W, b)
        got = _tc_like_layer(h, W, b)
        assert np.all((got >= lo) & (got <= hi)), l
        assert np.all(lo <= ex) and np.all(ex <= hi)
        wide = lo < hi
        assert wide.mean() < 0.02, wide.mean()
        # away from zero a wide interval spans exactly two BF16 values
        big = wide & (np.abs(ex) > 0.05)
        assert np.all(hi[big] == _bf16_next_up(lo[big]))
        h = got


def _bf16_next_up(x):
    """The next BF16 value above each BF16 value x (finite, x != -0)."""
    u = (np.asarray(x, np.float64).astype(np.float32).view(np.uint32) >> 16).astype(np.int64)
    neg = (u & 0x8000) != 0
    mag = u & 0x7FFF
    zero = mag == 0
    out = np.where(neg, u - 1, u + 1)
    out = np.where(zero, 1, out)                     # +0 or -0 -> the smallest positive subnormal
    out = np.where(neg & (mag == 1), 0, out)         # -min -> +0
    return (out.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def test_rounding_interval_detects_a_dropped_bias():
    """The interval is tight enough to catch an evaluation that drops the bias."""
    rng = np.random.default_rng(12)
    p = [(W.astype(np.float64), rng.normal(0, 0.05, W.shape[0])) for W, _ in syn.mlp_init(7)]
    h = mlp.bf16(rng.uniform(-1, 1, size=(500, 8)))
    W, b = p[0]
    _, lo, hi = mlp.hidden_layer_check(h, W, b)
    bad = _tc_like_layer(h, W, b, bias_scale=0.0)
    assert np.mean((bad < lo) | (bad > hi)) > 0.5
