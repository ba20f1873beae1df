"""MLP surrogate oracle: forward, backward and Adam in FP64, with BF16 rounding
(round-to-nearest-even) applied at exactly the points where the GPU kernels
round, so gradients can be compared tightly.

Oracle / test infrastructure only.

Network (the dynamic-aperture triage surrogate; the paper has no learned part):
  input 8 (x/25 mm, y/25 mm, 6 normalised lattice parameters)
  4 hidden layers Linear(-> 256) + GELU (erf form), then Linear(256 -> 1) logit.
Weights are BF16 copies of FP32 master weights; activations entering every
matrix product are BF16; products accumulate in FP32 on the GPU (FP64 here);
biases are FP32.  Loss: binary cross-entropy on the logit (label 1 = survives).

Rounding points (mirrored by the kernels):
  h_0 = bf16(x);  z_l = h_{l-1} bf16(W_l)^T + b_l;  h_l = bf16(gelu(z_l))
  logit = h_4 . bf16(w_5) + b_5
  dlogit = (sigmoid(logit) - y) / M
  dh_4 = dlogit bf16(w_5)^T;  dz_l = dh_l * gelu'(z_l);  dzb_l = bf16(dz_l)
  dW_l = dzb_l^T h_{l-1};  db_l = sum_m dz_l;  dh_{l-1} = dzb_l bf16(W_l)
  dw_5 = h_4^T dlogit;  db_5 = sum_m dlogit
"""
import math

import numpy as np
from scipy.special import erf

N_IN, WIDTH, N_HIDDEN = 8, 256, 4
SQRT1_2 = 1.0 / math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def bf16(x):
    """Round to BF16 (nearest, ties to even) via FP32; returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT1_2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z * SQRT1_2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def shapes():
    """[(out, in)] of the five linear layers."""
    dims = [N_IN] + [WIDTH] * N_HIDDEN
    return [(dims[i + 1], dims[i]) for i in range(N_HIDDEN)] + [(1, WIDTH)]


def _r(x, rounding):
    return bf16(x) if rounding else np.asarray(x, dtype=np.float64)


def forward(params, X, rounding=True):
    """params: list of (W, b) float arrays; returns (logits, cache)."""
    h = _r(X, rounding)
    cache = []
    for l in range(N_HIDDEN):
        W, b = params[l]
        z = h @ _r(W, rounding).T + b
        cache.append((h, z))
        h = _r(gelu(z), rounding)
    w5, b5 = params[N_HIDDEN]
    logit = h @ _r(w5, rounding).reshape(-1) + b5[0]
    cache.append((h, None))
    return logit, cache


# Error model of a float32 evaluation of one hidden layer (the GPU's): the K
# products of BF16 values are exact in float32, and the float32 sum of them,
# in whatever order the tensor core takes, is taken to lie within ACC_ULPS
# units of float32 rounding of sum |h W| (2^-24 sum |h W| each) of the exact
# sum; adding the bias rounds once more (2^-24 |z|).  GELU in float32 (z * c,
# erf to 2 ulp, 1 + erf, the final product) is within E_g of gelu at the
# float32 z, and |gelu'| <= 1.129, so the float32 activation lies within delta
# of gelu(z_exact) and rounds to a BF16 value in [bf16(g - delta), bf16(g + delta)].
# ACC_ULPS = 4 is a realistic scale, not the worst case (K units): measured on
# the GB300 tensor cores, the exact activation of every flipped BF16 rounding
# lay within 1.1e-7 sum |h W| (below 2 units) of the rounding midpoint.
GELU_GRAD_MAX = 1.1289
ACC_ULPS = 4


def layer_delta(h_prev, W, z, acc_ulps=ACC_ULPS):
    """Per-activation bound delta on |gelu_f32(z_f32) - gelu(z)| (see above)."""
    s_abs = np.abs(h_prev) @ np.abs(W).T
    ez = acc_ulps * 2.0 ** -24 * s_abs + 2.0 ** -24 * np.abs(z)
    g = gelu(z)
    eg = 0.5 * np.abs(z) * (2.0 ** -24 * np.abs(z) + 2.0 ** -21 + 2.0 ** -23) + 2.0 ** -23 * np.abs(g)
    return GELU_GRAD_MAX * ez + eg


def hidden_layer_check(h_prev, W, b, acc_ulps=ACC_ULPS):
    """One hidden layer on given BF16 inputs h_prev (exact values): returns
    (h, lo, hi) with h = bf16(gelu(z)) from the exact FP64 pre-activation
    z = h_prev bf16(W)^T + b, and [lo, hi] the BF16 values a float32 evaluation
    can round to: bf16(gelu(z) - delta) .. bf16(gelu(z) + delta).  Where lo < hi
    the exact activation sits within delta of a BF16 rounding midpoint, and
    either neighbour is a correct float32 result."""
    Wb = bf16(W)
    z = h_prev @ Wb.T + b
    g = gelu(z)
    d = layer_delta(h_prev, Wb, z, acc_ulps)
    return bf16(g), bf16(g - d), bf16(g + d)


def head_delta(h4, w5, logit):
    """Bound on |float32 logit - exact logit| for given h4: the 256-term float32
    dot product and the bias addition."""
    return 257 * 2.0 ** -23 * (np.abs(h4) @ np.abs(bf16(w5)).reshape(-1)) + 2.0 ** -23 * np.abs(logit)


def loss(logit, y):
    """Mean binary cross-entropy with logits."""
    return float(np.mean(np.logaddexp(0.0, logit) - y * logit))


def backward(params, cache, logit, y, rounding=True):
    M = logit.shape[0]
    dlogit = (1.0 / (1.0 + np.exp(-logit)) - y) / M
    grads = [None] * (N_HIDDEN + 1)
    h4 = cache[N_HIDDEN][0]
    w5 = params[N_HIDDEN][0]
    grads[N_HIDDEN] = ((dlogit @ h4).reshape(1, -1), np.array([dlogit.sum()]))
    dh = np.outer(dlogit, _r(w5, rounding).reshape(-1))
    for l in range(N_HIDDEN - 1, -1, -1):
        h_prev, z = cache[l]
        dz = dh * gelu_grad(z)
        dzb = _r(dz, rounding)
        grads[l] = (dzb.T @ h_prev, dz.sum(axis=0))
        if l > 0:
            dh = dzb @ _r(params[l][0], rounding)
    return grads


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on FP32 master weights held as float64."""
    state["t"] += 1
    t = state["t"]
    out = []
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for k, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][i][k] = beta1 * state["m"][i][k] + (1.0 - beta1) * g
            v = state["v"][i][k] = beta2 * state["v"][i][k] + (1.0 - beta2) * g * g
            mh = m / (1.0 - beta1 ** t)
            vh = v / (1.0 - beta2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out


def adam_state(params):
    return {"t": 0, "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]}
