"""GPU MLP surrogate kernels (BF16 tensor-core products, FP32 accumulation)
against the oracle at identical BF16 weights."""
import numpy as np
import pytest

import synthetic as syn
from oracle import mlp as om
from paper_1710_07350_gb300 import trk

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def params64(seed=7):
    rng = np.random.default_rng(seed)
    return [(W.astype(np.float64), rng.normal(0, 0.05, W.shape[0]).astype(np.float32).astype(np.float64))
            for W, _ in syn.mlp_init(seed)]


def data(n, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, 8)).astype(np.float32)
    y = ((X[:, 0] ** 2 + X[:, 1] ** 2) < 0.5).astype(np.float32)
    return X, y


def bf16_bits_to_f64(t):
    """int16 CUDA tensor of BF16 bit patterns -> float64 numpy values."""
    return (t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M", [1, 63, 1000, 70000])
def test_forward_matches_oracle(M):
    """Layer by layer from the GPU's own BF16 activations: each hidden layer's
    output equals the oracle's bf16(gelu(z)) on the same inputs, or -- where
    the exact activation lies within the float32 evaluation error of a BF16
    rounding midpoint -- the other neighbour (an admissible flip); the logit
    follows from the GPU's last hidden layer to float32 rounding.  End to end,
    every row the GPU rounded as the oracle matches the oracle's logit to 1e-5
    relative, so every larger difference comes from such flips."""
    p = params64()
    net = trk.trk_mlp_create(p)
    X, _ = data(M)
    got_t, hid = trk.trk_mlp_forward_hidden(net, torch.from_numpy(X).cuda())
    got = got_t.cpu().numpy().astype(np.float64)
    H = bf16_bits_to_f64(hid)
    plain = trk.trk_mlp_forward(net, torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    assert np.array_equal(plain, got)
    h = om.bf16(X.astype(np.float64))
    flipped_row = np.zeros(M, bool)
    for l in range(4):
        W, b = p[l]
        exact, lo, hi = om.hidden_layer_check(h, W, b)
        g = H[l]
        assert np.all((g >= lo) & (g <= hi)), "layer %d: activation outside the admissible BF16 roundings" % l
        flip = g != exact
        assert flip.mean() <= 1e-3, (l, flip.mean())
        flipped_row |= flip.any(axis=1)
        h = g
    w5, b5 = p[4]
    head = h @ om.bf16(w5).reshape(-1) + b5[0]
    assert np.all(np.abs(got - head) <= om.head_delta(h, w5, head))
    want, _ = om.forward(p, X.astype(np.float64))
    scale = np.maximum(np.abs(want), 0.1 * np.max(np.abs(want)))
    rel = np.abs(got - want) / scale
    assert np.all(rel[~flipped_row] <= 1e-5)
    assert np.median(rel) <= 1e-5


@pytest.mark.parametrize("M", [1000, 4096])
def test_gradients_match_oracle(M):
    p = params64(8)
    net = trk.trk_mlp_create(p)
    X, y = data(M, seed=2)
    loss = trk.trk_mlp_grad(net, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()).item()
    _, grads = trk.trk_mlp_get(net)
    logit, cache = om.forward(p, X.astype(np.float64))
    want = om.backward(p, cache, logit, y.astype(np.float64))
    assert abs(loss - om.loss(logit, y)) <= 1e-4 * abs(om.loss(logit, y))
    for l in range(5):
        for k in range(2):
            g = grads[l][k].astype(np.float64).reshape(want[l][k].shape)
            w = want[l][k]
            assert np.linalg.norm(g - w) <= 1e-2 * np.linalg.norm(w), (l, k)


def test_adam_step_matches_oracle():
    p = params64(9)
    net = trk.trk_mlp_create(p)
    X, y = data(512, seed=3)
    trk.trk_mlp_grad(net, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    _, g_gpu = trk.trk_mlp_get(net)
    trk.trk_mlp_adam(net, lr=1e-3)
    after, _ = trk.trk_mlp_get(net)
    p32 = [(W.astype(np.float32).astype(np.float64), b) for W, b in p]
    st = om.adam_state(p32)
    want = om.adam_step(p32, [(gW.astype(np.float64), gb.astype(np.float64)) for gW, gb in g_gpu], st, lr=1e-3)
    for l in range(5):
        assert np.allclose(after[l][0], want[l][0], rtol=0, atol=1e-6)
        assert np.allclose(after[l][1], want[l][1], rtol=0, atol=1e-6)


def test_training_learns_a_disc():
    X, y = data(32768, seed=4)
    net = trk.trk_mlp_create(syn.mlp_init(7))
    Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    g = np.random.default_rng(5)
    perm = torch.from_numpy(np.stack([g.permutation(len(X)) for _ in range(8)]).astype(np.int32)).cuda()
    hist = trk.trk_mlp_train(net, Xt, yt, batch=2048, epochs=8, perm=perm, lr=2e-3).cpu().numpy()
    assert hist[-1] < 0.25 * hist[0]
    Xv, yv = data(20000, seed=6)
    pred = (trk.trk_mlp_forward(net, torch.from_numpy(Xv).cuda()).cpu().numpy() > 0).astype(np.float32)
    assert np.mean(pred == yv) > 0.97


def test_gradients_and_training_are_deterministic():
    """The backward pass runs as a fork-join over several streams with
    programmatic dependent launch; every sum has one writer and a fixed order,
    so two runs on the same inputs give the same bits (gradients, loss history,
    weights), and a short last batch does too."""
    p = params64(11)
    X, y = data(5000, seed=12)
    Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    runs = []
    for _ in range(2):
        net = trk.trk_mlp_create(p)
        loss = trk.trk_mlp_grad(net, Xt, yt).item()
        _, g = trk.trk_mlp_get(net)
        runs.append((loss, g))
    assert runs[0][0] == runs[1][0]
    for l in range(5):
        for k in range(2):
            assert np.array_equal(runs[0][1][l][k], runs[1][1][l][k]), (l, k)
    gen = np.random.default_rng(13)
    perm = torch.from_numpy(np.stack([gen.permutation(len(X)) for _ in range(3)]).astype(np.int32)).cuda()
    out = []
    for _ in range(2):
        net = trk.trk_mlp_create(syn.mlp_init(7))
        hist = trk.trk_mlp_train(net, Xt, yt, batch=1024, epochs=3, perm=perm, lr=2e-3).cpu().numpy()
        w, _ = trk.trk_mlp_get(net)
        out.append((hist, w))
    assert np.array_equal(out[0][0], out[1][0])
    for l in range(5):
        assert np.array_equal(out[0][1][l][0], out[1][1][l][0]) and np.array_equal(out[0][1][l][1], out[1][1][l][1])
