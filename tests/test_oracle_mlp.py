"""Pins of the oracle MLP (learned implicit guess): gradients against finite
differences, bf16 rounding and Adam against library routines (no GPU)."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M

torch = pytest.importorskip("torch")


def _batch(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, 14))
    t = rng.normal(size=(B, 9))
    s = (rng.random(B) < 0.3).astype(float)
    m = np.array([1, 1, 1, 1, 1, 1, 0, 0.1, 0.1])
    return x, t, s, m


def test_gradient_matches_finite_differences():
    """Backpropagation (FP64 mode) equals central differences of the loss."""
    O.lib()
    P = M.init_params(1)
    x, t, s, m = _batch(5, 2)
    L, g = M.loss_grad(P, x, t, s, m, mode=1)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(P.size, 60, replace=False), np.arange(P.size - 9, P.size)])
    h = 1e-6
    for k in idx:
        e = np.zeros_like(P); e[k] = h
        fd = (M.loss_grad(P + e, x, t, s, m, 1, False) - M.loss_grad(P - e, x, t, s, m, 1, False)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * (abs(fd) + abs(g).max() * 1e-3), (k, fd, g[k])


def test_bf16_rounding_equals_torch():
    """Round-to-nearest-even bfloat16, bitwise equal to torch's conversion."""
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(size=10000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 10000),
                        np.array([0.0, -0.0, 1.0, 3.0e38, 1e-40], np.float32)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(M.bf16_round(x).view(np.uint32), ref.view(np.uint32))


def test_adam_equals_torch():
    """Adam (Kingma & Ba) step equals torch.optim.Adam on the same gradients."""
    rng = np.random.default_rng(5)
    P = rng.normal(size=300).astype(np.float32)
    mom = np.zeros_like(P); vel = np.zeros_like(P)
    tp = torch.nn.Parameter(torch.from_numpy(P.copy()))
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 4):
        g = rng.normal(size=300).astype(np.float32)
        M.adam(P, mom, vel, g, step)
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        assert np.allclose(P, tp.detach().numpy(), rtol=1e-6, atol=1e-7)


def test_bf16_model_close_to_exact_model():
    """The bf16-operand / FP32-accumulate forward stays within bf16 accuracy
    of the exact network."""
    P = M.init_params(7)
    x, _, _, _ = _batch(64, 8)
    y0 = M.forward(P, x, 0)
    y1 = M.forward(P, x, 1)
    assert np.abs(y0 - y1).max() < 3e-2 * np.abs(y1).max()


def _torch_forward(P, x, bf16):
    """The 14-128-128-128-9 ReLU network written with torch.nn.functional:
    y = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4, weights
    [out][in].  bf16: the tensor-core precision model (every GEMM operand
    rounded to bfloat16 by torch's own conversion, FP32 products and sums,
    FP32 biases); else FP64 throughout."""
    F = torch.nn.functional
    dt = torch.float32 if bf16 else torch.float64
    rnd = (lambda t: t.to(torch.bfloat16).to(dt)) if bf16 else (lambda t: t)
    h = rnd(torch.tensor(x, dtype=dt))
    for l, (W, b) in enumerate(M.unpack(np.asarray(P, np.float64))):
        z = F.linear(h, rnd(torch.tensor(W, dtype=dt)), torch.tensor(b, dtype=dt))
        h = z if l == 3 else rnd(F.relu(z))
    return h.double().numpy()


def test_forward_fp64_equals_torch_network():
    """The oracle forward pass in its exact mode is the network evaluated
    layer by layer by torch (FP64): any dropped bias, transposed weight,
    wrong layer order or misplaced ReLU fails this at rounding level."""
    P = M.init_params(21)
    x, _, _, _ = _batch(257, 22)
    y = M.forward(P, x, 1)
    ref = _torch_forward(P, x, bf16=False)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_forward_bf16_exact_on_integer_network():
    """With small-integer weights, biases and inputs (sparse rows of +-1 and
    +-2) every product and partial sum is an integer below 2^24, so the
    bf16-operand / FP32-accumulate forward has one correct answer whatever
    the summation order; the oracle's mode 0 equals torch's bf16-rounded
    FP32 network bit for bit, activations above 256 rounded to bf16
    included."""
    rng = np.random.default_rng(23)
    parts = []
    for l in range(4):
        ni, no = M.DIMS[l], M.DIMS[l + 1]
        W = np.zeros((no, ni))
        for o in range(no):
            cols = rng.choice(ni, min(ni, 6), replace=False)
            W[o, cols] = rng.choice([-2, -1, 1, 2], len(cols))
        parts += [W.ravel(), rng.integers(-3, 4, no).astype(float)]
    P = np.concatenate(parts)
    x = rng.integers(-8, 9, (300, 14)).astype(float)
    y = M.forward(P, x, 0)
    ref = _torch_forward(P, x, bf16=True)
    assert np.abs(y).max() > 256 and np.array_equal(y, ref)


def test_forward_bf16_equals_torch_network():
    """Random network and inputs in the bf16 model: the oracle's sequential
    FP32 sums against torch's own FP32 linear layers agree elementwise to
    1e-6 of the output scale (an order-of-summation difference could flip
    a bf16 activation rounding; none does here)."""
    P = M.init_params(25)
    x, _, _, _ = _batch(512, 26)
    y = M.forward(P, x, 0)
    ref = _torch_forward(P, x, bf16=True)
    err = np.abs(y - ref) / np.abs(ref).max()
    assert err.max() <= 1e-6, err.max()
