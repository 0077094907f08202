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
