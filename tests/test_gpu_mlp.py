"""GPU tests of the tensor-core (tcgen05) kernels of the learned guess:
the generic BF16 GEMM against torch, the fused MLP forward against the
oracle network."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from helpers import cuda_or_skip, fpic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    cuda_or_skip()
    return fpic()


@pytest.mark.parametrize("M_,N,K", [(128, 128, 16), (256, 128, 128), (200, 16, 64), (384, 48, 32),
                                    (128, 256, 512), (1000, 128, 144)])
def test_tensor_core_gemm_matches_torch(F, M_, N, K):
    """C = A B^T with bf16 operands and FP32 accumulation, exact products:
    agrees with an FP64 product of the same bf16 values to FP32 accumulation
    accuracy."""
    g = torch.Generator(device="cpu").manual_seed(M_ * 7 + N + K)
    A = torch.randn(M_, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C, err = F.fpic_mma_bf16(A, B)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = (A.double() @ B.double().T)
    tol = 1e-5 * K ** 0.5 * ref.abs().max().item()
    diff = (C.double() - ref).abs().max().item()
    if diff > tol:
        alt = (A.double() @ B.double().T).T  # diagnostics only
        pytest.fail(f"gemm mismatch {diff:.3e} > {tol:.3e}; C[0,:4]={C[0,:4].tolist()} ref={ref[0,:4].tolist()}")
    # accumulate into an existing C
    C2, err = F.fpic_mma_bf16(A, B, C=C.clone(), accumulate=True)
    torch.cuda.synchronize()
    assert (C2.double() - 2 * ref).abs().max().item() <= 2 * tol


def test_fused_forward_matches_oracle(F):
    """Fused tcgen05 forward of 5000 samples (39 tiles + a ragged tail) of a
    random network equals the oracle's bf16-operand / FP32-accumulate
    network to FP32 rounding, except for samples where a different
    summation order flips one bf16 activation rounding."""
    P = M.init_params(3)
    rng = np.random.default_rng(4)
    B = 5000
    X = rng.normal(size=(B, 14))
    y_or = M.forward(P, X, mode=0)
    net = F.MLP()
    net.set_params(torch.tensor(P, dtype=torch.float32, device="cuda"))
    Xg = torch.zeros(B, 16, dtype=torch.float32, device="cuda")
    Xg[:, :14] = torch.tensor(X, dtype=torch.float32)
    Y = net.forward(Xg)
    torch.cuda.synchronize()
    assert net.status() == 0
    y = Y[:, :9].double().cpu().numpy()
    err = np.abs(y - y_or) / np.abs(y_or).max()
    q = np.quantile(err, [0.5, 0.99])
    print("fused forward vs oracle, relative to scale: median %.2e, 99%% %.2e, max %.2e" % (q[0], q[1], err.max()))
    # FP32 sums in another order: most outputs agree to FP32 rounding; a
    # sample whose bf16 activation rounding flipped moves by ~1e-4 of scale
    assert q[0] <= 1e-7 and q[1] <= 1e-6 and err.max() <= 2e-3, (q, err.max())


def test_fused_forward_bit_exact_on_integer_network(F):
    """Small-integer weights, biases and inputs (sparse rows of +-1, +-2):
    every product and partial sum is an integer below 2^24, so the
    tensor-core forward has exactly one correct answer whatever its
    summation order, and it equals the oracle's bit for bit (bf16 rounding
    of activations above 256 included): 3000 samples, 23 tiles and a
    ragged tail."""
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
    B = 3000
    X = rng.integers(-8, 9, (B, 14)).astype(float)
    y_or = M.forward(P, X, mode=0)
    net = F.MLP()
    net.set_params(torch.tensor(P, dtype=torch.float32, device="cuda"))
    Xg = torch.zeros(B, 16, dtype=torch.float32, device="cuda")
    Xg[:, :14] = torch.tensor(X, dtype=torch.float32)
    Y = net.forward(Xg)
    torch.cuda.synchronize()
    assert net.status() == 0
    y = Y[:, :9].double().cpu().numpy()
    assert np.abs(y_or).max() > 256
    assert np.array_equal(y, y_or), np.abs(y - y_or).max()


def _batch(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, 14))
    t = np.zeros((B, 9)); t[:] = rng.normal(size=(B, 9)) * 0.5
    s = (rng.random(B) < 0.3).astype(float)
    lw = np.array([1, 1, 1, 1, 1, 1, 0, 0.1, 0.1])
    return x, t, s, lw


def _dev_batch(x, t, s):
    B = x.shape[0]
    X = torch.zeros(B, 16, dtype=torch.float32, device="cuda"); X[:, :14] = torch.tensor(x, dtype=torch.float32)
    T = torch.zeros(B, 16, dtype=torch.float32, device="cuda"); T[:, :9] = torch.tensor(t, dtype=torch.float32)
    S = torch.tensor(s, dtype=torch.float32, device="cuda")
    return X, T, S


def test_gradient_matches_oracle(F):
    """Backward on the tensor cores (split-K weight gradients, ReLU masks,
    bias column sums) against the oracle's bf16-operand / FP32-accumulate
    backpropagation, batch 1024."""
    P = M.init_params(11)
    x, t, s, lw = _batch(1024, 12)
    L_or, g_or = M.loss_grad(P, x, t, s, lw, mode=0)
    net = F.MLP()
    net.set_params(torch.tensor(P, dtype=torch.float32, device="cuda"))
    X, T, S = _dev_batch(x, t, s)
    L, g = net.grad(X, T, S, lw)
    torch.cuda.synchronize()
    assert net.status() == 0
    g = g.double().cpu().numpy()
    assert abs(L - L_or) <= 1e-3 * abs(L_or)
    rel = np.linalg.norm(g - g_or) / np.linalg.norm(g_or)
    assert rel <= 1e-2, rel
    assert np.abs(g - g_or).max() <= 5e-2 * np.abs(g_or).max()


def test_train_step_adam_and_learning(F):
    """fpic_mlp_train_step = the tensor-core gradient followed by the oracle's
    Adam step (same gradient), and repeated steps lower the loss."""
    P = M.init_params(5).astype(np.float32)
    x, t, s, lw = _batch(2048, 6)
    net = F.MLP()
    Pd = torch.tensor(P, device="cuda")
    net.set_params(Pd)
    X, T, S = _dev_batch(x, t, s)
    L0, g = net.grad(X, T, S, lw)
    mom = torch.zeros_like(Pd); vel = torch.zeros_like(Pd)
    net.train_step(Pd, mom, vel, X, T, S, lw, step=1, lr=1e-3)
    Pc = P.copy(); mc = np.zeros_like(P); vc = np.zeros_like(P)
    M.adam(Pc, mc, vc, g.cpu().numpy().astype(np.float32), 1, 1e-3)
    assert np.allclose(Pd.cpu().numpy(), Pc, rtol=1e-5, atol=1e-6)
    for step in range(2, 60):
        L = net.train_step(Pd, mom, vel, X, T, S, lw, step=step, lr=3e-3, want_loss=True)
    assert L < 0.7 * L0, (L0, L)
    assert net.status() == 0
