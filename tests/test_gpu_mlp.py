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
    """Fused tcgen05 forward of 5000 samples (39 tiles + a ragged tail) equals
    the oracle's bf16-operand / FP32-accumulate network within bf16
    accuracy."""
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
    scale = np.abs(y_or).max()
    err = np.abs(y - y_or)
    assert err.max() <= 2e-2 * scale, err.max() / scale
    assert err.mean() <= 2e-3 * scale
