"""The surrogate network's BF16 GEMM on the tensor cores (tcgen05 with TMA
loads) against a plain FP64 matrix product of the same BF16 operands.
Tolerance: FP32 accumulation, 1e-5 times the sum of the absolute products
(about 2^-17 per partial sum over K up to 2^14)."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_07638_gb300 import mc as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ws(mc):
    nb = ctypes.c_size_t(0)
    assert mc.lib().apm_mlp_workspace_size(0, ctypes.byref(nb)) == 0
    return torch.zeros(nb.value, dtype=torch.uint8, device="cuda")


def bf16(rng, shape, scale=1.0):
    return torch.as_tensor(rng.standard_normal(shape) * scale, dtype=torch.float32).to(torch.bfloat16)


def gemm(mc, ws, A, Bt, bias=None, relu=False, want32=True, wantb=False):
    M, K = A.shape
    N = Bt.shape[0]
    C32 = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda") if want32 else None
    Cb = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda") if wantb else None
    code = mc.lib().apm_mlp_gemm_tn(mc._p(A), mc._p(Bt), mc._p(bias), mc._p(C32), mc._p(Cb), M, N, K, int(relu),
                                    mc._p(ws), ws.numel(), mc._s(A))
    assert code == 0
    flags = ctypes.c_uint32(7)
    assert mc.lib().apm_mlp_status(mc._p(ws), ws.numel(), ctypes.byref(flags), mc._s(A)) == 0
    assert flags.value == 0
    return C32, Cb


def reference(A, Bt, bias=None, relu=False):
    a = A.float().cpu().double()
    b = Bt.float().cpu().double()
    ref = a @ b.T
    scale = a.abs() @ b.abs().T
    if bias is not None:
        ref = ref + bias.cpu().double()
        scale = scale + bias.cpu().double().abs()
    if relu:
        ref = ref.clamp_min(0.0)
    return ref.numpy(), scale.numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 256, 256), (64, 64, 64), (200, 128, 192),
                                   (1000, 256, 64), (16384, 256, 256), (256, 256, 16384), (256, 64, 4096),
                                   (130, 64, 1024)])
def test_fp32_result(mc, ws, M, N, K):
    """Full and ragged row tiles (M not a multiple of 128), both column tiles
    (BN = 128, 64), one to 256 K-blocks, with and without the K split."""
    rng = np.random.default_rng(M * 7 + N * 13 + K)
    A = bf16(rng, (M, K)).cuda()
    Bt = bf16(rng, (N, K)).cuda()
    C32, _ = gemm(mc, ws, A, Bt)
    ref, scale = reference(A, Bt)
    err = np.abs(C32.cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * scale + 1e-30), float(np.max(err / scale))


def test_bias_relu_and_bf16_copy(mc, ws):
    rng = np.random.default_rng(11)
    M, N, K = 384, 256, 256
    A = bf16(rng, (M, K)).cuda()
    Bt = bf16(rng, (N, K), 0.1).cuda()
    bias = torch.as_tensor(rng.standard_normal(N), dtype=torch.float32).cuda()
    C32, Cb = gemm(mc, ws, A, Bt, bias=bias, relu=True, wantb=True)
    ref, scale = reference(A, Bt, bias, relu=True)
    c = C32.cpu().numpy()
    assert np.all(np.abs(c - ref) <= 1e-5 * scale + 1e-30)
    assert np.all(c >= 0.0)
    # the BF16 copy is the FP32 result rounded to nearest
    assert torch.equal(Cb.cpu(), C32.cpu().to(torch.bfloat16))


def test_bf16_only_output(mc, ws):
    rng = np.random.default_rng(12)
    A = bf16(rng, (256, 64)).cuda()
    Bt = bf16(rng, (256, 64)).cuda()
    _, Cb = gemm(mc, ws, A, Bt, want32=False, wantb=True)
    ref, scale = reference(A, Bt)
    assert np.all(np.abs(Cb.float().cpu().numpy() - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * scale)


def test_split_k_is_deterministic(mc, ws):
    rng = np.random.default_rng(13)
    A = bf16(rng, (256, 16384)).cuda()
    Bt = bf16(rng, (256, 16384)).cuda()
    c1, _ = gemm(mc, ws, A, Bt)
    c2, _ = gemm(mc, ws, A, Bt)
    assert torch.equal(c1, c2)
