"""BF16 tensor-core GEMM (tcgen05) and the learned initialiser's kernels
against the double-precision oracle.

BF16 inputs are exact in both computations (products of BF16 values are exact
in FP32); the GPU accumulates in FP32, so each output may differ from the
double-precision sum by FP32 rounding of partial sums: the bar is 2e-5 of
sum_k |a_k b_k| (about 170 FP32 ulps of that scale)."""

import numpy as np
import pytest

from oracle import cnn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 2e-5


@pytest.fixture(scope="module")
def nat():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    return _native


def bf16_dev(x):
    bits = cnn.bf16_bits(x)
    return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()


def run_gemm(nat, a, b, bias=None, relu=False, splits=1, out="f32", lda=None, ldc=None):
    M, K = a.shape
    N = b.shape[0]
    lda = lda or -(-K // 8) * 8
    ldb = -(-K // 8) * 8
    A = np.zeros((M, lda), np.float32)
    A[:, :K] = a
    B = np.zeros((N, ldb), np.float32)
    B[:, :K] = b
    ldc = ldc or N
    dA, dB = bf16_dev(A), bf16_dev(B)
    dbias = torch.from_numpy(np.asarray(bias, np.float32)).cuda() if bias is not None else None
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    pb = nat.load().gs2d_gemm_partial_bytes(M, N, ldc, K, splits)
    part = torch.empty(max(pb // 4, 1), device="cuda")
    if out == "f32":
        C = torch.full((M, ldc), float("nan"), device="cuda")
        nat.gemm_bf16(dA.data_ptr(), lda, dB.data_ptr(), ldb, M, N, K,
                      dbias.data_ptr() if dbias is not None else 0, relu, C.data_ptr(), 0, ldc,
                      splits, part.data_ptr(), status.data_ptr(), 0)
        res = C.cpu().numpy()[:, :N].astype(np.float64)
    else:
        C = torch.zeros((M, ldc), dtype=torch.bfloat16, device="cuda")
        nat.gemm_bf16(dA.data_ptr(), lda, dB.data_ptr(), ldb, M, N, K,
                      dbias.data_ptr() if dbias is not None else 0, relu, 0, C.data_ptr(), ldc,
                      splits, part.data_ptr(), status.data_ptr(), 0)
        res = C.float().cpu().numpy()[:, :N].astype(np.float64)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return res


@pytest.mark.parametrize("M,N,K,splits", [
    (128, 32, 64, 1), (200, 64, 136, 1), (300, 384, 576, 1), (1000, 96, 2304, 4),
    (77, 256, 1152, 3), (4096, 192, 320, 1), (64, 16, 8, 1), (130, 300, 64, 1)])
def test_gemm_f32_matches_oracle(nat, M, N, K, splits):
    g = np.random.Generator(np.random.PCG64(M * 7 + N + K))
    a = cnn.bf16_round(g.normal(size=(M, K)))
    b = cnn.bf16_round(g.normal(size=(N, K)))
    got = run_gemm(nat, a, b, splits=splits)
    ref = cnn.gemm(a, b)
    bound = REL * cnn.gemm_abs(a, b) + 1e-30
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))


@pytest.mark.parametrize("splits", [1, 5])
def test_gemm_bias_relu_bf16_output(nat, splits):
    M, N, K = 256, 128, 320
    g = np.random.Generator(np.random.PCG64(9))
    a = cnn.bf16_round(g.normal(size=(M, K)))
    b = cnn.bf16_round(g.normal(size=(N, K)) * 0.1)
    bias = g.normal(size=N).astype(np.float32)
    got = run_gemm(nat, a, b, bias=bias, relu=True, splits=splits, out="bf16", ldc=136)
    ref = cnn.gemm(a, b, bias, relu=True)
    # the BF16 store rounds once more: half a BF16 ulp of the value
    bound = REL * (cnn.gemm_abs(a, b) + np.abs(bias)[None, :]) + np.abs(ref) * 2.0 ** -8
    assert np.all(np.abs(got - ref) <= bound + 1e-30)
    assert np.all(got >= 0.0)


def test_gemm_padded_leading_dimension(nat):
    M, N, K = 150, 40, 100
    g = np.random.Generator(np.random.PCG64(4))
    a = cnn.bf16_round(g.normal(size=(M, K)))
    b = cnn.bf16_round(g.normal(size=(N, K)))
    got = run_gemm(nat, a, b, lda=104, ldc=48)
    ref = cnn.gemm(a, b)
    assert np.all(np.abs(got - ref) <= REL * cnn.gemm_abs(a, b) + 1e-30)
