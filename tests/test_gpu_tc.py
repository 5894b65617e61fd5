"""Tensor-core building block (tcgen05.mma, TMEM, swizzled operand tiles) against an FP32 product."""
import pytest

from helpers import nqs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N,K", [(128, 64), (256, 128), (16, 64), (112, 192), (144, 256), (208, 128)])
def test_tc_gemm_matches_fp32_product(N, K):
    p = nqs()
    g = torch.Generator(device="cuda").manual_seed(N * 1000 + K)
    A = torch.randn((128, K), generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16)
    D, status = p.selftest_tc_gemm(A, B)
    torch.cuda.synchronize()
    assert status.item() == 0
    ref = A.double() @ B.double().T
    scale = (A.double().abs() @ B.double().abs().T)
    assert torch.all((D.double() - ref).abs() <= 1e-6 * scale + 1e-30), (D - ref.float()).abs().max()


@pytest.mark.parametrize("a_t,b_t", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("N,K", [(112, 128), (128, 64), (256, 256), (16, 192)])
def test_tc_gemm_mn_major_operands(N, K, a_t, b_t):
    p = nqs()
    g = torch.Generator(device="cuda").manual_seed(7 * N + K + 3 * a_t + b_t)
    A = torch.randn((128, K), generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16)
    D, status = p.selftest_tc_gemm(A.T.contiguous() if a_t else A, B.T.contiguous() if b_t else B, a_t, b_t)
    torch.cuda.synchronize()
    assert status.item() == 0
    ref = A.double() @ B.double().T
    scale = (A.double().abs() @ B.double().abs().T)
    assert torch.all((D.double() - ref).abs() <= 1e-6 * scale + 1e-30), (D - ref.float()).abs().max()


@pytest.mark.parametrize("n_rows,offs,base", [(128, [0], 0), (144, [0, 5, 16], 0), (256, [-13, -12, -11, -1, 0, 1, 11, 12], 13),
                                              (200, [-7, 9, 3], 40)])
def test_tc_shifted_row_product(n_rows, offs, base):
    # the implicit-GEMM product of the periodic convolutions: windows of A at row offsets
    p = nqs()
    g = torch.Generator(device="cuda").manual_seed(n_rows + base)
    A = torch.randn((n_rows, 16), generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn((len(offs), 16, 16), generator=g, device="cuda").to(torch.bfloat16)
    D, status = p.selftest_tc_shift(A, B, offs, base)
    torch.cuda.synchronize()
    assert status.item() == 0
    ref = sum(A[base + o: base + o + 128].double() @ B[t].double().T for t, o in enumerate(offs))
    scale = sum(A[base + o: base + o + 128].double().abs() @ B[t].double().abs().T for t, o in enumerate(offs))
    assert torch.all((D.double() - ref).abs() <= 1e-6 * scale + 1e-30), (D - ref.float()).abs().max()
