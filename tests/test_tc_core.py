"""The tcgen05 GEMM core in isolation (no PINN arithmetic): both operand layouts the
jet GEMMs use, against an FP32 matmul of the same BF16 (or TF32-truncated FP32) values.  Jet matrices are
tile-major: a logical [R][C] matrix is stored as [C/256][R][256]."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float((a - b).norm() / b.norm())


def _to_tiles(X):
    R, C = X.shape
    return X.reshape(R, C // 256, 256).permute(1, 0, 2).contiguous()


def _from_tiles(Xt):
    T, R, _ = Xt.shape
    return Xt.permute(1, 0, 2).reshape(R, T * 256)


@pytest.mark.parametrize("M,N,K,split", [(128, 256, 64, False), (256, 512, 320, False), (200, 768, 256, True),
                                         (24, 256, 16, False), (384, 1024, 512, True)])
def test_mn_major_b_operand(cuda_lib, M, N, K, split):
    from paper_2604_15645_gb300 import _lib
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).bfloat16()
    A2 = (torch.randn(M, K, device="cuda", generator=g) * 1e-3).bfloat16() if split else None
    B = torch.randn(K, N, device="cuda", generator=g).bfloat16()
    Bt = _to_tiles(B)
    Dt = torch.full((N // 256, M, 256), float("nan"), device="cuda")
    _lib.pinn_tc_selftest(0, M, N, K, A.data_ptr(), A2.data_ptr() if split else None, Bt.data_ptr(), Dt.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    D = _from_tiles(Dt)
    ref = A.float() @ B.float()
    if split:
        ref = ref + A2.float() @ B.float()
    assert torch.isfinite(D).all()
    assert _rel(D, ref) < 1e-5


@pytest.mark.parametrize("M,N,K", [(128, 256, 256), (256, 512, 4096), (200, 296, 1024), (8, 16, 256)])
def test_k_major_both_operands(cuda_lib, M, N, K):
    from paper_2604_15645_gb300 import _lib
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).bfloat16()
    B = torch.randn(N, K, device="cuda", generator=g).bfloat16()
    At, Bt = _to_tiles(A), _to_tiles(B)
    D = torch.full((M, N), float("nan"), device="cuda")
    _lib.pinn_tc_selftest(1, M, N, K, At.data_ptr(), None, Bt.data_ptr(), D.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    ref = A.float() @ B.float().T
    assert torch.isfinite(D).all()
    assert _rel(D, ref) < 1e-5


def _tf32(X):
    # the tensor cores read FP32 operands truncated to TF32 (10 explicit mantissa bits)
    return (X.view(torch.int32) & -8192).view(torch.float32)


def test_tf32_mn_major_is_refused(cuda_lib):
    from paper_2604_15645_gb300 import _lib
    A = torch.zeros(128, 64, device="cuda")
    B = torch.zeros(1, 64, 256, device="cuda")
    D = torch.zeros(1, 128, 256, device="cuda")
    with pytest.raises(_lib.PinnError):
        _lib.pinn_tc_selftest(2, 128, 256, 64, A.data_ptr(), None, B.data_ptr(), D.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("M,N,K", [(128, 256, 256), (200, 296, 1024)])
def test_tf32_k_major_both_operands(cuda_lib, M, N, K):
    from paper_2604_15645_gb300 import _lib
    g = torch.Generator(device="cuda").manual_seed(M * 3 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g)
    B = torch.randn(N, K, device="cuda", generator=g)
    D = torch.full((M, N), float("nan"), device="cuda")
    _lib.pinn_tc_selftest(3, M, N, K, _to_tiles(A).data_ptr(), None, _to_tiles(B).data_ptr(), D.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    ref = _tf32(A).double() @ _tf32(B).double().T
    assert torch.isfinite(D).all()
    assert _rel(D.double(), ref) < 1e-5


def test_fast_tanh_against_cuda_tanh(cuda_lib):
    """The BF16 epilogues' tanh (exponential form) against CUDA's tanh and a float64
    sech^2, including saturated arguments where 1 - tanh^2 would cancel."""
    from paper_2604_15645_gb300 import _lib
    z = torch.cat([torch.linspace(-12, 12, 200001, device="cuda"),
                   torch.tensor([0.0, -0.0, 1e-30, -1e-30, 1e-8, 20.0, -20.0, 50.0], device="cuda")])
    t = torch.empty_like(z)
    tp = torch.empty_like(z)
    _lib.pinn_tanh_selftest(z.numel(), z.data_ptr(), t.data_ptr(), tp.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref_t = torch.tanh(z)                                   # CUDA's tanh
    assert float((t - ref_t).abs().max()) < 4e-7
    zd = z.double()
    ref_tp = 1.0 / torch.cosh(zd) ** 2
    ok = ref_tp > 1e-30
    relerr = ((tp.double() - ref_tp).abs() / ref_tp)[ok]
    assert float(relerr.max()) < 2e-5
    assert torch.all(t.abs() <= 1) and torch.all(tp >= 0)
