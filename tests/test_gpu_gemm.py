"""The tcgen05 tensor-core GEMM (hrpp_gemm_bf16: C = A B^T, bf16 in, fp32
accumulated in tensor memory) against a plain PyTorch fp32 reference."""
import pytest

from gpu_util import hrpp_mod

pytestmark = pytest.mark.gpu

SHAPES = [(128, 128, 64), (128, 256, 64), (256, 256, 128), (384, 512, 192), (128, 4096, 256), (1024, 256, 4096),
          (256, 128, 1024)]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_gemm_matches_fp32_reference(m, n, k):
    import torch
    H = hrpp_mod()
    g = torch.Generator().manual_seed(m * 7 + n * 3 + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    ref = a.float() @ b.float().T            # products of bf16 values are exact in fp32
    c = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    da, db = a.cuda(), b.cuda()
    rc = H.hrpp_gemm_bf16(da.data_ptr(), db.data_ptr(), c.data_ptr(), m, n, k, None)
    assert rc == H.HRPP_OK, H.hrpp_last_error()
    out = c.cpu()
    assert torch.isfinite(out).all()
    # fp32 sums in another order: error bounded by k * eps * sum |a_i b_i|
    bound = 4 * k * 2.0 ** -24 * (a.float().abs() @ b.float().abs().T) + 1e-6
    assert ((out - ref).abs() <= bound).all(), float((out - ref).abs().max())


def test_gemm_rejects_bad_shapes():
    H = hrpp_mod()
    assert H.hrpp_gemm_bf16(None, None, None, 128, 128, 64, None) == H.HRPP_ERR_INVALID_ARG
    import torch
    x = torch.zeros(256, 128, dtype=torch.bfloat16, device="cuda")
    c = torch.zeros(100, 128, device="cuda")
    assert H.hrpp_gemm_bf16(x.data_ptr(), x.data_ptr(), c.data_ptr(), 100, 128, 64, None) == H.HRPP_ERR_INVALID_ARG
