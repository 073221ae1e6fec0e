"""The tcgen05 tensor-core GEMM (hrpp_gemm_bf16: C = A B^T, bf16 in, fp32
accumulated in tensor memory) against a plain PyTorch fp32 reference, with
K-major operands and (hrpp_gemm_bf16_ex) MN-major ones."""
import pytest

from gpu_util import hrpp_mod

pytestmark = pytest.mark.gpu

SHAPES = [(128, 128, 64), (128, 256, 64), (256, 256, 128), (384, 512, 192), (128, 4096, 256), (1024, 256, 4096),
          (256, 128, 1024),
          # two waves of 128 x 256 tiles or more: the persistent kernel (one
          # CTA per SM over the tiles, two TMEM accumulators); 624 tiles leave
          # a partial last round
          (4096, 4096, 512), (4992, 4096, 256)]


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


MN_SHAPES = [(128, 128, 64), (256, 256, 128), (4096, 256, 512), (256, 128, 1024), (384, 512, 192)]


@pytest.mark.parametrize("layout", [1, 2, 3])
@pytest.mark.parametrize("m,n,k", MN_SHAPES)
def test_gemm_mn_major_operands(m, n, k, layout):
    """A stored [k, m] and/or B stored [k, n] (the layout of the learned
    proposal's weight gradients, dW = dZ^T H): the same product as the
    K-major call, against fp32, for every K step and 64-wide slice."""
    import torch
    H = hrpp_mod()
    g = torch.Generator().manual_seed(m * 5 + n * 11 + k + layout)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    ref = a.float() @ b.float().T
    da = (a.T.contiguous() if layout & H.HRPP_GEMM_A_MN_MAJOR else a).cuda()
    db = (b.T.contiguous() if layout & H.HRPP_GEMM_B_MN_MAJOR else b).cuda()
    c = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    rc = H.hrpp_gemm_bf16_ex(da.data_ptr(), db.data_ptr(), c.data_ptr(), m, n, k, layout, None)
    assert rc == H.HRPP_OK, H.hrpp_last_error()
    out = c.cpu()
    bound = 4 * k * 2.0 ** -24 * (a.float().abs() @ b.float().abs().T) + 1e-6
    assert ((out - ref).abs() <= bound).all(), float((out - ref).abs().max())


def test_gemm_rejects_bad_shapes():
    H = hrpp_mod()
    assert H.hrpp_gemm_bf16(None, None, None, 128, 128, 64, None) == H.HRPP_ERR_INVALID_ARG
    import torch
    x = torch.zeros(256, 128, dtype=torch.bfloat16, device="cuda")
    c = torch.zeros(100, 128, device="cuda")
    assert H.hrpp_gemm_bf16(x.data_ptr(), x.data_ptr(), c.data_ptr(), 100, 128, 64, None) == H.HRPP_ERR_INVALID_ARG
    assert H.hrpp_gemm_bf16_ex(x.data_ptr(), x.data_ptr(), c.data_ptr(), 128, 128, 64, 4, None) == \
        H.HRPP_ERR_INVALID_ARG
    # the epilogue writes C 32 bytes at a time: a 16-byte offset is rejected
    c2 = torch.zeros(128 * 128 + 8, device="cuda")
    assert H.hrpp_gemm_bf16(x.data_ptr(), x.data_ptr(), c2.data_ptr() + 16, 128, 128, 64, None) == \
        H.HRPP_ERR_INVALID_ARG
