// Internal interface of the tcgen05 GEMM launchers (gemm.cu).
#pragma once

#include <cuda_runtime.h>

#include "umma.cuh"
#include "umma_softmax.cuh"

namespace hrpp {
bool gemm_shape_ok(int m, int n, int k, int bn);
// operand layout flags of gemm_bf16 (the same values as the public
// HRPP_GEMM_*_MN_MAJOR): A stored [K, M], B stored [K, N]
constexpr int GEMM_A_MN = 1, GEMM_B_MN = 2;
// C = A[M, K] * B[N, K]^T with the given epilogue (umma::Epilogue) and tile
// width bn (128 or 256); splits > 1 divides K across CTAs (EPI_F32_ATOMIC).
// layout 0: both operands K-major; MN-major layouts exist for EPI_F32, for
// EPI_F32_ATOMIC with both operands MN-major and for EPI_RELU_GRAD with B
// MN-major.
cudaError_t gemm_bf16(const void *a, const void *b, int epi, int bn, const umma::GemmArgs &g, int splits,
                      cudaStream_t s, int layout = 0);
// C = A B^T with the persistent kernel (EPI_F32, K-major operands, N a
// multiple of 256): one CTA per SM walks the tiles, the epilogue of one tile
// overlapping the MMAs of the next.
cudaError_t gemm_bf16_persistent(const void *a, const void *b, const umma::GemmArgs &g, cudaStream_t s);
// Fused output layer + softmax cross-entropy (umma_softmax.cuh): h2 [npad,
// 256] and w3 [4096, 256] bf16, K-major; writes dZ (both layouts), adds the
// loss and the labelled-row count.
cudaError_t softmax_xent(const void *h2, const void *w3, const umma::SoftmaxArgs &g, cudaStream_t s);
// The same kernel in prediction mode: per row, the first argmax of the output
// layer and its treelet node (g.out_classes / g.out_nodes, rows < g.n).
cudaError_t softmax_argmax(const void *h2, const void *w3, const umma::SoftmaxArgs &g, cudaStream_t s);
}  // namespace hrpp
