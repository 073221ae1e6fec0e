// Host launchers of the tcgen05 GEMM (umma.cuh): TMA tensor maps, tile and
// split choices, and the utility entry point hrpp_gemm_bf16.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "gemm.h"
#include "handles.h"
#include "hrpp.h"
#include "umma.cuh"

namespace hrpp {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mutex;

cudaError_t encoder(PFN_cuTensorMapEncodeTiled_v12000 *out)
{
    std::lock_guard<std::mutex> lk(g_encode_mutex);
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    *out = g_encode;
    return cudaSuccess;
}

// Raises a kernel's dynamic shared-memory limit once per device (the
// attribute belongs to the current device).  A failure is not remembered, so
// a later call retries.
class SmemAttr {
  public:
    cudaError_t set(const void *fn, size_t smem)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        std::lock_guard<std::mutex> lk(mu_);
        if ((done_ >> dev) & 1u) return cudaSuccess;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) done_ |= 1ull << dev;
        return e;
    }

  private:
    std::mutex mu_;
    uint64_t done_ = 0;
};

// K-major bf16 matrix [rows, k] as a TMA map with 64 x box_rows boxes and
// 128-byte swizzle (the layout the tcgen05 shared-memory descriptor expects).
cudaError_t make_map(CUtensorMap *map, const void *ptr, uint64_t rows, uint64_t k, uint32_t box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 encode;
    cudaError_t e = encoder(&encode);
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {k, rows};
    cuuint64_t strides[1] = {k * 2};
    cuuint32_t box[2] = {(cuuint32_t)umma::BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// MN-major bf16 matrix stored [k, mn] (mn contiguous) as a TMA map with
// 64 x 64 boxes (64 mn elements = one 128-byte swizzle row, 64 K rows).
cudaError_t make_map_mn(CUtensorMap *map, const void *ptr, uint64_t k, uint64_t mn)
{
    PFN_cuTensorMapEncodeTiled_v12000 encode;
    cudaError_t e = encoder(&encode);
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {mn, k};
    cuuint64_t strides[1] = {mn * 2};
    cuuint32_t box[2] = {64u, (cuuint32_t)umma::BK};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int EPI, int NST, bool AMN, bool BMN>
cudaError_t launch_stages(const void *a, const void *b, const umma::GemmArgs &g, int splits, cudaStream_t s)
{
    const size_t smem = umma::gemm_smem_bytes<BN, NST>();
    static SmemAttr attr;  // one per template instance
    cudaError_t e = attr.set((const void *)umma::k_gemm<BN, EPI, NST, AMN, BMN>, smem);
    if (e != cudaSuccess) return e;
    CUtensorMap ma, mb;
    e = AMN ? make_map_mn(&ma, a, (uint64_t)g.K, (uint64_t)g.M)
                        : make_map(&ma, a, (uint64_t)g.M, (uint64_t)g.K, umma::BM);
    if (e == cudaSuccess)
        e = BMN ? make_map_mn(&mb, b, (uint64_t)g.K, (uint64_t)g.N) : make_map(&mb, b, (uint64_t)g.N, (uint64_t)g.K, BN);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(g.N / BN), (unsigned)(g.M / umma::BM), (unsigned)splits);
    umma::k_gemm<BN, EPI, NST, AMN, BMN><<<grid, 128, smem, s>>>(ma, mb, g);
    return cudaGetLastError();
}

// short K ranges (at most 4 K blocks per CTA) take the 2-stage variant
template <int BN, int EPI, bool AMN = false, bool BMN = false>
cudaError_t launch(const void *a, const void *b, const umma::GemmArgs &g, int splits, cudaStream_t s)
{
    if (g.k_blocks_per_split <= 4) return launch_stages<BN, EPI, 2, AMN, BMN>(a, b, g, splits, s);
    return launch_stages<BN, EPI, umma::STAGES, AMN, BMN>(a, b, g, splits, s);
}

// The persistent kernel: one CTA per SM over 128 x 256 tiles (EPI_F32,
// K-major operands).
cudaError_t launch_persistent(const void *a, const void *b, const umma::GemmArgs &g, cudaStream_t s)
{
    const size_t smem = umma::gemm_persistent_smem_bytes<>();
    static SmemAttr attr;
    cudaError_t e = attr.set((const void *)umma::k_gemm_persistent<>, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    CUtensorMap ma, mb;
    e = make_map(&ma, a, (uint64_t)g.M, (uint64_t)g.K, umma::BM);
    if (e == cudaSuccess) e = make_map(&mb, b, (uint64_t)g.N, (uint64_t)g.K, umma::PG_BN);
    if (e != cudaSuccess) return e;
    const int tiles = (g.M / umma::BM) * (g.N / umma::PG_BN);
    const int grid = tiles < sms ? tiles : sms;
    umma::k_gemm_persistent<><<<grid, umma::PG_THREADS, smem, s>>>(ma, mb, g);
    return cudaGetLastError();
}

}  // namespace

namespace {

template <bool PREDICT>
cudaError_t launch_output_layer(const void *h2, const void *w3, const umma::SoftmaxArgs &g, cudaStream_t s)
{
    const size_t smem = umma::softmax_smem_bytes<>();
    static SmemAttr attr;  // one per instance
    cudaError_t e = attr.set((const void *)umma::k_softmax_xent<umma::SX_NST, PREDICT>, smem);
    if (e != cudaSuccess) return e;
    if (g.npad <= 0 || g.npad % umma::BM != 0 || ((uintptr_t)h2 & 15u) || ((uintptr_t)w3 & 15u)) return cudaErrorInvalidValue;
    // the epilogue reads the bias 16 bytes and writes dZ rows 32 bytes at a time
    if (!g.bias || ((uintptr_t)g.bias & 15u) || (!PREDICT && (!g.dz || ((uintptr_t)g.dz & 31u))))
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    e = make_map(&ma, h2, (uint64_t)g.npad, umma::SX_K, umma::BM);
    if (e == cudaSuccess) e = make_map(&mb, w3, umma::SX_CLASSES, umma::SX_K, umma::SX_BN);
    if (e != cudaSuccess) return e;
    umma::k_softmax_xent<umma::SX_NST, PREDICT><<<g.npad / umma::BM, umma::SX_THREADS, smem, s>>>(ma, mb, g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t softmax_xent(const void *h2, const void *w3, const umma::SoftmaxArgs &g, cudaStream_t s)
{
    return launch_output_layer<false>(h2, w3, g, s);
}

cudaError_t softmax_argmax(const void *h2, const void *w3, const umma::SoftmaxArgs &g, cudaStream_t s)
{
    return launch_output_layer<true>(h2, w3, g, s);
}

cudaError_t gemm_bf16_persistent(const void *a, const void *b, const umma::GemmArgs &g, cudaStream_t s)
{
    if (((uintptr_t)a & 15u) || ((uintptr_t)b & 15u) || ((uintptr_t)g.c32 & 31u) || g.N % umma::PG_BN != 0 ||
        g.M % umma::BM != 0 || g.K % umma::BK != 0)
        return cudaErrorInvalidValue;
    return launch_persistent(a, b, g, s);
}

bool gemm_shape_ok(int m, int n, int k, int bn)
{
    return m > 0 && n > 0 && k > 0 && m % umma::BM == 0 && n % bn == 0 && k % umma::BK == 0;
}

cudaError_t gemm_bf16(const void *a, const void *b, int epi, int bn, const umma::GemmArgs &g0, int splits,
                      cudaStream_t s, int layout)
{
    umma::GemmArgs g = g0;
    const int kb = g.K / umma::BK;
    if (splits < 1) splits = 1;
    if (splits > kb) splits = kb;
    g.k_blocks_per_split = (kb + splits - 1) / splits;
    splits = (kb + g.k_blocks_per_split - 1) / g.k_blocks_per_split;
    if (((uintptr_t)a & 15u) || ((uintptr_t)b & 15u)) return cudaErrorInvalidValue;
    // epilogue stores: 32 bytes per lane (plain fp32 and bf16 outputs), 16
    // bytes per atomic
    if ((epi == umma::EPI_F32 && ((uintptr_t)g.c32 & 31u)) || (epi == umma::EPI_F32_ATOMIC && ((uintptr_t)g.c32 & 15u)) ||
        ((epi == umma::EPI_BIAS_RELU || epi == umma::EPI_RELU_GRAD) && ((uintptr_t)g.c16 & 31u)))
        return cudaErrorInvalidValue;
    if (layout != 0) {
        // MN-major operands: the weight gradients of the training step
        // (split-K atomics, both MN-major), its dZ GEMMs (the weights as B,
        // MN-major) and the utility entry point (plain fp32)
#define HRPP_GEMM_MN(BN_, EPI_, L_)                                                                   \
    if (bn == BN_ && epi == EPI_ && layout == L_)                                                     \
        return launch<BN_, EPI_, (L_ & GEMM_A_MN) != 0, (L_ & GEMM_B_MN) != 0>(a, b, g, splits, s);
        HRPP_GEMM_MN(128, umma::EPI_F32, 1)
        HRPP_GEMM_MN(128, umma::EPI_F32, 2)
        HRPP_GEMM_MN(128, umma::EPI_F32, 3)
        HRPP_GEMM_MN(256, umma::EPI_F32, 1)
        HRPP_GEMM_MN(256, umma::EPI_F32, 2)
        HRPP_GEMM_MN(256, umma::EPI_F32, 3)
        HRPP_GEMM_MN(128, umma::EPI_F32_ATOMIC, 3)
        HRPP_GEMM_MN(256, umma::EPI_F32_ATOMIC, 3)
        HRPP_GEMM_MN(128, umma::EPI_RELU_GRAD, 2)
        HRPP_GEMM_MN(256, umma::EPI_RELU_GRAD, 2)
#undef HRPP_GEMM_MN
        return cudaErrorInvalidValue;
    }
#define HRPP_GEMM_CASE(BN_, EPI_) \
    if (bn == BN_ && epi == EPI_) return launch<BN_, EPI_>(a, b, g, splits, s);
    HRPP_GEMM_CASE(128, umma::EPI_F32)
    HRPP_GEMM_CASE(256, umma::EPI_F32)
    HRPP_GEMM_CASE(128, umma::EPI_F32_ATOMIC)
    HRPP_GEMM_CASE(256, umma::EPI_F32_ATOMIC)
    HRPP_GEMM_CASE(256, umma::EPI_BIAS_RELU)
    HRPP_GEMM_CASE(128, umma::EPI_BIAS_RELU)
    HRPP_GEMM_CASE(256, umma::EPI_RELU_GRAD)
    HRPP_GEMM_CASE(128, umma::EPI_RELU_GRAD)
#undef HRPP_GEMM_CASE
    return cudaErrorInvalidValue;
}

}  // namespace hrpp

extern "C" hrpp_status hrpp_gemm_bf16(const void *a, const void *b, float *c, int m, int n, int k, void *stream)
{
    return hrpp_gemm_bf16_ex(a, b, c, m, n, k, 0, stream);
}

extern "C" hrpp_status hrpp_gemm_bf16_ex(const void *a, const void *b, float *c, int m, int n, int k, int layout,
                                         void *stream)
{
    char msg[160];
    if (!a || !b || !c) return hrpp::report(HRPP_ERR_INVALID_ARG, "NULL matrix");
    if (layout < 0 || layout > (HRPP_GEMM_A_MN_MAJOR | HRPP_GEMM_B_MN_MAJOR))
        return hrpp::report(HRPP_ERR_INVALID_ARG, "unknown layout flags");
    if (((uintptr_t)a & 15u) || ((uintptr_t)b & 15u) || ((uintptr_t)c & 31u))
        return hrpp::report(HRPP_ERR_INVALID_ARG, "A and B must be 16-byte aligned, C 32-byte aligned");
    const int bn = (n % 256 == 0) ? 256 : 128;
    if (!hrpp::gemm_shape_ok(m, n, k, bn)) {
        snprintf(msg, sizeof msg, "shape %d x %d x %d: M must be a multiple of 128, N of 128, K of 64", m, n, k);
        return hrpp::report(HRPP_ERR_INVALID_ARG, msg);
    }
    unsigned int *err = nullptr;
    cudaError_t e = cudaMalloc(&err, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned int), (cudaStream_t)stream);
    if (e == cudaSuccess) {
        hrpp::umma::GemmArgs g = {};
        g.M = m;
        g.N = n;
        g.K = k;
        g.c32 = c;
        g.m_valid = m;
        g.error = err;
        // large K-major problems (two waves of 128 x 256 tiles or more) take
        // the persistent kernel
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            layout == 0 && n % 256 == 0 && (m / 128) * (n / 256) >= 2 * sms)
            e = hrpp::gemm_bf16_persistent(a, b, g, (cudaStream_t)stream);
        else
            e = hrpp::gemm_bf16(a, b, hrpp::umma::EPI_F32, bn, g, 1, (cudaStream_t)stream, layout);
    }
    unsigned int flag = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof flag, cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "gemm: %s", cudaGetErrorString(e));
        return hrpp::report(HRPP_ERR_CUDA, msg);
    }
    if (flag) return hrpp::report(HRPP_ERR_CUDA, "gemm: a pipeline wait timed out");
    return HRPP_OK;
}
