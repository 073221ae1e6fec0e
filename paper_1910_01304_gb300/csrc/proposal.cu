// Learned treelet proposal: a BF16 MLP 96 -> 256 -> 256 -> 4096 trained and
// evaluated on the tensor cores (tcgen05 GEMMs of gemm.cu), predicting per
// ray the root of a BVH treelet to traverse first.
//
// Training step on a minibatch of rows padded to a multiple of 128:
//   X  = features(rays)                      bf16 [B, 128]
//   H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2)   bf16 [B, 256]
//   Z  = H2 W3^T + b3                        fp32, never stored
//   dZ = softmax(Z) - onehot(label)          bf16 [B, 4096]
//   dW3 = dZ^T H2, dZ2 = (dZ W3) * (H2 > 0), dW2 = dZ2^T H1,
//   dZ1 = (dZ2 W2) * (H1 > 0), dW1 = dZ1^T X, db = column sums
//   Adam on fp32 master weights, scaled by 1 / (labelled rows); bf16 copies
//   refreshed, row-major ([out, in]).
// Every GEMM is C = A B^T.  The forward GEMMs read K-major operands; the dZ
// GEMMs read the weights [out, in] as MN-major B; the weight gradients reduce
// over the rows of the minibatch and read the row-major activations and
// gradients as MN-major operands.  Nothing is stored transposed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "gemm.h"
#include "handles.h"
#include "hrpp.h"

using namespace hrpp;

namespace {

constexpr int kIn = 128;    // 96 features padded with zeros to a 64-multiple K
constexpr int kFeat = HRPP_PROPOSAL_FEATURES;
constexpr int kHid = HRPP_PROPOSAL_HIDDEN;
constexpr int kCls = HRPP_PROPOSAL_CLASSES;
constexpr uint32_t kBmax = 16384;   // rows per training minibatch
constexpr uint32_t kBinfer = 65536; // rows per inference chunk
// master parameter layout (W1 padded to [256][128])
constexpr size_t oW1 = 0, ob1 = oW1 + (size_t)kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + (size_t)kHid * kHid,
                 oW3 = ob2 + kHid, ob3 = oW3 + (size_t)kCls * kHid, kMaster = ob3 + kCls;

hrpp_status pfail(hrpp_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return hrpp::report(s, buf);
}

uint16_t bf16_bits_rne(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x7FFFFFu)) return (uint16_t)((b >> 16) | 0x40u);
    const uint32_t rounded = b + 0x7FFFu + ((b >> 16) & 1u);
    return (uint16_t)(rounded >> 16);
}

uint64_t splitmix(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------- kernels --

__device__ __forceinline__ uint32_t quantise16(float u)
{
    if (!(u > 0.0f)) return 0u;
    if (u >= 65535.0f) return 65535u;
    return (uint32_t)u;
}

// Features of 128 rows per block.  Each thread builds its row's 128 bf16
// inputs in shared memory; the block then writes the tile row-major (one
// contiguous 32 KB span of X) with 16-byte stores.
constexpr int kFeatRows = 128;
constexpr int kFeatPitch = kIn + 8;  // bf16 elements per shared row (16-byte aligned, staggers banks)

__global__ void __launch_bounds__(kFeatRows) k_featurize(const float4 *rays, uint32_t n, uint32_t npad, float lox,
                                                         float loy, float loz, float sx, float sy, float sz,
                                                         const __nv_bfloat16 *sin_t, __nv_bfloat16 *X)
{
    __shared__ __align__(16) __nv_bfloat16 tile[kFeatRows * kFeatPitch];
    const uint32_t t = threadIdx.x, r0 = blockIdx.x * kFeatRows, r = r0 + t;
    uint32_t q[5] = {0, 0, 0, 0, 0};
    const bool live = r < n;
    if (live) {
        const float4 o = rays[2ull * r], d = rays[2ull * r + 1];
        q[0] = quantise16(__fmul_rn(__fsub_rn(o.x, lox), sx));
        q[1] = quantise16(__fmul_rn(__fsub_rn(o.y, loy), sy));
        q[2] = quantise16(__fmul_rn(__fsub_rn(o.z, loz), sz));
        const float l1 = __fadd_rn(__fadd_rn(fabsf(d.x), fabsf(d.y)), fabsf(d.z));
        const float px = __fdiv_rn(d.x, l1), py = __fdiv_rn(d.y, l1);
        const float sgx = px >= 0.0f ? 1.0f : -1.0f, sgy = py >= 0.0f ? 1.0f : -1.0f;
        float ux = px, uy = py;
        if (d.z < 0.0f) {
            ux = __fmul_rn(__fsub_rn(1.0f, fabsf(py)), sgx);
            uy = __fmul_rn(__fsub_rn(1.0f, fabsf(px)), sgy);
        }
        q[3] = quantise16(__fmul_rn(__fadd_rn(ux, 1.0f), 32767.5f));
        q[4] = quantise16(__fmul_rn(__fadd_rn(uy, 1.0f), 32767.5f));
    }
    __nv_bfloat16 *row = tile + t * kFeatPitch;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    if (live) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            row[i] = __float2bfloat16_rn(__fsub_rn(__fmul_rn((float)q[i], 1.0f / 32768.0f), 1.0f));
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const uint32_t ph = (q[i] << k) & 0xFFFFu;
                row[5 + 18 * i + 2 * k] = sin_t[ph];                          // sine
                row[6 + 18 * i + 2 * k] = sin_t[(ph + 16384u) & 0xFFFFu];     // cosine
            }
        }
        row[95] = __float2bfloat16_rn(1.0f);
    } else {
#pragma unroll
        for (int c = 0; c < kFeat; ++c) row[c] = zero;
    }
    // padding columns 96..127
    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int c = kFeat; c < kIn; c += 8) *reinterpret_cast<uint4 *>(row + c) = z4;
    __syncthreads();
    // row-major: the tile's rows are consecutive in X
    const uint32_t rows_here = npad - r0 < (uint32_t)kFeatRows ? npad - r0 : (uint32_t)kFeatRows;
    uint4 *dst = reinterpret_cast<uint4 *>(X + (size_t)r0 * kIn);
    for (uint32_t k = t; k < rows_here * (kIn / 8); k += kFeatRows) {
        const uint32_t rr = k / (kIn / 8), cc = (k % (kIn / 8)) * 8;
        dst[k] = *reinterpret_cast<const uint4 *>(tile + rr * kFeatPitch + cc);
    }
}

// out[c] += sum over rows of a bf16 [rows, cols] row-major matrix (the bias
// gradients; cols a multiple of 256), for one or two matrices of one shape
// (blockIdx.z picks the matrix).  A block of 32 x 8 threads covers 256
// columns and SPAN rows (a multiple of 64): thread (x, y) sums the 8
// adjacent columns of group x (one 16-byte load per row) over rows y, y + 8,
// ..., so each warp reads 512 contiguous bytes per row; the 8 partial sums of
// a column meet in shared memory and the block adds them with one atomic per
// column.  The host picks SPAN so that the grid fills the GPU.
struct ColsumJob {
    const __nv_bfloat16 *a[2];
    float *out[2];
};

template <uint32_t SPAN>
__global__ void __launch_bounds__(256) k_colsum(const ColsumJob job, uint32_t rows, uint32_t cols)
{
    static_assert(SPAN % 64u == 0u, "whole unrolled rounds of 8 rows per thread");
    __shared__ float part[8][32 * 8 + 4];
    const __nv_bfloat16 *a = blockIdx.z ? job.a[1] : job.a[0];
    float *out = blockIdx.z ? job.out[1] : job.out[0];
    const uint32_t x = threadIdx.x, y = threadIdx.y;
    const uint32_t c = 8u * (blockIdx.x * 32u + x);
    const uint32_t r0 = blockIdx.y * SPAN;
    const uint32_t r1 = r0 + SPAN < rows ? r0 + SPAN : rows;
    float acc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    const __nv_bfloat16 *p = a + (size_t)(r0 + y) * cols + c;
#pragma unroll 8
    for (uint32_t r = r0 + y; r < r1; r += 8u, p += 8ull * cols) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 f = __bfloat1622float2(h[j]);
            acc[2 * j] += f.x;
            acc[2 * j + 1] += f.y;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) part[y][8 * x + j] = acc[j];
    __syncthreads();
    // thread (x, y) now adds column 8x' + j' of the block for one (x', j')
    const uint32_t t = y * 32u + x;  // 0..255: one column of the block each
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += part[k][t];
    atomicAdd(out + 8u * blockIdx.x * 32u + t, sum);
}

// Column sums of a (and of a2 into out2, when a2 is not null; same shape).
// Rows per block: 256 when that still gives every SM work (a 16K x 4096
// matrix: 1,024 blocks), else 64 (two 16K x 256 matrices: 512 blocks, where
// 256 rows per block left most SMs idle).  A compile-time span lets the
// row loop run as whole unrolled rounds; a runtime span measured 15 % slower
// on the wide matrix.
void colsum(const __nv_bfloat16 *a, uint32_t rows, uint32_t cols, float *out, int sms, cudaStream_t s,
            const __nv_bfloat16 *a2 = nullptr, float *out2 = nullptr)
{
    const uint32_t mats = a2 ? 2u : 1u;
    const uint32_t col_blocks = cols / 256u;
    const ColsumJob job{{a, a2 ? a2 : a}, {out, a2 ? out2 : out}};
    const uint64_t blocks256 = (uint64_t)col_blocks * mats * ((rows + 255u) / 256u);
    if (blocks256 >= 4ull * (uint64_t)(sms > 0 ? sms : 1)) {
        const dim3 grid(col_blocks, (rows + 255u) / 256u, mats);
        k_colsum<256><<<grid, dim3(32, 8), 0, s>>>(job, rows, cols);
    } else {
        const dim3 grid(col_blocks, (rows + 63u) / 64u, mats);
        k_colsum<64><<<grid, dim3(32, 8), 0, s>>>(job, rows, cols);
    }
}

// Adam on every parameter in one launch (masters laid out W1 | b1 | W2 | b2 |
// W3 | b3, weights [rows, cols] row-major); the weights' bf16 copies are
// refreshed, row-major (the dZ GEMMs read W2 and W3 as MN-major operands).
struct AdamOut {
    __nv_bfloat16 *w1h, *w2h, *w3h;
};

__global__ void __launch_bounds__(256) k_adam(float *w, const float *g, float *m, float *v, float lr, float bc1,
                                              float bc2, const unsigned int *count, AdamOut out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMaster) return;
    const float scale = 1.0f / (float)(*count > 0u ? *count : 1u);
    const float gi = g[i] * scale;
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    w[i] = wi;
    const __nv_bfloat16 h = __float2bfloat16_rn(wi);
    if (i < ob1) {
        out.w1h[i - oW1] = h;
    } else if (i >= oW2 && i < ob2) {
        out.w2h[i - oW2] = h;
    } else if (i >= oW3 && i < ob3) {
        out.w3h[i - oW3] = h;
    }
}

// adds one minibatch's loss total and labelled-row count to the call's
__global__ void k_accumulate_loss(const float *loss_sum, const unsigned int *count, float *call_loss,
                                  unsigned int *call_count)
{
    *call_loss += *loss_sum;
    *call_count += *count;
}

__global__ void k_to_bf16(const float *w, uint32_t n, __nv_bfloat16 *wh)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wh[i] = __float2bfloat16_rn(w[i]);
}

__global__ void k_labels(const float4 *hits, uint32_t n, const int32_t *prim_class, uint32_t n_tris, int32_t *out)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t prim = __float_as_uint(hits[r].y);
    out[r] = prim < n_tris ? prim_class[prim] : -1;
}

}  // namespace

struct hrpp_proposal {
    int device, width;
    int sms;  // the device's SM count (grid sizes)
    uint32_t n_tris, n_nodes;
    float lo[3], scale[3];
    __nv_bfloat16 *sin_t;
    int32_t *class_node, *prim_class;
    std::vector<int32_t> h_class_node;
    float *master, *grad, *m, *v;
    __nv_bfloat16 *w1h, *w2h, *w3h;
    int step;
    __nv_bfloat16 *X, *H1, *H2, *dZ3, *dZ2, *dZ1;
    float *loss_sum;
    unsigned int *count, *err;
    float *call_loss;           // loss and labelled rows summed over one train call
    unsigned int *call_count;
    int32_t *lab;
    // inference chunk buffers (allocated on the first prediction)
    __nv_bfloat16 *Xi, *H1i, *H2i;
    // the backward's second stream and its fork / join events
    cudaStream_t side;
    cudaEvent_t fork_dz3, fork_dz2, join;
};

namespace {

void proposal_free(hrpp_proposal *p)
{
    if (!p) return;
    void *ptrs[] = {p->sin_t, p->class_node, p->prim_class, p->master, p->grad, p->m, p->v, p->w1h, p->w2h,
                    p->w3h, p->X, p->H1, p->H2, p->dZ3, p->dZ2, p->dZ1, p->loss_sum, p->count, p->err, p->call_loss, p->call_count,
                    p->lab, p->Xi, p->H1i, p->H2i};
    for (void *q : ptrs) cudaFree(q);
    if (p->side) cudaStreamDestroy(p->side);
    for (cudaEvent_t ev : {p->fork_dz3, p->fork_dz2, p->join})
        if (ev) cudaEventDestroy(ev);
    delete p;
}

struct Dev {
    int prev = -1;
    cudaError_t err;
    explicit Dev(int d)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != d) err = cudaSetDevice(d);
    }
    ~Dev()
    {
        int c = -1;
        if (prev >= 0 && cudaGetDevice(&c) == cudaSuccess && c != prev) cudaSetDevice(prev);
    }
};

cudaError_t refresh_bf16(hrpp_proposal *p, cudaStream_t s)
{
    auto run = [&](size_t off, uint32_t rows, uint32_t cols, __nv_bfloat16 *wh) {
        const uint32_t n = rows * cols;
        k_to_bf16<<<(n + 255) / 256, 256, 0, s>>>(p->master + off, n, wh);
    };
    run(oW1, kHid, kIn, p->w1h);
    run(oW2, kHid, kHid, p->w2h);
    run(oW3, kCls, kHid, p->w3h);
    return cudaGetLastError();
}

uint32_t pad128(uint32_t n) { return (n + 127u) & ~127u; }

// 256-wide tiles unless that leaves fewer than two CTAs per SM (152 SMs)
// Tile width: 256 when there are tiles for two waves, or when K is long
// enough (>= 2048) that one wave of wide tiles streams A once instead of
// splitting it over a partial second wave.
int tile_n(int m, int n, int k)
{
    const bool wide_ok = n % 256 == 0 && ((m / 128) * (n / 256) >= 2 * 152 || k >= 2048);
    return wide_ok ? 256 : 128;
}

umma::GemmArgs args(int m, int n, int k, hrpp_proposal *p)
{
    umma::GemmArgs g = {};
    g.M = m;
    g.N = n;
    g.K = k;
    g.m_valid = m;
    g.error = p->err;
    return g;
}

// Split-K factor for a weight gradient with m_tiles row tiles (one column
// tile): `ctas` CTAs in all, at most one K block per split.  dW3 (32 row
// tiles) takes 128 CTAs; the 256 x 256 and 256 x 128 hidden-layer gradients
// take 64, which halves their fp32 atomic traffic and measured 2 % faster
// per training minibatch than 128 (2 and 8 splits for dW3 were slower).
int splits_for(int m_tiles, int k, int ctas = 128)
{
    const int kb = k / umma::BK;
    int s = ctas / (m_tiles > 0 ? m_tiles : 1);
    if (s < 1) s = 1;
    if (s > kb) s = kb;
    return s;
}

// The gradients of one minibatch from dZ3 (softmax output minus one-hot):
// weight gradients and db3 on `side`, activation gradients and db2, db1 on
// `s`; `side` waits for dZ2 before dW2.  The caller forks `side` from `s`
// after dZ3 and joins it back.
cudaError_t backward(hrpp_proposal *p, uint32_t npad, cudaStream_t s, cudaStream_t side)
{
    cudaError_t e;
    umma::GemmArgs g;
    // the weight gradients reduce over rows: both operands MN-major
    constexpr int kMN = GEMM_A_MN | GEMM_B_MN;
    // side: db3, then dW3 = dZ3^T H2
    colsum(p->dZ3, npad, kCls, p->grad + ob3, p->sms, side);
    g = args(kCls, kHid, (int)npad, p);
    g.c32 = p->grad + oW3;
    if ((e = gemm_bf16(p->dZ3, p->H2, umma::EPI_F32_ATOMIC, 256, g, splits_for(kCls / 128, (int)npad), side, kMN)) !=
        cudaSuccess)
        return e;
    // s: dZ2 = (dZ3 W3) * (H2 > 0); B = W3 stored [4096, 256]: read MN-major
    g = args((int)npad, kHid, kCls, p);
    g.act = p->H2;
    g.c16 = p->dZ2;
    if ((e = gemm_bf16(p->dZ3, p->w3h, umma::EPI_RELU_GRAD, tile_n((int)npad, kHid, kCls), g, 1, s, GEMM_B_MN)) !=
        cudaSuccess)
        return e;
    if ((e = cudaEventRecord(p->fork_dz2, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, p->fork_dz2, 0)) != cudaSuccess) return e;
    // side: dW2 = dZ2^T H1
    g = args(kHid, kHid, (int)npad, p);
    g.c32 = p->grad + oW2;
    e = gemm_bf16(p->dZ2, p->H1, umma::EPI_F32_ATOMIC, 256, g, splits_for(kHid / 128, (int)npad, 64), side, kMN);
    if (e != cudaSuccess) return e;
    // s: dZ1 = (dZ2 W2) * (H1 > 0)
    g = args((int)npad, kHid, kHid, p);
    g.act = p->H1;
    g.c16 = p->dZ1;
    if ((e = gemm_bf16(p->dZ2, p->w2h, umma::EPI_RELU_GRAD, tile_n((int)npad, kHid, kHid), g, 1, s, GEMM_B_MN)) !=
        cudaSuccess)
        return e;
    // s: dW1 = dZ1^T X, then db2 and db1 in one launch
    g = args(kHid, kIn, (int)npad, p);
    g.c32 = p->grad + oW1;
    if ((e = gemm_bf16(p->dZ1, p->X, umma::EPI_F32_ATOMIC, 128, g, splits_for(kHid / 128, (int)npad, 64), s, kMN)) !=
        cudaSuccess)
        return e;
    colsum(p->dZ2, npad, kHid, p->grad + ob2, p->sms, s, p->dZ1, p->grad + ob1);
    return cudaGetLastError();
}

// forward (and, when train, the backward into p->grad) on rows [0, n) of
// rays, padded to npad rows; labels (device) when train
cudaError_t run_batch(hrpp_proposal *p, const hrpp_ray *rays, uint32_t n, const int32_t *labels, bool train,
                      bool argmax, cudaStream_t s, int32_t *out_nodes = nullptr, int32_t *out_classes = nullptr)
{
    const uint32_t npad = pad128(n);
    cudaError_t e;
    __nv_bfloat16 *X = argmax ? p->Xi : p->X, *H1 = argmax ? p->H1i : p->H1, *H2 = argmax ? p->H2i : p->H2;
    k_featurize<<<npad / kFeatRows, kFeatRows, 0, s>>>(reinterpret_cast<const float4 *>(rays), n, npad, p->lo[0],
                                                    p->lo[1], p->lo[2], p->scale[0], p->scale[1], p->scale[2],
                                                    p->sin_t, X);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    umma::GemmArgs g = args((int)npad, kHid, kIn, p);
    g.bias = p->master + ob1;
    g.c16 = H1;
    if ((e = gemm_bf16(X, p->w1h, umma::EPI_BIAS_RELU, tile_n((int)npad, kHid, kIn), g, 1, s)) != cudaSuccess) return e;
    g = args((int)npad, kHid, kHid, p);
    g.bias = p->master + ob2;
    g.c16 = H2;
    if ((e = gemm_bf16(H1, p->w2h, umma::EPI_BIAS_RELU, tile_n((int)npad, kHid, kHid), g, 1, s)) != cudaSuccess) return e;
    if (argmax) {
        // output layer and first argmax in one tensor-core pass
        umma::SoftmaxArgs sx = {};
        sx.bias = p->master + ob3;
        sx.n = (int)n;
        sx.npad = (int)npad;
        sx.out_classes = out_classes;
        sx.out_nodes = out_nodes;
        sx.class_node = p->class_node;
        sx.error = p->err;
        return softmax_argmax(H2, p->w3h, sx, s);
    }
    if (!train) return cudaErrorInvalidValue;  // forward passes end in the argmax above
    if ((e = cudaMemcpyAsync(p->lab, labels, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->loss_sum, 0, sizeof(float), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->count, 0, sizeof(unsigned int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->grad, 0, sizeof(float) * kMaster, s)) != cudaSuccess)
        return e;
    // logits, softmax cross-entropy and dZ3 in one tensor-core pass (the
    // logits never reach memory)
    umma::SoftmaxArgs sx = {};
    sx.bias = p->master + ob3;
    sx.labels = p->lab;
    sx.n = (int)n;
    sx.npad = (int)npad;
    sx.dz = p->dZ3;
    sx.loss_sum = p->loss_sum;
    sx.count = p->count;
    sx.error = p->err;
    if ((e = softmax_xent(H2, p->w3h, sx, s)) != cudaSuccess) return e;
    // The backward on two streams.  dZ3 feeds db3, dW3 and dZ2; dZ2 feeds dW2
    // and dZ1.  The weight gradients (and db3) go to p->side while the
    // activation gradients stay on s, so each pair shares the SMs (a 128-CTA
    // GEMM alone leaves 24 of 152 idle) and reads its common input once from
    // HBM while the other still finds it in L2.  The join comes before the
    // call returns, on every path, so that s orders everything after it.
    if ((e = cudaEventRecord(p->fork_dz3, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(p->side, p->fork_dz3, 0)) != cudaSuccess) return e;
    e = backward(p, npad, s, p->side);
    const cudaError_t ej = cudaEventRecord(p->join, p->side);
    const cudaError_t ew = ej == cudaSuccess ? cudaStreamWaitEvent(s, p->join, 0) : ej;
    if (e != cudaSuccess) return e;
    return ew != cudaSuccess ? ew : cudaGetLastError();
}

cudaError_t adam(hrpp_proposal *p, float lr, cudaStream_t s)
{
    p->step += 1;
    const float bc1 = 1.0f - std::pow(0.9f, (float)p->step), bc2 = 1.0f - std::pow(0.999f, (float)p->step);
    const AdamOut out = {p->w1h, p->w2h, p->w3h};
    k_adam<<<(unsigned)((kMaster + 255) / 256), 256, 0, s>>>(p->master, p->grad, p->m, p->v, lr, bc1, bc2, p->count,
                                                             out);
    return cudaGetLastError();
}

hrpp_status check_err(hrpp_proposal *p)
{
    unsigned int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, p->err, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "proposal: %s", cudaGetErrorString(e));
    if (flag) {
        cudaMemset(p->err, 0, sizeof(unsigned int));
        return pfail(HRPP_ERR_CUDA, "proposal: a tensor-core pipeline wait timed out");
    }
    return HRPP_OK;
}

// host copy of the masters in the API layout (W1 without its padding)
void masters_to_api(const std::vector<float> &m, float *out)
{
    size_t o = 0;
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c < kFeat; ++c) out[o++] = m[oW1 + (size_t)r * kIn + c];
    for (size_t i = ob1; i < kMaster; ++i) out[o++] = m[i];
}

void api_to_masters(const float *in, std::vector<float> &m)
{
    m.assign(kMaster, 0.0f);
    size_t o = 0;
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c < kFeat; ++c) m[oW1 + (size_t)r * kIn + c] = in[o++];
    for (size_t i = ob1; i < kMaster; ++i) m[i] = in[o++];
}

}  // namespace

extern "C" {

hrpp_status hrpp_proposal_create(const hrpp_scene *sc, const hrpp_bvh_node *nodes, uint32_t n_nodes, uint32_t root,
                                 const uint32_t *prim_index, uint32_t n_prim_index, uint64_t seed,
                                 hrpp_proposal **out)
{
    if (!sc || !nodes || !prim_index || !out) return pfail(HRPP_ERR_INVALID_ARG, "NULL argument");
    if (n_nodes != sc->n_nodes || n_prim_index != sc->n_tris || root >= n_nodes)
        return pfail(HRPP_ERR_INVALID_ARG, "the BVH does not match the scene");
    Dev dv(sc->device);
    if (dv.err != cudaSuccess) return pfail(HRPP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(dv.err));
    hrpp_proposal *p = new (std::nothrow) hrpp_proposal();
    if (!p) return pfail(HRPP_ERR_OOM, "host allocation");
    p->device = sc->device;
    p->width = sc->width;
    const cudaError_t ae = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, sc->device);
    if (ae != cudaSuccess) {
        delete p;
        return pfail(HRPP_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(ae));
    }
    p->n_tris = sc->n_tris;
    p->n_nodes = n_nodes;
    const hrpp_bvh_node &rn = nodes[root];
    for (int a = 0; a < 3; ++a) {
        p->lo[a] = rn.lo[a];
        p->scale[a] = 65535.0f / (rn.hi[a] - rn.lo[a]);
    }
    // classes: 12-bit path codes (one bit per level in BVH2, two in BVH4)
    const int bits = p->width == 2 ? 1 : 2, levels = 12 / bits;
    std::vector<int32_t> prim_class(sc->n_tris, -1);
    struct Item {
        uint32_t node;
        uint32_t code;
        int depth;
    };
    std::vector<Item> st{{root, 0u, 0}};
    while (!st.empty()) {
        const Item it = st.back();
        st.pop_back();
        const hrpp_bvh_node &n = nodes[it.node];
        if (n.count > 0) {
            const uint32_t code = it.depth <= levels ? it.code << (bits * (levels - it.depth)) : it.code;
            for (uint32_t j = 0; j < n.count && n.first + j < n_prim_index; ++j)
                if (prim_index[n.first + j] < sc->n_tris) prim_class[prim_index[n.first + j]] = (int32_t)code;
            continue;
        }
        for (int q = 0; q < 4; ++q) {
            const int32_t c = n.child[q];
            if (c < 0 || (uint32_t)c >= n_nodes) continue;
            if (it.depth < levels) st.push_back({(uint32_t)c, (it.code << bits) | (uint32_t)q, it.depth + 1});
            else st.push_back({(uint32_t)c, it.code, it.depth + 1});
        }
    }
    p->h_class_node.assign(kCls, (int32_t)root);
    for (int cls = 0; cls < kCls; ++cls) {
        uint32_t node = root;
        for (int lv = 0; lv < levels; ++lv) {
            if (nodes[node].count > 0) break;
            const int q = (cls >> (bits * (levels - 1 - lv))) & ((1 << bits) - 1);
            const int32_t c = nodes[node].child[q];
            if (c < 0 || (uint32_t)c >= n_nodes) break;
            node = (uint32_t)c;
        }
        p->h_class_node[cls] = (int32_t)node;
    }
    // sine table: sin(2 pi j / 65536) in double, rounded to float, then bf16
    std::vector<uint16_t> sin_h(65536);
    for (int j = 0; j < 65536; ++j) sin_h[j] = bf16_bits_rne((float)std::sin(2.0 * M_PI * j / 65536.0));
    // initial weights: He-uniform, zero biases, W1's padding columns zero
    std::vector<float> mh(kMaster, 0.0f);
    uint64_t rs = seed;
    auto uni = [&](float a) { return (float)(((splitmix(rs) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * a; };
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c < kFeat; ++c) mh[oW1 + (size_t)r * kIn + c] = uni(std::sqrt(6.0f / kFeat));
    for (size_t i = oW2; i < ob2; ++i) mh[i] = uni(std::sqrt(6.0f / kHid));
    for (size_t i = oW3; i < ob3; ++i) mh[i] = uni(std::sqrt(6.0f / kHid));
    const size_t rows = kBmax;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto **ptr, size_t bytes) {
        if (e == cudaSuccess) e = hrpp::device_malloc((void **)ptr, bytes);
    };
    alloc(&p->sin_t, 65536 * 2);
    alloc(&p->class_node, kCls * 4);
    alloc(&p->prim_class, (size_t)sc->n_tris * 4);
    alloc(&p->master, kMaster * 4);
    alloc(&p->grad, kMaster * 4);
    alloc(&p->m, kMaster * 4);
    alloc(&p->v, kMaster * 4);
    alloc(&p->w1h, (size_t)kHid * kIn * 2);
    alloc(&p->w2h, (size_t)kHid * kHid * 2);
    alloc(&p->w3h, (size_t)kCls * kHid * 2);
    alloc(&p->X, rows * kIn * 2);
    alloc(&p->H1, rows * kHid * 2);
    alloc(&p->H2, rows * kHid * 2);
    alloc(&p->dZ3, rows * kCls * 2);
    alloc(&p->dZ2, rows * kHid * 2);
    alloc(&p->dZ1, rows * kHid * 2);
    alloc(&p->loss_sum, 4);
    alloc(&p->count, 4);
    alloc(&p->err, 4);
    alloc(&p->call_loss, 4);
    alloc(&p->call_count, 4);
    alloc(&p->lab, rows * 4);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&p->fork_dz3, &p->fork_dz2, &p->join})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpy(p->sin_t, sin_h.data(), 65536 * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->class_node, p->h_class_node.data(), kCls * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->prim_class, prim_class.data(), (size_t)sc->n_tris * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->master, mh.data(), kMaster * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->m, 0, kMaster * 4);
    if (e == cudaSuccess) e = cudaMemset(p->v, 0, kMaster * 4);
    if (e == cudaSuccess) e = cudaMemset(p->err, 0, 4);
    if (e == cudaSuccess) e = refresh_bf16(p, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        proposal_free(p);
        return pfail(e == cudaErrorMemoryAllocation ? HRPP_ERR_OOM : HRPP_ERR_CUDA, "proposal: %s",
                     cudaGetErrorString(e));
    }
    *out = p;
    return HRPP_OK;
}

hrpp_status hrpp_proposal_features(hrpp_proposal *p, const hrpp_ray *rays, uint32_t n, void *out_bf16, void *stream)
{
    if (!p || (n && (!rays || !out_bf16))) return pfail(HRPP_ERR_INVALID_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(out_bf16) % 16) return pfail(HRPP_ERR_INVALID_ARG, "out_bf16 not 16-byte aligned");
    Dev dv(p->device);
    if (n == 0) return HRPP_OK;
    k_featurize<<<(n + kFeatRows - 1) / kFeatRows, kFeatRows, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4 *>(rays), n, n, p->lo[0], p->lo[1], p->lo[2], p->scale[0], p->scale[1],
        p->scale[2], p->sin_t, static_cast<__nv_bfloat16 *>(out_bf16));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "features: %s", cudaGetErrorString(e));
    return HRPP_OK;
}

hrpp_status hrpp_proposal_labels(hrpp_proposal *p, const hrpp_hit *hits, uint32_t n, int32_t *out_labels, void *stream)
{
    if (!p || (n && (!hits || !out_labels))) return pfail(HRPP_ERR_INVALID_ARG, "NULL argument");
    Dev dv(p->device);
    if (n == 0) return HRPP_OK;
    k_labels<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4 *>(hits), n,
                                                                 p->prim_class, p->n_tris, out_labels);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "labels: %s", cudaGetErrorString(e));
    return HRPP_OK;
}

hrpp_status hrpp_proposal_train(hrpp_proposal *p, const hrpp_ray *rays, const int32_t *labels, uint32_t n, float lr,
                                float *out_mean_loss, void *stream)
{
    hrpp::NvtxRange nvtx_range("hrpp_proposal_train");
    if (!p || (n && (!rays || !labels))) return pfail(HRPP_ERR_INVALID_ARG, "NULL argument");
    if (!(lr > 0.0f)) return pfail(HRPP_ERR_INVALID_ARG, "lr must be positive");
    Dev dv(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (out_mean_loss) {
        if ((e = cudaMemsetAsync(p->call_loss, 0, 4, s)) == cudaSuccess)
            e = cudaMemsetAsync(p->call_count, 0, 4, s);
    }
    for (uint32_t off = 0; off < n && e == cudaSuccess; off += kBmax) {
        const uint32_t b = n - off < kBmax ? n - off : kBmax;
        e = run_batch(p, rays + off, b, labels + off, true, false, s);
        if (e == cudaSuccess) e = adam(p, lr, s);
        if (e == cudaSuccess && out_mean_loss) {
            k_accumulate_loss<<<1, 1, 0, s>>>(p->loss_sum, p->count, p->call_loss, p->call_count);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "train: %s", cudaGetErrorString(e));
    if (out_mean_loss) {
        float sum = 0.0f;
        unsigned int cnt = 0;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess ||
            (e = cudaMemcpy(&sum, p->call_loss, 4, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&cnt, p->call_count, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return pfail(HRPP_ERR_CUDA, "train: %s", cudaGetErrorString(e));
        *out_mean_loss = cnt ? sum / (float)cnt : 0.0f;
        return check_err(p);
    }
    return HRPP_OK;
}

hrpp_status hrpp_proposal_gradients(hrpp_proposal *p, const hrpp_ray *rays, const int32_t *labels, uint32_t n,
                                    float *host_grads, float *out_mean_loss)
{
    if (!p || !rays || !labels || !host_grads || n == 0) return pfail(HRPP_ERR_INVALID_ARG, "NULL argument or n = 0");
    if (n > kBmax) return pfail(HRPP_ERR_INVALID_ARG, "at most %u rays", kBmax);
    Dev dv(p->device);
    cudaError_t e = run_batch(p, rays, n, labels, true, false, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    std::vector<float> g(kMaster);
    float sum = 0.0f;
    unsigned int cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpy(g.data(), p->grad, kMaster * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&sum, p->loss_sum, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&cnt, p->count, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "gradients: %s", cudaGetErrorString(e));
    const float scale = 1.0f / (float)(cnt ? cnt : 1u);
    for (float &x : g) x *= scale;
    masters_to_api(g, host_grads);
    if (out_mean_loss) *out_mean_loss = cnt ? sum / (float)cnt : 0.0f;
    return check_err(p);
}

hrpp_status hrpp_proposal_predict(hrpp_proposal *p, const hrpp_ray *rays, uint32_t n, int32_t *out_nodes,
                                  int32_t *out_classes, void *stream)
{
    hrpp::NvtxRange nvtx_range("hrpp_proposal_predict");
    if (!p || (n && (!rays || (!out_nodes && !out_classes)))) return pfail(HRPP_ERR_INVALID_ARG, "NULL argument");
    Dev dv(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!p->Xi) {
        if ((e = hrpp::device_malloc((void **)&p->Xi, (size_t)kBinfer * kIn * 2)) != cudaSuccess ||
            (e = hrpp::device_malloc((void **)&p->H1i, (size_t)kBinfer * kHid * 2)) != cudaSuccess ||
            (e = hrpp::device_malloc((void **)&p->H2i, (size_t)kBinfer * kHid * 2)) != cudaSuccess) {
            void *bufs[] = {p->Xi, p->H1i, p->H2i};
            for (void *q : bufs) cudaFree(q);
            p->Xi = p->H1i = p->H2i = nullptr;
            return pfail(e == cudaErrorMemoryAllocation ? HRPP_ERR_OOM : HRPP_ERR_CUDA, "predict buffers: %s",
                         cudaGetErrorString(e));
        }
    }
    for (uint32_t off = 0; off < n && e == cudaSuccess; off += kBinfer) {
        const uint32_t b = n - off < kBinfer ? n - off : kBinfer;
        e = run_batch(p, rays + off, b, nullptr, false, true, s, out_nodes ? out_nodes + off : nullptr,
                      out_classes ? out_classes + off : nullptr);
    }
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "predict: %s", cudaGetErrorString(e));
    return HRPP_OK;
}

hrpp_status hrpp_proposal_get_weights(const hrpp_proposal *p, float *host, size_t n_floats)
{
    if (!p || !host || n_floats != HRPP_PROPOSAL_PARAMS) return pfail(HRPP_ERR_INVALID_ARG, "need %u floats", HRPP_PROPOSAL_PARAMS);
    Dev dv(p->device);
    std::vector<float> mh(kMaster);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(mh.data(), p->master, kMaster * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "get_weights: %s", cudaGetErrorString(e));
    masters_to_api(mh, host);
    return HRPP_OK;
}

hrpp_status hrpp_proposal_set_weights(hrpp_proposal *p, const float *host, size_t n_floats)
{
    if (!p || !host || n_floats != HRPP_PROPOSAL_PARAMS) return pfail(HRPP_ERR_INVALID_ARG, "need %u floats", HRPP_PROPOSAL_PARAMS);
    Dev dv(p->device);
    std::vector<float> mh;
    api_to_masters(host, mh);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(p->master, mh.data(), kMaster * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->m, 0, kMaster * 4);
    if (e == cudaSuccess) e = cudaMemset(p->v, 0, kMaster * 4);
    if (e == cudaSuccess) e = refresh_bf16(p, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return pfail(HRPP_ERR_CUDA, "set_weights: %s", cudaGetErrorString(e));
    p->step = 0;
    return HRPP_OK;
}

hrpp_status hrpp_proposal_class_nodes(const hrpp_proposal *p, int32_t *host_nodes)
{
    if (!p || !host_nodes) return pfail(HRPP_ERR_INVALID_ARG, "NULL argument");
    memcpy(host_nodes, p->h_class_node.data(), sizeof(int32_t) * kCls);
    return HRPP_OK;
}

void hrpp_proposal_destroy(hrpp_proposal *p)
{
    if (!p) return;
    Dev dv(p->device);
    cudaDeviceSynchronize();
    proposal_free(p);
}

}  // extern "C"
