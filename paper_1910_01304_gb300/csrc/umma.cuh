// Tensor-core GEMM for sm_103a: tcgen05.mma with the accumulator in tensor
// memory (TMEM), operands staged in shared memory by TMA.
//
//   C[M, N] = A[M, K] * B[N, K]^T        A, B: bf16; accumulation fp32 in TMEM
//
// Each operand is K-major (stored [M or N][K], rows of K) or MN-major (stored
// [K][M or N]: the row-major activations and gradients of the training step,
// whose weight gradients reduce over rows), chosen per operand at compile time.
//
// One CTA computes a 128 x BN tile of C (BN = 128 or 256) over a K range:
//   warp 0 lane 0   TMA producer: per 64-wide K block, one 128 x 64 A tile
//                   and one BN x 64 B tile (128-byte swizzle) into a 4-stage
//                   ring guarded by full/empty mbarriers; an MN-major tile is
//                   loaded as 64-wide slices of 64 K rows, 8 KB apart
//   warp 1 lane 0   MMA issuer: 4 x tcgen05.mma (K = 16 each) per K block,
//                   tcgen05.commit frees the stage; a last commit signals the
//                   accumulator
//   warps 0-3       epilogue: thread t of warp w owns row 32w + t, reads its
//                   TMEM lane 16 columns at a time (tcgen05.ld 32x32b.x16)
// Every mbarrier wait is bounded; a wait that gives up sets an error flag,
// the kernel drains its outstanding copies (bounded again), frees its TMEM
// and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hrpp {
namespace umma {

constexpr int BM = 128;
constexpr int BK = 64;  // bf16 elements per 128-byte swizzle row
constexpr int STAGES = 4;
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait rounds before giving up

enum Epilogue : int {
    EPI_F32 = 0,        // C (+ bias per column) -> fp32 row-major
    EPI_F32_ATOMIC = 1, // split-K: atomicAdd into fp32 row-major
    EPI_BIAS_RELU = 2,  // relu(C + bias) -> bf16 row-major
    EPI_RELU_GRAD = 3   // C * (act > 0) -> bf16 row-major
};

struct GemmArgs {
    int M, N, K;             // full problem (M, N multiples of 128/BN; K of 64)
    int k_blocks_per_split;  // K blocks handled by one CTA (gridDim.z splits)
    float *c32;              // EPI_F32 / EPI_F32_ATOMIC output [M, N]
    __nv_bfloat16 *c16;      // bf16 output [M, N]
    const float *bias;       // per column (may be null)
    const __nv_bfloat16 *act;   // EPI_RELU_GRAD: activation [M, N] whose > 0 mask is applied
    int m_valid;             // rows >= m_valid are padding: not written
    unsigned int *error;     // set to 1 when a bounded wait gives up
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle.  K-major: rows of 128
// bytes (64 K elements), 8-row core groups 1024 bytes apart (the leading
// offset is unused).  MN-major: rows of 128 bytes hold 64 M (or N) elements
// of one K index; 8-row groups along K are 1024 bytes apart (stride offset)
// and 64-element slices along M (N) are kMnSliceBytes apart (leading offset).
constexpr uint32_t kMnSliceBytes = BK * 128;  // one 64 x 64 slice: 64 K rows of 128 bytes

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, bool mn_major = false)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);                          // start address
    d |= (uint64_t)((mn_major ? kMnSliceBytes : 16u) >> 4) << 16;      // leading byte offset
    d |= (uint64_t)(1024u >> 4) << 32;                                 // stride byte offset
    d |= (uint64_t)1u << 46;                                           // descriptor version
    d |= (uint64_t)2u << 61;                                           // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, M x N
// tile; a_mn / b_mn mark an MN-major operand (the transpose bits).
__host__ __device__ constexpr uint32_t instr_desc(int m, int n, bool a_mn = false, bool b_mn = false)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Byte offset of the k-th 16-deep K step inside one stage's operand tile:
// 32 bytes along a K-major row, two 8-row groups down an MN-major slice.
__host__ __device__ constexpr uint32_t kstep_offset(int k, bool mn_major)
{
    return mn_major ? 2048u * (uint32_t)k : 32u * (uint32_t)k;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One 32-byte global store (dst 32-byte aligned).  A lane's 32 bytes fill a
// whole sector, and a warp's store with each lane on its own row costs one L2
// request per row instead of two.
__device__ __forceinline__ void st_global_32b(void *dst, const uint32_t (&w)[8])
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN, int NST = STAGES>
constexpr size_t gemm_smem_bytes()
{
    return (size_t)NST * ((size_t)BM * BK * 2 + (size_t)BN * BK * 2) + 1024;
}

// NST pipeline stages: 4 for long K; 2 for short K, which halves the shared
// memory so two CTAs share an SM (their TMEM accumulators fit its 512
// columns) and one CTA's epilogue overlaps the other's loads
// AMN / BMN: A / B is MN-major (its tensor map is [K][M or N], 64 x 64 boxes).
template <int BN, int EPI, int NST = STAGES, bool AMN = false, bool BMN = false>
__global__ void __launch_bounds__(128, 1) k_gemm(const __grid_constant__ CUtensorMap tma_a,
                                                 const __grid_constant__ CUtensorMap tma_b, const GemmArgs g)
{
    static_assert(BN == 128 || BN == 256, "tile width");
    static_assert(NST >= 2 && NST <= STAGES, "stages");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], accum_bar;
    __shared__ uint32_t tmem_base;
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t kABytes = BM * BK * 2, kBBytes = BN * BK * 2;
    unsigned char *a_s = smem;
    unsigned char *b_s = smem + NST * kABytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb0 = blockIdx.z * g.k_blocks_per_split;
    int kb_end = kb0 + g.k_blocks_per_split;
    if (kb_end > g.K / BK) kb_end = g.K / BK;
    const int n_kb = kb_end > kb0 ? kb_end - kb0 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&accum_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool failed = false;
    int issued = 0;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int i = 0; i < n_kb; ++i) {
            const int s = i % NST;
            const uint32_t ph = (uint32_t)(i / NST) & 1u;
            if (!mbar_wait(&empty_bar[s], ph ^ 1u)) {
                failed = true;
                break;
            }
            mbar_expect_tx(&full_bar[s], kABytes + kBBytes);
            const int k0 = (kb0 + i) * BK;
            if (AMN) {
#pragma unroll
                for (int j = 0; j < BM / 64; ++j)
                    tma_load_2d(a_s + s * kABytes + j * kMnSliceBytes, &tma_a, m0 + 64 * j, k0, &full_bar[s]);
            } else {
                tma_load_2d(a_s + s * kABytes, &tma_a, k0, m0, &full_bar[s]);
            }
            if (BMN) {
#pragma unroll
                for (int j = 0; j < BN / 64; ++j)
                    tma_load_2d(b_s + s * kBBytes + j * kMnSliceBytes, &tma_b, n0 + 64 * j, k0, &full_bar[s]);
            } else {
                tma_load_2d(b_s + s * kBBytes, &tma_b, k0, n0, &full_bar[s]);
            }
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = instr_desc(BM, BN, AMN, BMN);
        for (int i = 0; i < n_kb; ++i) {
            const int s = i % NST;
            const uint32_t ph = (uint32_t)(i / NST) & 1u;
            if (!mbar_wait(&full_bar[s], ph)) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(a_s + s * kABytes), b0 = smem_u32(b_s + s * kBBytes);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
                mma_bf16(tmem, smem_desc(a0 + kstep_offset(k, AMN), AMN), smem_desc(b0 + kstep_offset(k, BMN), BMN),
                         idesc, (i > 0 || k > 0) ? 1u : 0u);
            mma_commit(&empty_bar[s]);
        }
        // tracks every MMA issued above, even after a timeout
        mma_commit(&accum_bar);
    }
    __syncwarp();

    // epilogue
    bool ready = n_kb > 0 && mbar_wait(&accum_bar, 0);
    if (!ready && n_kb > 0) failed = true;
    // tcgen05.ld is warp-collective: a warp reads TMEM only if all its lanes may
    ready = __all_sync(0xFFFFFFFFu, ready);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    if (ready) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(taddr + (uint32_t)c0, v);
            const int col0 = n0 + c0;
            if (row >= g.m_valid) continue;
            if (EPI == EPI_F32 || EPI == EPI_F32_ATOMIC) {
                float *dst = g.c32 + (size_t)row * g.N + col0;
                if (g.bias) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] += g.bias[col0 + j];
                }
                if (EPI == EPI_F32) {
                    // two 32-byte stores: each a full sector of the lane's row
#pragma unroll
                    for (int j = 0; j < 16; j += 8) {
                        uint32_t w[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) w[q] = __float_as_uint(v[j + q]);
                        st_global_32b(dst + j, w);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        atomicAdd(reinterpret_cast<float4 *>(dst + j), make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]));
                }
            } else if (EPI == EPI_BIAS_RELU || EPI == EPI_RELU_GRAD) {
                __align__(16) __nv_bfloat16 h[16];
                if (EPI == EPI_RELU_GRAD) {
                    __align__(16) __nv_bfloat16 a[16];
                    const uint4 *src = reinterpret_cast<const uint4 *>(g.act + (size_t)row * g.N + col0);
                    *reinterpret_cast<uint4 *>(a) = src[0];
                    *reinterpret_cast<uint4 *>(a + 8) = src[1];
#pragma unroll
                    for (int j = 0; j < 16; ++j) h[j] = __float2bfloat16_rn(__bfloat162float(a[j]) > 0.0f ? v[j] : 0.0f);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        h[j] = __float2bfloat16_rn(fmaxf(v[j] + (g.bias ? g.bias[col0 + j] : 0.0f), 0.0f));
                }
                st_global_32b(g.c16 + (size_t)row * g.N + col0, *reinterpret_cast<const uint32_t(*)[8]>(h));
            }
        }
    }
    if (failed && g.error) atomicExch(g.error, 1u);
    // a producer that gave up may still have copies in flight: wait for them
    if (warp == 0 && lane == 0 && failed) {
        for (int i = (issued > NST ? issued - NST : 0); i < issued; ++i)
            mbar_wait(&full_bar[i % NST], (uint32_t)(i / NST) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

// Persistent form of k_gemm for large fp32-output problems (EPI_F32, both
// operands K-major, 128 x 256 tiles): one CTA per SM walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  The TMA ring and its phases run on
// across tiles, and two TMEM accumulators of 256 columns let the epilogue of
// one tile overlap the MMAs of the next, so the tensor pipe does not wait for
// per-CTA set-up or for the epilogue.
//   warp 0 lane 0   TMA producer
//   warp 1 lane 0   MMA issuer
//   warps 2-5       epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows)
constexpr int PG_BN = 256;
constexpr int PG_THREADS = 6 * 32;

template <int NST = STAGES>
constexpr size_t gemm_persistent_smem_bytes()
{
    return (size_t)NST * ((size_t)BM * BK * 2 + (size_t)PG_BN * BK * 2) + 1024;
}

template <int NST = STAGES>
__global__ void __launch_bounds__(PG_THREADS, 1) k_gemm_persistent(const __grid_constant__ CUtensorMap tma_a,
                                                                 const __grid_constant__ CUtensorMap tma_b,
                                                                 const GemmArgs g)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], acc_full[2], acc_empty[2], drain;
    __shared__ uint32_t tmem_base;
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t kABytes = BM * BK * 2, kBBytes = PG_BN * BK * 2;
    unsigned char *a_s = smem;
    unsigned char *b_s = smem + NST * kABytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles_n = g.N / PG_BN;
    const int n_tiles = (g.M / BM) * n_tiles_n;
    const int n_kb = g.K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
        }
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2u * PG_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool failed = false;

    if (warp == 0) {
        if (lane == 0) {
            int i = 0, issued = 0;
            for (int t = blockIdx.x; t < n_tiles && !failed; t += gridDim.x) {
                const int m0 = (t / n_tiles_n) * BM, n0 = (t % n_tiles_n) * PG_BN;
                for (int kb = 0; kb < n_kb; ++kb, ++i) {
                    const int s = i % NST;
                    if (!mbar_wait(&empty_bar[s], ((uint32_t)(i / NST) & 1u) ^ 1u)) {
                        failed = true;
                        break;
                    }
                    mbar_expect_tx(&full_bar[s], kABytes + kBBytes);
                    tma_load_2d(a_s + s * kABytes, &tma_a, kb * BK, m0, &full_bar[s]);
                    tma_load_2d(b_s + s * kBBytes, &tma_b, kb * BK, n0, &full_bar[s]);
                    ++issued;
                }
            }
            // copies still in flight after a timeout land before the CTA exits
            if (failed)
                for (int q = (issued > NST ? issued - NST : 0); q < issued; ++q)
                    mbar_wait(&full_bar[q % NST], (uint32_t)(q / NST) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(BM, PG_BN);
            int i = 0, j = 0;
            for (int t = blockIdx.x; t < n_tiles && !failed; t += gridDim.x, ++j) {
                const int b = j & 1;
                if (!mbar_wait(&acc_empty[b], ((uint32_t)(j >> 1) & 1u) ^ 1u)) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * PG_BN);
                for (int kb = 0; kb < n_kb; ++kb, ++i) {
                    const int s = i % NST;
                    if (!mbar_wait(&full_bar[s], (uint32_t)(i / NST) & 1u)) {
                        failed = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(a_s + s * kABytes), b0 = smem_u32(b_s + s * kBBytes);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        mma_bf16(d, smem_desc(a0 + 32u * k), smem_desc(b0 + 32u * k), idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    mma_commit(&empty_bar[s]);
                }
                if (failed) break;
                mma_commit(&acc_full[b]);
            }
            // every MMA issued above completes before the CTA frees TMEM
            mma_commit(&drain);
            mbar_wait(&drain, 0);
        }
    } else {
        // epilogue: warp w owns TMEM lanes 32 (w % 4) .. and those rows of each tile
        const int q = warp & 3;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int j = 0;
        for (int t = blockIdx.x; t < n_tiles && !failed; t += gridDim.x, ++j) {
            const int b = j & 1;
            bool ok = mbar_wait(&acc_full[b], (uint32_t)(j >> 1) & 1u);
            // tcgen05.ld is warp-collective: a warp reads TMEM only if all its lanes may
            ok = __all_sync(0xFFFFFFFFu, ok);
            if (!ok) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (t / n_tiles_n) * BM, n0 = (t % n_tiles_n) * PG_BN;
            const int row = m0 + q * 32 + lane;
            const uint32_t taddr = tmem + lane_base + (uint32_t)(b * PG_BN);
#pragma unroll 1
            for (int c0 = 0; c0 < PG_BN; c0 += 16) {
                float v[16];
                tmem_ld16(taddr + (uint32_t)c0, v);
                if (row >= g.m_valid) continue;
                float *dst = g.c32 + (size_t)row * g.N + n0 + c0;
#pragma unroll
                for (int h = 0; h < 16; h += 8) {
                    uint32_t w[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) w[e] = __float_as_uint(v[h + e]);
                    st_global_32b(dst + h, w);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(&acc_empty[b]);
        }
    }
    if (failed && g.error) atomicExch(g.error, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * PG_BN) : "memory");
}

}  // namespace umma
}  // namespace hrpp
