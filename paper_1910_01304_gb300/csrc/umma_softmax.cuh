// Fused output layer and softmax cross-entropy of the learned proposal's
// training step, on the tensor cores (tcgen05):
//
//   Z    = H2 W3^T + b3            [rows, 4096], never written to memory
//   loss = log sum_j exp(Z_rj) - Z_r,label        per labelled row
//   dZ   = softmax(Z_r) - onehot(label)           bf16, row-major
//
// One CTA owns 128 rows and computes all 16 column tiles of 256 twice.  The
// first pass keeps each row's running maximum and sum of exponentials; the
// second recomputes each tile and writes the gradient.  The CTA's 128 x 256
// tile of H2 stays in shared memory; W3 streams from L2 in 256 x 64 blocks
// through a 4-stage ring; b3 is copied to shared memory once.  Two TMEM
// accumulators of 256 columns let the epilogue of one tile overlap the MMAs
// of the next.
//   warps 0-15 epilogue: warp w reads TMEM lanes 32(w%4).. (rows) and the
//              64-column slice w/4 of every tile; the four partial row
//              statistics of a row are combined in shared memory after pass 1
//   warp 16    TMA producer (one lane)
//   warp 17    MMA issuer (one lane)
// The prediction mode makes one pass and keeps each row's first maximum
// (argmax over the 4096 classes of Z), writing the class and its treelet node.
// Every mbarrier wait is bounded; a wait that gives up sets the error flag,
// the CTA drains its outstanding copies and MMAs (bounded again), frees its
// TMEM and returns.
#pragma once

#include "umma.cuh"

namespace hrpp {
namespace umma {

constexpr int SX_CLASSES = 4096;
constexpr int SX_K = 256;                       // hidden width
constexpr int SX_BN = 256;                      // columns per tile (one TMEM accumulator)
constexpr int SX_TILES = SX_CLASSES / SX_BN;    // 16 per pass
constexpr int SX_KB = SX_K / BK;                // 4 K blocks per tile
constexpr int SX_NST = 4;                       // W3 ring stages
constexpr uint32_t SX_A_BLOCK = BM * BK * 2;    // 16 KB
constexpr uint32_t SX_A_BYTES = SX_KB * SX_A_BLOCK;
constexpr uint32_t SX_B_BYTES = SX_BN * BK * 2; // 32 KB per stage
constexpr int SX_EPI_WARPS = 16;                // 4 row groups x 4 column slices
constexpr int SX_SLICE = SX_BN / 4;             // columns of a tile per epilogue warp
constexpr int SX_THREADS = (SX_EPI_WARPS + 2) * 32;

template <int NST = SX_NST>
constexpr size_t softmax_smem_bytes()
{
    return (size_t)SX_A_BYTES + (size_t)NST * SX_B_BYTES + SX_CLASSES * sizeof(float) + 1024;
}

struct SoftmaxArgs {
    const float *bias;      // b3 [4096]
    // prediction (PREDICT = true): first argmax per row, and its treelet node
    int32_t *out_classes;   // [n] (may be null)
    int32_t *out_nodes;     // [n] (may be null)
    const int32_t *class_node;  // [4096]
    const int32_t *labels;  // [npad]: class, or -1 for no target (read for rows < n)
    int n;                  // rows >= n are padding (no target)
    int npad;               // rows, a multiple of 128
    __nv_bfloat16 *dz;      // [npad, 4096]
    float *loss_sum;        // += loss of every labelled row
    unsigned int *count;    // += labelled rows
    unsigned int *error;    // set to 1 when a bounded wait gives up
};


// three-input maximum (one instruction); equals fmaxf twice for non-NaN inputs
__device__ __forceinline__ float max3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// v[j] = column j of a 16-column TMEM chunk + bias[j]; bias is in shared
// memory, 16-byte aligned and the same for every lane (a broadcast read)
__device__ __forceinline__ void chunk_plus_bias(const uint32_t (&r)[16], const float *bias, float (&v)[16])
{
    const float4 *b4 = reinterpret_cast<const float4 *>(bias);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 b = b4[j];
        v[4 * j] = __uint_as_float(r[4 * j]) + b.x;
        v[4 * j + 1] = __uint_as_float(r[4 * j + 1]) + b.y;
        v[4 * j + 2] = __uint_as_float(r[4 * j + 2]) + b.z;
        v[4 * j + 3] = __uint_as_float(r[4 * j + 3]) + b.w;
    }
}

// Issues a 16-column TMEM load of the warp's 32 lanes without waiting for it.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Waits for the thread's TMEM loads.  r passes through the instruction, so no
// read of the loaded registers can be scheduled above the wait.
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// Calls f(chunk, c0) on the 16-column chunks of a warp's column slice, in
// ascending order, loading chunk k + 1 while f works on chunk k.
template <typename F>
__device__ __forceinline__ void for_each_chunk(uint32_t taddr, F &&f)
{
    constexpr int kChunks = SX_SLICE / 16;
    static_assert(kChunks % 2 == 0, "chunks go in pairs");
    uint32_t ra[16], rb[16];
    tmem_ld16_issue(taddr, ra);
    tmem_wait16(ra);
#pragma unroll
    for (int k = 0; k < kChunks; k += 2) {
        tmem_ld16_issue(taddr + 16u * (uint32_t)(k + 1), rb);
        f(ra, 16 * k);
        tmem_wait16(rb);
        if (k + 2 < kChunks) tmem_ld16_issue(taddr + 16u * (uint32_t)(k + 2), ra);
        f(rb, 16 * (k + 1));
        if (k + 2 < kChunks) tmem_wait16(ra);
    }
}

// NST: stages of the W3 ring (a template so that every file that includes
// this header shares one instance).  PREDICT: one pass that keeps each row's
// first maximum instead of the two training passes.
template <int NST = SX_NST, bool PREDICT = false>
__global__ void __launch_bounds__(SX_THREADS, 1) k_softmax_xent(const __grid_constant__ CUtensorMap tma_a,
                                                         const __grid_constant__ CUtensorMap tma_b,
                                                         const SoftmaxArgs g)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full, full_bar[NST], empty_bar[NST], acc_full[2], acc_empty[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ float part_m[4][BM], part_s[4][BM], zl[BM];  // per column slice and row
    __shared__ int any_failed;
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *a_s = smem;
    unsigned char *b_s = smem + SX_A_BYTES;
    float *bias_s = reinterpret_cast<float *>(b_s + NST * SX_B_BYTES);  // b3, read by every epilogue warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM;
    constexpr int kTiles = PREDICT ? SX_TILES : 2 * SX_TILES;

    if (threadIdx.x == 0) {
        any_failed = 0;
        mbar_init(&a_full, 1);
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], SX_EPI_WARPS);  // one arrival per epilogue warp
        }
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < SX_CLASSES / 4; i += SX_THREADS)
        reinterpret_cast<float4 *>(bias_s)[i] = __ldg(reinterpret_cast<const float4 *>(g.bias) + i);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2u * SX_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool failed = false;

    if (warp == SX_EPI_WARPS) {
        if (lane == 0) {
            // H2 tile (4 K blocks, 64 KB), then W3 blocks for both passes
            mbar_expect_tx(&a_full, SX_A_BYTES);
            for (int kb = 0; kb < SX_KB; ++kb) tma_load_2d(a_s + kb * SX_A_BLOCK, &tma_a, kb * BK, m0, &a_full);
            int issued = 0;
            for (int i = 0; i < kTiles * SX_KB; ++i) {
                const int t = i / SX_KB, kb = i % SX_KB, s = i % NST;
                if (!mbar_wait(&empty_bar[s], ((uint32_t)(i / NST) & 1u) ^ 1u)) {
                    failed = true;
                    break;
                }
                mbar_expect_tx(&full_bar[s], SX_B_BYTES);
                tma_load_2d(b_s + s * SX_B_BYTES, &tma_b, kb * BK, (t % SX_TILES) * SX_BN, &full_bar[s]);
                ++issued;
            }
            // copies still in flight after a timeout land before the CTA exits
            mbar_wait(&a_full, 0);
            if (failed)
                for (int i = (issued > NST ? issued - NST : 0); i < issued; ++i)
                    mbar_wait(&full_bar[i % NST], (uint32_t)(i / NST) & 1u);
        }
    } else if (warp == SX_EPI_WARPS + 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(BM, SX_BN);
            if (!mbar_wait(&a_full, 0)) failed = true;
            int i = 0;
            for (int t = 0; t < kTiles && !failed; ++t) {
                const int b = t & 1;
                if (!mbar_wait(&acc_empty[b], ((uint32_t)(t >> 1) & 1u) ^ 1u)) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * SX_BN);
                for (int kb = 0; kb < SX_KB; ++kb, ++i) {
                    const int s = i % NST;
                    if (!mbar_wait(&full_bar[s], (uint32_t)(i / NST) & 1u)) {
                        failed = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(a_s + kb * SX_A_BLOCK), b0 = smem_u32(b_s + s * SX_B_BYTES);
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
        // epilogue: row group q (TMEM lanes 32q..), column slice cs of each tile
        const int q = warp & 3, cs = warp >> 2;
        const int r = q * 32 + lane;
        const int row = m0 + r;
        int lab = (!PREDICT && row < g.n) ? g.labels[row] : -1;
        if (lab >= SX_CLASSES) lab = -1;
        float m = -__int_as_float(0x7F800000), ssum = 0.0f, inv = 0.0f;
        int best = 0;  // PREDICT: this slice's first maximum
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        // pass 1: running maximum and sum of exponentials over this slice
        for (int t = 0; t < SX_TILES; ++t) {
            const int b = t & 1;
            bool ok = mbar_wait(&acc_full[b], (uint32_t)(t >> 1) & 1u);
            // tcgen05.ld is warp-collective: a warp reads TMEM only if all its lanes may
            ok = __all_sync(0xFFFFFFFFu, ok);
            if (!ok) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr = tmem + lane_base + (uint32_t)(b * SX_BN + cs * SX_SLICE);
            const int col0 = t * SX_BN + cs * SX_SLICE;
            for_each_chunk(taddr, [&](const uint32_t(&rc)[16], int c0) {
                float v[16];
                chunk_plus_bias(rc, bias_s + col0 + c0, v);
                if (PREDICT) {
                    // first maximum: columns arrive in ascending order
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (v[j] > m) {
                            m = v[j];
                            best = col0 + c0 + j;
                        }
                    }
                    return;
                }
                // the row's label logit, when its column is in this chunk
                const uint32_t off = (uint32_t)(lab - (col0 + c0));
                if (off < 16u) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if ((uint32_t)j == off) zl[r] = v[j];
                }
                float cm = m;
#pragma unroll
                for (int j = 0; j < 16; j += 2) cm = max3(cm, v[j], v[j + 1]);
                float acc = 0.0f;
#pragma unroll
                for (int j = 0; j < 16; ++j) acc += __expf(v[j] - cm);
                ssum = ssum * __expf(m - cm) + acc;
                m = cm;
            });
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(&acc_empty[b]);
        }
        // combine the four slices' statistics of each row; every epilogue warp
        // reaches this barrier once, also after a failed wait
        part_m[cs][r] = m;
        part_s[cs][r] = PREDICT ? __int_as_float(best) : ssum;
        if (failed) any_failed = 1;
        asm volatile("bar.sync 1, %0;" ::"n"(SX_EPI_WARPS * 32) : "memory");
        if (any_failed) failed = true;
        if (PREDICT) {
            // the row's first maximum: slices hold ascending column ranges
            if (!failed && cs == 0 && row < g.n) {
                float bm = part_m[0][r];
                int bc = __float_as_int(part_s[0][r]);
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    const float z = part_m[k][r];
                    const int c = __float_as_int(part_s[k][r]);
                    if (z > bm || (z == bm && c < bc)) {
                        bm = z;
                        bc = c;
                    }
                }
                if (g.out_classes) g.out_classes[row] = bc;
                if (g.out_nodes) g.out_nodes[row] = g.class_node[bc];
            }
        } else if (!failed) {
            m = fmaxf(fmaxf(part_m[0][r], part_m[1][r]), fmaxf(part_m[2][r], part_m[3][r]));
            ssum = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) ssum += part_s[k][r] * __expf(part_m[k][r] - m);
            inv = lab >= 0 ? 1.0f / ssum : 0.0f;
            if (cs == 0 && lab >= 0) {
                atomicAdd(g.loss_sum, logf(ssum) + m - zl[r]);
                atomicAdd(g.count, 1u);
            }
        }
        // pass 2: dZ = softmax - onehot (zero for rows without a target)
        for (int t = SX_TILES; !PREDICT && t < kTiles && !failed; ++t) {
            const int b = t & 1;
            bool ok = mbar_wait(&acc_full[b], (uint32_t)(t >> 1) & 1u);
            ok = __all_sync(0xFFFFFFFFu, ok);
            if (!ok) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr = tmem + lane_base + (uint32_t)(b * SX_BN + cs * SX_SLICE);
            const int col0 = (t - SX_TILES) * SX_BN + cs * SX_SLICE;
            for_each_chunk(taddr, [&](const uint32_t(&rc)[16], int c0) {
                float v[16];
                chunk_plus_bias(rc, bias_s + col0 + c0, v);
                // softmax (zero for rows without a target: inv = 0), minus
                // the one-hot of the label when its column is in this chunk
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __expf(v[j] - m) * inv;
                const uint32_t off = (uint32_t)(lab - (col0 + c0));
                if (off < 16u) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if ((uint32_t)j == off) v[j] -= 1.0f;
                }
                uint32_t w[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    w[j] = *reinterpret_cast<const uint32_t *>(&h);
                }
                // dZ: the lane's row, one 32-byte store (one full sector)
                st_global_32b(g.dz + (size_t)row * SX_CLASSES + col0 + c0, w);
            });
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(&acc_empty[b]);
        }
    }
    if (failed && g.error) atomicExch(g.error, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * SX_BN) : "memory");
}

}  // namespace umma
}  // namespace hrpp
