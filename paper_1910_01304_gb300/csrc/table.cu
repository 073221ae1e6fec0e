// Predictor table maintenance kernels.
#include <cuda_runtime.h>

#include "device.cuh"

namespace hrpp {

// Two-phase update, after the batch: each slot takes the word of the record
// with the highest ray index aimed at it (its index + 1 is in winner[slot]).
// The winning record writes the word and zeroes winner[slot] for the next
// call; a losing record reads either the winner's index or zero, never its
// own, so the outcome does not depend on scheduling.  The slot's old word
// (wanted only by the winner, for the eviction count) is read beside the
// winner index, so each record waits on two dependent loads, not three.
__device__ __forceinline__ void apply_records(uint64_t *table, uint32_t *winner, const Record *rec, Ctl *ctl,
                                              uint32_t max_records)
{
    const uint32_t n = min(ctl->n_records, max_records);
    uint32_t evict = 0, lost = 0;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const Record x = rec[r];
        const uint32_t w = __ldcg(winner + x.slot);
        const uint64_t old = __ldcg(reinterpret_cast<const unsigned long long *>(table) + x.slot);
        if (w == x.ray1) {
            table[x.slot] = x.word;
            winner[x.slot] = 0u;
            evict += old != HRPP_EMPTY_WORD;
        } else {
            ++lost;
        }
    }
    evict = __reduce_add_sync(0xFFFFFFFFu, evict);
    lost = __reduce_add_sync(0xFFFFFFFFu, lost);
    if ((threadIdx.x & 31u) == 0) {
        if (evict) atomicAdd(&ctl->stats[ST_EVICTIONS], (unsigned long long)evict);
        if (lost) atomicAdd(&ctl->stats[ST_DUP_INSERTS], (unsigned long long)lost);
    }
}

// The gate's decision reads only the call's counts, never the records, so
// the first thread of the grid takes it while the others apply records.
__global__ void __launch_bounds__(256) k_apply(uint64_t *table, uint32_t *winner, const Record *rec, Ctl *ctl,
                                               uint32_t max_records, uint32_t *gate, uint32_t gate_min_tp)
{
    if (gate && blockIdx.x == 0 && threadIdx.x == 0) gate_decide(gate, gate_min_tp, ctl);
    apply_records(table, winner, rec, ctl, max_records);
}

__global__ void k_gate(uint32_t *gate, uint32_t gate_min_tp, const Ctl *ctl)
{
    gate_decide(gate, gate_min_tp, ctl);
}

// one grid row per item of a batch (blockIdx.y)
__global__ void __launch_bounds__(256) k_apply_batch(const TraceParams *items, uint32_t max_records)
{
    const TraceParams &p = items[blockIdx.y];
    if (p.gate && blockIdx.x == 0 && threadIdx.x == 0) gate_decide(p.gate, p.gate_min_tp, p.ctl);
    if (!p.table || p.update_mode != HRPP_UPDATE_TWO_PHASE) return;
    apply_records(p.table, p.winner, p.records, p.ctl, min(max_records, p.n_rays));
}

__global__ void __launch_bounds__(256) k_fill(uint64_t *words, uint64_t n)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        words[i] = HRPP_EMPTY_WORD;
}

cudaError_t launch_table_apply(uint64_t *table, uint32_t *winner, const Record *records, Ctl *ctl,
                               uint32_t max_records, cudaStream_t stream, uint32_t *gate, uint32_t gate_min_tp)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // one record per thread while they last: the update is a chain of
    // dependent random reads, so it wants every resident warp in flight
    uint32_t blocks = (max_records + 255u) / 256u;
    if (blocks > (uint32_t)sms * 16u) blocks = (uint32_t)sms * 16u;
    if (blocks < 1) blocks = 1;
    k_apply<<<blocks, 256, 0, stream>>>(table, winner, records, ctl, max_records, gate, gate_min_tp);
    return cudaGetLastError();
}

cudaError_t launch_gate_update(uint32_t *gate, uint32_t gate_min_tp, const Ctl *ctl, cudaStream_t stream)
{
    k_gate<<<1, 1, 0, stream>>>(gate, gate_min_tp, ctl);
    return cudaGetLastError();
}

cudaError_t launch_table_apply_batch(const TraceParams *items, uint32_t n_items, uint32_t max_records,
                                     cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // the items share the resident warps of the single-call grid, 64 blocks each at least
    uint32_t cap = n_items ? (uint32_t)sms * 16u / n_items : 64u;
    if (cap < 64u) cap = 64u;
    uint32_t bx = (max_records + 255u) / 256u;
    if (bx > cap) bx = cap;
    if (bx < 1u) bx = 1u;
    k_apply_batch<<<dim3(bx, n_items), 256, 0, stream>>>(items, max_records);
    return cudaGetLastError();
}

cudaError_t launch_table_fill(uint64_t *words, uint64_t n_words, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (n_words + 255u) / 256u;
    if (blocks > (uint64_t)sms * 8u) blocks = (uint64_t)sms * 8u;
    if (blocks < 1) blocks = 1;
    k_fill<<<(unsigned)blocks, 256, 0, stream>>>(words, n_words);
    return cudaGetLastError();
}

}  // namespace hrpp
