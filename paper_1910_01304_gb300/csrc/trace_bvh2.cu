// Traversal kernels over binary BVHs (64-byte nodes holding both child boxes).
#include "compact.cuh"
#include "trace_kernel.cuh"

namespace hrpp {

cudaError_t launch_trace_w2(bool closest, bool stats, int schedule, const TraceParams &p, int block_threads, int blocks_per_sm_cap,
                            cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1, const L2Window *l2)
{
    return launch_width<2>(closest, stats, schedule, p, block_threads, blocks_per_sm_cap, stream, ev0, ev1, l2);
}

cudaError_t launch_batch_w2(bool closest, bool stats, const BatchDesc &b, int block_threads, cudaStream_t stream)
{
    return launch_batch_width<2>(closest, stats, b, block_threads, stream);
}

cudaError_t launch_compact_w2(bool closest, bool stats, const TraceParams &p, void *queue, int block_threads,
                              cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1)
{
    return launch_compact_width<2>(closest, stats, p, static_cast<QueueEntry *>(queue), block_threads, stream, ev0,
                                    ev1);
}

}  // namespace hrpp
