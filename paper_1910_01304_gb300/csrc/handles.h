// Internal definitions of the library's opaque handles, shared by the host
// translation units (api.cu, noalloc.cu).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>

#include "hrpp.h"

namespace hrpp {
// Host-side fault injection for tests: while the environment holds
// HRPP_FAIL_ALLOC_AFTER=N, every device allocation after the first N made
// since that value was set is refused (true: fail it, allocate nothing).
// device_malloc (every object-creating entry point) and hrpp_trace's per-call
// scratch consult it; hrpp_trace_noalloc allocates nothing and never does.
bool allocation_refused();
// cudaMalloc unless allocation_refused(), then cudaErrorMemoryAllocation.
cudaError_t device_malloc(void **ptr, size_t bytes);

// Names an entry point's host-side span in profiler timelines (NVTX; a no-op
// unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace hrpp

struct hrpp_scene {
    int device;
    uint64_t id;
    int width;
    uint32_t n_tris, n_interior, n_leaves, max_depth;
    int32_t root_ref;
    float4 *d_nodes;
    float4 *d_tris;
    uint32_t *d_error;
    int32_t *d_parent;       // per interior node (preorder index): its parent, -1 at the root
    int32_t *d_leaf_parent;  // per prim_index slot starting a leaf: the leaf's parent, else -1
    int32_t *d_canon_ref;    // per canonical node: its device ref (interior index or ~leaf), or empty
    uint32_t n_nodes;        // canonical node count
    uint64_t bytes;
};

struct hrpp_table {
    int device;
    int log2_entries, log2_ways, log2_sets;
    int precision, update_mode;
    int go_up;
    int hash_variant;  // HRPP_HASH_EXP_MSB or HRPP_HASH_EXP_LSB
    uint64_t *d_words;
    uint32_t *d_winner;
    uint32_t *d_gate;       // the gate word (nonzero = open), stored right after the table words
    uint32_t gate_min_tp;   // 0: no gate; else true positives per 65536 lookups that keep it open
    int gate_sample_log2;   // closed: every 2^s-th 32-ray chunk still consults the table
    uint64_t bound_scene;
};

namespace hrpp {
// Stores `message` as the calling thread's hrpp_last_error() text; returns s.
hrpp_status report(hrpp_status s, const char *message);
}  // namespace hrpp
