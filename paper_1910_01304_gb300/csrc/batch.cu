// Batched traces: many (scene, table, rays) items in one persistent launch
// per query mode (the two launches run side by side), captured once into a
// CUDA graph and replayed by hrpp_batch_run.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "handles.h"
#include "hrpp.h"

using namespace hrpp;

struct hrpp_batch {
    int device;
    int width;
    uint32_t n_items;
    bool stats;
    uint32_t block_threads;
    TraceParams *d_items;
    unsigned char *d_ctl;       // [cursors: 256 B][item 0 Ctl: 256 B]...[item n-1 Ctl]
    size_t ctl_bytes;
    Record *d_records;
    uint32_t *d_chunk_item, *d_chunk_first;
    uint32_t n_chunks;
    uint32_t n_closest_chunks;  // chunks of closest-hit items come first
    cudaStream_t capture_stream, side_stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaStream_t last_stream;
};

namespace {

hrpp_status bfail(hrpp_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return hrpp::report(s, buf);
}

bool on_device(const void *ptr, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

void release(hrpp_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->side_stream) cudaStreamDestroy(b->side_stream);
    cudaFree(b->d_items);
    cudaFree(b->d_ctl);
    cudaFree(b->d_records);
    cudaFree(b->d_chunk_item);
    cudaFree(b->d_chunk_first);
    delete b;
}

}  // namespace

extern "C" {

hrpp_status hrpp_batch_create(const hrpp_batch_item *items, uint32_t n_items, int collect_stats,
                              uint32_t block_threads, hrpp_batch **out)
{
    if (!out) return bfail(HRPP_ERR_INVALID_ARG, "out is NULL");
    if (!items || n_items == 0) return bfail(HRPP_ERR_INVALID_ARG, "no items");
    if (n_items > 65535u) return bfail(HRPP_ERR_UNSUPPORTED, "at most 65535 items per batch");
    if (block_threads == 0) block_threads = 128;
    if (block_threads != 64 && block_threads != 128 && block_threads != 256 && block_threads != 512)
        return bfail(HRPP_ERR_INVALID_ARG, "block_threads must be 64, 128, 256 or 512");
    const hrpp_scene *s0 = items[0].scene;
    if (!s0) return bfail(HRPP_ERR_INVALID_ARG, "item 0 has no scene");
    uint64_t total_chunks = 0;
    uint64_t total_records = 0;
    for (uint32_t k = 0; k < n_items; ++k) {
        const hrpp_batch_item &it = items[k];
        if (!it.scene) return bfail(HRPP_ERR_INVALID_ARG, "item %u has no scene", k);
        if (it.scene->device != s0->device || it.scene->width != s0->width)
            return bfail(HRPP_ERR_INVALID_ARG, "item %u: every scene of a batch must share one device and BVH width", k);
        if (it.mode != HRPP_ANY_HIT && it.mode != HRPP_CLOSEST_HIT) return bfail(HRPP_ERR_INVALID_ARG, "item %u: mode", k);
        if (it.n_rays > (1u << 31)) return bfail(HRPP_ERR_UNSUPPORTED, "item %u: more than 2^31 rays", k);
        if (it.n_rays && (!it.rays || !it.out_hits)) return bfail(HRPP_ERR_INVALID_ARG, "item %u: NULL buffer", k);
        if (((uintptr_t)it.rays & 15u) || ((uintptr_t)it.out_hits & (it.mode == HRPP_CLOSEST_HIT ? 15u : 3u)))
            return bfail(HRPP_ERR_INVALID_ARG, "item %u: misaligned buffer", k);
        if (it.n_rays && (!on_device(it.rays, s0->device) || !on_device(it.out_hits, s0->device)))
            return bfail(HRPP_ERR_INVALID_ARG, "item %u: rays and hits must be device memory of the scene's device", k);
        if (it.table) {
            if (it.table->device != s0->device) return bfail(HRPP_ERR_INVALID_ARG, "item %u: table on another device", k);
            if (it.table->bound_scene && it.table->bound_scene != it.scene->id)
                return bfail(HRPP_ERR_INVALID_ARG, "item %u: table bound to another scene; reset it first", k);
            for (uint32_t q = 0; q < k; ++q)
                if (items[q].table == it.table)
                    return bfail(HRPP_ERR_INVALID_ARG, "items %u and %u share a table; a table may serve one item", q, k);
            if (it.table->update_mode == HRPP_UPDATE_TWO_PHASE) total_records += it.n_rays;
        }
        total_chunks += (it.n_rays + 31u) / 32u;
    }
    if (total_chunks > 0xFFFFFFF0ull) return bfail(HRPP_ERR_UNSUPPORTED, "too many rays in one batch");

    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return bfail(HRPP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (prev != s0->device && (e = cudaSetDevice(s0->device)) != cudaSuccess)
        return bfail(HRPP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));

    hrpp_batch *b = new (std::nothrow) hrpp_batch;
    if (!b) return bfail(HRPP_ERR_OOM, "host allocation");
    memset(b, 0, sizeof *b);
    b->device = s0->device;
    b->width = s0->width;
    b->n_items = n_items;
    b->stats = collect_stats != 0;
    b->block_threads = block_threads;
    b->n_chunks = (uint32_t)total_chunks;
    b->ctl_bytes = 256ull * (n_items + 1);
    hrpp_status status = HRPP_OK;
    do {
        if ((e = hrpp::device_malloc((void **)&b->d_items, sizeof(TraceParams) * n_items)) != cudaSuccess ||
            (e = hrpp::device_malloc((void **)&b->d_ctl, b->ctl_bytes)) != cudaSuccess ||
            (e = hrpp::device_malloc((void **)&b->d_records, sizeof(Record) * (total_records ? total_records : 1))) != cudaSuccess ||
            (e = hrpp::device_malloc((void **)&b->d_chunk_item, sizeof(uint32_t) * (total_chunks ? total_chunks : 1))) != cudaSuccess ||
            (e = hrpp::device_malloc((void **)&b->d_chunk_first, sizeof(uint32_t) * (total_chunks ? total_chunks : 1))) != cudaSuccess) {
            status = bfail(e == cudaErrorMemoryAllocation ? HRPP_ERR_OOM : HRPP_ERR_CUDA, "batch allocation: %s",
                           cudaGetErrorString(e));
            break;
        }
        std::vector<TraceParams> h(n_items);
        std::vector<uint32_t> chunk_item, chunk_first;
        chunk_item.reserve(total_chunks);
        chunk_first.reserve(total_chunks);
        uint64_t rec_off = 0;
        uint32_t max_n = 0;
        bool any_gate = false;  // some item's table has a gate: k_apply_batch decides it
        std::vector<uint32_t> any_item, any_first;  // appended after the closest-hit chunks
        for (uint32_t k = 0; k < n_items; ++k) {
            const hrpp_batch_item &it = items[k];
            const hrpp_scene *sc = it.scene;
            TraceParams &p = h[k];
            memset(&p, 0, sizeof p);
            p.nodes = sc->d_nodes;
            p.tris = sc->d_tris;
            p.n_tris = sc->n_tris;
            p.root_ref = sc->root_ref;
            p.max_steps = sc->n_interior + sc->n_leaves + 8u;
            p.rays = reinterpret_cast<const float4 *>(it.rays);
            p.n_rays = it.n_rays;
            p.hits = it.out_hits;
            p.ctl = reinterpret_cast<Ctl *>(b->d_ctl + 256ull * (k + 1));
            p.error = sc->d_error;
            p.refill_min = 16;
            p.n_interior = sc->n_interior;
            p.parent = sc->d_parent;
            p.leaf_parent = sc->d_leaf_parent;
            p.closest = it.mode == HRPP_CLOSEST_HIT;
            if (it.table) {
                p.table = it.table->d_words;
                p.winner = it.table->d_winner;
                p.log2_sets = it.table->log2_sets;
                p.log2_ways = it.table->log2_ways;
                p.precision = it.table->precision;
                p.update_mode = it.table->update_mode;
                p.go_up = it.table->go_up;
                p.hash_variant = it.table->hash_variant;
                if (it.table->gate_min_tp) {
                    p.gate = it.table->d_gate;
                    p.gate_mask = (1u << it.table->gate_sample_log2) - 1u;
                    p.gate_min_tp = it.table->gate_min_tp;
                    any_gate = true;
                }
                if (it.table->update_mode == HRPP_UPDATE_TWO_PHASE) {
                    p.records = b->d_records + rec_off;
                    rec_off += it.n_rays;
                }
                it.table->bound_scene = sc->id;
            }
            if (it.n_rays > max_n) max_n = it.n_rays;
            for (uint32_t c = 0; c < (it.n_rays + 31u) / 32u; ++c) {
                (p.closest ? chunk_item : any_item).push_back(k);
                (p.closest ? chunk_first : any_first).push_back(32u * c);
            }
        }
        b->n_closest_chunks = (uint32_t)chunk_item.size();
        chunk_item.insert(chunk_item.end(), any_item.begin(), any_item.end());
        chunk_first.insert(chunk_first.end(), any_first.begin(), any_first.end());
        if ((e = cudaMemcpy(b->d_items, h.data(), sizeof(TraceParams) * n_items, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (total_chunks &&
             ((e = cudaMemcpy(b->d_chunk_item, chunk_item.data(), 4 * total_chunks, cudaMemcpyHostToDevice)) != cudaSuccess ||
              (e = cudaMemcpy(b->d_chunk_first, chunk_first.data(), 4 * total_chunks, cudaMemcpyHostToDevice)) != cudaSuccess)) ||
            (e = cudaMemset(b->d_ctl, 0, b->ctl_bytes)) != cudaSuccess) {
            status = bfail(HRPP_ERR_CUDA, "batch upload: %s", cudaGetErrorString(e));
            break;
        }
        // capture: zero the cursors and item control blocks; trace the
        // closest-hit items on the capture stream and the any-hit items on a
        // side stream, so the two launches overlap; then apply every
        // two-phase table's inserts
        if ((e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&b->side_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            status = bfail(HRPP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
            break;
        }
        const uint32_t n_any = b->n_chunks - b->n_closest_chunks;
        BatchDesc dc, da;
        dc.items = da.items = b->d_items;
        dc.chunk_item = b->d_chunk_item;
        dc.chunk_first = b->d_chunk_first;
        dc.n_chunks = b->n_closest_chunks;
        dc.cursor = reinterpret_cast<unsigned int *>(b->d_ctl);
        da.chunk_item = b->d_chunk_item + b->n_closest_chunks;
        da.chunk_first = b->d_chunk_first + b->n_closest_chunks;
        da.n_chunks = n_any;
        da.cursor = reinterpret_cast<unsigned int *>(b->d_ctl) + 1;
        cudaEvent_t fork = nullptr, join = nullptr;
        cudaError_t ec = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (ec == cudaSuccess) ec = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        if (ec == cudaSuccess) ec = cudaMemsetAsync(b->d_ctl, 0, b->ctl_bytes, b->capture_stream);
        const bool both = dc.n_chunks && da.n_chunks;
        if (ec == cudaSuccess && both) ec = cudaEventRecord(fork, b->capture_stream);
        if (ec == cudaSuccess && both) ec = cudaStreamWaitEvent(b->side_stream, fork, 0);
        if (ec == cudaSuccess && dc.n_chunks)
            ec = b->width == 2 ? launch_batch_w2(true, b->stats, dc, (int)block_threads, b->capture_stream)
                               : launch_batch_w4(true, b->stats, dc, (int)block_threads, b->capture_stream);
        cudaStream_t any_stream = both ? b->side_stream : b->capture_stream;
        if (ec == cudaSuccess && da.n_chunks)
            ec = b->width == 2 ? launch_batch_w2(false, b->stats, da, (int)block_threads, any_stream)
                               : launch_batch_w4(false, b->stats, da, (int)block_threads, any_stream);
        if (ec == cudaSuccess && both) ec = cudaEventRecord(join, b->side_stream);
        if (ec == cudaSuccess && both) ec = cudaStreamWaitEvent(b->capture_stream, join, 0);
        if (ec == cudaSuccess && (total_records || any_gate))
            ec = launch_table_apply_batch(b->d_items, n_items, max_n, b->capture_stream);
        e = cudaStreamEndCapture(b->capture_stream, &b->graph);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (ec != cudaSuccess || e != cudaSuccess) {
            status = bfail(HRPP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec != cudaSuccess ? ec : e));
            break;
        }
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
            status = bfail(HRPP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            break;
        }
    } while (false);
    int cur = -1;
    if (status != HRPP_OK) {
        release(b);
        b = nullptr;
    }
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    if (status == HRPP_OK) *out = b;
    return status;
}

hrpp_status hrpp_batch_run(hrpp_batch *b, void *stream)
{
    hrpp::NvtxRange nvtx_range("hrpp_batch_run");
    if (!b) return bfail(HRPP_ERR_INVALID_ARG, "batch is NULL");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != b->device) e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    b->last_stream = (cudaStream_t)stream;
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(HRPP_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return HRPP_OK;
}

hrpp_status hrpp_batch_get_stats(hrpp_batch *b, uint32_t item, hrpp_stats *host_stats)
{
    if (!b || !host_stats) return bfail(HRPP_ERR_INVALID_ARG, "NULL argument");
    if (item >= b->n_items) return bfail(HRPP_ERR_INVALID_ARG, "item %u out of range", item);
    if (!b->stats) return bfail(HRPP_ERR_INVALID_ARG, "the batch was created without statistics");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != b->device) e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->last_stream);
    if (e == cudaSuccess) {
        const Ctl *ctl = reinterpret_cast<const Ctl *>(b->d_ctl + 256ull * (item + 1));
        e = cudaMemcpy(host_stats, ctl->stats, sizeof(hrpp_stats), cudaMemcpyDeviceToHost);
    }
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(HRPP_ERR_CUDA, "reading batch stats: %s", cudaGetErrorString(e));
    return HRPP_OK;
}

void hrpp_batch_destroy(hrpp_batch *b)
{
    if (!b) return;
    int prev = -1, cur = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    release(b);
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

}  // extern "C"
