// hrpp_trace_noalloc: hrpp_trace for callers that must not allocate memory.
//
// hrpp_trace takes its per-call scratch (the ray pool cursor, the statistics
// block and, for two-phase tables, one 16-byte insert record per ray) from a
// stream-ordered memory pool.  Some callers cannot allow that: an engine that
// reserved all device memory for its own allocator at start-up (so any
// further cudaMalloc would fail), or a real-time frame loop that forbids
// allocation calls because they can stall or synchronise the device at an
// unpredictable moment.  This entry point runs the same kernels with the
// scratch taken from one fixed array in device memory that is part of the
// library image, so it never allocates.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "device.cuh"
#include "handles.h"
#include "hrpp.h"

using namespace hrpp;

// Library-owned scratch: the control block followed by the insert records of
// up to HRPP_NOALLOC_MAX_RAYS rays.  Every device that loads the library holds
// this array until the process exits.
constexpr size_t kNoallocCtlBytes = 256;
constexpr size_t kNoallocBytes = kNoallocCtlBytes + (size_t)HRPP_NOALLOC_MAX_RAYS * sizeof(Record);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[64] = {};  // device address of the array, per device

hrpp_status noalloc_fail(hrpp_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return hrpp::report(s, buf);
}

// Device address of the scratch array on the current device.  Host code only
// sees a host-side stand-in under the array's name, so the address has to be
// asked for once per device, with that device current.  The cached address
// lives as long as the device's context: cudaDeviceReset ends the context
// (and with it every scene and table of this library), so the library is
// not used across a reset.
cudaError_t scratch_on(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

bool device_pointer(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" hrpp_status hrpp_trace_noalloc(const hrpp_scene *sc, hrpp_table *table, const hrpp_ray *rays,
                                          uint32_t n_rays, hrpp_mode mode, void *out_hits, hrpp_stats *out_stats,
                                          void *stream_)
{
    hrpp::NvtxRange nvtx_range("hrpp_trace_noalloc");
    if (!sc) return noalloc_fail(HRPP_ERR_INVALID_ARG, "scene is NULL");
    if (mode != HRPP_ANY_HIT && mode != HRPP_CLOSEST_HIT) return noalloc_fail(HRPP_ERR_INVALID_ARG, "unknown mode");
    const bool closest = mode == HRPP_CLOSEST_HIT;
    if (n_rays > HRPP_NOALLOC_MAX_RAYS)
        return noalloc_fail(HRPP_ERR_INVALID_ARG, "n_rays %u exceeds the no-allocation limit of %u rays per call",
                            n_rays, (unsigned)HRPP_NOALLOC_MAX_RAYS);
    if (n_rays > 0 && (!rays || !out_hits)) return noalloc_fail(HRPP_ERR_INVALID_ARG, "NULL rays or out_hits");
    if (((uintptr_t)rays & 15u) != 0) return noalloc_fail(HRPP_ERR_INVALID_ARG, "rays must be 16-byte aligned");
    if (((uintptr_t)out_hits & (closest ? 15u : 3u)) != 0)
        return noalloc_fail(HRPP_ERR_INVALID_ARG, "out_hits misaligned");
    if (((uintptr_t)out_stats & 7u) != 0) return noalloc_fail(HRPP_ERR_INVALID_ARG, "out_stats must be 8-byte aligned");
    if (table && table->device != sc->device)
        return noalloc_fail(HRPP_ERR_INVALID_ARG, "table and scene on different devices");
    if (table && table->bound_scene && table->bound_scene != sc->id)
        return noalloc_fail(HRPP_ERR_INVALID_ARG, "table is bound to another scene; reset it first");

    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return noalloc_fail(HRPP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (prev != sc->device && (e = cudaSetDevice(sc->device)) != cudaSuccess)
        return noalloc_fail(HRPP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    hrpp_status status = HRPP_OK;
    cudaStream_t stream = (cudaStream_t)stream_;
    bool stats_host = false;
    do {
        if (n_rays > 0 && (!device_pointer(rays) || !device_pointer(out_hits))) {
            status = noalloc_fail(HRPP_ERR_INVALID_ARG, "rays and out_hits must be device memory");
            break;
        }
        if (out_stats) {
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, out_stats) != cudaSuccess) {
                cudaGetLastError();
                status = noalloc_fail(HRPP_ERR_INVALID_ARG, "out_stats is not a valid pointer");
                break;
            }
            stats_host = a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
        }
        if (n_rays == 0) {
            if (out_stats) {
                if (stats_host) memset(out_stats, 0, sizeof *out_stats);
                else if ((e = cudaMemsetAsync(out_stats, 0, sizeof *out_stats, stream)) != cudaSuccess)
                    status = noalloc_fail(HRPP_ERR_CUDA, "zeroing stats: %s", cudaGetErrorString(e));
            }
            break;
        }
        unsigned char *scratch = nullptr;
        if ((e = scratch_on(sc->device, &scratch)) != cudaSuccess) {
            status = noalloc_fail(HRPP_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            break;
        }
        Ctl *ctl = reinterpret_cast<Ctl *>(scratch);
        // the control block must start at zero; the records need no clearing
        if ((e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), stream)) != cudaSuccess) {
            status = noalloc_fail(HRPP_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
            break;
        }
        TraceParams p;
        memset(&p, 0, sizeof p);
        p.nodes = sc->d_nodes;
        p.tris = sc->d_tris;
        p.n_tris = sc->n_tris;
        p.root_ref = sc->root_ref;
        p.max_steps = sc->n_interior + sc->n_leaves + 8u;
        p.rays = reinterpret_cast<const float4 *>(rays);
        p.n_rays = n_rays;
        p.hits = out_hits;
        p.ctl = ctl;
        p.error = sc->d_error;
        p.refill_min = 16;
        p.n_interior = sc->n_interior;
        p.parent = sc->d_parent;
        p.leaf_parent = sc->d_leaf_parent;
        const bool two_phase = table && table->update_mode == HRPP_UPDATE_TWO_PHASE;
        if (table) {
            p.table = table->d_words;
            p.winner = table->d_winner;
            p.records = reinterpret_cast<Record *>(scratch + kNoallocCtlBytes);
            p.log2_sets = table->log2_sets;
            p.log2_ways = table->log2_ways;
            p.precision = table->precision;
            p.update_mode = table->update_mode;
            p.go_up = table->go_up;
            p.hash_variant = table->hash_variant;
            if (table->gate_min_tp) {
                p.gate = table->d_gate;
                p.gate_mask = (1u << table->gate_sample_log2) - 1u;
                p.gate_min_tp = table->gate_min_tp;
            }
        }
        e = sc->width == 2 ? launch_trace_w2(closest, out_stats != nullptr, 0, p, 128, 0, stream, nullptr, nullptr)
                           : launch_trace_w4(closest, out_stats != nullptr, 0, p, 128, 0, stream, nullptr, nullptr);
        if (e != cudaSuccess) {
            status = noalloc_fail(HRPP_ERR_CUDA, "trace launch: %s", cudaGetErrorString(e));
            break;
        }
        if (two_phase) e = launch_table_apply(table->d_words, table->d_winner, p.records, ctl, n_rays, stream, p.gate,
                                              p.gate_min_tp);
        else if (p.gate) e = launch_gate_update(p.gate, p.gate_min_tp, ctl, stream);
        if (e != cudaSuccess) {
            status = noalloc_fail(HRPP_ERR_CUDA, "table update launch: %s", cudaGetErrorString(e));
            break;
        }
        if (table) table->bound_scene = sc->id;
        if (out_stats) {
            e = cudaMemcpyAsync(out_stats, ctl->stats, sizeof(hrpp_stats),
                                stats_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, stream);
            if (e == cudaSuccess && stats_host) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) {
                status = noalloc_fail(HRPP_ERR_CUDA, "stats copy: %s", cudaGetErrorString(e));
                break;
            }
        }
        if (stats_host) {
            // the call has waited: report a ray stopped early exactly as
            // hrpp_trace does, and clear the scene's flag (a plain copy into a
            // host variable and a memset allocate nothing)
            uint32_t flag = 0;
            if ((e = cudaMemcpy(&flag, sc->d_error, sizeof flag, cudaMemcpyDeviceToHost)) != cudaSuccess) {
                status = noalloc_fail(HRPP_ERR_CUDA, "reading the error flag: %s", cudaGetErrorString(e));
                break;
            }
            if (flag) {
                cudaMemset(sc->d_error, 0, sizeof(uint32_t));
                status = noalloc_fail(HRPP_ERR_TRAVERSAL_LIMIT, "a ray was stopped early (flag %u)", flag);
                break;
            }
        }
    } while (false);
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    return status;
}
