// Host side of the HRPP C ABI (include/hrpp.h): argument checks, BVH
// validation and conversion to the device layouts, scene / table handles, and
// the per-call orchestration of hrpp_trace.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <vector>

#include "device.cuh"
#include "handles.h"
#include "hrpp.h"

using namespace hrpp;

bool hrpp::allocation_refused()
{
    static std::mutex mu;
    static std::string seen;
    static long long made = 0;
    const char *v = std::getenv("HRPP_FAIL_ALLOC_AFTER");
    std::lock_guard<std::mutex> lk(mu);
    if (!v || !*v) {
        seen.clear();  // unset: the next value counts from zero
        return false;
    }
    if (seen != v) {
        seen = v;
        made = 0;
    }
    return made++ >= std::atoll(v);
}

cudaError_t hrpp::device_malloc(void **ptr, size_t bytes)
{
    if (allocation_refused()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}


namespace {

// launch defaults (measured on GB300, see bench.py / the autotuner)
constexpr uint32_t kDefaultBlockThreads = 128;
constexpr uint32_t kDefaultSchedule = HRPP_SCHEDULE_BATCH;
constexpr uint32_t kDefaultRefillMin = 24;

thread_local std::string g_last_error;
std::atomic<uint64_t> g_next_scene_id{1};

hrpp_status fail(hrpp_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = std::string(hrpp_status_string(s)) + ": " + buf;
    return s;
}

hrpp_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return fail(HRPP_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(HRPP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Switches to `dev` for the lifetime of the guard, restoring the caller's device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// One stream-ordered memory pool per device for per-call scratch; it keeps
// freed blocks so repeated calls do not go back to the CUDA driver.
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[64] = {};

cudaError_t get_pool(int dev, cudaMemPool_t *pool)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pools[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        // never reuse a block by making the allocating stream wait for the
        // stream that freed it: a staged call's uploads (allocated on its
        // upload stream) would otherwise wait for the previous call's
        // downloads; the pool takes fresh memory instead
        int no = 0;
        cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    *pool = g_pools[dev];
    return cudaSuccess;
}

// Staged host buffers: at most kStagedChunks chunks of at least
// kStagedMinChunk rays (a chunk's launch still fills the GPU).
constexpr uint32_t kStagedChunks = 8;
constexpr uint32_t kStagedChunksAsync = 2;
constexpr uint64_t kStagedMinChunk = 1u << 18;

// A pair of library-owned copy streams (uploads, downloads) for one staged
// call; idle pairs are kept per device and reused, so concurrent staged calls
// from several host threads each get their own pair.
struct CopyStreams {
    cudaStream_t up = nullptr, down = nullptr;
};
std::mutex g_copy_mutex;
std::vector<CopyStreams> g_copy_idle[64];

cudaError_t acquire_copy_streams(int dev, CopyStreams *out)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(g_copy_mutex);
        if (!g_copy_idle[dev].empty()) {
            *out = g_copy_idle[dev].back();
            g_copy_idle[dev].pop_back();
            return cudaSuccess;
        }
    }
    CopyStreams c;
    cudaError_t e = cudaStreamCreateWithFlags(&c.up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.down, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (c.up) cudaStreamDestroy(c.up);
        return e;
    }
    *out = c;
    return cudaSuccess;
}

void release_copy_streams(int dev, const CopyStreams &c)
{
    std::lock_guard<std::mutex> lk(g_copy_mutex);
    g_copy_idle[dev].push_back(c);
}

// Staged calls in flight per device.  Each holds a staging block from the
// pool until its downloads are done; a caller that queues host_async calls
// without waiting would otherwise make the pool grow by one block per call
// (new device memory, mapped on the host thread inside the call).  A staged
// call that finds kStagedInFlight calls still holding staging waits on the
// host for the oldest one's block to be freed.  The work it waits for is
// already queued, so the wait ends.  Six (three two-batch frames ahead)
// measured as fast as 8 or 16 on the terrain frame loop; 4 sometimes stalled
// the uploads.
constexpr size_t kStagedInFlight = 6;
std::mutex g_inflight_mutex;
std::deque<cudaEvent_t> g_inflight[64];

cudaError_t wait_for_staging_slot(int dev)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    for (;;) {
        cudaEvent_t oldest = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_inflight_mutex);
            if (g_inflight[dev].size() < kStagedInFlight) return cudaSuccess;
            oldest = g_inflight[dev].front();
            g_inflight[dev].pop_front();
        }
        const cudaError_t e = cudaEventSynchronize(oldest);
        cudaEventDestroy(oldest);
        if (e != cudaSuccess) return e;
    }
}

// `freed` is recorded after a staged call's block is freed; the list owns it.
void note_staging_in_flight(int dev, cudaEvent_t freed)
{
    if (dev < 0 || dev >= 64) {
        cudaEventDestroy(freed);
        return;
    }
    std::lock_guard<std::mutex> lk(g_inflight_mutex);
    g_inflight[dev].push_back(freed);
}

bool is_host_pointer(const void *ptr, bool *ok, bool *pinned = nullptr)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ok = false;
        return false;
    }
    *ok = true;
    if (pinned) *pinned = a.type == cudaMemoryTypeHost;
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

uint32_t leaf_id(const hrpp_bvh_node &n) { return (n.first << 2) | (n.count - 1u); }

bool box_inside(const hrpp_bvh_node &c, const hrpp_bvh_node &p)
{
    for (int k = 0; k < 3; ++k)
        if (!(c.lo[k] >= p.lo[k]) || !(c.hi[k] <= p.hi[k])) return false;
    return true;
}

struct Validated {
    hrpp_scene_info info;
    std::vector<uint32_t> order;  // reachable interior nodes in preorder (device order)
};

hrpp_status validate(const float *tri_verts, uint32_t n_tris, const hrpp_bvh_node *nodes, uint32_t n_nodes,
                     uint32_t root, const uint32_t *prim_index, uint32_t n_prim_index, int width, Validated *out)
{
    if (width != 2 && width != 4) return fail(HRPP_ERR_INVALID_ARG, "width must be 2 or 4, got %d", width);
    if (n_tris == 0) return fail(HRPP_ERR_INVALID_ARG, "n_tris is 0");
    if (n_tris >= HRPP_MAX_TRIS) return fail(HRPP_ERR_UNSUPPORTED, "n_tris %u exceeds %u", n_tris, HRPP_MAX_TRIS - 1);
    if (!tri_verts || !nodes || !prim_index) return fail(HRPP_ERR_INVALID_ARG, "NULL scene array");
    if (n_nodes == 0 || root >= n_nodes) return fail(HRPP_ERR_INVALID_ARG, "root %u not below n_nodes %u", root, n_nodes);
    if (n_prim_index != n_tris) return fail(HRPP_ERR_INVALID_ARG, "n_prim_index %u != n_tris %u", n_prim_index, n_tris);
    for (uint64_t i = 0; i < 9ull * n_tris; ++i)
        if (!std::isfinite(tri_verts[i])) return fail(HRPP_ERR_INVALID_ARG, "non-finite vertex coordinate");
    std::vector<uint8_t> seen_prim(n_tris, 0), seen_slot(n_tris, 0), seen_node(n_nodes, 0);
    for (uint32_t k = 0; k < n_tris; ++k) {
        if (prim_index[k] >= n_tris) return fail(HRPP_ERR_INVALID_BVH, "prim_index[%u] = %u out of range", k, prim_index[k]);
        if (seen_prim[prim_index[k]]++) return fail(HRPP_ERR_INVALID_BVH, "prim %u listed twice", prim_index[k]);
    }
    Validated v;
    memset(&v.info, 0, sizeof v.info);
    v.info.width = (uint32_t)width;
    v.info.n_tris = n_tris;
    struct Item {
        uint32_t node, depth;
    };
    std::vector<Item> st;
    st.push_back({root, 0});
    seen_node[root] = 1;
    uint32_t max_depth = 0;
    while (!st.empty()) {
        const Item it = st.back();
        st.pop_back();
        const hrpp_bvh_node &n = nodes[it.node];
        if (n.count > 0) {
            if (n.count > HRPP_MAX_LEAF_TRIS)
                return fail(HRPP_ERR_UNSUPPORTED, "leaf %u holds %u triangles (max %d)", it.node, n.count, HRPP_MAX_LEAF_TRIS);
            if ((uint64_t)n.first + n.count > n_tris) return fail(HRPP_ERR_INVALID_BVH, "leaf %u range out of bounds", it.node);
            for (uint32_t j = 0; j < n.count; ++j) {
                const uint32_t slot = n.first + j;
                if (seen_slot[slot]++) return fail(HRPP_ERR_INVALID_BVH, "prim_index slot %u in two leaves", slot);
                const float *t = tri_verts + 9ull * prim_index[slot];
                for (int q = 0; q < 3; ++q)
                    for (int k = 0; k < 3; ++k)
                        if (!(t[3 * q + k] >= n.lo[k] && t[3 * q + k] <= n.hi[k]))
                            return fail(HRPP_ERR_INVALID_BVH, "leaf %u box does not hold prim %u", it.node, prim_index[slot]);
            }
            v.info.n_leaves++;
            if (it.depth > max_depth) max_depth = it.depth;
            continue;
        }
        v.order.push_back(it.node);
        v.info.n_interior++;
        int n_children = 0;
        for (int k = 0; k < 4; ++k) {
            const int32_t c = n.child[k];
            if (c == -1) continue;
            if (k >= width) return fail(HRPP_ERR_INVALID_BVH, "node %u uses child slot %d of a width-%d BVH", it.node, k, width);
            if (c < -1 || (uint32_t)c >= n_nodes) return fail(HRPP_ERR_INVALID_BVH, "node %u child %d out of range", it.node, c);
            if (seen_node[c]++) return fail(HRPP_ERR_INVALID_BVH, "node %d reached twice (cycle or shared child)", c);
            if (!box_inside(nodes[c], n)) return fail(HRPP_ERR_INVALID_BVH, "node %d box outside its parent %u", c, it.node);
            ++n_children;
        }
        if (n_children == 0) return fail(HRPP_ERR_INVALID_BVH, "interior node %u has no children", it.node);
        // preorder: push children in reverse slot order
        for (int k = 3; k >= 0; --k)
            if (n.child[k] != -1) st.push_back({(uint32_t)n.child[k], it.depth + 1});
    }
    for (uint32_t k = 0; k < n_tris; ++k)
        if (!seen_slot[k]) return fail(HRPP_ERR_INVALID_BVH, "prim_index slot %u in no leaf", k);
    v.info.max_depth = max_depth;
    v.info.root_is_leaf = nodes[root].count > 0;
    // nearest child is taken directly, the others pushed: (width-1) per level
    if ((uint64_t)max_depth * (uint64_t)(width - 1) > HRPP_MAX_STACK)
        return fail(HRPP_ERR_UNSUPPORTED, "BVH depth %u needs a stack deeper than %d", max_depth, HRPP_MAX_STACK);
    const uint64_t node_bytes = (uint64_t)v.info.n_interior * (width == 2 ? 64u : 128u);
    v.info.device_bytes = node_bytes + 48ull * n_tris + 256;
    if (out) *out = std::move(v);
    return HRPP_OK;
}

}  // namespace

hrpp_status hrpp::report(hrpp_status s, const char *message)
{
    g_last_error = std::string(hrpp_status_string(s)) + ": " + message;
    return s;
}

extern "C" {

const char *hrpp_status_string(hrpp_status s)
{
    switch (s) {
    case HRPP_OK: return "HRPP_OK";
    case HRPP_ERR_INVALID_ARG: return "HRPP_ERR_INVALID_ARG";
    case HRPP_ERR_INVALID_BVH: return "HRPP_ERR_INVALID_BVH";
    case HRPP_ERR_OOM: return "HRPP_ERR_OOM";
    case HRPP_ERR_CUDA: return "HRPP_ERR_CUDA";
    case HRPP_ERR_TRAVERSAL_LIMIT: return "HRPP_ERR_TRAVERSAL_LIMIT";
    case HRPP_ERR_UNSUPPORTED: return "HRPP_ERR_UNSUPPORTED";
    }
    return "HRPP_UNKNOWN_STATUS";
}

const char *hrpp_last_error(void) { return g_last_error.c_str(); }

int hrpp_version(void) { return HRPP_VERSION; }

hrpp_status hrpp_scene_validate(const float *tri_verts, uint32_t n_tris, const hrpp_bvh_node *nodes, uint32_t n_nodes,
                                uint32_t root, const uint32_t *prim_index, uint32_t n_prim_index, int width,
                                hrpp_scene_info *info)
{
    Validated v;
    hrpp_status s = validate(tri_verts, n_tris, nodes, n_nodes, root, prim_index, n_prim_index, width, &v);
    if (s == HRPP_OK && info) *info = v.info;
    return s;
}

hrpp_status hrpp_scene_create(const float *tri_verts, uint32_t n_tris, const hrpp_bvh_node *nodes, uint32_t n_nodes,
                              uint32_t root, const uint32_t *prim_index, uint32_t n_prim_index, int width,
                              hrpp_scene **out)
{
    if (!out) return fail(HRPP_ERR_INVALID_ARG, "out is NULL");
    Validated v;
    hrpp_status s = validate(tri_verts, n_tris, nodes, n_nodes, root, prim_index, n_prim_index, width, &v);
    if (s != HRPP_OK) return s;

    // device index of each reachable interior node: preorder position
    std::vector<int32_t> dev_index(n_nodes, -1);
    for (uint32_t k = 0; k < v.order.size(); ++k) dev_index[v.order[k]] = (int32_t)k;
    auto ref_of = [&](int32_t c) -> int32_t {
        const hrpp_bvh_node &n = nodes[c];
        if (n.count > 0) return (int32_t)~leaf_id(n);
        return dev_index[c];
    };
    // parent links for the Go Up Level (Sec. 6.2) and bottom-up verification:
    // interior node -> parent (also kept in the node's spare word), and a
    // leaf's first prim_index slot -> the leaf's parent (-1 at the root)
    std::vector<int32_t> h_parent(std::max<size_t>(1, v.order.size()), -1), h_leaf_parent(n_tris, -1);
    for (uint32_t k = 0; k < v.order.size(); ++k) {
        const hrpp_bvh_node &n = nodes[v.order[k]];
        for (int q = 0; q < 4; ++q) {
            const int32_t c = n.child[q];
            if (c == -1) continue;
            if (nodes[c].count > 0) h_leaf_parent[nodes[c].first] = (int32_t)k;
            else h_parent[dev_index[c]] = (int32_t)k;
        }
    }
    const size_t f4_per_node = width == 2 ? 4 : 8;
    std::vector<float4> h_nodes(std::max<size_t>(1, v.order.size() * f4_per_node));
    for (uint32_t k = 0; k < v.order.size(); ++k) {
        const hrpp_bvh_node &n = nodes[v.order[k]];
        int32_t refs[4] = {kEmptyRef, kEmptyRef, kEmptyRef, kEmptyRef};
        const hrpp_bvh_node *boxes[4] = {nullptr, nullptr, nullptr, nullptr};
        int m = 0;
        for (int q = 0; q < 4; ++q)
            if (n.child[q] != -1) {
                refs[m] = ref_of(n.child[q]);
                boxes[m] = &nodes[n.child[q]];
                ++m;
            }
        float4 *d = &h_nodes[k * f4_per_node];
        if (width == 2) {
            const hrpp_bvh_node *b0 = boxes[0], *b1 = boxes[1] ? boxes[1] : boxes[0];
            d[0] = make_float4(b0->lo[0], b0->hi[0], b0->lo[1], b0->hi[1]);
            d[1] = make_float4(b1->lo[0], b1->hi[0], b1->lo[1], b1->hi[1]);
            d[2] = make_float4(b0->lo[2], b0->hi[2], b1->lo[2], b1->hi[2]);
            int4 c = make_int4(refs[0], refs[1], h_parent[k], 0);
            memcpy(&d[3], &c, sizeof c);
        } else {
            float lo[3][4], hi[3][4];
            for (int q = 0; q < 4; ++q)
                for (int a = 0; a < 3; ++a) {
                    lo[a][q] = boxes[q] ? boxes[q]->lo[a] : 0.0f;
                    hi[a][q] = boxes[q] ? boxes[q]->hi[a] : 0.0f;
                }
            for (int a = 0; a < 3; ++a) {
                d[2 * a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
                d[2 * a + 1] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
            }
            int4 c = make_int4(refs[0], refs[1], refs[2], refs[3]);
            memcpy(&d[6], &c, sizeof c);
            int4 extra = make_int4(h_parent[k], 0, 0, 0);
            memcpy(&d[7], &extra, sizeof extra);
        }
    }
    // canonical node -> device ref, for per-ray predicted nodes
    std::vector<int32_t> h_canon(n_nodes, kEmptyRef);
    for (uint32_t k = 0; k < v.order.size(); ++k) {
        const hrpp_bvh_node &n = nodes[v.order[k]];
        h_canon[v.order[k]] = (int32_t)k;
        for (int q = 0; q < 4; ++q)
            if (n.child[q] != -1 && nodes[n.child[q]].count > 0) h_canon[n.child[q]] = (int32_t)~leaf_id(nodes[n.child[q]]);
    }
    if (nodes[root].count > 0) h_canon[root] = (int32_t)~leaf_id(nodes[root]);
    // triangles in leaf (prim_index) order: v0 with the prim id, then the edges
    std::vector<float4> h_tris(3ull * n_tris);
    for (uint32_t k = 0; k < n_tris; ++k) {
        const uint32_t prim = prim_index[k];
        const float *t = tri_verts + 9ull * prim;
        float pw;
        memcpy(&pw, &prim, 4);
        h_tris[3ull * k] = make_float4(t[0], t[1], t[2], pw);
        h_tris[3ull * k + 1] = make_float4(t[3] - t[0], t[4] - t[1], t[5] - t[2], 0.0f);
        h_tris[3ull * k + 2] = make_float4(t[6] - t[0], t[7] - t[1], t[8] - t[2], 0.0f);
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    hrpp_scene *sc = new (std::nothrow) hrpp_scene;
    if (!sc) return fail(HRPP_ERR_OOM, "host allocation");
    memset(sc, 0, sizeof *sc);
    sc->device = dev;
    sc->id = g_next_scene_id.fetch_add(1);
    sc->width = width;
    sc->n_tris = n_tris;
    sc->n_interior = v.info.n_interior;
    sc->n_leaves = v.info.n_leaves;
    sc->max_depth = v.info.max_depth;
    sc->root_ref = nodes[root].count > 0 ? (int32_t)~leaf_id(nodes[root]) : 0;
    const size_t nb = h_nodes.size() * sizeof(float4), tb = h_tris.size() * sizeof(float4);
    const size_t pb = h_parent.size() * sizeof(int32_t), lb = h_leaf_parent.size() * sizeof(int32_t);
    const size_t cb = h_canon.size() * sizeof(int32_t);
    sc->n_nodes = n_nodes;
    sc->bytes = nb + tb + pb + lb + cb + sizeof(uint32_t);
    if ((e = device_malloc((void **)&sc->d_nodes, nb)) != cudaSuccess || (e = device_malloc((void **)&sc->d_tris, tb)) != cudaSuccess ||
        (e = device_malloc((void **)&sc->d_error, sizeof(uint32_t))) != cudaSuccess ||
        (e = device_malloc((void **)&sc->d_parent, pb)) != cudaSuccess || (e = device_malloc((void **)&sc->d_leaf_parent, lb)) != cudaSuccess ||
        (e = device_malloc((void **)&sc->d_canon_ref, cb)) != cudaSuccess ||
        (e = cudaMemcpy(sc->d_canon_ref, h_canon.data(), cb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sc->d_nodes, h_nodes.data(), nb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sc->d_tris, h_tris.data(), tb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sc->d_parent, h_parent.data(), pb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sc->d_leaf_parent, h_leaf_parent.data(), lb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(sc->d_error, 0, sizeof(uint32_t))) != cudaSuccess) {
        hrpp_scene_destroy(sc);
        return cuda_fail(e, "scene upload");
    }
    *out = sc;
    return HRPP_OK;
}

hrpp_status hrpp_scene_get_info(const hrpp_scene *sc, hrpp_scene_info *info)
{
    if (!sc || !info) return fail(HRPP_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof *info);
    info->n_tris = sc->n_tris;
    info->n_interior = sc->n_interior;
    info->n_leaves = sc->n_leaves;
    info->max_depth = sc->max_depth;
    info->width = (uint32_t)sc->width;
    info->root_is_leaf = sc->root_ref < 0;
    info->device_bytes = sc->bytes;
    return HRPP_OK;
}

hrpp_status hrpp_scene_check(hrpp_scene *sc, void *stream)
{
    if (!sc) return fail(HRPP_ERR_INVALID_ARG, "scene is NULL");
    DeviceGuard g(sc->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    uint32_t flag = 0;
    if ((e = cudaMemcpy(&flag, sc->d_error, sizeof flag, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading the error flag");
    if (flag) {
        cudaMemset(sc->d_error, 0, sizeof(uint32_t));
        return fail(HRPP_ERR_TRAVERSAL_LIMIT, "a ray was stopped early (flag %u: %s)", flag,
                    (flag & kErrStack) ? "stack bound" : "step bound");
    }
    return HRPP_OK;
}

void hrpp_scene_destroy(hrpp_scene *sc)
{
    if (!sc) return;
    DeviceGuard g(sc->device);
    cudaFree(sc->d_nodes);
    cudaFree(sc->d_tris);
    cudaFree(sc->d_error);
    cudaFree(sc->d_parent);
    cudaFree(sc->d_leaf_parent);
    cudaFree(sc->d_canon_ref);
    delete sc;
}

hrpp_status hrpp_table_create(int log2_entries, int ways, hrpp_table **out)
{
    if (!out) return fail(HRPP_ERR_INVALID_ARG, "out is NULL");
    int log2_ways;
    switch (ways) {
    case 1: log2_ways = 0; break;
    case 2: log2_ways = 1; break;
    case 4: log2_ways = 2; break;
    case 8: log2_ways = 3; break;
    default: return fail(HRPP_ERR_INVALID_ARG, "ways must be 1, 2, 4 or 8, got %d", ways);
    }
    if (log2_entries < log2_ways || log2_entries > 28)
        return fail(HRPP_ERR_INVALID_ARG, "log2_entries must be in [%d, 28], got %d", log2_ways, log2_entries);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    hrpp_table *t = new (std::nothrow) hrpp_table;
    if (!t) return fail(HRPP_ERR_OOM, "host allocation");
    memset(t, 0, sizeof *t);
    t->device = dev;
    t->log2_entries = log2_entries;
    t->log2_ways = log2_ways;
    t->log2_sets = log2_entries - log2_ways;
    t->precision = 6;
    t->update_mode = HRPP_UPDATE_TWO_PHASE;
    const uint64_t n = 1ull << log2_entries;
    t->gate_sample_log2 = 5;
    // the gate word sits right after the table words, so one copy restores both
    e = device_malloc((void **)&t->d_words, n * 8 + 16);
    if (e == cudaSuccess) {
        t->d_gate = reinterpret_cast<uint32_t *>(t->d_words + n);
        e = device_malloc((void **)&t->d_winner, n * 4);
    }
    if (e == cudaSuccess) e = cudaMemset(t->d_words, 0xFF, n * 8);
    if (e == cudaSuccess) e = cudaMemset(t->d_winner, 0, n * 4);
    if (e == cudaSuccess) e = cudaMemset(t->d_gate, 1, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        hrpp_table_destroy(t);
        return cuda_fail(e, "table allocation");
    }
    *out = t;
    return HRPP_OK;
}

hrpp_status hrpp_table_configure(hrpp_table *t, int precision_bits, int update_mode)
{
    if (!t) return fail(HRPP_ERR_INVALID_ARG, "table is NULL");
    if (precision_bits < 1 || precision_bits > 7) return fail(HRPP_ERR_INVALID_ARG, "precision_bits must be in [1, 7]");
    if (update_mode < HRPP_UPDATE_TWO_PHASE || update_mode > HRPP_UPDATE_FROZEN)
        return fail(HRPP_ERR_INVALID_ARG, "unknown update_mode %d", update_mode);
    t->precision = precision_bits;
    t->update_mode = update_mode;
    return HRPP_OK;
}

hrpp_status hrpp_table_set_go_up(hrpp_table *t, int go_up_level)
{
    if (!t) return fail(HRPP_ERR_INVALID_ARG, "table is NULL");
    if (go_up_level < 0 || go_up_level > 15) return fail(HRPP_ERR_INVALID_ARG, "go_up_level must be in [0, 15]");
    t->go_up = go_up_level;
    return HRPP_OK;
}

hrpp_status hrpp_table_set_hash(hrpp_table *t, int hash_variant)
{
    if (!t) return fail(HRPP_ERR_INVALID_ARG, "table is NULL");
    if (hash_variant != HRPP_HASH_EXP_MSB && hash_variant != HRPP_HASH_EXP_LSB)
        return fail(HRPP_ERR_INVALID_ARG, "unknown hash variant %d", hash_variant);
    t->hash_variant = hash_variant;
    return HRPP_OK;
}

hrpp_status hrpp_table_set_gate(hrpp_table *t, uint32_t min_tp_per_65536, int sample_log2)
{
    if (!t) return fail(HRPP_ERR_INVALID_ARG, "table is NULL");
    if (min_tp_per_65536 > 65536u) return fail(HRPP_ERR_INVALID_ARG, "min_tp_per_65536 must be at most 65536");
    if (sample_log2 < 0 || sample_log2 > 20) return fail(HRPP_ERR_INVALID_ARG, "sample_log2 must be in [0, 20]");
    DeviceGuard g(t->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemset(t->d_gate, 1, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "gate reset");
    t->gate_min_tp = min_tp_per_65536;
    t->gate_sample_log2 = sample_log2;
    return HRPP_OK;
}

hrpp_status hrpp_table_get_gate(const hrpp_table *t, int *open)
{
    if (!t || !open) return fail(HRPP_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(t->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    uint32_t w = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&w, t->d_gate, sizeof w, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "gate read");
    *open = w != 0u;
    return HRPP_OK;
}

hrpp_status hrpp_table_reset(hrpp_table *t, void *stream)
{
    if (!t) return fail(HRPP_ERR_INVALID_ARG, "table is NULL");
    DeviceGuard g(t->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    const uint64_t n = 1ull << t->log2_entries;
    cudaError_t e = launch_table_fill(t->d_words, n, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->d_winner, 0, n * 4, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->d_gate, 1, sizeof(uint32_t), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "table reset");
    t->bound_scene = 0;
    return HRPP_OK;
}

hrpp_status hrpp_table_export(const hrpp_table *t, uint64_t *host_words, size_t n_words)
{
    if (!t || !host_words) return fail(HRPP_ERR_INVALID_ARG, "NULL argument");
    if (n_words != (1ull << t->log2_entries)) return fail(HRPP_ERR_INVALID_ARG, "n_words must be %llu", 1ull << t->log2_entries);
    DeviceGuard g(t->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host_words, t->d_words, n_words * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "table export");
    return HRPP_OK;
}

hrpp_status hrpp_table_import(hrpp_table *t, const uint64_t *host_words, size_t n_words)
{
    if (!t || !host_words) return fail(HRPP_ERR_INVALID_ARG, "NULL argument");
    if (n_words != (1ull << t->log2_entries)) return fail(HRPP_ERR_INVALID_ARG, "n_words must be %llu", 1ull << t->log2_entries);
    DeviceGuard g(t->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(t->d_words, host_words, n_words * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(t->d_winner, 0, n_words * 4);
    if (e == cudaSuccess) e = cudaMemset(t->d_gate, 1, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "table import");
    return HRPP_OK;
}

hrpp_status hrpp_table_copy(hrpp_table *dst, const hrpp_table *src, void *stream)
{
    if (!dst || !src) return fail(HRPP_ERR_INVALID_ARG, "NULL argument");
    if (dst == src) return HRPP_OK;
    if (dst->device != src->device) return fail(HRPP_ERR_INVALID_ARG, "tables on different devices");
    if (dst->log2_entries != src->log2_entries || dst->log2_ways != src->log2_ways ||
        dst->precision != src->precision || dst->go_up != src->go_up || dst->hash_variant != src->hash_variant)
        return fail(HRPP_ERR_INVALID_ARG, "tables differ in size, ways, precision, Go Up Level or hash variant");
    DeviceGuard g(dst->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    const uint64_t n = 1ull << dst->log2_entries;
    // the words and the gate word behind them, in one copy
    cudaError_t e = cudaMemcpyAsync(dst->d_words, src->d_words, n * 8 + sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "table copy");
    dst->bound_scene = src->bound_scene;
    return HRPP_OK;
}

hrpp_status hrpp_table_get_config(const hrpp_table *t, int *log2_entries, int *ways, int *precision_bits,
                                  int *update_mode)
{
    if (!t) return fail(HRPP_ERR_INVALID_ARG, "table is NULL");
    if (log2_entries) *log2_entries = t->log2_entries;
    if (ways) *ways = 1 << t->log2_ways;
    if (precision_bits) *precision_bits = t->precision;
    if (update_mode) *update_mode = t->update_mode;
    return HRPP_OK;
}

void hrpp_table_destroy(hrpp_table *t)
{
    if (!t) return;
    DeviceGuard g(t->device);
    cudaFree(t->d_words);  // holds the gate word too
    cudaFree(t->d_winner);
    delete t;
}

hrpp_status hrpp_trace(const hrpp_scene *sc, hrpp_table *table, const hrpp_ray *rays, uint32_t n_rays, hrpp_mode mode,
                       void *out_hits, hrpp_stats *out_stats, void *stream)
{
    return hrpp_trace_ex(sc, table, rays, n_rays, mode, out_hits, out_stats, stream, nullptr);
}

hrpp_status hrpp_trace_ex(const hrpp_scene *sc, hrpp_table *table, const hrpp_ray *rays, uint32_t n_rays,
                          hrpp_mode mode, void *out_hits, hrpp_stats *out_stats, void *stream_,
                          const hrpp_trace_opts *opts)
{
    hrpp::NvtxRange nvtx_range("hrpp_trace");
    if (!sc) return fail(HRPP_ERR_INVALID_ARG, "scene is NULL");
    if (mode != HRPP_ANY_HIT && mode != HRPP_CLOSEST_HIT) return fail(HRPP_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    const bool closest = mode == HRPP_CLOSEST_HIT;
    if (n_rays > 0 && (!rays || !out_hits)) return fail(HRPP_ERR_INVALID_ARG, "NULL rays or out_hits");
    // the ray pool's 32-bit cursor must not wrap: at most 2^31 rays per call
    if (n_rays > (1u << 31)) return fail(HRPP_ERR_UNSUPPORTED, "n_rays %u exceeds 2^31", n_rays);
    if (((uintptr_t)rays & 15u) != 0) return fail(HRPP_ERR_INVALID_ARG, "rays must be 16-byte aligned");
    if (((uintptr_t)out_hits & (closest ? 15u : 3u)) != 0)
        return fail(HRPP_ERR_INVALID_ARG, "out_hits must be %d-byte aligned", closest ? 16 : 4);
    if (((uintptr_t)out_stats & 7u) != 0) return fail(HRPP_ERR_INVALID_ARG, "out_stats must be 8-byte aligned");
    uint32_t block_threads = kDefaultBlockThreads;
    if (opts && opts->block_threads) {
        block_threads = opts->block_threads;
        if (block_threads != 64 && block_threads != 128 && block_threads != 256 && block_threads != 512)
            return fail(HRPP_ERR_INVALID_ARG, "block_threads must be 64, 128, 256 or 512");
    }
    uint32_t schedule = kDefaultSchedule, refill_min = kDefaultRefillMin;
    if (opts && opts->schedule) {
        if (opts->schedule != HRPP_SCHEDULE_BATCH && opts->schedule != HRPP_SCHEDULE_REFILL &&
            opts->schedule != HRPP_SCHEDULE_COMPACT)
            return fail(HRPP_ERR_INVALID_ARG, "unknown schedule %u", opts->schedule);
        schedule = opts->schedule;
    }
    if (opts && opts->refill_min) {
        if (opts->refill_min > 32) return fail(HRPP_ERR_INVALID_ARG, "refill_min must be in [1, 32]");
        refill_min = opts->refill_min;
    }
    if (opts && opts->verify != HRPP_VERIFY_ROOT && opts->verify != HRPP_VERIFY_BOTTOM_UP &&
        opts->verify != HRPP_VERIFY_NONE)
        return fail(HRPP_ERR_INVALID_ARG, "unknown verify mode %u", opts->verify);
    if (opts && opts->l2_persist > HRPP_L2_NODES)
        return fail(HRPP_ERR_INVALID_ARG, "unknown l2_persist value %u", opts->l2_persist);
    if (opts && opts->stage_chunks > 64) return fail(HRPP_ERR_INVALID_ARG, "stage_chunks must be at most 64");
    if (table && table->device != sc->device) return fail(HRPP_ERR_INVALID_ARG, "table and scene on different devices");
    if (table && table->bound_scene && table->bound_scene != sc->id)
        return fail(HRPP_ERR_INVALID_ARG, "table is bound to another scene; reset it first");
    DeviceGuard g(sc->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
    cudaStream_t stream = (cudaStream_t)stream_;
    cudaError_t e;

    bool stats_host = false;
    if (out_stats) {
        bool ok;
        stats_host = is_host_pointer(out_stats, &ok);
        if (!ok) return fail(HRPP_ERR_INVALID_ARG, "out_stats is not a valid pointer");
    }
    if (n_rays == 0) {
        if (out_stats) {
            if (stats_host) memset(out_stats, 0, sizeof *out_stats);
            else if ((e = cudaMemsetAsync(out_stats, 0, sizeof *out_stats, stream)) != cudaSuccess)
                return cuda_fail(e, "zeroing stats");
        }
        return HRPP_OK;
    }
    bool ok_r, ok_h, pinned_r = false, pinned_h = false;
    const bool rays_host = is_host_pointer(rays, &ok_r, &pinned_r);
    const bool hits_host = is_host_pointer(out_hits, &ok_h, &pinned_h);
    if (!ok_r || !ok_h) return fail(HRPP_ERR_INVALID_ARG, "rays / out_hits are not valid pointers");
    const bool host_async = opts && opts->host_async;
    if (host_async && ((rays_host && !pinned_r) || (hits_host && !pinned_h)))
        return fail(HRPP_ERR_INVALID_ARG, "host_async needs page-locked host buffers");

    cudaMemPool_t pool;
    if ((e = get_pool(sc->device, &pool)) != cudaSuccess) return cuda_fail(e, "memory pool");
    const bool two_phase = table && table->update_mode == HRPP_UPDATE_TWO_PHASE;
    // the two-pass schedule serves table lookups of leaves (Go Up Level 0)
    // with root or no verification; other calls run the BATCH schedule
    const bool compact = schedule == HRPP_SCHEDULE_COMPACT && table && table->go_up == 0 &&
                         !(opts && opts->predicted_nodes) && !(opts && opts->verify == HRPP_VERIFY_BOTTOM_UP);
    const size_t hit_size = closest ? sizeof(hrpp_hit) : sizeof(uint32_t);
    const size_t hit_bytes = (size_t)n_rays * hit_size;
    const size_t ray_bytes = (size_t)n_rays * sizeof(hrpp_ray);
    // Host buffers are staged in chunks (a multiple of 32 rays each): chunk
    // k+1 uploads on one copy stream and chunk k-1 downloads on another while
    // chunk k traces on the caller's stream.  Every chunk looks up the table
    // as the call found it; the two-phase update runs once, after the last.
    const bool staged = rays_host || hits_host;
    uint32_t n_chunks = 1, chunk = n_rays;
    if (staged) {
        // default: up to 8 chunks for a call that waits (its copies overlap
        // its own chunks' traces), 2 for host_async (its copies mostly
        // overlap the work queued around it, as a double-buffered frame
        // loop's do; 1 to 3 chunks measured within 1 % on the terrain frame)
        const uint32_t max_chunks = (opts && opts->stage_chunks) ? opts->stage_chunks
                                    : (host_async ? kStagedChunksAsync : kStagedChunks);
        n_chunks = (uint32_t)std::min<uint64_t>(max_chunks, (n_rays + kStagedMinChunk - 1) / kStagedMinChunk);
        if (n_chunks < 1) n_chunks = 1;
        chunk = (uint32_t)((((uint64_t)n_rays + n_chunks - 1) / n_chunks + 31u) & ~31ull);
        n_chunks = (uint32_t)(((uint64_t)n_rays + chunk - 1) / chunk);
    }
    // scratch on `stream`: control block, insert records, two-pass queue
    size_t off = 0;
    const size_t ctl_off = off;
    off += 256;
    const size_t rec_off = off;
    if (two_phase) off += (size_t)n_rays * sizeof(Record);
    const size_t queue_off = off;
    if (compact) off += (size_t)chunk * 16u;
    // staging buffers on the upload stream, so that the uploads need not
    // wait for earlier work on `stream` (an earlier call's traces)
    const size_t hit_stage_off = rays_host ? (ray_bytes + 255) & ~size_t(255) : 0;
    const size_t stage_bytes = hit_stage_off + (hits_host ? (hit_bytes + 255) & ~size_t(255) : 0);
    char *scratch = nullptr, *staging = nullptr;
    if (allocation_refused()) return cuda_fail(cudaErrorMemoryAllocation, "scratch allocation (injected)");
    if ((e = cudaMallocFromPoolAsync((void **)&scratch, off, pool, stream)) != cudaSuccess)
        return cuda_fail(e, "scratch allocation");
    Ctl *ctl = reinterpret_cast<Ctl *>(scratch + ctl_off);
    CopyStreams cs;
    std::vector<cudaEvent_t> events;
    auto event = [&](cudaEvent_t *ev) {
        cudaError_t err = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (err == cudaSuccess) events.push_back(*ev);
        return err;
    };
    hrpp_status status = HRPP_OK;
    char *d_rays = (char *)rays, *d_hits = (char *)out_hits;
    do {
        if ((e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), stream)) != cudaSuccess) { status = cuda_fail(e, "memset"); break; }
        if (staged) {
            if ((e = wait_for_staging_slot(sc->device)) != cudaSuccess) { status = cuda_fail(e, "staging wait"); break; }
            if ((e = acquire_copy_streams(sc->device, &cs)) != cudaSuccess) { status = cuda_fail(e, "copy streams"); break; }
            if (allocation_refused()) { status = cuda_fail(cudaErrorMemoryAllocation, "staging (injected)"); break; }
            if ((e = cudaMallocFromPoolAsync((void **)&staging, stage_bytes, pool, cs.up)) != cudaSuccess) {
                status = cuda_fail(e, "staging allocation");
                break;
            }
            if (rays_host) d_rays = staging;
            if (hits_host) d_hits = staging + hit_stage_off;
        }
        TraceParams p;
        memset(&p, 0, sizeof p);
        p.nodes = sc->d_nodes;
        p.tris = sc->d_tris;
        p.n_tris = sc->n_tris;
        p.root_ref = sc->root_ref;
        p.max_steps = sc->n_interior + sc->n_leaves + 8u;
        if (opts && opts->max_steps > 0u && opts->max_steps < p.max_steps) p.max_steps = opts->max_steps;
        p.verify = opts ? (int)opts->verify : 0;
        p.ctl = ctl;
        p.error = sc->d_error;
        p.refill_min = refill_min;
        p.n_interior = sc->n_interior;
        p.parent = sc->d_parent;
        p.leaf_parent = sc->d_leaf_parent;
        p.canon_ref = sc->d_canon_ref;
        p.n_nodes = sc->n_nodes;
        if (table) {
            p.table = table->d_words;
            p.winner = table->d_winner;
            p.records = reinterpret_cast<Record *>(scratch + rec_off);
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
        cudaEvent_t ev0 = opts ? (cudaEvent_t)opts->kernel_start : nullptr;
        cudaEvent_t ev1 = opts ? (cudaEvent_t)opts->kernel_stop : nullptr;
        const int sched = schedule == HRPP_SCHEDULE_REFILL ? 1 : 0;
        L2Window l2{nullptr, 0};
        if (opts && opts->l2_persist == HRPP_L2_TABLE && table)
            l2 = L2Window{table->d_words, sizeof(uint64_t) << table->log2_entries};
        else if (opts && opts->l2_persist == HRPP_L2_NODES)
            l2 = L2Window{sc->d_nodes, (size_t)sc->n_interior * (sc->width == 2 ? 64u : 128u)};
        for (uint32_t k = 0; k < n_chunks && status == HRPP_OK; ++k) {
            const uint64_t first = (uint64_t)k * chunk;
            const uint32_t cnt = (uint32_t)std::min<uint64_t>(chunk, n_rays - first);
            if (rays_host) {
                cudaEvent_t up_done;
                if ((e = cudaMemcpyAsync(d_rays + first * sizeof(hrpp_ray), (const char *)rays + first * sizeof(hrpp_ray),
                                         (size_t)cnt * sizeof(hrpp_ray), cudaMemcpyHostToDevice, cs.up)) != cudaSuccess ||
                    (e = event(&up_done)) != cudaSuccess || (e = cudaEventRecord(up_done, cs.up)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(stream, up_done, 0)) != cudaSuccess) {
                    status = cuda_fail(e, "ray upload");
                    break;
                }
            }
            // each chunk restarts the ray pool's cursor and the queue
            if (k > 0 && (e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned int), stream)) != cudaSuccess) {
                status = cuda_fail(e, "memset");
                break;
            }
            TraceParams pk = p;
            pk.rays = reinterpret_cast<const float4 *>(d_rays + first * sizeof(hrpp_ray));
            pk.hits = d_hits + first * hit_size;
            pk.n_rays = cnt;
            pk.ray_offset = (uint32_t)first;
            pk.predicted = (opts && opts->predicted_nodes) ? opts->predicted_nodes + first : nullptr;
            if (opts && out_stats) {
                pk.ray_outcome = opts->ray_outcome ? opts->ray_outcome + first : nullptr;
                pk.ray_box_tests = opts->ray_box_tests ? opts->ray_box_tests + first : nullptr;
            }
            cudaEvent_t e0 = k == 0 ? ev0 : nullptr, e1 = k + 1 == n_chunks ? ev1 : nullptr;
            if (compact)
                e = sc->width == 2 ? launch_compact_w2(closest, out_stats != nullptr, pk, scratch + queue_off, (int)block_threads,
                                                       stream, e0, e1)
                                   : launch_compact_w4(closest, out_stats != nullptr, pk, scratch + queue_off, (int)block_threads,
                                                       stream, e0, e1);
            else
                e = sc->width == 2 ? launch_trace_w2(closest, out_stats != nullptr, sched, pk, (int)block_threads, 0, stream, e0, e1, &l2)
                                   : launch_trace_w4(closest, out_stats != nullptr, sched, pk, (int)block_threads, 0, stream, e0, e1, &l2);
            if (e != cudaSuccess) { status = cuda_fail(e, "trace launch"); break; }
            if (hits_host) {
                cudaEvent_t traced;
                if ((e = event(&traced)) != cudaSuccess || (e = cudaEventRecord(traced, stream)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(cs.down, traced, 0)) != cudaSuccess ||
                    (e = cudaMemcpyAsync((char *)out_hits + first * hit_size, d_hits + first * hit_size, (size_t)cnt * hit_size,
                                         cudaMemcpyDeviceToHost, cs.down)) != cudaSuccess) {
                    status = cuda_fail(e, "hit download");
                    break;
                }
            }
        }
        if (status != HRPP_OK) break;
        if (two_phase) e = launch_table_apply(table->d_words, table->d_winner, p.records, ctl, n_rays, stream, p.gate,
                                              p.gate_min_tp);
        else if (p.gate) e = launch_gate_update(p.gate, p.gate_min_tp, ctl, stream);
        if (e != cudaSuccess) {
            status = cuda_fail(e, "table update launch");
            break;
        }
        if (table) table->bound_scene = sc->id;
        if (out_stats) {
            e = cudaMemcpyAsync(out_stats, ctl->stats, sizeof(hrpp_stats),
                                stats_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess) { status = cuda_fail(e, "stats copy"); break; }
        }
    } while (false);
    if (cs.up) {
        // the staging is freed in stream order on the download stream, after
        // the last chunk's trace and download; `stream` then waits for the
        // downloads, so the hits are in host memory when it gets there
        cudaEvent_t traced = nullptr, uploaded = nullptr, drained = nullptr;
        cudaError_t ed = event(&traced);
        if (ed == cudaSuccess) ed = cudaEventRecord(traced, stream);
        if (ed == cudaSuccess) ed = cudaStreamWaitEvent(cs.down, traced, 0);
        if (ed == cudaSuccess) ed = event(&uploaded);  // (uploads a failed call left unordered)
        if (ed == cudaSuccess) ed = cudaEventRecord(uploaded, cs.up);
        if (ed == cudaSuccess) ed = cudaStreamWaitEvent(cs.down, uploaded, 0);
        if (ed == cudaSuccess && staging) ed = cudaFreeAsync(staging, cs.down);
        if (ed == cudaSuccess && staging) {
            cudaEvent_t freed = nullptr;
            ed = cudaEventCreateWithFlags(&freed, cudaEventDisableTiming);
            if (ed == cudaSuccess && (ed = cudaEventRecord(freed, cs.down)) != cudaSuccess) cudaEventDestroy(freed);
            if (ed == cudaSuccess) note_staging_in_flight(sc->device, freed);
        }
        if (host_async && opts->host_done) {
            // the caller's event marks the hits in host memory; `stream`
            // goes on after the traces without waiting for the downloads
            if (ed == cudaSuccess) ed = cudaEventRecord((cudaEvent_t)opts->host_done, cs.down);
        } else {
            if (ed == cudaSuccess) ed = event(&drained);
            if (ed == cudaSuccess) ed = cudaEventRecord(drained, cs.down);
            if (ed == cudaSuccess) ed = cudaStreamWaitEvent(stream, drained, 0);
        }
        if (ed != cudaSuccess) {
            cudaStreamSynchronize(stream);
            cudaStreamSynchronize(cs.up);
            cudaStreamSynchronize(cs.down);
        }
        if (ed != cudaSuccess && status == HRPP_OK) status = cuda_fail(ed, "staging order");
    }
    cudaError_t ef = cudaFreeAsync(scratch, stream);
    // with device buffers the hits are final where `stream` gets to now
    if (!cs.up && host_async && opts->host_done && status == HRPP_OK) {
        if ((e = cudaEventRecord((cudaEvent_t)opts->host_done, stream)) != cudaSuccess)
            status = cuda_fail(e, "host_done record");
    }
    const bool wait = (staged && !host_async) || stats_host;
    if (wait) {
        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess && status == HRPP_OK)
            status = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (cs.up) release_copy_streams(sc->device, cs);
    for (cudaEvent_t ev : events) cudaEventDestroy(ev);
    if (status != HRPP_OK) return status;
    if (ef != cudaSuccess) return cuda_fail(ef, "scratch free");
    if (wait) {
        uint32_t flag = 0;
        if ((e = cudaMemcpy(&flag, sc->d_error, sizeof flag, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "reading the error flag");
        if (flag) {
            cudaMemset(sc->d_error, 0, sizeof(uint32_t));
            return fail(HRPP_ERR_TRAVERSAL_LIMIT, "a ray was stopped early (flag %u)", flag);
        }
    }
    return HRPP_OK;
}

hrpp_status hrpp_l2_set_aside(size_t bytes, size_t *granted)
{
    int dev = 0, max_persist = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev)) != cudaSuccess)
        return cuda_fail(e, "persisting L2 size");
    if (max_persist <= 0) return fail(HRPP_ERR_CUDA, "device %d has no persisting L2", dev);
    if (bytes > (size_t)max_persist) bytes = (size_t)max_persist;
    if (bytes == 0 && (e = cudaCtxResetPersistingL2Cache()) != cudaSuccess)
        return cuda_fail(e, "cudaCtxResetPersistingL2Cache");
    if ((e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceSetLimit(persisting L2)");
    if (granted) {
        size_t now = 0;
        if ((e = cudaDeviceGetLimit(&now, cudaLimitPersistingL2CacheSize)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetLimit(persisting L2)");
        *granted = now;
    }
    return HRPP_OK;
}

}  // extern "C"
