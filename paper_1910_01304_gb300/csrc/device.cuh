// Device-side definitions of the HRPP library: layouts, launch parameters and
// the per-ray arithmetic (Sec. 5 hash, table index, slab test, Moller-Trumbore).
//
// Every floating-point step below is written with an explicitly rounded
// intrinsic (__fmul_rn, __fadd_rn, __fsub_rn, __fmaf_rn, __frcp_rn), so the
// compiler cannot contract or reorder it: a given ray and triangle always give
// the same bits.
#pragma once

#include <cstdint>

#include "hrpp.h"

namespace hrpp {

constexpr int kTagBits = 36;
constexpr int kLeafBits = 28;
constexpr uint64_t kLeafMask = (1ull << kLeafBits) - 1ull;
constexpr uint64_t kTagMask = (1ull << kTagBits) - 1ull;
constexpr uint64_t kM48 = (1ull << 48) - 1ull;
constexpr int32_t kEmptyRef = INT32_MIN;  // no child in this slot
constexpr int kStack = HRPP_MAX_STACK;

// error bits of a scene's sticky device flag
constexpr uint32_t kErrStack = 1u;
constexpr uint32_t kErrSteps = 2u;

// statistics slots (hrpp_stats order)
enum Stat : int {
    ST_RAYS, ST_HITS, ST_LOOKUPS, ST_POSITIVES, ST_TRUE_POS, ST_FALSE_POS, ST_NEGATIVES, ST_TP_INEXACT,
    ST_INSERTS, ST_DUP_INSERTS, ST_EVICTIONS, ST_INTERIOR, ST_BOX_TESTS, ST_LEAVES, ST_TRI_TESTS,
    ST_PRED_LEAVES, ST_PRED_TRI_TESTS, ST_PRED_INTERIOR, ST_PRED_BOX_TESTS, ST_GATED, ST_N = 20
};

// Per-call device control block: the ray pool's cursor and the two-pass
// schedule's queue length (both restarted for every chunk of a staged call),
// the insert-record count, the table gate's counts (rays that consulted the
// table, and the true positives among them) and the statistics.  Zeroed
// before each call.
struct __align__(16) Ctl {
    unsigned int next_ray;
    unsigned int queue_len;
    unsigned int n_records;
    unsigned int gate_lookups;
    unsigned int gate_tp;
    unsigned int pad[3];
    unsigned long long stats[ST_N];
};
static_assert(sizeof(Ctl) <= 256, "the control block has 256 bytes of scratch");

// A table's gate word: nonzero = open (every ray consults the table), zero =
// closed (only the sampled 32-ray chunks do).
__device__ __forceinline__ bool gate_admits(const uint32_t *gate, uint32_t gate_mask, uint32_t ray)
{
    return gate == nullptr || ((ray >> 5) & gate_mask) == 0u || __ldg(gate) != 0u;
}

// After a call: the gate opens iff the call's true positives reach
// min_tp / 65536 of the rays that consulted the table; a call in which no ray
// consulted it leaves the gate as it was.
__device__ __forceinline__ void gate_decide(uint32_t *gate, uint32_t min_tp, const Ctl *ctl)
{
    const uint32_t look = ctl->gate_lookups, tp = ctl->gate_tp;
    if (look) *gate = ((uint64_t)tp << 16) >= (uint64_t)min_tp * look ? 1u : 0u;
}

// Two-phase insert record: table slot, ray index + 1, table word.
struct __align__(16) Record {
    uint32_t slot;
    uint32_t ray1;
    uint64_t word;
};

struct TraceParams {
    const float4 *nodes;     // width 2: 4 float4 per node; width 4: 8 float4 per node
    const float4 *tris;      // 3 float4 per triangle: (v0, prim bits), (v1 - v0), (v2 - v0)
    uint32_t n_tris;
    int32_t root_ref;        // >= 0 interior node, else ~leaf
    uint32_t max_steps;      // traversal steps per ray before the ray is stopped
    const float4 *rays;      // 2 float4 per ray
    uint32_t n_rays;
    void *hits;              // hrpp_hit[n] (closest) or uint32_t[n] (any)
    uint64_t *table;         // table words (NULL: plain traversal)
    uint32_t *winner;        // two-phase: highest ray index + 1 per slot
    Record *records;         // two-phase insert records
    int log2_sets, log2_ways, precision, update_mode;
    Ctl *ctl;
    uint32_t *error;         // scene's sticky error flag
    uint32_t refill_min;     // dynamic schedule: refill when this many lanes are idle
    int go_up;               // Go Up Level (Sec. 6.2): 0 = leaves are predicted
    uint32_t n_interior;
    const int32_t *parent;       // interior node -> parent (-1 at the root)
    const int32_t *leaf_parent;  // leaf's first prim_index slot -> parent (-1: root leaf)
    int closest;                 // batched launches: this item's query mode
    const int32_t *predicted;    // per ray: canonical node whose subtree is traversed first (-1: none)
    const int32_t *canon_ref;    // canonical node -> device ref
    uint32_t n_nodes;            // canonical node count
    int verify;                  // closest-hit true positives: 0 root traversal, 1 bottom-up climb
    int hash_variant;            // 0: exponent MSBs (Sec. 5), 1: exponent LSBs
    uint8_t *ray_outcome;        // per ray (statistics launches only; may be null)
    uint32_t *ray_box_tests;     // per ray (statistics launches only; may be null)
    uint32_t *gate;              // the table's gate word (null: no gate, every ray consults the table)
    uint32_t gate_mask;          // closed gate: 32-ray chunks c with (c & gate_mask) == 0 still consult it
    uint32_t gate_min_tp;        // true positives per 65536 lookups that keep the gate open
    uint32_t ray_offset;         // index of this launch's first ray in its call (a multiple of 32): rays,
                                 // hits and per-ray arrays start there, while insert order, the gate's
                                 // chunks and the online way use the call's ray index i + ray_offset
};

// 32 bytes through the read-only data path in one load (p 32-byte aligned):
// a BVH node arrives in 4 (4-wide) or 2 (binary) loads per lane instead of 8
// or 4 16-byte ones.
__device__ __forceinline__ void ldg32(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// ---------------------------------------------------------------- hashing --

// Sec. 5: sign bit, then the p most significant exponent bits, then the p most
// significant mantissa bits of the float's IEEE-754 encoding.  lsb: the
// tuning variant that keeps the p least significant exponent bits instead.
__device__ __forceinline__ uint32_t hash_float(float f, int p, bool lsb)
{
    const uint32_t b = __float_as_uint(f);
    // the p exponent bits in one shift and mask: the MSBs are bits 30..31-p
    // (shifting by 31 - p also brings the sign down, above them, and the
    // mask drops it); the LSBs are bits 23+p-1..23
    const uint32_t e = (b >> (lsb ? 23 : 31 - p)) & ((1u << p) - 1u);
    return ((b >> 31) << (2 * p)) | (e << p) | ((b & 0x7FFFFFu) >> (23 - p));
}

// Sec. 5: origin hashes XOR the swizzled direction hashes (o.x^d.z, o.y^d.y,
// o.z^d.x), packed into 16-bit fields of a 48-bit key.
__device__ __forceinline__ uint64_t ray_key(float4 o, float4 d, int p, bool lsb = false)
{
    const uint64_t h0 = hash_float(o.x, p, lsb) ^ hash_float(d.z, p, lsb);
    const uint64_t h1 = hash_float(o.y, p, lsb) ^ hash_float(d.y, p, lsb);
    const uint64_t h2 = hash_float(o.z, p, lsb) ^ hash_float(d.x, p, lsb);
    return h0 | (h1 << 16) | (h2 << 32);
}

// Bijection of 48-bit keys; its low bits pick the set, the rest is the tag.
__device__ __forceinline__ uint64_t mix48(uint64_t k)
{
    k &= kM48;
    k ^= k >> 23;
    k = (k * 0x9E3779B97F4Bull) & kM48;
    k ^= k >> 25;
    k = (k * 0xC2B2AE3D27D5ull) & kM48;
    k ^= k >> 21;
    return k;
}

__device__ __forceinline__ uint32_t way_of(uint32_t leaf, int log2_ways)
{
    return log2_ways == 0 ? 0u : (leaf * 0x9E3779B1u) >> (32 - log2_ways);
}

// ---------------------------------------------------------------- geometry --

struct RayInv {
    float ix, iy, iz;     // reciprocal direction
    float oix, oiy, oiz;  // origin * reciprocal direction
};

__device__ __forceinline__ float safe_rcp(float d)
{
    // |d| < 2^-80 -> copysign(2^-80, d): keeps the reciprocal finite
    const float m = 0x1p-80f;
    if (fabsf(d) < m) d = copysignf(m, d);
    return __frcp_rn(d);
}

__device__ __forceinline__ RayInv ray_inverse(float4 o, float4 d)
{
    RayInv r;
    r.ix = safe_rcp(d.x);
    r.iy = safe_rcp(d.y);
    r.iz = safe_rcp(d.z);
    r.oix = __fmul_rn(o.x, r.ix);
    r.oiy = __fmul_rn(o.y, r.iy);
    r.oiz = __fmul_rn(o.z, r.iz);
    return r;
}

// three-input min / max (one instruction each on sm_100 and later); for
// non-NaN inputs they equal the two-input forms applied twice
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Slab test: plane distances lo*inv - o*inv (one fused multiply-add each);
// entry = max(tmin, nearest planes), exit = min(tcur, farthest planes).
// Plane distances are finite (the reciprocal is), so no operand is NaN.
__device__ __forceinline__ bool slab(const RayInv &r, float tmin, float tcur, float lox, float hix, float loy,
                                     float hiy, float loz, float hiz, float &tn)
{
    const float x0 = __fmaf_rn(lox, r.ix, -r.oix), x1 = __fmaf_rn(hix, r.ix, -r.oix);
    const float y0 = __fmaf_rn(loy, r.iy, -r.oiy), y1 = __fmaf_rn(hiy, r.iy, -r.oiy);
    const float z0 = __fmaf_rn(loz, r.iz, -r.oiz), z1 = __fmaf_rn(hiz, r.iz, -r.oiz);
    tn = max3f(fminf(x0, x1), fminf(y0, y1), fmaxf(fminf(z0, z1), tmin));
    const float tf = min3f(fmaxf(x0, x1), fmaxf(y0, y1), fminf(fmaxf(z0, z1), tcur));
    return tn <= tf;
}

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz)
{
    return __fmaf_rn(ax, bx, __fmaf_rn(ay, by, __fmul_rn(az, bz)));
}

// Moller-Trumbore on a stored triangle (v0, e1 = v1 - v0, e2 = v2 - v0).
// Valid iff det != 0, u in [0,1], v >= 0, u + v <= 1, tmin < t < tmax.
__device__ __forceinline__ bool tri_test(float4 o, float4 d, float4 v0, float4 e1, float4 e2, float &t_out,
                                         float &u_out, float &v_out)
{
    // p = d x e2
    const float px = __fmaf_rn(d.y, e2.z, -__fmul_rn(d.z, e2.y));
    const float py = __fmaf_rn(d.z, e2.x, -__fmul_rn(d.x, e2.z));
    const float pz = __fmaf_rn(d.x, e2.y, -__fmul_rn(d.y, e2.x));
    const float det = dot3(e1.x, e1.y, e1.z, px, py, pz);
    if (det == 0.0f) return false;
    const float inv = __frcp_rn(det);
    const float sx = __fsub_rn(o.x, v0.x), sy = __fsub_rn(o.y, v0.y), sz = __fsub_rn(o.z, v0.z);
    const float u = __fmul_rn(dot3(sx, sy, sz, px, py, pz), inv);
    // q = s x e1
    const float qx = __fmaf_rn(sy, e1.z, -__fmul_rn(sz, e1.y));
    const float qy = __fmaf_rn(sz, e1.x, -__fmul_rn(sx, e1.z));
    const float qz = __fmaf_rn(sx, e1.y, -__fmul_rn(sy, e1.x));
    const float v = __fmul_rn(dot3(d.x, d.y, d.z, qx, qy, qz), inv);
    const float t = __fmul_rn(dot3(e2.x, e2.y, e2.z, qx, qy, qz), inv);
    if (!(u >= 0.0f && u <= 1.0f && v >= 0.0f && __fadd_rn(u, v) <= 1.0f && t > o.w && t < d.w)) return false;
    t_out = t;
    u_out = u;
    v_out = v;
    return true;
}

// A device range whose L2 hits the traversal launch marks persisting (an
// access-policy window on the launch; it takes effect only while the context
// has a persisting-L2 set-aside).
struct L2Window {
    const void *base;
    size_t bytes;
};

// host launchers (trace_bvh2.cu, trace_bvh4.cu, table.cu)
// schedule: 0 = each warp traces 32 rays to completion before taking the next
// 32; 1 = lanes that finish take new rays while the others keep traversing
cudaError_t launch_trace_w2(bool closest, bool stats, int schedule, const TraceParams &p, int block_threads,
                            int blocks_per_sm_cap, cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1,
                            const L2Window *l2 = nullptr);
cudaError_t launch_trace_w4(bool closest, bool stats, int schedule, const TraceParams &p, int block_threads,
                            int blocks_per_sm_cap, cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1,
                            const L2Window *l2 = nullptr);
// two-pass schedule (compact.cuh): k_predict, then k_trace_queue over the
// queue (16 bytes per ray of scratch, 16-byte aligned)
cudaError_t launch_compact_w2(bool closest, bool stats, const TraceParams &p, void *queue, int block_threads,
                              cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1);
cudaError_t launch_compact_w4(bool closest, bool stats, const TraceParams &p, void *queue, int block_threads,
                              cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1);
cudaError_t launch_table_apply(uint64_t *table, uint32_t *winner, const Record *records, Ctl *ctl,
                               uint32_t max_records, cudaStream_t stream, uint32_t *gate = nullptr,
                               uint32_t gate_min_tp = 0);
// the gate decision alone (tables whose updates need no k_apply)
cudaError_t launch_gate_update(uint32_t *gate, uint32_t gate_min_tp, const Ctl *ctl, cudaStream_t stream);
// batched launches (batch.cu): every item of one BVH width in one kernel, then
// the two-phase updates of every item's table in one kernel
struct BatchDesc {
    const TraceParams *items;    // per item; ctl/records point at the item's own scratch
    const uint32_t *chunk_item;  // item of each chunk
    const uint32_t *chunk_first; // first ray (within its item) of each chunk
    uint32_t n_chunks;
    unsigned int *cursor;        // the batch's chunk cursor (zeroed before each run)
};


// one launch per query mode: every chunk of b belongs to items of that mode
cudaError_t launch_batch_w2(bool closest, bool stats, const BatchDesc &b, int block_threads, cudaStream_t stream);
cudaError_t launch_batch_w4(bool closest, bool stats, const BatchDesc &b, int block_threads, cudaStream_t stream);
cudaError_t launch_table_apply_batch(const TraceParams *items, uint32_t n_items, uint32_t max_records,
                                     cudaStream_t stream);
cudaError_t launch_table_fill(uint64_t *words, uint64_t n_words, cudaStream_t stream);

}  // namespace hrpp
