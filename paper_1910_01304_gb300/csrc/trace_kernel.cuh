// Persistent HRPP traversal kernel (one template, instantiated per BVH width,
// query mode and statistics switch in trace_bvh2.cu / trace_bvh4.cu).
//
// Each warp repeatedly takes the next 32 rays from the call's ray pool (one
// atomic per warp on Ctl::next_ray) and traces one ray per lane:
//   1. HRPP lookup (Sec. 4.2, Sec. 5): hash the ray, read its set, collect the
//      ways whose tag matches; test those predicted leaves' triangles.
//   2. Outcome (Sec. 4.3): no prediction -> negative; a predicted leaf holds a
//      valid hit -> true positive (any-hit rays are done, no interior node is
//      touched); otherwise false positive.
//   3. Traversal from the root unless an any-hit ray is done.  Closest-hit
//      true positives traverse with the predicted hit as the initial bound,
//      so the answer stays exact.  Children are visited nearest first, ties
//      by slot; the stack lives in local memory (HRPP_MAX_STACK entries).
//   4. A ray whose traversal produced its final hit inserts that hit's leaf:
//      two-phase mode records it (atomicMax on the slot's winner + a record
//      appended with one atomic per warp); online mode exchanges the word.
#pragma once

#include <cuda_runtime.h>

#include "device.cuh"

namespace hrpp {

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// order-preserving float -> unsigned map (for (entry t, slot) sort keys);
// -0 is folded into +0 first so equal distances compare equal
__device__ __forceinline__ uint32_t ordered(float f)
{
    const uint32_t b = __float_as_uint(__fadd_rn(f, 0.0f));
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ void cswap(uint64_t &a, uint64_t &b)
{
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

__device__ __forceinline__ int32_t pick4(int4 c, uint32_t s)
{
    return s == 0 ? c.x : s == 1 ? c.y : s == 2 ? c.z : c.w;
}

template <bool STATS>
struct Counters {
    uint32_t c[ST_N];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int k = 0; k < ST_N; ++k) c[k] = 0;
    }
    __device__ __forceinline__ void add(int k, uint32_t v = 1)
    {
        if (STATS) c[k] += v;
    }
};

struct Best {
    float t, u, v;
    uint32_t prim, leaf;
    bool found, from_trav;
};

// Tests the triangles of one leaf.  Any-hit: returns true at the first valid
// hit.  Closest: keeps the lexicographic minimum (t, prim).
template <bool CLOSEST, bool STATS>
__device__ __forceinline__ bool test_leaf(const TraceParams &p, uint32_t leaf, float4 o, float4 d, Best &b,
                                          float &tcur, bool in_traversal, Counters<STATS> &cnt, int tri_stat)
{
    const uint32_t first = leaf >> 2, count = (leaf & 3u) + 1u;
    const float4 *tr = p.tris + 3ull * first;
    for (uint32_t j = 0; j < count; ++j) {
        const float4 v0 = __ldg(tr + 3 * j), e1 = __ldg(tr + 3 * j + 1), e2 = __ldg(tr + 3 * j + 2);
        cnt.add(tri_stat);
        float t, u, v;
        if (!tri_test(o, d, v0, e1, e2, t, u, v)) continue;
        const uint32_t prim = __float_as_uint(v0.w);
        if (!CLOSEST) {
            b.t = t; b.u = u; b.v = v; b.prim = prim; b.leaf = leaf;
            b.found = true;
            b.from_trav = in_traversal;
            return true;
        }
        if (!b.found || t < b.t || (t == b.t && prim < b.prim)) {
            b.t = t; b.u = u; b.v = v; b.prim = prim; b.leaf = leaf;
            b.found = true;
            b.from_trav = in_traversal;
            tcur = t;
        }
    }
    return false;
}

template <int W, bool CLOSEST, bool STATS>
__device__ __forceinline__ void traverse(const TraceParams &p, float4 o, float4 d, Best &b, Counters<STATS> &cnt)
{
    const RayInv ri = ray_inverse(o, d);
    float tcur = (CLOSEST && b.found) ? b.t : d.w;
    int32_t stack[kStack];
    int sp = 0;
    int32_t ref = p.root_ref;
    uint32_t steps = 0;
    for (;;) {
        if (++steps > p.max_steps) {
            atomicOr(p.error, kErrSteps);
            return;
        }
        if (ref >= 0) {
            cnt.add(ST_INTERIOR);
            if (W == 2) {
                const float4 *n = p.nodes + 4ull * (uint32_t)ref;
                const float4 a = __ldg(n), bb = __ldg(n + 1), c = __ldg(n + 2);
                const int4 e = __ldg(reinterpret_cast<const int4 *>(n + 3));
                float t0, t1;
                const bool h0 = slab(ri, o.w, tcur, a.x, a.y, a.z, a.w, c.x, c.y, t0);
                const bool v1 = e.y != kEmptyRef;
                const bool h1 = v1 && slab(ri, o.w, tcur, bb.x, bb.y, bb.z, bb.w, c.z, c.w, t1);
                cnt.add(ST_BOX_TESTS, 1u + (v1 ? 1u : 0u));
                if (h0 && h1) {
                    const bool swap = t1 < t0;
                    if (sp >= kStack) {
                        atomicOr(p.error, kErrStack);
                        return;
                    }
                    stack[sp++] = swap ? e.x : e.y;
                    ref = swap ? e.y : e.x;
                    continue;
                }
                if (h0) { ref = e.x; continue; }
                if (h1) { ref = e.y; continue; }
            } else {
                const float4 *n = p.nodes + 8ull * (uint32_t)ref;
                const float4 lx = __ldg(n), hx = __ldg(n + 1), ly = __ldg(n + 2), hy = __ldg(n + 3);
                const float4 lz = __ldg(n + 4), hz = __ldg(n + 5);
                const int4 ch = __ldg(reinterpret_cast<const int4 *>(n + 6));
                uint64_t k0 = ~0ull, k1 = ~0ull, k2 = ~0ull, k3 = ~0ull;
                float t;
                uint32_t nvalid = 0, nhit = 0;
                if (ch.x != kEmptyRef) {
                    ++nvalid;
                    if (slab(ri, o.w, tcur, lx.x, hx.x, ly.x, hy.x, lz.x, hz.x, t)) { k0 = ((uint64_t)ordered(t) << 2) | 0u; ++nhit; }
                }
                if (ch.y != kEmptyRef) {
                    ++nvalid;
                    if (slab(ri, o.w, tcur, lx.y, hx.y, ly.y, hy.y, lz.y, hz.y, t)) { k1 = ((uint64_t)ordered(t) << 2) | 1u; ++nhit; }
                }
                if (ch.z != kEmptyRef) {
                    ++nvalid;
                    if (slab(ri, o.w, tcur, lx.z, hx.z, ly.z, hy.z, lz.z, hz.z, t)) { k2 = ((uint64_t)ordered(t) << 2) | 2u; ++nhit; }
                }
                if (ch.w != kEmptyRef) {
                    ++nvalid;
                    if (slab(ri, o.w, tcur, lx.w, hx.w, ly.w, hy.w, lz.w, hz.w, t)) { k3 = ((uint64_t)ordered(t) << 2) | 3u; ++nhit; }
                }
                cnt.add(ST_BOX_TESTS, nvalid);
                if (nhit > 0) {
                    // sort (entry t, slot) ascending: 5 compare-exchanges
                    cswap(k0, k1);
                    cswap(k2, k3);
                    cswap(k0, k2);
                    cswap(k1, k3);
                    cswap(k1, k2);
                    if (sp + (int)nhit - 1 > kStack) {
                        atomicOr(p.error, kErrStack);
                        return;
                    }
                    if (nhit > 3) stack[sp++] = pick4(ch, (uint32_t)k3 & 3u);
                    if (nhit > 2) stack[sp++] = pick4(ch, (uint32_t)k2 & 3u);
                    if (nhit > 1) stack[sp++] = pick4(ch, (uint32_t)k1 & 3u);
                    ref = pick4(ch, (uint32_t)k0 & 3u);
                    continue;
                }
            }
        } else {
            // leaf
            cnt.add(ST_LEAVES);
            if (test_leaf<CLOSEST, STATS>(p, ~(uint32_t)ref, o, d, b, tcur, true, cnt, ST_TRI_TESTS)) return;
        }
        if (sp == 0) return;
        ref = stack[--sp];
    }
}

template <int W, bool CLOSEST, bool STATS>
__global__ void __launch_bounds__(512) k_trace(const TraceParams p)
{
    const uint32_t lane = threadIdx.x & 31u;
    Counters<STATS> cnt;
    cnt.init();
    const bool hrpp = p.table != nullptr;
    const uint32_t ways = 1u << p.log2_ways;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&p.ctl->next_ray, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= p.n_rays) break;
        const uint32_t i = base + lane;
        bool want_insert = false;
        uint32_t slot = 0;
        uint64_t word = 0;
        if (i < p.n_rays) {
            const float4 o = __ldg(p.rays + 2ull * i), d = __ldg(p.rays + 2ull * i + 1);
            Best b;
            b.t = __int_as_float(0x7F800000);
            b.u = b.v = 0.0f;
            b.prim = HRPP_NO_HIT;
            b.leaf = 0;
            b.found = b.from_trav = false;
            cnt.add(ST_RAYS);
            bool run_traversal = true;
            bool positive = false;
            uint64_t set = 0, tag = 0;
            if (hrpp) {
                cnt.add(ST_LOOKUPS);
                const uint64_t m = mix48(ray_key(o, d, p.precision));
                set = m & ((1ull << p.log2_sets) - 1ull);
                tag = (m >> p.log2_sets) & kTagMask;
                const uint64_t *s = p.table + (set << p.log2_ways);
                float tdummy = 0.0f;
                bool done = false;
                for (uint32_t w = 0; w < ways && !done; ++w) {
                    const uint64_t wd = p.update_mode == HRPP_UPDATE_ONLINE ? __ldcg(s + w) : __ldg(s + w);
                    if (wd == HRPP_EMPTY_WORD || (wd >> kLeafBits) != tag) continue;
                    positive = true;
                    const uint32_t leaf = (uint32_t)(wd & kLeafMask);
                    if ((leaf >> 2) + (leaf & 3u) + 1u > p.n_tris) continue;  // not a leaf of this scene
                    cnt.add(ST_PRED_LEAVES);
                    done = test_leaf<CLOSEST, STATS>(p, leaf, o, d, b, tdummy, false, cnt, ST_PRED_TRI_TESTS);
                }
                if (!positive) {
                    cnt.add(ST_NEGATIVES);
                } else {
                    cnt.add(ST_POSITIVES);
                    if (b.found) {
                        cnt.add(ST_TRUE_POS);
                        if (!CLOSEST) run_traversal = false;
                    } else {
                        cnt.add(ST_FALSE_POS);
                    }
                }
            }
            if (run_traversal) {
                const bool predicted_hit = b.found;
                traverse<W, CLOSEST, STATS>(p, o, d, b, cnt);
                if (CLOSEST && predicted_hit && b.from_trav) cnt.add(ST_TP_INEXACT);
                if (hrpp && b.from_trav && p.update_mode != HRPP_UPDATE_FROZEN) {
                    cnt.add(ST_INSERTS);
                    slot = (uint32_t)((set << p.log2_ways) | way_of(b.leaf, p.log2_ways));
                    word = (tag << kLeafBits) | b.leaf;
                    if (p.update_mode == HRPP_UPDATE_ONLINE) {
                        const unsigned long long old =
                            atomicExch(reinterpret_cast<unsigned long long *>(p.table + slot), word);
                        if (old == word) cnt.add(ST_DUP_INSERTS);
                        else if (old != HRPP_EMPTY_WORD) cnt.add(ST_EVICTIONS);
                    } else {
                        atomicMax(p.winner + slot, i + 1u);
                        want_insert = true;
                    }
                }
            }
            if (b.found) cnt.add(ST_HITS);
            if (CLOSEST) {
                reinterpret_cast<float4 *>(p.hits)[i] = make_float4(b.t, __uint_as_float(b.prim), b.u, b.v);
            } else {
                reinterpret_cast<uint32_t *>(p.hits)[i] = b.found ? b.prim : HRPP_NO_HIT;
            }
        }
        // two-phase insert records: one atomic per warp
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, want_insert);
        if (m) {
            const uint32_t leader = __ffs(m) - 1;
            uint32_t rb = 0;
            if (lane == leader) rb = atomicAdd(&p.ctl->n_records, (uint32_t)__popc(m));
            rb = __shfl_sync(0xFFFFFFFFu, rb, leader);
            if (want_insert) {
                Record r;
                r.slot = slot;
                r.ray1 = i + 1u;
                r.word = word;
                p.records[rb + __popc(m & lanemask_lt())] = r;
            }
        }
    }
    if (STATS) {
#pragma unroll
        for (int k = 0; k < ST_PRED_TRI_TESTS + 1; ++k) {
            const uint32_t v = __reduce_add_sync(0xFFFFFFFFu, cnt.c[k]);
            if (lane == 0 && v) atomicAdd(&p.ctl->stats[k], (unsigned long long)v);
        }
    }
}

template <int W>
cudaError_t launch_width(bool closest, bool stats, const TraceParams &p, int block_threads, int blocks_per_sm_cap,
                         cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1)
{
    const void *fn;
    if (closest) fn = stats ? (const void *)k_trace<W, true, true> : (const void *)k_trace<W, true, false>;
    else fn = stats ? (const void *)k_trace<W, false, true> : (const void *)k_trace<W, false, false>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block_threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm_cap > 0 && per_sm > blocks_per_sm_cap) per_sm = blocks_per_sm_cap;
    // never more warps than 32-ray batches
    const uint64_t warps_needed = (p.n_rays + 31ull) / 32ull;
    uint64_t blocks = (uint64_t)sms * per_sm;
    const uint64_t warps_per_block = block_threads / 32;
    if (blocks * warps_per_block > warps_needed) blocks = (warps_needed + warps_per_block - 1) / warps_per_block;
    if (blocks < 1) blocks = 1;
    if (ev0) cudaEventRecord(ev0, stream);
    void *args[] = {(void *)&p};
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(block_threads), args, 0, stream);
    if (ev1) cudaEventRecord(ev1, stream);
    return e;
}

}  // namespace hrpp
