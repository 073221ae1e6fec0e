// Persistent HRPP traversal kernels (templates instantiated per BVH width,
// query mode and statistics switch in trace_bvh2.cu / trace_bvh4.cu).
//
// Per ray:
//   1. HRPP lookup (Sec. 4.2, Sec. 5): hash the ray, read its set, collect the
//      ways whose tag matches; test those predicted leaves' triangles.
//   2. Outcome (Sec. 4.3): no prediction -> negative; a predicted leaf holds a
//      valid hit -> true positive (any-hit rays are done, no interior node is
//      touched); otherwise false positive.
//   3. Traversal from the root unless an any-hit ray is done.  Closest-hit
//      true positives traverse with the predicted hit as the initial bound,
//      so the answer stays exact; or (bottom-up verification) they climb from
//      the predicted hit's leaf to the root and traverse only the siblings
//      met on the way.  Children are visited nearest first, ties by slot; the
//      stack lives in local memory (HRPP_MAX_STACK entries).
//   4. A ray whose traversal produced its final hit inserts that hit's leaf:
//      two-phase mode records it (atomicMax on the slot's winner + a record
//      appended with one atomic per warp); online mode claims a way by CAS.
//
// Two schedules over the ray pool (Ctl::next_ray), identical per-ray work:
//   k_trace      a warp takes 32 rays, traces them to completion, repeats.
//   k_trace_dyn  lanes whose ray finished take new rays (one atomic per warp
//                for all of them) once refill_min lanes are idle, while the
//                other lanes keep traversing; every iteration each lane visits
//                one node, as in k_trace, between two warp votes (refill,
//                finished rays).
#pragma once

#include <cuda_runtime.h>

#include <cstring>

#include "device.cuh"

namespace hrpp {

constexpr int32_t kDoneRef = INT32_MIN + 1;  // traversal finished
constexpr int kMaxWarps = 16;                // warps per block (512 threads)
constexpr uint32_t kNoRay = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
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
    __device__ __forceinline__ void flush(Ctl *ctl, uint32_t lane)
    {
        if (STATS) {
#pragma unroll
            for (int k = 0; k < ST_N; ++k) {
                const uint32_t v = __reduce_add_sync(0xFFFFFFFFu, c[k]);
                if (lane == 0 && v) atomicAdd(&ctl->stats[k], (unsigned long long)v);
            }
        }
    }
};

// Gate counts of the rays a warp just finished (all 32 lanes call this
// together): gflags bit 0 = the ray consulted the table, bit 1 = it was a
// true positive.  Two warp votes, summed by lane 0 into the warp's own
// shared-memory slot (no register stays live across the traversal, and no
// global atomic per chunk); gate_flush adds the slot to the call's counts.
constexpr uint32_t kGateLooked = 1u, kGateTp = 2u;

__device__ __forceinline__ void gate_count(const TraceParams &p, uint32_t lane, uint32_t gflags, uint2 &acc)
{
    if (!p.gate) return;  // warp-uniform
    const uint32_t l = __popc(__ballot_sync(0xFFFFFFFFu, gflags & kGateLooked));
    const uint32_t t = __popc(__ballot_sync(0xFFFFFFFFu, gflags & kGateTp));
    if (lane == 0) {
        acc.x += l;
        acc.y += t;
    }
}

__device__ __forceinline__ void gate_flush(const TraceParams &p, uint32_t lane, uint2 &acc)
{
    if (lane == 0) {
        if (p.gate && acc.x) atomicAdd(&p.ctl->gate_lookups, acc.x);
        if (p.gate && acc.y) atomicAdd(&p.ctl->gate_tp, acc.y);
        acc = make_uint2(0u, 0u);
    }
    __syncwarp();
}

struct Best {
    float t, u, v;
    uint32_t prim, leaf;
    bool found, from_trav;
};

// Everything one lane keeps about its ray between traversal rounds.
struct RayState {
    float4 o, d;
    RayInv ri;
    float tcur;
    Best b;
    int sp;
    int32_t ref;
    uint32_t steps;
    bool predicted_hit;
    uint32_t set;
    uint64_t tag;
    int32_t from;      // bottom-up verification: the ref the climb is at (kDoneRef: not climbing)
    bool climb_visit;  // the next interior visit is the climb's ancestor (then from moves up)
    uint8_t outcome;   // HRPP_OUTCOME_* (written out by statistics launches)
    uint32_t box0;     // the lane's box-test counter when this ray's traversal began
};

// Tests triangle j of a leaf (triangles from tr).  Any-hit: returns true at a
// valid hit.  Closest: keeps the lexicographic minimum (t, prim).
template <bool CLOSEST, bool STATS>
__device__ __forceinline__ bool test_tri(const float4 *tr, uint32_t j, uint32_t leaf, float4 o, float4 d, Best &b,
                                         float &tcur, bool in_traversal, Counters<STATS> &cnt, int tri_stat)
{
    const float4 v0 = __ldg(tr + 3 * j), e1 = __ldg(tr + 3 * j + 1), e2 = __ldg(tr + 3 * j + 2);
    cnt.add(tri_stat);
    float t, u, v;
    if (!tri_test(o, d, v0, e1, e2, t, u, v)) return false;
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
    return false;
}

// Tests the triangles of one leaf in order.  Any-hit: returns true at the
// first valid hit.  The closest-hit loop is unrolled over the (at most 4)
// triangles, which measured faster for closest-hit rays and slower for
// any-hit rays.
template <bool CLOSEST, bool STATS>
__device__ __forceinline__ bool test_leaf(const TraceParams &p, uint32_t leaf, float4 o, float4 d, Best &b,
                                          float &tcur, bool in_traversal, Counters<STATS> &cnt, int tri_stat)
{
    const uint32_t first = leaf >> 2, count = (leaf & 3u) + 1u;
    const float4 *tr = p.tris + 3ull * first;
    if constexpr (CLOSEST) {
#pragma unroll
        for (uint32_t j = 0; j < (uint32_t)HRPP_MAX_LEAF_TRIS; ++j) {
            if (j >= count) break;
            test_tri<CLOSEST, STATS>(tr, j, leaf, o, d, b, tcur, in_traversal, cnt, tri_stat);
        }
        return false;
    } else {
        for (uint32_t j = 0; j < count; ++j)
            if (test_tri<CLOSEST, STATS>(tr, j, leaf, o, d, b, tcur, in_traversal, cnt, tri_stat)) return true;
        return false;
    }
}

__device__ __forceinline__ int32_t pop(int32_t *stack, int &sp) { return sp > 0 ? stack[--sp] : kDoneRef; }

// Visits the interior node s.ref: tests its children's boxes against the
// current bound and moves to the nearest hit child, pushing the others
// (farthest deepest); with no hit child it pops.
// PRED: the node belongs to a predicted subtree (Go Up Level > 0), counted
// apart from the traversal from the root.  SKIP: the child ref `skip` is
// left out (the child a bottom-up climb came from).
template <int W, bool STATS, bool PRED = false, bool SKIP = false>
__device__ __forceinline__ void visit_interior(const TraceParams &p, RayState &s, int32_t *stack, Counters<STATS> &cnt,
                                               int32_t skip = kDoneRef)
{
    constexpr int kBoxStat = PRED ? ST_PRED_BOX_TESTS : ST_BOX_TESTS;
    cnt.add(PRED ? ST_PRED_INTERIOR : ST_INTERIOR);
    const float tmin = s.o.w;
    if (W == 2) {
        const float4 *n = p.nodes + 4ull * (uint32_t)s.ref;
        float4 a, bb, c, ef;
        ldg32(n, a, bb);
        ldg32(n + 2, c, ef);
        const int4 e = make_int4(__float_as_int(ef.x), __float_as_int(ef.y), __float_as_int(ef.z), __float_as_int(ef.w));
        float t0, t1;
        const bool v0 = !SKIP || e.x != skip;
        const bool h0 = v0 && slab(s.ri, tmin, s.tcur, a.x, a.y, a.z, a.w, c.x, c.y, t0);
        const bool v1 = e.y != kEmptyRef && (!SKIP || e.y != skip);
        const bool h1 = v1 && slab(s.ri, tmin, s.tcur, bb.x, bb.y, bb.z, bb.w, c.z, c.w, t1);
        cnt.add(kBoxStat, (v0 ? 1u : 0u) + (v1 ? 1u : 0u));
        if (h0 && h1) {
            if (s.sp >= kStack) {
                atomicOr(p.error, kErrStack);
                s.ref = kDoneRef;
                return;
            }
            const bool swap = t1 < t0;
            stack[s.sp++] = swap ? e.x : e.y;
            s.ref = swap ? e.y : e.x;
        } else if (h0) {
            s.ref = e.x;
        } else if (h1) {
            s.ref = e.y;
        } else {
            s.ref = pop(stack, s.sp);
        }
        return;
    }
    const float4 *n = p.nodes + 8ull * (uint32_t)s.ref;
    float4 lx, hx, ly, hy, lz, hz, cf, spare;
    ldg32(n, lx, hx);
    ldg32(n + 2, ly, hy);
    ldg32(n + 4, lz, hz);
    ldg32(n + 6, cf, spare);  // children, then the parent row (unused here)
    const int4 ch = make_int4(__float_as_int(cf.x), __float_as_int(cf.y), __float_as_int(cf.z), __float_as_int(cf.w));
    const float inf = __int_as_float(0x7F800000);
    float t0 = inf, t1 = inf, t2 = inf, t3 = inf, t;
    bool h0 = false, h1 = false, h2 = false, h3 = false;
    uint32_t nvalid = 0;
    if (ch.x != kEmptyRef && (!SKIP || ch.x != skip)) { ++nvalid; if ((h0 = slab(s.ri, tmin, s.tcur, lx.x, hx.x, ly.x, hy.x, lz.x, hz.x, t))) t0 = t; }
    if (ch.y != kEmptyRef && (!SKIP || ch.y != skip)) { ++nvalid; if ((h1 = slab(s.ri, tmin, s.tcur, lx.y, hx.y, ly.y, hy.y, lz.y, hz.y, t))) t1 = t; }
    if (ch.z != kEmptyRef && (!SKIP || ch.z != skip)) { ++nvalid; if ((h2 = slab(s.ri, tmin, s.tcur, lx.z, hx.z, ly.z, hy.z, lz.z, hz.z, t))) t2 = t; }
    if (ch.w != kEmptyRef && (!SKIP || ch.w != skip)) { ++nvalid; if ((h3 = slab(s.ri, tmin, s.tcur, lx.w, hx.w, ly.w, hy.w, lz.w, hz.w, t))) t3 = t; }
    cnt.add(kBoxStat, nvalid);
    const int nhit = (int)h0 + (int)h1 + (int)h2 + (int)h3;
    if (nhit == 0) {
        s.ref = pop(stack, s.sp);
        return;
    }
    if (nhit == 1) {  // one hit child (most visits of short rays): nothing to order or push
        s.ref = h0 ? ch.x : (h1 ? ch.y : (h2 ? ch.z : ch.w));
        return;
    }
    if (s.sp + nhit - 1 > kStack) {
        atomicOr(p.error, kErrStack);
        s.ref = kDoneRef;
        return;
    }
    // rank of each child in (entry t, slot) order; missed children sit at +inf
    // behind every hit one.  For slots i < j, j goes first iff t_j < t_i.
    int r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    bool c;
    c = t1 < t0; r0 += c; r1 += !c;
    c = t2 < t0; r0 += c; r2 += !c;
    c = t3 < t0; r0 += c; r3 += !c;
    c = t2 < t1; r1 += c; r2 += !c;
    c = t3 < t1; r1 += c; r3 += !c;
    c = t3 < t2; r2 += c; r3 += !c;
    // rank 0 is visited next; rank k > 0 goes to stack slot sp + nhit - 1 - k
    const int top = s.sp + nhit - 1;
    if (h0) { if (r0 == 0) s.ref = ch.x; else stack[top - r0] = ch.x; }
    if (h1) { if (r1 == 0) s.ref = ch.y; else stack[top - r1] = ch.y; }
    if (h2) { if (r2 == 0) s.ref = ch.z; else stack[top - r2] = ch.z; }
    if (h3) { if (r3 == 0) s.ref = ch.w; else stack[top - r3] = ch.w; }
    s.sp = top;
}

// Tests the leaf s.ref; any-hit rays end at the first valid hit, otherwise the
// traversal pops the next node.
template <bool CLOSEST, bool STATS, bool PRED = false>
__device__ __forceinline__ void visit_leaf(const TraceParams &p, RayState &s, int32_t *stack, Counters<STATS> &cnt)
{
    cnt.add(PRED ? ST_PRED_LEAVES : ST_LEAVES);
    if (test_leaf<CLOSEST, STATS>(p, ~(uint32_t)s.ref, s.o, s.d, s.b, s.tcur, !PRED, cnt,
                                  PRED ? ST_PRED_TRI_TESTS : ST_TRI_TESTS)) {
        s.ref = kDoneRef;
        return;
    }
    s.ref = pop(stack, s.sp);
}

__device__ __forceinline__ bool over_budget(const TraceParams &p, RayState &s)
{
    if (++s.steps > p.max_steps) {
        atomicOr(p.error, kErrSteps);
        s.ref = kDoneRef;
        s.from = kDoneRef;
        return true;
    }
    return false;
}

// Loads ray i and runs the HRPP lookup (Sec. 4.2): each predicted leaf is
// tested; with Go Up Level > 0 each predicted interior node's subtree is
// traversed (Sec. 6.2).  Returns true when the ray still has to traverse from
// the root (then s.ref is the root).
template <int W, bool CLOSEST, bool STATS, bool BU = false>
__device__ __forceinline__ bool start_ray(const TraceParams &p, uint32_t i, RayState &s, int32_t *stack,
                                          Counters<STATS> &cnt)
{
    s.o = __ldg(p.rays + 2ull * i);
    s.d = __ldg(p.rays + 2ull * i + 1);
    s.b.t = __int_as_float(0x7F800000);
    s.b.u = s.b.v = 0.0f;
    s.b.prim = HRPP_NO_HIT;
    s.b.leaf = 0;
    s.b.found = s.b.from_trav = false;
    s.set = 0;
    s.tag = 0;
    s.from = kDoneRef;
    s.climb_visit = false;
    s.outcome = HRPP_OUTCOME_PLAIN;
    cnt.add(ST_RAYS);
    bool traverse = true, have_inverse = false;
    const bool learned = p.predicted != nullptr;
    // a closed gate leaves the table to the sampled chunks' rays (finish_ray
    // takes the same decision again instead of keeping it in a register)
    const bool consult = p.table != nullptr && gate_admits(p.gate, p.gate_mask, i + p.ray_offset);
    if (p.table && !consult) cnt.add(ST_GATED);
    if (consult || learned) {
        cnt.add(ST_LOOKUPS);
        float tdummy = 0.0f;
        bool positive = false, done = false;
        if (learned) {
            // a predicted treelet (learned proposal): traverse its subtree first
            const int32_t c = __ldg(p.predicted + i);
            const int32_t ref = (c >= 0 && (uint32_t)c < p.n_nodes) ? __ldg(p.canon_ref + c) : kEmptyRef;
            if (ref != kEmptyRef) {
                positive = true;
                s.ri = ray_inverse(s.o, s.d);
                have_inverse = true;
                s.tcur = s.d.w;
                s.sp = 0;
                s.ref = ref;
                s.steps = 0;
                while (s.ref != kDoneRef) {
                    if (over_budget(p, s)) break;
                    if (s.ref >= 0) visit_interior<W, STATS, true>(p, s, stack, cnt);
                    else visit_leaf<CLOSEST, STATS, true>(p, s, stack, cnt);
                }
                done = !CLOSEST && s.b.found;
            }
        }
        const uint32_t ways = consult ? (1u << p.log2_ways) : 0u;
        const uint64_t *set = nullptr;
        if (consult) {
            const uint64_t m = mix48(ray_key(s.o, s.d, p.precision, p.hash_variant == HRPP_HASH_EXP_LSB));
            s.set = (uint32_t)(m & ((1ull << p.log2_sets) - 1ull));
            s.tag = (m >> p.log2_sets) & kTagMask;
            set = p.table + ((uint64_t)s.set << p.log2_ways);
        }
        if (p.go_up == 0) {
            // the predicted leaves of this scene, in way order, wait in the
            // (still empty) traversal stack; their triangles are then tested
            // in one loop, so a warp takes as many steps as its longest list
            // rather than, way by way, its largest leaf
            uint32_t nc = 0;
            for (uint32_t w = 0; w < ways && !done; ++w) {
                const uint64_t wd = p.update_mode == HRPP_UPDATE_ONLINE ? __ldcg(set + w) : __ldg(set + w);
                if (wd == HRPP_EMPTY_WORD || (wd >> kLeafBits) != s.tag) continue;
                positive = true;
                const uint32_t node = (uint32_t)(wd & kLeafMask);
                if ((node >> 2) + (node & 3u) + 1u > p.n_tris) continue;  // not a leaf of this scene
                stack[nc++] = (int32_t)node;
            }
            if (nc) {
                uint32_t k = 0, j = 0, node = (uint32_t)stack[0];
                cnt.add(ST_PRED_LEAVES);
                for (;;) {
                    // any-hit: the first hit ends the lookup
                    if (test_tri<CLOSEST, STATS>(p.tris + 3ull * (node >> 2), j, node, s.o, s.d, s.b, tdummy, false,
                                                 cnt, ST_PRED_TRI_TESTS))
                        break;
                    if (++j > (node & 3u)) {
                        if (++k == nc) break;
                        node = (uint32_t)stack[k];
                        j = 0;
                        cnt.add(ST_PRED_LEAVES);
                    }
                }
            }
        }
        // Go Up Level > 0: each predicted subtree is traversed in way order
        for (uint32_t w = 0; p.go_up != 0 && w < ways && !done; ++w) {
            const uint64_t wd = p.update_mode == HRPP_UPDATE_ONLINE ? __ldcg(set + w) : __ldg(set + w);
            if (wd == HRPP_EMPTY_WORD || (wd >> kLeafBits) != s.tag) continue;
            positive = true;
            const uint32_t node = (uint32_t)(wd & kLeafMask);
            if (node >= p.n_interior) continue;  // not an interior node of this scene
            if (!have_inverse) {
                s.ri = ray_inverse(s.o, s.d);
                have_inverse = true;
            }
            s.tcur = (CLOSEST && s.b.found) ? s.b.t : s.d.w;
            s.sp = 0;
            s.ref = (int32_t)node;
            s.steps = 0;
            while (s.ref != kDoneRef) {
                if (over_budget(p, s)) break;
                if (s.ref >= 0) visit_interior<W, STATS, true>(p, s, stack, cnt);
                else visit_leaf<CLOSEST, STATS, true>(p, s, stack, cnt);
            }
            done = !CLOSEST && s.b.found;
        }
        if (!positive) {
            cnt.add(ST_NEGATIVES);
            s.outcome = HRPP_OUTCOME_NEGATIVE;
        } else {
            cnt.add(ST_POSITIVES);
            if (s.b.found) {
                cnt.add(ST_TRUE_POS);
                s.outcome = HRPP_OUTCOME_TRUE_POS;
                // any-hit: answered; closest-hit without verification (the
                // paper's semantics, not exact): the predicted hit stands
                if (!CLOSEST || p.verify == HRPP_VERIFY_NONE) traverse = false;
            } else {
                cnt.add(ST_FALSE_POS);
                s.outcome = HRPP_OUTCOME_FALSE_POS;
            }
        }
    }
    s.predicted_hit = s.b.found;
    if (STATS) s.box0 = cnt.c[ST_BOX_TESTS];
    if (traverse) {
        if (!have_inverse) s.ri = ray_inverse(s.o, s.d);
        s.tcur = (CLOSEST && s.b.found) ? s.b.t : s.d.w;
        s.sp = 0;
        s.ref = p.root_ref;
        s.steps = 0;
        if (BU && CLOSEST && s.b.found) {
            // climb from the predicted hit's leaf (climb() visits the ancestors)
            s.ref = kDoneRef;
            s.from = (int32_t)~s.b.leaf;
        }
    } else {
        s.ref = kDoneRef;
    }
    return traverse;
}

// Online insert (Sec. 5: the node a conflicting ray reached joins its entry,
// with no duplicate nodes): a 64-bit compare-and-swap claims the set's first
// empty way or, with every way valid, replaces way (ray mod W).  A CAS that
// another ray beat re-reads the set, and finding its own word there makes it
// a duplicate.  After kOnlineTries lost attempts the insert is dropped and
// counted as a duplicate; results never depend on the table's contents.
constexpr int kOnlineTries = 4;

template <bool STATS>
__device__ __forceinline__ void online_insert(const TraceParams &p, uint32_t set, uint32_t ray, uint64_t word,
                                              Counters<STATS> &cnt)
{
    unsigned long long *base = reinterpret_cast<unsigned long long *>(p.table) + ((uint64_t)set << p.log2_ways);
    const uint32_t ways = 1u << p.log2_ways;
    for (int attempt = 0; attempt < kOnlineTries; ++attempt) {
        uint32_t target = ways;
        for (uint32_t k = 0; k < ways; ++k) {
            const unsigned long long wd = __ldcg(base + k);
            if (wd == word) {
                cnt.add(ST_DUP_INSERTS);
                return;
            }
            if (wd == HRPP_EMPTY_WORD && target == ways) target = k;
        }
        unsigned long long expected = HRPP_EMPTY_WORD;
        if (target == ways) {
            target = ray & (ways - 1u);
            expected = __ldcg(base + target);
            if (expected == HRPP_EMPTY_WORD) continue;  // emptied meanwhile: rescan
        }
        const unsigned long long old = atomicCAS(base + target, expected, (unsigned long long)word);
        if (old == expected) {
            if (expected != HRPP_EMPTY_WORD) cnt.add(ST_EVICTIONS);
            return;
        }
        if (old == word) {
            cnt.add(ST_DUP_INSERTS);
            return;
        }
    }
    cnt.add(ST_DUP_INSERTS);
}

// Writes ray i's result and decides its insert (two-phase: returns the record
// to append; online: inserts the word now).
template <bool CLOSEST, bool STATS>
__device__ __forceinline__ bool finish_ray(const TraceParams &p, uint32_t i, const RayState &s, Counters<STATS> &cnt,
                                           uint32_t &gflags, uint32_t &slot, uint64_t &word)
{
    bool want_record = false;
    const bool consulted = p.table != nullptr && gate_admits(p.gate, p.gate_mask, i + p.ray_offset);
    gflags = consulted ? (kGateLooked | (s.outcome == HRPP_OUTCOME_TRUE_POS ? kGateTp : 0u)) : 0u;
    if (CLOSEST && s.predicted_hit && s.b.from_trav) cnt.add(ST_TP_INEXACT);
    // Sec. 5: a ray that traversed inserts the node of its final hit (the leaf,
    // or its ancestor go_up levels up, Sec. 6.2) unless its entry holds it
    // already.  Any-hit true positives (and closest-hit ones left unverified)
    // were answered by the predictor.
    const bool traversed = !s.predicted_hit || (CLOSEST && p.verify != HRPP_VERIFY_NONE);
    if (consulted && traversed && s.b.found && p.update_mode != HRPP_UPDATE_FROZEN) {
        uint32_t node = s.b.leaf;
        bool storable = true;
        if (p.go_up > 0) {
            int32_t a = __ldg(p.leaf_parent + (s.b.leaf >> 2));
            storable = a >= 0;
            for (int g = 1; storable && g < p.go_up; ++g) {
                const int32_t q = __ldg(p.parent + a);
                if (q < 0) break;
                a = q;
            }
            node = (uint32_t)a;
        }
        const uint64_t w = (s.tag << kLeafBits) | node;
        const uint64_t *set = p.table + ((uint64_t)s.set << p.log2_ways);
        bool present = false;
        for (uint32_t k = 0; k < (1u << p.log2_ways); ++k)
            present |= (p.update_mode == HRPP_UPDATE_ONLINE ? __ldcg(set + k) : __ldg(set + k)) == w;
        if (storable && !present) {
            cnt.add(ST_INSERTS);
            word = w;
            if (p.update_mode == HRPP_UPDATE_ONLINE) {
                online_insert(p, s.set, i + p.ray_offset, word, cnt);
            } else {
                slot = (s.set << p.log2_ways) | way_of(node, p.log2_ways);
                want_record = true;  // append_records claims the slot
            }
        }
    }
    if (s.b.found) cnt.add(ST_HITS);
    if (STATS) {
        if (p.ray_outcome) p.ray_outcome[i] = s.outcome;
        if (p.ray_box_tests) p.ray_box_tests[i] = cnt.c[ST_BOX_TESTS] - s.box0;
    }
    if (CLOSEST) {
        reinterpret_cast<float4 *>(p.hits)[i] = make_float4(s.b.t, __uint_as_float(s.b.prim), s.b.u, s.b.v);
    } else {
        reinterpret_cast<uint32_t *>(p.hits)[i] = s.b.found ? s.b.prim : HRPP_NO_HIT;
    }
    return want_record;
}

// Two-phase inserts of the lanes that want one (all 32 lanes call this
// together).  A slot goes to the highest ray index aimed at it.  LANE_ORDERED
// (the warp's rays rise with the lane): of the lanes aimed at one slot only
// the highest lane can win, so the others are counted as lost inserts here
// (k_apply counts the rest) and leave no record.  The remaining lanes claim
// their slots (atomicMax of ray + 1) and append their records with one atomic
// per warp.
template <bool LANE_ORDERED, bool STATS>
__device__ __forceinline__ void append_records(const TraceParams &p, uint32_t lane, bool want, uint32_t slot,
                                               uint32_t ray, uint64_t word, Counters<STATS> &cnt)
{
    if (!__any_sync(0xFFFFFFFFu, want)) return;
    if (LANE_ORDERED) {
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, want ? slot : 0xFFFFFFFFu);
        if (want && lane != 31u - (uint32_t)__clz(peers)) {
            cnt.add(ST_DUP_INSERTS);
            want = false;
        }
    }
    if (want) atomicMax(p.winner + slot, p.ray_offset + ray + 1u);
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, want);
    const uint32_t leader = __ffs(m) - 1;
    uint32_t rb = 0;
    if (lane == leader) rb = atomicAdd(&p.ctl->n_records, (uint32_t)__popc(m));
    rb = __shfl_sync(0xFFFFFFFFu, rb, leader);
    if (want) {
        Record r;
        r.slot = slot;
        r.ray1 = p.ray_offset + ray + 1u;
        r.word = word;
        p.records[rb + __popc(m & lanemask_lt())] = r;
    }
}

// Parent of interior node `node`, kept in the node's spare word.
template <int W>
__device__ __forceinline__ int32_t node_parent(const TraceParams &p, int32_t node)
{
    if (W == 2) return __ldg(reinterpret_cast<const int32_t *>(p.nodes + 4ull * (uint32_t)node + 3) + 2);
    return __ldg(reinterpret_cast<const int32_t *>(p.nodes + 8ull * (uint32_t)node + 7));
}

// Bottom-up verification: once everything below the climb is traversed,
// the ray moves to the parent of s.from; that visit (an ordinary interior
// visit) tests only the children other than s.from and then the climb is at
// the parent.  Returns false when the climb is over (past the root) or none
// runs.
template <int W>
__device__ __forceinline__ bool climb(const TraceParams &p, RayState &s)
{
    if (s.from == kDoneRef) return false;
    const int32_t up = s.from >= 0 ? node_parent<W>(p, s.from) : __ldg(p.leaf_parent + ((uint32_t)~s.from >> 2));
    if (up < 0) {
        s.from = kDoneRef;
        return false;
    }
    s.ref = up;
    s.climb_visit = true;
    return true;
}

// One interior visit of the main traversal.  With bottom-up verification
// (BU) the visit leaves out the child the climb came from; no other node has
// that child, so passing it on every visit only matters at the climb's
// ancestor.
template <int W, bool BU, bool STATS>
__device__ __forceinline__ void traverse_interior(const TraceParams &p, RayState &s, int32_t *stack,
                                                  Counters<STATS> &cnt)
{
    if (!BU) {
        visit_interior<W, STATS>(p, s, stack, cnt);
        return;
    }
    const int32_t node = s.ref;
    visit_interior<W, STATS, false, true>(p, s, stack, cnt, s.from);
    if (s.climb_visit) {
        s.from = node;
        s.climb_visit = false;
    }
}

// The whole of one ray: lookup, traversal, result, insert decision.  BU:
// closest-hit true positives verify bottom-up; a lane whose stack runs dry
// climbs within the same loop, without waiting for the rest of its warp.
template <int W, bool CLOSEST, bool STATS, bool BU = false>
__device__ __forceinline__ bool trace_one(const TraceParams &p, uint32_t i, int32_t *stack, Counters<STATS> &cnt,
                                          uint32_t &gflags, uint32_t &slot, uint64_t &word)
{
    static_assert(CLOSEST || !BU, "bottom-up verification is for closest-hit rays");
    RayState s;
    if (start_ray<W, CLOSEST, STATS, BU>(p, i, s, stack, cnt)) {
        if (!BU) {
            while (s.ref != kDoneRef) {
                if (over_budget(p, s)) break;
                if (s.ref >= 0) visit_interior<W, STATS>(p, s, stack, cnt);
                else visit_leaf<CLOSEST, STATS>(p, s, stack, cnt);
            }
        } else {
            for (;;) {
                if (s.ref == kDoneRef && !climb<W>(p, s)) break;
                if (over_budget(p, s)) break;
                if (s.ref >= 0) traverse_interior<W, BU, STATS>(p, s, stack, cnt);
                else visit_leaf<CLOSEST, STATS>(p, s, stack, cnt);
            }
        }
    }
    return finish_ray<CLOSEST, STATS>(p, i, s, cnt, gflags, slot, word);
}

template <int W, bool CLOSEST, bool STATS, bool BU = false>
__global__ void __launch_bounds__(512) k_trace(const TraceParams p)
{
    __shared__ uint2 gate_acc[kMaxWarps];
    const uint32_t lane = threadIdx.x & 31u;
    uint2 &gacc = gate_acc[threadIdx.x >> 5];
    if (lane == 0) gacc = make_uint2(0u, 0u);
    __syncwarp();
    Counters<STATS> cnt;
    cnt.init();
    int32_t stack[kStack];
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&p.ctl->next_ray, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= p.n_rays) break;
        const uint32_t i = base + lane;
        bool want = false;
        uint32_t slot = 0, gflags = 0;
        uint64_t word = 0;
        if (i < p.n_rays) want = trace_one<W, CLOSEST, STATS, BU>(p, i, stack, cnt, gflags, slot, word);
        append_records<true>(p, lane, want, slot, i, word, cnt);
        gate_count(p, lane, gflags, gacc);
    }
    cnt.flush(p.ctl, lane);
    gate_flush(p, lane, gacc);
}

// Many (scene, table, rays) items of one query mode in one persistent
// launch (a batch runs one launch per mode).  The rays of all items are cut
// into 32-ray chunks (a chunk never spans two items); a warp takes the next
// chunk from the launch's cursor, copies that item's parameters into shared
// memory when the item changes, traces the chunk exactly as k_trace would,
// and adds its counters to the item's own control block.
constexpr int kBatchMaxWarps = 16;  // up to 512 threads per block

template <int W, bool CLOSEST, bool STATS>
__global__ void __launch_bounds__(512) k_trace_batch(const BatchDesc b)
{
    __shared__ TraceParams item_params[kBatchMaxWarps];
    __shared__ uint2 gate_acc[kBatchMaxWarps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    TraceParams &p = item_params[warp];
    uint2 &gacc = gate_acc[warp];
    if (lane == 0) gacc = make_uint2(0u, 0u);
    Counters<STATS> cnt;
    cnt.init();
    int32_t stack[kStack];
    uint32_t cur = 0xFFFFFFFFu;
    for (;;) {
        uint32_t chunk = 0;
        if (lane == 0) chunk = atomicAdd(b.cursor, 1u);
        chunk = __shfl_sync(0xFFFFFFFFu, chunk, 0);
        if (chunk >= b.n_chunks) break;
        const uint32_t item = __ldg(b.chunk_item + chunk);
        if (item != cur) {
            if (cur != 0xFFFFFFFFu) {
                cnt.flush(p.ctl, lane);
                gate_flush(p, lane, gacc);
            }
            cnt.init();
            __syncwarp();
            const uint32_t *src = reinterpret_cast<const uint32_t *>(b.items + item);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&p);
            for (uint32_t k = lane; k < sizeof(TraceParams) / 4; k += 32) dst[k] = __ldg(src + k);
            __syncwarp();
            cur = item;
        }
        const uint32_t i = __ldg(b.chunk_first + chunk) + lane;
        bool want = false;
        uint32_t slot = 0, gflags = 0;
        uint64_t word = 0;
        if (i < p.n_rays) want = trace_one<W, CLOSEST, STATS>(p, i, stack, cnt, gflags, slot, word);
        append_records<true>(p, lane, want, slot, i, word, cnt);
        gate_count(p, lane, gflags, gacc);
    }
    if (cur != 0xFFFFFFFFu) {
        cnt.flush(p.ctl, lane);
        gate_flush(p, lane, gacc);
    }
}

template <int W>
cudaError_t launch_batch_width(bool closest, bool stats, const BatchDesc &b, int block_threads, cudaStream_t stream)
{
    const void *fn = closest ? (stats ? (const void *)k_trace_batch<W, true, true> : (const void *)k_trace_batch<W, true, false>)
                             : (stats ? (const void *)k_trace_batch<W, false, true> : (const void *)k_trace_batch<W, false, false>);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block_threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t warps_per_block = block_threads / 32;
    uint64_t blocks = (uint64_t)sms * per_sm;
    if (blocks * warps_per_block > b.n_chunks) blocks = (b.n_chunks + warps_per_block - 1) / warps_per_block;
    if (blocks < 1) blocks = 1;
    void *args[] = {(void *)&b};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(block_threads), args, 0, stream);
}

// REFILL schedule: node visits per lane between the warp's votes (refill,
// finish).  One visit per vote cost 37 % on terrain AO rays; 16 keeps the
// votes rare while idle lanes still refill within a few dozen visits.
constexpr int kRefillSteps = 16;

template <int W, bool CLOSEST, bool STATS, bool BU = false>
__global__ void __launch_bounds__(512) k_trace_dyn(const TraceParams p)
{
    __shared__ uint2 gate_acc[kMaxWarps];
    const uint32_t lane = threadIdx.x & 31u;
    uint2 &gacc = gate_acc[threadIdx.x >> 5];
    if (lane == 0) gacc = make_uint2(0u, 0u);
    __syncwarp();
    Counters<STATS> cnt;
    cnt.init();
    int32_t stack[kStack];
    RayState s;
    uint32_t ray = kNoRay;
    bool pool_open = true;  // warp-uniform
    for (;;) {
        // refill idle lanes from the ray pool
        const uint32_t idle = __ballot_sync(0xFFFFFFFFu, ray == kNoRay);
        if (pool_open && (uint32_t)__popc(idle) >= p.refill_min) {
            const uint32_t need = __popc(idle);
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&p.ctl->next_ray, need);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base + need >= p.n_rays) pool_open = false;
            if (ray == kNoRay) {
                const uint32_t mine = base + __popc(idle & lanemask_lt());
                if (mine < p.n_rays) {
                    ray = mine;
                    start_ray<W, CLOSEST, STATS, BU>(p, ray, s, stack, cnt);
                }
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, ray != kNoRay) == 0) {
            if (!pool_open) break;
            continue;
        }
        // up to kRefillSteps node visits per lane between two warp votes; a
        // lane whose ray ends early waits for the vote
        if (ray != kNoRay) {
#pragma unroll 1
            for (int k = 0; k < kRefillSteps; ++k) {
                if (s.ref == kDoneRef) {
                    if (!BU || !climb<W>(p, s)) break;
                    continue;
                }
                if (over_budget(p, s)) break;
                if (s.ref >= 0) traverse_interior<W, BU, STATS>(p, s, stack, cnt);
                else visit_leaf<CLOSEST, STATS>(p, s, stack, cnt);
            }
        }
        const bool done = ray != kNoRay && s.ref == kDoneRef && s.from == kDoneRef;
        if (__any_sync(0xFFFFFFFFu, done)) {
            bool want = false;
            uint32_t slot = 0, gflags = 0;
            uint64_t word = 0;
            if (done) want = finish_ray<CLOSEST, STATS>(p, ray, s, cnt, gflags, slot, word);
            append_records<false>(p, lane, want, slot, ray, word, cnt);
            gate_count(p, lane, gflags, gacc);
            if (done) ray = kNoRay;
        }
    }
    cnt.flush(p.ctl, lane);
    gate_flush(p, lane, gacc);
}

template <int W>
cudaError_t launch_width(bool closest, bool stats, int schedule, const TraceParams &p, int block_threads,
                         int blocks_per_sm_cap, cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1,
                         const L2Window *l2 = nullptr)
{
    const void *fn;
    const bool bu = closest && p.verify == HRPP_VERIFY_BOTTOM_UP;
    if (schedule == 1) {
        if (bu) fn = stats ? (const void *)k_trace_dyn<W, true, true, true> : (const void *)k_trace_dyn<W, true, false, true>;
        else if (closest) fn = stats ? (const void *)k_trace_dyn<W, true, true> : (const void *)k_trace_dyn<W, true, false>;
        else fn = stats ? (const void *)k_trace_dyn<W, false, true> : (const void *)k_trace_dyn<W, false, false>;
    } else {
        if (bu) fn = stats ? (const void *)k_trace<W, true, true, true> : (const void *)k_trace<W, true, false, true>;
        else if (closest) fn = stats ? (const void *)k_trace<W, true, true> : (const void *)k_trace<W, true, false>;
        else fn = stats ? (const void *)k_trace<W, false, true> : (const void *)k_trace<W, false, false>;
    }
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
    // persisting-L2 window: only while the context has a set-aside, and no
    // larger than the device allows
    cudaLaunchAttribute attr;
    unsigned n_attr = 0;
    if (l2 && l2->base && l2->bytes) {
        size_t set_aside = 0;
        int max_window = 0;
        if ((e = cudaDeviceGetLimit(&set_aside, cudaLimitPersistingL2CacheSize)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev)) != cudaSuccess)
            return e;
        if (set_aside > 0 && max_window > 0) {
            const size_t bytes = l2->bytes < (size_t)max_window ? l2->bytes : (size_t)max_window;
            memset(&attr, 0, sizeof attr);
            attr.id = cudaLaunchAttributeAccessPolicyWindow;
            attr.val.accessPolicyWindow.base_ptr = const_cast<void *>(l2->base);
            attr.val.accessPolicyWindow.num_bytes = bytes;
            attr.val.accessPolicyWindow.hitRatio = set_aside >= bytes ? 1.0f : (float)((double)set_aside / bytes);
            attr.val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
            attr.val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
            n_attr = 1;
        }
    }
    if (ev0) cudaEventRecord(ev0, stream);
    void *args[] = {(void *)&p};
    if (n_attr) {
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof cfg);
        cfg.gridDim = dim3((unsigned)blocks);
        cfg.blockDim = dim3(block_threads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = stream;
        cfg.attrs = &attr;
        cfg.numAttrs = n_attr;
        e = cudaLaunchKernelExC(&cfg, fn, args);
    } else {
        e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(block_threads), args, 0, stream);
    }
    if (ev1) cudaEventRecord(ev1, stream);
    return e;
}

}  // namespace hrpp
