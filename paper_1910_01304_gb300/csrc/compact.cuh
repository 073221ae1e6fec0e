// Two-pass HRPP: the paper's ray pool (Sec. 4.1-4.2).  A ray whose
// prediction answers its query leaves after the lookup; every other ray is
// "added back into the ray pool" -- here a compacted queue -- and traverses in
// a second launch whose warps hold only rays that really traverse, instead of
// idling the lanes of the rays that were answered.
//
//   k_predict      one thread per ray (Go Up Level 0, no learned treelets):
//                  hash (Sec. 5), set read, predicted-leaf tests (Sec. 4.2).
//                  An any-hit true positive -- and, with verification off
//                  (the paper's own semantics), a closest-hit one -- writes
//                  its result and is done (Sec. 4.3).  Every other ray is
//                  appended to the queue with its mixed key; a closest-hit
//                  true positive also keeps its predicted leaf, and its
//                  predicted hit waits in the output buffer as the bound of
//                  its exact traversal.  Each block appends its rays in ray
//                  order with one atomic.
//   k_trace_queue  persistent warps take 32 queue entries at a time and
//                  traverse them exactly as k_trace traverses its rays, then
//                  decide the inserts; lanes aimed at one slot leave only the
//                  highest ray's record.
//
// Per ray, the work, results, counters, table updates and gate decision are
// those of the fused kernels: pass 1 counts the lookup (rays, lookups,
// outcome classes, predicted-leaf tests, gated), pass 2 the traversal and the
// insert, and each ray's result is written by exactly one of them.
#pragma once

#include "trace_kernel.cuh"

namespace hrpp {

// One queued ray: its index, its predicted leaf (closest-hit true positives)
// with the lookup's outcome in the top bits, and mix48 of its key.
struct __align__(16) QueueEntry {
    uint32_t ray;
    uint32_t leaf_flags;
    uint64_t m;
};
constexpr uint32_t kQConsulted = 1u << 28, kQTruePos = 2u << 28, kQFalsePos = 4u << 28;
constexpr uint32_t kQLeafMask = (1u << 28) - 1u;

constexpr int kPredictThreads = 256;
// k_predict waits on dependent loads (ray, set, triangles): 6 resident blocks
// per SM (40 registers) ran the lookups of 1.14M terrain shadow rays faster
// than 5 (48 registers, nothing spilled) or 8 (32 registers, more spills).
constexpr int kPredictMinBlocks = 6;

// The lookup of ray i (Go Up Level 0): fills s (hit found in a predicted
// leaf, outcome, set and tag) and returns m = mix48(key) (0 when the table
// was not consulted).  The ray's predicted leaves go to its column of `cand`
// (shared memory, kPredictThreads entries per row) and are tested in one
// loop over their triangles in way order, so a warp takes as many steps as
// its longest list, not the sum over ways of each way's largest leaf.
template <bool CLOSEST, bool STATS>
__device__ __forceinline__ uint64_t predict_ray(const TraceParams &p, uint32_t i, RayState &s, Counters<STATS> &cnt,
                                                bool &consulted, uint32_t *cand)
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
    consulted = gate_admits(p.gate, p.gate_mask, i + p.ray_offset);
    uint64_t m = 0;
    if (!consulted) {
        cnt.add(ST_GATED);
    } else {
        cnt.add(ST_LOOKUPS);
        m = mix48(ray_key(s.o, s.d, p.precision, p.hash_variant == HRPP_HASH_EXP_LSB));
        s.set = (uint32_t)(m & ((1ull << p.log2_sets) - 1ull));
        s.tag = (m >> p.log2_sets) & kTagMask;
        const uint64_t *set = p.table + ((uint64_t)s.set << p.log2_ways);
        const uint32_t ways = 1u << p.log2_ways;
        bool positive = false;
        // the set's words first, all loads in flight together
        uint64_t words[8];
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            if (w < ways) words[w] = p.update_mode == HRPP_UPDATE_ONLINE ? __ldcg(set + w) : __ldg(set + w);
        // the predicted leaves of this scene, in way order; each one's
        // triangles (48 to 192 bytes: the lines holding its first and last
        // byte) start towards L1 before the first test waits on one
        uint32_t nc = 0;
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w) {
            if (w >= ways) break;
            const uint64_t wd = words[w];
            if (wd == HRPP_EMPTY_WORD || (wd >> kLeafBits) != s.tag) continue;
            positive = true;
            const uint32_t node = (uint32_t)(wd & kLeafMask);
            if ((node >> 2) + (node & 3u) + 1u > p.n_tris) continue;  // not a leaf of this scene
            cand[nc * kPredictThreads] = node;
            ++nc;
            const char *tri = reinterpret_cast<const char *>(p.tris + 3ull * (node >> 2));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(tri));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(tri + 48u * ((node & 3u) + 1u) - 1u));
        }
        if (nc) {
            float tdummy = 0.0f;
            uint32_t k = 0, j = 0, node = cand[0];
            cnt.add(ST_PRED_LEAVES);
            for (;;) {
                // any-hit: the first hit ends the lookup
                if (test_tri<CLOSEST, STATS>(p.tris + 3ull * (node >> 2), j, node, s.o, s.d, s.b, tdummy, false, cnt,
                                             ST_PRED_TRI_TESTS))
                    break;
                if (++j > (node & 3u)) {
                    if (++k == nc) break;
                    node = cand[k * kPredictThreads];
                    j = 0;
                    cnt.add(ST_PRED_LEAVES);
                }
            }
        }
        if (!positive) {
            cnt.add(ST_NEGATIVES);
            s.outcome = HRPP_OUTCOME_NEGATIVE;
        } else {
            cnt.add(ST_POSITIVES);
            if (s.b.found) {
                cnt.add(ST_TRUE_POS);
                s.outcome = HRPP_OUTCOME_TRUE_POS;
            } else {
                cnt.add(ST_FALSE_POS);
                s.outcome = HRPP_OUTCOME_FALSE_POS;
            }
        }
    }
    s.predicted_hit = s.b.found;
    if (STATS) s.box0 = cnt.c[ST_BOX_TESTS];
    return m;
}

template <bool CLOSEST, bool STATS>
__global__ void __launch_bounds__(kPredictThreads, kPredictMinBlocks) k_predict(const TraceParams p, QueueEntry *queue)
{
    __shared__ uint32_t warp_base[kPredictThreads / 32];
    __shared__ uint32_t block_base;
    __shared__ uint2 gate_acc[kPredictThreads / 32];
    __shared__ uint32_t cand[8 * kPredictThreads];  // predicted leaves, one column per thread
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t i = blockIdx.x * (uint32_t)kPredictThreads + threadIdx.x;
    Counters<STATS> cnt;
    cnt.init();
    bool enqueue = false;
    uint32_t gflags = 0;
    QueueEntry e;
    e.ray = i;
    e.leaf_flags = 0;
    e.m = 0;
    if (i < p.n_rays) {
        RayState s;
        bool consulted = false;
        e.m = predict_ray<CLOSEST, STATS>(p, i, s, cnt, consulted, cand + threadIdx.x);
        // answered by the prediction: any-hit true positives, and closest-hit
        // ones when they are not verified (the paper's semantics)
        const bool answered = s.b.found && (!CLOSEST || p.verify == HRPP_VERIFY_NONE);
        if (answered) {
            uint32_t slot = 0;
            uint64_t word = 0;
            finish_ray<CLOSEST, STATS>(p, i, s, cnt, gflags, slot, word);  // no insert: it did not traverse
        } else {
            enqueue = true;
            e.leaf_flags = (consulted ? kQConsulted : 0u) |
                           (s.outcome == HRPP_OUTCOME_TRUE_POS ? kQTruePos | (s.b.leaf & kQLeafMask) : 0u) |
                           (s.outcome == HRPP_OUTCOME_FALSE_POS ? kQFalsePos : 0u);
            if (CLOSEST && s.b.found)  // the bound of its exact traversal, read back by pass 2
                reinterpret_cast<float4 *>(p.hits)[i] = make_float4(s.b.t, __uint_as_float(s.b.prim), s.b.u, s.b.v);
            if (STATS && p.ray_outcome) p.ray_outcome[i] = s.outcome;
        }
    }
    if (lane == 0) gate_acc[warp] = make_uint2(0u, 0u);
    gate_count(p, lane, gflags, gate_acc[warp]);
    // append the block's queued rays in ray order: warp counts, a prefix over
    // the block's warps, one atomic for the block (the gate's counts of the
    // rays answered here likewise meet in one atomic per block)
    const uint32_t ball = __ballot_sync(0xFFFFFFFFu, enqueue);
    if (lane == 0) warp_base[warp] = __popc(ball);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t total = 0;
        uint2 g = make_uint2(0u, 0u);
        for (int w = 0; w < kPredictThreads / 32; ++w) {
            const uint32_t c = warp_base[w];
            warp_base[w] = total;
            total += c;
            g.x += gate_acc[w].x;
            g.y += gate_acc[w].y;
        }
        block_base = total ? atomicAdd(&p.ctl->queue_len, total) : 0u;
        if (p.gate && g.x) atomicAdd(&p.ctl->gate_lookups, g.x);
        if (p.gate && g.y) atomicAdd(&p.ctl->gate_tp, g.y);
    }
    __syncthreads();
    if (enqueue) queue[block_base + warp_base[warp] + __popc(ball & lanemask_lt())] = e;
    cnt.flush(p.ctl, lane);
}

// Two-phase inserts of a pass-2 warp, whose lanes hold queue entries in no
// particular ray order: of the lanes aimed at one slot only the highest ray
// can win it, so the others are counted as lost inserts and leave no record
// (as append_records does for a lane-ordered warp).
template <bool STATS>
__device__ __forceinline__ void append_records_any_order(const TraceParams &p, uint32_t lane, bool want,
                                                         uint32_t slot, uint32_t ray, uint64_t word,
                                                         Counters<STATS> &cnt)
{
    if (!__any_sync(0xFFFFFFFFu, want)) return;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, want ? slot : 0xFFFFFFFFu);
    if (want) {
        const uint32_t top = __reduce_max_sync(peers, ray);
        if (ray != top) {
            cnt.add(ST_DUP_INSERTS);
            want = false;
        }
    }
    append_records<false>(p, lane, want, slot, ray, word, cnt);
}

// Pass 2: the queued rays' traversal from the root (closest-hit true
// positives bounded by their predicted hit), result and insert decision.
template <int W, bool CLOSEST, bool STATS>
__global__ void __launch_bounds__(512) k_trace_queue(const TraceParams p, const QueueEntry *queue)
{
    __shared__ uint2 gate_acc[kMaxWarps];
    const uint32_t lane = threadIdx.x & 31u;
    uint2 &gacc = gate_acc[threadIdx.x >> 5];
    if (lane == 0) gacc = make_uint2(0u, 0u);
    __syncwarp();
    const uint32_t n = p.ctl->queue_len;  // final: pass 1 ended before this launch
    Counters<STATS> cnt;
    cnt.init();
    int32_t stack[kStack];
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&p.ctl->next_ray, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        const uint32_t k = base + lane;
        bool want = false;
        uint32_t slot = 0, gflags = 0, i = 0;
        uint64_t word = 0;
        if (k < n) {
            const QueueEntry e = queue[k];
            i = e.ray;
            RayState s;
            s.o = __ldg(p.rays + 2ull * i);
            s.d = __ldg(p.rays + 2ull * i + 1);
            s.b.u = s.b.v = 0.0f;
            s.b.found = s.b.from_trav = false;
            s.b.t = __int_as_float(0x7F800000);
            s.b.prim = HRPP_NO_HIT;
            s.b.leaf = 0;
            if (CLOSEST && (e.leaf_flags & kQTruePos)) {
                const float4 h = reinterpret_cast<const float4 *>(p.hits)[i];
                s.b.t = h.x;
                s.b.prim = __float_as_uint(h.y);
                s.b.u = h.z;
                s.b.v = h.w;
                s.b.leaf = e.leaf_flags & kQLeafMask;
                s.b.found = true;
            }
            s.predicted_hit = s.b.found;
            s.set = (uint32_t)(e.m & ((1ull << p.log2_sets) - 1ull));
            s.tag = (e.m >> p.log2_sets) & kTagMask;
            s.from = kDoneRef;
            s.climb_visit = false;
            s.outcome = !(e.leaf_flags & kQConsulted) ? HRPP_OUTCOME_PLAIN
                        : (e.leaf_flags & kQTruePos)  ? HRPP_OUTCOME_TRUE_POS
                        : (e.leaf_flags & kQFalsePos) ? HRPP_OUTCOME_FALSE_POS
                                                      : HRPP_OUTCOME_NEGATIVE;
            if (STATS) s.box0 = cnt.c[ST_BOX_TESTS];
            s.ri = ray_inverse(s.o, s.d);
            s.tcur = s.b.found ? s.b.t : s.d.w;
            s.sp = 0;
            s.ref = p.root_ref;
            s.steps = 0;
            while (s.ref != kDoneRef) {
                if (over_budget(p, s)) break;
                if (s.ref >= 0) visit_interior<W, STATS>(p, s, stack, cnt);
                else visit_leaf<CLOSEST, STATS>(p, s, stack, cnt);
            }
            want = finish_ray<CLOSEST, STATS>(p, i, s, cnt, gflags, slot, word);
        }
        append_records_any_order<STATS>(p, lane, want, slot, i, word, cnt);
        gate_count(p, lane, gflags, gacc);
    }
    cnt.flush(p.ctl, lane);
    gate_flush(p, lane, gacc);
}

template <int W>
cudaError_t launch_compact_width(bool closest, bool stats, const TraceParams &p, QueueEntry *queue, int block_threads,
                                 cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1)
{
    const void *f1 = closest ? (stats ? (const void *)k_predict<true, true> : (const void *)k_predict<true, false>)
                             : (stats ? (const void *)k_predict<false, true> : (const void *)k_predict<false, false>);
    const void *f2 = closest ? (stats ? (const void *)k_trace_queue<W, true, true> : (const void *)k_trace_queue<W, true, false>)
                             : (stats ? (const void *)k_trace_queue<W, false, true> : (const void *)k_trace_queue<W, false, false>);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f2, block_threads, 0)) != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t warps_per_block = block_threads / 32;
    uint64_t blocks2 = (uint64_t)sms * per_sm;
    const uint64_t warps_needed = (p.n_rays + 31ull) / 32ull;  // the queue holds at most n_rays
    if (blocks2 * warps_per_block > warps_needed) blocks2 = (warps_needed + warps_per_block - 1) / warps_per_block;
    if (blocks2 < 1) blocks2 = 1;
    const uint64_t blocks1 = (p.n_rays + kPredictThreads - 1ull) / kPredictThreads;
    if (ev0) cudaEventRecord(ev0, stream);
    void *args[] = {(void *)&p, (void *)&queue};
    e = cudaLaunchKernel(f1, dim3((unsigned)blocks1), dim3(kPredictThreads), args, 0, stream);
    if (e == cudaSuccess) e = cudaLaunchKernel(f2, dim3((unsigned)blocks2), dim3(block_threads), args, 0, stream);
    if (ev1) cudaEventRecord(ev1, stream);
    return e;
}

}  // namespace hrpp
