/*
 * hrpp.h -- C ABI of the GB300 Hash-Based Ray Path Prediction library.
 *
 * HRPP (Demoullin, Gubran, Aamodt: "Hash-Based Ray Path Prediction: Skipping
 * BVH Traversal Computation by Exploiting Ray Locality") fronts BVH ray
 * traversal with a predictor table.  Each ray is hashed from the IEEE-754 bits
 * of its origin and direction (Sec. 5); the table maps the hash to leaf nodes
 * that earlier rays with the same hash reached (Sec. 4.2).  A ray first tests
 * the predicted leaves; when that answers the query the interior traversal is
 * skipped, otherwise the ray traverses the BVH as usual and its leaf is
 * inserted (Sec. 4.2-4.3, Sec. 5).  Results are exactly those of plain
 * traversal: any-hit rays stop at a hit found in a predicted leaf, and
 * closest-hit rays use the predicted hit only to bound an exact traversal.
 *
 * Conventions for every entry point:
 *   - Errors are returned as hrpp_status codes; nothing aborts or throws.
 *     hrpp_last_error() gives a message for the calling thread's last
 *     non-OK status.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Device work is enqueued asynchronously on it.
 *   - Handles are opaque; destroy(NULL) is a no-op.  The library copies every
 *     host array it is given; the caller keeps ownership of its buffers.
 *   - Objects live on the CUDA device that was current when they were made;
 *     calls switch to that device and restore the caller's afterwards.
 *   - Concurrency: a scene may be traced by any number of calls at once (it
 *     is read-only on the GPU, but its error flag is shared).  A table, a
 *     batch or a proposal must not be used by two calls whose GPU work
 *     overlaps (two streams, or two host threads): order them on one stream
 *     or with events.  Host-side calls are thread-safe otherwise.
 */
#ifndef HRPP_H
#define HRPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HRPP_VERSION 1
#define HRPP_NO_HIT 0xFFFFFFFFu
#define HRPP_EMPTY_WORD 0xFFFFFFFFFFFFFFFFull
#define HRPP_MAX_LEAF_TRIS 4      /* triangles per leaf */
#define HRPP_MAX_TRIS (1u << 26)  /* triangles per scene */
#define HRPP_MAX_STACK 64         /* traversal stack entries per ray */

typedef enum {
    HRPP_OK = 0,
    HRPP_ERR_INVALID_ARG = 1,     /* NULL where a pointer is required, bad size, mode or alignment */
    HRPP_ERR_INVALID_BVH = 2,     /* the node array is not a tree over all triangles */
    HRPP_ERR_OOM = 3,             /* a device or host allocation failed */
    HRPP_ERR_CUDA = 4,            /* a CUDA runtime call failed */
    HRPP_ERR_TRAVERSAL_LIMIT = 5, /* a ray exceeded its traversal step or stack bound */
    HRPP_ERR_UNSUPPORTED = 6      /* valid but beyond the library's compiled limits (HRPP_MAX_*) */
} hrpp_status;

/* Query paradigms (Sec. 4.1): shadow rays look for any intersection
 * ("hit-any"); most others need the closest one ("hit-all"). */
typedef enum { HRPP_ANY_HIT = 0, HRPP_CLOSEST_HIT = 1 } hrpp_mode;

/* When a ray's insert lands in the table.
 *   TWO_PHASE  every lookup of one hrpp_trace call sees the table as it was
 *              when the call started; after the batch, each slot keeps the
 *              insert of the highest ray index aimed at it.  Deterministic:
 *              results, table and statistics repeat bit for bit.
 *   ONLINE     inserts are written while the batch runs, so later rays may
 *              see them: a 64-bit compare-and-swap claims the set's first
 *              empty way or, with every way valid, replaces way (ray index
 *              mod ways); a CAS beaten by another ray re-reads the set (at
 *              most 4 attempts, then the insert is dropped as a duplicate).
 *              Results stay exact; table contents and statistics depend on
 *              scheduling, except when no two rays of a call share a set.
 *   FROZEN     lookups only; the table is never written. */
typedef enum { HRPP_UPDATE_TWO_PHASE = 0, HRPP_UPDATE_ONLINE = 1, HRPP_UPDATE_FROZEN = 2 } hrpp_update_mode;

/* Canonical BVH node (48 bytes; host memory).  A node is a leaf iff count > 0;
 * a leaf covers triangles prim_index[first .. first+count).  An interior
 * node's non-negative child entries index the node array; -1 = no child.
 * lo/hi bound the node's triangles; every child box must lie inside its
 * parent's.  Width 2 uses child[0..1], width 4 child[0..3]. */
typedef struct hrpp_bvh_node {
    float lo[3], hi[3];
    int32_t child[4];
    uint32_t first, count;
} hrpp_bvh_node;

/* Ray (32 bytes, 16-byte aligned): origin, tmin, direction, tmax.  A hit at
 * distance t counts iff tmin < t < tmax.  The direction is hashed exactly as
 * given (callers normally pass unit vectors). */
typedef struct hrpp_ray {
    float ox, oy, oz, tmin;
    float dx, dy, dz, tmax;
} hrpp_ray;

/* Closest-hit result (16 bytes): distance, triangle index in the caller's
 * tri_verts order, barycentrics of v1 (u) and v2 (v).  A miss is
 * (+inf, HRPP_NO_HIT, 0, 0).  Any-hit results are one uint32 per ray: the
 * index of a triangle the ray hits, or HRPP_NO_HIT. */
typedef struct hrpp_hit {
    float t;
    uint32_t prim;
    float u, v;
} hrpp_hit;

/* Counters of one hrpp_trace call (Sec. 4.3 outcome classes and node work).
 *   lookups           rays that consulted the table
 *   positives         lookups that found at least one predicted leaf
 *   true_pos          positives whose predicted leaves held a valid hit
 *   false_pos         positives whose predicted leaves held none
 *   negatives         lookups with no predicted leaf
 *   tp_inexact        closest-hit true positives whose exact traversal found
 *                     a closer hit than the predicted leaves (Sec. 4.3)
 *   inserts           rays that asked to insert the leaf they reached
 *   dup_inserts       two-phase: inserts that lost their slot to a later ray
 *                     of the same batch; online: inserts whose word another
 *                     ray of the call stored first, or that lost 4 CAS tries
 *   evictions         inserts that overwrote a valid table word
 *   interior_nodes,   interior nodes entered, child boxes tested, leaves
 *   box_tests,        entered and triangles tested by traversal
 *   leaves, tri_tests
 *   pred_leaves,      leaves and triangles tested inside predicted leaves or
 *   pred_tri_tests    subtrees, before (or instead of) traversal from the root
 *   pred_interior_nodes, pred_box_tests
 *                     interior nodes entered and child boxes tested inside
 *                     predicted subtrees (Go Up Level > 0, Sec. 6.2)
 *   gated             rays that skipped the table because its gate was
 *                     closed (hrpp_table_set_gate): no lookup, no insert */
typedef struct hrpp_stats {
    uint64_t rays, hits, lookups, positives, true_pos, false_pos, negatives, tp_inexact;
    uint64_t inserts, dup_inserts, evictions;
    uint64_t interior_nodes, box_tests, leaves, tri_tests, pred_leaves, pred_tri_tests;
    uint64_t pred_interior_nodes, pred_box_tests;
    uint64_t gated;
} hrpp_stats;

typedef struct hrpp_scene_info {
    uint32_t n_tris, n_interior, n_leaves, max_depth;
    uint32_t width, root_is_leaf;
    uint64_t device_bytes;
} hrpp_scene_info;

/* Per-call options of hrpp_trace_ex (all fields may be zero).  Results and
 * table words never depend on them, except that a max_steps budget a ray
 * runs out of stops that ray early; verify changes node counters; the
 * others change only speed.
 *   kernel_start/kernel_stop  cudaEvent_t (as void*) recorded on `stream`
 *                             immediately before and after the traversal
 *                             kernel (both launches of the COMPACT
 *                             schedule), for timing it alone
 *   block_threads             threads per block of the traversal kernel:
 *                             0 = default, else 64, 128, 256 or 512
 *   schedule                  how warps take rays from the batch:
 *                             HRPP_SCHEDULE_DEFAULT, HRPP_SCHEDULE_BATCH (a
 *                             warp traces 32 rays to completion, then takes
 *                             32 more), HRPP_SCHEDULE_REFILL (lanes whose
 *                             ray is done take new rays while the rest of
 *                             the warp keeps traversing) or
 *                             HRPP_SCHEDULE_COMPACT (the paper's ray pool,
 *                             Sec. 4.1-4.2, in two launches: every ray's
 *                             lookup first, one thread per ray; rays whose
 *                             prediction answered them -- any-hit true
 *                             positives, and closest-hit ones under
 *                             HRPP_VERIFY_NONE -- are done, and only the
 *                             others are queued and traversed, so no warp
 *                             carries answered rays; 16 bytes of scratch per
 *                             ray.  It applies to table lookups of leaves
 *                             (Go Up Level 0) without learned predictions
 *                             or bottom-up verification; other calls, and
 *                             calls without a table, run BATCH.  No L2
 *                             window is set on its launches.)
 *   refill_min                REFILL: idle lanes needed before a warp refills,
 *                             1..32 (0 = default, 24)
 *   max_steps                 node visits allowed per traversal (0 = the
 *                             default, interior nodes + leaves + 8, which a
 *                             traversal of a valid tree never reaches; larger
 *                             values are clamped to it).  A ray that runs out
 *                             keeps its best hit so far and sets the scene's
 *                             error flag: the call returns
 *                             HRPP_ERR_TRAVERSAL_LIMIT when it synchronises
 *                             (host stats), else the next hrpp_scene_check
 *                             does.  For failure-detection tests.
 *   verify                    how a closest-hit true positive proves that no
 *                             closer hit exists (Sec. 4.3 admits the
 *                             unverified prediction can be wrong):
 *                             HRPP_VERIFY_ROOT (default) traverses from the
 *                             root bounded by the predicted hit;
 *                             HRPP_VERIFY_BOTTOM_UP climbs from the predicted
 *                             hit's leaf to the root, testing at each ancestor
 *                             only the children off the climb's path and
 *                             traversing those hit, bounded by the best hit.
 *                             Both return exactly the plain closest hit and
 *                             leave the same table; the climb skips one box
 *                             test per level and the predicted leaf's
 *                             re-test.  HRPP_VERIFY_NONE is the paper's own
 *                             semantics and NOT exact: a true positive
 *                             returns its predicted hit, which may not be the
 *                             closest, and does no traversal and no insert.
 *                             Other values: HRPP_ERR_INVALID_ARG.
 *   l2_persist                which device range the traversal launch marks
 *                             persisting in L2 (an access-policy window on
 *                             the launch): HRPP_L2_NONE (default),
 *                             HRPP_L2_TABLE (the table's words; nothing
 *                             without a table) or HRPP_L2_NODES (the scene's
 *                             interior nodes).  It takes effect only while
 *                             the context has a persisting-L2 set-aside
 *                             (hrpp_l2_set_aside); the window is clipped to
 *                             the device's maximum and its hit ratio is
 *                             set-aside / window bytes (at most 1).  Other
 *                             values: HRPP_ERR_INVALID_ARG. */
#define HRPP_SCHEDULE_DEFAULT 0u
#define HRPP_SCHEDULE_BATCH 1u
#define HRPP_SCHEDULE_REFILL 2u
#define HRPP_SCHEDULE_COMPACT 3u
#define HRPP_VERIFY_ROOT 0u
#define HRPP_VERIFY_BOTTOM_UP 1u
#define HRPP_VERIFY_NONE 2u
#define HRPP_L2_NONE 0u
#define HRPP_L2_TABLE 1u
#define HRPP_L2_NODES 2u
typedef struct hrpp_trace_opts {
    void *kernel_start, *kernel_stop;
    const int32_t *predicted_nodes;  /* device, one canonical node index per ray
                                        (-1 = none), e.g. from
                                        hrpp_proposal_predict: the ray
                                        traverses that node's subtree first */
    uint32_t block_threads;
    uint32_t schedule;
    uint32_t refill_min;
    uint32_t max_steps;
    uint32_t verify;
    uint32_t l2_persist;
    uint8_t *ray_outcome;     /* device, one per ray, or NULL: HRPP_OUTCOME_* */
    uint32_t *ray_box_tests;  /* device, one per ray, or NULL: box tests of the
                                 ray's traversal from the root (0 for an
                                 any-hit true positive; predicted subtrees
                                 not included) */
    uint32_t host_async;      /* host ray/hit buffers: 0 = the call returns
                                 with the hits in host memory; 1 = it returns
                                 at once, like a call on device buffers, and
                                 the hits are in host memory when `stream`
                                 reaches the end of the call's work (wait for
                                 the stream or an event recorded after the
                                 call).  The host buffers must be page-locked
                                 (HRPP_ERR_INVALID_ARG otherwise) and stay
                                 valid, the rays unmodified, until then.  A
                                 stopped ray is then reported by
                                 hrpp_scene_check; host out_stats still make
                                 the call wait.  At most 6 staged calls per
                                 device hold staging memory at once: a
                                 further one first waits on the host for
                                 the oldest one's downloads to finish. */
    void *host_done;          /* host_async: NULL, or a cudaEvent_t (as void*)
                                 that the library records once the hits are
                                 in host memory (device buffers: once they
                                 are final); `stream` then waits only for the
                                 traces, not for the hits' download, so later
                                 work on it (the next frame's traces)
                                 overlaps the download.  Wait for this event
                                 before reading the hits. */
    uint32_t stage_chunks;    /* host ray/hit buffers: at most this many
                                 staging chunks (each at least 2^18 rays);
                                 0 = the default, 8 for a call that waits
                                 (its copies overlap its own chunks'
                                 traces) and 2 for host_async (its copies
                                 mostly overlap the work queued around it);
                                 at most 64, else HRPP_ERR_INVALID_ARG */
} hrpp_trace_opts;
/* Per-ray outcome codes (Sec. 4.3).  The per-ray outputs above are filled
 * only when the call also collects statistics (out_stats != NULL). */
#define HRPP_OUTCOME_PLAIN 0      /* no lookup (no table, no prediction) */
#define HRPP_OUTCOME_NEGATIVE 1   /* nothing predicted */
#define HRPP_OUTCOME_FALSE_POS 2  /* predicted nodes held no valid hit */
#define HRPP_OUTCOME_TRUE_POS 3   /* a predicted node held a valid hit */

typedef struct hrpp_scene hrpp_scene;
typedef struct hrpp_table hrpp_table;

/* Checks a scene description on the host without touching any GPU.
 * tri_verts: 9 floats per triangle (v0, v1, v2).  nodes/root: the BVH
 * (canonical format above).  prim_index: n_prim_index == n_tris entries, a
 * permutation of 0..n_tris-1 in leaf order.  width: 2 or 4.  Accepts iff the
 * nodes reachable from root form a tree (no cycles, no node reached twice),
 * every triangle lies in exactly one leaf, leaves hold 1..HRPP_MAX_LEAF_TRIS
 * triangles, every child box lies inside its parent's, every leaf box holds
 * its triangles, and the traversal stack fits HRPP_MAX_STACK.  Fills *info
 * when info != NULL.  Returns INVALID_ARG / INVALID_BVH / UNSUPPORTED. */
hrpp_status hrpp_scene_validate(const float *tri_verts, uint32_t n_tris, const hrpp_bvh_node *nodes,
                                uint32_t n_nodes, uint32_t root, const uint32_t *prim_index,
                                uint32_t n_prim_index, int width, hrpp_scene_info *info);

/* Validates (as hrpp_scene_validate), converts the BVH to the device layout
 * (width 2: 64-byte nodes holding both child boxes; width 4: 128-byte SoA
 * nodes; triangles stored as v0, v1-v0, v2-v0 in leaf order), and uploads it
 * to the current device.  Blocking.  *out is set only on success. */
hrpp_status hrpp_scene_create(const float *tri_verts, uint32_t n_tris, const hrpp_bvh_node *nodes,
                              uint32_t n_nodes, uint32_t root, const uint32_t *prim_index,
                              uint32_t n_prim_index, int width, hrpp_scene **out);
hrpp_status hrpp_scene_get_info(const hrpp_scene *scene, hrpp_scene_info *info);
/* Waits for `stream`, then reads and clears the scene's sticky device error
 * flag: TRAVERSAL_LIMIT if a kernel on this scene stopped a ray early. */
hrpp_status hrpp_scene_check(hrpp_scene *scene, void *stream);
void hrpp_scene_destroy(hrpp_scene *scene);

/* Predictor table of 2^log2_entries 64-bit words in 2^log2_entries / ways
 * sets of `ways` words (ways in {1,2,4,8}; log2_entries in [ways' log2, 28]).
 * A word holds (tag << 28 | leaf), leaf = first_prim_index_slot << 2 |
 * (count - 1), or HRPP_EMPTY_WORD.  Paper Sec. 4.2: the table maps ray
 * hashes to leaf nodes; the paper's table is unbounded (Sec. 4.3, 6), this
 * one has fixed size: a leaf goes to way (leaf * 0x9E3779B1) >> (32 -
 * log2 ways) of its set, so one hash can hold up to `ways` distinct leaves.
 * Starts empty, precision 6 (Table 1), TWO_PHASE.  Blocking. */
hrpp_status hrpp_table_create(int log2_entries, int ways, hrpp_table **out);
/* precision_bits in [1, 7]: bits kept from each float's exponent and
 * mantissa by the Sec. 5 hash.  update_mode: hrpp_update_mode. */
hrpp_status hrpp_table_configure(hrpp_table *table, int precision_bits, int update_mode);
/* Go Up Level (Sec. 6.2), 0..15, default 0.  0: the table predicts leaves
 * (word leaf field = first_prim_index_slot << 2 | count - 1).  G > 0: it
 * predicts the ancestor G levels above the leaf a ray reached (the root if
 * the leaf is shallower), stored as that interior node's preorder rank
 * (children in slot order); a predicted ray traverses that subtree first.
 * Scenes whose root is a leaf store nothing for G > 0.  Changing G makes the
 * stored words meaningless: reset the table with it. */
hrpp_status hrpp_table_set_go_up(hrpp_table *table, int go_up_level);
/* Which exponent bits the ray hash keeps (a tuning knob; results never
 * depend on it): HRPP_HASH_EXP_MSB (default) takes the p most significant
 * exponent bits, as Sec. 5 defines the hash; HRPP_HASH_EXP_LSB takes the p
 * least significant ones, which separates neighbouring binades (1.0, 0.5,
 * 0.25 ...) that the Sec. 5 hash files under one key.  Sign and mantissa
 * bits are as in Sec. 5.  Changing it makes the stored words meaningless:
 * reset the table with it.  Other values: HRPP_ERR_INVALID_ARG. */
#define HRPP_HASH_EXP_MSB 0
#define HRPP_HASH_EXP_LSB 1
hrpp_status hrpp_table_set_hash(hrpp_table *table, int hash_variant);
/* Gate: lets a table stop predicting while its predictions do not pay (the
 * paper's predictor is always consulted; this is a policy on top of it, with
 * no counterpart in the paper).  min_tp_per_65536 == 0 (the default) turns
 * the gate off: every ray consults the table.  Otherwise the gate starts
 * open, and after each hrpp_trace / batch run it is set from that call alone:
 * open iff its true positives reach min_tp_per_65536 / 65536 of the rays
 * that consulted the table (a call in which none did leaves it as it was).
 * While it is closed, only the rays of every 2^sample_log2-th 32-ray chunk
 * (rays i with ((i >> 5) mod 2^sample_log2) == 0) consult and update the
 * table; every other ray traverses from the root with no lookup and no
 * insert and is counted in hrpp_stats.gated.  Results stay exact, and the
 * gate is deterministic: it depends only on the calls' rays and table.
 * sample_log2 in [0, 20] (default 5), else INVALID_ARG.  Blocking; opens
 * the gate.  hrpp_table_reset, hrpp_table_import and hrpp_table_set_gate
 * open it; hrpp_table_copy copies it. */
hrpp_status hrpp_table_set_gate(hrpp_table *table, uint32_t min_tp_per_65536, int sample_log2);
/* *open = 1 if the table's gate is open (always, without a gate).  Blocking. */
hrpp_status hrpp_table_get_gate(const hrpp_table *table, int *open);
/* Empties the table (asynchronous on stream) and unbinds it from its scene.
 * A table binds to the first scene it is traced with; tracing it with
 * another scene returns INVALID_ARG until it is reset. */
hrpp_status hrpp_table_reset(hrpp_table *table, void *stream);
/* Copies the 2^log2_entries table words to / from host memory (blocking;
 * n_words must equal the table size).  Import validates nothing about the
 * words' leaves: import only tables exported from the same scene. */
hrpp_status hrpp_table_export(const hrpp_table *table, uint64_t *host_words, size_t n_words);
hrpp_status hrpp_table_import(hrpp_table *table, const uint64_t *host_words, size_t n_words);
/* Device-to-device copy of src's words (and gate state) into dst, asynchronous on `stream`
 * (e.g. to restore a warm snapshot before each frame without a host round
 * trip).  Both tables must be on the same device with the same
 * log2_entries, ways, precision, Go Up Level and hash variant, else
 * HRPP_ERR_INVALID_ARG;
 * dst takes src's scene binding.  The update mode of dst is unchanged. */
hrpp_status hrpp_table_copy(hrpp_table *dst, const hrpp_table *src, void *stream);
hrpp_status hrpp_table_get_config(const hrpp_table *table, int *log2_entries, int *ways, int *precision_bits,
                                  int *update_mode);
void hrpp_table_destroy(hrpp_table *table);

/* Traces n_rays rays against scene.  table == NULL: plain BVH traversal.
 * Otherwise HRPP against table (Sec. 4.2-4.3), which it may update.
 *   rays      n_rays hrpp_ray, 16-byte aligned, device or host memory
 *   out_hits  closest: n_rays hrpp_hit (16-byte aligned); any: n_rays uint32
 *             (4-byte aligned); device or host memory
 *   out_stats NULL, or one hrpp_stats in device or host memory.  A host
 *             pointer makes the call wait for its kernels.
 * Host ray/hit buffers are staged through device memory the call allocates
 * and frees (stream-ordered), in chunks of a multiple of 32 rays (by default
 * up to 8 chunks of at least 2^18 rays; hrpp_trace_opts.stage_chunks):
 * chunk k+1 uploads on a library-owned copy
 * stream and chunk k-1 downloads on another while chunk k traces on
 * `stream`, so page-locked (pinned) buffers overlap copies with tracing.
 * Every chunk looks up the table as the call found it and two-phase inserts
 * land once, after the last chunk: results, counters and table equal those
 * of the same call on device buffers.  The uploads start at once, without
 * waiting for earlier work on `stream`: host rays that such work writes
 * must be complete before the call.  The call returns after the results
 * are back in host memory (or at once, with hrpp_trace_opts.host_async).
 * Device buffers keep the call fully asynchronous.
 * Calls that use the same table must be ordered on one stream.
 * n_rays == 0 does nothing (stats, if requested, are zeroed); n_rays above
 * 2^31 returns UNSUPPORTED.
 * Returns TRAVERSAL_LIMIT when the call waited and a ray was stopped early
 * (see hrpp_scene_check otherwise). */
hrpp_status hrpp_trace(const hrpp_scene *scene, hrpp_table *table, const hrpp_ray *rays, uint32_t n_rays,
                       hrpp_mode mode, void *out_hits, hrpp_stats *out_stats, void *stream);
/* hrpp_trace with per-call options (opts may be NULL). */
hrpp_status hrpp_trace_ex(const hrpp_scene *scene, hrpp_table *table, const hrpp_ray *rays, uint32_t n_rays,
                          hrpp_mode mode, void *out_hits, hrpp_stats *out_stats, void *stream,
                          const hrpp_trace_opts *opts);

/* Sets the current device's persisting-L2 set-aside (the part of L2 that
 * lines from an hrpp_trace_opts.l2_persist window may keep) to `bytes`,
 * clipped to the device's maximum, and writes the size in force to *granted
 * (may be NULL).  bytes == 0 releases it and returns lines already marked
 * persisting to normal.  The setting belongs to this process's CUDA context
 * on the current device: it applies to every kernel of the process that
 * uses an access-policy window and ends with the context.  Returns
 * HRPP_ERR_CUDA when the device has no persisting L2. */
hrpp_status hrpp_l2_set_aside(size_t bytes, size_t *granted);

/* hrpp_trace for callers that must not allocate device memory.  The paper
 * has no counterpart; this is a library-usage entry point.  hrpp_trace takes
 * its per-call scratch from a stream-ordered pool, which some callers cannot
 * allow: an engine whose own allocator reserved all device memory up front
 * (any further allocation would fail), or a real-time loop that bans
 * allocation calls because they can stall or synchronise the device.  This
 * variant allocates nothing: its scratch (a 256-byte control block plus one
 * 16-byte insert record per ray) lives in one fixed array of 256 B +
 * 16 B x HRPP_NOALLOC_MAX_RAYS (16 MiB) that every device loading the
 * library holds until the process exits.
 *   - rays and out_hits must be device memory (host buffers would need
 *     staging); out_stats may be NULL, device or host (host waits).
 *   - n_rays above HRPP_NOALLOC_MAX_RAYS returns INVALID_ARG; split larger
 *     batches into several calls.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture.
 *   - All calls on a device share its one array, which keeps the last
 *     call's contents (each call clears the control block it needs): calls
 *     whose work overlaps on the GPU, e.g. on two streams, race; order them,
 *     for instance on one stream.
 *   - The array's address is kept for the life of the device's context.
 *     cudaDeviceReset ends that context and every scene and table with it:
 *     the library is not used across a reset.
 * Results, statistics, table updates and the returned status equal
 * hrpp_trace's: with host out_stats the call waits, and a ray stopped early
 * returns HRPP_ERR_TRAVERSAL_LIMIT (clearing the scene's flag). */
#define HRPP_NOALLOC_MAX_RAYS (1u << 20)
hrpp_status hrpp_trace_noalloc(const hrpp_scene *scene, hrpp_table *table, const hrpp_ray *rays, uint32_t n_rays,
                               hrpp_mode mode, void *out_hits, hrpp_stats *out_stats, void *stream);

/* Batched traces: many (scene, table, rays) items -- scenes of different
 * sizes, batches of uneven lengths -- traced by one persistent kernel launch
 * per query mode (the closest-hit and any-hit launches run side by side),
 * plus one launch applying every two-phase table's inserts, recorded once
 * into a CUDA graph and replayed by hrpp_batch_run.  Per item the results,
 * counters and table updates are exactly those of hrpp_trace on that item.
 *   scene, table  as for hrpp_trace; all scenes of a batch share one device
 *                 and one BVH width; a table may serve one item only.
 *   rays, out_hits  device memory (16-byte aligned; hits 16/4-byte for
 *                 closest/any); the batch keeps these addresses: refill the
 *                 same buffers between runs.
 * Table settings (precision, update mode, Go Up Level) are read when the
 * batch is created. */
typedef struct hrpp_batch_item {
    const hrpp_scene *scene;
    hrpp_table *table;
    const hrpp_ray *rays;
    uint32_t n_rays;
    int mode;  /* hrpp_mode */
    void *out_hits;
} hrpp_batch_item;
typedef struct hrpp_batch hrpp_batch;
/* Validates the items, uploads the work list (32-ray chunks, each within one
 * item), allocates the batch's scratch and captures its graph.  collect_stats
 * != 0 keeps per-item counters (hrpp_batch_get_stats).  block_threads: 0
 * (default) or 64/128/256/512.  Blocking. */
hrpp_status hrpp_batch_create(const hrpp_batch_item *items, uint32_t n_items, int collect_stats,
                              uint32_t block_threads, hrpp_batch **out);
/* Replays the batch's graph on `stream` (asynchronous).  Runs of one batch,
 * and of batches sharing a table, must be ordered. */
hrpp_status hrpp_batch_run(hrpp_batch *batch, void *stream);
/* Waits for the batch's last run and copies item `item`'s counters. */
hrpp_status hrpp_batch_get_stats(hrpp_batch *batch, uint32_t item, hrpp_stats *host_stats);
void hrpp_batch_destroy(hrpp_batch *batch);

/* Learned treelet proposal (BASELINE's learned-proposal extension; no
 * counterpart in the paper, whose predictor is the hash table).  A small
 * BF16 MLP, 96 -> 256 -> 256 -> 4096 with ReLU and fp32 accumulation on the
 * tensor cores, predicts for each ray a BVH treelet: one of 4096 classes,
 * each a 12-bit path code from the root (BVH2: one child-slot bit per level;
 * BVH4: two bits per level), whose root is the deepest node that code
 * reaches.  A ray traverses its predicted treelet first (hrpp_trace_opts
 * predicted_nodes), so an any-hit ray answered there skips the rest, and
 * then traverses from the root exactly as without a prediction.
 * Inputs (96): the origin quantised to 16 bits per axis within the root
 * box, the octahedral-encoded direction quantised to 16 bits per component,
 * those 5 values as bf16(q / 32768 - 1), their Fourier terms
 * sin/cos(2 pi ((q << k) mod 2^16) / 2^16) for k = 0..8 from a bf16 sine
 * table, and a constant 1.  Training minimises the mean softmax
 * cross-entropy against the class of the leaf holding each ray's closest
 * hit (Adam, fp32 master weights). */
#define HRPP_PROPOSAL_FEATURES 96
#define HRPP_PROPOSAL_HIDDEN 256
#define HRPP_PROPOSAL_CLASSES 4096
/* weights as floats: W1 [256][96], b1 [256], W2 [256][256], b2 [256],
 * W3 [4096][256], b3 [4096] */
#define HRPP_PROPOSAL_PARAMS (256u * 96u + 256u + 256u * 256u + 256u + 4096u * 256u + 4096u)
typedef struct hrpp_proposal hrpp_proposal;
/* Makes a proposal network for `scene`, whose canonical BVH (as given to
 * hrpp_scene_create) defines the classes; weights drawn from `seed`
 * (He-uniform weights, zero biases).  Blocking. */
hrpp_status hrpp_proposal_create(const hrpp_scene *scene, const hrpp_bvh_node *nodes, uint32_t n_nodes, uint32_t root,
                                 const uint32_t *prim_index, uint32_t n_prim_index, uint64_t seed,
                                 hrpp_proposal **out);
/* Network inputs of n rays: bf16 [n][128] (96 features, 32 zeros), device;
 * out_bf16 must be 16-byte aligned (HRPP_ERR_INVALID_ARG otherwise). */
hrpp_status hrpp_proposal_features(hrpp_proposal *p, const hrpp_ray *rays, uint32_t n, void *out_bf16, void *stream);
/* Training labels from closest-hit results (device): the class of the leaf
 * holding each hit's triangle, -1 for a miss. */
hrpp_status hrpp_proposal_labels(hrpp_proposal *p, const hrpp_hit *hits, uint32_t n, int32_t *out_labels,
                                 void *stream);
/* One Adam step per minibatch of up to 16384 rays (device rays and labels;
 * label -1 = no target).  *out_mean_loss (host, may be NULL) receives the
 * mean loss over every labelled ray of the call, each minibatch's loss
 * taken before its own step (the call then waits); 0 if none was labelled.
 * Each minibatch's backward pass forks onto a stream the network owns and
 * joins `stream` again before its Adam step, so the call is ordered on
 * `stream` like a single-stream one.  Calls on one network must not run
 * concurrently. */
hrpp_status hrpp_proposal_train(hrpp_proposal *p, const hrpp_ray *rays, const int32_t *labels, uint32_t n, float lr,
                                float *out_mean_loss, void *stream);
/* Loss and gradients of one batch (n <= 16384) without updating: host_grads
 * receives HRPP_PROPOSAL_PARAMS floats in the weight layout above.  Waits. */
hrpp_status hrpp_proposal_gradients(hrpp_proposal *p, const hrpp_ray *rays, const int32_t *labels, uint32_t n,
                                    float *host_grads, float *out_mean_loss);
/* Predicted treelet root (canonical node index) and class per ray, device
 * outputs (out_classes may be NULL). */
hrpp_status hrpp_proposal_predict(hrpp_proposal *p, const hrpp_ray *rays, uint32_t n, int32_t *out_nodes,
                                  int32_t *out_classes, void *stream);
hrpp_status hrpp_proposal_get_weights(const hrpp_proposal *p, float *host, size_t n_floats);
hrpp_status hrpp_proposal_set_weights(hrpp_proposal *p, const float *host, size_t n_floats);
/* Class -> treelet root (canonical node) table, 4096 entries, host. */
hrpp_status hrpp_proposal_class_nodes(const hrpp_proposal *p, int32_t *host_nodes);
void hrpp_proposal_destroy(hrpp_proposal *p);

/* Utility (no counterpart in the paper; the learned treelet proposal's
 * building block, exposed for testing): C[m, n] = A[m, k] * B[n, k]^T on the
 * tensor cores (tcgen05.mma, fp32 accumulation in tensor memory, operands
 * loaded by TMA).  A, B: bf16, row-major with k contiguous (K-major), device
 * memory, 16-byte aligned; C: fp32 row-major [m, n], device memory, 32-byte
 * aligned.  m and n must be multiples of 128 and k of 64 (INVALID_ARG
 * otherwise, and for misaligned pointers).  Waits for the result. */
hrpp_status hrpp_gemm_bf16(const void *a, const void *b, float *c, int m, int n, int k, void *stream);
/* hrpp_gemm_bf16 with operand layouts (layout 0 is hrpp_gemm_bf16):
 *   HRPP_GEMM_A_MN_MAJOR  A is stored [k, m] (m contiguous), i.e. the
 *                         product uses its transpose without copying it
 *   HRPP_GEMM_B_MN_MAJOR  B is stored [k, n] (n contiguous)
 * Other bits: INVALID_ARG.  The learned proposal's weight gradients
 * (dW = dZ^T H over the rows of a minibatch) take both operands MN-major. */
#define HRPP_GEMM_A_MN_MAJOR 1
#define HRPP_GEMM_B_MN_MAJOR 2
hrpp_status hrpp_gemm_bf16_ex(const void *a, const void *b, float *c, int m, int n, int k, int layout,
                              void *stream);

const char *hrpp_last_error(void);
const char *hrpp_status_string(hrpp_status status);
int hrpp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HRPP_H */
