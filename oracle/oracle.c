/*
 * HRPP oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of what the HRPP hot path
 * computes.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg and reference arm may load it; the library's product path never does.
 * It shares no code with the CUDA path (no headers, helpers or tables); the
 * two meet only at the input arrays the seeded generators make.
 *
 * Arithmetic is IEEE-754 single precision, the precision the paper states for
 * ray origin and direction (Sec. 5).  Build with -ffp-contract=off so every
 * product and sum rounds where it is written; fmaf() is a fused multiply-add
 * with one rounding, called where the definition below uses one.
 *
 * What each function follows:
 *   orc_hash_float / orc_ray_key     Sec. 5: sign bit, the p most significant
 *                                    exponent bits and the p most significant
 *                                    mantissa bits of each float; the origin
 *                                    hashes XORed with the swizzled direction
 *                                    hashes (ox^dz, oy^dy, oz^dx) and packed
 *                                    into at most 48 bits (16-bit fields).
 *   orc_hash_float_variant           the same with the p least significant
 *                                    exponent bits (a tuning variant, not
 *                                    the paper's definition).
 *   orc_mix48, set/tag, way          the bounded table's index (the paper
 *                                    indexes an unbounded map by the key,
 *                                    Sec. 4.2; a bounded table needs a set
 *                                    index and a tag -- our reading).
 *   orc_ray_triangle                 Moller-Trumbore (1997) with one fixed
 *                                    operation order; edges inclusive.
 *   orc_ray_box                      slab test with precomputed reciprocal
 *                                    direction and origin*reciprocal.
 *   orc_brute                        the result's plain definition: the
 *                                    lexicographic minimum (t, prim) over all
 *                                    triangles (closest) / existence of a
 *                                    valid hit (any).
 *   traversal (orc_trace, no table)  stack traversal from the root, children
 *                                    near-first (Sec. 3, 4.1).
 *   orc_trace with a table           Sec. 4.2-4.3: hash, look up, test the
 *                                    predicted leaves, skip interior traversal
 *                                    on a true positive, else traverse and
 *                                    insert the leaf reached (Sec. 5: no
 *                                    duplicate nodes per entry).
 *   verify_bottom_up                 exact verification of a closest-hit true
 *                                    positive by climbing from the predicted
 *                                    hit's leaf and traversing the siblings
 *                                    met on the way (the alternative to a
 *                                    bounded traversal from the root).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float lo[3], hi[3];
    int32_t child[4];
    uint32_t first, count;
} orc_node;

typedef struct {
    const float *tris;         /* 9 floats per triangle, caller order = prim id */
    uint32_t n_tris;
    const orc_node *nodes;
    uint32_t n_nodes;
    uint32_t root;
    const uint32_t *prim_index;
    uint32_t n_prim_index;
} orc_scene;

enum { ORC_ANY = 0, ORC_CLOSEST = 1 };
/* when and where inserts land: after the batch (two-phase), before the next
 * ray in the leaf's hashed way (sequential), in the unbounded map, or before
 * the next ray in the set's first empty way, else way (ray index mod W)
 * (online: the GPU's compare-and-swap placement, without its races) */
enum { ORC_TWO_PHASE = 0, ORC_SEQUENTIAL = 1, ORC_UNBOUNDED = 2, ORC_ONLINE = 3 };
/* how a closest-hit true positive is verified: a traversal from the root
 * bounded by the predicted hit, a climb from the predicted leaf testing the
 * siblings on the way up, or not at all (the paper's semantics, Sec. 4.3:
 * the predicted hit is returned as it is, and may not be the closest) */
enum { ORC_VERIFY_ROOT = 0, ORC_VERIFY_BOTTOM_UP = 1, ORC_VERIFY_NONE = 2 };

typedef struct {
    uint64_t *words;  /* 2^log2_sets * 2^log2_ways table words (bounded modes) */
    int log2_sets, log2_ways, precision;
    int update_mode;
    void *unbounded;  /* private state of the unbounded map */
    int go_up;        /* Sec. 6.2 Go Up Level: 0 = leaves, G > 0 = the ancestor G levels up */
    int hash_variant; /* ORC_HASH_EXP_MSB (Sec. 5, the default) or ORC_HASH_EXP_LSB */
    /* the gate (a policy on top of the method, not in the paper): with
     * gate_min_tp > 0, a call decides from its own rays whether the next call
     * consults the table: open iff true positives * 65536 >= gate_min_tp *
     * (rays that consulted the table).  While closed, only rays in 32-ray
     * chunks c with c mod 2^gate_sample_log2 == 0 consult (and update) it. */
    uint32_t gate_min_tp;
    int gate_sample_log2;
    int gate_open;
} orc_table;

/* Which exponent bits the per-float hash keeps: the p most significant ones
 * (Sec. 5 as written) or, as a tuning variant, the p least significant ones,
 * which tell neighbouring binades apart. */
enum { ORC_HASH_EXP_MSB = 0, ORC_HASH_EXP_LSB = 1 };

/* statistics counters, in this order */
enum {
    S_RAYS, S_HITS, S_LOOKUPS, S_POSITIVES, S_TRUE_POS, S_FALSE_POS, S_NEGATIVES, S_TP_INEXACT,
    S_INSERTS, S_DUP_INSERTS, S_EVICTIONS, S_INTERIOR, S_BOX_TESTS, S_LEAVES, S_TRI_TESTS,
    S_PRED_LEAVES, S_PRED_TRI_TESTS, S_PRED_INTERIOR, S_PRED_BOX_TESTS, S_GATED, S_COUNT = 20
};

/* per-ray outcome codes */
enum { OUT_PLAIN = 0, OUT_NEGATIVE = 1, OUT_FALSE_POS = 2, OUT_TRUE_POS = 3 };

#define NO_HIT 0xFFFFFFFFu
#define EMPTY_WORD 0xFFFFFFFFFFFFFFFFull
#define M48 0xFFFFFFFFFFFFull
#define TAG_BITS 36
#define LEAF_BITS 28

/* ------------------------------------------------------------- hashing -- */

/* Sec. 5: sign | top p exponent bits | top p mantissa bits, MSB to LSB. */
uint32_t orc_hash_float(float f, int p)
{
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    uint32_t sign = b >> 31;
    uint32_t expo = (b >> 23) & 0xFFu;
    uint32_t mant = b & 0x7FFFFFu;
    return (sign << (2 * p)) | ((expo >> (8 - p)) << p) | (mant >> (23 - p));
}

/* The exponent-LSB variant: sign, then the p least significant exponent
 * bits, then the p most significant mantissa bits (same field layout). */
uint32_t orc_hash_float_variant(float f, int p, int variant)
{
    if (variant != ORC_HASH_EXP_LSB) return orc_hash_float(f, p);
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    uint32_t sign = b >> 31;
    uint32_t expo = (b >> 23) & 0xFFu;
    uint32_t mant = b & 0x7FFFFFu;
    return (sign << (2 * p)) | ((expo & ((1u << p) - 1u)) << p) | (mant >> (23 - p));
}

/* Sec. 5: XOR origin hashes with swizzled direction hashes, pack to 48 bits. */
uint64_t orc_ray_key_variant(const float *ray, int p, int variant)
{
    uint64_t h0 = orc_hash_float_variant(ray[0], p, variant) ^ orc_hash_float_variant(ray[6], p, variant);
    uint64_t h1 = orc_hash_float_variant(ray[1], p, variant) ^ orc_hash_float_variant(ray[5], p, variant);
    uint64_t h2 = orc_hash_float_variant(ray[2], p, variant) ^ orc_hash_float_variant(ray[4], p, variant);
    return h0 | (h1 << 16) | (h2 << 32);
}

uint64_t orc_ray_key(const float *ray, int p) { return orc_ray_key_variant(ray, p, ORC_HASH_EXP_MSB); }

/* Bijective 48-bit mixer (xorshift-multiply rounds, odd multipliers). */
uint64_t orc_mix48(uint64_t k)
{
    k &= M48;
    k ^= k >> 23;
    k = (k * 0x9E3779B97F4Bull) & M48;
    k ^= k >> 25;
    k = (k * 0xC2B2AE3D27D5ull) & M48;
    k ^= k >> 21;
    return k;
}

/* Leaf identity: first prim_index slot and triangle count of a leaf node. */
static uint32_t leaf_id(const orc_node *n) { return (n->first << 2) | (n->count - 1u); }

static uint32_t way_of(uint32_t leaf, int log2_ways)
{
    if (log2_ways == 0) return 0;
    return (uint32_t)(leaf * 0x9E3779B1u) >> (32 - log2_ways);
}

/* ------------------------------------------------------------ geometry -- */

static float dot3(const float *a, const float *b) { return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2])); }

static void cross3(const float *a, const float *b, float *o)
{
    o[0] = fmaf(a[1], b[2], -(a[2] * b[1]));
    o[1] = fmaf(a[2], b[0], -(a[0] * b[2]));
    o[2] = fmaf(a[0], b[1], -(a[1] * b[0]));
}

/* Moller-Trumbore.  Valid iff det != 0, u >= 0, u <= 1, v >= 0, u + v <= 1,
 * tmin < t < tmax (tmax = the ray's own).  Writes t, u, v when valid. */
int orc_ray_triangle(const float *ray, const float *v0, const float *v1, const float *v2, float *t_out,
                     float *u_out, float *v_out)
{
    const float *o = ray, *d = ray + 4;
    float e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    float e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    float p[3];
    cross3(d, e2, p);
    float det = dot3(e1, p);
    if (det == 0.0f) return 0;
    float inv = 1.0f / det;
    float s[3] = {o[0] - v0[0], o[1] - v0[1], o[2] - v0[2]};
    float u = dot3(s, p) * inv;
    float q[3];
    cross3(s, e1, q);
    float v = dot3(d, q) * inv;
    float t = dot3(e2, q) * inv;
    if (!(u >= 0.0f && u <= 1.0f && v >= 0.0f && u + v <= 1.0f && t > ray[3] && t < ray[7])) return 0;
    *t_out = t;
    *u_out = u;
    *v_out = v;
    return 1;
}

/* Reciprocal direction; components with |d| < 2^-80 are replaced by
 * copysign(2^-80, d) so the reciprocal stays finite. */
void orc_ray_inverse(const float *ray, float *inv, float *oinv)
{
    for (int k = 0; k < 3; ++k) {
        float d = ray[4 + k];
        if (fabsf(d) < 0x1p-80f) d = copysignf(0x1p-80f, d);
        inv[k] = 1.0f / d;
        oinv[k] = ray[k] * inv[k];
    }
}

/* Slab test against [lo, hi]: t = lo*inv - o*inv per plane (one fused
 * multiply-add), entry tn = max(tmin, per-axis near), exit tf = min(tcur,
 * per-axis far); hit iff tn <= tf. */
int orc_ray_box(const float *inv, const float *oinv, float tmin, float tcur, const float *lo, const float *hi,
                float *tn_out)
{
    float near[3], far[3];
    for (int k = 0; k < 3; ++k) {
        float t0 = fmaf(lo[k], inv[k], -oinv[k]);
        float t1 = fmaf(hi[k], inv[k], -oinv[k]);
        near[k] = fminf(t0, t1);
        far[k] = fmaxf(t0, t1);
    }
    float tn = fmaxf(fmaxf(near[0], near[1]), fmaxf(near[2], tmin));
    float tf = fminf(fminf(far[0], far[1]), fminf(far[2], tcur));
    *tn_out = tn;
    return tn <= tf;
}

/* ---------------------------------------------------------- brute force -- */

/* Closest: (t, prim, u, v) of the lexicographic minimum (t, prim) over all
 * valid hits, or (+inf, NO_HIT, 0, 0).  near_tie[i] = 1 when another prim's
 * valid hit has |t2 - t1| <= 1e-6 t1.  Any: the lowest prim id with a valid
 * hit, or NO_HIT. */
void orc_brute(const float *rays, uint32_t n_rays, const float *tris, uint32_t n_tris, int mode, void *out,
               uint8_t *near_tie)
{
    for (uint32_t i = 0; i < n_rays; ++i) {
        const float *r = rays + 8ull * i;
        float bt = INFINITY, bu = 0.0f, bv = 0.0f;
        uint32_t bp = NO_HIT;
        for (uint32_t j = 0; j < n_tris; ++j) {
            const float *tr = tris + 9ull * j;
            float t, u, v;
            if (!orc_ray_triangle(r, tr, tr + 3, tr + 6, &t, &u, &v)) continue;
            if (mode == ORC_ANY) {
                bp = j;
                break;
            }
            if (t < bt || (t == bt && j < bp)) {
                bt = t;
                bu = u;
                bv = v;
                bp = j;
            }
        }
        if (mode == ORC_ANY) {
            ((uint32_t *)out)[i] = bp;
            continue;
        }
        float *h = (float *)out + 4ull * i;
        h[0] = bt;
        memcpy(&h[1], &bp, 4);
        h[2] = bu;
        h[3] = bv;
        if (near_tie) {
            uint8_t flag = 0;
            if (bp != NO_HIT) {
                for (uint32_t j = 0; j < n_tris; ++j) {
                    if (j == bp) continue;
                    const float *tr = tris + 9ull * j;
                    float t, u, v;
                    if (orc_ray_triangle(r, tr, tr + 3, tr + 6, &t, &u, &v) && fabsf(t - bt) <= 1e-6f * bt) flag = 1;
                }
            }
            near_tie[i] = flag;
        }
    }
}

/* ------------------------------------------------------------ traversal -- */

typedef struct {
    float t, u, v;
    uint32_t prim;
    uint32_t leaf;
    int found;
} best_hit;

typedef struct {
    uint32_t *stack;
    uint32_t cap;
} workspace;

/* Tests the triangles of leaf node n.  Any: stop at the first valid hit.
 * Closest: keep the lexicographic minimum (t, prim).  Returns 1 when an
 * any-hit query is answered. */
static int test_leaf(const orc_scene *sc, const orc_node *n, const float *ray, int mode, best_hit *b,
                     uint64_t *tri_counter)
{
    for (uint32_t j = 0; j < n->count; ++j) {
        uint32_t prim = sc->prim_index[n->first + j];
        const float *tr = sc->tris + 9ull * prim;
        float t, u, v;
        *tri_counter += 1;
        if (!orc_ray_triangle(ray, tr, tr + 3, tr + 6, &t, &u, &v)) continue;
        if (mode == ORC_ANY) {
            b->t = t;
            b->u = u;
            b->v = v;
            b->prim = prim;
            b->leaf = leaf_id(n);
            b->found = 1;
            return 1;
        }
        if (!b->found || t < b->t || (t == b->t && prim < b->prim)) {
            b->t = t;
            b->u = u;
            b->v = v;
            b->prim = prim;
            b->leaf = leaf_id(n);
            b->found = 1;
        }
    }
    return 0;
}

/* Which counters a traversal adds to: the main traversal, or the traversal
 * of a predicted subtree. */
typedef struct {
    int interior, box_tests, leaves, tri_tests;
} counter_set;

static const counter_set MAIN_COUNTERS = {S_INTERIOR, S_BOX_TESTS, S_LEAVES, S_TRI_TESTS};
static const counter_set PRED_COUNTERS = {S_PRED_INTERIOR, S_PRED_BOX_TESTS, S_PRED_LEAVES, S_PRED_TRI_TESTS};

/* Tests the boxes of interior node n's children (all but the child `skip`;
 * -1 skips none) against [tmin, tcur] and pushes the hit ones so that the
 * nearest, by (entry t, slot), is popped first.  Returns the box tests made. */
static uint32_t push_children(const orc_scene *sc, const orc_node *n, int32_t skip, const float *inv,
                              const float *oinv, const float *ray, float tcur, workspace *ws, uint32_t *sp)
{
    float tn[4];
    int slot[4], cnt = 0;
    uint32_t box_tests = 0;
    for (int s = 0; s < 4; ++s) {
        if (n->child[s] < 0 || n->child[s] == skip) continue;
        const orc_node *c = &sc->nodes[n->child[s]];
        box_tests += 1;
        float t;
        if (orc_ray_box(inv, oinv, ray[3], tcur, c->lo, c->hi, &t)) {
            tn[cnt] = t;
            slot[cnt] = s;
            ++cnt;
        }
    }
    /* insertion sort by (tn, slot); slots arrive ascending */
    for (int i = 1; i < cnt; ++i) {
        float kt = tn[i];
        int ks = slot[i], j = i - 1;
        while (j >= 0 && (tn[j] > kt || (tn[j] == kt && slot[j] > ks))) {
            tn[j + 1] = tn[j];
            slot[j + 1] = slot[j];
            --j;
        }
        tn[j + 1] = kt;
        slot[j + 1] = ks;
    }
    for (int i = cnt - 1; i >= 0; --i) ws->stack[(*sp)++] = (uint32_t)n->child[slot[i]];
    return box_tests;
}

/* Runs the stack until it is empty (or an any-hit ray is answered): leaves
 * test their triangles, interior nodes push their hit children with the
 * current bound (the ray's tmax, or the best hit so far in closest mode).
 * Returns 1 if the best hit changed. */
static int run_stack(const orc_scene *sc, const float *ray, const float *inv, const float *oinv, int mode,
                     best_hit *b, workspace *ws, uint32_t *sp, uint64_t *st, counter_set cs, uint32_t *box_tests)
{
    int changed = 0;
    while (*sp > 0) {
        const orc_node *n = &sc->nodes[ws->stack[--(*sp)]];
        if (n->count > 0) {
            st[cs.leaves] += 1;
            best_hit before = *b;
            int done = test_leaf(sc, n, ray, mode, b, &st[cs.tri_tests]);
            if (b->found && (!before.found || b->prim != before.prim || b->t != before.t)) changed = 1;
            if (done) break;
            continue;
        }
        st[cs.interior] += 1;
        float tcur = (mode == ORC_CLOSEST && b->found) ? b->t : ray[7];
        *box_tests += push_children(sc, n, -1, inv, oinv, ray, tcur, ws, sp);
    }
    return changed;
}

/* Stack traversal of the subtree under `start` (the root for the main
 * traversal), children that are hit visited nearest first, ordered by
 * (entry t, slot).  Returns 1 if the best hit changed during this traversal. */
static int traverse_from(const orc_scene *sc, uint32_t start, const float *ray, int mode, best_hit *b,
                         workspace *ws, uint64_t *st, counter_set cs, uint32_t *box_tests_out)
{
    float inv[3], oinv[3];
    orc_ray_inverse(ray, inv, oinv);
    uint32_t sp = 0, box_tests = 0;
    ws->stack[sp++] = start;
    int changed = run_stack(sc, ray, inv, oinv, mode, b, ws, &sp, st, cs, &box_tests);
    st[cs.box_tests] += box_tests;
    if (box_tests_out) *box_tests_out = box_tests;
    return changed;
}

static int traverse(const orc_scene *sc, const float *ray, int mode, best_hit *b, workspace *ws, uint64_t *st,
                    uint32_t *box_tests_out)
{
    return traverse_from(sc, sc->root, ray, mode, b, ws, st, MAIN_COUNTERS, box_tests_out);
}

/* Tree facts the Go Up Level needs (Sec. 6.2): each node's parent, and each
 * interior node's identity = its rank in preorder from the root with
 * children taken in slot order. */
typedef struct {
    int32_t *parent;      /* per node; -1 for the root and unreached nodes */
    int32_t *rank;        /* per node: preorder rank among interior nodes, else -1 */
    int32_t *by_rank;     /* rank -> node */
    int32_t *leaf_at;     /* prim_index slot -> the leaf node starting there, else -1 */
    uint32_t n_interior;
} tree_info;

static void tree_info_free(tree_info *t)
{
    free(t->parent);
    free(t->rank);
    free(t->by_rank);
    free(t->leaf_at);
}

static int tree_info_build(const orc_scene *sc, tree_info *t)
{
    memset(t, 0, sizeof *t);
    t->parent = (int32_t *)malloc(sizeof(int32_t) * sc->n_nodes);
    t->rank = (int32_t *)malloc(sizeof(int32_t) * sc->n_nodes);
    t->by_rank = (int32_t *)malloc(sizeof(int32_t) * sc->n_nodes);
    t->leaf_at = (int32_t *)malloc(sizeof(int32_t) * (sc->n_prim_index ? sc->n_prim_index : 1));
    uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * (sc->n_nodes + 4));
    if (!t->parent || !t->rank || !t->by_rank || !t->leaf_at || !stack) {
        free(stack);
        tree_info_free(t);
        return 1;
    }
    for (uint32_t i = 0; i < sc->n_nodes; ++i) t->parent[i] = t->rank[i] = -1;
    for (uint32_t i = 0; i < sc->n_prim_index; ++i) t->leaf_at[i] = -1;
    uint32_t sp = 0;
    stack[sp++] = sc->root;
    while (sp > 0) {
        uint32_t ni = stack[--sp];
        const orc_node *n = &sc->nodes[ni];
        if (n->count > 0) {
            if (n->first < sc->n_prim_index) t->leaf_at[n->first] = (int32_t)ni;
            continue;
        }
        t->rank[ni] = (int32_t)t->n_interior;
        t->by_rank[t->n_interior++] = (int32_t)ni;
        for (int s = 3; s >= 0; --s)
            if (n->child[s] >= 0) {
                t->parent[n->child[s]] = (int32_t)ni;
                stack[sp++] = (uint32_t)n->child[s];
            }
    }
    free(stack);
    return 0;
}

/* Table node of the leaf where a hit was found: the leaf itself (G = 0) or
 * its ancestor G levels up, stopping at the root (G > 0; then the preorder
 * rank).  Returns -1 when there is nothing to store (the root is a leaf). */
static int64_t predicted_node(const orc_scene *sc, const tree_info *t, uint32_t leaf, int go_up)
{
    if (go_up == 0) return leaf;
    int32_t n = t->leaf_at[leaf >> 2];
    if (n < 0 || t->parent[n] < 0) return -1;
    n = t->parent[n];
    for (int g = 1; g < go_up && t->parent[n] >= 0; ++g) n = t->parent[n];
    return t->rank[n];
}

/* Bottom-up verification of a closest-hit true positive (the exact
 * alternative to re-traversing from the root, Sec. 4.3 / Sec. 6.2): from the
 * leaf holding the best hit so far, climb to the root; at each ancestor, test
 * the boxes of its children other than the one the climb came from against
 * [tmin, best t] and traverse the hit ones nearest first, as the main
 * traversal would.  Every leaf but the starting one lies under exactly one
 * of those siblings, so the final hit is the plain closest hit.  Counts the
 * ancestors as interior nodes and their sibling boxes as box tests.  Returns
 * 1 if the best hit changed. */
static int verify_bottom_up(const orc_scene *sc, const tree_info *t, const float *ray, best_hit *b, workspace *ws,
                            uint64_t *st, uint32_t *box_tests_out)
{
    float inv[3], oinv[3];
    orc_ray_inverse(ray, inv, oinv);
    int32_t from = t->leaf_at[b->leaf >> 2];
    int32_t a = from >= 0 ? t->parent[from] : -1;
    uint32_t sp = 0, box_tests = 0;
    int changed = 0;
    while (a >= 0) {
        st[S_INTERIOR] += 1;
        box_tests += push_children(sc, &sc->nodes[a], from, inv, oinv, ray, b->t, ws, &sp);
        changed |= run_stack(sc, ray, inv, oinv, ORC_CLOSEST, b, ws, &sp, st, MAIN_COUNTERS, &box_tests);
        from = a;
        a = t->parent[a];
    }
    st[S_BOX_TESTS] += box_tests;
    if (box_tests_out) *box_tests_out = box_tests;
    return changed;
}

/* ------------------------------------------------------- unbounded map -- */

typedef struct {
    uint64_t key;
    uint32_t n, cap;
    uint32_t *leaves;
} ub_entry;

typedef struct {
    ub_entry *slots;
    uint64_t cap, used;
} ub_map;

static ub_entry *ub_find(ub_map *m, uint64_t key, int create)
{
    if (!m->slots) {
        if (!create) return NULL;
        m->cap = 1024;
        m->slots = (ub_entry *)calloc(m->cap, sizeof(ub_entry));
        for (uint64_t i = 0; i < m->cap; ++i) m->slots[i].key = EMPTY_WORD;
    }
    if (create && 2 * (m->used + 1) > m->cap) {
        ub_entry *old = m->slots;
        uint64_t oc = m->cap;
        m->cap *= 2;
        m->slots = (ub_entry *)calloc(m->cap, sizeof(ub_entry));
        for (uint64_t i = 0; i < m->cap; ++i) m->slots[i].key = EMPTY_WORD;
        for (uint64_t i = 0; i < oc; ++i) {
            if (old[i].key == EMPTY_WORD) continue;
            uint64_t h = orc_mix48(old[i].key) & (m->cap - 1);
            while (m->slots[h].key != EMPTY_WORD) h = (h + 1) & (m->cap - 1);
            m->slots[h] = old[i];
        }
        free(old);
    }
    uint64_t h = orc_mix48(key) & (m->cap - 1);
    while (m->slots[h].key != EMPTY_WORD) {
        if (m->slots[h].key == key) return &m->slots[h];
        h = (h + 1) & (m->cap - 1);
    }
    if (!create) return NULL;
    m->slots[h].key = key;
    m->slots[h].n = m->slots[h].cap = 0;
    m->slots[h].leaves = NULL;
    m->used += 1;
    return &m->slots[h];
}

/* Number of keys and of stored leaves in the unbounded map. */
void orc_unbounded_size(const orc_table *tab, uint64_t *keys, uint64_t *leaves)
{
    *keys = *leaves = 0;
    const ub_map *m = (const ub_map *)tab->unbounded;
    if (!m || !m->slots) return;
    for (uint64_t i = 0; i < m->cap; ++i)
        if (m->slots[i].key != EMPTY_WORD) {
            *keys += 1;
            *leaves += m->slots[i].n;
        }
}

void orc_unbounded_free(orc_table *tab)
{
    ub_map *m = (ub_map *)tab->unbounded;
    if (!m) return;
    if (m->slots)
        for (uint64_t i = 0; i < m->cap; ++i) free(m->slots[i].leaves);
    free(m->slots);
    free(m);
    tab->unbounded = NULL;
}

/* ----------------------------------------------------------------- trace -- */

typedef struct {
    uint32_t slot;
    uint64_t value;
} record;

static const orc_node *find_leaf(const orc_scene *sc, uint32_t leaf)
{
    /* the predictor stores (first << 2 | count - 1); rebuild a leaf node view */
    static __thread orc_node tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.first = leaf >> 2;
    tmp.count = (leaf & 3u) + 1u;
    if (tmp.first + tmp.count > sc->n_prim_index) return NULL;
    return &tmp;
}

/*
 * Traces n rays.  table == NULL: plain traversal.  Otherwise HRPP (Sec. 4.2-4.3):
 *   1. key = hash of the ray (Sec. 5); m = mix48(key); set = m mod S,
 *      tag = (m >> log2 S) mod 2^36.
 *   2. candidates = leaves of the set's ways whose tag matches, in way order
 *      (unbounded mode: every leaf stored under the key, in insertion order).
 *   3. no candidate: negative -> traverse from the root.
 *      any-hit: a valid hit in a candidate leaf is a true positive and ends
 *      the ray with no interior traversal; otherwise a false positive ->
 *      traverse.  closest-hit: no valid candidate hit is a false positive ->
 *      traverse; otherwise a true positive -> traverse from the root bounded
 *      by the candidates' best hit, so the result is exact (a closer hit found
 *      there counts as tp_inexact).
 *   4. a ray that traversed and hit, in a leaf that was not a candidate,
 *      inserts (tag, leaf) at way way_of(leaf) of its set.  Two-phase: every
 *      lookup of the batch sees the table as it was at batch start, and the
 *      highest ray index targeting a slot wins it after the batch; a record
 *      that loses counts as dup_inserts, a winner that overwrites a valid
 *      word as an eviction.  Sequential: each insert lands before the next
 *      ray.  Online: each insert lands before the next ray, in the set's
 *      first empty way, else in way (ray index mod W) as an eviction.
 *      Unbounded: the leaf is appended to the key's list.
 * out: closest -> 4 words per ray (t, prim, u, v); any -> prim or NO_HIT.
 * outcome (optional): OUT_* code per ray.  ray_box_tests (optional): box tests
 * each ray's traversal made.  Returns 0, or 1 on bad arguments / no memory.
 */
int orc_trace(const orc_scene *sc, const float *rays, uint32_t n_rays, int mode, orc_table *tab, void *out,
              uint64_t *stats, uint8_t *outcome, uint32_t *ray_box_tests, const int32_t *predicted, int verify)
{
    if (!sc || (!rays && n_rays) || (!out && n_rays) || !stats) return 1;
    workspace ws;
    ws.cap = sc->n_nodes * 4u + 8u;
    ws.stack = (uint32_t *)malloc(sizeof(uint32_t) * ws.cap);
    record *recs = NULL;
    uint32_t n_recs = 0;
    int bounded = tab && tab->update_mode != ORC_UNBOUNDED;
    uint32_t ways = tab ? (1u << tab->log2_ways) : 1u;
    if (tab && tab->update_mode == ORC_TWO_PHASE) recs = (record *)malloc(sizeof(record) * (n_rays ? n_rays : 1));
    if (tab && tab->update_mode == ORC_UNBOUNDED && !tab->unbounded) tab->unbounded = calloc(1, sizeof(ub_map));
    tree_info ti;
    int go_up = tab ? tab->go_up : 0;
    if (!ws.stack || (tab && tab->update_mode == ORC_TWO_PHASE && !recs) || tree_info_build(sc, &ti)) {
        free(ws.stack);
        free(recs);
        return 1;
    }
    /* the gate as the call starts (its state changes only after the batch) */
    const int gated_table = tab && tab->gate_min_tp > 0;
    const int admit_all = !gated_table || tab->gate_open;
    const uint32_t sample_mask = gated_table ? (1u << tab->gate_sample_log2) - 1u : 0u;
    uint64_t gate_lookups = 0, gate_tp = 0;
    for (uint32_t i = 0; i < n_rays; ++i) {
        const float *ray = rays + 8ull * i;
        /* does this ray consult the table?  every ray while the gate is open;
         * while it is closed, the rays of the sampled 32-ray chunks */
        const int consult = tab && (admit_all || ((i >> 5) & sample_mask) == 0u);
        best_hit b;
        memset(&b, 0, sizeof b);
        b.t = INFINITY;
        b.prim = NO_HIT;
        stats[S_RAYS] += 1;
        uint8_t oc = OUT_PLAIN;
        int run_traversal = 1;
        uint32_t cand_local[8];
        const uint32_t *cand = cand_local;
        uint32_t n_cand = 0;
        uint64_t set = 0, tag = 0;
        uint64_t key = 0;
        int learned_positive = 0;
        if (predicted) {
            /* a predicted treelet (learned proposal): traverse the subtree of
             * the given node first, when it is a node of the tree */
            int32_t c = predicted[i];
            int reachable = 0;
            if (c >= 0 && (uint32_t)c < sc->n_nodes) {
                const orc_node *pn = &sc->nodes[c];
                reachable = pn->count > 0 ? (pn->first < sc->n_prim_index && ti.leaf_at[pn->first] == c)
                                          : ti.rank[c] >= 0;
            }
            if (reachable) {
                learned_positive = 1;
                traverse_from(sc, (uint32_t)c, ray, mode, &b, &ws, stats, PRED_COUNTERS, NULL);
            }
        }
        if (tab && !consult) stats[S_GATED] += 1;
        if (consult || predicted) {
            stats[S_LOOKUPS] += 1;
            if (!consult) {
                /* learned proposal only */
            } else if ((key = orc_ray_key_variant(ray, tab->precision, tab->hash_variant)), bounded) {
                uint64_t m = orc_mix48(key);
                set = m & ((1ull << tab->log2_sets) - 1ull);
                tag = (m >> tab->log2_sets) & ((1ull << TAG_BITS) - 1ull);
                for (uint32_t w = 0; w < ways; ++w) {
                    uint64_t word = tab->words[set * ways + w];
                    if (word != EMPTY_WORD && (word >> LEAF_BITS) == tag)
                        cand_local[n_cand++] = (uint32_t)(word & ((1u << LEAF_BITS) - 1u));
                }
            } else {
                ub_entry *e = ub_find((ub_map *)tab->unbounded, key, 0);
                if (e) {
                    cand = e->leaves;
                    n_cand = e->n;
                }
            }
            if (n_cand == 0 && !learned_positive) {
                oc = OUT_NEGATIVE;
                stats[S_NEGATIVES] += 1;
            } else {
                stats[S_POSITIVES] += 1;
                int answered = mode == ORC_ANY && b.found;
                for (uint32_t k = 0; k < n_cand && !answered; ++k) {
                    if (go_up == 0) {
                        const orc_node *lf = find_leaf(sc, cand[k]);
                        if (!lf) continue;
                        stats[S_PRED_LEAVES] += 1;
                        answered = test_leaf(sc, lf, ray, mode, &b, &stats[S_PRED_TRI_TESTS]);
                    } else {
                        /* Sec. 6.2: a predicted interior node; the ray traverses its subtree */
                        if (cand[k] >= ti.n_interior) continue;
                        best_hit before = b;
                        traverse_from(sc, (uint32_t)ti.by_rank[cand[k]], ray, mode, &b, &ws, stats, PRED_COUNTERS, NULL);
                        answered = mode == ORC_ANY && b.found && !before.found;
                    }
                }
                if (b.found) {
                    oc = OUT_TRUE_POS;
                    stats[S_TRUE_POS] += 1;
                    if (mode == ORC_ANY || verify == ORC_VERIFY_NONE) run_traversal = 0;
                } else {
                    oc = OUT_FALSE_POS;
                    stats[S_FALSE_POS] += 1;
                }
            }
        }
        if (run_traversal) {
            best_hit pred = b;
            int changed;
            if (verify == ORC_VERIFY_BOTTOM_UP && mode == ORC_CLOSEST && oc == OUT_TRUE_POS)
                changed = verify_bottom_up(sc, &ti, ray, &b, &ws, stats, ray_box_tests ? &ray_box_tests[i] : NULL);
            else
                changed = traverse(sc, ray, mode, &b, &ws, stats, ray_box_tests ? &ray_box_tests[i] : NULL);
            if (oc == OUT_TRUE_POS && changed && (b.prim != pred.prim || b.t != pred.t)) stats[S_TP_INEXACT] += 1;
            int64_t node = (consult && b.found) ? predicted_node(sc, &ti, b.leaf, go_up) : -1;
            if (node >= 0) {
                int is_cand = 0;
                for (uint32_t k = 0; k < n_cand; ++k) is_cand |= cand[k] == (uint32_t)node;
                if (!is_cand) {
                    stats[S_INSERTS] += 1;
                    if (bounded) {
                        uint32_t slot = (uint32_t)(set * ways + way_of((uint32_t)node, tab->log2_ways));
                        uint64_t value = (tag << LEAF_BITS) | (uint64_t)node;
                        if (tab->update_mode == ORC_SEQUENTIAL) {
                            uint64_t old = tab->words[slot];
                            if (old == value) stats[S_DUP_INSERTS] += 1;
                            else if (old != EMPTY_WORD) stats[S_EVICTIONS] += 1;
                            tab->words[slot] = value;
                        } else if (tab->update_mode == ORC_ONLINE) {
                            /* the set's first empty way; with none, way (i mod W) */
                            uint64_t *sw = tab->words + set * ways;
                            uint32_t k = 0;
                            while (k < ways && sw[k] != EMPTY_WORD) ++k;
                            if (k == ways) {
                                k = i & (ways - 1u);
                                stats[S_EVICTIONS] += 1;
                            }
                            sw[k] = value;
                        } else {
                            recs[n_recs].slot = slot;
                            recs[n_recs].value = value;
                            ++n_recs;
                        }
                    } else {
                        ub_entry *e = ub_find((ub_map *)tab->unbounded, key, 1);
                        if (e->n == e->cap) {
                            e->cap = e->cap ? 2 * e->cap : 4;
                            e->leaves = (uint32_t *)realloc(e->leaves, sizeof(uint32_t) * e->cap);
                        }
                        e->leaves[e->n++] = (uint32_t)node;
                    }
                }
            }
        } else if (ray_box_tests) {
            ray_box_tests[i] = 0;
        }
        if (b.found) stats[S_HITS] += 1;
        if (consult) {
            gate_lookups += 1;
            gate_tp += oc == OUT_TRUE_POS;
        }
        if (outcome) outcome[i] = oc;
        if (mode == ORC_ANY) {
            ((uint32_t *)out)[i] = b.found ? b.prim : NO_HIT;
        } else {
            float *h = (float *)out + 4ull * i;
            h[0] = b.found ? b.t : INFINITY;
            uint32_t p = b.found ? b.prim : NO_HIT;
            memcpy(&h[1], &p, 4);
            h[2] = b.found ? b.u : 0.0f;
            h[3] = b.found ? b.v : 0.0f;
        }
    }
    if (recs) {
        /* after the batch, in ascending ray order: the last record aimed at a
         * slot is the one that stays; walking backwards, the first sighting
         * of each slot is that winner */
        uint64_t n_slots = (1ull << tab->log2_sets) * ways;
        uint8_t *seen = (uint8_t *)calloc((n_slots + 7) / 8, 1);
        for (uint32_t k = n_recs; k-- > 0;) {
            uint32_t s = recs[k].slot;
            if (seen[s >> 3] & (1u << (s & 7))) {
                stats[S_DUP_INSERTS] += 1;
                continue;
            }
            seen[s >> 3] |= (uint8_t)(1u << (s & 7));
            if (tab->words[s] != EMPTY_WORD) stats[S_EVICTIONS] += 1;
            tab->words[s] = recs[k].value;
        }
        free(seen);
    }
    /* the gate for the next call, from this call's rays that consulted the table */
    if (gated_table && gate_lookups) tab->gate_open = (gate_tp << 16) >= (uint64_t)tab->gate_min_tp * gate_lookups;
    free(recs);
    free(ws.stack);
    tree_info_free(&ti);
    return 0;
}
