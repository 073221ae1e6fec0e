/*
 * Seeded synthetic inputs for HRPP workloads: scenes, BVHs and rays.
 *
 * This module is the one place both sides of a parity check draw their inputs
 * from.  It holds none of the method's arithmetic: no ray hash, no predictor
 * table, no ray-box or ray-triangle test and no traversal.  It makes
 *   - triangle soups for the stand-in scenes (icosphere, quad grid, value-noise
 *     terrain, uniform triangle soup),
 *   - deterministic binary BVHs (binned surface-area heuristic, or median
 *     split) and their 4-wide collapse, written in the canonical node format
 *     `hrpp_scene_create` takes,
 *   - camera, shadow, ambient-occlusion and uniform-sphere rays.
 * Random numbers come from PCG32 (O'Neill 2014, "PCG: A Family of Simple Fast
 * Space-Efficient Statistically Good Algorithms for Random Number Generation")
 * and the splitmix64 finaliser (Steele, Lea, Flood 2014), both written from
 * their published definitions.
 *
 * All generated geometry is computed in double precision and rounded to
 * IEEE-754 single precision once, so the float arrays are identical on every
 * host that runs this file (no x86- or Arm-specific code).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Canonical node: 48 bytes, identical in layout to hrpp_bvh_node. */
typedef struct {
    float lo[3], hi[3];
    int32_t child[4]; /* -1 = no child */
    uint32_t first, count; /* leaf iff count > 0: prim_index[first .. first+count) */
} sg_node;

/* ------------------------------------------------------------------ RNG -- */

uint64_t sg_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct {
    uint64_t state, inc;
} pcg32_t;

static uint32_t pcg32_next(pcg32_t *r)
{
    uint64_t old = r->state;
    r->state = old * 6364136223846793005ull + r->inc;
    uint32_t xorshifted = (uint32_t)(((old >> 18u) ^ old) >> 27u);
    uint32_t rot = (uint32_t)(old >> 59u);
    return (xorshifted >> rot) | (xorshifted << ((-rot) & 31u));
}

static void pcg32_seed(pcg32_t *r, uint64_t initstate, uint64_t initseq)
{
    r->state = 0u;
    r->inc = (initseq << 1u) | 1u;
    pcg32_next(r);
    r->state += initstate;
    pcg32_next(r);
}

/* uniform double in [0, 1) with 53 random bits */
static double pcg32_unit(pcg32_t *r)
{
    uint64_t hi = pcg32_next(r) >> 5;  /* 27 bits */
    uint64_t lo = pcg32_next(r) >> 6;  /* 26 bits */
    return (double)((hi << 26) | lo) * (1.0 / 9007199254740992.0);
}

/* n raw outputs of PCG32 seeded with (initstate, initseq); lets callers check
 * the generator against its published reference sequence. */
void sg_pcg32_stream(uint64_t initstate, uint64_t initseq, uint32_t n, uint32_t *out)
{
    pcg32_t r;
    pcg32_seed(&r, initstate, initseq);
    for (uint32_t i = 0; i < n; ++i) out[i] = pcg32_next(&r);
}

/* ------------------------------------------------------------- geometry -- */

static void put_tri(float *out, uint32_t idx, const double a[3], const double b[3], const double c[3])
{
    float *o = out + 9ull * idx;
    for (int k = 0; k < 3; ++k) {
        o[k] = (float)a[k];
        o[3 + k] = (float)b[k];
        o[6 + k] = (float)c[k];
    }
}

static void normalize3(double v[3])
{
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l;
    v[1] /= l;
    v[2] /= l;
}

typedef struct {
    double a[3], b[3], c[3];
} dtri;

static void icosphere_rec(const dtri *t, int depth, double cx, double cy, double cz, double r,
                          float *out, uint32_t *cursor)
{
    if (depth == 0) {
        double a[3], b[3], c[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = t->a[k] * r;
            b[k] = t->b[k] * r;
            c[k] = t->c[k] * r;
        }
        a[0] += cx; a[1] += cy; a[2] += cz;
        b[0] += cx; b[1] += cy; b[2] += cz;
        c[0] += cx; c[1] += cy; c[2] += cz;
        if (out) put_tri(out, *cursor, a, b, c);
        *cursor += 1;
        return;
    }
    /* midpoints: normalize(p + q) is symmetric in p, q, so shared edges split
     * at the same point in both neighbours and the sphere stays watertight */
    double ab[3], bc[3], ca[3];
    for (int k = 0; k < 3; ++k) {
        ab[k] = t->a[k] + t->b[k];
        bc[k] = t->b[k] + t->c[k];
        ca[k] = t->c[k] + t->a[k];
    }
    normalize3(ab);
    normalize3(bc);
    normalize3(ca);
    dtri s[4];
    memcpy(s[0].a, t->a, sizeof ab); memcpy(s[0].b, ab, sizeof ab); memcpy(s[0].c, ca, sizeof ab);
    memcpy(s[1].a, t->b, sizeof ab); memcpy(s[1].b, bc, sizeof ab); memcpy(s[1].c, ab, sizeof ab);
    memcpy(s[2].a, t->c, sizeof ab); memcpy(s[2].b, ca, sizeof ab); memcpy(s[2].c, bc, sizeof ab);
    memcpy(s[3].a, ab, sizeof ab);   memcpy(s[3].b, bc, sizeof ab); memcpy(s[3].c, ca, sizeof ab);
    for (int i = 0; i < 4; ++i) icosphere_rec(&s[i], depth - 1, cx, cy, cz, r, out, cursor);
}

/* Icosahedron subdivided `subdiv` times: 20 * 4^subdiv triangles on a sphere
 * of radius r about (cx, cy, cz).  out may be NULL to count. */
uint32_t sg_icosphere(int subdiv, float cx, float cy, float cz, float r, float *out)
{
    const double g = (1.0 + sqrt(5.0)) / 2.0;
    double v[12][3] = {{-1, g, 0}, {1, g, 0}, {-1, -g, 0}, {1, -g, 0}, {0, -1, g}, {0, 1, g},
                       {0, -1, -g}, {0, 1, -g}, {g, 0, -1}, {g, 0, 1}, {-g, 0, -1}, {-g, 0, 1}};
    static const int f[20][3] = {{0, 11, 5}, {0, 5, 1}, {0, 1, 7}, {0, 7, 10}, {0, 10, 11},
                                 {1, 5, 9}, {5, 11, 4}, {11, 10, 2}, {10, 7, 6}, {7, 1, 8},
                                 {3, 9, 4}, {3, 4, 2}, {3, 2, 6}, {3, 6, 8}, {3, 8, 9},
                                 {4, 9, 5}, {2, 4, 11}, {6, 2, 10}, {8, 6, 7}, {9, 8, 1}};
    for (int i = 0; i < 12; ++i) normalize3(v[i]);
    uint32_t cursor = 0;
    for (int i = 0; i < 20; ++i) {
        dtri t;
        memcpy(t.a, v[f[i][0]], sizeof t.a);
        memcpy(t.b, v[f[i][1]], sizeof t.a);
        memcpy(t.c, v[f[i][2]], sizeof t.a);
        icosphere_rec(&t, subdiv, cx, cy, cz, r, out, &cursor);
    }
    return cursor;
}

/* ---- value noise (lattice values from splitmix64, smoothstep blend) ---- */

static double lattice(uint64_t seed, int64_t i, int64_t j, int octave)
{
    uint64_t h = sg_splitmix64(seed ^ 0xD1B54A32D192ED03ull);
    h = sg_splitmix64(h ^ (uint64_t)i);
    h = sg_splitmix64(h ^ ((uint64_t)j * 0x9E3779B97F4A7C15ull));
    h = sg_splitmix64(h ^ (uint64_t)octave);
    return (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0; /* [-1, 1) */
}

static double smooth(double x) { return x * x * (3.0 - 2.0 * x); }

static double value_noise(uint64_t seed, double x, double z, int octave)
{
    double fi = floor(x), fj = floor(z);
    int64_t i = (int64_t)fi, j = (int64_t)fj;
    double sx = smooth(x - fi), sz = smooth(z - fj);
    double a = lattice(seed, i, j, octave), b = lattice(seed, i + 1, j, octave);
    double c = lattice(seed, i, j + 1, octave), d = lattice(seed, i + 1, j + 1, octave);
    double ab = a + (b - a) * sx, cd = c + (d - c) * sx;
    return ab + (cd - ab) * sz;
}

/* Terrain height: sum over octaves o of amp * 0.5^o * noise(x * freq * 2^o). */
double sg_terrain_height(uint64_t seed, int octaves, double amp, double freq, double x, double z)
{
    double h = 0.0, a = amp, f = freq;
    for (int o = 0; o < octaves; ++o) {
        h += a * value_noise(seed, x * f, z * f, o);
        a *= 0.5;
        f *= 2.0;
    }
    return h;
}

/* nx * nz quads over [x0,x1] x [z0,z1], two triangles each, split along the
 * (i,j)->(i+1,j+1) diagonal.  Heights are y0 when octaves == 0, else the
 * value-noise terrain.  out may be NULL to count. */
uint32_t sg_grid(int nx, int nz, float x0, float x1, float z0, float z1, float y0, uint64_t seed,
                 int octaves, float amp, float freq, float *out)
{
    uint32_t n = 2u * (uint32_t)nx * (uint32_t)nz;
    if (!out) return n;
    uint32_t cursor = 0;
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nx; ++i) {
            double p[4][3];
            for (int k = 0; k < 4; ++k) {
                int ii = i + (k & 1), jj = j + (k >> 1);
                double x = (double)x0 + ((double)x1 - (double)x0) * (double)ii / (double)nx;
                double z = (double)z0 + ((double)z1 - (double)z0) * (double)jj / (double)nz;
                double y = octaves > 0 ? sg_terrain_height(seed, octaves, amp, freq, x, z) : (double)y0;
                p[k][0] = x;
                p[k][1] = y;
                p[k][2] = z;
            }
            /* p[0]=(i,j) p[1]=(i+1,j) p[2]=(i,j+1) p[3]=(i+1,j+1) */
            put_tri(out, cursor++, p[0], p[1], p[3]);
            put_tri(out, cursor++, p[0], p[3], p[2]);
        }
    }
    return cursor;
}

/* n triangles with centroids uniform in [lo,hi]^3 and vertex offsets uniform
 * in +-extent about the centroid. */
uint32_t sg_soup(uint32_t n, uint64_t seed, float lo, float hi, float extent, float *out)
{
    pcg32_t r;
    pcg32_seed(&r, seed, 0x50u);
    for (uint32_t t = 0; t < n; ++t) {
        double c[3], v[3][3];
        for (int k = 0; k < 3; ++k) c[k] = lo + (hi - lo) * pcg32_unit(&r);
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < 3; ++k) v[q][k] = c[k] + extent * (2.0 * pcg32_unit(&r) - 1.0);
        put_tri(out, t, v[0], v[1], v[2]);
    }
    return n;
}

/* Places `count` spheres with radius log-uniform in [rmin, rmax] and centre
 * xz uniform over [x0,x1] x [z0,z1], resting on the value-noise terrain.
 * Writes (cx, cy, cz, r) per sphere. */
void sg_place_spheres(uint32_t count, uint64_t seed, float rmin, float rmax, float x0, float x1,
                      float z0, float z1, uint64_t terrain_seed, int octaves, float amp, float freq,
                      float *out4)
{
    pcg32_t r;
    pcg32_seed(&r, seed, 0x5E5u);
    for (uint32_t s = 0; s < count; ++s) {
        double rad = (double)rmin * pow((double)rmax / (double)rmin, pcg32_unit(&r));
        double x = x0 + rad + ((double)x1 - x0 - 2 * rad) * pcg32_unit(&r);
        double z = z0 + rad + ((double)z1 - z0 - 2 * rad) * pcg32_unit(&r);
        double y = octaves > 0 ? sg_terrain_height(terrain_seed, octaves, amp, freq, x, z) : 0.0;
        out4[4 * s + 0] = (float)x;
        out4[4 * s + 1] = (float)(y + rad);
        out4[4 * s + 2] = (float)z;
        out4[4 * s + 3] = (float)rad;
    }
}

/* ------------------------------------------------------------------ BVH -- */

typedef struct {
    const float *tris;
    float *cent; /* 3 per triangle */
    uint32_t *idx;
    sg_node *nodes;
    uint32_t n_nodes, cap;
    int max_leaf;
    uint64_t rng;
    int axis;
    int err;
    float *tb; /* SAH builder: 6 per triangle, its box (lo xyz, hi xyz) */
    double trav_cost; /* SAH builder: > 0 lets small nodes split when that is cheaper */
} bctx;

static int key_less(const bctx *c, uint32_t a, uint32_t b)
{
    float ka = c->cent[3ull * a + c->axis], kb = c->cent[3ull * b + c->axis];
    if (ka < kb) return 1;
    if (ka > kb) return 0;
    return a < b;
}

/* Rearranges idx[lo, hi) so that position k holds the element of rank k under
 * (centroid[axis], prim index), smaller elements before it and larger after. */
static void select_kth(bctx *c, uint32_t lo, uint32_t hi, uint32_t k)
{
    uint32_t *a = c->idx;
    while (hi - lo > 1) {
        c->rng = c->rng * 6364136223846793005ull + 1442695040888963407ull;
        uint32_t pi = lo + (uint32_t)((c->rng >> 33) % (hi - lo));
        uint32_t pv = a[pi];
        a[pi] = a[hi - 1];
        a[hi - 1] = pv;
        uint32_t store = lo;
        for (uint32_t i = lo; i < hi - 1; ++i) {
            if (key_less(c, a[i], pv)) {
                uint32_t t = a[i];
                a[i] = a[store];
                a[store] = t;
                ++store;
            }
        }
        a[hi - 1] = a[store];
        a[store] = pv;
        if (store == k) return;
        if (k < store) hi = store;
        else lo = store + 1;
    }
}

static int32_t build_rec(bctx *c, uint32_t begin, uint32_t end)
{
    if (c->n_nodes >= c->cap) {
        c->err = 1;
        return -1;
    }
    int32_t id = (int32_t)c->n_nodes++;
    sg_node *n = &c->nodes[id];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = begin; i < end; ++i) {
        const float *t = c->tris + 9ull * c->idx[i];
        const float *ce = c->cent + 3ull * c->idx[i];
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < 3; ++k) {
                if (t[3 * q + k] < lo[k]) lo[k] = t[3 * q + k];
                if (t[3 * q + k] > hi[k]) hi[k] = t[3 * q + k];
            }
        for (int k = 0; k < 3; ++k) {
            if (ce[k] < clo[k]) clo[k] = ce[k];
            if (ce[k] > chi[k]) chi[k] = ce[k];
        }
    }
    memcpy(n->lo, lo, sizeof lo);
    memcpy(n->hi, hi, sizeof hi);
    n->child[0] = n->child[1] = n->child[2] = n->child[3] = -1;
    if (end - begin <= (uint32_t)c->max_leaf) {
        n->first = begin;
        n->count = end - begin;
        return id;
    }
    n->first = 0;
    n->count = 0;
    /* longest centroid axis, ties to the lower axis */
    int axis = 0;
    float ext = chi[0] - clo[0];
    for (int k = 1; k < 3; ++k)
        if (chi[k] - clo[k] > ext) {
            ext = chi[k] - clo[k];
            axis = k;
        }
    c->axis = axis;
    uint32_t mid = begin + (end - begin) / 2;
    select_kth(c, begin, end, mid);
    int32_t l = build_rec(c, begin, mid);
    int32_t r = build_rec(c, mid, end);
    c->nodes[id].child[0] = l;
    c->nodes[id].child[1] = r;
    return id;
}

static void pad_boxes(const float *tris, uint32_t n_tris, sg_node *nodes, uint32_t n_nodes)
{
    /* pad = 2^-20 * max |coordinate|; every coordinate is <= M, so one ulp of
     * it is < pad and lo - pad, hi + pad move strictly outward */
    double m = 1.0;
    for (uint64_t i = 0; i < 9ull * n_tris; ++i) {
        double a = fabs((double)tris[i]);
        if (a > m) m = a;
    }
    float pad = (float)(m * ldexp(1.0, -20));
    for (uint32_t i = 0; i < n_nodes; ++i)
        for (int k = 0; k < 3; ++k) {
            nodes[i].lo[k] = nodes[i].lo[k] - pad;
            nodes[i].hi[k] = nodes[i].hi[k] + pad;
        }
}

/* Median-split binary BVH, <= max_leaf triangles per leaf, nodes in preorder
 * (root 0, left subtree before right).  nodes must hold 2*n_tris entries and
 * prim_index n_tris entries.  Returns 0 on success. */
int sg_build_bvh2(const float *tris, uint32_t n_tris, int max_leaf, sg_node *nodes, uint32_t *n_nodes,
                  uint32_t *prim_index)
{
    if (n_tris == 0 || max_leaf < 1) return 1;
    bctx c;
    memset(&c, 0, sizeof c);
    c.tris = tris;
    c.cent = (float *)malloc(sizeof(float) * 3ull * n_tris);
    if (!c.cent) return 2;
    for (uint32_t t = 0; t < n_tris; ++t)
        for (int k = 0; k < 3; ++k)
            c.cent[3ull * t + k] =
                (float)(((double)tris[9ull * t + k] + tris[9ull * t + 3 + k] + tris[9ull * t + 6 + k]) / 3.0);
    c.idx = prim_index;
    for (uint32_t t = 0; t < n_tris; ++t) prim_index[t] = t;
    c.nodes = nodes;
    c.cap = 2u * n_tris;
    c.max_leaf = max_leaf;
    c.rng = 0x853C49E6748FEA9Bull;
    build_rec(&c, 0, n_tris);
    free(c.cent);
    if (c.err) return 3;
    pad_boxes(tris, n_tris, nodes, c.n_nodes);
    *n_nodes = c.n_nodes;
    return 0;
}

/* Binned surface-area-heuristic split (Wald 2007, "On fast Construction of
 * SAH-based Bounding Volume Hierarchies"): each axis's centroid range is cut
 * into SAH_BINS bins; the plane between two bins with the least
 * area(left) * count(left) + area(right) * count(right) wins (ties to the lower
 * axis, then the lower plane).  Nodes of at most max_leaf triangles are
 * leaves; a node whose centroids all fall in one bin on every axis is split
 * at its median instead.  Partitions are stable, so the tree depends only on
 * the input. */
#define SAH_BINS 32

typedef struct {
    float lo[3], hi[3];
    uint32_t n;
} sbin;

static uint32_t bin_of(float cent, float clo, double scale)
{
    double b = ((double)cent - (double)clo) * scale;
    if (!(b > 0.0)) return 0;
    if (b >= (double)(SAH_BINS - 1)) return SAH_BINS - 1;
    return (uint32_t)b;
}

static double box_area(const float lo[3], const float hi[3])
{
    double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

static void box_grow(float lo[3], float hi[3], const float blo[3], const float bhi[3])
{
    for (int k = 0; k < 3; ++k) {
        if (blo[k] < lo[k]) lo[k] = blo[k];
        if (bhi[k] > hi[k]) hi[k] = bhi[k];
    }
}

static int32_t sah_rec(bctx *c, uint32_t *tmp, uint32_t begin, uint32_t end)
{
    if (c->n_nodes >= c->cap) {
        c->err = 1;
        return -1;
    }
    int32_t id = (int32_t)c->n_nodes++;
    sg_node *n = &c->nodes[id];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = begin; i < end; ++i) {
        const float *tb = c->tb + 6ull * c->idx[i];
        const float *ce = c->cent + 3ull * c->idx[i];
        box_grow(lo, hi, tb, tb + 3);
        box_grow(clo, chi, ce, ce);
    }
    memcpy(n->lo, lo, sizeof lo);
    memcpy(n->hi, hi, sizeof hi);
    n->child[0] = n->child[1] = n->child[2] = n->child[3] = -1;
    const uint32_t count = end - begin;
    if (count == 1 || (count <= (uint32_t)c->max_leaf && !(c->trav_cost > 0.0))) {
        n->first = begin;
        n->count = count;
        return id;
    }
    n->first = 0;
    n->count = 0;
    /* bin every triangle on the three axes in one pass */
    sbin bins[3][SAH_BINS];
    double scale[3];
    int live[3];
    for (int axis = 0; axis < 3; ++axis) {
        const float ext = chi[axis] - clo[axis];
        live[axis] = ext > 0.0f;
        scale[axis] = live[axis] ? (double)SAH_BINS / (double)ext : 0.0;
        for (int b = 0; b < SAH_BINS; ++b) {
            for (int k = 0; k < 3; ++k) {
                bins[axis][b].lo[k] = INFINITY;
                bins[axis][b].hi[k] = -INFINITY;
            }
            bins[axis][b].n = 0;
        }
    }
    for (uint32_t i = begin; i < end; ++i) {
        const uint32_t t = c->idx[i];
        const float *tb = c->tb + 6ull * t;
        const float *ce = c->cent + 3ull * t;
        for (int axis = 0; axis < 3; ++axis) {
            if (!live[axis]) continue;
            sbin *bn = &bins[axis][bin_of(ce[axis], clo[axis], scale[axis])];
            box_grow(bn->lo, bn->hi, tb, tb + 3);
            ++bn->n;
        }
    }
    double best = INFINITY;
    int best_axis = -1;
    uint32_t best_plane = 0;
    for (int axis = 0; axis < 3; ++axis) {
        if (!live[axis]) continue;
        /* left sweep: area and count of bins [0, b] */
        double left_area[SAH_BINS];
        uint32_t left_n[SAH_BINS];
        float l_lo[3] = {INFINITY, INFINITY, INFINITY}, l_hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        uint32_t ln = 0;
        for (int b = 0; b < SAH_BINS - 1; ++b) {
            if (bins[axis][b].n) box_grow(l_lo, l_hi, bins[axis][b].lo, bins[axis][b].hi);
            ln += bins[axis][b].n;
            left_n[b] = ln;
            left_area[b] = ln ? box_area(l_lo, l_hi) : 0.0;
        }
        /* right sweep: the plane below bin b splits [0, b) from [b, SAH_BINS) */
        float r_lo[3] = {INFINITY, INFINITY, INFINITY}, r_hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        uint32_t rn = 0;
        double right_cost[SAH_BINS];
        for (int b = SAH_BINS - 1; b >= 1; --b) {
            if (bins[axis][b].n) box_grow(r_lo, r_hi, bins[axis][b].lo, bins[axis][b].hi);
            rn += bins[axis][b].n;
            right_cost[b] = rn ? box_area(r_lo, r_hi) * (double)rn : 0.0;
        }
        for (int b = 1; b < SAH_BINS; ++b) {
            const uint32_t nl = left_n[b - 1], nr = (end - begin) - nl;
            if (nl == 0 || nr == 0) continue;
            const double cost = left_area[b - 1] * (double)nl + right_cost[b];
            if (cost < best) {
                best = cost;
                best_axis = axis;
                best_plane = (uint32_t)b;
            }
        }
    }
    if (count <= (uint32_t)c->max_leaf) {
        /* a node that may be a leaf splits only if the split's expected cost,
         * trav_cost x area + the children's area x count, is below the leaf's
         * area x count (triangle tests costing 1) */
        const double a = box_area(lo, hi);
        if (best_axis < 0 || !(c->trav_cost * a + best < a * (double)count)) {
            n->first = begin;
            n->count = count;
            return id;
        }
    }
    uint32_t mid;
    if (best_axis < 0) {
        /* every centroid in one bin: the median on the longest centroid axis */
        int axis = 0;
        float ext = chi[0] - clo[0];
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > ext) {
                ext = chi[k] - clo[k];
                axis = k;
            }
        c->axis = axis;
        mid = begin + (end - begin) / 2;
        select_kth(c, begin, end, mid);
    } else {
        uint32_t nl = 0, nr = 0;
        for (uint32_t i = begin; i < end; ++i) {
            const uint32_t t = c->idx[i];
            if (bin_of(c->cent[3ull * t + best_axis], clo[best_axis], scale[best_axis]) < best_plane)
                c->idx[begin + nl++] = t;
            else
                tmp[nr++] = t;
        }
        memcpy(c->idx + begin + nl, tmp, sizeof(uint32_t) * nr);
        mid = begin + nl;
    }
    int32_t l = sah_rec(c, tmp, begin, mid);
    int32_t r = sah_rec(c, tmp, mid, end);
    c->nodes[id].child[0] = l;
    c->nodes[id].child[1] = r;
    return id;
}

/* Binned-SAH binary BVH, <= max_leaf triangles per leaf, nodes in preorder,
 * boxes padded as sg_build_bvh2's.  Same arguments and results. */
int sg_build_bvh2_sah(const float *tris, uint32_t n_tris, int max_leaf, double trav_cost, sg_node *nodes,
                      uint32_t *n_nodes, uint32_t *prim_index)
{
    if (n_tris == 0 || max_leaf < 1) return 1;
    bctx c;
    memset(&c, 0, sizeof c);
    c.tris = tris;
    c.cent = (float *)malloc(sizeof(float) * 3ull * n_tris);
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_tris);
    c.tb = (float *)malloc(sizeof(float) * 6ull * n_tris);
    if (!c.cent || !tmp || !c.tb) {
        free(c.cent);
        free(tmp);
        free(c.tb);
        return 2;
    }
    for (uint32_t t = 0; t < n_tris; ++t) {
        const float *v = tris + 9ull * t;
        float *tb = c.tb + 6ull * t;
        for (int k = 0; k < 3; ++k) {
            c.cent[3ull * t + k] = (float)(((double)v[k] + v[3 + k] + v[6 + k]) / 3.0);
            tb[k] = fminf(fminf(v[k], v[3 + k]), v[6 + k]);
            tb[3 + k] = fmaxf(fmaxf(v[k], v[3 + k]), v[6 + k]);
        }
    }
    c.idx = prim_index;
    for (uint32_t t = 0; t < n_tris; ++t) prim_index[t] = t;
    c.nodes = nodes;
    c.cap = 2u * n_tris;
    c.max_leaf = max_leaf;
    c.trav_cost = trav_cost;
    c.rng = 0x853C49E6748FEA9Bull;
    sah_rec(&c, tmp, 0, n_tris);
    free(c.cent);
    free(tmp);
    free(c.tb);
    if (c.err) return 3;
    pad_boxes(tris, n_tris, nodes, c.n_nodes);
    *n_nodes = c.n_nodes;
    return 0;
}

static double area(const sg_node *n)
{
    double dx = (double)n->hi[0] - n->lo[0], dy = (double)n->hi[1] - n->lo[1], dz = (double)n->hi[2] - n->lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

typedef struct {
    const sg_node *in;
    sg_node *out;
    uint32_t n_out;
} cctx;

static int32_t collapse_rec(cctx *c, int32_t src)
{
    int32_t id = (int32_t)c->n_out++;
    const sg_node *s = &c->in[src];
    c->out[id] = *s;
    if (s->count > 0) return id;
    int32_t list[4];
    int cnt = 0;
    for (int k = 0; k < 4; ++k)
        if (s->child[k] >= 0) list[cnt++] = s->child[k];
    /* open the interior child with the largest surface area until 4 */
    while (cnt < 4) {
        int best = -1;
        double best_a = -1.0;
        for (int k = 0; k < cnt; ++k) {
            const sg_node *ch = &c->in[list[k]];
            int nch = 0;
            for (int q = 0; q < 4; ++q) nch += ch->child[q] >= 0;
            if (ch->count == 0 && cnt - 1 + nch <= 4 && area(ch) > best_a) {
                best_a = area(ch);
                best = k;
            }
        }
        if (best < 0) break;
        const sg_node *ch = &c->in[list[best]];
        int32_t kids[4];
        int nk = 0;
        for (int q = 0; q < 4; ++q)
            if (ch->child[q] >= 0) kids[nk++] = ch->child[q];
        for (int k = cnt - 1; k > best; --k) list[k + nk - 1] = list[k];
        for (int q = 0; q < nk; ++q) list[best + q] = kids[q];
        cnt += nk - 1;
    }
    int32_t out_children[4] = {-1, -1, -1, -1};
    for (int k = 0; k < cnt; ++k) out_children[k] = collapse_rec(c, list[k]);
    memcpy(c->out[id].child, out_children, sizeof out_children);
    return id;
}

/* Collapses a binary BVH (root 0) into a 4-wide one in preorder.  Boxes and
 * leaves are unchanged; out must hold n_in entries. */
int sg_collapse_bvh4(const sg_node *in, uint32_t n_in, sg_node *out, uint32_t *n_out)
{
    if (n_in == 0) return 1;
    cctx c = {in, out, 0};
    collapse_rec(&c, 0);
    *n_out = c.n_out;
    return 0;
}

/* ----------------------------------------------------------------- rays -- */

static void put_ray(float *out, uint64_t i, const double o[3], double tmin, const double d[3], double tmax)
{
    float *r = out + 8ull * i;
    r[0] = (float)o[0];
    r[1] = (float)o[1];
    r[2] = (float)o[2];
    r[3] = (float)tmin;
    r[4] = (float)d[0];
    r[5] = (float)d[1];
    r[6] = (float)d[2];
    r[7] = (float)tmax;
}

/* Pinhole camera rays, tmin 0, tmax +inf, written tile by tile (tile_w x
 * tile_h pixels, tiles in row-major order) so neighbouring rays are adjacent.
 * frame 0 uses pixel centres; frame f > 0 jitters each pixel by a PCG32 offset
 * in [-0.5, 0.5)^2 drawn from stream (seed, f). */
void sg_pinhole(const float eye[3], const float target[3], float vfov_deg, uint32_t w, uint32_t h,
                uint64_t seed, uint32_t frame, uint32_t tile_w, uint32_t tile_h, float *out)
{
    double e[3] = {eye[0], eye[1], eye[2]};
    double fw[3] = {(double)target[0] - e[0], (double)target[1] - e[1], (double)target[2] - e[2]};
    normalize3(fw);
    double up[3] = {0, 1, 0};
    double rt[3] = {fw[1] * up[2] - fw[2] * up[1], fw[2] * up[0] - fw[0] * up[2], fw[0] * up[1] - fw[1] * up[0]};
    normalize3(rt);
    double cu[3] = {rt[1] * fw[2] - rt[2] * fw[1], rt[2] * fw[0] - rt[0] * fw[2], rt[0] * fw[1] - rt[1] * fw[0]};
    double th = tan(0.5 * vfov_deg * 3.14159265358979323846 / 180.0);
    double aspect = (double)w / (double)h;
    pcg32_t r;
    pcg32_seed(&r, seed, 0x1000u + frame);
    if (tile_w == 0) tile_w = 1;
    if (tile_h == 0) tile_h = 1;
    uint32_t tiles_x = (w + tile_w - 1) / tile_w, tiles_y = (h + tile_h - 1) / tile_h;
    uint64_t k = 0;
    for (uint32_t ty = 0; ty < tiles_y; ++ty)
        for (uint32_t tx = 0; tx < tiles_x; ++tx)
            for (uint32_t yy = 0; yy < tile_h; ++yy)
                for (uint32_t xx = 0; xx < tile_w; ++xx) {
                    uint32_t px = tx * tile_w + xx, py = ty * tile_h + yy;
                    if (px >= w || py >= h) continue;
                    double jx = 0.0, jy = 0.0;
                    if (frame > 0) {
                        jx = pcg32_unit(&r) - 0.5;
                        jy = pcg32_unit(&r) - 0.5;
                    }
                    double sx = (2.0 * (px + 0.5 + jx) / w - 1.0) * th * aspect;
                    double sy = (1.0 - 2.0 * (py + 0.5 + jy) / h) * th;
                    double d[3];
                    for (int q = 0; q < 3; ++q) d[q] = fw[q] + sx * rt[q] + sy * cu[q];
                    normalize3(d);
                    put_ray(out, k++, e, 0.0, d, INFINITY);
                }
}

/* hit point and geometric normal facing the incoming ray */
static void hit_frame(const float *ray, float t, const float *tri, double p[3], double n[3])
{
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        p[k] = (double)ray[k] + (double)t * ray[4 + k];
        e1[k] = (double)tri[3 + k] - tri[k];
        e2[k] = (double)tri[6 + k] - tri[k];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    normalize3(n);
    if (n[0] * ray[4] + n[1] * ray[5] + n[2] * ray[6] > 0.0) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
    }
}

#define SG_NO_HIT 0xFFFFFFFFu

/* One shadow ray per hit toward a point light.  origin = p + 1e-4 n, tmax =
 * distance * (1 - 1e-4).  Returns the number written; src[i] = primary index. */
uint32_t sg_shadow_rays(const float *rays, const float *hit_t, const uint32_t *hit_prim, uint32_t n,
                        const float *tris, const float light[3], float *out, uint32_t *src)
{
    uint32_t k = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (hit_prim[i] == SG_NO_HIT) continue;
        double p[3], nn[3];
        hit_frame(rays + 8ull * i, hit_t[i], tris + 9ull * hit_prim[i], p, nn);
        double o[3], d[3];
        for (int q = 0; q < 3; ++q) o[q] = p[q] + 1e-4 * nn[q];
        for (int q = 0; q < 3; ++q) d[q] = (double)light[q] - o[q];
        double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int q = 0; q < 3; ++q) d[q] /= dist;
        put_ray(out, k, o, 0.0, d, dist * (1.0 - 1e-4));
        if (src) src[k] = i;
        ++k;
    }
    return k;
}

/* orthonormal basis about unit n (Duff et al. 2017, "Building an Orthonormal
 * Basis, Revisited") */
static void onb(const double n[3], double b1[3], double b2[3])
{
    double s = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (s + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + s * n[0] * n[0] * a;
    b1[1] = s * b;
    b1[2] = -s * n[0];
    b2[0] = b;
    b2[1] = s + n[1] * n[1] * a;
    b2[2] = -n[1];
}

/* per_hit cosine-weighted ambient-occlusion rays per hit (Malley's method:
 * uniform disk sample lifted onto the hemisphere about the geometric normal),
 * origin p + 1e-4 n, tmin 0, tmax `tmax`.  Random numbers from PCG32 stream
 * (seed, 0x2000 + frame).  Returns the number written. */
uint32_t sg_ao_rays(const float *rays, const float *hit_t, const uint32_t *hit_prim, uint32_t n,
                    const float *tris, uint32_t per_hit, float tmax, uint64_t seed, uint32_t frame,
                    float *out, uint32_t *src)
{
    pcg32_t r;
    pcg32_seed(&r, seed, 0x2000u + frame);
    uint32_t k = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (hit_prim[i] == SG_NO_HIT) continue;
        double p[3], nn[3], b1[3], b2[3];
        hit_frame(rays + 8ull * i, hit_t[i], tris + 9ull * hit_prim[i], p, nn);
        onb(nn, b1, b2);
        double o[3];
        for (int q = 0; q < 3; ++q) o[q] = p[q] + 1e-4 * nn[q];
        for (uint32_t s = 0; s < per_hit; ++s) {
            double u1 = pcg32_unit(&r), u2 = pcg32_unit(&r);
            double rad = sqrt(u1), phi = 2.0 * 3.14159265358979323846 * u2;
            double x = rad * cos(phi), y = rad * sin(phi), z = sqrt(1.0 - u1 > 0.0 ? 1.0 - u1 : 0.0);
            double d[3];
            for (int q = 0; q < 3; ++q) d[q] = x * b1[q] + y * b2[q] + z * nn[q];
            normalize3(d);
            put_ray(out, k, o, 0.0, d, tmax);
            if (src) src[k] = i;
            ++k;
        }
    }
    return k;
}

/* n rays with origins uniform in [lo,hi]^3 and directions uniform on the unit
 * sphere, tmin 0, tmax `tmax`. */
void sg_sphere_rays(uint32_t n, uint64_t seed, float lo, float hi, float tmax, float *out)
{
    pcg32_t r;
    pcg32_seed(&r, seed, 0x3000u);
    for (uint32_t i = 0; i < n; ++i) {
        double o[3], d[3];
        for (int q = 0; q < 3; ++q) o[q] = lo + ((double)hi - lo) * pcg32_unit(&r);
        double z = 2.0 * pcg32_unit(&r) - 1.0, phi = 2.0 * 3.14159265358979323846 * pcg32_unit(&r);
        double s = sqrt(1.0 - z * z > 0.0 ? 1.0 - z * z : 0.0);
        d[0] = s * cos(phi);
        d[1] = s * sin(phi);
        d[2] = z;
        normalize3(d);
        put_ray(out, i, o, 0.0, d, tmax);
    }
}
