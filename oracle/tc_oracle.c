/*
 * tc_oracle.c -- plain FP64 CPU oracle of the treecode force phase.
 *
 * TEST INFRASTRUCTURE ONLY (see tc_oracle.h).  Slow and direct on purpose:
 * every quantity is computed from its definition, in the order the paper
 * describes the method (Sec. 3.1): build the oct-tree by recursive
 * subdivision, give every cell its mass and centre of mass, walk the tree
 * from the root building an interaction list, loop over the list with the
 * force law, then move the bodies.
 *
 * Readings of what the paper leaves open (it names no bounding box, key,
 * threshold rule, opening test, softening or integrator):
 *   R1 root cube: a power-of-two cube on a 2^21 grid, so that every cell
 *      corner is an exact binary fraction (or_root_cube).
 *   R2 subdivision: a cube is split while it holds MORE than leaf_max
 *      bodies and is above level 21; empty sub-cubes are not kept.
 *   R3 bodies sharing a leaf are ordered by Morton key, then by original
 *      index (a stable sort).
 *   R4 groups: contiguous runs of at most gmax bodies that share one walk
 *      (or_tree_make_groups).
 *   R5 "distant enough": a cell of side s whose centre of mass lies at
 *      distance d from the group's bounding box is accepted iff it holds
 *      none of the group's bodies and s < theta * d.
 *   R6 force law with Plummer softening eps:
 *      a_i = G sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2).
 *   R7 kick-drift-kick leapfrog.
 */
#include "tc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* R1: root cube.                                                      */
/* The cube side is the smallest power of two L with                   */
/* L >= extent * (1 + 2^-20), extent the largest axis range; the grid  */
/* step is h = L / 2^21 and the corner c0 = floor(min / h) * h on each */
/* axis.  With this choice the largest body still falls strictly       */
/* inside the cube (extent <= L - 2h and c0 > min - h).                */
/* ------------------------------------------------------------------ */
static double next_pow2(double t)
{
    int e;
    double m = frexp(t, &e); /* t = m * 2^e, m in [0.5, 1) */
    if (m == 0.5)
        return t;
    return ldexp(1.0, e);
}

int or_root_cube(const float *pos, int64_t n, double *out5)
{
    if (n < 1)
        return -1;
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (int64_t i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++) {
            double x = (double)pos[3 * i + a];
            if (!isfinite(x))
                return -1;
            if (x < lo[a])
                lo[a] = x;
            if (x > hi[a])
                hi[a] = x;
        }
    }
    double extent = 0.0;
    for (int a = 0; a < 3; a++)
        if (hi[a] - lo[a] > extent)
            extent = hi[a] - lo[a];
    double target = extent * (1.0 + ldexp(1.0, -20));
    double L = (target > 0.0) ? next_pow2(target) : 1.0; /* all bodies coincide: unit cube */
    double h = L / 2097152.0;                             /* 2^21 */
    for (int a = 0; a < 3; a++)
        out5[a] = floor(lo[a] / h) * h;
    out5[3] = L;
    out5[4] = h;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Morton keys.  Each coordinate is quantised to a 21-bit cell index   */
/* q = floor((x - c0) / h), clamped to [0, 2^21 - 1]; the key takes    */
/* one bit of each axis per level, most significant level first, with  */
/* the x bit highest in each 3-bit digit.  The digit at level l        */
/* (1..21) is the octant (4*xbit + 2*ybit + zbit) of the level-l cube  */
/* inside its parent.                                                  */
/* ------------------------------------------------------------------ */
static uint64_t quantise(double x, double c0, double h)
{
    /* (x - c0) / h evaluated exactly: h is a power of two and c0 an integer
     * multiple of h, so x / h and c0 / h are exact and so is the difference
     * of their integer parts */
    double q = floor(x / h) - c0 / h;
    if (q < 0.0)
        q = 0.0;
    if (q > 2097151.0)
        q = 2097151.0;
    return (uint64_t)q;
}

void or_keys(const float *pos, int64_t n, const double *cube5, uint64_t *keys)
{
    for (int64_t i = 0; i < n; i++) {
        uint64_t q[3];
        for (int a = 0; a < 3; a++)
            q[a] = quantise((double)pos[3 * i + a], cube5[a], cube5[4]);
        uint64_t k = 0;
        for (int b = 20; b >= 0; b--) {
            uint64_t digit = (((q[0] >> b) & 1u) << 2) | (((q[1] >> b) & 1u) << 1) | ((q[2] >> b) & 1u);
            k = (k << 3) | digit;
        }
        keys[i] = k;
    }
}

static int digit_at(uint64_t key, int level) /* level 1..21 */
{
    return (int)((key >> (3 * (OR_MAX_LEVEL - level))) & 7u);
}

/* ------------------------------------------------------------------ */
/* Tree storage.                                                       */
/* ------------------------------------------------------------------ */
struct or_tree {
    int64_t n;
    int leaf_max;
    double cube[5];
    uint64_t *keys; /* sorted */
    uint32_t *perm; /* sorted position -> original index */
    double *xs;     /* sorted positions, n x 3 */
    double *ms;     /* sorted masses */

    int64_t M; /* nodes, breadth-first order */
    int32_t *level;
    uint64_t *prefix;
    int64_t *first, *count, *child_first, *parent;
    int32_t *nchild;
    double *mass, *com, *quad;

    int64_t G; /* groups */
    int64_t *gfirst, *gcount, *gref;
};

typedef struct {
    uint64_t key;
    uint32_t idx;
} kv_t;

static int cmp_kv(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/* Pre-order record produced by the recursive subdivision. */
typedef struct {
    int32_t level;
    uint64_t prefix;
    int64_t first, count, parent_pre;
} rec_t;

typedef struct {
    rec_t *v;
    int64_t n, cap;
} recvec_t;

static int64_t push_rec(recvec_t *r, rec_t x)
{
    if (r->n == r->cap) {
        r->cap = r->cap ? 2 * r->cap : 1024;
        r->v = (rec_t *)realloc(r->v, (size_t)r->cap * sizeof(rec_t));
    }
    r->v[r->n] = x;
    return r->n++;
}

/* R2: recursive subdivision (Sec. 3.1).  The bodies of the cube
 * (level, prefix) are the sorted range [first, first + count); its
 * non-empty octants are consecutive sub-ranges because keys are sorted. */
static void subdivide(const or_tree *t, recvec_t *out, int level, uint64_t prefix,
                      int64_t first, int64_t count, int64_t parent_pre)
{
    rec_t me = {level, prefix, first, count, parent_pre};
    int64_t self = push_rec(out, me);
    if (count <= t->leaf_max || level == OR_MAX_LEVEL)
        return; /* leaf */
    int64_t s = first, end = first + count;
    for (int o = 0; o < 8; o++) {
        int64_t e = s;
        while (e < end && digit_at(t->keys[e], level + 1) == o)
            e++;
        if (e > s)
            subdivide(t, out, level + 1, (prefix << 3) | (uint64_t)o, s, e - s, self);
        s = e;
    }
}

static const rec_t *g_sort_recs; /* qsort context (single-threaded oracle) */
static int cmp_bfs(const void *a, const void *b)
{
    const rec_t *x = &g_sort_recs[*(const int64_t *)a];
    const rec_t *y = &g_sort_recs[*(const int64_t *)b];
    if (x->level != y->level)
        return x->level < y->level ? -1 : 1;
    return x->first < y->first ? -1 : (x->first > y->first);
}

or_tree *or_tree_build(const float *pos, const float *mass, int64_t n, int leaf_max)
{
    if (n < 1 || leaf_max < 1)
        return NULL;
    for (int64_t i = 0; i < n; i++) /* masses must be finite and positive */
        if (!isfinite((double)mass[i]) || !(mass[i] > 0.0f))
            return NULL;
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    t->n = n;
    t->leaf_max = leaf_max;
    if (or_root_cube(pos, n, t->cube) != 0) {
        free(t);
        return NULL;
    }

    /* keys, then the stable (key, index) sort (R3) */
    uint64_t *k = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    or_keys(pos, n, t->cube, k);
    kv_t *kv = (kv_t *)malloc((size_t)n * sizeof(kv_t));
    for (int64_t i = 0; i < n; i++) {
        kv[i].key = k[i];
        kv[i].idx = (uint32_t)i;
    }
    qsort(kv, (size_t)n, sizeof(kv_t), cmp_kv);
    free(k);
    t->keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    t->perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    t->xs = (double *)malloc((size_t)n * 3 * sizeof(double));
    t->ms = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        t->keys[i] = kv[i].key;
        t->perm[i] = kv[i].idx;
        for (int a = 0; a < 3; a++)
            t->xs[3 * i + a] = (double)pos[3 * (int64_t)kv[i].idx + a];
        t->ms[i] = (double)mass[kv[i].idx];
    }
    free(kv);

    /* the oct-tree in pre-order, then re-ordered breadth-first */
    recvec_t recs = {0};
    subdivide(t, &recs, 0, 0, 0, n, -1);
    int64_t M = recs.n;
    int64_t *order = (int64_t *)malloc((size_t)M * sizeof(int64_t));
    for (int64_t i = 0; i < M; i++)
        order[i] = i;
    g_sort_recs = recs.v;
    qsort(order, (size_t)M, sizeof(int64_t), cmp_bfs);
    int64_t *bfs_of_pre = (int64_t *)malloc((size_t)M * sizeof(int64_t));
    for (int64_t b = 0; b < M; b++)
        bfs_of_pre[order[b]] = b;

    t->M = M;
    t->level = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    t->prefix = (uint64_t *)malloc((size_t)M * sizeof(uint64_t));
    t->first = (int64_t *)malloc((size_t)M * sizeof(int64_t));
    t->count = (int64_t *)malloc((size_t)M * sizeof(int64_t));
    t->child_first = (int64_t *)malloc((size_t)M * sizeof(int64_t));
    t->parent = (int64_t *)malloc((size_t)M * sizeof(int64_t));
    t->nchild = (int32_t *)calloc((size_t)M, sizeof(int32_t));
    for (int64_t b = 0; b < M; b++) {
        const rec_t *r = &recs.v[order[b]];
        t->level[b] = r->level;
        t->prefix[b] = r->prefix;
        t->first[b] = r->first;
        t->count[b] = r->count;
        t->parent[b] = r->parent_pre < 0 ? -1 : bfs_of_pre[r->parent_pre];
        t->child_first[b] = -1;
    }
    for (int64_t b = 0; b < M; b++) {
        int64_t p = t->parent[b];
        if (p < 0)
            continue;
        t->nchild[p]++;
        if (t->child_first[p] < 0 || b < t->child_first[p])
            t->child_first[p] = b;
    }
    free(order);
    free(bfs_of_pre);
    free(recs.v);

    /* mass, centre of mass and second moments of every cell, each from
     * the definition over the cell's own bodies (Sec. 3.1: a cell stands
     * for its bodies by one body of their total mass at their centre of
     * mass). */
    t->mass = (double *)malloc((size_t)M * sizeof(double));
    t->com = (double *)malloc((size_t)M * 3 * sizeof(double));
    t->quad = (double *)malloc((size_t)M * 6 * sizeof(double));
    for (int64_t v = 0; v < M; v++) {
        double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t j = t->first[v]; j < t->first[v] + t->count[v]; j++) {
            m += t->ms[j];
            sx += t->ms[j] * t->xs[3 * j + 0];
            sy += t->ms[j] * t->xs[3 * j + 1];
            sz += t->ms[j] * t->xs[3 * j + 2];
        }
        double c[3] = {sx / m, sy / m, sz / m};
        double q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = t->first[v]; j < t->first[v] + t->count[v]; j++) {
            double dx = t->xs[3 * j + 0] - c[0];
            double dy = t->xs[3 * j + 1] - c[1];
            double dz = t->xs[3 * j + 2] - c[2];
            double mj = t->ms[j];
            q[0] += mj * dx * dx;
            q[1] += mj * dx * dy;
            q[2] += mj * dx * dz;
            q[3] += mj * dy * dy;
            q[4] += mj * dy * dz;
            q[5] += mj * dz * dz;
        }
        t->mass[v] = m;
        for (int a = 0; a < 3; a++)
            t->com[3 * v + a] = c[a];
        for (int a = 0; a < 6; a++)
            t->quad[6 * v + a] = q[a];
    }
    return t;
}

void or_tree_free(or_tree *t)
{
    if (!t)
        return;
    free(t->keys);
    free(t->perm);
    free(t->xs);
    free(t->ms);
    free(t->level);
    free(t->prefix);
    free(t->first);
    free(t->count);
    free(t->child_first);
    free(t->parent);
    free(t->nchild);
    free(t->mass);
    free(t->com);
    free(t->quad);
    free(t->gfirst);
    free(t->gcount);
    free(t->gref);
    free(t);
}

int64_t or_tree_nnodes(const or_tree *t) { return t->M; }
int64_t or_tree_nbodies(const or_tree *t) { return t->n; }
void or_tree_get_cube(const or_tree *t, double *out5) { memcpy(out5, t->cube, 5 * sizeof(double)); }
void or_tree_get_perm(const or_tree *t, uint32_t *perm) { memcpy(perm, t->perm, (size_t)t->n * sizeof(uint32_t)); }
void or_tree_get_keys(const or_tree *t, uint64_t *k) { memcpy(k, t->keys, (size_t)t->n * sizeof(uint64_t)); }

void or_tree_get_nodes(const or_tree *t, int32_t *level, uint64_t *prefix, int64_t *first,
                       int64_t *count, int64_t *child_first, int32_t *nchild, int64_t *parent)
{
    size_t M = (size_t)t->M;
    if (level)
        memcpy(level, t->level, M * sizeof(int32_t));
    if (prefix)
        memcpy(prefix, t->prefix, M * sizeof(uint64_t));
    if (first)
        memcpy(first, t->first, M * sizeof(int64_t));
    if (count)
        memcpy(count, t->count, M * sizeof(int64_t));
    if (child_first)
        memcpy(child_first, t->child_first, M * sizeof(int64_t));
    if (nchild)
        memcpy(nchild, t->nchild, M * sizeof(int32_t));
    if (parent)
        memcpy(parent, t->parent, M * sizeof(int64_t));
}

void or_tree_get_moments(const or_tree *t, double *mass, double *com, double *quad)
{
    size_t M = (size_t)t->M;
    if (mass)
        memcpy(mass, t->mass, M * sizeof(double));
    if (com)
        memcpy(com, t->com, M * 3 * sizeof(double));
    if (quad)
        memcpy(quad, t->quad, M * 6 * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* R4: groups.  The paper walks the tree once per body (Sec. 3.2); the */
/* walk here is shared by a group of at most gmax bodies that are      */
/* contiguous in Morton order (gmax = 1 is the per-body walk).  Rule,  */
/* applied from the root down:                                         */
/*   - a cube holding at most gmax bodies that is the root is a group; */
/*   - a leaf holding more than gmax bodies is cut into consecutive    */
/*     chunks of gmax (the last one shorter);                          */
/*   - the children of an internal cube holding more than gmax bodies  */
/*     are taken in octant order: a child holding more than gmax is    */
/*     handled by these rules in turn; runs of consecutive children    */
/*     holding at most gmax each are packed greedily, left to right,   */
/*     into groups of at most gmax bodies.                             */
/* Each group has a reference cube: the cube itself for a single cube  */
/* or a chunk of a leaf, the common parent for several packed children.*/
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t *first, *count, *ref;
    int64_t n, cap;
} grpvec_t;

static void push_group(grpvec_t *g, int64_t first, int64_t count, int64_t ref)
{
    if (g->n == g->cap) {
        g->cap = g->cap ? 2 * g->cap : 1024;
        g->first = (int64_t *)realloc(g->first, (size_t)g->cap * sizeof(int64_t));
        g->count = (int64_t *)realloc(g->count, (size_t)g->cap * sizeof(int64_t));
        g->ref = (int64_t *)realloc(g->ref, (size_t)g->cap * sizeof(int64_t));
    }
    g->first[g->n] = first;
    g->count[g->n] = count;
    g->ref[g->n] = ref;
    g->n++;
}

static void group_cube(const or_tree *t, grpvec_t *out, int64_t v, int gmax)
{
    if (t->count[v] <= gmax) { /* only the root gets here */
        push_group(out, t->first[v], t->count[v], v);
        return;
    }
    if (t->nchild[v] == 0) { /* over-full leaf: chunks */
        for (int64_t s = 0; s < t->count[v]; s += gmax) {
            int64_t c = t->count[v] - s < gmax ? t->count[v] - s : gmax;
            push_group(out, t->first[v] + s, c, v);
        }
        return;
    }
    int64_t run_first = -1, run_count = 0, run_len = 0, run_only = -1;
    for (int64_t c = t->child_first[v]; c < t->child_first[v] + t->nchild[v]; c++) {
        if (t->count[c] > gmax || run_count + t->count[c] > gmax) {
            if (run_len > 0)
                push_group(out, run_first, run_count, run_len == 1 ? run_only : v);
            run_len = 0;
            run_count = 0;
        }
        if (t->count[c] > gmax) {
            group_cube(t, out, c, gmax);
            continue;
        }
        if (run_len == 0) {
            run_first = t->first[c];
            run_only = c;
        }
        run_count += t->count[c];
        run_len++;
    }
    if (run_len > 0)
        push_group(out, run_first, run_count, run_len == 1 ? run_only : v);
}

int64_t or_tree_make_groups(or_tree *t, int gmax)
{
    if (gmax < 1)
        return -1;
    grpvec_t g = {0};
    group_cube(t, &g, 0, gmax);
    free(t->gfirst);
    free(t->gcount);
    free(t->gref);
    t->gfirst = g.first;
    t->gcount = g.count;
    t->gref = g.ref;
    t->G = g.n;
    return g.n;
}

void or_tree_get_groups(const or_tree *t, int64_t *first, int64_t *count, int64_t *ref)
{
    size_t G = (size_t)t->G;
    if (first)
        memcpy(first, t->gfirst, G * sizeof(int64_t));
    if (count)
        memcpy(count, t->gcount, G * sizeof(int64_t));
    if (ref)
        memcpy(ref, t->gref, G * sizeof(int64_t));
}

/* ------------------------------------------------------------------ */
/* R5: the opening test ("distant enough", Sec. 3.1).                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t gfirst, gcount;
    double lo[3], hi[3]; /* tight box of the group's bodies */
    double theta;
    int flagged;
    /* lists */
    int64_t *cells, ncells, cap_c;
    int64_t *leaves, nleaves, cap_l;
    int64_t nbody;
} walk_t;

static double cube_side(const or_tree *t, int64_t v) { return ldexp(t->cube[3], -t->level[v]); }

static double dist_to_box(const double *p, const double *lo, const double *hi)
{
    double s = 0.0;
    for (int a = 0; a < 3; a++) {
        double e = 0.0;
        if (p[a] < lo[a])
            e = lo[a] - p[a];
        else if (p[a] > hi[a])
            e = p[a] - hi[a];
        s += e * e;
    }
    return sqrt(s);
}

/* 0 = open (holds a body of the group), 1 = open (too close), 2 = accept */
static int decide(const or_tree *t, walk_t *w, int64_t v)
{
    int64_t a0 = t->first[v], a1 = t->first[v] + t->count[v];
    if (a0 < w->gfirst + w->gcount && w->gfirst < a1)
        return 0;
    double s = cube_side(t, v);
    double d = dist_to_box(&t->com[3 * v], w->lo, w->hi);
    double td = w->theta * d;
    if (fabs(s - td) <= 1e-6 * td)
        w->flagged = 1;
    return (s < td) ? 2 : 1;
}

static void push_i64(int64_t **a, int64_t *n, int64_t *cap, int64_t x)
{
    if (*n == *cap) {
        *cap = *cap ? 2 * *cap : 256;
        *a = (int64_t *)realloc(*a, (size_t)*cap * sizeof(int64_t));
    }
    (*a)[(*n)++] = x;
}

/* v has been opened: a leaf gives its bodies to the list, an internal
 * cube has each child tested in turn (traversal continues recursively). */
static void open_cube(const or_tree *t, walk_t *w, int64_t v)
{
    if (t->nchild[v] == 0) {
        push_i64(&w->leaves, &w->nleaves, &w->cap_l, v);
        w->nbody += t->count[v];
        return;
    }
    for (int64_t c = t->child_first[v]; c < t->child_first[v] + t->nchild[v]; c++) {
        if (decide(t, w, c) == 2)
            push_i64(&w->cells, &w->ncells, &w->cap_c, c);
        else
            open_cube(t, w, c);
    }
}

static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* R6: softened monopole force of a point mass m at y on a body at x. */
static void add_force(const double *x, const double *y, double m, double eps2, double G,
                      double *a, double *phi, double *mag)
{
    double dx = y[0] - x[0], dy = y[1] - x[1], dz = y[2] - x[2];
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    double rinv = 1.0 / sqrt(r2);
    double f = G * m * rinv * rinv * rinv;
    a[0] += f * dx;
    a[1] += f * dy;
    a[2] += f * dz;
    *phi -= G * m * rinv;
    *mag += fabs(f) * sqrt(dx * dx + dy * dy + dz * dz);
}

/* Quadrupole term of a cell (mass centre y, second moments Q about it) on a
 * body at x, from the second-order Taylor expansion of the softened
 * potential -G m / sqrt(|x - y'|^2 + eps^2) about y'= y: with d = y - x and
 * rho^2 = |d|^2 + eps^2,
 *   phi_Q = -(G/2) (3 d.Qd / rho^5 - tr Q / rho^3)
 *   a_Q   = G (-3 Qd / rho^5 + (7.5 d.Qd / rho^7 - 1.5 tr Q / rho^5) d). */
static void add_quad(const double *x, const double *y, const double *q, double eps2, double G, double *a,
                     double *phi, double *mag)
{
    double d[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
    double Qd[3] = {q[0] * d[0] + q[1] * d[1] + q[2] * d[2], q[1] * d[0] + q[3] * d[1] + q[4] * d[2],
                    q[2] * d[0] + q[4] * d[1] + q[5] * d[2]};
    double dQd = d[0] * Qd[0] + d[1] * Qd[1] + d[2] * Qd[2];
    double tr = q[0] + q[3] + q[5];
    double rho2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
    double ri = 1.0 / sqrt(rho2);
    double ri2 = ri * ri, ri3 = ri2 * ri, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
    double c = 7.5 * dQd * ri7 - 1.5 * tr * ri5;
    for (int k = 0; k < 3; k++) {
        double term = G * (-3.0 * Qd[k] * ri5 + c * d[k]);
        a[k] += term;
        *mag += fabs(term);
    }
    *phi -= 0.5 * G * (3.0 * dQd * ri5 - tr * ri3);
}

int or_tree_test(const or_tree *t, int64_t group, int64_t node, double theta)
{
    walk_t w;
    memset(&w, 0, sizeof(w));
    w.gfirst = t->gfirst[group];
    w.gcount = t->gcount[group];
    for (int a = 0; a < 3; a++) {
        w.lo[a] = INFINITY;
        w.hi[a] = -INFINITY;
    }
    for (int64_t j = w.gfirst; j < w.gfirst + w.gcount; j++)
        for (int a = 0; a < 3; a++) {
            if (t->xs[3 * j + a] < w.lo[a])
                w.lo[a] = t->xs[3 * j + a];
            if (t->xs[3 * j + a] > w.hi[a])
                w.hi[a] = t->xs[3 * j + a];
        }
    w.theta = theta;
    return decide(t, &w, node);
}

int64_t or_tree_walk(const or_tree *t, double theta, double eps, double G, int64_t g_begin,
                     int64_t g_end, double *acc, double *pot, double *amag, int64_t *ncell,
                     int64_t *nbody, uint64_t *hash, int32_t *flag)
{
    return or_tree_walk_order(t, theta, eps, G, 0, g_begin, g_end, acc, pot, amag, ncell, nbody, hash, flag);
}

int64_t or_tree_walk_order(const or_tree *t, double theta, double eps, double G, int quadrupole,
                           int64_t g_begin, int64_t g_end, double *acc, double *pot, double *amag,
                           int64_t *ncell, int64_t *nbody, uint64_t *hash, int32_t *flag)
{
    int64_t inter = 0;
    double eps2 = eps * eps;
    walk_t w;
    memset(&w, 0, sizeof(w));
    for (int64_t g = g_begin; g < g_end; g++) {
        w.gfirst = t->gfirst[g];
        w.gcount = t->gcount[g];
        w.theta = theta;
        w.flagged = 0;
        w.ncells = w.nleaves = w.nbody = 0;
        for (int a = 0; a < 3; a++) {
            w.lo[a] = INFINITY;
            w.hi[a] = -INFINITY;
        }
        for (int64_t j = w.gfirst; j < w.gfirst + w.gcount; j++)
            for (int a = 0; a < 3; a++) {
                if (t->xs[3 * j + a] < w.lo[a])
                    w.lo[a] = t->xs[3 * j + a];
                if (t->xs[3 * j + a] > w.hi[a])
                    w.hi[a] = t->xs[3 * j + a];
            }
        /* the walk starts at the root, which holds every body and so is
         * always opened */
        open_cube(t, &w, 0);

        /* loop through the accumulated list for every body of the group */
        for (int64_t i = w.gfirst; i < w.gfirst + w.gcount; i++) {
            double a[3] = {0, 0, 0}, phi = 0.0, mag = 0.0;
            const double *xi = &t->xs[3 * i];
            for (int64_t k = 0; k < w.ncells; k++) {
                int64_t c = w.cells[k];
                add_force(xi, &t->com[3 * c], t->mass[c], eps2, G, a, &phi, &mag);
                if (quadrupole)
                    add_quad(xi, &t->com[3 * c], &t->quad[6 * c], eps2, G, a, &phi, &mag);
            }
            for (int64_t k = 0; k < w.nleaves; k++) {
                int64_t v = w.leaves[k];
                for (int64_t j = t->first[v]; j < t->first[v] + t->count[v]; j++) {
                    double dummy = 0.0;
                    add_force(xi, &t->xs[3 * j], t->ms[j], eps2, G, a, j == i ? &dummy : &phi, &mag);
                }
            }
            int64_t o = (int64_t)t->perm[i];
            if (acc) {
                acc[3 * o + 0] = a[0];
                acc[3 * o + 1] = a[1];
                acc[3 * o + 2] = a[2];
            }
            if (pot)
                pot[o] = phi;
            if (amag)
                amag[o] = mag;
        }
        inter += w.gcount * (w.ncells + w.nbody);
        if (ncell)
            ncell[g] = w.ncells;
        if (nbody)
            nbody[g] = w.nbody;
        if (flag)
            flag[g] = w.flagged;
        if (hash) {
            uint64_t hsum = 0;
            for (int64_t k = 0; k < w.ncells; k++)
                hsum += mix64(2 * (uint64_t)w.cells[k] + 1);
            for (int64_t k = 0; k < w.nleaves; k++)
                hsum += mix64(2 * (uint64_t)w.leaves[k] + 2);
            hash[g] = hsum;
        }
    }
    free(w.cells);
    free(w.leaves);
    return inter;
}

/* ------------------------------------------------------------------ */
/* Direct summation: the exact O(N^2) result the treecode approximates.*/
/* ------------------------------------------------------------------ */
void or_direct64(const double *pos, const double *mass, int64_t n, double eps, double G,
                 const int64_t *idx, int64_t ns, double *acc, double *pot)
{
    double eps2 = eps * eps;
    for (int64_t s = 0; s < ns; s++) {
        int64_t i = idx[s];
        double a[3] = {0, 0, 0}, phi = 0.0, mag = 0.0;
        for (int64_t j = 0; j < n; j++) {
            double dummy = 0.0;
            add_force(&pos[3 * i], &pos[3 * j], mass[j], eps2, G, a, j == i ? &dummy : &phi, &mag);
        }
        acc[3 * s + 0] = a[0];
        acc[3 * s + 1] = a[1];
        acc[3 * s + 2] = a[2];
        if (pot)
            pot[s] = phi;
    }
}

void or_direct(const float *pos, const float *mass, int64_t n, double eps, double G,
               const int64_t *idx, int64_t ns, double *acc, double *pot)
{
    double *p = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *m = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t j = 0; j < n; j++) {
        for (int a = 0; a < 3; a++)
            p[3 * j + a] = (double)pos[3 * j + a];
        m[j] = (double)mass[j];
    }
    or_direct64(p, m, n, eps, G, idx, ns, acc, pot);
    free(p);
    free(m);
}

/* ------------------------------------------------------------------ */
/* R7: kick-drift-kick leapfrog (Sec. 3.1: bodies update position and  */
/* velocity from the computed forces).                                  */
/* ------------------------------------------------------------------ */
void or_kick(double *vel, const double *acc, int64_t n, double h)
{
    for (int64_t i = 0; i < 3 * n; i++)
        vel[i] += acc[i] * h;
}

void or_drift(double *pos, const double *vel, int64_t n, double dt)
{
    for (int64_t i = 0; i < 3 * n; i++)
        pos[i] += vel[i] * dt;
}

void or_diag(const double *pos, const double *vel, const double *mass, const double *pot,
             int64_t n, double *out8)
{
    memset(out8, 0, 8 * sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        const double *x = &pos[3 * i], *v = &vel[3 * i];
        double m = mass[i];
        out8[0] += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (pot)
            out8[1] += 0.5 * m * pot[i];
        out8[2] += m * v[0];
        out8[3] += m * v[1];
        out8[4] += m * v[2];
        out8[5] += m * (x[1] * v[2] - x[2] * v[1]);
        out8[6] += m * (x[2] * v[0] - x[0] * v[2]);
        out8[7] += m * (x[0] * v[1] - x[1] * v[0]);
    }
}

/* ------------------------------------------------------------------ */
/* Learned far-field correction: features, labels and the MLP.        */
/* ------------------------------------------------------------------ */
void or_mlp_features(const or_tree *t, int64_t v, const double *x, double eps, double msys, double *f)
{
    double s = cube_side(t, v);
    double d[3], r2 = 0.0;
    for (int a = 0; a < 3; a++) {
        d[a] = t->com[3 * v + a] - x[a];
        r2 += d[a] * d[a];
    }
    double r = sqrt(r2);
    double M = t->mass[v];
    for (int a = 0; a < 3; a++)
        f[a] = d[a] / s;
    f[3] = s / r;
    f[4] = eps / s;
    f[5] = log2((double)t->count[v]);
    f[6] = M / msys;
    for (int k = 0; k < 6; k++)
        f[7 + k] = t->quad[6 * v + k] / (M * s * s);
}

/* G M s^2 / r^4: the acceleration unit of a label (the scaling of the
 * quadrupole term, so that labels depend on direction and shape only). */
double or_mlp_factor(const or_tree *t, int64_t v, const double *x, double G)
{
    double s = cube_side(t, v), r2 = 0.0;
    for (int a = 0; a < 3; a++) {
        double d = t->com[3 * v + a] - x[a];
        r2 += d * d;
    }
    return G * t->mass[v] * s * s / (r2 * r2);
}

void or_mlp_label(const or_tree *t, int64_t v, const double *x, double eps, double G, double *out)
{
    double eps2 = eps * eps, phi = 0.0, mag = 0.0;
    double ae[3] = {0, 0, 0}, am[3] = {0, 0, 0};
    for (int64_t j = t->first[v]; j < t->first[v] + t->count[v]; j++)
        add_force(x, &t->xs[3 * j], t->ms[j], eps2, G, ae, &phi, &mag);
    add_force(x, &t->com[3 * v], t->mass[v], eps2, G, am, &phi, &mag);
    double fac = or_mlp_factor(t, v, x, G);
    for (int a = 0; a < 3; a++)
        out[a] = (ae[a] - am[a]) / fac;
}

#define H 64
static void mlp_layers(const double *p, const double *x, double *h1, double *h2, double *y)
{
    const double *W1 = p, *b1 = W1 + 13 * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H * 3;
    for (int j = 0; j < H; j++) {
        double z = b1[j];
        for (int i = 0; i < 13; i++)
            z += x[i] * W1[i * H + j];
        h1[j] = z > 0.0 ? z : 0.0;
    }
    for (int j = 0; j < H; j++) {
        double z = b2[j];
        for (int i = 0; i < H; i++)
            z += h1[i] * W2[i * H + j];
        h2[j] = z > 0.0 ? z : 0.0;
    }
    for (int k = 0; k < 3; k++) {
        double z = b3[k];
        for (int i = 0; i < H; i++)
            z += h2[i] * W3[i * 3 + k];
        y[k] = z;
    }
}

void or_mlp_forward(const double *p, const double *X, int64_t n, double *Y)
{
    double h1[H], h2[H];
    for (int64_t i = 0; i < n; i++)
        mlp_layers(p, &X[13 * i], h1, h2, &Y[3 * i]);
}

double or_mlp_grad(const double *p, const double *X, const double *T, const double *w, int64_t n, double *g)
{
    const double *W2 = p + 13 * H + H, *W3 = W2 + H * H + H;
    double *gW1 = g, *gb1 = gW1 + 13 * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + H * 3;
    memset(g, 0, OR_MLP_NPARAM * sizeof(double));
    double loss = 0.0;
    double h1[H], h2[H], y[3], dy[3], dh2[H], dh1[H];
    for (int64_t i = 0; i < n; i++) {
        const double *x = &X[13 * i];
        mlp_layers(p, x, h1, h2, y);
        double wi = w ? w[i] : 1.0;
        for (int k = 0; k < 3; k++) {
            double e = y[k] - T[3 * i + k];
            loss += wi * e * e;
            dy[k] = 2.0 * wi * e / (double)n;
        }
        /* output layer */
        for (int k = 0; k < 3; k++) {
            gb3[k] += dy[k];
            for (int j = 0; j < H; j++)
                gW3[j * 3 + k] += h2[j] * dy[k];
        }
        for (int j = 0; j < H; j++) {
            double z = 0.0;
            for (int k = 0; k < 3; k++)
                z += W3[j * 3 + k] * dy[k];
            dh2[j] = h2[j] > 0.0 ? z : 0.0;
        }
        /* second hidden layer */
        for (int j = 0; j < H; j++) {
            gb2[j] += dh2[j];
            for (int i2 = 0; i2 < H; i2++)
                gW2[i2 * H + j] += h1[i2] * dh2[j];
        }
        for (int i2 = 0; i2 < H; i2++) {
            double z = 0.0;
            for (int j = 0; j < H; j++)
                z += W2[i2 * H + j] * dh2[j];
            dh1[i2] = h1[i2] > 0.0 ? z : 0.0;
        }
        /* first hidden layer */
        for (int j = 0; j < H; j++) {
            gb1[j] += dh1[j];
            for (int i1 = 0; i1 < 13; i1++)
                gW1[i1 * H + j] += x[i1] * dh1[j];
        }
    }
    return loss / (double)n;
}
#undef H

/* ------------------------------------------------------------------ */
/* BF16 rounding model of the network.                                  */
/* The network above is exact (FP64).  A tensor-core implementation    */
/* rounds some operands to bfloat16 (an 8-bit significand) and adds in */
/* FP32.  The model below rounds the same operands at the same points  */
/* -- the normalised inputs, the weights, the hidden activations after */
/* the ReLU and, in the backward pass, the operands of the products    */
/* that form the gradients -- and keeps every sum exact.  Beside each  */
/* value it carries a radius: how far an implementation that performs */
/* the same roundings on FP32 sums (each addition off by at most one   */
/* FP32 ulp of the largest partial magnitude) can land from the model  */
/* value.  Rounding to nearest is monotone, so a value known to lie in */
/* [v - r, v + r] before a rounding lies in [bf16(v - r), bf16(v + r)] */
/* after it; most hidden units are far from a rounding boundary and    */
/* keep radius 0 there.  The model is a reading of the precision the   */
/* learned correction runs at, not a copy of any kernel's structure.   */
/* ------------------------------------------------------------------ */
#define RM_U32 (1.0 / 8388608.0) /* 2^-23: one FP32 ulp at 1 */

/* nearest number with an 8-bit significand, ties to even (the bfloat16
 * value of x, for x in the normal range of float) */
double or_bf16(double x)
{
    if (x == 0.0 || !isfinite(x))
        return x;
    int e;
    double m = frexp(x, &e);         /* x = m 2^e, 0.5 <= |m| < 1 */
    double t = ldexp(m, 8);          /* 128 <= |t| < 256: 8 significant bits */
    double r = nearbyint(t);         /* round half to even (default mode) */
    return ldexp(r, e - 8);
}

/* model value of bf16(relu?(v)) and the largest distance to the values an
 * implementation reaches from [v - r, v + r] */
static double bf16_iv(double v, double r, int relu, double *rad)
{
    double lo = v - r, hi = v + r;
    if (relu) {
        v = v > 0.0 ? v : 0.0;
        lo = lo > 0.0 ? lo : 0.0;
        hi = hi > 0.0 ? hi : 0.0;
    }
    double m = or_bf16(v), a = or_bf16(lo), b = or_bf16(hi);
    *rad = (b - m > m - a) ? b - m : m - a;
    return m;
}

/* z_j = b_j + sum_i a_i bf16(W[i][j]) exactly, and the radius of an FP32
 * accumulation (kacc additions) of inputs known within da_i of a_i */
static void layer_iv(const double *W, const double *b, int nin, int nout, int kacc, const double *a,
                     const double *da, double *z, double *dz)
{
    for (int j = 0; j < nout; j++) {
        double s = b[j], mag = fabs(b[j]), prop = 0.0;
        for (int i = 0; i < nin; i++) {
            double w = or_bf16(W[i * nout + j]);
            s += a[i] * w;
            mag += (fabs(a[i]) + da[i]) * fabs(w);
            prop += da[i] * fabs(w);
        }
        z[j] = s;
        dz[j] = prop + (double)(kacc + 1) * RM_U32 * mag;
    }
}

#define RH 64
typedef struct {
    double x[13], dx[13];
    double z1[RH], dz1[RH], h1[RH], dh1[RH];
    double z2[RH], dz2[RH], h2[RH], dh2[RH];
    double y[3], dy[3];
} rm_fwd_t;

static void rm_forward(const double *p, const double *x, const double *xr, rm_fwd_t *f)
{
    const double *W1 = p, *b1 = W1 + 13 * RH, *W2 = b1 + RH, *b2 = W2 + RH * RH, *W3 = b2 + RH, *b3 = W3 + RH * 3;
    for (int i = 0; i < 13; i++)
        f->x[i] = bf16_iv(x[i], xr ? xr[i] : 0.0, 0, &f->dx[i]);
    layer_iv(W1, b1, 13, RH, 16, f->x, f->dx, f->z1, f->dz1);
    for (int j = 0; j < RH; j++)
        f->h1[j] = bf16_iv(f->z1[j], f->dz1[j], 1, &f->dh1[j]);
    layer_iv(W2, b2, RH, RH, RH, f->h1, f->dh1, f->z2, f->dz2);
    for (int j = 0; j < RH; j++)
        f->h2[j] = bf16_iv(f->z2[j], f->dz2[j], 1, &f->dh2[j]);
    layer_iv(W3, b3, RH, 3, RH, f->h2, f->dh2, f->y, f->dy);
}

void or_mlp_forward_bf16(const double *p, const double *X, const double *Xr, int64_t n, double *Y, double *R)
{
    rm_fwd_t f;
    for (int64_t i = 0; i < n; i++) {
        rm_forward(p, &X[13 * i], Xr ? &Xr[13 * i] : NULL, &f);
        for (int k = 0; k < 3; k++) {
            Y[3 * i + k] = f.y[k];
            if (R)
                R[3 * i + k] = f.dy[k];
        }
    }
}

/* a masked product z * [h > 0] where the implementation's z lies within r
 * and its pre-activation (model zh) within rh: value and radius (an
 * uncertain mask allows 0 as well) */
static double mask_iv(double z, double r, double zh, double rh, double *rad)
{
    if (zh - rh > 0.0) {
        *rad = r;
        return z;
    }
    if (zh + rh <= 0.0) {
        *rad = 0.0;
        return 0.0;
    }
    *rad = fabs(z) + r;
    return zh > 0.0 ? z : 0.0;
}

/* Loss and gradient of the rounding model (layout as or_mlp_grad).  Per
 * row: e = y - T, dY = 2 w e / n; the products dW3 = H2^T dY,
 * dH2 = dY W3^T, dW2 = H1^T dH2, dH1 = dH2 W2^T, dW1 = X^T dH1 take BF16
 * operands (dY, dH2, dH1 rounded before use); the bias gradients sum the
 * unrounded dY, dH2, dH1.  grad_rad (nullable) receives the radius of an
 * implementation that accumulates every sum -- over k and over the n rows
 * -- in FP32; *loss_rad (nullable) that of the loss. */
double or_mlp_grad_bf16(const double *p, const double *X, const double *Xr, const double *T, const double *w,
                        int64_t n, double *g, double *grad_rad, double *loss_rad)
{
    const double *W2 = p + 13 * RH + RH, *W3 = W2 + RH * RH + RH;
    double *gW1 = g, *gb1 = gW1 + 13 * RH, *gW2 = gb1 + RH, *gb2 = gW2 + RH * RH, *gW3 = gb2 + RH,
           *gb3 = gW3 + RH * 3;
    /* per element: sum of term radii and sum of |terms| (for the FP32
     * accumulation over rows) */
    double *er = (double *)calloc(OR_MLP_NPARAM, sizeof(double));
    double *em = (double *)calloc(OR_MLP_NPARAM, sizeof(double));
    memset(g, 0, OR_MLP_NPARAM * sizeof(double));
    double loss = 0.0, lr = 0.0, lmag = 0.0;
    rm_fwd_t f;
    double dyv[3], ddy[3], dyb[3], ddyb[3];
    double dh2[RH], rdh2[RH], dh2b[RH], rdh2b[RH], dh1[RH], rdh1[RH], dh1b[RH], rdh1b[RH];
    for (int64_t i = 0; i < n; i++) {
        rm_forward(p, &X[13 * i], Xr ? &Xr[13 * i] : NULL, &f);
        double wi = w ? w[i] : 1.0;
        for (int k = 0; k < 3; k++) {
            double e = f.y[k] - T[3 * i + k];
            double re = f.dy[k] + RM_U32 * (fabs(e) + f.dy[k]);
            loss += wi * e * e;
            lr += wi * (2.0 * fabs(e) * re + re * re);
            lmag += wi * (fabs(e) + re) * (fabs(e) + re);
            dyv[k] = 2.0 * wi * e / (double)n;
            /* 2 w e / n formed in FP32: a few roundings */
            ddy[k] = 2.0 * wi * re / (double)n + 4.0 * RM_U32 * fabs(dyv[k]);
            dyb[k] = bf16_iv(dyv[k], ddy[k], 0, &ddyb[k]);
        }
        /* output layer */
        for (int k = 0; k < 3; k++) {
            gb3[k] += dyv[k];
            er[13 * RH + RH + RH * RH + RH + RH * 3 + k] += ddy[k];
            em[13 * RH + RH + RH * RH + RH + RH * 3 + k] += fabs(dyv[k]) + ddy[k];
            for (int j = 0; j < RH; j++) {
                int o = 13 * RH + RH + RH * RH + RH + j * 3 + k;
                gW3[j * 3 + k] += f.h2[j] * dyb[k];
                er[o] += fabs(f.h2[j]) * ddyb[k] + fabs(dyb[k]) * f.dh2[j] + f.dh2[j] * ddyb[k];
                em[o] += (fabs(f.h2[j]) + f.dh2[j]) * (fabs(dyb[k]) + ddyb[k]);
            }
        }
        for (int j = 0; j < RH; j++) {
            double z = 0.0, mag = 0.0, pr = 0.0;
            for (int k = 0; k < 3; k++) {
                double w3 = or_bf16(W3[j * 3 + k]);
                z += w3 * dyb[k];
                mag += fabs(w3) * (fabs(dyb[k]) + ddyb[k]);
                pr += fabs(w3) * ddyb[k];
            }
            dh2[j] = mask_iv(z, pr + 17.0 * RM_U32 * mag, f.z2[j], f.dz2[j], &rdh2[j]);
            dh2b[j] = bf16_iv(dh2[j], rdh2[j], 0, &rdh2b[j]);
        }
        /* second hidden layer */
        for (int j = 0; j < RH; j++) {
            int ob = 13 * RH + RH + RH * RH + j;
            gb2[j] += dh2[j];
            er[ob] += rdh2[j];
            em[ob] += fabs(dh2[j]) + rdh2[j];
            for (int i2 = 0; i2 < RH; i2++) {
                int o = 13 * RH + RH + i2 * RH + j;
                gW2[i2 * RH + j] += f.h1[i2] * dh2b[j];
                er[o] += fabs(f.h1[i2]) * rdh2b[j] + fabs(dh2b[j]) * f.dh1[i2] + f.dh1[i2] * rdh2b[j];
                em[o] += (fabs(f.h1[i2]) + f.dh1[i2]) * (fabs(dh2b[j]) + rdh2b[j]);
            }
        }
        for (int i2 = 0; i2 < RH; i2++) {
            double z = 0.0, mag = 0.0, pr = 0.0;
            for (int j = 0; j < RH; j++) {
                double w2 = or_bf16(W2[i2 * RH + j]);
                z += w2 * dh2b[j];
                mag += fabs(w2) * (fabs(dh2b[j]) + rdh2b[j]);
                pr += fabs(w2) * rdh2b[j];
            }
            dh1[i2] = mask_iv(z, pr + (RH + 1) * RM_U32 * mag, f.z1[i2], f.dz1[i2], &rdh1[i2]);
            dh1b[i2] = bf16_iv(dh1[i2], rdh1[i2], 0, &rdh1b[i2]);
        }
        /* first hidden layer */
        for (int j = 0; j < RH; j++) {
            int ob = 13 * RH + j;
            gb1[j] += dh1[j];
            er[ob] += rdh1[j];
            em[ob] += fabs(dh1[j]) + rdh1[j];
            for (int i1 = 0; i1 < 13; i1++) {
                int o = i1 * RH + j;
                gW1[o] += f.x[i1] * dh1b[j];
                er[o] += fabs(f.x[i1]) * rdh1b[j] + fabs(dh1b[j]) * f.dx[i1] + f.dx[i1] * rdh1b[j];
                em[o] += (fabs(f.x[i1]) + f.dx[i1]) * (fabs(dh1b[j]) + rdh1b[j]);
            }
        }
    }
    if (grad_rad)
        for (int k = 0; k < OR_MLP_NPARAM; k++)
            grad_rad[k] = er[k] + (double)(n + 17) * RM_U32 * em[k];
    if (loss_rad)
        *loss_rad = (lr + (double)(n + 17) * RM_U32 * lmag) / (double)n;
    free(er);
    free(em);
    return loss / (double)n;
}
#undef RH

/* Radius of a feature an FP32 implementation computes at the same point
 * (an error analysis of FP32 evaluation of the definitions in
 * or_mlp_features, with a margin of 4): offsets d/s carry the rounding of
 * the cell's centre of mass and of the group's centre relative to its
 * reference cube (side sref); s/r those of r and of one reciprocal square
 * root (2 ulps); log2(count) a fast logarithm (2^-21 absolute); the moment
 * ratios two roundings of the inputs and one approximate division, plus the
 * error of second moments accumulated in FP32 (a few roundings per body of
 * a leaf of at most leaf_max bodies and per child above it, each at most
 * half an FP32 ulp of a term no larger than M s^2). */
static void feature_radius(const double *f, double s, double sref, double r, int leaf_max, double *fr)
{
    const double u = RM_U32, off = 4.0 * (2.0 * u * (fabs(f[0]) + fabs(f[1]) + fabs(f[2])) + u + 4.0 * u * sref / s);
    for (int a = 0; a < 3; a++)
        fr[a] = off;
    fr[3] = 4.0 * f[3] * (2.0 * u + off * s / r);
    fr[4] = 4.0 * u * f[4];
    fr[5] = 4.0 * (4.0 * u * (1.0 + f[5]));
    fr[6] = 4.0 * (4.0 * u * f[6]);
    /* the moment ratios also carry the FP32 second moments' error:
     * (leaf_max + 122) 2^-26 in units of M s^2 (taken as leaf_max + 128),
     * twice */
    for (int k = 7; k < 13; k++)
        fr[k] = 4.0 * (4.0 * u * fabs(f[k])) + (double)(leaf_max + 128) * u / 4.0;
}

/* Learned correction of the group walk.  For each group: the accepted cells
 * v of its walk holding two or more bodies with s >= band * d (d = distance
 * from v's centre of mass to the group's box) are evaluated at the centre
 * x_g of the group's box, and F y is added to every body of the group, with
 * F = G M_v s^2 / r^4 (r = |com_v - x_g|, s the cell side: the scale of the
 * quadrupole term).  y = network((f - mean) * scale) * yscale with maps =
 * 13 means, 13 scales, 3 output scales; with params NULL, y is the exact
 * label at x_g instead (what a perfect model would give); with rm the
 * network is its BF16 rounding model and crad gets the radius of an FP32
 * implementation. */
static int64_t learned_walk(const or_tree *t, double theta, double eps, double G, double band,
                            const double *params, const double *maps, int64_t g_begin, int64_t g_end, int rm,
                            double *corr, double *crad, int32_t *flag)
{
    int64_t evals = 0;
    walk_t w;
    memset(&w, 0, sizeof(w));
    double msys = t->mass[0];
    for (int64_t g = g_begin; g < g_end; g++) {
        w.gfirst = t->gfirst[g];
        w.gcount = t->gcount[g];
        w.theta = theta;
        w.flagged = 0;
        w.ncells = w.nleaves = w.nbody = 0;
        for (int a = 0; a < 3; a++) {
            w.lo[a] = INFINITY;
            w.hi[a] = -INFINITY;
        }
        for (int64_t j = w.gfirst; j < w.gfirst + w.gcount; j++)
            for (int a = 0; a < 3; a++) {
                if (t->xs[3 * j + a] < w.lo[a])
                    w.lo[a] = t->xs[3 * j + a];
                if (t->xs[3 * j + a] > w.hi[a])
                    w.hi[a] = t->xs[3 * j + a];
            }
        open_cube(t, &w, 0);
        double xg[3], cg[3] = {0, 0, 0}, cr[3] = {0, 0, 0}, cm[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++)
            xg[a] = 0.5 * (w.lo[a] + w.hi[a]);
        double sref = cube_side(t, t->gref[g]);
        int64_t nev = 0;
        for (int64_t k = 0; k < w.ncells; k++) {
            int64_t v = w.cells[k];
            if (t->count[v] < 2)
                continue;
            double s = cube_side(t, v);
            double bd = band * dist_to_box(&t->com[3 * v], w.lo, w.hi);
            if (fabs(s - bd) <= 1e-6 * bd)
                w.flagged = 1;
            if (s < bd)
                continue;
            double y[3], yr[3] = {0, 0, 0};
            if (params) {
                double f[13], h1[64], h2[64];
                or_mlp_features(t, v, xg, eps, msys, f);
                if (rm) {
                    /* normalised inputs and their radius: the feature's own,
                     * scaled, plus the two FP32 roundings of (f - mean) scale */
                    double fr[13], xr[13];
                    double r2 = 0.0;
                    for (int a = 0; a < 3; a++)
                        r2 += (t->com[3 * v + a] - xg[a]) * (t->com[3 * v + a] - xg[a]);
                    feature_radius(f, s, sref, sqrt(r2), t->leaf_max, fr);
                    for (int i = 0; i < 13; i++) {
                        double xn = (f[i] - maps[i]) * maps[13 + i];
                        xr[i] = fabs(maps[13 + i]) * fr[i] + 2.0 * RM_U32 * (fabs(maps[i] * maps[13 + i]) + fabs(xn));
                        f[i] = xn;
                    }
                    rm_fwd_t fw;
                    rm_forward(params, f, xr, &fw);
                    for (int a = 0; a < 3; a++) {
                        y[a] = fw.y[a] * maps[26 + a];
                        yr[a] = fabs(maps[26 + a]) * fw.dy[a] + RM_U32 * fabs(y[a]);
                    }
                } else {
                    for (int i = 0; i < 13; i++)
                        f[i] = (f[i] - maps[i]) * maps[13 + i];
                    mlp_layers(params, f, h1, h2, y);
                    for (int a = 0; a < 3; a++)
                        y[a] *= maps[26 + a];
                }
            } else {
                or_mlp_label(t, v, xg, eps, G, y);
            }
            double fac = or_mlp_factor(t, v, xg, G);
            for (int a = 0; a < 3; a++) {
                cg[a] += fac * y[a];
                if (rm) {
                    /* the factor G M s^2 / r^4 in FP32: a few roundings and
                     * the reciprocal square root, plus r's own radius */
                    double r2 = 0.0;
                    for (int b = 0; b < 3; b++)
                        r2 += (t->com[3 * v + b] - xg[b]) * (t->com[3 * v + b] - xg[b]);
                    double dr = 4.0 * (2.0 * RM_U32 * sqrt(r2) + 4.0 * RM_U32 * (s + sref));
                    double frel = 16.0 * RM_U32 + 4.0 * dr / sqrt(r2);
                    cr[a] += fabs(fac) * yr[a] + frel * fabs(fac * y[a]);
                    cm[a] += fabs(fac) * (fabs(y[a]) + yr[a]);
                }
            }
            evals++;
            nev++;
        }
        for (int64_t i = w.gfirst; i < w.gfirst + w.gcount; i++) {
            int64_t o = (int64_t)t->perm[i];
            for (int a = 0; a < 3; a++) {
                corr[3 * o + a] = cg[a];
                /* FP32 sums over the group's cells: one ulp per addition */
                if (crad)
                    crad[3 * o + a] = cr[a] + (double)(nev + 6) * RM_U32 * cm[a];
            }
        }
        if (flag)
            flag[g] = w.flagged;
    }
    free(w.cells);
    free(w.leaves);
    return evals;
}

int64_t or_tree_learned(const or_tree *t, double theta, double eps, double G, double band,
                        const double *params, const double *maps, int64_t g_begin, int64_t g_end,
                        double *corr, int32_t *flag)
{
    return learned_walk(t, theta, eps, G, band, params, maps, g_begin, g_end, 0, corr, NULL, flag);
}

int64_t or_tree_learned_bf16(const or_tree *t, double theta, double eps, double G, double band,
                             const double *params, const double *maps, int64_t g_begin, int64_t g_end,
                             double *corr, double *crad, int32_t *flag)
{
    if (!params)
        return -1;
    return learned_walk(t, theta, eps, G, band, params, maps, g_begin, g_end, 1, corr, crad, flag);
}

/* The interaction list of one group at theta: accepted cells and opened
 * leaves in the walk's order (depth first, children in octant order).
 * Writes at most cap_c / cap_l entries; *nc / *nl get the full lengths. */
void or_tree_group_list(const or_tree *t, double theta, int64_t g, int64_t *cells, int64_t cap_c,
                        int64_t *leaves, int64_t cap_l, int64_t *nc, int64_t *nl)
{
    walk_t w;
    memset(&w, 0, sizeof(w));
    w.gfirst = t->gfirst[g];
    w.gcount = t->gcount[g];
    w.theta = theta;
    for (int a = 0; a < 3; a++) {
        w.lo[a] = INFINITY;
        w.hi[a] = -INFINITY;
    }
    for (int64_t j = w.gfirst; j < w.gfirst + w.gcount; j++)
        for (int a = 0; a < 3; a++) {
            if (t->xs[3 * j + a] < w.lo[a])
                w.lo[a] = t->xs[3 * j + a];
            if (t->xs[3 * j + a] > w.hi[a])
                w.hi[a] = t->xs[3 * j + a];
        }
    open_cube(t, &w, 0);
    for (int64_t k = 0; k < w.ncells && k < cap_c; k++)
        cells[k] = w.cells[k];
    for (int64_t k = 0; k < w.nleaves && k < cap_l; k++)
        leaves[k] = w.leaves[k];
    *nc = w.ncells;
    *nl = w.nleaves;
    free(w.cells);
    free(w.leaves);
}

/* ------------------------------------------------------------------ */
/* Fast multipole method (Sec. 5 names it as the treecode's O(N)       */
/* successor; the paper gives no formulation, so this is a reading,    */
/* stated in full).  Same tree as the treecode.                        */
/*   Expansion centres: every cell's centre of mass c_X.               */
/*   Multipoles: the monopole, mass M_X at c_X.                        */
/*   Radii: r_X bounds the distance of X's bodies from c_X: a leaf's    */
/*     farthest body; above, the farthest child sphere,                 */
/*     max over children (|c_child - c_X| + r_child).                   */
/*   Local expansions, third order about c_B: the field at x near B is  */
/*     a(x) = L0 + L1 dx + (1/2) L2 dx dx + (1/6) L3 dx dx dx,           */
/*     dx = x - c_B; L0 a vector, L1 the field's Jacobian (symmetric),   */
/*     L2 and L3 its second and third derivatives (symmetric tensors).   */
/*   Acceptance of a pair of disjoint cells: r_A + r_B < theta |c_A - c_B|*/
/*     (the spheres about the centres, shrunk by theta, are disjoint);  */
/*     a pair within 1e-6 relative of the bound is counted (ties).      */
/*   Dual traversal from (root, root):                                  */
/*     (X, X): a leaf -> P2P within it; otherwise every (child, child).  */
/*     (A, B), A != B: accepted -> M2L(A -> B); both leaves -> P2P(A ->  */
/*     B); otherwise split B if it is internal and (A is a leaf or      */
/*     r_B >= r_A), else split A.  Per target cell this is a walk: a    */
/*     target B refines each candidate source wider than itself until   */
/*     it is accepted, a leaf or no wider, and hands the unresolved     */
/*     ones, with its own children, to its children as their candidates.*/
/*   M2L(A -> B): d = c_A - c_B, rho^2 = |d|^2 + eps^2, the softened     */
/*     field G M_A d / rho^3 and its derivatives at c_B:                 */
/*     L0_i += G M d_i / rho^3                                           */
/*     L1_ij += G M (3 d_i d_j / rho^5 - delta_ij / rho^3)               */
/*     L2_ijk += G M (15 d_i d_j d_k / rho^7                             */
/*               - 3 (delta_ij d_k + delta_ik d_j + delta_jk d_i) / rho^5)*/
/*     L3_ijkl += G M (105 d_i d_j d_k d_l / rho^9                       */
/*               - 15 (the 6 terms delta_ab d_c d_e) / rho^7             */
/*               + 3 (the 3 terms delta_ab delta_ce) / rho^5)            */
/*   L2L, parents before children, t = c_c - c_p: each coefficient       */
/*     gains its parent's Taylor series moved by t:                      */
/*     L0_c += L0_p + L1_p t + (1/2) L2_p t t + (1/6) L3_p t t t,        */
/*     L1_c += L1_p + L2_p t + (1/2) L3_p t t, L2_c += L2_p + L3_p t,    */
/*     L3_c += L3_p.                                                     */
/*   L2P: a_i += L0 + L1 dx + (1/2) L2 dx dx + (1/6) L3 dx dx dx over a   */
/*     leaf's bodies.                                                    */
/*   P2P(A -> B): a_i += G m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^1.5,*/
/*     i in B, j in A, j != i.                                           */
/* Every ordered pair of bodies is reached through exactly one M2L or    */
/* P2P: the traversal splits pairs down to disjoint cells or leaves.     */
/* ------------------------------------------------------------------ */
typedef struct {
    const or_tree *t;
    double theta, eps2, G;
    double *L0, *L1, *L2, *L3; /* M x 3, M x 9, M x 27, M x 81 (full index ranges) */
    double *rad;     /* M: radius about the centre of mass */
    double *acc;     /* sorted order, n x 3 */
    int64_t n_m2l, n_p2p, ties;
    uint64_t h_m2l, h_p2p; /* order-independent hashes of the pair sets */
    /* per target cell (nullable) */
    int64_t *nm2l, *np2p;
    uint64_t *hm2l, *hp2p;
    int32_t *flag;
} fmm_t;

static uint64_t fmm_mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void fmm_p2p(fmm_t *f, int64_t A, int64_t B)
{
    const or_tree *t = f->t;
    const uint64_t h = fmm_mix(((uint64_t)A << 32) ^ (uint64_t)B);
    f->n_p2p++;
    f->h_p2p += h;
    if (f->np2p) {
        f->np2p[B]++;
        f->hp2p[B] += h;
    }
    double phi = 0.0, mag = 0.0;
    for (int64_t i = t->first[B]; i < t->first[B] + t->count[B]; i++)
        for (int64_t j = t->first[A]; j < t->first[A] + t->count[A]; j++) {
            if (j == i)
                continue;
            add_force(&t->xs[3 * i], &t->xs[3 * j], t->ms[j], f->eps2, f->G, &f->acc[3 * i], &phi, &mag);
        }
}

static void fmm_m2l(fmm_t *f, int64_t A, int64_t B)
{
    const or_tree *t = f->t;
    const uint64_t h = fmm_mix(((uint64_t)A << 32) ^ (uint64_t)B);
    f->n_m2l++;
    f->h_m2l += h;
    if (f->nm2l) {
        f->nm2l[B]++;
        f->hm2l[B] += h;
    }
    double d[3];
    for (int a = 0; a < 3; a++)
        d[a] = t->com[3 * A + a] - t->com[3 * B + a];
    double rho2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + f->eps2;
    double ri = 1.0 / sqrt(rho2);
    double ri3 = ri * ri * ri, ri5 = ri3 * ri * ri;
    double gm = f->G * t->mass[A];
    double ri7 = ri5 * ri * ri;
    double ri9 = ri7 * ri * ri;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int c = 0; c < 3; c++)
                for (int e = 0; e < 3; e++) {
                    const double dd = (a == b ? d[c] * d[e] : 0.0) + (a == c ? d[b] * d[e] : 0.0) +
                                      (a == e ? d[b] * d[c] : 0.0) + (b == c ? d[a] * d[e] : 0.0) +
                                      (b == e ? d[a] * d[c] : 0.0) + (c == e ? d[a] * d[b] : 0.0);
                    const double d2 = (a == b && c == e ? 1.0 : 0.0) + (a == c && b == e ? 1.0 : 0.0) +
                                      (a == e && b == c ? 1.0 : 0.0);
                    f->L3[81 * B + 27 * a + 9 * b + 3 * c + e] +=
                        gm * (105.0 * d[a] * d[b] * d[c] * d[e] * ri9 - 15.0 * dd * ri7 + 3.0 * d2 * ri5);
                }
    for (int a = 0; a < 3; a++) {
        f->L0[3 * B + a] += gm * d[a] * ri3;
        for (int b = 0; b < 3; b++) {
            f->L1[9 * B + 3 * a + b] += gm * (3.0 * d[a] * d[b] * ri5 - (a == b ? ri3 : 0.0));
            for (int c = 0; c < 3; c++)
                f->L2[27 * B + 9 * a + 3 * b + c] +=
                    gm * (15.0 * d[a] * d[b] * d[c] * ri7 -
                          3.0 * ((a == b ? d[c] : 0.0) + (a == c ? d[b] : 0.0) + (b == c ? d[a] : 0.0)) * ri5);
        }
    }
}

static void fmm_pair(fmm_t *f, int64_t A, int64_t B)
{
    const or_tree *t = f->t;
    const int leafA = t->nchild[A] == 0, leafB = t->nchild[B] == 0;
    if (A == B) {
        if (leafA) {
            fmm_p2p(f, A, A);
            return;
        }
        for (int64_t ca = t->child_first[A]; ca < t->child_first[A] + t->nchild[A]; ca++)
            for (int64_t cb = t->child_first[A]; cb < t->child_first[A] + t->nchild[A]; cb++)
                fmm_pair(f, ca, cb);
        return;
    }
    const double rA = f->rad[A], rB = f->rad[B];
    double d2 = 0.0;
    for (int a = 0; a < 3; a++) {
        double e = t->com[3 * A + a] - t->com[3 * B + a];
        d2 += e * e;
    }
    const double lhs = rA + rB, rhs = f->theta * sqrt(d2);
    /* rhs = 0 (theta = 0, or coincident centres) rejects exactly */
    if (rhs > 0.0 && fabs(lhs - rhs) <= 1e-6 * rhs) {
        f->ties++;
        if (f->flag)
            f->flag[B] = 1;
    }
    if (lhs < rhs) {
        fmm_m2l(f, A, B);
        return;
    }
    if (leafA && leafB) {
        fmm_p2p(f, A, B);
        return;
    }
    if (!leafB && (leafA || rB >= rA)) {
        for (int64_t cb = t->child_first[B]; cb < t->child_first[B] + t->nchild[B]; cb++)
            fmm_pair(f, A, cb);
    } else {
        for (int64_t ca = t->child_first[A]; ca < t->child_first[A] + t->nchild[A]; ca++)
            fmm_pair(f, ca, B);
    }
}

/* r_X of every cell: children come after their parent in breadth-first
 * order, so one backward sweep sees every child before its parent. */
void or_fmm_radii(const or_tree *t, double *rad)
{
    for (int64_t v = t->M - 1; v >= 0; v--) {
        const double *c = &t->com[3 * v];
        double r = 0.0;
        if (t->nchild[v] == 0) {
            for (int64_t i = t->first[v]; i < t->first[v] + t->count[v]; i++) {
                const double *x = &t->xs[3 * i];
                double e = sqrt((x[0] - c[0]) * (x[0] - c[0]) + (x[1] - c[1]) * (x[1] - c[1]) +
                                (x[2] - c[2]) * (x[2] - c[2]));
                if (e > r)
                    r = e;
            }
        } else {
            for (int64_t k = t->child_first[v]; k < t->child_first[v] + t->nchild[v]; k++) {
                const double *q = &t->com[3 * k];
                double e = sqrt((q[0] - c[0]) * (q[0] - c[0]) + (q[1] - c[1]) * (q[1] - c[1]) +
                                (q[2] - c[2]) * (q[2] - c[2])) + rad[k];
                if (e > r)
                    r = e;
            }
        }
        rad[v] = r;
    }
}

/* Accelerations (n x 3, ORIGINAL order) of the FMM at opening parameter
 * theta; stats[0..4] (nullable) = M2L pairs, P2P pairs, ties, and the two
 * pair-set hashes (as int64 bit patterns). */
void or_fmm(const or_tree *t, double theta, double eps, double G, double *acc_out, int64_t *stats)
{
    or_fmm_nodes(t, theta, eps, G, acc_out, stats, NULL, NULL, NULL, NULL, NULL);
}

void or_fmm_nodes(const or_tree *t, double theta, double eps, double G, double *acc_out, int64_t *stats,
                  int64_t *nm2l, int64_t *np2p, uint64_t *hm2l, uint64_t *hp2p, int32_t *flag)
{
    fmm_t f;
    memset(&f, 0, sizeof(f));
    int64_t *own_n = NULL;
    uint64_t *own_h = NULL;
    int32_t *own_f = NULL;
    if (nm2l || np2p || hm2l || hp2p || flag) {
        /* the records are kept together; absent ones go to scratch */
        own_n = (int64_t *)calloc((size_t)t->M * 2, sizeof(int64_t));
        own_h = (uint64_t *)calloc((size_t)t->M * 2, sizeof(uint64_t));
        own_f = (int32_t *)calloc((size_t)t->M, sizeof(int32_t));
        f.nm2l = nm2l ? nm2l : own_n;
        f.np2p = np2p ? np2p : own_n + t->M;
        f.hm2l = hm2l ? hm2l : own_h;
        f.hp2p = hp2p ? hp2p : own_h + t->M;
        f.flag = flag ? flag : own_f;
        memset(f.nm2l, 0, (size_t)t->M * sizeof(int64_t));
        memset(f.np2p, 0, (size_t)t->M * sizeof(int64_t));
        memset(f.hm2l, 0, (size_t)t->M * sizeof(uint64_t));
        memset(f.hp2p, 0, (size_t)t->M * sizeof(uint64_t));
        memset(f.flag, 0, (size_t)t->M * sizeof(int32_t));
    }
    f.t = t;
    f.theta = theta;
    f.eps2 = eps * eps;
    f.G = G;
    f.L0 = (double *)calloc((size_t)t->M * 3, sizeof(double));
    f.L1 = (double *)calloc((size_t)t->M * 9, sizeof(double));
    f.L2 = (double *)calloc((size_t)t->M * 27, sizeof(double));
    f.L3 = (double *)calloc((size_t)t->M * 81, sizeof(double));
    f.acc = (double *)calloc((size_t)t->n * 3, sizeof(double));
    f.rad = (double *)calloc((size_t)t->M, sizeof(double));
    or_fmm_radii(t, f.rad);
    fmm_pair(&f, 0, 0);
    /* L2L: breadth-first order puts every parent before its children */
    for (int64_t v = 1; v < t->M; v++) {
        int64_t p = t->parent[v];
        double dc[3];
        for (int a = 0; a < 3; a++)
            dc[a] = t->com[3 * v + a] - t->com[3 * p + a];
        for (int a = 0; a < 3; a++) {
            double s = f.L0[3 * p + a];
            for (int b = 0; b < 3; b++) {
                s += f.L1[9 * p + 3 * a + b] * dc[b];
                for (int c = 0; c < 3; c++) {
                    s += 0.5 * f.L2[27 * p + 9 * a + 3 * b + c] * dc[b] * dc[c];
                    for (int e = 0; e < 3; e++)
                        s += f.L3[81 * p + 27 * a + 9 * b + 3 * c + e] * dc[b] * dc[c] * dc[e] / 6.0;
                }
            }
            f.L0[3 * v + a] += s;
            for (int b = 0; b < 3; b++) {
                double u = f.L1[9 * p + 3 * a + b];
                for (int c = 0; c < 3; c++) {
                    u += f.L2[27 * p + 9 * a + 3 * b + c] * dc[c];
                    for (int e = 0; e < 3; e++)
                        u += 0.5 * f.L3[81 * p + 27 * a + 9 * b + 3 * c + e] * dc[c] * dc[e];
                }
                f.L1[9 * v + 3 * a + b] += u;
                for (int c = 0; c < 3; c++) {
                    double w = f.L2[27 * p + 9 * a + 3 * b + c];
                    for (int e = 0; e < 3; e++)
                        w += f.L3[81 * p + 27 * a + 9 * b + 3 * c + e] * dc[e];
                    f.L2[27 * v + 9 * a + 3 * b + c] += w;
                    for (int e = 0; e < 3; e++)
                        f.L3[81 * v + 27 * a + 9 * b + 3 * c + e] += f.L3[81 * p + 27 * a + 9 * b + 3 * c + e];
                }
            }
        }
    }
    /* L2P */
    for (int64_t v = 0; v < t->M; v++) {
        if (t->nchild[v] != 0)
            continue;
        for (int64_t i = t->first[v]; i < t->first[v] + t->count[v]; i++) {
            double dx[3];
            for (int a = 0; a < 3; a++)
                dx[a] = t->xs[3 * i + a] - t->com[3 * v + a];
            for (int a = 0; a < 3; a++) {
                double s = f.L0[3 * v + a];
                for (int b = 0; b < 3; b++) {
                    s += f.L1[9 * v + 3 * a + b] * dx[b];
                    for (int c = 0; c < 3; c++) {
                        s += 0.5 * f.L2[27 * v + 9 * a + 3 * b + c] * dx[b] * dx[c];
                        for (int e = 0; e < 3; e++)
                            s += f.L3[81 * v + 27 * a + 9 * b + 3 * c + e] * dx[b] * dx[c] * dx[e] / 6.0;
                    }
                }
                f.acc[3 * i + a] += s;
            }
        }
    }
    for (int64_t i = 0; i < t->n; i++)
        for (int a = 0; a < 3; a++)
            acc_out[3 * (int64_t)t->perm[i] + a] = f.acc[3 * i + a];
    if (stats) {
        stats[0] = f.n_m2l;
        stats[1] = f.n_p2p;
        stats[2] = f.ties;
        stats[3] = (int64_t)f.h_m2l;
        stats[4] = (int64_t)f.h_p2p;
    }
    /* a flagged cell hands its (possibly flipped) pairs to its subtree */
    if (f.flag)
        for (int64_t v = 1; v < t->M; v++)
            if (f.flag[t->parent[v]])
                f.flag[v] = 1;
    free(own_n);
    free(own_h);
    free(own_f);
    free(f.rad);
    free(f.L0);
    free(f.L1);
    free(f.L2);
    free(f.L3);
    free(f.acc);
}
