/*
 * rs_oracle.c -- float64 CPU oracle for the ROCKSTAR hot path.
 *
 * TEST INFRASTRUCTURE, NOT THE PRODUCT.  Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg load this library.  It shares no code,
 * header, table or helper with the CUDA library, and neither side includes
 * the other.
 *
 * Every routine below is a plain, slow statement of a definition from
 * Behroozi, Wechsler & Wu, "The ROCKSTAR phase-space temporal halo finder"
 * (arXiv:1110.4372), computed in float64 on float32 inputs promoted exactly:
 *
 *   or_fof3d         3D friends-of-friends, periodic minimum image (Sec. 3.1)
 *   or_grid_*        the same graph queried one component at a time (Sec. 3.1)
 *   or_fof3d_accel   the paper's accelerated variant: dense particles join
 *                    everything within 2l and their neighbours skip their
 *                    own search (Sec. 3.1)
 *   or_refine        per-group phase-space hierarchy (Sec. 3.2, Eq. 1)
 *   or_refine_sampled  the same, with the linking length of a node above a
 *                    size limit taken from the nearest-neighbour distances
 *                    of a random subset of its members (Sec. 3.2)
 *   or_sample_key    the counter-based generator that draws those subsets
 *   or_assign        seeds, seed merge (Eq. 2), r_dyn,vir (Eq. 4) and the
 *                    hierarchical particle assignment with Eq. 3 (Sec. 3.3)
 *   or_halo_props    halo centres (Poisson-minimising node, Sec. 3.5.1) and
 *                    the host/subhalo relation (Sec. 3.4)
 *   or_unbind        single-pass unbinding with the exact potential
 *                    (Sec. 3.4, App. B)
 *
 * Readings taken where the paper is silent are written beside the code.
 * Compile with -ffp-contract=off so that no multiply-add is fused and the
 * arithmetic is the same on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 3
#define OR_ERR_EXTENT 7

/* Relative half-width of the tie band around a linking length: a pair whose
 * float64 distance d satisfies |d - l| <= 1e-6 l is a tie-band pair. */
#define TIE_REL 1e-6

int64_t or_version(void) { return 3; }

/* ------------------------------------------------------------------------ */
/* periodic minimum image of a float64 difference, into [-box/2, box/2]      */
/* ------------------------------------------------------------------------ */
static double min_image(double d, double box)
{
    if (d > 0.5 * box) d -= box;
    else if (d < -0.5 * box) d += box;
    return d;
}

static double dist2_3d(const float *pos, int64_t i, int64_t j, double box)
{
    double s = 0.0;
    for (int a = 0; a < 3; a++) {
        double d = min_image((double)pos[3 * i + a] - (double)pos[3 * j + a], box);
        s += d * d;
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* union-find on int32 indices; the root of every set is its smallest index  */
/* ------------------------------------------------------------------------ */
static int32_t uf_find(int32_t *p, int32_t x)
{
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

static void uf_union(int32_t *p, int32_t a, int32_t b)
{
    int32_t ra = uf_find(p, a), rb = uf_find(p, b);
    if (ra == rb) return;
    if (ra < rb) p[rb] = ra;
    else p[ra] = rb;
}

/* ======================================================================== */
/* 3D friends-of-friends (Sec. 3.1)                                          */
/* Two particles are friends when their periodic distance is <= l; groups    */
/* are the connected components.  The neighbour search uses a grid of cells  */
/* no smaller than l, so every friend of a particle lies in the 27 cells     */
/* around its own.                                                           */
/* ======================================================================== */
typedef struct {
    int64_t key;
    int64_t idx;
} kv_t;

struct or_grid {
    const float *pos;
    int64_t n;
    double box, l;
    int64_t G;      /* cells per side; 1 means "one cell, test all pairs" */
    kv_t *cells;    /* (cell key, particle) sorted by key then particle */
    uint32_t *stamp;
    uint32_t cur;
};
typedef struct or_grid or_grid;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static int64_t cell_coord(double x, double box, int64_t G)
{
    int64_t c = (int64_t)floor(x / box * (double)G);
    if (c < 0) c = 0;
    if (c >= G) c = G - 1;
    return c;
}

or_grid *or_grid_build(const float *pos, int64_t n, double box, double l)
{
    if (n < 0 || !(box > 0) || !(l >= 0)) return NULL;
    or_grid *g = (or_grid *)calloc(1, sizeof(or_grid));
    if (!g) return NULL;
    g->pos = pos;
    g->n = n;
    g->box = box;
    g->l = l;
    /* cell side box/G >= l (with a margin far above float64 rounding) */
    int64_t G = (l > 0) ? (int64_t)floor(box / (l * (1.0 + 1e-9))) : 1;
    if (G < 3) G = 1; /* fewer than 3 cells per side would alias neighbours */
    if (G > 2000000) G = 2000000;
    g->G = G;
    g->cells = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
    g->stamp = (uint32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint32_t));
    if (!g->cells || !g->stamp) {
        free(g->cells);
        free(g->stamp);
        free(g);
        return NULL;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t cx = cell_coord(pos[3 * i + 0], box, G);
        int64_t cy = cell_coord(pos[3 * i + 1], box, G);
        int64_t cz = cell_coord(pos[3 * i + 2], box, G);
        g->cells[i].key = (cz * G + cy) * G + cx;
        g->cells[i].idx = i;
    }
    qsort(g->cells, (size_t)n, sizeof(kv_t), kv_cmp);
    return g;
}

void or_grid_free(or_grid *g)
{
    if (!g) return;
    free(g->cells);
    free(g->stamp);
    free(g);
}

/* first position in the sorted cell list whose key is >= key */
static int64_t lower_bound_key(const or_grid *g, int64_t key)
{
    int64_t lo = 0, hi = g->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->cells[mid].key < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Calls visit(j) for every particle j != i within l of particle i.
 * Returns the number of such particles. */
typedef void (*visit_fn)(void *arg, int64_t i, int64_t j, double d2);

static int64_t grid_radius(const or_grid *g, int64_t i, double l2, visit_fn visit, void *arg);

static int64_t grid_neighbours(const or_grid *g, int64_t i, visit_fn visit, void *arg)
{
    return grid_radius(g, i, g->l * g->l, visit, arg);
}

/* The same for every particle within sqrt(l2) <= the grid's cell radius. */
static int64_t grid_radius(const or_grid *g, int64_t i, double l2, visit_fn visit, void *arg)
{
    int64_t found = 0;
    if (g->G == 1) {
        for (int64_t j = 0; j < g->n; j++) {
            if (j == i) continue;
            double d2 = dist2_3d(g->pos, i, j, g->box);
            if (d2 <= l2) {
                found++;
                if (visit) visit(arg, i, j, d2);
            }
        }
        return found;
    }
    const int64_t G = g->G;
    int64_t cx = cell_coord(g->pos[3 * i + 0], g->box, G);
    int64_t cy = cell_coord(g->pos[3 * i + 1], g->box, G);
    int64_t cz = cell_coord(g->pos[3 * i + 2], g->box, G);
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int64_t x = (cx + dx + G) % G, y = (cy + dy + G) % G, z = (cz + dz + G) % G;
                int64_t key = (z * G + y) * G + x;
                for (int64_t p = lower_bound_key(g, key); p < g->n && g->cells[p].key == key; p++) {
                    int64_t j = g->cells[p].idx;
                    if (j == i) continue;
                    double d2 = dist2_3d(g->pos, i, j, g->box);
                    if (d2 <= l2) {
                        found++;
                        if (visit) visit(arg, i, j, d2);
                    }
                }
            }
    return found;
}

typedef struct {
    int32_t *parent;
    int64_t tie;
    double l;
} fof_arg;

static void fof_visit(void *a, int64_t i, int64_t j, double d2)
{
    fof_arg *f = (fof_arg *)a;
    if (j <= i) return; /* each unordered pair once */
    uf_union(f->parent, (int32_t)i, (int32_t)j);
    double d = sqrt(d2);
    if (f->l > 0 && fabs(d - f->l) <= TIE_REL * f->l) f->tie++;
}

/* Labels every particle with the smallest index in its FOF group.
 * n_tieband receives the number of pairs with |d - l| <= 1e-6 l (d <= l side
 * only: pairs beyond l are not visited). */
int or_fof3d(const float *pos, int64_t n, double box, double l, int32_t *labels, int64_t *n_tieband)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || !(box > 0) || !(l >= 0)) return OR_ERR_ARG;
    or_grid *g = or_grid_build(pos, n, box, l);
    if (!g) return OR_ERR_OOM;
    for (int64_t i = 0; i < n; i++) labels[i] = (int32_t)i;
    fof_arg a = {labels, 0, l};
    for (int64_t i = 0; i < n; i++) grid_neighbours(g, i, fof_visit, &a);
    for (int64_t i = 0; i < n; i++) labels[i] = uf_find(labels, (int32_t)i);
    if (n_tieband) *n_tieband = a.tie;
    or_grid_free(g);
    return OR_OK;
}

/* ---- accelerated 3D FOF (Sec. 3.1) ---------------------------------------
 * The paper's faster variant.  Particles are visited in index order (reading:
 * the paper leaves the order to its tree walk).  A visited particle with at
 * most dense_n neighbours within l (the paper's 16; the particle itself not
 * counted) is joined with those neighbours as in plain FOF.  One with more
 * is joined with every particle within 2l instead, and each of its
 * neighbours within l is marked so that its own neighbour search is skipped
 * when its turn comes.  The groups are unions of plain FOF groups. */
typedef struct {
    int64_t *list;
    int64_t len, cap;
    int oom;
} list_arg;

static void list_visit(void *a, int64_t i, int64_t j, double d2)
{
    (void)i;
    (void)d2;
    list_arg *L = (list_arg *)a;
    if (L->len == L->cap) {
        int64_t c = L->cap ? 2 * L->cap : 64;
        int64_t *p = (int64_t *)realloc(L->list, sizeof(int64_t) * (size_t)c);
        if (!p) {
            L->oom = 1;
            return;
        }
        L->list = p;
        L->cap = c;
    }
    L->list[L->len++] = j;
}

static void join_visit(void *a, int64_t i, int64_t j, double d2)
{
    (void)d2;
    uf_union((int32_t *)a, (int32_t)i, (int32_t)j);
}

int or_fof3d_accel(const float *pos, int64_t n, double box, double l, int64_t dense_n, int32_t *labels,
                   int64_t *n_centres)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || !(box > 0) || !(l >= 0) || dense_n < 0) return OR_ERR_ARG;
    /* cells of side >= 2l, so both searches look at the 27 nearest cells */
    or_grid *g = or_grid_build(pos, n, box, 2.0 * l);
    if (!g) return OR_ERR_OOM;
    unsigned char *skip = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!skip) {
        or_grid_free(g);
        return OR_ERR_OOM;
    }
    for (int64_t i = 0; i < n; i++) labels[i] = (int32_t)i;
    const double l2 = l * l, r2 = (2.0 * l) * (2.0 * l);
    list_arg nb = {NULL, 0, 0, 0};
    int64_t centres = 0;
    for (int64_t i = 0; i < n; i++) {
        if (skip[i]) continue;
        nb.len = 0;
        grid_radius(g, i, l2, list_visit, &nb);
        if (nb.oom) break;
        if (nb.len > dense_n) {
            for (int64_t a = 0; a < nb.len; a++) skip[nb.list[a]] = 1;
            grid_radius(g, i, r2, join_visit, labels);
            centres++;
        } else {
            for (int64_t a = 0; a < nb.len; a++) uf_union(labels, (int32_t)i, (int32_t)nb.list[a]);
        }
    }
    const int oom = nb.oom;
    free(nb.list);
    free(skip);
    or_grid_free(g);
    if (oom) return OR_ERR_OOM;
    for (int64_t i = 0; i < n; i++) labels[i] = uf_find(labels, (int32_t)i);
    if (n_centres) *n_centres = centres;
    return OR_OK;
}

/* Pairs (i<j) whose distance lies within the tie band of l on either side. */
int64_t or_fof3d_tieband(const float *pos, int64_t n, double box, double l)
{
    double lw = l * (1.0 + 2.0 * TIE_REL);
    or_grid *g = or_grid_build(pos, n, box, lw);
    if (!g) return -1;
    int64_t tie = 0;
    for (int64_t i = 0; i < n; i++) {
        /* enumerate neighbours within the widened radius */
        const int64_t G = g->G;
        if (G == 1) {
            for (int64_t j = i + 1; j < n; j++) {
                double d = sqrt(dist2_3d(pos, i, j, box));
                if (l > 0 && fabs(d - l) <= TIE_REL * l) tie++;
            }
            continue;
        }
        int64_t cx = cell_coord(pos[3 * i + 0], box, G);
        int64_t cy = cell_coord(pos[3 * i + 1], box, G);
        int64_t cz = cell_coord(pos[3 * i + 2], box, G);
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int64_t x = (cx + dx + G) % G, y = (cy + dy + G) % G, z = (cz + dz + G) % G;
                    int64_t key = (z * G + y) * G + x;
                    for (int64_t p = lower_bound_key(g, key); p < n && g->cells[p].key == key; p++) {
                        int64_t j = g->cells[p].idx;
                        if (j <= i) continue;
                        double d = sqrt(dist2_3d(pos, i, j, box));
                        if (l > 0 && fabs(d - l) <= TIE_REL * l) tie++;
                    }
                }
    }
    or_grid_free(g);
    return tie;
}

/* All j != i within l of particle i, ascending.  Returns the count, or -1 if
 * more than cap were found. */
typedef struct {
    int32_t *out;
    int64_t cap, k;
} coll_arg;

static void coll_visit(void *a, int64_t i, int64_t j, double d2)
{
    (void)i;
    (void)d2;
    coll_arg *c = (coll_arg *)a;
    if (c->k < c->cap) c->out[c->k] = (int32_t)j;
    c->k++;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t or_grid_neighbours(or_grid *g, int64_t i, int32_t *out, int64_t cap)
{
    coll_arg c = {out, cap, 0};
    grid_neighbours(g, i, coll_visit, &c);
    if (c.k > cap) return -1;
    qsort(out, (size_t)c.k, sizeof(int32_t), cmp_i32);
    return c.k;
}

/* The FOF group of particle `seed`, found by breadth-first search over the
 * friendship graph.  Members are written ascending; returns the count, or -1
 * if the group has more than cap members. */
typedef struct {
    or_grid *g;
    int32_t *queue;
    int64_t cap, tail;
    int overflow;
} bfs_arg;

static void bfs_visit(void *a, int64_t i, int64_t j, double d2)
{
    (void)i;
    (void)d2;
    bfs_arg *b = (bfs_arg *)a;
    if (b->g->stamp[j] == b->g->cur) return;
    b->g->stamp[j] = b->g->cur;
    if (b->tail >= b->cap) {
        b->overflow = 1;
        return;
    }
    b->queue[b->tail++] = (int32_t)j;
}

int64_t or_grid_component(or_grid *g, int64_t seed, int32_t *out, int64_t cap)
{
    if (!g || seed < 0 || seed >= g->n || cap < 1) return -1;
    g->cur++;
    if (g->cur == 0) {
        memset(g->stamp, 0, sizeof(uint32_t) * (size_t)g->n);
        g->cur = 1;
    }
    bfs_arg b = {g, out, cap, 0, 0};
    g->stamp[seed] = g->cur;
    out[b.tail++] = (int32_t)seed;
    for (int64_t head = 0; head < b.tail && !b.overflow; head++) grid_neighbours(g, out[head], bfs_visit, &b);
    if (b.overflow) return -1;
    qsort(out, (size_t)b.tail, sizeof(int32_t), cmp_i32);
    return b.tail;
}

/* ======================================================================== */
/* Phase-space hierarchy (Sec. 3.2)                                          */
/* ======================================================================== */

/* Neumaier-compensated running sum */
typedef struct {
    double s, c;
} ksum;

static void ks_add(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}

static double ks_val(const ksum *k) { return k->s + k->c; }

/* Mean and dispersion of positions and velocities of a member list.
 * Reading: the dispersion is the 3D total, sigma_x^2 = (1/n) sum |x - xbar|^2
 * (and likewise sigma_v); the paper does not fix the per-axis/total or the
 * 1/n vs 1/(n-1) choice, and the subgroup partition does not depend on it
 * because a common factor on both sigmas rescales every distance and the
 * linking length alike.  Positions are unwrapped to the periodic image
 * nearest the member with the smallest index; the mean is wrapped back into
 * [0, box).  Returns OR_ERR_EXTENT if the unwrapped members span half the box
 * or more on some axis (the unwrap would be ambiguous). */
typedef struct {
    double xbar[3], vbar[3], sigx, sigv;
} moments_t;

static int moments_of(const float *pos, const float *vel, const int32_t *mem, int64_t n, double box,
                      moments_t *m)
{
    int32_t ref = mem[0];
    for (int64_t a = 1; a < n; a++)
        if (mem[a] < ref) ref = mem[a];
    ksum sx[3] = {{0, 0}, {0, 0}, {0, 0}}, sv[3] = {{0, 0}, {0, 0}, {0, 0}};
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int64_t a = 0; a < n; a++) {
        int32_t i = mem[a];
        for (int d = 0; d < 3; d++) {
            double dx = min_image((double)pos[3 * (int64_t)i + d] - (double)pos[3 * (int64_t)ref + d], box);
            double dv = (double)vel[3 * (int64_t)i + d] - (double)vel[3 * (int64_t)ref + d];
            ks_add(&sx[d], dx);
            ks_add(&sv[d], dv);
            if (dx < lo[d]) lo[d] = dx;
            if (dx > hi[d]) hi[d] = dx;
        }
    }
    for (int d = 0; d < 3; d++)
        if (hi[d] - lo[d] >= 0.5 * box) return OR_ERR_EXTENT;
    double mx[3], mv[3];
    for (int d = 0; d < 3; d++) {
        mx[d] = ks_val(&sx[d]) / (double)n;
        mv[d] = ks_val(&sv[d]) / (double)n;
    }
    ksum qx = {0, 0}, qv = {0, 0};
    for (int64_t a = 0; a < n; a++) {
        int32_t i = mem[a];
        for (int d = 0; d < 3; d++) {
            double dx = min_image((double)pos[3 * (int64_t)i + d] - (double)pos[3 * (int64_t)ref + d], box) - mx[d];
            double dv = ((double)vel[3 * (int64_t)i + d] - (double)vel[3 * (int64_t)ref + d]) - mv[d];
            ks_add(&qx, dx * dx);
            ks_add(&qv, dv * dv);
        }
    }
    for (int d = 0; d < 3; d++) {
        double x = (double)pos[3 * (int64_t)ref + d] + mx[d];
        x = fmod(x, box);
        if (x < 0) x += box;
        if (x >= box) x -= box;
        m->xbar[d] = x;
        m->vbar[d] = (double)vel[3 * (int64_t)ref + d] + mv[d];
    }
    m->sigx = sqrt(ks_val(&qx) / (double)n);
    m->sigv = sqrt(ks_val(&qv) / (double)n);
    return OR_OK;
}

/* Eq. 1: squared phase-space distance between particles i and j of a group
 * with dispersions sigx, sigv.  Reading: a zero dispersion drops its term
 * (then every member shares that coordinate and the difference is zero). */
static double dist2_6d(const float *pos, const float *vel, int32_t i, int32_t j, double box, double sigx,
                       double sigv)
{
    double sx = 0.0, sv = 0.0;
    for (int d = 0; d < 3; d++) {
        double dx = min_image((double)pos[3 * (int64_t)i + d] - (double)pos[3 * (int64_t)j + d], box);
        double dv = (double)vel[3 * (int64_t)i + d] - (double)vel[3 * (int64_t)j + d];
        sx += dx * dx;
        sv += dv * dv;
    }
    double r = 0.0;
    if (sigx > 0) r += sx / (sigx * sigx);
    if (sigv > 0) r += sv / (sigv * sigv);
    return r;
}

/* ---- a 6D k-d tree over normalised coordinates, used only to prune ------ */
/* Distances are always re-evaluated with dist2_6d on the raw coordinates;    */
/* the tree only decides which members can be skipped, with a safety factor  */
/* far above the rounding difference between the two forms.                  */
typedef struct {
    int64_t n;
    double *u;          /* n x 6 normalised coordinates, by local index */
    int32_t *idx;       /* local indices, permuted into tree order */
    int32_t *lo, *hi;   /* node ranges into idx */
    int32_t *left, *right;
    int8_t *dim;
    double *split;
    int32_t nnodes, cap;
} kdtree;

#define KD_LEAF 8
#define KD_SLACK (1.0 + 1e-9)

static int g_kd_threshold = 1024; /* brute force at or below this many members */

void or_set_kd_threshold(int t) { g_kd_threshold = t; }

static double *g_sort_u;
static int g_sort_dim;
static int cmp_by_dim(const void *a, const void *b)
{
    double x = g_sort_u[6 * (*(const int32_t *)a) + g_sort_dim];
    double y = g_sort_u[6 * (*(const int32_t *)b) + g_sort_dim];
    if (x < y) return -1;
    if (x > y) return 1;
    int32_t p = *(const int32_t *)a, q = *(const int32_t *)b;
    return (p > q) - (p < q);
}

static int32_t kd_build_rec(kdtree *t, int32_t lo, int32_t hi)
{
    int32_t me = t->nnodes++;
    t->lo[me] = lo;
    t->hi[me] = hi;
    t->left[me] = t->right[me] = -1;
    t->dim[me] = -1;
    if (hi - lo <= KD_LEAF) return me;
    double best = -1.0;
    int bd = 0;
    for (int d = 0; d < 6; d++) {
        double a = INFINITY, b = -INFINITY;
        for (int32_t p = lo; p < hi; p++) {
            double x = t->u[6 * t->idx[p] + d];
            if (x < a) a = x;
            if (x > b) b = x;
        }
        if (b - a > best) {
            best = b - a;
            bd = d;
        }
    }
    if (!(best > 0)) return me; /* all coincide: keep as one leaf */
    g_sort_u = t->u;
    g_sort_dim = bd;
    qsort(t->idx + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_by_dim);
    int32_t mid = lo + (hi - lo) / 2;
    t->dim[me] = (int8_t)bd;
    t->split[me] = t->u[6 * t->idx[mid] + bd];
    int32_t L = kd_build_rec(t, lo, mid);
    int32_t R = kd_build_rec(t, mid, hi);
    t->left[me] = L;
    t->right[me] = R;
    return me;
}

static int kd_build(kdtree *t, const double *u, int64_t n)
{
    memset(t, 0, sizeof(*t));
    t->n = n;
    t->u = (double *)u;
    t->cap = (int32_t)(2 * (n / (KD_LEAF / 2) + 1) + 8);
    t->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    t->lo = (int32_t *)malloc(sizeof(int32_t) * (size_t)t->cap);
    t->hi = (int32_t *)malloc(sizeof(int32_t) * (size_t)t->cap);
    t->left = (int32_t *)malloc(sizeof(int32_t) * (size_t)t->cap);
    t->right = (int32_t *)malloc(sizeof(int32_t) * (size_t)t->cap);
    t->dim = (int8_t *)malloc((size_t)t->cap);
    t->split = (double *)malloc(sizeof(double) * (size_t)t->cap);
    if (!t->idx || !t->lo || !t->hi || !t->left || !t->right || !t->dim || !t->split) return OR_ERR_OOM;
    for (int64_t i = 0; i < n; i++) t->idx[i] = (int32_t)i;
    kd_build_rec(t, 0, (int32_t)n);
    return OR_OK;
}

static void kd_free(kdtree *t)
{
    free(t->idx);
    free(t->lo);
    free(t->hi);
    free(t->left);
    free(t->right);
    free(t->dim);
    free(t->split);
}

/* group-local view of the member list for distance evaluation */
typedef struct {
    const float *pos, *vel;
    const int32_t *mem;
    double box, sigx, sigv;
} grp_t;

static double gdist2(const grp_t *g, int32_t a, int32_t b)
{
    return dist2_6d(g->pos, g->vel, g->mem[a], g->mem[b], g->box, g->sigx, g->sigv);
}

static void kd_nn_rec(const kdtree *t, const grp_t *g, int32_t node, int32_t q, double *best)
{
    if (t->dim[node] < 0) {
        for (int32_t p = t->lo[node]; p < t->hi[node]; p++) {
            int32_t j = t->idx[p];
            if (j == q) continue;
            double d2 = gdist2(g, q, j);
            if (d2 < *best) *best = d2;
        }
        return;
    }
    int d = t->dim[node];
    double diff = t->u[6 * q + d] - t->split[node];
    int32_t nearc = diff < 0 ? t->left[node] : t->right[node];
    int32_t farc = diff < 0 ? t->right[node] : t->left[node];
    kd_nn_rec(t, g, nearc, q, best);
    if (diff * diff <= (*best) * KD_SLACK) kd_nn_rec(t, g, farc, q, best);
}

typedef struct {
    int32_t *parent;
    double l2, l, lo2, hi2;
    int64_t tie;
} link_arg;

/* The linking length is itself the distance of one member pair, so that
 * pair always sits exactly on l; only pairs whose distance differs from l
 * and lies within 1e-6 l of it count as tie-band pairs. */
static void link_pair(link_arg *a, int32_t i, int32_t j, double d2)
{
    if (d2 <= a->l2) uf_union(a->parent, i, j);
    if (a->l > 0 && d2 != a->l2 && d2 >= a->lo2 && d2 <= a->hi2) {
        double d = sqrt(d2);
        if (fabs(d - a->l) <= TIE_REL * a->l) a->tie++;
    }
}

static void kd_range_rec(const kdtree *t, const grp_t *g, int32_t node, int32_t q, double r2, link_arg *a)
{
    if (t->dim[node] < 0) {
        for (int32_t p = t->lo[node]; p < t->hi[node]; p++) {
            int32_t j = t->idx[p];
            if (j <= q) continue;
            double d2 = gdist2(g, q, j);
            if (d2 <= r2) link_pair(a, q, j, d2);
        }
        return;
    }
    int d = t->dim[node];
    double diff = t->u[6 * q + d] - t->split[node];
    int32_t nearc = diff < 0 ? t->left[node] : t->right[node];
    int32_t farc = diff < 0 ? t->right[node] : t->left[node];
    kd_range_rec(t, g, nearc, q, r2, a);
    if (diff * diff <= r2 * KD_SLACK) kd_range_rec(t, g, farc, q, r2, a);
}

static int cmp_f64(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* ---- the hierarchy ------------------------------------------------------ */
typedef struct {
    int32_t parent, level, minidx, group, nchild;
    int64_t first, count, tie, child_span;
    double lnk, xbar[3], vbar[3], sigx, sigv;
} or_node;

struct or_tree {
    const float *pos, *vel;
    int64_t n_total;
    double box, f;
    int32_t min_n;
    int64_t sub_n;      /* nodes above this size use a subset of sub_n members for l (0: never) */
    uint64_t sub_seed;  /* seed of the subset keys */
    int32_t *mem;       /* member particle indices, groups back to back */
    int64_t n_mem;
    or_node *nodes;
    int64_t n_nodes, cap_nodes;
    /* assignment results */
    int64_t n_halos;
    int32_t *halo_id_of_leaf; /* per node: merged halo id for leaves, -1 otherwise */
    int32_t *h_id;
    int64_t *h_ncore;
    int32_t *h_nseeds;
    double *h_xbar, *h_vbar, *h_sigv, *h_rdyn2;
    int status;
};
typedef struct or_tree or_tree;

static int64_t push_node(or_tree *t, or_node nd)
{
    if (t->n_nodes == t->cap_nodes) {
        int64_t c = t->cap_nodes ? 2 * t->cap_nodes : 1024;
        or_node *p = (or_node *)realloc(t->nodes, sizeof(or_node) * (size_t)c);
        if (!p) return -1;
        t->nodes = p;
        t->cap_nodes = c;
    }
    t->nodes[t->n_nodes] = nd;
    return t->n_nodes++;
}

typedef struct {
    int32_t comp_min; /* smallest particle index of the member's component */
    int32_t comp_size;
    int32_t pidx;     /* particle index */
    int32_t is_child;
} sort_rec;

static int cmp_sort_rec(const void *a, const void *b)
{
    const sort_rec *x = (const sort_rec *)a, *y = (const sort_rec *)b;
    if (x->is_child != y->is_child) return y->is_child - x->is_child; /* children first */
    if (x->is_child && x->comp_min != y->comp_min) return (x->comp_min > y->comp_min) - (x->comp_min < y->comp_min);
    return (x->pidx > y->pidx) - (x->pidx < y->pidx);
}

/* ---- random subsets for the linking length (Sec. 3.2) -------------------
 * Nodes with more members than a limit s take their linking length from the
 * nearest-neighbour distances of s randomly chosen members instead of all of
 * them.  The randomness is SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: particle i gets the (i+1)-th output of the stream whose state
 * starts at the seed, i.e. the finaliser applied to seed + (i+1)*gamma.  The
 * finaliser is a bijection of 64-bit words and gamma is odd, so distinct
 * particles get distinct keys; a node's subset is its s members with the
 * smallest keys, which is a uniformly random s-subset. */
#define SM64_GAMMA 0x9e3779b97f4a7c15ULL

static uint64_t sm64_finalise(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t or_sample_key(uint64_t seed, int64_t i) { return sm64_finalise(seed + (uint64_t)(i + 1) * SM64_GAMMA); }

/* keys of particles first .. first+count-1 */
void or_sample_keys(uint64_t seed, int64_t first, int64_t count, uint64_t *out)
{
    for (int64_t i = 0; i < count; i++) out[i] = or_sample_key(seed, first + i);
}

typedef struct {
    uint64_t key;
    int64_t slot;
} key_slot;

static int cmp_key_slot(const void *a, const void *b)
{
    const key_slot *x = (const key_slot *)a, *y = (const key_slot *)b;
    return (x->key > y->key) - (x->key < y->key);
}

/* Marks in `in` (0/1 per slot) the s members of mem[0..n) with the smallest
 * keys. */
static int sample_subset(const int32_t *mem, int64_t n, int64_t s, uint64_t seed, unsigned char *in)
{
    key_slot *ks = (key_slot *)malloc(sizeof(key_slot) * (size_t)n);
    if (!ks) return OR_ERR_OOM;
    for (int64_t a = 0; a < n; a++) {
        ks[a].key = or_sample_key(seed, mem[a]);
        ks[a].slot = a;
        in[a] = 0;
    }
    qsort(ks, (size_t)n, sizeof(key_slot), cmp_key_slot);
    for (int64_t a = 0; a < s && a < n; a++) in[ks[a].slot] = 1;
    free(ks);
    return OR_OK;
}

/* Refines one node (Sec. 3.2) and recurses into its children. */
static int refine_node(or_tree *t, int64_t id)
{
    or_node nd = t->nodes[id];
    const int64_t n = nd.count;
    int32_t *mem = t->mem + nd.first;
    moments_t m;
    int st = moments_of(t->pos, t->vel, mem, n, t->box, &m);
    if (st) return st;
    for (int d = 0; d < 3; d++) {
        nd.xbar[d] = m.xbar[d];
        nd.vbar[d] = m.vbar[d];
    }
    nd.sigx = m.sigx;
    nd.sigv = m.sigv;
    grp_t g = {t->pos, t->vel, mem, t->box, m.sigx, m.sigv};

    /* nearest-neighbour distance under Eq. 1 of every member, or of the
     * random subset's members when the node is above the subset size (the
     * neighbour is still searched among all members); the others get -1 */
    double *dnn2 = (double *)malloc(sizeof(double) * (size_t)n);
    double *u = NULL;
    kdtree kd;
    int use_kd = n > g_kd_threshold;
    if (!dnn2) return OR_ERR_OOM;
    const int sampled = t->sub_n > 0 && n > t->sub_n;
    const int64_t n_eff = sampled ? t->sub_n : n;
    unsigned char *in = (unsigned char *)malloc((size_t)n);
    if (!in) return OR_ERR_OOM;
    if (sampled) {
        st = sample_subset(mem, n, t->sub_n, t->sub_seed, in);
        if (st) return st;
    } else {
        memset(in, 1, (size_t)n);
    }
    if (use_kd) {
        int32_t ref = mem[0];
        for (int64_t a = 1; a < n; a++)
            if (mem[a] < ref) ref = mem[a];
        u = (double *)malloc(sizeof(double) * 6 * (size_t)n);
        if (!u) return OR_ERR_OOM;
        for (int64_t a = 0; a < n; a++) {
            for (int d = 0; d < 3; d++) {
                double dx = min_image((double)t->pos[3 * (int64_t)mem[a] + d] - (double)t->pos[3 * (int64_t)ref + d], t->box);
                double dv = (double)t->vel[3 * (int64_t)mem[a] + d] - (double)t->vel[3 * (int64_t)ref + d];
                u[6 * a + d] = m.sigx > 0 ? dx / m.sigx : 0.0;
                u[6 * a + 3 + d] = m.sigv > 0 ? dv / m.sigv : 0.0;
            }
        }
        if (kd_build(&kd, u, n)) return OR_ERR_OOM;
        for (int64_t a = 0; a < n; a++) {
            double best = INFINITY;
            if (!in[a]) {
                dnn2[a] = -1.0;
                continue;
            }
            kd_nn_rec(&kd, &g, 0, (int32_t)a, &best);
            dnn2[a] = best;
        }
    } else {
        for (int64_t a = 0; a < n; a++) {
            double best = INFINITY;
            if (!in[a]) {
                dnn2[a] = -1.0;
                continue;
            }
            for (int64_t b = 0; b < n; b++) {
                if (b == a) continue;
                double d2 = gdist2(&g, (int32_t)a, (int32_t)b);
                if (d2 < best) best = d2;
            }
            dnn2[a] = best;
        }
    }

    /* linking length: the k-th smallest nearest-neighbour distance with
     * k = ceil(f n), so that at least a fraction f of the members have a
     * friend within it (reading of "a constant fraction f ... are linked");
     * over the subset, with n its size, when the node is sampled */
    int64_t k = (int64_t)ceil(t->f * (double)n_eff);
    if (k < 1) k = 1;
    if (k > n_eff) k = n_eff;
    double *srt = (double *)malloc(sizeof(double) * (size_t)n_eff);
    if (!srt) return OR_ERR_OOM;
    int64_t ns = 0;
    for (int64_t a = 0; a < n; a++)
        if (in[a]) srt[ns++] = dnn2[a];
    free(in);
    qsort(srt, (size_t)ns, sizeof(double), cmp_f64);
    double l2 = srt[k - 1];
    free(srt);
    double l = sqrt(l2);
    nd.lnk = l;

    /* friends-of-friends at l inside the node (inclusive: d <= l) */
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!par) return OR_ERR_OOM;
    for (int64_t a = 0; a < n; a++) par[a] = (int32_t)a;
    link_arg la = {par, l2, l, 0, 0, 0};
    double lo = l * (1.0 - TIE_REL), hi = l * (1.0 + TIE_REL);
    la.lo2 = lo * lo * (1.0 - 1e-12);
    la.hi2 = hi * hi * (1.0 + 1e-12);
    double r2 = la.hi2 > l2 ? la.hi2 : l2;
    if (use_kd) {
        for (int64_t a = 0; a < n; a++)
            if (dnn2[a] <= r2) kd_range_rec(&kd, &g, 0, (int32_t)a, r2, &la);
        kd_free(&kd);
        free(u);
    } else {
        for (int64_t a = 0; a < n; a++) {
            if (dnn2[a] > r2) continue;
            for (int64_t b = a + 1; b < n; b++) {
                double d2 = gdist2(&g, (int32_t)a, (int32_t)b);
                if (d2 <= r2) link_pair(&la, (int32_t)a, (int32_t)b, d2);
            }
        }
    }
    nd.tie = la.tie;
    free(dnn2);

    /* components: size and smallest particle index */
    int32_t *csize = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *cmin = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    sort_rec *rec = (sort_rec *)malloc(sizeof(sort_rec) * (size_t)n);
    if (!csize || !cmin || !rec) return OR_ERR_OOM;
    for (int64_t a = 0; a < n; a++) cmin[a] = INT32_MAX;
    for (int64_t a = 0; a < n; a++) {
        int32_t r = uf_find(par, (int32_t)a);
        csize[r]++;
        if (mem[a] < cmin[r]) cmin[r] = mem[a];
    }
    /* children: components with at least min_n members that are strictly
     * smaller than the node (a component equal to the whole node makes no
     * progress and is not a subgroup -- reading, needed for termination
     * when duplicate points give a zero linking length) */
    for (int64_t a = 0; a < n; a++) {
        int32_t r = uf_find(par, (int32_t)a);
        rec[a].comp_min = cmin[r];
        rec[a].comp_size = csize[r];
        rec[a].pidx = mem[a];
        rec[a].is_child = (csize[r] >= t->min_n && csize[r] < n) ? 1 : 0;
    }
    free(par);
    free(csize);
    free(cmin);
    qsort(rec, (size_t)n, sizeof(sort_rec), cmp_sort_rec);
    for (int64_t a = 0; a < n; a++) mem[a] = rec[a].pidx;
    /* children occupy the front of the node's range, ordered by their
     * smallest particle index; the remaining members follow by index */
    int32_t nchild = 0;
    int64_t a = 0;
    int64_t child_first[4096];
    int64_t *cf = child_first;
    int64_t cf_cap = 4096;
    int64_t child_cnt[4096];
    int64_t *cc = child_cnt;
    int heap = 0;
    while (a < n && rec[a].is_child) {
        int64_t b = a;
        while (b < n && rec[b].is_child && rec[b].comp_min == rec[a].comp_min) b++;
        if (nchild == cf_cap) {
            int64_t nc = cf_cap * 2;
            int64_t *ncf = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
            int64_t *ncc = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
            if (!ncf || !ncc) return OR_ERR_OOM;
            memcpy(ncf, cf, sizeof(int64_t) * (size_t)cf_cap);
            memcpy(ncc, cc, sizeof(int64_t) * (size_t)cf_cap);
            if (heap) {
                free(cf);
                free(cc);
            }
            cf = ncf;
            cc = ncc;
            cf_cap = nc;
            heap = 1;
        }
        cf[nchild] = a;
        cc[nchild] = b - a;
        nchild++;
        a = b;
    }
    free(rec);
    nd.nchild = nchild;
    nd.child_span = a;
    t->nodes[id] = nd;
    int64_t *kids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nchild > 0 ? nchild : 1));
    if (!kids) return OR_ERR_OOM;
    for (int32_t c = 0; c < nchild; c++) {
        or_node ch;
        memset(&ch, 0, sizeof(ch));
        ch.parent = (int32_t)id;
        ch.level = nd.level + 1;
        ch.group = nd.group;
        ch.first = nd.first + cf[c];
        ch.count = cc[c];
        int32_t mn = INT32_MAX;
        for (int64_t q = 0; q < ch.count; q++)
            if (t->mem[ch.first + q] < mn) mn = t->mem[ch.first + q];
        ch.minidx = mn;
        kids[c] = push_node(t, ch);
        if (kids[c] < 0) return OR_ERR_OOM;
    }
    if (heap) {
        free(cf);
        free(cc);
    }
    for (int32_t c = 0; c < nchild; c++) {
        st = refine_node(t, kids[c]);
        if (st) {
            free(kids);
            return st;
        }
    }
    free(kids);
    return OR_OK;
}

/* Builds the phase-space hierarchy of every group (Sec. 3.2).  `members`
 * lists the particles of each group back to back, group g occupying
 * members[group_offsets[g] .. group_offsets[g+1]).  Groups with fewer than
 * min_n members are not refined (reading: the recursion floor applies to the
 * 3D groups too).  Recursion stops at nodes without a subgroup of at least
 * min_n members; those nodes are the seed halos (Sec. 3.3).  With sub_n > 0
 * a node of more than sub_n members takes its linking length from the
 * nearest-neighbour distances of sub_n of its members, drawn with the keys of
 * or_sample_key(sub_seed, .), and k = ceil(f sub_n) (Sec. 3.2: above 10,000
 * members the paper computes them for a random 10,000-member subset). */
or_tree *or_refine_sampled(const float *pos, const float *vel, int64_t n_total, double box, const int32_t *members,
                           const int64_t *group_offsets, int64_t n_groups, double f, int32_t min_n, int64_t sub_n,
                           uint64_t sub_seed, int *status)
{
    *status = OR_ERR_ARG;
    if (!(box > 0) || !(f > 0 && f < 1) || min_n < 2 || n_groups < 0 || sub_n < 0) return NULL;
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    if (!t) {
        *status = OR_ERR_OOM;
        return NULL;
    }
    t->pos = pos;
    t->vel = vel;
    t->n_total = n_total;
    t->box = box;
    t->f = f;
    t->min_n = min_n;
    t->sub_n = sub_n;
    t->sub_seed = sub_seed;
    t->n_mem = group_offsets[n_groups] - group_offsets[0];
    t->mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(t->n_mem > 0 ? t->n_mem : 1));
    if (!t->mem) {
        free(t);
        *status = OR_ERR_OOM;
        return NULL;
    }
    memcpy(t->mem, members + group_offsets[0], sizeof(int32_t) * (size_t)t->n_mem);
    for (int64_t gi = 0; gi < n_groups; gi++) {
        int64_t first = group_offsets[gi] - group_offsets[0];
        int64_t cnt = group_offsets[gi + 1] - group_offsets[gi];
        if (cnt < min_n) continue;
        qsort(t->mem + first, (size_t)cnt, sizeof(int32_t), cmp_i32);
        or_node root;
        memset(&root, 0, sizeof(root));
        root.parent = -1;
        root.level = 0;
        root.group = (int32_t)gi;
        root.first = first;
        root.count = cnt;
        root.minidx = t->mem[first];
        int64_t id = push_node(t, root);
        if (id < 0) {
            *status = OR_ERR_OOM;
            return t;
        }
        int st = refine_node(t, id);
        if (st) {
            *status = st;
            t->status = st;
            return t;
        }
    }
    *status = OR_OK;
    return t;
}

/* Every member's nearest-neighbour distance enters the linking length. */
or_tree *or_refine(const float *pos, const float *vel, int64_t n_total, double box, const int32_t *members,
                   const int64_t *group_offsets, int64_t n_groups, double f, int32_t min_n, int *status)
{
    return or_refine_sampled(pos, vel, n_total, box, members, group_offsets, n_groups, f, min_n, 0, 0, status);
}

int64_t or_tree_n_nodes(const or_tree *t) { return t->n_nodes; }
int64_t or_tree_n_members(const or_tree *t) { return t->n_mem; }

void or_tree_export(const or_tree *t, int32_t *parent, int32_t *level, int64_t *first, int64_t *count,
                    int32_t *minidx, int32_t *group, int32_t *nchild, double *lnk, double *xbar, double *vbar,
                    double *sigx, double *sigv, int64_t *tie)
{
    for (int64_t i = 0; i < t->n_nodes; i++) {
        const or_node *nd = &t->nodes[i];
        parent[i] = nd->parent;
        level[i] = nd->level;
        first[i] = nd->first;
        count[i] = nd->count;
        minidx[i] = nd->minidx;
        group[i] = nd->group;
        nchild[i] = nd->nchild;
        lnk[i] = nd->lnk;
        for (int d = 0; d < 3; d++) {
            xbar[3 * i + d] = nd->xbar[d];
            vbar[3 * i + d] = nd->vbar[d];
        }
        sigx[i] = nd->sigx;
        sigv[i] = nd->sigv;
        tie[i] = nd->tie;
    }
}

void or_tree_members(const or_tree *t, int32_t *out) { memcpy(out, t->mem, sizeof(int32_t) * (size_t)t->n_mem); }

void or_tree_free(or_tree *t)
{
    if (!t) return;
    free(t->mem);
    free(t->nodes);
    free(t->halo_id_of_leaf);
    free(t->h_id);
    free(t->h_ncore);
    free(t->h_nseeds);
    free(t->h_xbar);
    free(t->h_vbar);
    free(t->h_sigv);
    free(t->h_rdyn2);
    free(t);
}

/* ======================================================================== */
/* Seeds, merge and assignment (Sec. 3.3)                                    */
/* ======================================================================== */

/* zero-dispersion reading for ratios: 0/0 contributes 0, x/0 is infinite */
static double ratio2(double num2, double den2)
{
    if (den2 > 0) return num2 / den2;
    return num2 > 0 ? INFINITY : 0.0;
}


/* Eq. 2: phase-space separation of two seeds in units of the Poisson
 * uncertainties mu_x = sigma_x / sqrt(n), mu_v = sigma_v / sqrt(n) of the
 * smaller seed (fewer members; on a tie, the one with the larger smallest
 * particle index -- reading).  The seeds merge when this is below 10 sqrt 2. */
double merge_distance(int64_t na, int32_t mina, const double *xa, const double *va, double sxa, double sva,
                      int64_t nb, int32_t minb, const double *xb, const double *vb, double sxb, double svb,
                      double box)
{
    int a_small = (na != nb) ? (na < nb) : (mina > minb);
    double n = (double)(a_small ? na : nb);
    double sx = a_small ? sxa : sxb, sv = a_small ? sva : svb;
    double rn = sqrt(n);
    double mux = sx / rn, muv = sv / rn;
    double dx2 = 0, dv2 = 0;
    for (int d = 0; d < 3; d++) {
        double dx = min_image(xa[d] - xb[d], box);
        double dv = va[d] - vb[d];
        dx2 += dx * dx;
        dv2 += dv * dv;
    }
    return sqrt(ratio2(dx2, mux * mux) + ratio2(dv2, muv * muv));
}

/* Eq. 4: r_dyn,vir^2 = v_max^2 / (4/3 pi G rho_vir) with v_max^2 the largest
 * G M(<r)/r over the members (Sec. 3.4.4) and rho_vir = delta_vir m nbar.
 * With M(<r_(k)) = k m for the k-th smallest member radius r_(k) about the
 * centre, G and m cancel:  r_dyn^2 = max_k (k / r_(k)) / (4/3 pi delta_vir
 * nbar), over radii r_(k) > 0.  Returns -1 on allocation failure. */
double rdyn2_of(const float *pos, const int32_t *mem, int64_t n, double box, const double *xbar, double delta_vir,
                double nbar)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r) return -1.0;
    for (int64_t p = 0; p < n; p++) {
        double s = 0;
        for (int d = 0; d < 3; d++) {
            double dx = min_image((double)pos[3 * (int64_t)mem[p] + d] - xbar[d], box);
            s += dx * dx;
        }
        r[p] = sqrt(s);
    }
    qsort(r, (size_t)n, sizeof(double), cmp_f64);
    double best = 0.0;
    for (int64_t p = 0; p < n; p++)
        if (r[p] > 0) {
            double v = (double)(p + 1) / r[p];
            if (v > best) best = v;
        }
    free(r);
    return best / ((4.0 / 3.0) * M_PI * delta_vir * nbar);
}

/* moments of an arbitrary member list (exposed for the tests) */
int or_moments(const float *pos, const float *vel, const int32_t *mem, int64_t n, double box, double *out8)
{
    moments_t m;
    int st = moments_of(pos, vel, mem, n, box, &m);
    if (st) return st;
    out8[0] = m.sigx;
    out8[1] = m.sigv;
    for (int d = 0; d < 3; d++) {
        out8[2 + d] = m.xbar[d];
        out8[5 + d] = m.vbar[d];
    }
    return OR_OK;
}

typedef struct {
    int64_t first;
    int64_t node;
} leaf_ref;

static int cmp_leaf_ref(const void *a, const void *b)
{
    const leaf_ref *x = (const leaf_ref *)a, *y = (const leaf_ref *)b;
    return (x->first > y->first) - (x->first < y->first);
}

/* Seed halos are the nodes without subgroups (Sec. 3.3).  Within each 3D
 * group, two seeds merge when Eq. 2 holds with the Poisson uncertainties
 * mu = sigma / sqrt(n) of the seed with fewer members (tie: the one with the
 * larger smallest-index); every pair is tested with the seeds' own (unmerged)
 * properties and merges close transitively (readings).  A merged halo is
 * identified by the smallest particle index among its seeds' members, and its
 * centre, bulk velocity, sigma_v and v_max come from the union of those
 * members.  r_dyn,vir (Eq. 4) = v_max / sqrt(4/3 pi G rho_vir) with
 * rho_vir = delta_vir * m * nbar; G and the particle mass m cancel:
 * r_dyn^2 = max_k (k / r_(k)) / (4/3 pi delta_vir nbar), r_(k) the k-th
 * smallest distance of a member from the centre, k counting every member up
 * to that radius.  Each particle of a refined group is then decided at the
 * deepest node that holds it: members of a seed go to that seed's halo; the
 * other members of a node go to its only halo when its seeds form one halo,
 * else to the halo nearest under Eq. 3 (ties to the smaller halo id).
 * Particles outside refined groups get -1. */
int or_assign(or_tree *t, double delta_vir, double nbar, double merge_thresh, int32_t *halo_id,
              int64_t *n_halos_out)
{
    const float *pos = t->pos, *vel = t->vel;
    const double box = t->box;
    const int64_t NN = t->n_nodes;
    for (int64_t i = 0; i < t->n_total; i++) halo_id[i] = -1;
    free(t->halo_id_of_leaf);
    t->halo_id_of_leaf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(NN > 0 ? NN : 1));
    int64_t nleaf = 0;
    for (int64_t i = 0; i < NN; i++) {
        t->halo_id_of_leaf[i] = -1;
        if (t->nodes[i].nchild == 0) nleaf++;
    }
    leaf_ref *leaves = (leaf_ref *)malloc(sizeof(leaf_ref) * (size_t)(nleaf > 0 ? nleaf : 1));
    int32_t *uf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nleaf > 0 ? nleaf : 1));
    if (!leaves || !uf || !t->halo_id_of_leaf) return OR_ERR_OOM;
    int64_t q = 0;
    for (int64_t i = 0; i < NN; i++)
        if (t->nodes[i].nchild == 0) {
            leaves[q].first = t->nodes[i].first;
            leaves[q].node = i;
            q++;
        }
    /* leaves ordered by their place in the member array: every node's seeds
     * are then a contiguous run of this list (nested member ranges) */
    qsort(leaves, (size_t)nleaf, sizeof(leaf_ref), cmp_leaf_ref);
    for (int64_t a = 0; a < nleaf; a++) uf[a] = (int32_t)a;

    /* seed merge, pairs within one 3D group (Eq. 2) */
    const double thr = merge_thresh;
    int64_t a0 = 0;
    while (a0 < nleaf) {
        int32_t grp = t->nodes[leaves[a0].node].group;
        int64_t a1 = a0;
        while (a1 < nleaf && t->nodes[leaves[a1].node].group == grp) a1++;
        for (int64_t a = a0; a < a1; a++)
            for (int64_t b = a + 1; b < a1; b++) {
                const or_node *A = &t->nodes[leaves[a].node], *B = &t->nodes[leaves[b].node];
                double D = merge_distance(A->count, A->minidx, A->xbar, A->vbar, A->sigx, A->sigv, B->count,
                                          B->minidx, B->xbar, B->vbar, B->sigx, B->sigv, box);
                if (D < thr) uf_union(uf, (int32_t)a, (int32_t)b);
            }
        a0 = a1;
    }

    /* merged halos: members, id, properties */
    int64_t nh = 0;
    int32_t *hslot = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nleaf > 0 ? nleaf : 1));
    if (!hslot) return OR_ERR_OOM;
    for (int64_t a = 0; a < nleaf; a++) hslot[a] = -1;
    for (int64_t a = 0; a < nleaf; a++) {
        int32_t r = uf_find(uf, (int32_t)a);
        if (hslot[r] < 0) hslot[r] = (int32_t)nh++;
    }
    free(t->h_id);
    free(t->h_ncore);
    free(t->h_nseeds);
    free(t->h_xbar);
    free(t->h_vbar);
    free(t->h_sigv);
    free(t->h_rdyn2);
    size_t hsz = (size_t)(nh > 0 ? nh : 1);
    t->h_id = (int32_t *)malloc(sizeof(int32_t) * hsz);
    t->h_ncore = (int64_t *)calloc(hsz, sizeof(int64_t));
    t->h_nseeds = (int32_t *)calloc(hsz, sizeof(int32_t));
    t->h_xbar = (double *)malloc(sizeof(double) * 3 * hsz);
    t->h_vbar = (double *)malloc(sizeof(double) * 3 * hsz);
    t->h_sigv = (double *)malloc(sizeof(double) * hsz);
    t->h_rdyn2 = (double *)malloc(sizeof(double) * hsz);
    if (!t->h_id || !t->h_ncore || !t->h_nseeds || !t->h_xbar || !t->h_vbar || !t->h_sigv || !t->h_rdyn2)
        return OR_ERR_OOM;
    t->n_halos = nh;
    for (int64_t a = 0; a < nleaf; a++) {
        int32_t h = hslot[uf_find(uf, (int32_t)a)];
        t->h_ncore[h] += t->nodes[leaves[a].node].count;
        t->h_nseeds[h]++;
    }
    /* gather members per halo */
    int64_t *hoff = (int64_t *)calloc(hsz + 1, sizeof(int64_t));
    if (!hoff) return OR_ERR_OOM;
    for (int64_t h = 0; h < nh; h++) hoff[h + 1] = hoff[h] + t->h_ncore[h];
    int64_t *hfill = (int64_t *)calloc(hsz, sizeof(int64_t));
    int32_t *hmem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(hoff[nh] > 0 ? hoff[nh] : 1));
    if (!hfill || !hmem) return OR_ERR_OOM;
    for (int64_t a = 0; a < nleaf; a++) {
        int32_t h = hslot[uf_find(uf, (int32_t)a)];
        const or_node *L = &t->nodes[leaves[a].node];
        for (int64_t p = 0; p < L->count; p++) hmem[hoff[h] + hfill[h]++] = t->mem[L->first + p];
    }
    for (int64_t h = 0; h < nh; h++) {
        int32_t *hm = hmem + hoff[h];
        int64_t cnt = hoff[h + 1] - hoff[h];
        int32_t mn = INT32_MAX;
        for (int64_t p = 0; p < cnt; p++)
            if (hm[p] < mn) mn = hm[p];
        t->h_id[h] = mn;
        moments_t m;
        int st = moments_of(pos, vel, hm, cnt, box, &m);
        if (st) return st;
        for (int d = 0; d < 3; d++) {
            t->h_xbar[3 * h + d] = m.xbar[d];
            t->h_vbar[3 * h + d] = m.vbar[d];
        }
        t->h_sigv[h] = m.sigv;
        double r2 = rdyn2_of(pos, hm, cnt, box, m.xbar, delta_vir, nbar);
        if (r2 < 0) return OR_ERR_OOM;
        t->h_rdyn2[h] = r2;
    }
    free(hfill);
    free(hmem);
    free(hoff);

    /* per-leaf halo id; leaf members go to their own halo */
    for (int64_t a = 0; a < nleaf; a++) {
        int32_t h = hslot[uf_find(uf, (int32_t)a)];
        const or_node *L = &t->nodes[leaves[a].node];
        t->halo_id_of_leaf[leaves[a].node] = t->h_id[h];
        for (int64_t p = 0; p < L->count; p++) halo_id[t->mem[L->first + p]] = t->h_id[h];
    }
    /* inner nodes: members outside every child */
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nleaf > 0 ? nleaf : 1));
    if (!cand) return OR_ERR_OOM;
    for (int64_t i = 0; i < NN; i++) {
        const or_node *N = &t->nodes[i];
        if (N->nchild == 0) continue;
        /* leaves under N: first within [N->first, N->first + N->count) */
        int64_t lo = 0, hi = nleaf;
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (leaves[mid].first < N->first) lo = mid + 1;
            else hi = mid;
        }
        int64_t nc = 0;
        for (int64_t a = lo; a < nleaf && leaves[a].first < N->first + N->count; a++) {
            int32_t h = hslot[uf_find(uf, (int32_t)a)];
            int dup = 0;
            for (int64_t c = 0; c < nc; c++)
                if (cand[c] == h) dup = 1;
            if (!dup) cand[nc++] = h;
        }
        /* children sit at the front of N's range: the tail starts after them */
        int64_t tail = N->first + N->child_span;
        for (int64_t p = tail; p < N->first + N->count; p++) {
            int32_t pi = t->mem[p];
            if (nc == 1) {
                halo_id[pi] = t->h_id[cand[0]];
                continue;
            }
            double best = INFINITY;
            int32_t bid = INT32_MAX;
            for (int64_t c = 0; c < nc; c++) {
                int32_t h = cand[c];
                double dx2 = 0, dv2 = 0;
                for (int d = 0; d < 3; d++) {
                    double dx = min_image(t->h_xbar[3 * h + d] - (double)pos[3 * (int64_t)pi + d], box);
                    double dv = t->h_vbar[3 * h + d] - (double)vel[3 * (int64_t)pi + d];
                    dx2 += dx * dx;
                    dv2 += dv * dv;
                }
                double d2 = ratio2(dx2, t->h_rdyn2[h]) + ratio2(dv2, t->h_sigv[h] * t->h_sigv[h]);
                if (d2 < best || (d2 == best && t->h_id[h] < bid)) {
                    best = d2;
                    bid = t->h_id[h];
                }
            }
            halo_id[pi] = bid;
        }
    }
    free(cand);
    free(hslot);
    free(uf);
    free(leaves);
    *n_halos_out = nh;
    return OR_OK;
}

void or_halos_export(const or_tree *t, int32_t *id, int64_t *ncore, int32_t *nseeds, double *xbar, double *vbar,
                     double *sigv, double *rdyn2)
{
    for (int64_t h = 0; h < t->n_halos; h++) {
        id[h] = t->h_id[h];
        ncore[h] = t->h_ncore[h];
        nseeds[h] = t->h_nseeds[h];
        for (int d = 0; d < 3; d++) {
            xbar[3 * h + d] = t->h_xbar[3 * h + d];
            vbar[3 * h + d] = t->h_vbar[3 * h + d];
        }
        sigv[h] = t->h_sigv[h];
        rdyn2[h] = t->h_rdyn2[h];
    }
}

void or_leaf_halo(const or_tree *t, int32_t *out)
{
    for (int64_t i = 0; i < t->n_nodes; i++) out[i] = t->halo_id_of_leaf ? t->halo_id_of_leaf[i] : -1;
}

/* ---- halo centres and the host/subhalo relation (Sec. 3.4, 3.5.1) -------
 * After the assignment.  Centre (Sec. 3.5.1): among the nodes whose seeds
 * all belong to the halo (the halo's own part of the hierarchy), the one
 * whose Poisson error sigma_x / sqrt(n) is smallest; the halo's centre and
 * velocity are that node's mean position and velocity (reading: the paper's
 * velocity from the innermost tenth of the halo radius needs the spherical-
 * overdensity radius, which is not computed here).  Ties go to the node with
 * the smaller smallest member, then the smaller level.
 * Host (Sec. 3.4): each halo's centre is treated as a particle and measured
 * with the metric of Eq. 3 against every halo of the same 3D group with more
 * assigned particles, using that halo's centre, r_dyn,vir and sigma_v; the
 * closest is its host (ties to the smaller halo id), none means a host halo.
 * Outputs are per halo in the order of or_halos_export. */
typedef struct {
    int32_t id;
    int32_t slot;
} id_slot;

static int cmp_id_slot(const void *a, const void *b)
{
    const id_slot *x = (const id_slot *)a, *y = (const id_slot *)b;
    return (x->id > y->id) - (x->id < y->id);
}

static int32_t slot_of(const id_slot *map, int64_t H, int32_t id)
{
    int64_t lo = 0, hi = H;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (map[mid].id < id) lo = mid + 1;
        else hi = mid;
    }
    return (lo < H && map[lo].id == id) ? map[lo].slot : -1;
}

static id_slot *halo_map(const or_tree *t)
{
    const int64_t H = t->n_halos;
    id_slot *map = (id_slot *)malloc(sizeof(id_slot) * (size_t)(H > 0 ? H : 1));
    if (!map) return NULL;
    for (int64_t h = 0; h < H; h++) {
        map[h].id = t->h_id[h];
        map[h].slot = (int32_t)h;
    }
    qsort(map, (size_t)H, sizeof(id_slot), cmp_id_slot);
    return map;
}

int or_halo_props(const or_tree *t, const int32_t *halo_id, int32_t *centre_node, double *xc, double *vc,
                  int64_t *n_assigned, int32_t *host)
{
    const int64_t NN = t->n_nodes, H = t->n_halos;
    if (!t->halo_id_of_leaf) return OR_ERR_ARG; /* or_assign first */
    id_slot *map = halo_map(t);
    int32_t *pure = (int32_t *)malloc(sizeof(int32_t) * (size_t)(NN > 0 ? NN : 1));
    int32_t *group = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H > 0 ? H : 1));
    if (!map || !pure || !group) return OR_ERR_OOM;
    /* the halo whose seeds fill each node (-1: seeds of several halos);
     * children come after their parents in the node list */
    for (int64_t i = 0; i < NN; i++)
        pure[i] = t->nodes[i].nchild == 0 ? slot_of(map, H, t->halo_id_of_leaf[i]) : -2;
    for (int64_t i = NN - 1; i >= 0; i--) {
        const int32_t p = t->nodes[i].parent;
        if (p < 0) continue;
        if (pure[p] == -2) pure[p] = pure[i];
        else if (pure[p] != pure[i]) pure[p] = -1;
    }
    for (int64_t h = 0; h < H; h++) centre_node[h] = -1;
    for (int64_t i = 0; i < NN; i++) {
        const int32_t h = pure[i];
        if (h < 0) continue;
        const or_node *N = &t->nodes[i];
        const double e = N->sigx * N->sigx / (double)N->count; /* (Poisson error)^2 */
        const int32_t b = centre_node[h];
        int better = b < 0;
        if (!better) {
            const or_node *B = &t->nodes[b];
            const double eb = B->sigx * B->sigx / (double)B->count;
            better = e < eb || (e == eb && (N->minidx < B->minidx || (N->minidx == B->minidx && N->level < B->level)));
        }
        if (better) centre_node[h] = (int32_t)i;
    }
    for (int64_t h = 0; h < H; h++) {
        const or_node *N = &t->nodes[centre_node[h]];
        for (int d = 0; d < 3; d++) {
            xc[3 * h + d] = N->xbar[d];
            vc[3 * h + d] = N->vbar[d];
        }
        group[h] = N->group;
        n_assigned[h] = 0;
    }
    for (int64_t i = 0; i < t->n_total; i++)
        if (halo_id[i] >= 0) {
            const int32_t h = slot_of(map, H, halo_id[i]);
            if (h >= 0) n_assigned[h]++;
        }
    for (int64_t s2 = 0; s2 < H; s2++) {
        double best = INFINITY;
        int32_t bid = -1;
        for (int64_t h = 0; h < H; h++) {
            if (group[h] != group[s2] || n_assigned[h] <= n_assigned[s2]) continue;
            double dx2 = 0, dv2 = 0;
            for (int d = 0; d < 3; d++) {
                const double dx = min_image(xc[3 * h + d] - xc[3 * s2 + d], t->box);
                const double dv = vc[3 * h + d] - vc[3 * s2 + d];
                dx2 += dx * dx;
                dv2 += dv * dv;
            }
            const double d2 = ratio2(dx2, t->h_rdyn2[h]) + ratio2(dv2, t->h_sigv[h] * t->h_sigv[h]);
            if (d2 < best || (d2 == best && bid >= 0 && t->h_id[h] < bid)) {
                best = d2;
                bid = t->h_id[h];
            }
        }
        host[s2] = bid;
    }
    free(map);
    free(pure);
    free(group);
    return OR_OK;
}

/* ---- unbinding (Sec. 3.4, App. B) ----------------------------------------
 * Single pass.  The particles of a halo for this purpose are those assigned
 * to it or to any halo below it in the host relation (its substructure);
 * their mean velocity is the halo's bulk velocity (Sec. 3.5.1).  A particle
 * is bound to the halo when 1/2 |v - v_bulk|^2 + phi < 0 with the exact
 * potential per unit mass phi = -Gm sum_j 1 / sqrt(r^2 + eps^2) over the
 * other particles of the set (periodic minimum image; with eps = 0 a pair at
 * zero separation is left out).  The paper approximates phi with a tree to
 * 4% (App. B); this is the direct sum that bounds such an approximation.
 * Outputs per halo (order of or_halos_export): the set's size, its bound
 * count and bulk velocity; per particle: bound to its own halo's set (-1 for
 * particles outside every halo).  host holds each halo's host id or -1. */
/* The bound test on one particle set mem[0..n): bulk velocity vb (3), the
 * exact potential per unit mass of every member (phi, optional) and its
 * flag; returns the number bound. */
int64_t or_unbind_set(const float *pos, const float *vel, double box, const int32_t *mem, int64_t n, double gm,
                      double eps, double *vb, double *phi_out, int8_t *flag)
{
    const double eps2 = eps * eps;
    ksum sv[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t a = 0; a < n; a++)
        for (int d = 0; d < 3; d++) ks_add(&sv[d], (double)vel[3 * (int64_t)mem[a] + d]);
    for (int d = 0; d < 3; d++) vb[d] = n > 0 ? ks_val(&sv[d]) / (double)n : 0.0;
    int64_t nb = 0;
    for (int64_t a = 0; a < n; a++) {
        const int32_t i = mem[a];
        ksum phi = {0, 0};
        for (int64_t b = 0; b < n; b++) {
            if (b == a) continue;
            const int32_t j = mem[b];
            double r2 = 0;
            for (int d = 0; d < 3; d++) {
                const double dx = min_image((double)pos[3 * (int64_t)j + d] - (double)pos[3 * (int64_t)i + d], box);
                r2 += dx * dx;
            }
            r2 += eps2;
            if (r2 > 0) ks_add(&phi, -gm / sqrt(r2));
        }
        double ke = 0;
        for (int d = 0; d < 3; d++) {
            const double dv = (double)vel[3 * (int64_t)i + d] - vb[d];
            ke += dv * dv;
        }
        if (phi_out) phi_out[a] = ks_val(&phi);
        flag[a] = (int8_t)(0.5 * ke + ks_val(&phi) < 0);
        nb += flag[a];
    }
    return nb;
}

int or_unbind(const or_tree *t, const int32_t *halo_id, const int32_t *host, double gm, double eps, int64_t *n_part,
              int64_t *n_bound, double *vbulk, int8_t *bound_own)
{
    const int64_t H = t->n_halos, N = t->n_total;
    const float *pos = t->pos, *vel = t->vel;
    id_slot *map = halo_map(t);
    int32_t *up = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H > 0 ? H : 1));
    int64_t *off = (int64_t *)calloc((size_t)H + 1, sizeof(int64_t));
    if (!map || !up || !off) return OR_ERR_OOM;
    for (int64_t h = 0; h < H; h++) up[h] = host[h] >= 0 ? slot_of(map, H, host[h]) : -1;
    /* every particle belongs to its halo's set and to each set up the chain */
    for (int64_t i = 0; i < N; i++) {
        bound_own[i] = -1;
        if (halo_id[i] < 0) continue;
        int64_t guard = 0;
        for (int32_t h = slot_of(map, H, halo_id[i]); h >= 0 && guard <= H; h = up[h], guard++) off[h + 1]++;
        if (guard > H) return OR_ERR_ARG; /* the host relation has a cycle */
    }
    for (int64_t h = 0; h < H; h++) off[h + 1] += off[h];
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[H] > 0 ? off[H] : 1));
    int64_t *fill = (int64_t *)calloc((size_t)(H > 0 ? H : 1), sizeof(int64_t));
    if (!mem || !fill) return OR_ERR_OOM;
    for (int64_t i = 0; i < N; i++) {
        if (halo_id[i] < 0) continue;
        for (int32_t h = slot_of(map, H, halo_id[i]); h >= 0; h = up[h]) mem[off[h] + fill[h]++] = (int32_t)i;
    }
    int8_t *flags = (int8_t *)malloc((size_t)(off[H] > 0 ? off[H] : 1));
    if (!flags) return OR_ERR_OOM;
    for (int64_t h = 0; h < H; h++) {
        const int32_t *m = mem + off[h];
        const int64_t n = off[h + 1] - off[h];
        n_part[h] = n;
        n_bound[h] = or_unbind_set(pos, vel, t->box, m, n, gm, eps, vbulk + 3 * h, NULL, flags + off[h]);
        for (int64_t a = 0; a < n; a++)
            if (slot_of(map, H, halo_id[m[a]]) == (int32_t)h) bound_own[m[a]] = flags[off[h] + a];
    }
    free(flags);
    free(map);
    free(up);
    free(off);
    free(mem);
    free(fill);
    return OR_OK;
}

/* Brute-force nearest-neighbour distances and linking length of one member
 * list, exposed for the tests: dnn2[a] = min_b dist^2 (Eq. 1), returns l^2. */
double or_node_dnn(const float *pos, const float *vel, const int32_t *mem, int64_t n, double box, double f,
                   double *dnn2, double *sig_out)
{
    moments_t m;
    if (moments_of(pos, vel, mem, n, box, &m)) return NAN;
    grp_t g = {pos, vel, mem, box, m.sigx, m.sigv};
    for (int64_t a = 0; a < n; a++) {
        double best = INFINITY;
        for (int64_t b = 0; b < n; b++)
            if (b != a) {
                double d2 = gdist2(&g, (int32_t)a, (int32_t)b);
                if (d2 < best) best = d2;
            }
        dnn2[a] = best;
    }
    if (sig_out) {
        sig_out[0] = m.sigx;
        sig_out[1] = m.sigv;
        for (int d = 0; d < 3; d++) {
            sig_out[2 + d] = m.xbar[d];
            sig_out[5 + d] = m.vbar[d];
        }
    }
    int64_t k = (int64_t)ceil(f * (double)n);
    if (k < 1) k = 1;
    if (k > n) k = n;
    double *srt = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(srt, dnn2, sizeof(double) * (size_t)n);
    qsort(srt, (size_t)n, sizeof(double), cmp_f64);
    double l2 = srt[k - 1];
    free(srt);
    return l2;
}
