/*
 * FP64 CPU oracle for the tree side of the P3T scheme (Iwasawa, Portegies
 * Zwart & Makino, arXiv:1506.04553).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it; the
 * library itself never does.  It shares no source, header, table or helper
 * with the CUDA path.
 *
 * Everything here is deliberately plain: loops over particles in the order the
 * definitions are written, FP64 arithmetic, no blocking or reordering beyond
 * what a definition states.  It is compiled with -ffp-contract=off so that
 * every float/double expression is evaluated exactly as written (IEEE
 * round-to-nearest, one rounding per operation).
 *
 * What follows the paper, and where:
 *   - cut-off function K(x) ............ Eq. 12-15 (Sect. 2.1)
 *   - transition function W(y; gamma) .. Eq. 16-17, with the sign of G's
 *                                         numerator reversed (the printed sign
 *                                         violates Eq. 9; see orc_W)
 *   - soft / hard / Newtonian forces ... Eq. 7-9 with the softened distance of
 *                                         Eq. 2-3
 *   - soft potential ................... Eq. 6
 *   - Barnes-Hut tree to quadrupole .... Sect. 2.2 (tree for F_soft on all
 *                                         particles, up to the quadrupole)
 *   - neighbour list within h .......... Sect. 2.2 (list of particles within
 *                                         distance h of each particle)
 *   - velocity kick / drift ............ Eq. 11 and the step procedure of
 *                                         Sect. 2.2 (half kicks by F_soft,
 *                                         drift r <- r + dt v)
 * Items the paper leaves unstated (key quantisation, leaf and group rules,
 * the opening test, the quadrupole convention) follow one fixed reading that
 * is written out at each function.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LEVEL 21

/* ------------------------------------------------------------------------ */
/* Cut-off function and transition function (Sect. 2.1)                     */
/* ------------------------------------------------------------------------ */

/* Eq. 12: K(x) = 0 for x < 0, -20x^7 + 70x^6 - 84x^5 + 35x^4 on [0, 1),
 * 1 for x >= 1. */
double orc_K(double x)
{
    if (x < 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    double x2 = x * x;
    double x3 = x2 * x;
    double x4 = x2 * x2;
    double x5 = x4 * x;
    double x6 = x3 * x3;
    double x7 = x6 * x;
    return -20.0 * x7 + 70.0 * x6 - 84.0 * x5 + 35.0 * x4;
}

/* dK/dx of Eq. 12 (used by the analytic gradient). */
double orc_dKdx(double x)
{
    if (x <= 0.0 || x >= 1.0) return 0.0;
    double x2 = x * x;
    double x3 = x2 * x;
    double x4 = x2 * x2;
    double x5 = x4 * x;
    double x6 = x3 * x3;
    return -140.0 * x6 + 420.0 * x5 - 420.0 * x4 + 140.0 * x3;
}

/* Eq. 13-15: K as a function of the softened distance s, with y = s/r_cut,
 * x = (y - gamma)/(1 - gamma). */
double orc_K_of_s(double s, double r_cut, double gamma)
{
    double y = s / r_cut;
    double x = (y - gamma) / (1.0 - gamma);
    return orc_K(x);
}

/* Eq. 17 as printed, G_printed(y; gamma). */
static double orc_G_printed(double y, double g)
{
    double g2 = g * g, g3 = g2 * g, g4 = g3 * g, g5 = g4 * g, g6 = g5 * g,
           g7 = g6 * g;
    double y2 = y * y, y3 = y2 * y, y4 = y3 * y, y5 = y4 * y, y6 = y5 * y,
           y7 = y6 * y;
    double num = (-10.0 / 3.0) * y7
               + 14.0 * (g + 1.0) * y6
               - 21.0 * (g2 + 3.0 * g + 1.0) * y5
               + (35.0 * (g3 + 9.0 * g2 + 9.0 * g + 1.0) / 3.0) * y4
               - 70.0 * (g3 + 3.0 * g2 + g) * y3
               + 210.0 * (g3 + g2) * y2
               - 140.0 * g3 * y * log(y)
               + (g7 - 7.0 * g6 + 21.0 * g5 - 35.0 * g4);
    double d = 1.0 - g;
    double d7 = d * d * d * d * d * d * d;
    return num / d7;
}

/* Slope of W below r_in (first branch of Eq. 16). */
double orc_W_inner_slope(double g)
{
    double g2 = g * g, g3 = g2 * g, g4 = g3 * g, g5 = g4 * g, g6 = g5 * g;
    double gm1 = g - 1.0;
    double gm17 = gm1 * gm1 * gm1 * gm1 * gm1 * gm1 * gm1;
    return 7.0 * (g6 - 9.0 * g5 + 45.0 * g4 - 60.0 * g3 * log(g) - 45.0 * g2
                  + 9.0 * g - 1.0)
           / (3.0 * gm17);
}

/* Eq. 16: the potential transition function W(y; gamma).
 * Reading: the middle branch uses G = -G_printed.  With the printed sign,
 * W - y dW/dy differs from K by O(1) on (gamma, 1) and W jumps at y = gamma,
 * contradicting Eq. 9; with the numerator's sign reversed Eq. 9 holds and W
 * is continuous at y = gamma and y = 1. */
double orc_W(double y, double g)
{
    if (y >= 1.0) return 1.0;
    if (y < g) return orc_W_inner_slope(g) * y;
    double G1 = -orc_G_printed(1.0, g);
    return -orc_G_printed(y, g) + (1.0 - G1) * y;
}

/* W(s/r_cut)/s, the soft pair potential per unit G m_i m_j (Eq. 6), with its
 * finite limit inside r_in where W is linear in y. */
static double orc_W_over_s(double s, double r_cut, double g)
{
    double y = s / r_cut;
    if (y < g) return orc_W_inner_slope(g) / r_cut;
    return orc_W(y, g) / s;
}

/* ------------------------------------------------------------------------ */
/* A plain parallel-for over index ranges (used only to make the oracle     */
/* finish in reasonable time; each index is computed independently).        */
/* ------------------------------------------------------------------------ */

typedef void (*orc_range_fn)(void *arg, int64_t lo, int64_t hi);

typedef struct {
    orc_range_fn fn;
    void *arg;
    int64_t lo, hi;
} orc_job;

static void *orc_job_main(void *p)
{
    orc_job *j = (orc_job *)p;
    j->fn(j->arg, j->lo, j->hi);
    return NULL;
}

static void orc_parallel_for(int64_t n, int nthreads, orc_range_fn fn,
                             void *arg)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 2 * nthreads || nthreads == 1) {
        fn(arg, 0, n);
        return;
    }
    pthread_t th[256];
    orc_job jobs[256];
    /* interleave work in small chunks so uneven per-index costs balance */
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].arg = arg;
        jobs[t].lo = (n * t) / nthreads;
        jobs[t].hi = (n * (t + 1)) / nthreads;
        pthread_create(&th[t], NULL, orc_job_main, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Direct summation (the plain definition of Eq. 7-9 and Eq. 6)             */
/* ------------------------------------------------------------------------ */

enum { ORC_SOFT = 0, ORC_HARD = 1, ORC_NEWTON = 2 };

typedef struct {
    int64_t n;
    const double *pos; /* n x 3, row-major */
    const double *m;
    double G, gamma;
    double eps[3], r_cut[3]; /* per pair type (see orc_direct_species) */
    int64_t n_fs;
    int kind;
    double *acc; /* n x 3 */
    double *pot; /* n or NULL */
    const int64_t *rows; /* NULL: all i; else the i to evaluate */
} orc_direct_args;

/* Pair weight for the force (Eq. 7 hard: 1-K, Eq. 8 soft: K, Newton: 1). */
static double orc_force_weight(int kind, double s, double r_cut, double g)
{
    if (kind == ORC_NEWTON) return 1.0;
    double K = orc_K_of_s(s, r_cut, g);
    return kind == ORC_SOFT ? K : 1.0 - K;
}

/* Pair potential per unit G m_j: soft W/s (Eq. 6), hard (1-W)/s (Eq. 5). */
static double orc_pot_weight(int kind, double s, double r_cut, double g)
{
    if (kind == ORC_NEWTON) return 1.0 / s;
    double wos = orc_W_over_s(s, r_cut, g);
    return kind == ORC_SOFT ? wos : 1.0 / s - wos;
}

static void orc_direct_range(void *p, int64_t lo, int64_t hi)
{
    orc_direct_args *a = (orc_direct_args *)p;
    for (int64_t r = lo; r < hi; ++r) {
        int64_t i = a->rows ? a->rows[r] : r;
        double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
        for (int64_t j = 0; j < a->n; ++j) {
            if (j == i) continue;
            const int t = (i >= a->n_fs) + (j >= a->n_fs);
            const double eps2 = a->eps[t] * a->eps[t], r_cut = a->r_cut[t];
            /* q_ij = q_i - q_j (Eq. 3), s_ij = sqrt(|q_ij|^2 + eps^2) (Eq. 2) */
            double qx = a->pos[3 * i + 0] - a->pos[3 * j + 0];
            double qy = a->pos[3 * i + 1] - a->pos[3 * j + 1];
            double qz = a->pos[3 * i + 2] - a->pos[3 * j + 2];
            double s2 = qx * qx + qy * qy + qz * qz + eps2;
            double s = sqrt(s2);
            double w = orc_force_weight(a->kind, s, r_cut, a->gamma);
            if (w != 0.0) {
                /* acceleration of i: F_i / m_i = -G m_j w q_ij / s^3 */
                double f = -a->G * a->m[j] * w / (s2 * s);
                ax += f * qx;
                ay += f * qy;
                az += f * qz;
            }
            if (a->pot) ph -= a->G * a->m[j]
                              * orc_pot_weight(a->kind, s, r_cut, a->gamma);
        }
        a->acc[3 * r + 0] = ax;
        a->acc[3 * r + 1] = ay;
        a->acc[3 * r + 2] = az;
        if (a->pot) a->pot[r] = ph;
    }
}

/* Acceleration (and optionally potential) by direct summation over all
 * j != i.  rows == NULL evaluates every particle; otherwise only rows[0..nr)
 * and the outputs are indexed by position in rows. */
void orc_direct(int64_t n, const double *pos, const double *m, double G,
                double eps, double r_cut, double gamma, int kind,
                const int64_t *rows, int64_t nr, double *acc, double *pot,
                int nthreads)
{
    orc_direct_args a = {n, pos, m, G, gamma, {eps, eps, eps},
                         {r_cut, r_cut, r_cut}, INT64_MAX, kind, acc, pot,
                         rows};
    orc_parallel_for(rows ? nr : n, nthreads, orc_direct_range, &a);
}

/* The same with two species (Sect. 3.2.2): the last n_bh particles are black
 * holes, and a pair of type t (0 star-star, 1 black hole-star, 2 black
 * hole-black hole) takes eps[t] and r_cut[t].  r_cut = infinity means the
 * force is not split: K = 0, all of it hard (the black hole pair). */
void orc_direct_species(int64_t n, int64_t n_bh, const double *pos,
                        const double *m, double G, const double *eps,
                        const double *r_cut, double gamma, int kind,
                        const int64_t *rows, int64_t nr, double *acc,
                        double *pot, int nthreads)
{
    orc_direct_args a = {n, pos, m, G, gamma, {eps[0], eps[1], eps[2]},
                         {r_cut[0], r_cut[1], r_cut[2]}, n - n_bh, kind, acc,
                         pot, rows};
    orc_parallel_for(rows ? nr : n, nthreads, orc_direct_range, &a);
}

/* ------------------------------------------------------------------------ */
/* Neighbour lists by brute force (Sect. 2.2: particles within distance h)  */
/* Predicate: j != i and ((dx*dx + dy*dy) + dz*dz) < h*h in FP64, with      */
/* dx = x_i - x_j; the unsoftened distance, strict inequality.              */
/* ------------------------------------------------------------------------ */

int orc_is_neighbour(const double *pi, const double *pj, double h)
{
    double dx = pi[0] - pj[0];
    double dy = pi[1] - pj[1];
    double dz = pi[2] - pj[2];
    double r2 = (dx * dx + dy * dy) + dz * dz;
    return r2 < h * h;
}

typedef struct {
    int64_t n;
    const double *pos;
    double h[3];  /* per pair type */
    int64_t n_fs;
    const int64_t *rows;
    int64_t *count; /* per row */
    const int64_t *offsets; /* NULL in the counting pass */
    int32_t *idx;
} orc_ngb_args;

static void orc_ngb_range(void *p, int64_t lo, int64_t hi)
{
    orc_ngb_args *a = (orc_ngb_args *)p;
    for (int64_t r = lo; r < hi; ++r) {
        int64_t i = a->rows ? a->rows[r] : r;
        int64_t c = 0;
        for (int64_t j = 0; j < a->n; ++j) {
            if (j == i) continue;
            const int t = (i >= a->n_fs) + (j >= a->n_fs);
            if (orc_is_neighbour(a->pos + 3 * i, a->pos + 3 * j, a->h[t])) {
                if (a->offsets) a->idx[a->offsets[r] + c] = (int32_t)j;
                ++c;
            }
        }
        a->count[r] = c;
    }
}

/* Counting pass: count[r] = number of neighbours of row r. */
void orc_neighbours_count(int64_t n, const double *pos, double h,
                          const int64_t *rows, int64_t nr, int64_t *count,
                          int nthreads)
{
    orc_ngb_args a = {n, pos, {h, h, h}, INT64_MAX, rows, count, NULL, NULL};
    orc_parallel_for(rows ? nr : n, nthreads, orc_ngb_range, &a);
}

/* Filling pass: indices of row r (ascending j) at idx[offsets[r] ...]. */
void orc_neighbours_fill(int64_t n, const double *pos, double h,
                         const int64_t *rows, int64_t nr,
                         const int64_t *offsets, int32_t *idx, int64_t *count,
                         int nthreads)
{
    orc_ngb_args a = {n, pos, {h, h, h}, INT64_MAX, rows, count, offsets, idx};
    orc_parallel_for(rows ? nr : n, nthreads, orc_ngb_range, &a);
}

/* Both passes with two species (Sect. 3.2.2): the last n_bh particles are
 * black holes and a pair of type t (0 star-star, 1 black hole-star, 2 black
 * hole-black hole) is a neighbour pair within h[t]; h = infinity makes every
 * such pair one (the black holes, whose force is not split).  rows == NULL
 * takes every particle, else rows[0..nr) (outputs by position in rows).
 * offsets == NULL counts, else fills. */
void orc_neighbours_species(int64_t n, int64_t n_bh, const double *pos,
                            const double *h, const int64_t *rows, int64_t nr,
                            const int64_t *offsets, int32_t *idx,
                            int64_t *count, int nthreads)
{
    orc_ngb_args a = {n, pos, {h[0], h[1], h[2]}, n - n_bh, rows, count,
                      offsets, idx};
    orc_parallel_for(rows ? nr : n, nthreads, orc_ngb_range, &a);
}

/* ------------------------------------------------------------------------ */
/* Leapfrog pieces (Eq. 11; Sect. 2.2 steps: kick by F_soft for dt/2,       */
/* drift r <- r + dt v)                                                     */
/* ------------------------------------------------------------------------ */

void orc_kick(int64_t n3, double *v, const float *a, double dt_half)
{
    for (int64_t k = 0; k < n3; ++k) v[k] = v[k] + dt_half * (double)a[k];
}

void orc_drift(int64_t n3, double *x, const double *v, double dt)
{
    for (int64_t k = 0; k < n3; ++k) x[k] = x[k] + dt * v[k];
}

/* ------------------------------------------------------------------------ */
/* Barnes-Hut octree to quadrupole order (Sect. 2.2)                        */
/* ------------------------------------------------------------------------ */

typedef struct orc_tree {
    int64_t n;
    int n_leaf, n_group;
    double lo[3], size;
    uint64_t *key;   /* keys in sorted order */
    int64_t *order;  /* order[k] = original index of the k-th sorted particle */
    double *x;       /* sorted positions, n x 3 */
    double *m;       /* sorted masses */
    /* cells, in breadth-first order; children of a cell are contiguous and
     * in Morton (digit) order */
    int64_t ncell, cap_cell;
    int32_t *level;
    int64_t *first, *count, *parent, *child_first;
    int32_t *nchild;
    double *M, *com, *Q;   /* Q: xx, yy, zz, xy, xz, yz */
    double *bmin, *bmax;   /* member bounding box, FP64 */
    float *fmin, *fmax;    /* the same box rounded outward to FP32 */
    /* groups (i-particle sets sharing one interaction list) */
    int64_t ngroup, cap_group;
    int64_t *g_first, *g_count;
    float *g_fmin, *g_fmax;
    /* interaction lists, filled by orc_tree_walk */
    int walked;
    int64_t *pc_off, *ppn_off, *ppf_off; /* ngroup + 1 */
    int64_t *pc, *ppn, *ppf;             /* cell ids / sorted particle ids */
} orc_tree;

/* Level-L Morton digit (L = 1..21): three bits, x highest. */
static int orc_digit(uint64_t key, int L)
{
    return (int)((key >> (3 * (ORC_MAX_LEVEL - L))) & 7u);
}

/* Quantised integer coordinate along one axis: floor((x - lo)/size * 2^21),
 * clamped to [0, 2^21 - 1], each operation rounded once in FP64. */
static int64_t orc_quantise(double x, double lo, double size)
{
    double t = x - lo;
    double u = t / size;
    double v = u * 2097152.0;
    int64_t q = (int64_t)floor(v);
    if (q < 0) q = 0;
    if (q > 2097151) q = 2097151;
    return q;
}

/* 63-bit Morton key: for bit b = 20..0 the triple (x_b, y_b, z_b), x highest. */
uint64_t orc_morton_key(double x, double y, double z, const double *lo,
                        double size)
{
    int64_t q[3] = {orc_quantise(x, lo[0], size), orc_quantise(y, lo[1], size),
                    orc_quantise(z, lo[2], size)};
    uint64_t key = 0;
    for (int b = ORC_MAX_LEVEL - 1; b >= 0; --b) {
        key = (key << 3) | ((uint64_t)((q[0] >> b) & 1) << 2)
              | ((uint64_t)((q[1] >> b) & 1) << 1) | (uint64_t)((q[2] >> b) & 1);
    }
    return key;
}

/* Root cube: lo = componentwise minimum; ext = largest extent; size =
 * ext * (1 + 2^-20) so the cube strictly encloses every particle; size = 1
 * when all particles coincide. */
void orc_root_box(int64_t n, const double *pos, double *lo, double *size)
{
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = pos[a];
        mx[a] = pos[a];
    }
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (pos[3 * i + a] < mn[a]) mn[a] = pos[3 * i + a];
            if (pos[3 * i + a] > mx[a]) mx[a] = pos[3 * i + a];
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = mx[a] - mn[a];
        if (e > ext) ext = e;
        lo[a] = mn[a];
    }
    *size = (ext == 0.0) ? 1.0 : ext * (1.0 + 0x1p-20);
}

/* FP64 -> FP32 rounded toward -inf / +inf. */
static float orc_round_down(double v)
{
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return f;
}
static float orc_round_up(double v)
{
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}

typedef struct {
    uint64_t key;
    int64_t idx;
} orc_kv;

static int orc_kv_cmp(const void *a, const void *b)
{
    const orc_kv *p = (const orc_kv *)a, *q = (const orc_kv *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
    return 0;
}

static void orc_cell_reserve(orc_tree *t)
{
    if (t->ncell < t->cap_cell) return;
    int64_t c = t->cap_cell ? 2 * t->cap_cell : 1024;
    t->level = realloc(t->level, c * sizeof(int32_t));
    t->first = realloc(t->first, c * sizeof(int64_t));
    t->count = realloc(t->count, c * sizeof(int64_t));
    t->parent = realloc(t->parent, c * sizeof(int64_t));
    t->child_first = realloc(t->child_first, c * sizeof(int64_t));
    t->nchild = realloc(t->nchild, c * sizeof(int32_t));
    t->cap_cell = c;
}

static int64_t orc_cell_add(orc_tree *t, int level, int64_t first,
                            int64_t count, int64_t parent)
{
    orc_cell_reserve(t);
    int64_t c = t->ncell++;
    t->level[c] = level;
    t->first[c] = first;
    t->count[c] = count;
    t->parent[c] = parent;
    t->child_first[c] = -1;
    t->nchild[c] = 0;
    return c;
}

/* Multipole moments of a cell directly from its member particles:
 * M = sum m, com = sum m x / M, Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab)
 * with d = x - com (traceless quadrupole about the centre of mass). */
static void orc_cell_moments(orc_tree *t, int64_t c)
{
    int64_t f = t->first[c], n = t->count[c];
    double M = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    for (int64_t k = f; k < f + n; ++k) {
        M += t->m[k];
        cx += t->m[k] * t->x[3 * k + 0];
        cy += t->m[k] * t->x[3 * k + 1];
        cz += t->m[k] * t->x[3 * k + 2];
    }
    cx /= M;
    cy /= M;
    cz /= M;
    double Q[6] = {0, 0, 0, 0, 0, 0};
    double bmn[3], bmx[3];
    for (int a = 0; a < 3; ++a) {
        bmn[a] = t->x[3 * f + a];
        bmx[a] = t->x[3 * f + a];
    }
    for (int64_t k = f; k < f + n; ++k) {
        double dx = t->x[3 * k + 0] - cx;
        double dy = t->x[3 * k + 1] - cy;
        double dz = t->x[3 * k + 2] - cz;
        double d2 = dx * dx + dy * dy + dz * dz;
        double mk = t->m[k];
        Q[0] += mk * (3.0 * dx * dx - d2);
        Q[1] += mk * (3.0 * dy * dy - d2);
        Q[2] += mk * (3.0 * dz * dz - d2);
        Q[3] += mk * (3.0 * dx * dy);
        Q[4] += mk * (3.0 * dx * dz);
        Q[5] += mk * (3.0 * dy * dz);
        for (int a = 0; a < 3; ++a) {
            if (t->x[3 * k + a] < bmn[a]) bmn[a] = t->x[3 * k + a];
            if (t->x[3 * k + a] > bmx[a]) bmx[a] = t->x[3 * k + a];
        }
    }
    t->M[c] = M;
    t->com[3 * c + 0] = cx;
    t->com[3 * c + 1] = cy;
    t->com[3 * c + 2] = cz;
    for (int q = 0; q < 6; ++q) t->Q[6 * c + q] = Q[q];
    for (int a = 0; a < 3; ++a) {
        t->bmin[3 * c + a] = bmn[a];
        t->bmax[3 * c + a] = bmx[a];
        t->fmin[3 * c + a] = orc_round_down(bmn[a]);
        t->fmax[3 * c + a] = orc_round_up(bmx[a]);
    }
}

static int orc_is_leaf(const orc_tree *t, int64_t c)
{
    return t->nchild[c] == 0;
}

static void orc_group_add(orc_tree *t, int64_t first, int64_t count)
{
    if (t->ngroup == t->cap_group) {
        int64_t c = t->cap_group ? 2 * t->cap_group : 1024;
        t->g_first = realloc(t->g_first, c * sizeof(int64_t));
        t->g_count = realloc(t->g_count, c * sizeof(int64_t));
        t->cap_group = c;
    }
    t->g_first[t->ngroup] = first;
    t->g_count[t->ngroup] = count;
    t->ngroup++;
}

/* A range larger than n_group is cut into consecutive chunks of n_group. */
static void orc_group_add_chunked(orc_tree *t, int64_t first, int64_t count)
{
    for (int64_t k = 0; k < count; k += t->n_group) {
        int64_t c = count - k < t->n_group ? count - k : t->n_group;
        orc_group_add(t, first + k, c);
    }
}

/* Groups.  A container is a cell holding at most 16 n_group particles whose
 * parent holds more (or a leaf whose parent holds more, or the root if it
 * qualifies); the particles of each container are cut into consecutive
 * chunks of n_group in Morton order, the last one partial.  Containers are
 * visited depth first in Morton order. */
static void orc_groups_below(orc_tree *t, int64_t c)
{
    const int64_t cap = 16 * (int64_t)t->n_group;
    if (t->count[c] <= cap || orc_is_leaf(t, c)) {
        orc_group_add_chunked(t, t->first[c], t->count[c]);
        return;
    }
    for (int k = 0; k < t->nchild[c]; ++k)
        orc_groups_below(t, t->child_first[c] + k);
}

/* Build the tree for n particles (pos n x 3 row-major, masses m > 0).
 * Steps: root cube, Morton keys, sort by (key, original index), split every
 * cell holding more than n_leaf particles (and above level 21) into its
 * non-empty octants, moments per cell, groups (chunks of n_group inside
 * cells of at most 16 n_group particles). */
orc_tree *orc_tree_build(int64_t n, const double *pos, const double *m,
                         int n_leaf, int n_group)
{
    orc_tree *t = calloc(1, sizeof(orc_tree));
    t->n = n;
    t->n_leaf = n_leaf;
    t->n_group = n_group;
    if (n <= 0) return t;
    orc_root_box(n, pos, t->lo, &t->size);

    orc_kv *kv = malloc(n * sizeof(orc_kv));
    for (int64_t i = 0; i < n; ++i) {
        kv[i].key = orc_morton_key(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2],
                                   t->lo, t->size);
        kv[i].idx = i;
    }
    qsort(kv, n, sizeof(orc_kv), orc_kv_cmp);
    t->key = malloc(n * sizeof(uint64_t));
    t->order = malloc(n * sizeof(int64_t));
    t->x = malloc(3 * n * sizeof(double));
    t->m = malloc(n * sizeof(double));
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = kv[k].idx;
        t->key[k] = kv[k].key;
        t->order[k] = i;
        for (int a = 0; a < 3; ++a) t->x[3 * k + a] = pos[3 * i + a];
        t->m[k] = m[i];
    }
    free(kv);

    /* breadth-first split */
    orc_cell_add(t, 0, 0, n, -1);
    for (int64_t c = 0; c < t->ncell; ++c) {
        if (t->count[c] <= n_leaf || t->level[c] >= ORC_MAX_LEVEL) continue;
        int L = t->level[c] + 1;
        int64_t f = t->first[c], e = f + t->count[c];
        int64_t start = f;
        t->child_first[c] = t->ncell;
        while (start < e) {
            int d = orc_digit(t->key[start], L);
            int64_t stop = start;
            while (stop < e && orc_digit(t->key[stop], L) == d) ++stop;
            orc_cell_add(t, L, start, stop - start, c);
            t->nchild[c]++;
            start = stop;
        }
    }

    int64_t C = t->ncell;
    t->M = malloc(C * sizeof(double));
    t->com = malloc(3 * C * sizeof(double));
    t->Q = malloc(6 * C * sizeof(double));
    t->bmin = malloc(3 * C * sizeof(double));
    t->bmax = malloc(3 * C * sizeof(double));
    t->fmin = malloc(3 * C * sizeof(float));
    t->fmax = malloc(3 * C * sizeof(float));
    for (int64_t c = 0; c < C; ++c) orc_cell_moments(t, c);

    orc_groups_below(t, 0);
    t->g_fmin = malloc(3 * t->ngroup * sizeof(float));
    t->g_fmax = malloc(3 * t->ngroup * sizeof(float));
    for (int64_t g = 0; g < t->ngroup; ++g) {
        int64_t f = t->g_first[g];
        for (int a = 0; a < 3; ++a) {
            double mn = t->x[3 * f + a], mx = t->x[3 * f + a];
            for (int64_t k = f; k < f + t->g_count[g]; ++k) {
                if (t->x[3 * k + a] < mn) mn = t->x[3 * k + a];
                if (t->x[3 * k + a] > mx) mx = t->x[3 * k + a];
            }
            t->g_fmin[3 * g + a] = orc_round_down(mn);
            t->g_fmax[3 * g + a] = orc_round_up(mx);
        }
    }
    return t;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    void *ptrs[] = {t->key, t->order, t->x, t->m, t->level, t->first,
                    t->count, t->parent, t->child_first, t->nchild, t->M,
                    t->com, t->Q, t->bmin, t->bmax, t->fmin, t->fmax,
                    t->g_first, t->g_count, t->g_fmin, t->g_fmax, t->pc_off,
                    t->ppn_off, t->ppf_off, t->pc, t->ppn, t->ppf};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(t);
}

/* ---- accessors for the Python side ---- */
int64_t orc_tree_n(const orc_tree *t) { return t->n; }
int64_t orc_tree_ncell(const orc_tree *t) { return t->ncell; }
int64_t orc_tree_ngroup(const orc_tree *t) { return t->ngroup; }
void orc_tree_root(const orc_tree *t, double *lo3, double *size)
{
    for (int a = 0; a < 3; ++a) lo3[a] = t->lo[a];
    *size = t->size;
}
void orc_tree_particles(const orc_tree *t, uint64_t *key, int64_t *order)
{
    memcpy(key, t->key, t->n * sizeof(uint64_t));
    memcpy(order, t->order, t->n * sizeof(int64_t));
}
void orc_tree_cells(const orc_tree *t, int32_t *level, int64_t *first,
                    int64_t *count, int64_t *parent, int64_t *child_first,
                    int32_t *nchild, double *M, double *com, double *Q,
                    float *fmin, float *fmax)
{
    int64_t C = t->ncell;
    memcpy(level, t->level, C * sizeof(int32_t));
    memcpy(first, t->first, C * sizeof(int64_t));
    memcpy(count, t->count, C * sizeof(int64_t));
    memcpy(parent, t->parent, C * sizeof(int64_t));
    memcpy(child_first, t->child_first, C * sizeof(int64_t));
    memcpy(nchild, t->nchild, C * sizeof(int32_t));
    memcpy(M, t->M, C * sizeof(double));
    memcpy(com, t->com, 3 * C * sizeof(double));
    memcpy(Q, t->Q, 6 * C * sizeof(double));
    memcpy(fmin, t->fmin, 3 * C * sizeof(float));
    memcpy(fmax, t->fmax, 3 * C * sizeof(float));
}
void orc_tree_groups(const orc_tree *t, int64_t *first, int64_t *count,
                     float *fmin, float *fmax)
{
    memcpy(first, t->g_first, t->ngroup * sizeof(int64_t));
    memcpy(count, t->g_count, t->ngroup * sizeof(int64_t));
    memcpy(fmin, t->g_fmin, 3 * t->ngroup * sizeof(float));
    memcpy(fmax, t->g_fmax, 3 * t->ngroup * sizeof(float));
}

/* ---- the opening test (paper: "opening criterion theta"; form unstated) ----
 * Reading used here.  For group box B_g and cell member box B_c (both the
 * FP64 boxes rounded outward to FP32), with all arithmetic in FP32, one
 * rounding per operation, in this order:
 *   gap_a = max(max(cmin_a - gmax_a, gmin_a - cmax_a), 0)
 *   d2    = (gap_x*gap_x + gap_y*gap_y) + gap_z*gap_z
 *   l     = max(max(cmax_x - cmin_x, cmax_y - cmin_y), cmax_z - cmin_z)
 *   accept  <=>  l*l < theta2*d2  and  d2 > hg2
 * with theta2 = fl(theta)*fl(theta) and hg2 = (hg*hg)*(1 + 2^-10),
 * hg = fl(max(h, r_cut)).  The second clause keeps every pair closer than
 * max(h, r_cut) out of the cell list, so cells are evaluated with K = 1 and
 * every neighbour candidate is met particle by particle. */
typedef struct {
    float theta2, hg2;
} orc_mac;

static orc_mac orc_mac_make(double theta, double h, double r_cut)
{
    orc_mac k;
    float th = (float)theta;
    k.theta2 = th * th;
    float hg = (float)(h > r_cut ? h : r_cut);
    float hh = hg * hg;
    k.hg2 = hh * 1.0009765625f;
    return k;
}

static float orc_box_d2(const float *gmin, const float *gmax,
                        const float *cmin, const float *cmax)
{
    float gap[3];
    for (int a = 0; a < 3; ++a) {
        float u = cmin[a] - gmax[a];
        float v = gmin[a] - cmax[a];
        float w = fmaxf(u, v);
        gap[a] = fmaxf(w, 0.0f);
    }
    float gx2 = gap[0] * gap[0];
    float gy2 = gap[1] * gap[1];
    float gz2 = gap[2] * gap[2];
    float s = gx2 + gy2;
    return s + gz2;
}

static float orc_box_side(const float *cmin, const float *cmax)
{
    float lx = cmax[0] - cmin[0];
    float ly = cmax[1] - cmin[1];
    float lz = cmax[2] - cmin[2];
    return fmaxf(fmaxf(lx, ly), lz);
}

/* growable int64 list */
typedef struct {
    int64_t *v;
    int64_t n, cap;
} orc_vec;
static void orc_vec_push(orc_vec *a, int64_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 256;
        a->v = realloc(a->v, a->cap * sizeof(int64_t));
    }
    a->v[a->n++] = x;
}

/* Visit cell c for group g: accepted -> cell list; a leaf that is not
 * accepted -> its particles go to the near list (d2 <= hg2) or the far list;
 * otherwise descend into the children. */
static void orc_visit(const orc_tree *t, int64_t g, int64_t c, orc_mac mac,
                      orc_vec *pc, orc_vec *ppn, orc_vec *ppf)
{
    const float *gmin = t->g_fmin + 3 * g, *gmax = t->g_fmax + 3 * g;
    const float *cmin = t->fmin + 3 * c, *cmax = t->fmax + 3 * c;
    float d2 = orc_box_d2(gmin, gmax, cmin, cmax);
    float l = orc_box_side(cmin, cmax);
    float ll = l * l;
    float td = mac.theta2 * d2;
    if (ll < td && d2 > mac.hg2) {
        orc_vec_push(pc, c);
        return;
    }
    if (orc_is_leaf(t, c)) {
        orc_vec *dst = (d2 <= mac.hg2) ? ppn : ppf;
        for (int64_t k = t->first[c]; k < t->first[c] + t->count[c]; ++k)
            orc_vec_push(dst, k);
        return;
    }
    for (int k = 0; k < t->nchild[c]; ++k)
        orc_visit(t, g, t->child_first[c] + k, mac, pc, ppn, ppf);
}

typedef struct {
    const orc_tree *t;
    orc_mac mac;
    orc_vec *pc, *ppn, *ppf;
} orc_walk_args;

static void orc_walk_range(void *p, int64_t lo, int64_t hi)
{
    orc_walk_args *a = (orc_walk_args *)p;
    for (int64_t g = lo; g < hi; ++g)
        orc_visit(a->t, g, 0, a->mac, &a->pc[g], &a->ppn[g], &a->ppf[g]);
}

/* Interaction lists of every group.  Returns total sizes through out3
 * (cells, near particles, far particles). */
void orc_tree_walk(orc_tree *t, double theta, double h, double r_cut,
                   int nthreads, int64_t *out3)
{
    int64_t G = t->ngroup;
    orc_walk_args a;
    a.t = t;
    a.mac = orc_mac_make(theta, h, r_cut);
    a.pc = calloc(G ? G : 1, sizeof(orc_vec));
    a.ppn = calloc(G ? G : 1, sizeof(orc_vec));
    a.ppf = calloc(G ? G : 1, sizeof(orc_vec));
    orc_parallel_for(G, nthreads, orc_walk_range, &a);
    free(t->pc_off); free(t->ppn_off); free(t->ppf_off);
    free(t->pc); free(t->ppn); free(t->ppf);
    t->pc_off = calloc(G + 1, sizeof(int64_t));
    t->ppn_off = calloc(G + 1, sizeof(int64_t));
    t->ppf_off = calloc(G + 1, sizeof(int64_t));
    for (int64_t g = 0; g < G; ++g) {
        t->pc_off[g + 1] = t->pc_off[g] + a.pc[g].n;
        t->ppn_off[g + 1] = t->ppn_off[g] + a.ppn[g].n;
        t->ppf_off[g + 1] = t->ppf_off[g] + a.ppf[g].n;
    }
    t->pc = malloc((t->pc_off[G] + 1) * sizeof(int64_t));
    t->ppn = malloc((t->ppn_off[G] + 1) * sizeof(int64_t));
    t->ppf = malloc((t->ppf_off[G] + 1) * sizeof(int64_t));
    for (int64_t g = 0; g < G; ++g) {
        if (a.pc[g].n)
            memcpy(t->pc + t->pc_off[g], a.pc[g].v, a.pc[g].n * sizeof(int64_t));
        if (a.ppn[g].n)
            memcpy(t->ppn + t->ppn_off[g], a.ppn[g].v,
                   a.ppn[g].n * sizeof(int64_t));
        if (a.ppf[g].n)
            memcpy(t->ppf + t->ppf_off[g], a.ppf[g].v,
                   a.ppf[g].n * sizeof(int64_t));
        free(a.pc[g].v);
        free(a.ppn[g].v);
        free(a.ppf[g].v);
    }
    free(a.pc);
    free(a.ppn);
    free(a.ppf);
    t->walked = 1;
    out3[0] = t->pc_off[G];
    out3[1] = t->ppn_off[G];
    out3[2] = t->ppf_off[G];
}

void orc_tree_lists(const orc_tree *t, int64_t *pc_off, int64_t *pc,
                    int64_t *ppn_off, int64_t *ppn, int64_t *ppf_off,
                    int64_t *ppf)
{
    int64_t G = t->ngroup;
    memcpy(pc_off, t->pc_off, (G + 1) * sizeof(int64_t));
    memcpy(ppn_off, t->ppn_off, (G + 1) * sizeof(int64_t));
    memcpy(ppf_off, t->ppf_off, (G + 1) * sizeof(int64_t));
    memcpy(pc, t->pc, t->pc_off[G] * sizeof(int64_t));
    memcpy(ppn, t->ppn, t->ppn_off[G] * sizeof(int64_t));
    memcpy(ppf, t->ppf, t->ppf_off[G] * sizeof(int64_t));
}

/* ---- tree forces ---- */

/* Softened quadrupole expansion about the cell's centre of mass.  With
 * r = x_i - com and s^2 = |r|^2 + eps^2:
 *   phi = -G M / s - (G/2) r.Q.r / s^5
 *   a   = -grad phi = -G M r / s^3 + G Q r / s^5 - (5/2) G (r.Q.r) r / s^7 */
static void orc_cell_accel(const orc_tree *t, int64_t c, const double *xi,
                           double G, double eps2, double *acc, double *pot)
{
    const double *Q = t->Q + 6 * c;
    double rx = xi[0] - t->com[3 * c + 0];
    double ry = xi[1] - t->com[3 * c + 1];
    double rz = xi[2] - t->com[3 * c + 2];
    double s2 = rx * rx + ry * ry + rz * rz + eps2;
    double s = sqrt(s2);
    double s3 = s2 * s, s5 = s3 * s2, s7 = s5 * s2;
    double Qrx = Q[0] * rx + Q[3] * ry + Q[4] * rz;
    double Qry = Q[3] * rx + Q[1] * ry + Q[5] * rz;
    double Qrz = Q[4] * rx + Q[5] * ry + Q[2] * rz;
    double rQr = rx * Qrx + ry * Qry + rz * Qrz;
    double M = t->M[c];
    acc[0] += -G * M * rx / s3 + G * Qrx / s5 - 2.5 * G * rQr * rx / s7;
    acc[1] += -G * M * ry / s3 + G * Qry / s5 - 2.5 * G * rQr * ry / s7;
    acc[2] += -G * M * rz / s3 + G * Qrz / s5 - 2.5 * G * rQr * rz / s7;
    *pot += -G * M / s - 0.5 * G * rQr / s5;
}

/* Soft pair term of Eq. 8 (per unit m_i) and Eq. 6 for sorted particle j. */
static void orc_pair_soft(const orc_tree *t, int64_t j, const double *xi,
                          double G, double eps2, double r_cut, double gamma,
                          double *acc, double *pot)
{
    double qx = xi[0] - t->x[3 * j + 0];
    double qy = xi[1] - t->x[3 * j + 1];
    double qz = xi[2] - t->x[3 * j + 2];
    double s2 = qx * qx + qy * qy + qz * qz + eps2;
    double s = sqrt(s2);
    double K = orc_K_of_s(s, r_cut, gamma);
    if (K != 0.0) {
        double f = -G * t->m[j] * K / (s2 * s);
        acc[0] += f * qx;
        acc[1] += f * qy;
        acc[2] += f * qz;
    }
    *pot += -G * t->m[j] * orc_W_over_s(s, r_cut, gamma);
}

typedef struct {
    const orc_tree *t;
    double G, eps2, r_cut, gamma;
    const int64_t *groups; /* groups to evaluate, NULL = all */
    const int64_t *ids;    /* or: sorted particles to evaluate (with groups[r]
                              their groups) */
    double *acc, *pot;     /* indexed by ORIGINAL particle index */
} orc_force_args;

/* Acceleration and soft potential of sorted particle i of group g over the
 * group's lists. */
static void orc_force_one(const orc_force_args *a, int64_t g, int64_t i)
{
    const orc_tree *t = a->t;
    const double *xi = t->x + 3 * i;
    double acc[3] = {0, 0, 0}, pot = 0.0;
    for (int64_t k = t->pc_off[g]; k < t->pc_off[g + 1]; ++k)
        orc_cell_accel(t, t->pc[k], xi, a->G, a->eps2, acc, &pot);
    for (int64_t k = t->ppf_off[g]; k < t->ppf_off[g + 1]; ++k)
        orc_pair_soft(t, t->ppf[k], xi, a->G, a->eps2, a->r_cut, a->gamma,
                      acc, &pot);
    for (int64_t k = t->ppn_off[g]; k < t->ppn_off[g + 1]; ++k) {
        if (t->ppn[k] == i) continue;
        orc_pair_soft(t, t->ppn[k], xi, a->G, a->eps2, a->r_cut, a->gamma,
                      acc, &pot);
    }
    int64_t o = t->order[i];
    for (int c = 0; c < 3; ++c) a->acc[3 * o + c] = acc[c];
    if (a->pot) a->pot[o] = pot;
}

static void orc_force_range(void *p, int64_t lo, int64_t hi)
{
    orc_force_args *a = (orc_force_args *)p;
    const orc_tree *t = a->t;
    for (int64_t r = lo; r < hi; ++r) {
        int64_t g = a->groups ? a->groups[r] : r;
        if (a->ids) {
            orc_force_one(a, g, a->ids[r]);
            continue;
        }
        for (int64_t i = t->g_first[g]; i < t->g_first[g] + t->g_count[g]; ++i)
            orc_force_one(a, g, i);
    }
}

/* Tree acceleration (and soft potential) of the particles of the listed
 * groups (all groups if groups == NULL), written at their ORIGINAL indices
 * of acc (n x 3) and pot (n).  Requires orc_tree_walk first. */
int orc_tree_force(const orc_tree *t, double G, double eps, double r_cut,
                   double gamma, const int64_t *groups, int64_t ng,
                   double *acc, double *pot, int nthreads)
{
    if (!t->walked) return -1;
    orc_force_args a = {t, G, eps * eps, r_cut, gamma, groups, NULL, acc, pot};
    orc_parallel_for(groups ? ng : t->ngroup, nthreads, orc_force_range, &a);
    return 0;
}

/* The same for cnt single particles: sorted particle ids[r], a member of
 * group groups[r]. */
int orc_tree_force_particles(const orc_tree *t, double G, double eps,
                             double r_cut, double gamma, const int64_t *ids,
                             const int64_t *groups, int64_t cnt, double *acc,
                             double *pot, int nthreads)
{
    if (!t->walked) return -1;
    for (int64_t r = 0; r < cnt; ++r) {
        int64_t g = groups[r];
        if (g < 0 || g >= t->ngroup || ids[r] < t->g_first[g]
            || ids[r] >= t->g_first[g] + t->g_count[g])
            return -1;
    }
    orc_force_args a = {t, G, eps * eps, r_cut, gamma, groups, ids, acc, pot};
    orc_parallel_for(cnt, nthreads, orc_force_range, &a);
    return 0;
}

/* Group that holds sorted particle k (groups are disjoint contiguous ranges
 * whose union is [0, n)). */
int64_t orc_tree_group_of(const orc_tree *t, int64_t k)
{
    for (int64_t g = 0; g < t->ngroup; ++g)
        if (k >= t->g_first[g] && k < t->g_first[g] + t->g_count[g]) return g;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Gradients of L = sum_i w_i . a_i (no counterpart in the paper)           */
/*                                                                          */
/* The tree force is a function of positions and masses once the tree      */
/* topology, the groups and the interaction lists are held fixed; these     */
/* functions give its vector-Jacobian product.  Pair term (Eq. 8, per unit  */
/* m_i) with d = x_j - x_i, s^2 = |d|^2 + eps^2:                            */
/*     f = G m_j K(s) d / s^3,                                               */
/*     df/dd = G m_j [ (K / s^3) I + (K'(s) / s^4 - 3 K / s^5) d d^T ],     */
/* K'(s) = dK/dx / ((1 - gamma) r_cut).  Cell term with d = com - x_i:      */
/*     f = G [ M d / s^3 - Q d / s^5 + (5/2) (d.Q.d) d / s^7 ].             */
/* Cell adjoints (dL/dM, dL/dcom, dL/dQ) are pushed to every member k with  */
/* dM/dm_k = 1, dcom/dx_k = m_k / M, dcom/dm_k = e_k / M and                 */
/* dQ_ab/dx_k,c = m_k (3 (delta_ac e_b + e_a delta_bc) - 2 e_c delta_ab),   */
/* dQ_ab/dm_k = 3 e_a e_b - |e|^2 delta_ab, e_k = x_k - com (the dependence */
/* of Q on com vanishes because sum_k m_k e_k = 0).                          */
/* ------------------------------------------------------------------------ */

static double orc_dK_ds(double s, double r_cut, double gamma)
{
    double x = (s / r_cut - gamma) / (1.0 - gamma);
    return orc_dKdx(x) / ((1.0 - gamma) * r_cut);
}

/* Pair contribution: adds -J w to gi, +J w to gj and w.(f/m_j) to gmj. */
static void orc_pair_vjp(const double *xi, const double *xj, double mj,
                         const double *w, double G, double eps2, double r_cut,
                         double gamma, double *gi, double *gj, double *gmj)
{
    double d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
    double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
    if (s2 == 0.0) return;
    double s = sqrt(s2);
    double K = orc_K_of_s(s, r_cut, gamma);
    double Kp = orc_dK_ds(s, r_cut, gamma);
    if (K == 0.0 && Kp == 0.0) return;
    double s3 = s2 * s, s4 = s2 * s2, s5 = s4 * s;
    double phi = K / s3;
    double psi = Kp / s4 - 3.0 * K / s5;
    double wd = w[0] * d[0] + w[1] * d[1] + w[2] * d[2];
    for (int a = 0; a < 3; ++a) {
        double Jw = G * mj * (phi * w[a] + psi * d[a] * wd);
        gi[a] -= Jw;
        gj[a] += Jw;
    }
    *gmj += G * phi * wd;
}

typedef struct {
    const orc_tree *t;
    double G, eps2, r_cut, gamma;
    const double *w;   /* n x 3, original order */
    double *gx, *gm;   /* per thread: n x 3, n, sorted order */
    double *aM, *acom, *aQ; /* per thread cell adjoints: C, C x 3, C x 9 */
} orc_vjp_args;

static void orc_vjp_group(orc_vjp_args *a, int64_t g)
{
    const orc_tree *t = a->t;
    for (int64_t i = t->g_first[g]; i < t->g_first[g] + t->g_count[g]; ++i) {
        const double *xi = t->x + 3 * i;
        const double *w = a->w + 3 * t->order[i];
        double *gi = a->gx + 3 * i;
        for (int64_t k = t->pc_off[g]; k < t->pc_off[g + 1]; ++k) {
            int64_t c = t->pc[k];
            const double *Q6 = t->Q + 6 * c;
            double Q[3][3] = {{Q6[0], Q6[3], Q6[4]}, {Q6[3], Q6[1], Q6[5]},
                              {Q6[4], Q6[5], Q6[2]}};
            double d[3];
            for (int q = 0; q < 3; ++q) d[q] = t->com[3 * c + q] - xi[q];
            double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + a->eps2;
            double s = sqrt(s2);
            double s3 = s2 * s, s5 = s3 * s2, s7 = s5 * s2, s9 = s7 * s2;
            double M = t->M[c];
            double Qd[3], dQd = 0.0, wd = 0.0, wQd = 0.0;
            for (int p = 0; p < 3; ++p) {
                Qd[p] = Q[p][0] * d[0] + Q[p][1] * d[1] + Q[p][2] * d[2];
            }
            for (int p = 0; p < 3; ++p) {
                dQd += d[p] * Qd[p];
                wd += w[p] * d[p];
                wQd += w[p] * Qd[p];
            }
            /* (J^T w)_b = sum_a w_a J_ab with J = df/dd */
            double JTw[3];
            for (int b = 0; b < 3; ++b) {
                double wQ_b = w[0] * Q[0][b] + w[1] * Q[1][b] + w[2] * Q[2][b];
                double v = M * (w[b] / s3 - 3.0 * wd * d[b] / s5)
                           - (wQ_b / s5 - 5.0 * wQd * d[b] / s7)
                           + 2.5 * (2.0 * wd * Qd[b] / s7 + dQd * w[b] / s7
                                    - 7.0 * dQd * wd * d[b] / s9);
                JTw[b] = a->G * v;
            }
            for (int b = 0; b < 3; ++b) {
                gi[b] -= JTw[b];
                a->acom[3 * c + b] += JTw[b];
            }
            a->aM[c] += a->G * wd / s3;
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q)
                    a->aQ[9 * c + 3 * p + q] +=
                        a->G * (-w[p] * d[q] / s5 + 2.5 * wd * d[p] * d[q] / s7);
        }
        for (int pass = 0; pass < 2; ++pass) {
            const int64_t *off = pass ? t->ppf_off : t->ppn_off;
            const int64_t *lst = pass ? t->ppf : t->ppn;
            for (int64_t k = off[g]; k < off[g + 1]; ++k) {
                int64_t j = lst[k];
                if (j == i) continue;
                orc_pair_vjp(xi, t->x + 3 * j, t->m[j], w, a->G, a->eps2,
                             a->r_cut, a->gamma, gi, a->gx + 3 * j, a->gm + j);
            }
        }
    }
}

typedef struct {
    orc_vjp_args *args;
    int64_t ng;
    int nthreads, id;
} orc_vjp_job;

static void *orc_vjp_main(void *p)
{
    orc_vjp_job *j = (orc_vjp_job *)p;
    for (int64_t g = j->id; g < j->ng; g += j->nthreads)
        orc_vjp_group(&j->args[j->id], g);
    return NULL;
}

/* Gradient of sum_i w_i . a_i over the current lists (orc_tree_walk first).
 * w, gx: n x 3 in ORIGINAL order; gm: n.  Returns 0 on success. */
int orc_tree_vjp(const orc_tree *t, double G, double eps, double r_cut,
                 double gamma, const double *w, double *gx, double *gm,
                 int nthreads)
{
    if (!t->walked) return -1;
    int64_t n = t->n, C = t->ncell;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    orc_vjp_args *args = calloc(nthreads, sizeof(orc_vjp_args));
    for (int k = 0; k < nthreads; ++k) {
        args[k].t = t;
        args[k].G = G;
        args[k].eps2 = eps * eps;
        args[k].r_cut = r_cut;
        args[k].gamma = gamma;
        args[k].w = w;
        args[k].gx = calloc(3 * n + 1, sizeof(double));
        args[k].gm = calloc(n + 1, sizeof(double));
        args[k].aM = calloc(C + 1, sizeof(double));
        args[k].acom = calloc(3 * C + 1, sizeof(double));
        args[k].aQ = calloc(9 * C + 1, sizeof(double));
    }
    pthread_t th[64];
    orc_vjp_job jobs[64];
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].args = args;
        jobs[k].ng = t->ngroup;
        jobs[k].nthreads = nthreads;
        jobs[k].id = k;
        pthread_create(&th[k], NULL, orc_vjp_main, &jobs[k]);
    }
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    /* reduce the per-thread buffers into thread 0's */
    orc_vjp_args *r = &args[0];
    for (int k = 1; k < nthreads; ++k) {
        for (int64_t q = 0; q < 3 * n; ++q) r->gx[q] += args[k].gx[q];
        for (int64_t q = 0; q < n; ++q) r->gm[q] += args[k].gm[q];
        for (int64_t q = 0; q < C; ++q) r->aM[q] += args[k].aM[q];
        for (int64_t q = 0; q < 3 * C; ++q) r->acom[q] += args[k].acom[q];
        for (int64_t q = 0; q < 9 * C; ++q) r->aQ[q] += args[k].aQ[q];
    }
    /* push the cell adjoints to every member particle */
    for (int64_t c = 0; c < C; ++c) {
        double S[3][3], tr = 0.0;
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q)
                S[p][q] = 0.5 * (r->aQ[9 * c + 3 * p + q] + r->aQ[9 * c + 3 * q + p]);
        tr = S[0][0] + S[1][1] + S[2][2];
        double aM = r->aM[c];
        const double *ac = r->acom + 3 * c;
        if (aM == 0.0 && ac[0] == 0.0 && ac[1] == 0.0 && ac[2] == 0.0 &&
            tr == 0.0 && S[0][1] == 0.0 && S[0][2] == 0.0 && S[1][2] == 0.0 &&
            S[0][0] == 0.0 && S[1][1] == 0.0)
            continue;
        double M = t->M[c];
        for (int64_t k = t->first[c]; k < t->first[c] + t->count[c]; ++k) {
            double e[3];
            for (int q = 0; q < 3; ++q) e[q] = t->x[3 * k + q] - t->com[3 * c + q];
            double Se[3], eSe = 0.0, ee = 0.0, eac = 0.0;
            for (int p = 0; p < 3; ++p) {
                Se[p] = S[p][0] * e[0] + S[p][1] * e[1] + S[p][2] * e[2];
            }
            for (int p = 0; p < 3; ++p) {
                eSe += e[p] * Se[p];
                ee += e[p] * e[p];
                eac += e[p] * ac[p];
            }
            double mk = t->m[k];
            for (int q = 0; q < 3; ++q)
                r->gx[3 * k + q] += (mk / M) * ac[q] + mk * (6.0 * Se[q] - 2.0 * tr * e[q]);
            r->gm[k] += aM + eac / M + 3.0 * eSe - ee * tr;
        }
    }
    for (int64_t k = 0; k < n; ++k) {
        int64_t o = t->order[k];
        for (int q = 0; q < 3; ++q) gx[3 * o + q] = r->gx[3 * k + q];
        gm[o] = r->gm[k];
    }
    for (int k = 0; k < nthreads; ++k) {
        free(args[k].gx);
        free(args[k].gm);
        free(args[k].aM);
        free(args[k].acom);
        free(args[k].aQ);
    }
    free(args);
    return 0;
}

/* Direct-summation gradient of sum_i w_i . a_soft,i (all pairs, Eq. 8). */
void orc_direct_vjp(int64_t n, const double *pos, const double *m, double G,
                    double eps, double r_cut, double gamma, const double *w,
                    double *gx, double *gm, int nthreads)
{
    (void)nthreads;
    memset(gx, 0, 3 * n * sizeof(double));
    memset(gm, 0, n * sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            orc_pair_vjp(pos + 3 * i, pos + 3 * j, m[j], w + 3 * i, G,
                         eps * eps, r_cut, gamma, gx + 3 * i, gx + 3 * j,
                         gm + j);
        }
}

/* New positions / masses (original order) for the same tree: the sorted
 * copies and all cell moments are recomputed; keys, topology, groups and
 * interaction lists are kept (the frozen-structure function the gradients
 * above differentiate). */
void orc_tree_update(orc_tree *t, const double *pos, const double *m)
{
    for (int64_t k = 0; k < t->n; ++k) {
        int64_t i = t->order[k];
        for (int a = 0; a < 3; ++a) t->x[3 * k + a] = pos[3 * i + a];
        t->m[k] = m[i];
    }
    for (int64_t c = 0; c < t->ncell; ++c) orc_cell_moments(t, c);
}

/* ------------------------------------------------------------------------ */
/* Hard part (Sect. 2.1 and 2.2): F_hard over the neighbour lists and the   */
/* fourth-order Hermite integrator with block timesteps                     */
/* ------------------------------------------------------------------------ */
/* Positions and velocities are n x 3 row-major; neighbour rows are CSR
 * (off[n+1], idx) in ascending j, as the neighbour search returns them.
 * Every expression is written in the order it is evaluated. */

/* ---- The oracle proper: the hard part as the paper writes it ----
 *
 * Plain FP64 with one rounding per written operation (the file is compiled
 * with -ffp-contract=off): the pair force of Eq. 7 and its time derivative
 * with K of Eq. 12 in its monomial form (orc_K, orc_dKdx), the timestep
 * criteria of Eq. 18-20 in their printed form, dt <= eta sqrt(num / den)
 * (Eq. 18 read with |a^(1)| |a^(3)| in the denominator, see below), and the
 * Hermite predictor and corrector of Makino & Aarseth (1992) as written
 * below.  The mirror further down evaluates the same formulas in the GPU
 * path's fused order; only that mirror, not this code, is bit-identical to
 * the GPU. */

/* Per pair type (Sect. 3.2.2; 0 star-star, 1 black hole-star, 2 black
 * hole-black hole): softening and cut-off.  r_cut = infinity means the pair
 * is not split: y = s / r_cut = 0, x < 0 and K = 0, so all of it is hard. */
typedef struct {
    double eps, r_cut;
} orc_plain_pair;

typedef struct {
    double G, gamma, alpha;
    orc_plain_pair pt[3];
    int64_t n_fs;       /* particles [n_fs, n) are black holes */
    double a0_rcut[2];  /* per species: the r_cut of a_0 (Eq. 19) */
    double eta[2];      /* per species: eta of Eq. 18 */
} orc_plain_par;

static orc_plain_par orc_plain_par_make(double G, double eps, double r_cut,
                                        double gamma, double alpha, double eta)
{
    orc_plain_par P;
    P.G = G;
    P.gamma = gamma;
    P.alpha = alpha;
    for (int t = 0; t < 3; ++t) {
        P.pt[t].eps = eps;
        P.pt[t].r_cut = r_cut;
    }
    P.n_fs = INT64_MAX;
    P.a0_rcut[0] = P.a0_rcut[1] = r_cut;
    P.eta[0] = P.eta[1] = eta;
    return P;
}

static double orc_norm3(const double *a)
{
    return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
}

/* Hard acceleration and jerk of particle i from its neighbour row, Eq. 7 as
 * written: with q = x_i - x_j, u = v_i - v_j, s = sqrt(|q|^2 + eps^2)
 * (Eq. 2), y = s / r_cut, x = (y - gamma) / (1 - gamma) (Eq. 13-15),
 *   a_i  = -sum_j G m_j (1 - K(x)) q / s^3,
 *   da_i = -sum_j G m_j [ (1 - K) (u / s^3 - 3 (q.u) q / s^5)
 *                         - (dK/ds) ((q.u) / s) q / s^3 ],
 * dK/ds = (dK/dx) / ((1 - gamma) r_cut), ds/dt = (q.u) / s. */
static void orc_hard_one(int64_t i, const double *x, const double *v,
                         const double *m, const int64_t *off,
                         const int32_t *idx, const orc_plain_par *P,
                         double *a, double *jk)
{
    double acc[3] = {0.0, 0.0, 0.0}, jrk[3] = {0.0, 0.0, 0.0};
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        int64_t j = idx[e];
        const orc_plain_pair *pp = &P->pt[(i >= P->n_fs) + (j >= P->n_fs)];
        double q[3], u[3];
        for (int c = 0; c < 3; ++c) {
            q[c] = x[3 * i + c] - x[3 * j + c];
            u[c] = v[3 * i + c] - v[3 * j + c];
        }
        double s = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + pp->eps * pp->eps);
        double y = s / pp->r_cut;
        double xk = (y - P->gamma) / (1.0 - P->gamma);
        double K = orc_K(xk);
        double dKds = orc_dKdx(xk) / ((1.0 - P->gamma) * pp->r_cut);
        double qu = q[0] * u[0] + q[1] * u[1] + q[2] * u[2];
        double s3 = s * s * s;
        double s5 = s3 * s * s;
        double Gm = P->G * m[j];
        for (int c = 0; c < 3; ++c) {
            acc[c] -= Gm * (1.0 - K) * q[c] / s3;
            jrk[c] -= Gm * ((1.0 - K) * (u[c] / s3 - 3.0 * qu * q[c] / s5)
                            - dKds * (qu / s) * q[c] / s3);
        }
    }
    for (int c = 0; c < 3; ++c) {
        a[c] = acc[c];
        jk[c] = jrk[c];
    }
}

/* Hard acceleration and jerk of every particle (a, jk: n x 3). */
void orc_hard_force(int64_t n, const double *x, const double *v,
                    const double *m, const int64_t *off, const int32_t *idx,
                    double G, double eps, double r_cut, double gamma,
                    double *a, double *jk)
{
    orc_plain_par P = orc_plain_par_make(G, eps, r_cut, gamma, 0.0, 0.0);
    for (int64_t i = 0; i < n; ++i)
        orc_hard_one(i, x, v, m, off, idx, &P, a + 3 * i, jk + 3 * i);
}

/* The same with two species: the last n_bh particles are black holes and a
 * pair of type t takes eps[t] and r_cut[t]. */
void orc_hard_force_species(int64_t n, int64_t n_bh, const double *x,
                            const double *v, const double *m,
                            const int64_t *off, const int32_t *idx, double G,
                            const double *eps, const double *r_cut,
                            double gamma, double *a, double *jk)
{
    orc_plain_par P = orc_plain_par_make(G, eps[0], r_cut[0], gamma, 0.0, 0.0);
    for (int t = 1; t < 3; ++t) {
        P.pt[t].eps = eps[t];
        P.pt[t].r_cut = r_cut[t];
    }
    P.n_fs = n - n_bh;
    for (int64_t i = 0; i < n; ++i)
        orc_hard_one(i, x, v, m, off, idx, &P, a + 3 * i, jk + 3 * i);
}

/* Block level from a criterion dt_crit (Eq. 18 or Eq. 20, before the min
 * with dt_max): the smallest k in [kmin, kmax] whose step dt_max 2^-k is at
 * most dt_crit (kmax, and *capped set, when none is).  *margin receives the
 * least relative distance |dt_k - dt_crit| / dt_crit over the steps
 * compared, the size of the rounding change that could flip the decision. */
static int orc_plain_level(double dt_crit, double dt_max, int kmin, int kmax,
                           int *capped, double *margin)
{
    int k = kmin;
    for (;;) {
        double dt_k = ldexp(dt_max, -k);
        double d = fabs(dt_k - dt_crit) / dt_crit;
        if (d < *margin) *margin = d;
        if (dt_k <= dt_crit) {
            *capped = 0;
            return k;
        }
        if (k == kmax) {
            *capped = 1;
            return k;
        }
        ++k;
    }
}

/* Eq. 18-20 in the printed form.  A criterion whose denominator vanishes
 * (no hard force) puts no limit on the step. */
static double orc_plain_crit(double eta, double num, double den)
{
    if (den == 0.0) return INFINITY;
    return eta * sqrt(num / den);
}

/* Fourth-order Hermite integration (Makino & Aarseth 1992) of every
 * particle with a non-empty neighbour row over dt_soft under H_hard, with
 * individual block timesteps (the sixth step of Sect. 2.2); particles with
 * an empty row are isolated and drift, x <- x + dt_soft v (the fifth).
 *
 * Time is counted in ticks of dt_max 2^-kmax, dt_max = dt_soft 2^-p.  A
 * particle at level k steps h = dt_max 2^-k and its time is a multiple of h.
 *   - First level: Eq. 20, dt = eta_s sqrt((|a|^2 + a0^2) / |j|^2),
 *     eta_s = eta / 10, a0 = alpha G m_i / r_cut^2 (Eq. 19).
 *   - Later levels: Eq. 18,
 *       dt = eta sqrt((sqrt(|a|^2 + a0^2) |a2| + |j|^2) / (|j| |a3| + |a2|^2))
 *     with a, j at the end of the step and a2, a3 the Hermite
 *     interpolation's, a2 advanced to the end of the step (a2 + h a3).  The
 *     step may at most double, and is halved until the current time is a
 *     multiple of it.
 *   - Block step: t_n is the least t_i + h_i; every particle is predicted
 *       xp = x + v d + a d^2 / 2 + j d^3 / 6,  vp = v + a d + j d^2 / 2
 *     (d = t_n - t_i); the particles due at t_n get a1, j1 from the
 *     predicted values of their rows and are corrected:
 *       a2 = (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2
 *       a3 = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3
 *       x = xp + a2 h^4 / 24 + a3 h^5 / 120,  v = vp + a2 h^3 / 6 + a3 h^4 / 24.
 * stats (may be NULL): [0] block steps, [1] particle steps, [2] pair
 * evaluations, [3] steps whose level was capped at kmax.  Per particle (each
 * may be NULL): nstep, its number of steps; lev0, its first level; margin,
 * the least relative distance of any of its level decisions from a tie
 * (orc_plain_level; +infinity for an isolated particle).
 * Returns 0, or -1 on bad arguments or allocation failure. */
static int orc_hermite_run(int64_t n, double *x, double *v, const double *m,
                           const int64_t *off, const int32_t *idx,
                           const orc_plain_par *P, double dt_soft, int p,
                           int kmax, int64_t *stats, int64_t *nstep,
                           int32_t *lev0, double *margin)
{
    if (n < 0 || p < 0 || kmax < 0 || p + kmax > 60) return -1;
    const double dt_max = ldexp(dt_soft, -p);
    const double tick = ldexp(dt_max, -kmax);
    const int64_t T = (int64_t)1 << (p + kmax);
    int capped = 0;
    int64_t st[4] = {0, 0, 0, 0};
    double *a = malloc(3 * n * sizeof(double) + 1);
    double *jk = malloc(3 * n * sizeof(double) + 1);
    double *xp = malloc(3 * n * sizeof(double) + 1);
    double *vp = malloc(3 * n * sizeof(double) + 1);
    int64_t *t = malloc(n * sizeof(int64_t) + 1);
    int *lev = malloc(n * sizeof(int) + 1);
    int64_t *ns = malloc(n * sizeof(int64_t) + 1);
    double *mg = malloc(n * sizeof(double) + 1);
    if (!a || !jk || !xp || !vp || !t || !lev || !ns || !mg) {
        free(a); free(jk); free(xp); free(vp); free(t); free(lev); free(ns);
        free(mg);
        return -1;
    }
    /* start: forces at t = 0 and the first levels (Eq. 20) */
    for (int64_t i = 0; i < n; ++i) {
        t[i] = 0;
        lev[i] = 0;
        ns[i] = 0;
        mg[i] = INFINITY;
        if (off[i + 1] == off[i]) continue;
        orc_hard_one(i, x, v, m, off, idx, P, a + 3 * i, jk + 3 * i);
        st[2] += off[i + 1] - off[i];
        const int sp = i >= P->n_fs;
        double rc = P->a0_rcut[sp];
        double a0 = P->alpha * P->G * m[i] / (rc * rc);
        double an = orc_norm3(a + 3 * i), jn = orc_norm3(jk + 3 * i);
        double eta_s = P->eta[sp] / 10.0;
        double crit = orc_plain_crit(eta_s, an * an + a0 * a0, jn * jn);
        lev[i] = orc_plain_level(crit, dt_max, 0, kmax, &capped, &mg[i]);
        st[3] += capped;
    }
    if (lev0)
        for (int64_t i = 0; i < n; ++i) lev0[i] = lev[i];
    for (;;) {
        int64_t tn = T;
        int any = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (off[i + 1] == off[i] || t[i] == T) continue;
            int64_t e = t[i] + ((int64_t)1 << (kmax - lev[i]));
            if (e < tn) tn = e;
            any = 1;
        }
        if (!any) break;
        ++st[0];
        /* predict every non-isolated particle to tn */
        for (int64_t i = 0; i < n; ++i) {
            if (off[i + 1] == off[i]) continue;
            double d = (double)(tn - t[i]) * tick;
            for (int c = 0; c < 3; ++c) {
                int64_t k = 3 * i + c;
                xp[k] = x[k] + v[k] * d + a[k] * (d * d / 2.0)
                        + jk[k] * (d * d * d / 6.0);
                vp[k] = v[k] + a[k] * d + jk[k] * (d * d / 2.0);
            }
        }
        /* evaluate and correct the particles due at tn */
        for (int64_t i = 0; i < n; ++i) {
            if (off[i + 1] == off[i]) continue;
            int64_t step = (int64_t)1 << (kmax - lev[i]);
            if (t[i] + step != tn) continue;
            double a1[3], j1[3];
            orc_hard_one(i, xp, vp, m, off, idx, P, a1, j1);
            ++st[1];
            ++ns[i];
            st[2] += off[i + 1] - off[i];
            double h = (double)step * tick;
            double h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h;
            double a2[3], a3[3], a2e[3];
            for (int c = 0; c < 3; ++c) {
                int64_t k = 3 * i + c;
                double a0c = a[k], j0c = jk[k];
                a2[c] = (-6.0 * (a0c - a1[c]) - h * (4.0 * j0c + 2.0 * j1[c])) / h2;
                a3[c] = (12.0 * (a0c - a1[c]) + 6.0 * h * (j0c + j1[c])) / h3;
                x[k] = xp[k] + a2[c] * h4 / 24.0 + a3[c] * h5 / 120.0;
                v[k] = vp[k] + a2[c] * h3 / 6.0 + a3[c] * h4 / 24.0;
                a[k] = a1[c];
                jk[k] = j1[c];
                a2e[c] = a2[c] + h * a3[c];
            }
            t[i] = tn;
            if (tn == T) continue;
            /* Eq. 18, with |a^(1)| |a^(3)| as the first term of the
             * denominator: as printed, |a^(0)| |a^(3)| has the dimension
             * L^2 T^-7 beside |a^(2)|^2 of L^2 T^-8, so the printed step
             * would change with the unit of time; with |a^(1)| the ratio is
             * a time squared, as in the Aarseth criterion that Eq. 18
             * extends by a_0. */
            const int sp = i >= P->n_fs;
            double rc = P->a0_rcut[sp];
            double a0 = P->alpha * P->G * m[i] / (rc * rc);
            double an = orc_norm3(a1), jn = orc_norm3(j1);
            double a2n = orc_norm3(a2e), a3n = orc_norm3(a3);
            double num = sqrt(an * an + a0 * a0) * a2n + jn * jn;
            double den = jn * a3n + a2n * a2n;
            double crit = orc_plain_crit(P->eta[sp], num, den);
            int kmin = lev[i] > 0 ? lev[i] - 1 : 0;
            int k = orc_plain_level(crit, dt_max, kmin, kmax, &capped, &mg[i]);
            st[3] += capped;
            while (tn % ((int64_t)1 << (kmax - k)) != 0) ++k;
            lev[i] = k;
        }
    }
    /* isolated particles drift (Sect. 2.2, step 5) */
    for (int64_t i = 0; i < n; ++i) {
        if (off[i + 1] != off[i]) continue;
        for (int c = 0; c < 3; ++c) x[3 * i + c] = x[3 * i + c] + dt_soft * v[3 * i + c];
    }
    if (stats)
        for (int k = 0; k < 4; ++k) stats[k] = st[k];
    if (nstep)
        for (int64_t i = 0; i < n; ++i) nstep[i] = ns[i];
    if (margin)
        for (int64_t i = 0; i < n; ++i) margin[i] = mg[i];
    free(a); free(jk); free(xp); free(vp); free(t); free(lev); free(ns);
    free(mg);
    return 0;
}

int orc_hermite(int64_t n, double *x, double *v, const double *m,
                const int64_t *off, const int32_t *idx, double G, double eps,
                double r_cut, double gamma, double eta, double alpha,
                double dt_soft, int p, int kmax, int64_t *stats,
                int64_t *nstep, int32_t *lev0, double *margin)
{
    orc_plain_par P = orc_plain_par_make(G, eps, r_cut, gamma, alpha, eta);
    return orc_hermite_run(n, x, v, m, off, idx, &P, dt_soft, p, kmax, stats,
                           nstep, lev0, margin);
}

/* The same with two species (Sect. 3.2.2): the last n_bh particles are black
 * holes.  Pair type t takes eps[t] and r_cut[t] (r_cut[2] = infinity: not
 * split, K = 0); species s takes eta[s] (eta / 10 on the first step) and
 * a_0 = alpha G m_i / r_cut[s]^2, the cut-off of its own pairs with stars. */
int orc_hermite_species(int64_t n, int64_t n_bh, double *x, double *v,
                        const double *m, const int64_t *off,
                        const int32_t *idx, double G, const double *eps,
                        const double *r_cut, double gamma, const double *eta,
                        double alpha, double dt_soft, int p, int kmax,
                        int64_t *stats, int64_t *nstep, int32_t *lev0,
                        double *margin)
{
    if (n_bh < 0 || n_bh > n) return -1;
    orc_plain_par P = orc_plain_par_make(G, eps[0], r_cut[0], gamma, alpha,
                                         eta[0]);
    for (int t = 1; t < 3; ++t) {
        P.pt[t].eps = eps[t];
        P.pt[t].r_cut = r_cut[t];
    }
    P.n_fs = n - n_bh;
    P.a0_rcut[1] = r_cut[1];
    P.eta[1] = eta[1];
    return orc_hermite_run(n, x, v, m, off, idx, &P, dt_soft, p, kmax, stats,
                           nstep, lev0, margin);
}

/* ---- The fused-order mirror of the GPU's hard part ----
 *
 * NOT the oracle: a second, separately named check.  It evaluates the same
 * formulas as the code above in the order the GPU kernels do: every product
 * that feeds a sum as one fused multiply-add, K and dK/dx in Horner form,
 * reciprocal powers of s, and the timestep criteria compared in squares
 * (dt^2 den <= eta^2 num, with sqrt(A) sqrt(B) taken as sqrt(A B)).  It
 * agrees with the GPU bit for bit, which checks the GPU's block schedule
 * and component bookkeeping exactly; the oracle above checks the GPU's
 * arithmetic against the printed formulas within a rounding tolerance. */
/* The hard part evaluates its formulas with fused multiply-adds: fma(a, b, c)
 * is a b + c with one rounding (IEEE 754 fusedMultiplyAdd), written out at
 * every use so that the order of operations is explicit.  The same holds
 * for the GPU path, so the two agree bit for bit. */
static double orc_mirror_dot3(const double *a, const double *b)
{
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

/* K and dK/dx of Eq. 12 in Horner form for the hard part:
 *   K = x^4 (35 + x (-84 + x (70 - 20 x))),
 *   dK/dx = 140 x^3 (1 - x)^3 = x^3 (140 + x (-420 + x (420 - 140 x))). */
static double orc_mirror_K(double x)
{
    if (x < 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    double x2 = x * x, x4 = x2 * x2;
    return x4 * fma(fma(fma(-20.0, x, 70.0), x, -84.0), x, 35.0);
}

static double orc_mirror_dK(double x)
{
    if (x <= 0.0 || x >= 1.0) return 0.0;
    double x3 = x * x * x;
    return x3 * fma(fma(fma(-140.0, x, 420.0), x, -420.0), x, 140.0);
}

/* Per pair type: softening and cut-off.  Types (Sect. 3.2.2): 0 star-star,
 * 1 black hole-star, 2 black hole-black hole.  The black holes are the last
 * n_bh particles; the type of (i, j) is [i >= n_fs] + [j >= n_fs].  Between
 * black holes the force is not split (F_soft = 0): 1 / r_cut = 0, so that
 * x = -gamma / (1 - gamma) < 0 and K = 0. */
typedef struct {
    double eps2;
    double irc;    /* 1 / r_cut (0: not split) */
    double iomgrc; /* 1 / ((1 - gamma) r_cut) */
} orc_mirror_pair;

/* Constants of the hard part, each computed once in this order. */
typedef struct {
    double G, gamma;
    double iomg;   /* 1 / (1 - gamma) */
    orc_mirror_pair pt[3];
    int64_t n_fs;  /* particles [n_fs, n) are black holes */
    double a0c[2]; /* per species: alpha G / r_cut^2, a_0 = a0c m_i (Eq. 19) */
    double c6, c24, c120;  /* 1/6, 1/24, 1/120 */
    double eta2[2];   /* per species: eta^2 (later steps) */
    double eta_s2[2]; /* per species: eta_s^2 (first steps) */
} orc_mirror_par;

static orc_mirror_pair orc_mirror_pair_make(double eps, double r_cut, double gamma)
{
    orc_mirror_pair q;
    q.eps2 = eps * eps;
    q.irc = isinf(r_cut) ? 0.0 : 1.0 / r_cut;
    q.iomgrc = isinf(r_cut) ? 0.0 : 1.0 / ((1.0 - gamma) * r_cut);
    return q;
}

/* One species (every particle a star): the parameters of the plain path. */
static orc_mirror_par orc_mirror_par_make(double G, double eps, double r_cut,
                                      double gamma, double alpha)
{
    orc_mirror_par P;
    P.G = G;
    P.gamma = gamma;
    P.iomg = 1.0 / (1.0 - gamma);
    P.pt[0] = orc_mirror_pair_make(eps, r_cut, gamma);
    P.pt[1] = P.pt[0];
    P.pt[2] = P.pt[0];
    P.n_fs = INT64_MAX;
    P.a0c[0] = alpha * G / (r_cut * r_cut);
    P.a0c[1] = P.a0c[0];
    P.c6 = 1.0 / 6.0;
    P.c24 = 1.0 / 24.0;
    P.c120 = 1.0 / 120.0;
    return P;
}

/* Hard acceleration and jerk of particle i from its neighbour row: the pair
 * force of Eq. 7 (weight 1 - K(s), s of Eq. 2, q = x_i - x_j) and its time
 * derivative along u = v_i - v_j, with ds/dt = (q.u)/s:
 *   a_i  = -sum G m_j (1-K) q / s^3
 *   da_i = -sum G m_j [ (1-K) (u - 3 (q.u) q / s^2) / s^3
 *                       - (dK/ds) ((q.u) / s) q / s^3 ].
 * One square root and one division per pair: 1/s, then its powers. */
static void orc_mirror_hard_one(int64_t i, const double *x, const double *v,
                         const double *m, const int64_t *off,
                         const int32_t *idx, const orc_mirror_par *P,
                         double *a, double *jk)
{
    double acc[3] = {0.0, 0.0, 0.0}, jrk[3] = {0.0, 0.0, 0.0};
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        int64_t j = idx[e];
        const orc_mirror_pair *pp = &P->pt[(i >= P->n_fs) + (j >= P->n_fs)];
        double q[3], u[3];
        for (int c = 0; c < 3; ++c) {
            q[c] = x[3 * i + c] - x[3 * j + c];
            u[c] = v[3 * i + c] - v[3 * j + c];
        }
        double s2 = fma(q[0], q[0], fma(q[1], q[1], fma(q[2], q[2], pp->eps2)));
        double s = sqrt(s2);
        double ri = 1.0 / s;
        double ri2 = ri * ri;
        double ri3 = ri2 * ri;
        double xk = fma(s, pp->irc, -P->gamma) * P->iomg;
        double w = 1.0 - orc_mirror_K(xk);
        double dKds = orc_mirror_dK(xk) * pp->iomgrc;
        double rv = orc_mirror_dot3(q, u);
        double gm = P->G * m[j];
        double fa = gm * w * ri3;
        double c1 = 3.0 * rv * ri2;
        double fb = gm * (dKds * rv * ri) * ri3;
        for (int c = 0; c < 3; ++c) {
            acc[c] = fma(-fa, q[c], acc[c]);
            jrk[c] = fma(-fa, fma(-c1, q[c], u[c]), fma(fb, q[c], jrk[c]));
        }
    }
    for (int c = 0; c < 3; ++c) {
        a[c] = acc[c];
        jk[c] = jrk[c];
    }
}

/* Hard acceleration and jerk of every particle (a, jk: n x 3). */
void orc_mirror_hard_force(int64_t n, const double *x, const double *v,
                    const double *m, const int64_t *off, const int32_t *idx,
                    double G, double eps, double r_cut, double gamma,
                    double *a, double *jk)
{
    orc_mirror_par P = orc_mirror_par_make(G, eps, r_cut, gamma, 0.0);
    for (int64_t i = 0; i < n; ++i)
        orc_mirror_hard_one(i, x, v, m, off, idx, &P, a + 3 * i, jk + 3 * i);
}

/* The same with two species: the last n_bh particles are black holes and a
 * pair of type t takes eps[t] and r_cut[t] (as orc_mirror_hermite_species). */
void orc_mirror_hard_force_species(int64_t n, int64_t n_bh, const double *x,
                            const double *v, const double *m,
                            const int64_t *off, const int32_t *idx, double G,
                            const double *eps, const double *r_cut,
                            double gamma, double *a, double *jk)
{
    orc_mirror_par P = orc_mirror_par_make(G, eps[0], r_cut[0], gamma, 0.0);
    for (int t = 1; t < 3; ++t) P.pt[t] = orc_mirror_pair_make(eps[t], r_cut[t], gamma);
    P.n_fs = n - n_bh;
    for (int64_t i = 0; i < n; ++i)
        orc_mirror_hard_one(i, x, v, m, off, idx, &P, a + 3 * i, jk + 3 * i);
}

/* Block level for a step dt of at most eta sqrt(num / den) (Eq. 18
 * and Eq. 20), tested in squares so that it needs neither a division nor the
 * outer square root: dt^2 den <= eta^2 num with e = eta^2 num and
 * dm2 = dt_max^2.  The smallest k in [kmin, kmax] with
 * (dt_max 2^-k)^2 den <= e (kmax when none is); *capped is set when even
 * kmax fails. */
static int orc_mirror_level(double den, double e, double dm2, int kmin, int kmax,
                     int *capped)
{
    int k = kmin;
    double q = ldexp(dm2, -2 * k);
    while (k < kmax && q * den > e) {
        ++k;
        q = q * 0.25;
    }
    *capped = k == kmax && q * den > e;
    return k;
}

/* Fourth-order Hermite integration (Makino & Aarseth 1992) of every
 * particle with a non-empty neighbour row over dt_soft under H_hard, with
 * individual block timesteps (the third step of the P3T procedure of
 * Sect. 2.1 / the sixth of Sect. 2.2); particles with an empty row are
 * isolated and drift, x <- x + dt_soft v (the fifth step of Sect. 2.2).
 *
 * Products that feed a sum are fused (fma, one rounding each).
 * Divisions are few: 1/s per pair, 1/h per correction, and constants
 * (1/r_cut, 1/(1 - gamma), alpha G / r_cut^2, 1/6, 1/24, 1/120) formed once;
 * the timestep criteria are tested in squares (orc_mirror_level).
 * Time is counted in ticks of dt_max 2^-kmax, dt_max = dt_soft 2^-p.  A
 * particle at level k steps dt_max 2^-k; its time is always a multiple of
 * its step.  First step: Eq. 20 with eta_s = eta / 10; later steps:
 * Eq. 18, a_0 = alpha G m_i / r_cut^2, with a^(2) and a^(3) from
 * the Hermite interpolation of the last step; the level may rise by at most
 * one per step (the step at most doubles) and is raised further until the
 * current time is a multiple of the step.  Each block step: the next time
 * t_n is the smallest t_i + dt_i; every particle is predicted to t_n
 *   xp = x + v d + a (d^2 / 2) + j (d^3 / 6),  vp = v + a d + j (d^2 / 2),
 * the particles with t_i + dt_i = t_n get a, j at t_n from the predicted
 * values (own and neighbours') and are corrected, with h = their step:
 *   a2 = (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2
 *   a3 = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3
 *   x = xp + a2 h^4 / 24 + a3 h^5 / 120,  v = vp + a2 h^3 / 6 + a3 h^4 / 24.
 * stats (may be NULL): [0] block steps, [1] particle steps, [2] pair
 * evaluations, [3] steps whose level was capped at kmax.
 * Returns 0, or -1 on bad arguments or allocation failure. */
static int orc_mirror_hermite_run(int64_t n, double *x, double *v, const double *m,
                           const int64_t *off, const int32_t *idx,
                           orc_mirror_par P, double dt_soft, int p, int kmax,
                           int64_t *stats);

int orc_mirror_hermite(int64_t n, double *x, double *v, const double *m,
                const int64_t *off, const int32_t *idx, double G, double eps,
                double r_cut, double gamma, double eta, double alpha,
                double dt_soft, int p, int kmax, int64_t *stats)
{
    orc_mirror_par P = orc_mirror_par_make(G, eps, r_cut, gamma, alpha);
    const double eta_s = eta / 10.0;
    P.eta2[0] = P.eta2[1] = eta * eta;
    P.eta_s2[0] = P.eta_s2[1] = eta_s * eta_s;
    return orc_mirror_hermite_run(n, x, v, m, off, idx, P, dt_soft, p, kmax, stats);
}

/* The same with two species (Sect. 3.2.2): the last n_bh particles are black
 * holes.  Pair types 0 star-star, 1 black hole-star, 2 black hole-black
 * hole take eps[t] and r_cut[t] (r_cut[2] = infinity: not split, K = 0);
 * species s takes eta[s] (eta_s = eta / 10 on the first step) and
 * a_0 = alpha G m_i / r_cut^2 with the cut-off of its own pairs with stars,
 * r_cut[s]. */
int orc_mirror_hermite_species(int64_t n, int64_t n_bh, double *x, double *v,
                        const double *m, const int64_t *off,
                        const int32_t *idx, double G, const double *eps,
                        const double *r_cut, double gamma, const double *eta,
                        double alpha, double dt_soft, int p, int kmax,
                        int64_t *stats)
{
    if (n_bh < 0 || n_bh > n) return -1;
    orc_mirror_par P = orc_mirror_par_make(G, eps[0], r_cut[0], gamma, alpha);
    for (int t = 1; t < 3; ++t) P.pt[t] = orc_mirror_pair_make(eps[t], r_cut[t], gamma);
    P.n_fs = n - n_bh;
    P.a0c[1] = alpha * G / (r_cut[1] * r_cut[1]);
    for (int sp = 0; sp < 2; ++sp) {
        const double eta_s = eta[sp] / 10.0;
        P.eta2[sp] = eta[sp] * eta[sp];
        P.eta_s2[sp] = eta_s * eta_s;
    }
    return orc_mirror_hermite_run(n, x, v, m, off, idx, P, dt_soft, p, kmax, stats);
}

static int orc_mirror_hermite_run(int64_t n, double *x, double *v, const double *m,
                           const int64_t *off, const int32_t *idx,
                           orc_mirror_par P, double dt_soft, int p, int kmax,
                           int64_t *stats)
{
    if (n < 0 || p < 0 || kmax < 0 || p + kmax > 60) return -1;
    const double dt_max = ldexp(dt_soft, -p);
    const double tick = ldexp(dt_max, -kmax);
    const int64_t T = (int64_t)1 << (p + kmax);
    const double dm2 = dt_max * dt_max;
    int capped = 0;
    int64_t st[4] = {0, 0, 0, 0};
    double *a = malloc(3 * n * sizeof(double) + 1);
    double *jk = malloc(3 * n * sizeof(double) + 1);
    double *xp = malloc(3 * n * sizeof(double) + 1);
    double *vp = malloc(3 * n * sizeof(double) + 1);
    int64_t *t = malloc(n * sizeof(int64_t) + 1);
    int *lev = malloc(n * sizeof(int) + 1);
    if (!a || !jk || !xp || !vp || !t || !lev) {
        free(a); free(jk); free(xp); free(vp); free(t); free(lev);
        return -1;
    }
    /* start: forces at t = 0 and the first-step levels */
    for (int64_t i = 0; i < n; ++i) {
        t[i] = 0;
        lev[i] = 0;
        if (off[i + 1] == off[i]) continue;
        orc_mirror_hard_one(i, x, v, m, off, idx, &P, a + 3 * i, jk + 3 * i);
        st[2] += off[i + 1] - off[i];
        /* Eq. 20: dt^2 |j|^2 <= eta_s^2 (|a|^2 + a0^2) */
        const int sp = i >= P.n_fs;
        double a0 = P.a0c[sp] * m[i];
        double jj = orc_mirror_dot3(jk + 3 * i, jk + 3 * i);
        double e = P.eta_s2[sp] * fma(a0, a0, orc_mirror_dot3(a + 3 * i, a + 3 * i));
        lev[i] = orc_mirror_level(jj, e, dm2, 0, kmax, &capped);
        st[3] += capped;
    }
    for (;;) {
        int64_t tn = T;
        int any = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (off[i + 1] == off[i] || t[i] == T) continue;
            int64_t e = t[i] + ((int64_t)1 << (kmax - lev[i]));
            if (e < tn) tn = e;
            any = 1;
        }
        if (!any) break;
        ++st[0];
        /* predict every non-isolated particle to tn */
        for (int64_t i = 0; i < n; ++i) {
            if (off[i + 1] == off[i]) continue;
            double d = (double)(tn - t[i]) * tick;
            double d2 = d * d * 0.5;
            double d3 = d * d * d * P.c6;
            for (int c = 0; c < 3; ++c) {
                int64_t k = 3 * i + c;
                xp[k] = fma(jk[k], d3, fma(a[k], d2, fma(v[k], d, x[k])));
                vp[k] = fma(jk[k], d2, fma(a[k], d, v[k]));
            }
        }
        /* evaluate and correct the particles due at tn */
        for (int64_t i = 0; i < n; ++i) {
            if (off[i + 1] == off[i]) continue;
            int64_t step = (int64_t)1 << (kmax - lev[i]);
            if (t[i] + step != tn) continue;
            double a1[3], j1[3];
            orc_mirror_hard_one(i, xp, vp, m, off, idx, &P, a1, j1);
            ++st[1];
            st[2] += off[i + 1] - off[i];
            double h = (double)step * tick;
            double ih = 1.0 / h;
            double ih2 = ih * ih, ih3 = ih2 * ih;
            double h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h;
            double h3c6 = h3 * P.c6, h4c24 = h4 * P.c24, h5c120 = h5 * P.c120;
            double a2[3], a3[3], a2e[3];
            for (int c = 0; c < 3; ++c) {
                int64_t k = 3 * i + c;
                double da = a[k] - a1[c];
                a2[c] = fma(-h, fma(4.0, jk[k], 2.0 * j1[c]), -6.0 * da) * ih2;
                a3[c] = fma(6.0 * h, jk[k] + j1[c], 12.0 * da) * ih3;
                x[k] = fma(a3[c], h5c120, fma(a2[c], h4c24, xp[k]));
                v[k] = fma(a3[c], h4c24, fma(a2[c], h3c6, vp[k]));
                a[k] = a1[c];
                jk[k] = j1[c];
                a2e[c] = fma(a3[c], h, a2[c]);
            }
            t[i] = tn;
            if (tn == T) continue;
            /* Eq. 18, with sqrt(A) sqrt(B) taken as sqrt(A B) and |j| |a3|
             * in the denominator (as the oracle above):
             * dt^2 (sqrt(|j|^2 |a3|^2) + |a2|^2)
             *     <= eta^2 (sqrt((|a|^2 + a0^2) |a2|^2) + |j|^2) */
            const int sp = i >= P.n_fs;
            double a0 = P.a0c[sp] * m[i];
            double aa = orc_mirror_dot3(a1, a1);
            double jj = orc_mirror_dot3(j1, j1);
            double a2sq = orc_mirror_dot3(a2e, a2e);
            double num = sqrt(fma(a0, a0, aa) * a2sq) + jj;
            double den = sqrt(jj * orc_mirror_dot3(a3, a3)) + a2sq;
            int kmin = lev[i] > 0 ? lev[i] - 1 : 0;
            int k = orc_mirror_level(den, P.eta2[sp] * num, dm2, kmin, kmax, &capped);
            st[3] += capped;
            while (tn % ((int64_t)1 << (kmax - k)) != 0) ++k;
            lev[i] = k;
        }
    }
    /* isolated particles drift (Sect. 2.2, step 5) */
    for (int64_t i = 0; i < n; ++i) {
        if (off[i + 1] != off[i]) continue;
        for (int c = 0; c < 3; ++c) x[3 * i + c] = x[3 * i + c] + dt_soft * v[3 * i + c];
    }
    if (stats)
        for (int k = 0; k < 4; ++k) stats[k] = st[k];
    free(a); free(jk); free(xp); free(vp); free(t); free(lev);
    return 0;
}
