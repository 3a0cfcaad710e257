/*
 * gr_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU implementation of the five readability
 * metrics of "Scalable Readability Evaluation for Graph Layouts: 2D Geometric
 * Distributed Algorithms" (arXiv 2411.09809), Sec. 2.1 and Algorithms 1-5.
 * It exists so that the tests, `__graft_entry__.smoke()` and the CPU-baseline
 * leg of `bench.py` can check and time the CUDA library against something
 * independent.  Nothing in the product path may link, load or call it, and it
 * shares no code, header, table or helper with the CUDA library.
 *
 * Every metric is computed by its plain definition: brute force over all
 * unordered vertex pairs / edge pairs, exact 64-bit integer orientation
 * predicates on int32 coordinates in [0, 65536), FP64 for everything that is
 * not an integer, Neumaier-compensated sums.  No grid, no sort beyond the
 * per-vertex angular sort that the minimum-angle definition itself states.
 * OpenMP parallelises only the outermost loop; per-thread partial results are
 * combined in thread order, so results do not depend on scheduling.
 *
 * Readings of the paper where it is silent or ambiguous (the same readings the
 * library implements):
 *   - edges that share a vertex id never cross (the literal <= 0 predicate of
 *     Algorithm 4 would count every adjacent pair);
 *   - a zero-length edge (distinct ids, coincident coordinates) takes part in
 *     no crossing and no angle; it is reported once per edge;
 *   - a collinear pair whose 1-D extents meet (overlap or a single common
 *     point) is counted in a separate counter, and is NOT part of E_c / E_ca
 *     (Sec. 3.1.4 leaves collinear pairs out);
 *   - E_c = proper crossings + touching pairs (an endpoint on the other
 *     segment), which is what the <= 0 predicate of Algorithm 4 counts;
 *   - the crossing angle is the acute angle between the two lines, in
 *     [0, pi/2] (consistent with the category bounds of Eq. 1);
 *   - E_ca = 1 when E_c = 0;
 *   - M_a = 1 - (1/n) sum d_v over the n vertices with >= 2 non-zero-length
 *     incident edges (Algorithm 2 writes 1 - sum d_v, unnormalised); S and n
 *     are returned so other normalisations are a host division;
 *   - M_l counts every edge once (N_e = |E|, Algorithm 3), l = 0 for a
 *     zero-length edge; M_l = 0 when N_e <= 1 or the mean length is 0.
 *
 * Parity: pinned by the CPU tests against closed forms (K_n in convex
 * position, axis-parallel grids, lattices, stars, two-length edge sets),
 * against a rational-arithmetic brute force that decides intersections by
 * solving the two line equations (a different algorithm), against the known
 * probability 25/108 that two random segments in a square cross, and by
 * invariance under relabelling, reordering, translation, rotation and
 * reflection.  The float-coordinate functions at the end are pinned the same
 * way (see their comment).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_COORD_LIMIT 65536

/* ---------------------------------------------------------------- helpers */

/* Neumaier-compensated accumulator (a published improvement of Kahan
 * summation; Neumaier 1974). */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_value(const nsum *a) { return a->s + a->c; }

static int num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* Orientation of the ordered triple (p, q, r): sign of (q - p) x (r - p).
 * Algorithm 4's CCW(A, B, C) takes the sign of CA x AB, which is the same
 * quantity up to a global sign; Algorithm 4 only ever uses products of two
 * orientations, where a global sign cancels.  Coordinates are < 2^16, so the
 * products are < 2^34 and exact in int64. */
static int orient(int64_t px, int64_t py, int64_t qx, int64_t qy,
                  int64_t rx, int64_t ry)
{
    int64_t v = (qx - px) * (ry - py) - (qy - py) * (rx - px);
    return (v > 0) - (v < 0);
}

/* Lexicographic (x, then y) comparison of two points. */
static int lex_cmp(int64_t ax, int64_t ay, int64_t bx, int64_t by)
{
    if (ax != bx) return ax < bx ? -1 : 1;
    if (ay != by) return ay < by ? -1 : 1;
    return 0;
}

/* Validates a layout: vertex ids in [0, V), no self-loop, coordinates in
 * [0, 65536).  Returns 0 when valid, 1 for a bad id / self-loop, 2 for a
 * coordinate out of range. */
int oracle_validate(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E)
{
    for (int64_t v = 0; v < V; ++v)
        for (int k = 0; k < 2; ++k)
            if (xy[2 * v + k] < 0 || xy[2 * v + k] >= ORACLE_COORD_LIMIT) return 2;
    for (int64_t e = 0; e < E; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= V || b >= V || a == b) return 1;
    }
    return 0;
}

/* ------------------------------------------------------ node occlusion N_c */

/* Sec. 2.1 and Algorithm 1: the number of unordered vertex pairs {v, u},
 * v < u, with ||p_v - p_u||^2 < (2r)^2.  `d` is the diameter 2r; the
 * inequality is strict.  Returns -1 for d < 0. */
int64_t oracle_node_occlusion(const int32_t *xy, int64_t V, int64_t d)
{
    if (d < 0) return -1;
    const int64_t d2 = d * d;
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t v = 0; v < V; ++v) {
        const int64_t xv = xy[2 * v], yv = xy[2 * v + 1];
        for (int64_t u = v + 1; u < V; ++u) {
            const int64_t dx = xv - xy[2 * u], dy = yv - xy[2 * u + 1];
            if (dx * dx + dy * dy < d2) ++total;
        }
    }
    return total;
}

/* ------------------------------------------- edge crossings E_c and E_ca */

enum { PAIR_NONE = 0, PAIR_PROPER = 1, PAIR_TOUCHING = 2, PAIR_COLLINEAR = 3 };

/* Classifies the unordered edge pair {e, f} (Algorithm 4's join predicate,
 * with the readings stated in the file header).  For PAIR_PROPER and
 * PAIR_TOUCHING, *angle receives the acute crossing angle a_c in [0, pi/2]
 * (Sec. 3.1.5): atan2(|u x v|, |u . v|) of the exact integer cross and dot
 * products of the two direction vectors. */
static int classify_pair(const int32_t *xy, const int32_t *e, const int32_t *f,
                         double *angle)
{
    const int32_t ia = e[0], ib = e[1], ic = f[0], id = f[1];
    if (ia == ic || ia == id || ib == ic || ib == id) return PAIR_NONE;

    const int64_t ax = xy[2 * ia], ay = xy[2 * ia + 1];
    const int64_t bx = xy[2 * ib], by = xy[2 * ib + 1];
    const int64_t cx = xy[2 * ic], cy = xy[2 * ic + 1];
    const int64_t dx = xy[2 * id], dy = xy[2 * id + 1];
    if ((ax == bx && ay == by) || (cx == dx && cy == dy)) return PAIR_NONE;

    const int o1 = orient(ax, ay, bx, by, cx, cy);
    const int o2 = orient(ax, ay, bx, by, dx, dy);
    const int o3 = orient(cx, cy, dx, dy, ax, ay);
    const int o4 = orient(cx, cy, dx, dy, bx, by);

    if (o1 == 0 && o2 == 0 && o3 == 0 && o4 == 0) {
        /* Both segments lie on one line; lexicographic order is a linear
         * order along that line, so the segments meet iff the larger of the
         * two lexicographic minima is <= the smaller of the two maxima. */
        int64_t e_lo_x = ax, e_lo_y = ay, e_hi_x = bx, e_hi_y = by;
        if (lex_cmp(bx, by, ax, ay) < 0) { e_lo_x = bx; e_lo_y = by; e_hi_x = ax; e_hi_y = ay; }
        int64_t f_lo_x = cx, f_lo_y = cy, f_hi_x = dx, f_hi_y = dy;
        if (lex_cmp(dx, dy, cx, cy) < 0) { f_lo_x = dx; f_lo_y = dy; f_hi_x = cx; f_hi_y = cy; }
        int64_t lo_x = e_lo_x, lo_y = e_lo_y;
        if (lex_cmp(f_lo_x, f_lo_y, lo_x, lo_y) > 0) { lo_x = f_lo_x; lo_y = f_lo_y; }
        int64_t hi_x = e_hi_x, hi_y = e_hi_y;
        if (lex_cmp(f_hi_x, f_hi_y, hi_x, hi_y) < 0) { hi_x = f_hi_x; hi_y = f_hi_y; }
        return lex_cmp(lo_x, lo_y, hi_x, hi_y) <= 0 ? PAIR_COLLINEAR : PAIR_NONE;
    }

    int kind;
    if (o1 * o2 < 0 && o3 * o4 < 0)
        kind = PAIR_PROPER;
    else if (o1 * o2 <= 0 && o3 * o4 <= 0)
        kind = PAIR_TOUCHING;
    else
        return PAIR_NONE;

    const int64_t ux = bx - ax, uy = by - ay, vx = dx - cx, vy = dy - cy;
    const int64_t cross = ux * vy - uy * vx;
    const int64_t dot = ux * vx + uy * vy;
    *angle = atan2(fabs((double)cross), fabs((double)dot));
    return kind;
}

static int64_t count_zero_length(const int32_t *xy, const int32_t *edges, int64_t E)
{
    int64_t z = 0;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (xy[2 * a] == xy[2 * b] && xy[2 * a + 1] == xy[2 * b + 1]) ++z;
    }
    return z;
}

/* Edge crossings (Sec. 2.1, Algorithm 4) and edge crossing angle (Sec. 2.1,
 * Algorithm 5) by brute force over all unordered edge pairs e < f.
 *   counts[0] = proper crossings, counts[1] = touching pairs,
 *   counts[2] = collinear overlaps, counts[3] = zero-length edges,
 *   counts[4] = E_c = proper + touching.
 *   fvals[0]  = sum over the E_c pairs of |ideal - a_c| (radians),
 *   fvals[1]  = E_ca = 1 - (1 / E_c) sum |ideal - a_c| / ideal (1 if E_c = 0).
 * Returns 0, or -1 for ideal outside (0, pi/2]. */
int oracle_crossings(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E,
                     double ideal, int64_t *counts, double *fvals)
{
    (void)V;
    if (!(ideal > 0.0 && ideal <= M_PI / 2 + 1e-15)) return -1;
    const int nt = num_threads();
    int64_t *acc = calloc((size_t)nt * 3, sizeof(int64_t));
    nsum *sums = calloc((size_t)nt, sizeof(nsum));
#pragma omp parallel
    {
        const int t = thread_id();
        int64_t proper = 0, touching = 0, collinear = 0;
        nsum s = {0.0, 0.0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < E; ++i) {
            for (int64_t j = i + 1; j < E; ++j) {
                double ac = 0.0;
                const int k = classify_pair(xy, edges + 2 * i, edges + 2 * j, &ac);
                if (k == PAIR_PROPER) { ++proper; nsum_add(&s, fabs(ideal - ac)); }
                else if (k == PAIR_TOUCHING) { ++touching; nsum_add(&s, fabs(ideal - ac)); }
                else if (k == PAIR_COLLINEAR) ++collinear;
            }
        }
        acc[3 * t] = proper; acc[3 * t + 1] = touching; acc[3 * t + 2] = collinear;
        sums[t] = s;
    }
    int64_t proper = 0, touching = 0, collinear = 0;
    nsum total = {0.0, 0.0};
    for (int t = 0; t < nt; ++t) {
        proper += acc[3 * t]; touching += acc[3 * t + 1]; collinear += acc[3 * t + 2];
        nsum_add(&total, sums[t].s);
        nsum_add(&total, sums[t].c);
    }
    free(acc); free(sums);
    const int64_t ec = proper + touching;
    counts[0] = proper; counts[1] = touching; counts[2] = collinear;
    counts[3] = count_zero_length(xy, edges, E); counts[4] = ec;
    const double dev = nsum_value(&total);
    fvals[0] = dev;
    fvals[1] = ec > 0 ? 1.0 - dev / (ideal * (double)ec) : 1.0;
    return 0;
}

/* Per-edge crossing data for a sample of edges: for each sampled edge e,
 * over all f != e, the number of proper crossings, touching pairs and
 * collinear overlaps it takes part in, and the sum of |ideal - a_c| over its
 * E_c partners.  Used to check large layouts edge by edge. */
int oracle_crossings_of_edges(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E,
                              double ideal, const int64_t *sample, int64_t n_sample,
                              int64_t *out_counts /* [n_sample][3] */,
                              double *out_dev /* [n_sample] */)
{
    (void)V;
    if (!(ideal > 0.0 && ideal <= M_PI / 2 + 1e-15)) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_sample; ++s) {
        const int64_t e = sample[s];
        int64_t proper = 0, touching = 0, collinear = 0;
        nsum dev = {0.0, 0.0};
        for (int64_t f = 0; f < E; ++f) {
            if (f == e) continue;
            double ac = 0.0;
            const int k = classify_pair(xy, edges + 2 * e, edges + 2 * f, &ac);
            if (k == PAIR_PROPER) { ++proper; nsum_add(&dev, fabs(ideal - ac)); }
            else if (k == PAIR_TOUCHING) { ++touching; nsum_add(&dev, fabs(ideal - ac)); }
            else if (k == PAIR_COLLINEAR) ++collinear;
        }
        out_counts[3 * s] = proper; out_counts[3 * s + 1] = touching;
        out_counts[3 * s + 2] = collinear;
        out_dev[s] = nsum_value(&dev);
    }
    return 0;
}

/* ------------------------------------------------------- minimum angle M_a */

typedef struct { int64_t x, y; int64_t edge; } dir_t;

/* 0 for directions with angle in [0, pi), 1 for [pi, 2 pi). */
static int half_plane(int64_t x, int64_t y) { return (y < 0 || (y == 0 && x < 0)) ? 1 : 0; }

/* Exact order of directions by their angle with the x-axis in [0, 2 pi);
 * equal directions are ordered by edge index. */
static int dir_cmp(const void *pa, const void *pb)
{
    const dir_t *a = pa, *b = pb;
    const int ha = half_plane(a->x, a->y), hb = half_plane(b->x, b->y);
    if (ha != hb) return ha - hb;
    const int64_t c = a->x * b->y - a->y * b->x;
    if (c > 0) return -1;
    if (c < 0) return 1;
    return (a->edge > b->edge) - (a->edge < b->edge);
}

/* Counter-clockwise angle from direction p to direction q, in [0, 2 pi). */
static double ccw_gap(const dir_t *p, const dir_t *q)
{
    const double cr = (double)(p->x * q->y - p->y * q->x);
    const double dt = (double)(p->x * q->x + p->y * q->y);
    double g = atan2(cr, dt);
    if (g < 0) g += 2.0 * M_PI;
    return g;
}

/* Minimum angle (Sec. 2.1, Algorithm 2).  For every vertex v: collect the
 * directions of its non-zero-length incident edges, sort them by angle,
 * take the smallest counter-clockwise gap between neighbours in sorted
 * order, the wrap-around gap included (GetMinAngle), and
 * d_v = (2 pi / deg - min) / (2 pi / deg).  A vertex of degree 1 has a single
 * gap of 2 pi, so d_v = 0.  out[0] = M_a = 1 - S / n, out[1] = S = sum d_v,
 * out[2] = n = number of vertices with deg >= 2 (M_a = 1 when n = 0). */
int oracle_min_angle(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E,
                     double *out)
{
    int64_t *deg = calloc((size_t)V + 1, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (xy[2 * a] == xy[2 * b] && xy[2 * a + 1] == xy[2 * b + 1]) continue;
        deg[a]++; deg[b]++;
    }
    int64_t *off = malloc(sizeof(int64_t) * ((size_t)V + 1));
    off[0] = 0;
    for (int64_t v = 0; v < V; ++v) off[v + 1] = off[v] + deg[v];
    dir_t *dirs = malloc(sizeof(dir_t) * ((size_t)off[V] + 1));
    int64_t *fill = calloc((size_t)V + 1, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        const int64_t dx = (int64_t)xy[2 * b] - xy[2 * a], dy = (int64_t)xy[2 * b + 1] - xy[2 * a + 1];
        if (dx == 0 && dy == 0) continue;
        dirs[off[a] + fill[a]++] = (dir_t){dx, dy, e};
        dirs[off[b] + fill[b]++] = (dir_t){-dx, -dy, e};
    }
    nsum S = {0.0, 0.0};
    int64_t n = 0;
    for (int64_t v = 0; v < V; ++v) {
        const int64_t k = deg[v];
        if (k < 2) continue;
        dir_t *d = dirs + off[v];
        qsort(d, (size_t)k, sizeof(dir_t), dir_cmp);
        double mn = ccw_gap(&d[k - 1], &d[0]);
        for (int64_t i = 1; i < k; ++i) {
            const double g = ccw_gap(&d[i - 1], &d[i]);
            if (g < mn) mn = g;
        }
        const double ideal = 2.0 * M_PI / (double)k;
        nsum_add(&S, (ideal - mn) / ideal);
        ++n;
    }
    free(deg); free(off); free(dirs); free(fill);
    const double s = nsum_value(&S);
    out[0] = n > 0 ? 1.0 - s / (double)n : 1.0;
    out[1] = s;
    out[2] = (double)n;
    return 0;
}

/* ------------------------------------------------ edge length variation M_l */

/* Edge length variation (Sec. 2.1, Algorithm 3): with l_e the Euclidean
 * length of edge e, N_e = |E| and l_mu the mean,
 * M_l = sqrt(sum_e (l_e - l_mu)^2 / (N_e l_mu^2)) / sqrt(N_e - 1).
 * Two passes; 0 when N_e <= 1 or l_mu = 0. */
double oracle_edge_length_variation(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E)
{
    (void)V;
    if (E <= 1) return 0.0;
    nsum sl = {0.0, 0.0};
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        const double dx = (double)xy[2 * b] - xy[2 * a], dy = (double)xy[2 * b + 1] - xy[2 * a + 1];
        nsum_add(&sl, sqrt(dx * dx + dy * dy));
    }
    const double mu = nsum_value(&sl) / (double)E;
    if (mu == 0.0) return 0.0;
    nsum ss = {0.0, 0.0};
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        const double dx = (double)xy[2 * b] - xy[2 * a], dy = (double)xy[2 * b + 1] - xy[2 * a + 1];
        const double t = sqrt(dx * dx + dy * dy) - mu;
        nsum_add(&ss, t * t);
    }
    return sqrt(nsum_value(&ss) / ((double)E * mu * mu)) / sqrt((double)E - 1.0);
}

/* Threads OpenMP will use (reported beside CPU timings). */
int oracle_num_threads(void) { return num_threads(); }

/* ======================================================================
 * FP32 coordinates: the differentiable form (any finite coordinates).
 *
 * Orientation signs on FP32 inputs are decided exactly with floating-point
 * expansion arithmetic (Shewchuk, "Adaptive Precision Floating-Point
 * Arithmetic and Fast Robust Geometric Predicates", 1997): the inputs are
 * exact in FP64, every difference is carried as a two-term expansion
 * (two_diff), every product of terms as a two-term expansion (two_prod with
 * a fused multiply-add), and the terms are summed into a non-overlapping
 * expansion (grow_expansion) whose largest component carries the sign.
 * Parity: pinned by the CPU tests against exact rational arithmetic
 * (Python fractions) on random FP32 inputs spanning many exponents and on
 * exactly collinear constructions, and the FP32 metrics against the
 * integer oracle on coordinates k / 65536 (the same geometry scaled by a
 * power of two).  The gradients are pinned against central differences of
 * this FP64 forward.
 * ====================================================================== */

static void two_sum(double a, double b, double *x, double *y)
{
    const double s = a + b;
    const double bv = s - a;
    const double av = s - bv;
    *x = s;
    *y = (a - av) + (b - bv);
}

static void two_prod(double a, double b, double *x, double *y)
{
    const double p = a * b;
    *x = p;
    *y = fma(a, b, -p);
}

/* h = e + b for a non-overlapping expansion e of n components sorted by
 * increasing magnitude; zero components are dropped.  Returns |h|. */
static int grow_expansion(int n, const double *e, double b, double *h)
{
    double q = b;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        double s, t;
        two_sum(q, e[i], &s, &t);
        q = s;
        if (t != 0.0) h[m++] = t;
    }
    if (q != 0.0 || m == 0) h[m++] = q;
    return m;
}

/* Exact sign of (b - a) x (c - a) for FP32 points, always by expansions. */
int oracle_orient_f32_exact(float ax, float ay, float bx, float by, float cx, float cy)
{
    double u[2][2], w[2][2];  /* u = b - a, w = c - a as two-term expansions (hi, lo) */
    two_sum((double)bx, -(double)ax, &u[0][0], &u[0][1]);
    two_sum((double)by, -(double)ay, &u[1][0], &u[1][1]);
    two_sum((double)cx, -(double)ax, &w[0][0], &w[0][1]);
    two_sum((double)cy, -(double)ay, &w[1][0], &w[1][1]);
    /* det = u_x w_y - u_y w_x: 16 two-term products */
    double e[40], h[40];
    int n = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double p, q;
            two_prod(u[0][i], w[1][j], &p, &q);
            n = grow_expansion(n, e, p, h); memcpy(e, h, sizeof(double) * n);
            n = grow_expansion(n, e, q, h); memcpy(e, h, sizeof(double) * n);
            two_prod(-u[1][i], w[0][j], &p, &q);
            n = grow_expansion(n, e, p, h); memcpy(e, h, sizeof(double) * n);
            n = grow_expansion(n, e, q, h); memcpy(e, h, sizeof(double) * n);
        }
    const double top = e[n - 1];
    return (top > 0) - (top < 0);
}

/* Exact sign of (b - a) x (c - a) for FP32 points: Shewchuk's adaptive
 * scheme, first stage.  The determinant t1 - t2 evaluated in FP64 (unit
 * roundoff e = 2^-53) carries the true sign whenever its magnitude exceeds
 * (3 + 16 e) e (|t1| + |t2|) (Shewchuk 1997, the orient2d error bound; FP32
 * inputs can neither underflow nor overflow FP64 here).  Otherwise the
 * expansion evaluation above decides. */
int oracle_orient_f32(float ax, float ay, float bx, float by, float cx, float cy)
{
    const double e = 1.1102230246251565e-16;  /* 2^-53 */
    const double t1 = ((double)bx - (double)ax) * ((double)cy - (double)ay);
    const double t2 = ((double)by - (double)ay) * ((double)cx - (double)ax);
    const double det = t1 - t2;
    const double bound = (3.0 + 16.0 * e) * e * (fabs(t1) + fabs(t2));
    if (det > bound) return 1;
    if (-det > bound) return -1;
    return oracle_orient_f32_exact(ax, ay, bx, by, cx, cy);
}

static int lex_cmp_f(float ax, float ay, float bx, float by)
{
    if (ax != bx) return ax < bx ? -1 : 1;
    if (ay != by) return ay < by ? -1 : 1;
    return 0;
}

/* Classification of an edge pair with FP32 coordinates: the rules of
 * classify_pair with exact orientations; the angle from FP64 cross and dot
 * products of the FP64 direction vectors. */
static int classify_pair_f32(const float *xy, const int32_t *e, const int32_t *f, double *angle)
{
    const int32_t ia = e[0], ib = e[1], ic = f[0], id = f[1];
    if (ia == ic || ia == id || ib == ic || ib == id) return PAIR_NONE;
    const float ax = xy[2 * ia], ay = xy[2 * ia + 1], bx = xy[2 * ib], by = xy[2 * ib + 1];
    const float cx = xy[2 * ic], cy = xy[2 * ic + 1], dx = xy[2 * id], dy = xy[2 * id + 1];
    if ((ax == bx && ay == by) || (cx == dx && cy == dy)) return PAIR_NONE;
    const int o1 = oracle_orient_f32(ax, ay, bx, by, cx, cy);
    const int o2 = oracle_orient_f32(ax, ay, bx, by, dx, dy);
    const int o3 = oracle_orient_f32(cx, cy, dx, dy, ax, ay);
    const int o4 = oracle_orient_f32(cx, cy, dx, dy, bx, by);
    if (o1 == 0 && o2 == 0 && o3 == 0 && o4 == 0) {
        float elx = ax, ely = ay, ehx = bx, ehy = by;
        if (lex_cmp_f(bx, by, ax, ay) < 0) { elx = bx; ely = by; ehx = ax; ehy = ay; }
        float flx = cx, fly = cy, fhx = dx, fhy = dy;
        if (lex_cmp_f(dx, dy, cx, cy) < 0) { flx = dx; fly = dy; fhx = cx; fhy = cy; }
        float lx = elx, ly = ely;
        if (lex_cmp_f(flx, fly, lx, ly) > 0) { lx = flx; ly = fly; }
        float hx = ehx, hy = ehy;
        if (lex_cmp_f(fhx, fhy, hx, hy) < 0) { hx = fhx; hy = fhy; }
        return lex_cmp_f(lx, ly, hx, hy) <= 0 ? PAIR_COLLINEAR : PAIR_NONE;
    }
    int kind;
    if (o1 * o2 < 0 && o3 * o4 < 0) kind = PAIR_PROPER;
    else if (o1 * o2 <= 0 && o3 * o4 <= 0) kind = PAIR_TOUCHING;
    else return PAIR_NONE;
    const double ux = (double)bx - ax, uy = (double)by - ay, vx = (double)dx - cx, vy = (double)dy - cy;
    *angle = atan2(fabs(ux * vy - uy * vx), fabs(ux * vx + uy * vy));
    return kind;
}

/* Row i of the pair triangle (pairs (i, j), j > i) on FP32 coordinates:
 * class counts into c[0..2] (proper, touching, collinear), |ideal - a_c|
 * into s, and, when `out` is not NULL, the first `limit` E_c pairs of the
 * row (in increasing j) into out. */
static void crossings_row_f32(const float *xy, const int32_t *edges, int64_t E, int64_t i, double ideal,
                              int64_t *c, nsum *s, int32_t *out, int64_t limit)
{
    int64_t n = 0;
    for (int64_t j = i + 1; j < E; ++j) {
        double ac = 0.0;
        const int k = classify_pair_f32(xy, edges + 2 * i, edges + 2 * j, &ac);
        if (k == PAIR_COLLINEAR) { ++c[2]; continue; }
        if (k == PAIR_NONE) continue;
        ++c[k == PAIR_PROPER ? 0 : 1];
        nsum_add(s, fabs(ideal - ac));
        if (out && n < limit) { out[2 * n] = (int32_t)i; out[2 * n + 1] = (int32_t)j; }
        ++n;
    }
}

/* Edge crossings and crossing angle on FP32 coordinates; counts/fvals as
 * oracle_crossings.  When `pairs` is not NULL, the E_c pairs (edge indices,
 * e < f, in increasing (e, f) order) are written to it, at most max_pairs of
 * them: a second pass over the rows, each starting at its offset. */
static int crossings_f32_impl(const float *xy, const int32_t *edges, int64_t E, double ideal, int64_t *counts,
                              double *fvals, int32_t *pairs, int64_t max_pairs, int32_t **alloc_pairs)
{
    if (!(ideal > 0.0 && ideal <= M_PI / 2 + 1e-15)) return -1;
    const int nt = num_threads();
    int64_t *acc = calloc((size_t)nt * 3, sizeof(int64_t));
    nsum *sums = calloc((size_t)nt, sizeof(nsum));
    int64_t *row = (pairs || alloc_pairs) ? calloc((size_t)E + 1, sizeof(int64_t)) : NULL;
#pragma omp parallel
    {
        const int t = thread_id();
        int64_t c[3] = {0, 0, 0};
        nsum s = {0.0, 0.0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < E; ++i) {
            const int64_t before = c[0] + c[1];
            crossings_row_f32(xy, edges, E, i, ideal, c, &s, NULL, 0);
            if (row) row[i] = c[0] + c[1] - before;
        }
        acc[3 * t] = c[0]; acc[3 * t + 1] = c[1]; acc[3 * t + 2] = c[2];
        sums[t] = s;
    }
    int64_t proper = 0, touching = 0, collinear = 0, zero = 0;
    nsum total = {0.0, 0.0};
    for (int t = 0; t < nt; ++t) {
        proper += acc[3 * t]; touching += acc[3 * t + 1]; collinear += acc[3 * t + 2];
        nsum_add(&total, sums[t].s);
        nsum_add(&total, sums[t].c);
    }
    free(acc); free(sums);
    if (alloc_pairs) {  /* a buffer of exactly E_c pairs, owned by the caller */
        max_pairs = proper + touching;
        pairs = malloc(sizeof(int32_t) * 2 * (size_t)(max_pairs > 0 ? max_pairs : 1));
        *alloc_pairs = pairs;
    }
    if (row) {
        int64_t off = 0;  /* exclusive offsets of the rows */
        for (int64_t i = 0; i < E; ++i) { const int64_t n = row[i]; row[i] = off; off += n; }
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < E; ++i) {
            if (row[i] >= max_pairs) continue;
            int64_t c[3] = {0, 0, 0};
            nsum s = {0.0, 0.0};
            crossings_row_f32(xy, edges, E, i, ideal, c, &s, pairs + 2 * row[i], max_pairs - row[i]);
        }
        free(row);
    }
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (xy[2 * a] == xy[2 * b] && xy[2 * a + 1] == xy[2 * b + 1]) ++zero;
    }
    const int64_t ec = proper + touching;
    counts[0] = proper; counts[1] = touching; counts[2] = collinear; counts[3] = zero; counts[4] = ec;
    fvals[0] = nsum_value(&total);
    fvals[1] = ec > 0 ? 1.0 - fvals[0] / (ideal * (double)ec) : 1.0;
    return 0;
}

int oracle_crossings_f32(const float *xy, int64_t V, const int32_t *edges, int64_t E, double ideal,
                         int64_t *counts, double *fvals, int32_t *pairs, int64_t max_pairs)
{
    (void)V;
    return crossings_f32_impl(xy, edges, E, ideal, counts, fvals, pairs, max_pairs, NULL);
}

/* Direction angle of (dx, dy) in [0, 2 pi). */
static double dir_angle(double dx, double dy)
{
    double t = atan2(dy, dx);
    if (t < 0) t += 2.0 * M_PI;
    return t;
}

typedef struct { double ang; int32_t other; int64_t edge; } fdir_t;

static int fdir_cmp(const void *pa, const void *pb)
{
    const fdir_t *a = pa, *b = pb;
    if (a->ang != b->ang) return a->ang < b->ang ? -1 : 1;
    return (a->edge > b->edge) - (a->edge < b->edge);
}

/* Minimum angle on FP32 coordinates (Algorithm 2 with FP64 direction angles
 * sorted, the smallest gap including the wrap-around one).  out as
 * oracle_min_angle.  When `arg` is not NULL, arg[v] = (i, j): the vertices
 * at the far ends of the two edges whose directions bound v's smallest gap
 * (the gap runs counter-clockwise from the edge to i to the edge to j), or
 * (-1, -1) for vertices with fewer than two edges. */
int oracle_min_angle_f32(const float *xy, int64_t V, const int32_t *edges, int64_t E, double *out, int32_t *arg)
{
    int64_t *deg = calloc((size_t)V + 1, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (xy[2 * a] == xy[2 * b] && xy[2 * a + 1] == xy[2 * b + 1]) continue;
        deg[a]++; deg[b]++;
    }
    int64_t *off = malloc(sizeof(int64_t) * ((size_t)V + 1));
    off[0] = 0;
    for (int64_t v = 0; v < V; ++v) off[v + 1] = off[v] + deg[v];
    fdir_t *d = malloc(sizeof(fdir_t) * ((size_t)off[V] + 1));
    int64_t *fill = calloc((size_t)V + 1, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        const double dx = (double)xy[2 * b] - xy[2 * a], dy = (double)xy[2 * b + 1] - xy[2 * a + 1];
        if (dx == 0 && dy == 0) continue;
        d[off[a] + fill[a]++] = (fdir_t){dir_angle(dx, dy), b, e};
        d[off[b] + fill[b]++] = (fdir_t){dir_angle(-dx, -dy), a, e};
    }
    nsum S = {0.0, 0.0};
    int64_t n = 0;
    for (int64_t v = 0; v < V; ++v) {
        const int64_t k = deg[v];
        if (arg) { arg[2 * v] = -1; arg[2 * v + 1] = -1; }
        if (k < 2) continue;
        fdir_t *q = d + off[v];
        qsort(q, (size_t)k, sizeof(fdir_t), fdir_cmp);
        double mn = 2.0 * M_PI - q[k - 1].ang + q[0].ang;
        int32_t bi = q[k - 1].other, bj = q[0].other;
        for (int64_t i = 1; i < k; ++i) {
            const double g = q[i].ang - q[i - 1].ang;
            if (g < mn) { mn = g; bi = q[i - 1].other; bj = q[i].other; }
        }
        const double ideal = 2.0 * M_PI / (double)k;
        nsum_add(&S, (ideal - mn) / ideal);
        ++n;
        if (arg) { arg[2 * v] = bi; arg[2 * v + 1] = bj; }
    }
    free(deg); free(off); free(d); free(fill);
    const double s = nsum_value(&S);
    out[0] = n > 0 ? 1.0 - s / (double)n : 1.0;
    out[1] = s;
    out[2] = (double)n;
    return 0;
}

double oracle_edge_length_variation_f32(const float *xy, int64_t V, const int32_t *edges, int64_t E)
{
    (void)V;
    if (E <= 1) return 0.0;
    nsum sl = {0.0, 0.0};
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        const double dx = (double)xy[2 * b] - xy[2 * a], dy = (double)xy[2 * b + 1] - xy[2 * a + 1];
        nsum_add(&sl, sqrt(dx * dx + dy * dy));
    }
    const double mu = nsum_value(&sl) / (double)E;
    if (mu == 0.0) return 0.0;
    nsum ss = {0.0, 0.0};
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        const double dx = (double)xy[2 * b] - xy[2 * a], dy = (double)xy[2 * b + 1] - xy[2 * a + 1];
        const double t = sqrt(dx * dx + dy * dy) - mu;
        nsum_add(&ss, t * t);
    }
    return sqrt(nsum_value(&ss) / ((double)E * mu * mu)) / sqrt((double)E - 1.0);
}

/* Gradient of (theta(q - p)) with respect to q, for the direction angle of
 * the vector q - p: (-dy, dx) / |q - p|^2; with respect to p it is the
 * negative. */
static void dtheta(double dx, double dy, double *gx, double *gy)
{
    const double r2 = dx * dx + dy * dy;
    *gx = -dy / r2;
    *gy = dx / r2;
}

/* The three terms of the differentiable loss and their gradients with
 * respect to every coordinate (FP64), with the crossing set and every
 * vertex's smallest gap held fixed:
 *   terms[0] = E_ca, terms[1] = M_l, terms[2] = M_a;
 *   g_eca, g_ml, g_ma: [V][2] gradients of E_ca, M_l and M_a.
 * E_ca: a_c is the acute angle between the lines, a function of the two
 * direction angles; d|ideal - a_c| / d a_c = sign(a_c - ideal) (0 at 0).
 * M_l: with S = sum (l_e - mu)^2, dM_l / dl_e = M_l ((l_e - mu) / S - 1 / (N mu)).
 * M_a: d(M_a) / d(min_v) = deg_v / (2 pi n) for each counted vertex; the
 * gap runs counter-clockwise between two fixed incident edges. */
int oracle_diff_terms_and_grads(const float *xy, int64_t V, const int32_t *edges, int64_t E, double ideal,
                                double *terms, double *g_eca, double *g_ml, double *g_ma, int64_t *counts_out)
{
    memset(g_eca, 0, sizeof(double) * 2 * (size_t)V);
    memset(g_ml, 0, sizeof(double) * 2 * (size_t)V);
    memset(g_ma, 0, sizeof(double) * 2 * (size_t)V);
    /* E_ca and its gradient */
    int64_t counts[5];
    double fv[2];
    int32_t *pairs = NULL;
    if (crossings_f32_impl(xy, edges, E, ideal, counts, fv, NULL, 0, &pairs) != 0) return -1;
    const int64_t ec = counts[4];
    if (counts_out) memcpy(counts_out, counts, sizeof(counts));
    terms[0] = fv[1];
    for (int64_t p = 0; p < ec; ++p) {
        const int32_t *e = edges + 2 * pairs[2 * p], *f = edges + 2 * pairs[2 * p + 1];
        const int32_t a = e[0], b = e[1], c = f[0], d = f[1];
        const double ux = (double)xy[2 * b] - xy[2 * a], uy = (double)xy[2 * b + 1] - xy[2 * a + 1];
        const double vx = (double)xy[2 * d] - xy[2 * c], vy = (double)xy[2 * d + 1] - xy[2 * c + 1];
        /* a_c = acute angle between the lines; delta = theta_u - theta_v mod pi */
        double delta = fmod(dir_angle(ux, uy) - dir_angle(vx, vy), M_PI);
        if (delta < 0) delta += M_PI;
        const double ac = delta <= M_PI / 2 ? delta : M_PI - delta;
        const double s_ac = delta <= M_PI / 2 ? 1.0 : -1.0; /* d a_c / d theta_u */
        const double dev_sign = ac > ideal ? 1.0 : (ac < ideal ? -1.0 : 0.0);
        /* E_ca = 1 - sum |ideal - a_c| / (ideal E_c) */
        const double coef = -dev_sign * s_ac / (ideal * (double)ec);
        double gux, guy, gvx, gvy;
        dtheta(ux, uy, &gux, &guy);
        dtheta(vx, vy, &gvx, &gvy);
        g_eca[2 * b] += coef * gux; g_eca[2 * b + 1] += coef * guy;
        g_eca[2 * a] -= coef * gux; g_eca[2 * a + 1] -= coef * guy;
        g_eca[2 * d] -= coef * gvx; g_eca[2 * d + 1] -= coef * gvy;
        g_eca[2 * c] += coef * gvx; g_eca[2 * c + 1] += coef * gvy;
    }
    free(pairs);
    /* M_l and its gradient */
    terms[1] = oracle_edge_length_variation_f32(xy, V, edges, E);
    if (E > 1) {
        nsum sl = {0.0, 0.0};
        for (int64_t e = 0; e < E; ++e) {
            const double dx = (double)xy[2 * edges[2 * e + 1]] - xy[2 * edges[2 * e]];
            const double dy = (double)xy[2 * edges[2 * e + 1] + 1] - xy[2 * edges[2 * e] + 1];
            nsum_add(&sl, sqrt(dx * dx + dy * dy));
        }
        const double mu = nsum_value(&sl) / (double)E;
        nsum ss = {0.0, 0.0};
        for (int64_t e = 0; e < E; ++e) {
            const double dx = (double)xy[2 * edges[2 * e + 1]] - xy[2 * edges[2 * e]];
            const double dy = (double)xy[2 * edges[2 * e + 1] + 1] - xy[2 * edges[2 * e] + 1];
            const double t = sqrt(dx * dx + dy * dy) - mu;
            nsum_add(&ss, t * t);
        }
        const double S = nsum_value(&ss), Ml = terms[1];
        if (S > 0 && mu > 0) {
            for (int64_t e = 0; e < E; ++e) {
                const int32_t a = edges[2 * e], b = edges[2 * e + 1];
                const double dx = (double)xy[2 * b] - xy[2 * a], dy = (double)xy[2 * b + 1] - xy[2 * a + 1];
                const double l = sqrt(dx * dx + dy * dy);
                if (l == 0.0) continue;
                const double dl = Ml * ((l - mu) / S - 1.0 / ((double)E * mu));
                g_ml[2 * b] += dl * dx / l; g_ml[2 * b + 1] += dl * dy / l;
                g_ml[2 * a] -= dl * dx / l; g_ml[2 * a + 1] -= dl * dy / l;
            }
        }
    }
    /* M_a and its gradient */
    double ma[3];
    int32_t *arg = malloc(sizeof(int32_t) * 2 * (size_t)(V > 0 ? V : 1));
    oracle_min_angle_f32(xy, V, edges, E, ma, arg);
    terms[2] = ma[0];
    const int64_t n = (int64_t)ma[2];
    if (n > 0) {
        int64_t *deg = calloc((size_t)V + 1, sizeof(int64_t));
        for (int64_t e = 0; e < E; ++e) {
            const int32_t a = edges[2 * e], b = edges[2 * e + 1];
            if (xy[2 * a] == xy[2 * b] && xy[2 * a + 1] == xy[2 * b + 1]) continue;
            deg[a]++; deg[b]++;
        }
        for (int64_t v = 0; v < V; ++v) {
            if (arg[2 * v] < 0) continue;
            const int32_t i = arg[2 * v], j = arg[2 * v + 1];
            /* min_v = theta(p_j - p_v) - theta(p_i - p_v) (mod 2 pi) */
            const double c = (double)deg[v] / (2.0 * M_PI * (double)n);
            double gix, giy, gjx, gjy;
            dtheta((double)xy[2 * i] - xy[2 * v], (double)xy[2 * i + 1] - xy[2 * v + 1], &gix, &giy);
            dtheta((double)xy[2 * j] - xy[2 * v], (double)xy[2 * j + 1] - xy[2 * v + 1], &gjx, &gjy);
            g_ma[2 * j] += c * gjx; g_ma[2 * j + 1] += c * gjy;
            g_ma[2 * v] -= c * gjx; g_ma[2 * v + 1] -= c * gjy;
            g_ma[2 * i] -= c * gix; g_ma[2 * i + 1] -= c * giy;
            g_ma[2 * v] += c * gix; g_ma[2 * v + 1] += c * giy;
        }
        free(deg);
    }
    free(arg);
    return 0;
}
