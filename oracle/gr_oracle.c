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
