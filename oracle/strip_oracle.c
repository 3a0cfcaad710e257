/*
 * strip_oracle.c -- TEST INFRASTRUCTURE ONLY (part of the oracle library).
 *
 * The approximate "enhanced" edge-crossing and crossing-angle algorithms of
 * arXiv 2411.09809, Sec. 3.2.2 and Sec. 3.2.3, followed step by step on the
 * CPU.  Nothing in the product path may link, load or call it; it shares no
 * code with the CUDA library.
 *
 * Sec. 3.2.2.  The plane is cut only vertically, by the lines x = s * l
 * (strip s spans [s l, (s + 1) l]).  Two segments are comparable in strip s
 * when both cross both of its lines; there they cross if and only if the
 * order of their y values at the left line is the reverse of the order at the
 * right line.  Per strip: the y values l_i (left line) and r_i (right line)
 * of the comparable segments, a sorted array L of the l_i, a sweep over L in
 * non-decreasing order that keeps the r values seen so far in an ordered
 * structure R and, for the current segment i, counts the members of R greater
 * than r_i.  The sum over strips is the estimate of E_c.  Horizontal strips
 * are the same with x and y exchanged ("grid orientation", Table 4).
 *
 * Sec. 3.2.3.  For each current segment i the crossing segments j found in R
 * are split into the 8 angle categories of theta_j relative to theta_i
 * (theta in [0, pi), the angle of the segment's line with the x axis):
 * LIL [t, t+v), LIG [t+v, t+pi/2), LOG [t+pi/2, t+pi-v), LOL [t+pi-v, t+pi),
 * RIL [t-v, t), RIG [t-pi/2, t-v), ROG [t-pi+v, t-pi/2), ROL [t-pi, t-pi+v)
 * (t = theta_i, v = the ideal angle), and Eq. 1 turns each category's count
 * |C| and angle sum sum(C) into sum_j |v - angle(i, j)|.  The crossing angle
 * estimate is E_ca = 1 - (sum over i of Eq. 1 / v) / E_c.
 *
 * Readings (the paper is silent on them):
 *   - y at a strip line is the exact rational y0 + (X - x0) dy / dx, used as
 *     the integer key floor(y * 2^30) (exact 64-bit integer arithmetic), so
 *     that every comparison is exact and reproducible;
 *   - a segment crosses a line when the line lies within its closed x range;
 *     segments with dx = 0 (parallel to the lines) and zero-length segments
 *     take no part;
 *   - order reversal is strict: pairs with equal keys at either line (a
 *     crossing on a strip line, a shared endpoint, collinear segments) are not
 *     counted.  The sweep takes L in non-decreasing order of (l, r), so a
 *     segment with the same l as the current one never has a greater r and R
 *     only yields l_j < l_i;
 *   - R, the paper's balanced binary tree, is a Fenwick tree over the ranks
 *     of the strip's r keys (the same order statistics); the 2-D segment tree
 *     of Sec. 3.2.3 is replaced by a plain pass over the segments in R whose
 *     r is greater, which yields the same category counts and sums;
 *   - Eq. 1's left-hand side carries the 1/v factor that its right-hand side
 *     omits: the per-pair term is |v - angle| / v, as in Algorithm 5;
 *   - "both" orientations: the one with the larger count is reported (each
 *     orientation only misses pairs, never adds one).
 *
 * Pinned by the CPU tests against a pairwise brute force of the same
 * definition (every pair of comparable segments of every strip, key orders
 * compared directly), against the direct per-pair sum of |v - angle| / v for
 * Eq. 1, against closed forms (segments spanning the whole strip range, whose
 * every crossing off the strip lines is counted), against the exact count
 * (never above it; each counted pair crosses), and by the exchange of x and y
 * between the two orientations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define STRIP_KEY_SHIFT 30

typedef struct {
    int64_t l, r; /* keys at the left and right line of the strip */
    double theta; /* angle of the segment's line with the x axis, [0, pi) */
} strip_rec;

static int rec_cmp(const void *pa, const void *pb)
{
    const strip_rec *a = (const strip_rec *)pa, *b = (const strip_rec *)pb;
    if (a->l != b->l) return a->l < b->l ? -1 : 1;
    if (a->r != b->r) return a->r < b->r ? -1 : 1;
    return 0;
}

static int i64_cmp(const void *pa, const void *pb)
{
    const int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* floor(y(X) * 2^30) for the segment (x0, y0)-(x1, y1), x0 < x1, at x0 <= X <= x1. */
static int64_t y_key(int64_t x0, int64_t y0, int64_t x1, int64_t y1, int64_t X)
{
    const int64_t dx = x1 - x0, dy = y1 - y0;
    const int64_t num = y0 * dx + (X - x0) * dy; /* = dx * y(X), in [0, 2^32) */
    return (num << STRIP_KEY_SHIFT) / dx;
}

/* Line angle with the x axis in [0, pi). */
static double line_theta(double dx, double dy)
{
    double t = atan2(dy, dx);
    if (t < 0.0) t += M_PI;
    if (t >= M_PI) t -= M_PI;
    return t;
}

/* Eq. 1 for one segment: category counts n[8] and angle sums S[8] (order LIL,
 * LIG, LOG, LOL, RIL, RIG, ROG, ROL) -> sum_j |v - angle(i, j)|. */
double oracle_strip_eq1(double t, double v, const int64_t *n, const double *S)
{
    const double pi = M_PI;
    double x = 0.0;
    x += v * n[0] - (S[0] - t * n[0]);
    x += (S[1] - t * n[1]) - v * n[1];
    x += (t * n[2] - (S[2] - pi * n[2])) - v * n[2];
    x += v * n[3] - (t * n[3] - (S[3] - pi * n[3]));
    x += v * n[4] - (t * n[4] - S[4]);
    x += (t * n[5] - S[5]) - v * n[5];
    x += ((S[6] + pi * n[6]) - t * n[6]) - v * n[6];
    x += v * n[7] - ((S[7] + pi * n[7]) - t * n[7]);
    return x;
}

/* Category of theta_j relative to theta_i = t (Sec. 3.2.3). */
int oracle_strip_category(double t, double tj, double v)
{
    const double pi = M_PI;
    if (tj >= t && tj < t + v) return 0;                 /* LIL */
    if (tj >= t + v && tj < t + pi / 2) return 1;        /* LIG */
    if (tj >= t + pi / 2 && tj < t + pi - v) return 2;   /* LOG */
    if (tj >= t + pi - v && tj < t + pi) return 3;       /* LOL */
    if (tj >= t - v && tj < t) return 4;                 /* RIL */
    if (tj >= t - pi / 2 && tj < t - v) return 5;        /* RIG */
    if (tj >= t - pi + v && tj < t - pi / 2) return 6;   /* ROG */
    return 7;                                            /* ROL: [t - pi, t - pi + v) */
}

/* One strip [X, X + l]: sweep of Sec. 3.2.2 (count) and Sec. 3.2.3 (angles). */
static void strip_sweep(strip_rec *rec, int64_t n, double v, int64_t *count, double *term)
{
    qsort(rec, (size_t)n, sizeof(strip_rec), rec_cmp); /* the sorted array L */
    int64_t *rs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fen = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) rs[i] = rec[i].r;
    qsort(rs, (size_t)n, sizeof(int64_t), i64_cmp);
    for (int64_t i = 0; i < n; ++i)
        if (m == 0 || rs[m - 1] != rs[i]) rs[m++] = rs[i];
    int64_t c = 0;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        /* rank of r_i among the distinct r keys (1-based) */
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (rs[mid] < rec[i].r) lo = mid + 1; else hi = mid;
        }
        const int64_t rank = lo + 1;
        /* members of R with r <= r_i, then those greater */
        int64_t le = 0;
        for (int64_t k = rank; k > 0; k -= k & (-k)) le += fen[k];
        const int64_t greater = i - le;
        c += greater;
        if (greater > 0) {
            int64_t cn[8] = {0};
            double cs[8] = {0};
            for (int64_t j = 0; j < i; ++j) {
                if (rec[j].r <= rec[i].r) continue;
                const int g = oracle_strip_category(rec[i].theta, rec[j].theta, v);
                cn[g] += 1;
                cs[g] += rec[j].theta;
            }
            s += oracle_strip_eq1(rec[i].theta, v, cn, cs) / v;
        }
        for (int64_t k = rank; k <= m; k += k & (-k)) fen[k] += 1; /* insert r_i into R */
    }
    free(rs);
    free(fen);
    *count = c;
    *term = s;
}

/*
 * Strip estimate of E_c and of sum |v - angle| / v over the counted pairs.
 * orient 0: vertical strips (lines x = s l); 1: horizontal (lines y = s l).
 * Returns 0, or -1 for a bad argument (l < 1, bad ids).
 */
int oracle_strip_crossings(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E, int64_t l, int orient,
                           double ideal, int64_t *count_out, double *term_out, int64_t *records_out)
{
    if (l < 1 || (orient != 0 && orient != 1)) return -1;
    const int64_t S = 65536 / l + 1; /* strips s with (s + 1) l <= 65535 are all below this */
    int64_t *cnt = (int64_t *)calloc((size_t)S + 1, sizeof(int64_t));
    /* records per strip */
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= V || b >= V || a == b) {
            free(cnt);
            return -1;
        }
        int64_t x0 = xy[2 * a + orient], x1 = xy[2 * b + orient];
        if (x0 == x1) continue;
        if (x0 > x1) { const int64_t t = x0; x0 = x1; x1 = t; }
        const int64_t s0 = (x0 + l - 1) / l, s1 = x1 / l - 1;
        for (int64_t s = s0; s <= s1; ++s) cnt[s] += 1;
    }
    int64_t *off = (int64_t *)calloc((size_t)S + 2, sizeof(int64_t));
    for (int64_t s = 0; s <= S; ++s) off[s + 1] = off[s] + cnt[s];
    const int64_t R = off[S + 1];
    strip_rec *rec = (strip_rec *)malloc(sizeof(strip_rec) * (size_t)(R > 0 ? R : 1));
    memset(cnt, 0, sizeof(int64_t) * ((size_t)S + 1));
    for (int64_t e = 0; e < E; ++e) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        int64_t x0 = xy[2 * a + orient], y0 = xy[2 * a + 1 - orient];
        int64_t x1 = xy[2 * b + orient], y1 = xy[2 * b + 1 - orient];
        if (x0 == x1) continue;
        if (x0 > x1) {
            int64_t t = x0; x0 = x1; x1 = t;
            t = y0; y0 = y1; y1 = t;
        }
        const double theta = line_theta((double)(x1 - x0), (double)(y1 - y0));
        const int64_t s0 = (x0 + l - 1) / l, s1 = x1 / l - 1;
        for (int64_t s = s0; s <= s1; ++s) {
            strip_rec *q = &rec[off[s] + cnt[s]++];
            q->l = y_key(x0, y0, x1, y1, s * l);
            q->r = y_key(x0, y0, x1, y1, (s + 1) * l);
            q->theta = theta;
        }
    }
    int64_t *sc = (int64_t *)calloc((size_t)S + 1, sizeof(int64_t));
    double *st = (double *)calloc((size_t)S + 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s <= S; ++s) strip_sweep(rec + off[s], off[s + 1] - off[s], ideal, &sc[s], &st[s]);
    int64_t c = 0;
    double t = 0.0;
    for (int64_t s = 0; s <= S; ++s) { /* strips in order: the result does not depend on scheduling */
        c += sc[s];
        t += st[s];
    }
    *count_out = c;
    *term_out = t;
    if (records_out) *records_out = R;
    free(cnt);
    free(off);
    free(rec);
    free(sc);
    free(st);
    return 0;
}
