// grid_common.cuh -- device code shared by the single-layout grid path
// (k_grid.cu) and the batched evaluator (batch.cu): the integer DDA walk of
// a segment through the cells of side 2^k it meets, and the per-cell pair
// tests with the owner-cell rules.
#pragma once

#include <cuda_fp16.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

constexpr int TILE = 32;  // segments per tile (one per lane)

// floor(num / den) for 0 <= num < 2^36, 1 <= den < 2^16: an FP32 estimate,
// then exact integer correction (the estimate is off by at most a few units).
// The operands reach FP32 without a 64-bit conversion instruction.
__device__ __forceinline__ int floordiv_pos(long long num, int den) {
    int q = (int)__fdividef(ll2f_rn(num), i2f_exact(den));
    long long r = num - (long long)q * den;
    while (r < 0) { --q; r += den; }
    while (r >= den) { ++q; r -= den; }
    return q;
}

// A segment walked along its major axis: coordinates swapped when |dy| > |dx|
// (tr), then ordered so that x0 <= x1; afterwards |y1 - y0| <= x1 - x0 and
// x1 > x0 (zero-length segments never reach the grid).
struct DdaSeg {
    int x0, y0, x1, y1;
    bool tr;
};

__device__ __forceinline__ DdaSeg dda_norm(SegRec r) {
    int ax = px(r.x), ay = py(r.x), bx = px(r.y), by = py(r.y);
    const bool tr = abs(by - ay) > abs(bx - ax);
    if (tr) {
        int t = ax; ax = ay; ay = t;
        t = bx; bx = by; by = t;
    }
    if (ax > bx) {
        int t = ax; ax = bx; bx = t;
        t = ay; ay = by; by = t;
    }
    return DdaSeg{ax, ay, bx, by, tr};
}

// Minor-axis cell index of the segment at major coordinate X, x0 <= X <= x1:
// floor(y(X) / 2^k) with y(X) = y0 + (X - x0) (y1 - y0) / (x1 - x0), exact.
__device__ __forceinline__ int minor_at(const DdaSeg &s, int X, int k) {
    if (X == s.x0) return s.y0 >> k;
    if (X == s.x1) return s.y1 >> k;
    const int dx = s.x1 - s.x0, dy = s.y1 - s.y0;
    return floordiv_pos((long long)s.y0 * dx + (long long)(X - s.x0) * dy, dx) >> k;
}

// The cells of major line c: minor indices between those at the line's two
// ends, closed at both (a superset of the half-open cells the segment meets).
// Along one line the major coordinate advances by at most w and the slope is
// at most 1, so the minor index changes by at most one: at most two cells.
// Writes their ids (base + cy * G + cx) and returns how many.
__device__ __forceinline__ int line_cells(const DdaSeg &s, int c, int k, int G, uint32_t base, int (&out)[2]) {
    const int ra = minor_at(s, max(s.x0, c << k), k);
    const int rb = minor_at(s, min(s.x1, (c + 1) << k), k);
    const int lo = min(ra, rb);
    const int n = min(max(ra, rb) - lo + 1, 2);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int q = lo + i;
        out[i] = (int)(base + (uint32_t)(s.tr ? (c * G + q) : (q * G + c)));
    }
    return n;
}

constexpr int SHORT_LINES = 2;  // segments spanning more major lines are "long": walked by a warp

// Whether a segment is long in a grid of side 2^k.  Pairs of two long
// segments are left to the all-pairs tiles: a grid prunes nothing there (two
// long segments share about as many cells as they have pairs) and would only
// add records and owner tests.
__device__ __forceinline__ bool is_long_seg(SegRec r, int k) {
    const DdaSeg s = dda_norm(r);
    return (s.x1 >> k) - (s.x0 >> k) + 1 > SHORT_LINES;
}

// Calls f(ids, n, record, edge id, direction, split_long) for the cells of
// side 2^k that the segment held by this lane (valid if `ok`) meets, a batch
// of at most two cells at a time (so a callback can issue its atomics before
// its stores).  Segments spanning at most SHORT_LINES major lines are walked
// by their own lane; longer ones by the whole warp, one line per lane, so
// that a few long edges do not serialise their warp.  Every lane of the warp
// must call it.  Both DDA passes use it, so they enumerate the same cells.
// `k`, the cell-id `base` and `split` may differ between lanes (several
// grids); split_long is true for the cells of a long segment whose lane
// passed `split`.
template <class F>
__device__ __forceinline__ void warp_for_each_cell(SegRec r, int32_t eid, uint32_t th, bool ok, int k, uint32_t base,
                                                   bool split, F &&f) {
    const int lane = threadIdx.x & 31;
    const int G = 65536 >> k;
    const DdaSeg s = dda_norm(r);
    const int nl = ok ? (s.x1 >> k) - (s.x0 >> k) + 1 : 0;
    const bool is_long = nl > SHORT_LINES;
    if (ok && !is_long) {
        for (int c = s.x0 >> k, e = s.x1 >> k; c <= e; ++c) {
            int ids[2];
            const int n = line_cells(s, c, k, G, base, ids);
            f(ids, n, r, eid, th, false);
        }
    }
    unsigned m = __ballot_sync(0xffffffffu, is_long);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        SegRec q;
        q.x = __shfl_sync(0xffffffffu, r.x, src);
        q.y = __shfl_sync(0xffffffffu, r.y, src);
        q.z = __shfl_sync(0xffffffffu, r.z, src);
        q.w = __shfl_sync(0xffffffffu, r.w, src);
        const int32_t qe = __shfl_sync(0xffffffffu, eid, src);
        const uint32_t qt = __shfl_sync(0xffffffffu, th, src);
        const int qk = __shfl_sync(0xffffffffu, k, src);
        const uint32_t qb = __shfl_sync(0xffffffffu, base, src);
        const bool qs = __shfl_sync(0xffffffffu, split ? 1 : 0, src) != 0;
        const int qG = 65536 >> qk;
        const DdaSeg t = dda_norm(q);
        for (int c = (t.x0 >> qk) + lane, e = t.x1 >> qk; c <= e; c += 32) {
            int ids[2];
            const int n = line_cells(t, c, qk, qG, qb, ids);
            f(ids, n, q, qe, qt, qs);
        }
    }
}

// Owner test of an E_c pair in cell-relative integer coordinates (the cell
// spans [0, w)^2): the intersection point P = a + u t with
// t = ((c - a) x v) / (u x v) lies in the half-open cell.  Exact in int64
// (|P_x * den| < 2^51).
__device__ __forceinline__ bool owns_crossing(int ax, int ay, int ux, int uy, int cx, int cy, int vx, int vy,
                                              int w) {
    long long den = (long long)ux * vy - (long long)uy * vx;
    long long num = (long long)(cx - ax) * vy - (long long)(cy - ay) * vx;
    if (den < 0) { den = -den; num = -num; }
    const long long X = (long long)ax * den + (long long)ux * num;
    const long long Y = (long long)ay * den + (long long)uy * num;
    const long long W = (long long)w * den;
    return 0 <= X && X < W && 0 <= Y && Y < W;
}

// A segment in the coordinates of the cell being processed (origin at the
// cell's lower-left corner), in the FP32 form the pair test uses.  When
// |u_x|, |u_y| <= 2^10 and every coordinate is within 2^12 of the origin,
// u x p - k and all its partial sums are integers of magnitude <= 2^24, so
// the FP32 evaluation is exact ("exact" below); otherwise (relative
// coordinates still below 2^16 in magnitude) its error is below 1,792, under
// the filter bound kOrientFilter.
struct __align__(16) GSeg {
    float ax, ay, bx, by;
    float ux, uy, nk;  // nk = -(u x a), rounded
    uint32_t th;
    uint32_t ida, idb;
    int exact;
    int32_t eid;
};

constexpr float kOrientFilter = 4096.f;

__device__ __forceinline__ GSeg make_gseg(const GridRec &g, int x0, int y0) {
    GSeg r;
    const int ax = px(g.s.x) - x0, ay = py(g.s.x) - y0, bx = px(g.s.y) - x0, by = py(g.s.y) - y0;
    const int ux = bx - ax, uy = by - ay;
    r.ax = i2f_exact(ax); r.ay = i2f_exact(ay); r.bx = i2f_exact(bx); r.by = i2f_exact(by);
    r.ux = i2f_exact(ux); r.uy = i2f_exact(uy);
    r.nk = -ll2f_rn((long long)ux * ay - (long long)uy * ax);
    r.th = g.x.y;
    r.ida = g.s.z; r.idb = g.s.w;
    r.eid = (int32_t)g.x.x;
    const int m = max(max(abs(ax), abs(ay)), max(abs(bx), abs(by)));
    r.exact = (abs(ux) <= 1024 && abs(uy) <= 1024 && m <= 4096) ? 1 : 0;
    return r;
}

// Exact int64 classification of a pair whose FP32 orientations were not
// conclusive, on the absolute coordinates (cell origin x0, y0 added back).
__device__ __forceinline__ int classify_exact(const GSeg &r, const GSeg &c, int x0, int y0) {
    const SegRec a = make_uint4(uint32_t((int)r.ax + x0) | (uint32_t((int)r.ay + y0) << 16),
                                uint32_t((int)r.bx + x0) | (uint32_t((int)r.by + y0) << 16), r.ida, r.idb);
    const SegRec b = make_uint4(uint32_t((int)c.ax + x0) | (uint32_t((int)c.ay + y0) << 16),
                                uint32_t((int)c.bx + x0) | (uint32_t((int)c.by + y0) << 16), c.ida, c.idb);
    return classify_kind(make_row(a, r.th), make_col(b, c.th));
}

// Owner of a collinear overlap: the cell holding the lexicographically
// smallest point of the overlap, an endpoint of one of the segments.
__device__ __forceinline__ bool owns_collinear(const GSeg &r, const GSeg &c, int w) {
    // compare (x, y) lexicographically on the relative integer coordinates
    int ex0 = (int)r.ax, ey0 = (int)r.ay, ex1 = (int)r.bx, ey1 = (int)r.by;
    if (ex1 < ex0 || (ex1 == ex0 && ey1 < ey0)) { int t = ex0; ex0 = ex1; ex1 = t; t = ey0; ey0 = ey1; ey1 = t; }
    int fx0 = (int)c.ax, fy0 = (int)c.ay, fx1 = (int)c.bx, fy1 = (int)c.by;
    if (fx1 < fx0 || (fx1 == fx0 && fy1 < fy0)) { int t = fx0; fx0 = fx1; fx1 = t; t = fy0; fy0 = fy1; fy1 = t; }
    int lx = ex0, ly = ey0;
    if (fx0 > lx || (fx0 == lx && fy0 > ly)) { lx = fx0; ly = fy0; }
    return 0 <= lx && lx < w && 0 <= ly && ly < w;
}

// Owner test with FP32 fast paths.  For two "exact" segments (see GSeg)
// num = (c - a) x v and den = u x v are exact integers in FP32 (|den| <= 2^21,
// |num| <= 2^24), t = num / den carries a relative error below 2^-21 and
// P_x = a_x + u_x t an absolute error below 2^-11 (|u_x t| <= 2^10, |P_x| <
// 2^13).  P is decided inside or outside the half-open cell [0, w)^2 when it
// is further than 2^-9 from the cell's border.  For other segments (cell-
// relative integer coordinates below 2^17, so every input and difference is
// exact in FP32) each product carries a relative error of at most 2^-24, so
// |den~ - den| <= bd = 2^-22 (|u_x v_y| + |u_y v_x|) and likewise bn for num
// (a factor 4 to spare); when |den~| > 4 bd, t~ = num~ / den~ (the fast
// division, within 2 units in the last place) is within
// et = (bn + |t~| bd) / (|den~| - 2 bd) + 2^-20 |t~| of t, and P~ within
// |u| et + 2^-22 (|P~| + 1) of P, a margin doubled again for the decision.
// Otherwise, and near a border, the exact int64 test decides.
__device__ __forceinline__ bool owns_crossing_fast(const GSeg &r, const GSeg &c, int w) {
    const float fw = (float)w;
    if (r.exact & c.exact) {
        const float den = r.ux * c.uy - r.uy * c.ux;
        const float num = (c.ax - r.ax) * c.uy - (c.ay - r.ay) * c.ux;
        const float t = __fdividef(num, den);
        const float X = fmaf(r.ux, t, r.ax), Y = fmaf(r.uy, t, r.ay);
        const float e = 1.0f / 512.0f;
        const bool in = X >= e && X < fw - e && Y >= e && Y < fw - e;
        const bool out = X < -e || X >= fw + e || Y < -e || Y >= fw + e;
        if (in) return true;
        if (out) return false;
    } else {
        const float p1 = r.ux * c.uy, p2 = r.uy * c.ux;
        const float dx = c.ax - r.ax, dy = c.ay - r.ay;
        const float q1 = dx * c.uy, q2 = dy * c.ux;
        const float den = p1 - p2, num = q1 - q2;
        const float bd = 0x1p-22f * (fabsf(p1) + fabsf(p2)), bn = 0x1p-22f * (fabsf(q1) + fabsf(q2));
        if (fabsf(den) > 4.0f * bd) {
            const float t = __fdividef(num, den);
            const float at = fabsf(t);
            const float et = __fdividef(bn + at * bd, fabsf(den) - 2.0f * bd) * 1.001f + 0x1p-20f * at;
            const float X = fmaf(r.ux, t, r.ax), Y = fmaf(r.uy, t, r.ay);
            const float ex = 2.0f * (fabsf(r.ux) * et + 0x1p-22f * (fabsf(X) + 1.0f));
            const float ey = 2.0f * (fabsf(r.uy) * et + 0x1p-22f * (fabsf(Y) + 1.0f));
            const bool in = X >= ex && X < fw - ex && Y >= ey && Y < fw - ey;
            const bool out = X < -ex || X >= fw + ex || Y < -ey || Y >= fw + ey;
            if (in) return true;
            if (out) return false;
        }
    }
    const int iax = (int)r.ax, iay = (int)r.ay, icx = (int)c.ax, icy = (int)c.ay;
    return owns_crossing(iax, iay, (int)r.bx - iax, (int)r.by - iay, icx, icy, (int)c.bx - icx, (int)c.by - icy, w);
}

// Work items of the per-cell pair kernel.  A cell's records are its `ns`
// short segments followed by its long ones; an item is a tile of up to 32
// row records against a tile of up to 32 column records:
//   short x short  row tile ti <= column tile tj of the short records
//                  (ti == tj: a diagonal tile, each pair once);
//   long x short   row tile tl of the long records against column tile ts of
//                  the short ones (long x long pairs are not items: they go
//                  to the all-pairs tiles, or, without the split, every
//                  record counts as short).
// Packed as {flag long-x-short << 31 | a << 16 | b}; tiles < 2^15 per cell.
struct ItemTiles {
    int row0, mr, col0, mc;
    bool diag;
};

// T: segments per tile, 32 (one warp per item) or 16 (two items per warp,
// one per half-warp; fewer idle lanes in cells of few records).
template <int T = TILE>
__device__ __forceinline__ ItemTiles item_tiles(uint32_t n, uint32_t ns, uint32_t w) {
    const int a = (int)((w >> 16) & 0x7fffu), b = (int)(w & 0xffffu);
    ItemTiles t;
    if (w >> 31) {
        t.row0 = (int)ns + a * T;
        t.mr = min(T, (int)n - t.row0);
        t.col0 = b * T;
        t.mc = min(T, (int)ns - t.col0);
        t.diag = false;
    } else {
        t.row0 = a * T;
        t.mr = min(T, (int)ns - t.row0);
        t.col0 = b * T;
        t.mc = min(T, (int)ns - t.col0);
        t.diag = a == b;
    }
    return t;
}

constexpr uint32_t kMaxCellTiles = 1u << 15;

// Work items of a cell with n records, ns of them short (see ItemTiles).
template <int T = TILE>
__device__ __forceinline__ uint64_t cell_item_count(uint64_t n, uint64_t ns, bool *overflow) {
    const uint64_t nl = n - ns, Ts = (ns + T - 1) / T, Tl = (nl + T - 1) / T;
    *overflow = Ts >= kMaxCellTiles || Tl >= kMaxCellTiles;
    return (ns >= 2 ? Ts * (Ts + 1) / 2 : 0) + (ns >= 1 ? Tl * Ts : 0);
}

// Writes the descriptors' tile words of a cell's items, in the order
// counted by cell_item_count, via emit(q, word) for q in [q0, q_end).
template <int T = TILE, class F>
__device__ __forceinline__ void cell_item_words(uint32_t n, uint32_t ns, uint32_t q, uint32_t q_end, F &&emit) {
    const uint32_t nl = n - ns, Ts = (ns + T - 1) / T, Tl = (nl + T - 1) / T;
    if (ns >= 2)
        for (uint32_t ti = 0; ti < Ts && q < q_end; ++ti)
            for (uint32_t tj = ti; tj < Ts && q < q_end; ++tj, ++q) emit(q, (ti << 16) | tj);
    if (ns >= 1)
        for (uint32_t tl = 0; tl < Tl && q < q_end; ++tl)
            for (uint32_t ts = 0; ts < Ts && q < q_end; ++ts, ++q) emit(q, (1u << 31) | (tl << 16) | ts);
}

// The pair tests of one work item: records [row0, row0 + mr) of the cell
// against records [col0, col0 + mc) (diag: the same records, each pair once),
// where `cell_rec` holds the records of one cell whose lower-left corner is
// (x0, y0), side 2^k, and `cs` is this warp's 32-slot staging area.
// Off-diagonal items test all rows x columns; diagonal items use a
// rotation schedule (round q pairs lane i with (i + q) mod m) so that every
// lane has work in every round.  Orientations are evaluated in FP32 in the
// cell's coordinates: exact for pairs of short segments near the cell,
// filtered for the rest.  The rounds only record, per lane, bitmasks of the
// columns that are E_c candidates, collinear candidates or inconclusive; each
// lane then settles its own bits (exact int64 for the inconclusive ones) and
// applies the owner rules: a pair in E_c counts only if this cell owns its
// intersection point, a collinear overlap only if this cell owns the
// lexicographically smallest point of the overlap.  Every lane of the warp
// must call it.
template <bool PER_EDGE, int T = TILE>
__device__ __forceinline__ void grid_item(const GridRec *__restrict__ cell_rec, const ItemTiles t, int x0, int y0,
                                          int k, GSeg *cs, uint32_t ideal, PairCounts &pc, PerEdge pe) {
    const int lane = threadIdx.x & (T - 1);  // the lane within this item's T lanes
    const int w = 1 << k;
    const int mr = t.mr, mc = t.mc;

    __syncwarp();
    if (lane < mc) cs[lane] = make_gseg(cell_rec[t.col0 + lane], x0, y0);
    GSeg rs;
    if (lane < mr) rs = make_gseg(cell_rec[t.row0 + lane], x0, y0);
    __syncwarp();
    if (lane >= mr) return;

    uint32_t m_ec = 0, m_prop = 0, m_coll = 0, m_unsure = 0;
    const bool diag = t.diag;
    const int rounds = diag ? mr / 2 : mc;
    for (int s = 0; s < rounds; ++s) {
        int jj;
        if (diag) {
            const int qq = s + 1;
            if (2 * qq == mr && lane >= mr / 2) continue;
            jj = lane + qq;
            if (jj >= mr) jj -= mr;
        } else {
            jj = s;
        }
        const GSeg c = cs[jj];
        const float o1 = fmaf(rs.ux, c.ay, fmaf(-rs.uy, c.ax, rs.nk));
        const float o2 = fmaf(rs.ux, c.by, fmaf(-rs.uy, c.bx, rs.nk));
        const float o3 = fmaf(c.ux, rs.ay, fmaf(-c.uy, rs.ax, c.nk));
        const float o4 = fmaf(c.ux, rs.by, fmaf(-c.uy, rs.bx, c.nk));
        const float mn = fminf(fminf(fabsf(o1), fabsf(o2)), fminf(fabsf(o3), fabsf(o4)));
        const uint32_t bit = 1u << jj;
        const bool sure = (rs.exact & c.exact) || mn > kOrientFilter;
        const bool shared = (rs.ida == c.ida) | (rs.ida == c.idb) | (rs.idb == c.ida) | (rs.idb == c.idb);
        const float p12 = o1 * o2, p34 = o3 * o4;
        const bool cand = !shared && p12 <= 0.f && p34 <= 0.f;
        const bool coll = o1 == 0.f && o2 == 0.f;
        m_unsure |= sure ? 0u : bit;
        m_ec |= (sure && cand && !coll) ? bit : 0u;
        m_prop |= (sure && p12 < 0.f && p34 < 0.f) ? bit : 0u;
        m_coll |= (sure && cand && coll) ? bit : 0u;
    }
    // inconclusive pairs: exact int64
    while (m_unsure) {
        const int jj = __ffs(m_unsure) - 1;
        m_unsure &= m_unsure - 1;
        const int kind = classify_exact(rs, cs[jj], x0, y0);
        const uint32_t bit = 1u << jj;
        if (kind == PAIR_PROPER) { m_ec |= bit; m_prop |= bit; }
        else if (kind == PAIR_TOUCHING) m_ec |= bit;
        else if (kind == PAIR_COLLINEAR) m_coll |= bit;
    }
    // collinear candidates: the extents must meet, and this cell must own
    // the smallest point of the overlap (coordinates exact in FP32)
    while (m_coll) {
        const int jj = __ffs(m_coll) - 1;
        m_coll &= m_coll - 1;
        const GSeg c = cs[jj];
        const bool ar = rs.ax < rs.bx || (rs.ax == rs.bx && rs.ay <= rs.by);
        const bool ac = c.ax < c.bx || (c.ax == c.bx && c.ay <= c.by);
        const float elx = ar ? rs.ax : rs.bx, ely = ar ? rs.ay : rs.by;
        const float ehx = ar ? rs.bx : rs.ax, ehy = ar ? rs.by : rs.ay;
        const float flx = ac ? c.ax : c.bx, fly = ac ? c.ay : c.by;
        const float fhx = ac ? c.bx : c.ax, fhy = ac ? c.by : c.ay;
        const bool lo_e = elx > flx || (elx == flx && ely >= fly);
        const float lx = lo_e ? elx : flx, ly = lo_e ? ely : fly;
        const bool hi_e = ehx < fhx || (ehx == fhx && ehy <= fhy);
        const float hx = hi_e ? ehx : fhx, hy = hi_e ? ehy : fhy;
        if (!(lx < hx || (lx == hx && ly <= hy))) continue;
        if (!owns_collinear(rs, c, w)) continue;
        ++pc.collinear;
        if (PER_EDGE) {
            atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)rs.eid + 2], 1ull);
            atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)c.eid + 2], 1ull);
        }
    }
    // E_c candidates: owner of the intersection point
    while (m_ec) {
        const int jj = __ffs(m_ec) - 1;
        const uint32_t bit = 1u << jj;
        m_ec &= m_ec - 1;
        const GSeg c = cs[jj];
        if (!owns_crossing_fast(rs, c, w)) continue;
        const uint32_t qd = dev_term(rs.th, c.th, ideal);
        const bool prop = (m_prop & bit) != 0;
        pc.dev += qd;
        if (prop) ++pc.proper; else ++pc.touching;
        if (PER_EDGE) {
            const int slot = prop ? 0 : 1;
            atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)rs.eid + slot], 1ull);
            atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)c.eid + slot], 1ull);
            atomicAdd((unsigned long long *)&pe.dev[rs.eid], (unsigned long long)qd);
            atomicAdd((unsigned long long *)&pe.dev[c.eid], (unsigned long long)qd);
        }
    }
}

}  // namespace gr

namespace gr {

// ------------------------------------------------ rotation work items (a6)
// All pairs of a cell's n records in the rotation order: row i meets rows
// (i + q) mod n for q = 1 .. n/2, except that for even n the offset n/2 is
// taken from rows i < n/2 only; every unordered pair of the cell appears
// exactly once.  A work item is one warp's share of a chunk of m rows (32,
// or n mod 32 for a cell's last chunk): s streams of the m rows (s = 1 for a
// full chunk, up to 3 for a short last chunk, so that fewer lanes idle), each
// stream taking RQ consecutive offsets, stream sigma the offsets
// q0 + sigma RQ ... .  The item's columns form a window the warp stages in
// shared memory: stream sigma's rows 32 c + r meet, at their t-th offset,
// window slot sigma (m + RQ - 1) + r + t, which holds row
// 32 c + q0 + sigma RQ + r + t (mod n) of the cell.
constexpr int RQ = 16;                 // rotation offsets per stream of a work item
constexpr int RQ_HALF = RQ / 2;        // the kernel settles its queue after each half
constexpr int RSTREAMS = 3;            // at most this many streams of a short last chunk
constexpr int RWIN = 75;               // window slots: max over m of s (m + RQ - 1)

// Streams of a chunk of m rows in a cell with P offset pieces.
__host__ __device__ __forceinline__ int rot_streams(int m, int P) {
    int s = 1;  // min(RSTREAMS, 32 / m) for m < 32, without a division
#pragma unroll
    for (int k = 2; k <= RSTREAMS; ++k) s += (m < 32 && k * m <= 32) ? 1 : 0;
    return min(s, max(1, P));
}

// Work items of a cell with n records; overflow when the item word cannot
// hold the chunk or offset index.
__device__ __forceinline__ uint64_t rot_item_count(uint64_t n, bool *overflow) {
    *overflow = false;
    if (n < 2) return 0;
    const uint64_t Q = n >> 1, Ff = n >> 5, m = n & 31, P = (Q + RQ - 1) / RQ;
    *overflow = Ff + 1 > (1u << 15) || P >= (1u << 16);
    uint64_t items = Ff * P;
    if (m) {
        const uint64_t s = (uint64_t)rot_streams((int)m, (int)min(P, (uint64_t)RSTREAMS));
        items += (P + s - 1) / s;
    }
    return items;
}

// The item words of a cell, in the order counted by rot_item_count, via
// emit(i, word) for i in [q, q_end): chunk c and piece group p (of s pieces
// for the last chunk) as c << 16 | p.
template <class F>
__device__ __forceinline__ void rot_item_words(uint32_t n, uint32_t q, uint32_t q_end, F &&emit) {
    if (n < 2) return;
    const uint32_t Q = n >> 1, Ff = n >> 5, m = n & 31, P = (Q + RQ - 1) / RQ;
    for (uint32_t c = 0; c < Ff && q < q_end; ++c)
        for (uint32_t p = 0; p < P && q < q_end; ++p, ++q) emit(q, (c << 16) | p);
    if (m) {
        const uint32_t s = (uint32_t)rot_streams((int)m, (int)min(P, (uint32_t)RSTREAMS));
        for (uint32_t p = 0; p < (P + s - 1) / s && q < q_end; ++p, ++q) emit(q, (Ff << 16) | p);
    }
}

// A lane's share of a rotation item: row i of the cell, its first offset q0,
// the number of offsets it takes (0: none) and its first window slot; and the
// item's stream layout (m rows, s streams, first window row of stream 0).
struct RotLane {
    int i, q0, cnt, slot;
    int m, s;
    uint32_t first;
};

__device__ __forceinline__ RotLane rot_lane(int n, uint32_t w, int lane) {
    const int Q = n >> 1, c = (int)((w >> 16) & 0x7fffu), p = (int)(w & 0xffffu);
    const int P = (Q + RQ - 1) / RQ;
    RotLane r;
    r.m = min(32, n - 32 * c);
    r.s = rot_streams(r.m, min(P, RSTREAMS));
    // the lane's stream: lane / m where below s, at least s otherwise (then
    // the lane takes no offsets), without a division
    int sig = 0;
#pragma unroll
    for (int k = 1; k <= RSTREAMS; ++k) sig += lane >= k * r.m ? 1 : 0;
    const int row = lane - sig * r.m;
    const int piece = (r.m == 32 ? p : p * r.s) + sig;
    r.i = 32 * c + row;
    r.q0 = 1 + piece * RQ;
    r.first = (uint32_t)(32 * c + 1 + (r.m == 32 ? p : p * r.s) * RQ);
    r.slot = sig * (r.m + RQ - 1) + row;
    const int Qi = ((n & 1) == 0 && r.i >= (n >> 1)) ? Q - 1 : Q;
    r.cnt = (sig < r.s && piece < P) ? max(0, min(Qi, r.q0 + RQ - 1) - r.q0 + 1) : 0;
    if (r.cnt == 0) { r.i = 0; r.slot = 0; }
    return r;
}

// The FP32 form of a record for the rotation kernel, written by the scatter
// into three arrays of float4 (one row each per record): its segment in the
// coordinates of its cell (origin at the cell's lower-left corner)
//   a = {ax, ay, bx, by},
//   b = {ux, uy, nk, v}, nk = -(u x a) rounded and v its margin code,
//   c = {E0x, E0y, E1x, E1y}, the part of the segment inside the closed cell.
// A segment is "exact" when |u_x|, |u_y| <= 2^10 and its coordinates lie
// within 2^12 of the origin (then its line evaluated at integer points within
// 2^12 of the origin is an exact FP32 integer: products and sums below 2^24),
// and "whole" when it lies inside the closed cell (its clip points are its
// own integer endpoints).  v = 0 for an exact whole segment, 64 for another
// exact one, 8192 otherwise.  kRotFilter is the bound on the FP32 error of
// one orientation of two records: with |u|, |coordinates| < 2^16 the rounded
// nk (< 2^33) errs by at most 256, the inner fused multiply-add (< 2^34) by
// 512 and the outer (< 2^35) by 1024: 1792 in all.
constexpr float kRotFilter = 4096.f;
constexpr float kClipExact = 64.f;    // margin of a clip test against an exact line
constexpr float kClipFiltered = 8192.f;  // ... against any other line

// The clipped part [E0, E1] is computed by Liang and Barsky's parametric
// clipping against the box [0, w]^2: the parameters t of the box lines are
// quotients of integers from the fast division (within 2 ulp: |t| error
// below 2^-23 for t in [0, 1], where t is clamped), E = a + t u rounded, so
// each coordinate of E is within |u| 2^-23 + ulp(w) / 2 < 2^-6 of the exact
// point; a whole segment keeps its endpoints exactly.  A segment lying on a
// line of the cell's border (its clipped part on the border itself) gets NaN
// clip points, which make every clip test inconclusive.
__device__ __forceinline__ void make_rgeo(SegRec s, int x0, int y0, int w, float4 &a, float4 &b, float4 &c) {
    const int ax = px(s.x) - x0, ay = py(s.x) - y0, bx = px(s.y) - x0, by = py(s.y) - y0;
    const int ux = bx - ax, uy = by - ay;
    const float fax = i2f_exact(ax), fay = i2f_exact(ay), fbx = i2f_exact(bx), fby = i2f_exact(by);
    const float fux = i2f_exact(ux), fuy = i2f_exact(uy);
    a = make_float4(fax, fay, fbx, fby);
    const int m = max(max(abs(ax), abs(ay)), max(abs(bx), abs(by)));
    const bool exact = abs(ux) <= 1024 && abs(uy) <= 1024 && m <= 4096;
    const bool whole = min(min(ax, ay), min(bx, by)) >= 0 && max(max(ax, ay), max(bx, by)) <= w;
    b = make_float4(fux, fuy, -ll2f_rn((long long)ux * ay - (long long)uy * ax),
                    exact ? (whole ? 0.f : kClipExact) : kClipFiltered);
    const bool on_border = (uy == 0 && (ay == 0 || ay == w)) || (ux == 0 && (ax == 0 || ax == w));
    if (on_border) {
        const float nan = __int_as_float(0x7fc00000);
        c = make_float4(nan, nan, nan, nan);
        return;
    }
    if (whole) {
        c = make_float4(fax, fay, fbx, fby);
        return;
    }
    float t0 = 0.f, t1 = 1.f;
    if (ux != 0) {
        const float ta = __fdividef(i2f_exact(-ax), fux), tb = __fdividef(i2f_exact(w - ax), fux);
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (uy != 0) {
        const float ta = __fdividef(i2f_exact(-ay), fuy), tb = __fdividef(i2f_exact(w - ay), fuy);
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (t1 < t0) t1 = t0;
    c = make_float4(fmaf(t0, fux, fax), fmaf(t0, fuy, fay), fmaf(t1, fux, fax), fmaf(t1, fuy, fay));
}

// The FP16 form of a record for the rotation kernel's first test, in cell
// units centred on the cell (the cell is [-1/2, 1/2]^2): the signed distance
// to its line
//   f(p) = hx p_y + hy p_x + hc,  hx = u_x / |u|, hy = -u_y / |u|,
//   hc = nk / (|u| w) + (hx + hy) / 2,
// and its clipped part E0, E1 as E / w - 1/2, as eight halves
// {hx, hy, hc, E0x, E0y, E1x, E1y, 0} (two per word, the first in the low
// half).  The line meets the closed cell, so |hc| <= sqrt(2) / 2 (the
// distance from the centre).  Error of f at the true clipped part, evaluated
// as two fused FP16 multiply-adds fma(hx, E_y, fma(hy, E_x, hc)) (round to
// nearest; |inner| <= 1.25 and |f| <= 1.75, so each rounding is <= 2^-11):
//   coefficients rounded to FP16 (|hx|, |hy| <= 1 against |p| <= 1/2,
//   |hc| < 1; FP32 errors below 2^-20)                          <= 2^-12 + 2^-12 + 2^-20;
//   clip points: FP32 error 2^-6 / w plus FP16 rounding 2^-13, times
//   |hx| + |hy| <= sqrt(2)                                      <= sqrt(2) (2^-13 + 2^-6 / w);
//   the two roundings of the multiply-adds                      <= 2 2^-11;
// in all below 0.00165 + 0.0221 / w, under half_margin(w) = 2^-9 + 2^-4 / w.
// A zero-length line or a border record (NaN clip points) gets NaN halves,
// which leave every pair with it to the FP32 test.
__host__ __device__ __forceinline__ float half_margin(int w) { return 0.001953125f + 0.0625f / (float)w; }

__device__ __forceinline__ uint32_t pack_halves(float lo, float hi) {
    return (uint32_t)__half_as_ushort(__float2half_rn(lo)) | ((uint32_t)__half_as_ushort(__float2half_rn(hi)) << 16);
}

__device__ __forceinline__ uint4 make_hgeo(const float4 &b, const float4 &c, int w) {
    const float inv_w = 1.f / (float)w;  // exact: w is a power of two
    const float len = sqrtf(b.x * b.x + b.y * b.y);
    const float hx = b.x / len, hy = -b.y / len;
    const float hc = b.z * inv_w / len + 0.5f * (hx + hy);
    if (!(len > 0.f) || !(fabsf(hc) <= 0.75f)) {
        const uint32_t nan2 = 0x7e007e00u;
        return make_uint4(nan2, nan2, nan2, nan2);
    }
    return make_uint4(pack_halves(hx, hy), pack_halves(hc, fmaf(c.x, inv_w, -0.5f)),
                      pack_halves(fmaf(c.y, inv_w, -0.5f), fmaf(c.z, inv_w, -0.5f)),
                      pack_halves(fmaf(c.w, inv_w, -0.5f), 0.f));
}

// The clip test of a pair: the row's clipped part against the column's line
// (s0, s1) and the column's clipped part against the row's line (s2, s3).
// The error of s0, s1 is the column line's FP32 error at the row's clip
// points plus |u_col| times their error: at most 1792 + 2 * 2^16 * 2^-6 =
// 3840 for a filtered line (margin 8192), 12 + 32 for an exact one (margin
// 64) and none for an exact line at a whole exact segment's endpoints
// (margin 0); the margin of s0, s1 is max(v_col as a line, v_row as points),
// where a record's "points" margin is min(v, 64).  Both clipped parts lie in
// the closed cell, so the pair can count here only if each clipped part
// meets the other's line: a pair is surely outside (clip_out) when either
// part lies strictly beyond the margin on one side.  clip_in: the row's part
// strictly straddles the column's line, so an intersection point on the row's
// segment lies strictly inside it, hence in the open cell (the open part of
// a segment that does not run along the border lies in the cell's interior).
// both: each part strictly straddles the other's line, so the parts meet in
// one point inside both: a proper crossing of the segments, in the open cell.
struct ClipTest {
    bool out, in, both;
};

__device__ __forceinline__ ClipTest clip_test(const float4 &rb, const float4 &rc, float r_pts, const float4 &cb,
                                              const float4 &cc) {
    const float s0 = fmaf(cb.x, rc.y, fmaf(-cb.y, rc.x, cb.z));
    const float s1 = fmaf(cb.x, rc.w, fmaf(-cb.y, rc.z, cb.z));
    const float s2 = fmaf(rb.x, cc.y, fmaf(-rb.y, cc.x, rb.z));
    const float s3 = fmaf(rb.x, cc.w, fmaf(-rb.y, cc.z, rb.z));
    const float M01 = fmaxf(cb.w, r_pts), M23 = fmaxf(rb.w, fminf(cb.w, kClipExact));
    const float lo01 = fminf(s0, s1), hi01 = fmaxf(s0, s1), lo23 = fminf(s2, s3), hi23 = fmaxf(s2, s3);
    ClipTest t;
    t.out = (lo01 > M01) | (hi01 < -M01) | (lo23 > M23) | (hi23 < -M23);
    t.in = (lo01 < -M01) & (hi01 > M01);
    t.both = t.in & (lo23 < -M23) & (hi23 > M23);
    return t;
}

// The four orientations of a pair: o1, o2 of c's endpoints against r's line,
// o3, o4 of r's endpoints against c's line.
struct Orient4 {
    float o1, o2, o3, o4;
};

__device__ __forceinline__ Orient4 orient4(const float4 &ra, const float4 &rb, const float4 &ca, const float4 &cb) {
    Orient4 o;
    o.o1 = fmaf(rb.x, ca.y, fmaf(-rb.y, ca.x, rb.z));
    o.o2 = fmaf(rb.x, ca.w, fmaf(-rb.y, ca.z, rb.z));
    o.o3 = fmaf(cb.x, ra.y, fmaf(-cb.y, ra.x, cb.z));
    o.o4 = fmaf(cb.x, ra.w, fmaf(-cb.y, ra.z, cb.z));
    return o;
}

// Whether the pair is surely disjoint: one segment's endpoints lie strictly
// on one side of the other's line, beyond the filter F.
__device__ __forceinline__ bool surely_apart(const Orient4 &o, float F) {
    const float lo12 = fminf(o.o1, o.o2), hi12 = fmaxf(o.o1, o.o2);
    const float lo34 = fminf(o.o3, o.o4), hi34 = fmaxf(o.o3, o.o4);
    return (lo12 > F) | (hi12 < -F) | (lo34 > F) | (hi34 < -F);
}

// Lexicographic (x, then y) order of two integer points in signed
// coordinates: a <= b.
__device__ __forceinline__ bool lex_le(int ax, int ay, int bx, int by) { return ax < bx || (ax == bx && ay <= by); }

// Exact int64 classification (classify_kind's rules) of a pair given in the
// integer coordinates of one cell (|values| < 2^17, products below 2^35).
__device__ __forceinline__ int classify_rel(const float4 &ra, const float4 &ca, uint32_t ida, uint32_t idb,
                                            uint32_t idc, uint32_t idd) {
    if ((ida == idc) | (ida == idd) | (idb == idc) | (idb == idd)) return PAIR_NONE;
    const int ax = (int)ra.x, ay = (int)ra.y, bx = (int)ra.z, by = (int)ra.w;
    const int cx = (int)ca.x, cy = (int)ca.y, dx = (int)ca.z, dy = (int)ca.w;
    const long long ux = bx - ax, uy = by - ay, vx = dx - cx, vy = dy - cy;
    const long long o1 = ux * (cy - ay) - uy * (cx - ax);
    const long long o2 = ux * (dy - ay) - uy * (dx - ax);
    if ((o1 > 0 && o2 > 0) || (o1 < 0 && o2 < 0)) return PAIR_NONE;
    const long long o3 = vx * (ay - cy) - vy * (ax - cx);
    const long long o4 = vx * (by - cy) - vy * (bx - cx);
    if ((o3 > 0 && o4 > 0) || (o3 < 0 && o4 < 0)) return PAIR_NONE;
    if (o1 == 0 && o2 == 0) {
        // collinear: the extents along the line meet (lexicographic order is
        // a linear order of the points of one line)
        int lx = ax, ly = ay, hx = bx, hy = by;
        if (!lex_le(lx, ly, hx, hy)) { lx = bx; ly = by; hx = ax; hy = ay; }
        int mx = cx, my = cy, nx = dx, ny = dy;
        if (!lex_le(mx, my, nx, ny)) { mx = dx; my = dy; nx = cx; ny = cy; }
        if (lex_le(lx, ly, mx, my)) { lx = mx; ly = my; }  // larger low end
        if (lex_le(nx, ny, hx, hy)) { hx = nx; hy = ny; }  // smaller high end
        return lex_le(lx, ly, hx, hy) ? PAIR_COLLINEAR : PAIR_NONE;
    }
    return (o1 != 0 && o2 != 0 && o3 != 0 && o4 != 0) ? PAIR_PROPER : PAIR_TOUCHING;
}

// Owner of a collinear overlap in its cell's coordinates: the cell holding
// the lexicographically smallest point of the overlap (the larger of the two
// segments' smaller endpoints).
__device__ __forceinline__ bool owns_collinear_rel(const float4 &ra, const float4 &ca, int w) {
    int ex = (int)ra.x, ey = (int)ra.y;
    if (!lex_le(ex, ey, (int)ra.z, (int)ra.w)) { ex = (int)ra.z; ey = (int)ra.w; }
    int fx = (int)ca.x, fy = (int)ca.y;
    if (!lex_le(fx, fy, (int)ca.z, (int)ca.w)) { fx = (int)ca.z; fy = (int)ca.w; }
    if (lex_le(ex, ey, fx, fy)) { ex = fx; ey = fy; }
    return 0 <= ex && ex < w && 0 <= ey && ey < w;
}

}  // namespace gr
