// allpairs_common.cuh -- one square tile of the all-pairs crossing test (a7),
// shared by the single-layout kernel (every pair of a layout, or the pairs of
// its long segments) and the batched kernel (the long segments of each
// layout).
#pragma once

#include <math.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

// t = r (r + 1) / 2 + c with c <= r; (bi, bj) = (c, r)
__device__ __forceinline__ void decode_tile(int64_t t, int &bi, int &bj) {
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    bj = (int)r;
    bi = (int)(t - r * (r + 1) / 2);
}

// FP32 fast path with an exact fallback.  For integer coordinates below 2^16
// the orientation u x p - k (k rounded to FP32, |k| < 2^33) evaluated as
// fma(u_x, p_y, fma(-u_y, p_x, -k)) is off by at most 256 + 512 + 1024 =
// 1792 (half an ulp of k, of the inner fma result < 2^34 and of the outer one
// < 2^35).  When all four orientations of a pair exceed kAllPairsFilter in
// magnitude their signs are exact and none is zero, so the pair crosses
// properly iff both sign products are negative.  Any pair with a smaller
// orientation -- which includes every pair sharing an endpoint, every
// collinear and every touching pair -- is re-decided exactly in int64.
constexpr float kAllPairsFilter = 4096.f;

// Tile shapes: THREADS threads holding RPT rows each, THREADS * RPT columns
// (square tiles: the diagonal test is local j > local i).  Large lists take
// the big tile (fewer column stagings per pair), short lists the small one
// (enough tiles to fill the GPU, less padding).
constexpr int AG_THREADS = 256;
constexpr int AG_RPT = 2;
constexpr int AG_ROWS = AG_THREADS * AG_RPT;
constexpr int AS_THREADS = 128;
constexpr int AS_RPT = 2;
constexpr int AS_ROWS = AS_THREADS * AS_RPT;

struct __align__(16) FCol {
    float cx, cy, dx, dy;
    float vx, vy, nk;  // v = d - c, nk = -(v x c) rounded
    uint32_t th;
};

struct FRow {
    float ax, ay, bx, by;
    float ux, uy, nk;
    uint32_t th;
};

__device__ __forceinline__ FRow make_frow(SegRec s, uint32_t th) {
    FRow r;
    const int ax = px(s.x), ay = py(s.x), bx = px(s.y), by = py(s.y);
    const int ux = bx - ax, uy = by - ay;
    r.ax = i2f_exact(ax); r.ay = i2f_exact(ay); r.bx = i2f_exact(bx); r.by = i2f_exact(by);
    r.ux = i2f_exact(ux); r.uy = i2f_exact(uy);
    r.nk = -ll2f_rn((long long)ux * ay - (long long)uy * ax);
    r.th = th;
    return r;
}

__device__ __forceinline__ FCol make_fcol(SegRec s, uint32_t th) {
    FCol c;
    const int cx = px(s.x), cy = py(s.x), dx = px(s.y), dy = py(s.y);
    const int vx = dx - cx, vy = dy - cy;
    c.cx = i2f_exact(cx); c.cy = i2f_exact(cy); c.dx = i2f_exact(dx); c.dy = i2f_exact(dy);
    c.vx = i2f_exact(vx); c.vy = i2f_exact(vy);
    c.nk = -ll2f_rn((long long)vx * cy - (long long)vy * cx);
    c.th = th;
    return c;
}

// Shared-memory staging of one tile's columns.
template <int COLS>
struct AllPairsSmem {
    FCol fc[COLS];
    SegRec raw[COLS];
};

// Tile (bi, bj), bi <= bj, of the n segments at seg/theta: rows bi, columns
// bj (THREADS * RPT each); diagonal tiles keep column > row.  Tallies go to
// pc.  Every thread of the THREADS-thread block must call it with the same
// arguments; it synchronises the block.
template <int THREADS, int RPT>
__device__ __forceinline__ void allpairs_tile(const SegRec *__restrict__ seg, const uint32_t *__restrict__ theta,
                                              int n, int bi, int bj, uint32_t ideal,
                                              AllPairsSmem<THREADS * RPT> &sm, PairCounts &pc) {
    constexpr int ROWS = THREADS * RPT, COLS = ROWS;
    const int j0 = bj * COLS;
    if (j0 >= n) return;
    const int nc = min(COLS, n - j0);
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += THREADS) {
        const SegRec s = seg[j0 + c];
        sm.raw[c] = s;
        sm.fc[c] = make_fcol(s, theta[j0 + c]);
    }
    FRow rs[RPT];
    SegRec rr[RPT];
    bool rok[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int i = bi * ROWS + threadIdx.x + k * THREADS;
        rok[k] = i < n;
        rr[k] = rok[k] ? seg[i] : make_uint4(0, 0, 0, 0);
        rs[k] = make_frow(rr[k], rok[k] ? theta[i] : 0u);
    }
    __syncthreads();
    // a pair counts when its column index exceeds lim (diagonal tiles: the row's own index)
    int lim[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        lim[k] = !rok[k] ? 0x7fffffff : (bi == bj ? (int)threadIdx.x + k * THREADS : -1);
    // columns in chunks of 32: the sure crossings and the inconclusive pairs
    // are marked in per-row bitmasks; the angle terms of the crossings and the
    // exact re-decisions run per set bit after each chunk
    for (int c0 = 0; c0 < nc; c0 += 32) {
        const int ce = min(32, nc - c0);
        uint32_t hm[RPT], um[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) hm[k] = um[k] = 0u;
#pragma unroll 2
        for (int q = 0; q < ce; ++q) {
            const int jj = c0 + q;
            const FCol c = sm.fc[jj];
            const uint32_t bit = 1u << q;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const FRow &r = rs[k];
                const float o1 = fmaf(r.ux, c.cy, fmaf(-r.uy, c.cx, r.nk));
                const float o2 = fmaf(r.ux, c.dy, fmaf(-r.uy, c.dx, r.nk));
                const float o3 = fmaf(c.vx, r.ay, fmaf(-c.vy, r.ax, c.nk));
                const float o4 = fmaf(c.vx, r.by, fmaf(-c.vy, r.bx, c.nk));
                const float mn = fminf(fminf(fabsf(o1), fabsf(o2)), fminf(fabsf(o3), fabsf(o4)));
                const bool valid = jj > lim[k];
                const bool sure = mn > kAllPairsFilter;
                const int sx = (__float_as_int(o1) ^ __float_as_int(o2)) & (__float_as_int(o3) ^ __float_as_int(o4));
                if (valid && sure && sx < 0) hm[k] |= bit;
                if (valid && !sure) um[k] |= bit;
            }
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            pc.proper += (uint32_t)__popc(hm[k]);
            for (uint32_t m = hm[k]; m; m &= m - 1) pc.dev += dev_term(rs[k].th, sm.fc[c0 + __ffs(m) - 1].th, ideal);
            for (uint32_t m = um[k]; m; m &= m - 1) {
                const int jj = c0 + __ffs(m) - 1;
                const RowSeg er = make_row(rr[k], rs[k].th);
                const ColSeg ec = make_col(sm.raw[jj], sm.fc[jj].th);
                const int kind = classify_kind(er, ec);
                if (kind == PAIR_COLLINEAR) {
                    ++pc.collinear;
                } else if (kind != PAIR_NONE) {
                    if (kind == PAIR_PROPER) ++pc.proper; else ++pc.touching;
                    pc.dev += dev_term(er.th, ec.th, ideal);
                }
            }
        }
    }
}

}  // namespace gr
