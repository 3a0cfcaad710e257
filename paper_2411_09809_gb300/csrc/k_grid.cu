// k_grid.cu -- the uniform-grid crossing path (a2-a6).
//
// The paper's enhanced algorithm (Sec. 3.2.2) cuts the plane into strips so
// that independent groups replace a global join, and accepts an error for
// pairs that do not share two strip lines.  Here the plane is cut into square
// cells of side w = 2^k and the count stays exact:
//   a2  every segment walks the cells its closed segment meets (integer DDA,
//       exact floor divisions) and counts them per cell;
//   a3  an exclusive scan turns the per-cell counts into cell offsets;
//   a4  a second DDA walk scatters the segment records into their cells (a
//       counting sort by cell id; the order inside a cell is irrelevant);
//   a6  a pair kernel tests every pair of segments that share a cell and
//       counts a pair only in the cell that owns its exactly computed
//       intersection point (half-open cells), so each pair counts once.
// Every cell met by a segment holds it, so the owner cell of an intersection
// point, which lies on both segments, holds both of them.
#include <math.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

namespace {

constexpr int GP_WARPS = 8;  // warps per block of the pair kernel
constexpr int TILE = 32;     // segments per tile (one per lane)

// floor(num / den) for 0 <= num < 2^36, 1 <= den < 2^16: an FP32 estimate,
// then exact integer correction (the estimate is off by at most a few units).
__device__ __forceinline__ int floordiv_pos(long long num, int den) {
    int q = (int)__fdividef((float)num, (float)den);
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
// ends, closed at both (a superset of the half-open cells the segment meets;
// the slope is at most 1, so there are at most three).
template <class F>
__device__ __forceinline__ void dda_line(const DdaSeg &s, int c, int k, SegRec r, int32_t eid, uint32_t th,
                                         F &f) {
    const int ra = minor_at(s, max(s.x0, c << k), k);
    const int rb = minor_at(s, min(s.x1, (c + 1) << k), k);
    for (int q = min(ra, rb); q <= max(ra, rb); ++q) {
        if (s.tr) f(q, c, r, eid, th); else f(c, q, r, eid, th);
    }
}

constexpr int LONG_LINES = 8;  // segments spanning more lines are walked by a warp

// Calls f(cx, cy, record, edge id, direction) for every cell of side 2^k that the
// segment held by this lane (valid if `ok`) meets.  Short segments are walked
// by their own lane; long ones by the whole warp, one major line per lane, so
// that a few long edges do not serialise their warp.  Every lane of the warp
// must call it.  Both DDA passes use it, so they enumerate the same cells.
template <class F>
__device__ __forceinline__ void warp_for_each_cell(SegRec r, int32_t eid, uint32_t th, bool ok, int k, F &&f) {
    const int lane = threadIdx.x & 31;
    const DdaSeg s = dda_norm(r);
    const int nl = ok ? (s.x1 >> k) - (s.x0 >> k) + 1 : 0;
    const bool is_long = nl > LONG_LINES;
    if (ok && !is_long) {
        for (int c = s.x0 >> k, e = s.x1 >> k; c <= e; ++c) dda_line(s, c, k, r, eid, th, f);
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
        const DdaSeg t = dda_norm(q);
        for (int c = (t.x0 >> k) + lane, e = t.x1 >> k; c <= e; c += 32) dda_line(t, c, k, q, qe, qt, f);
    }
}

// a2 -- per-cell record counts.
__global__ void __launch_bounds__(256) k_grid_count(const SegRec *__restrict__ seg,
                                                    const DevAcc *__restrict__ acc, int k,
                                                    uint32_t *__restrict__ cell_cnt) {
    const int64_t n = acc->n_seg;
    const int G = 65536 >> k;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const SegRec r = ok ? seg[i] : make_uint4(0, 0, 0, 0);
        warp_for_each_cell(r, 0, 0u, ok, k, [&](int cx, int cy, SegRec, int32_t, uint32_t) {
            atomicAdd(&cell_cnt[cy * G + cx], 1u);
        });
    }
}

// Work items of the pair kernel: a cell with n segments has T = ceil(n / 32)
// tiles and T (T + 1) / 2 tile pairs.  Also sums the candidate pairs
// n (n - 1) / 2 of all cells.
__global__ void __launch_bounds__(256) k_cell_items(const uint32_t *__restrict__ cell_off, int C,
                                                    uint32_t *__restrict__ item_cnt, DevAcc *acc) {
    __shared__ uint64_t sh[32];
    uint64_t w = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const uint32_t n = cell_off[c + 1] - cell_off[c];
        const uint64_t T = (n + TILE - 1) / TILE;
        const uint64_t items = n < 2 ? 0 : T * (T + 1) / 2;
        if (items > 0x7fffffffull) atomicOr(&acc->grid_flags, GF_ITEMS_OVERFLOW);
        item_cnt[c] = (uint32_t)min(items, (uint64_t)0x7fffffffull);
        w += (uint64_t)n * (n - (n > 0)) / 2;
    }
    w = block_sum<uint64_t>(w, sh);
    if (threadIdx.x == 0) atomic_add_u64(&acc->grid_work, w);
}

// a4 -- scatter of the records into their cells: the segment record and its
// edge id go to cell_off[c] + (running count of cell c).
__global__ void __launch_bounds__(256) k_grid_fill(const SegRec *__restrict__ seg,
                                                   const int32_t *__restrict__ seg_eid,
                                                   const uint32_t *__restrict__ seg_theta,
                                                   const DevAcc *__restrict__ acc, int k,
                                                   const uint32_t *__restrict__ cell_off,
                                                   uint32_t *__restrict__ cell_fill, uint64_t cap,
                                                   SegRec *__restrict__ rec, int32_t *__restrict__ rec_eid,
                                                   uint32_t *__restrict__ rec_theta, uint32_t *status) {
    const int64_t n = acc->n_seg;
    const int G = 65536 >> k;
    if (acc->records > cap) {  // sized from the same counts; cannot happen unless inputs changed
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_OVERFLOW);
        return;
    }
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const SegRec r = ok ? seg[i] : make_uint4(0, 0, 0, 0);
        const int32_t eid = ok ? seg_eid[i] : 0;
        const uint32_t th = ok ? seg_theta[i] : 0u;
        warp_for_each_cell(r, eid, th, ok, k, [&](int cx, int cy, SegRec q, int32_t qe, uint32_t qt) {
            const int c = cy * G + cx;
            const uint32_t pos = cell_off[c] + atomicAdd(&cell_fill[c], 1u);
            rec[pos] = q;
            rec_eid[pos] = qe;
            rec_theta[pos] = qt;
        });
    }
}

// Owner test of an E_c pair: the intersection point P = a + u t with
// t = ((c - a) x v) / (u x v) lies in the half-open cell [x0, x0 + w) x
// [y0, y0 + w).  All products are exact in int64 (|P_x * den| < 2^52).
__device__ __forceinline__ bool owns_crossing(const RowSeg &r, const ColSeg &c, int x0, int y0, int w) {
    long long den = (long long)r.ux * c.vy - (long long)r.uy * c.vx;
    long long num = (long long)(c.cx - r.ax) * c.vy - (long long)(c.cy - r.ay) * c.vx;
    if (den < 0) { den = -den; num = -num; }
    const long long X = (long long)r.ax * den + (long long)r.ux * num;
    const long long Y = (long long)r.ay * den + (long long)r.uy * num;
    return (long long)x0 * den <= X && X < (long long)(x0 + w) * den &&
           (long long)y0 * den <= Y && Y < (long long)(y0 + w) * den;
}

// Owner of a collinear overlap: the cell of the lexicographically smallest
// point of the overlap, which is an endpoint of one of the segments.
__device__ __forceinline__ bool owns_collinear(const RowSeg &r, const ColSeg &c, int cx, int cy, int k) {
    const uint32_t ka = lex_key(r.ax, r.ay), kb = lex_key(r.bx, r.by);
    const uint32_t kc = lex_key(c.cx, c.cy), kd = lex_key(c.dx, c.dy);
    const uint32_t lo = max(min(ka, kb), min(kc, kd));
    return (int(lo >> 16) >> k) == cx && (int(lo & 0xffffu) >> k) == cy;
}

// a6 -- one warp per work item (cell, row tile ti, column tile tj), items in a
// warp-strided static order.  Off-diagonal items test all rows x columns;
// diagonal items use a rotation schedule (round q pairs lane i with
// (i + q) mod m) so that every lane has work in every round.
template <bool PER_EDGE>
__global__ void __launch_bounds__(GP_WARPS * 32) k_grid_pairs(
    const SegRec *__restrict__ rec, const int32_t *__restrict__ rec_eid, const uint32_t *__restrict__ rec_theta,
    const uint32_t *__restrict__ cell_off, const uint32_t *__restrict__ item_off, int C, int k,
    DevAcc *acc, uint32_t ideal, PerEdge pe) {
    __shared__ ColSeg cs[GP_WARPS][TILE];
    __shared__ int32_t ceid[GP_WARPS][PER_EDGE ? TILE : 1];
    __shared__ uint64_t shu[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int G = 65536 >> k, w = 1 << k;
    const uint32_t n_items = item_off[C];
    PairCounts pc;
    for (uint32_t it = blockIdx.x * GP_WARPS + wid; it < n_items; it += gridDim.x * GP_WARPS) {
        // cell of this item: largest c with item_off[c] <= it (binary search)
        int lo = 0, hi = C - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const int cell = lo;
        const uint32_t q = it - item_off[cell];
        int r = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
        while (r * (r + 1) / 2 > (int)q) --r;
        while ((r + 1) * (r + 2) / 2 <= (int)q) ++r;
        const int tj = r, ti = (int)q - r * (r + 1) / 2;
        const uint32_t base = cell_off[cell];
        const int n = (int)(cell_off[cell + 1] - base);
        const int cx = cell % G, cy = cell / G;
        const int x0 = cx << k, y0 = cy << k;
        const int mr = min(TILE, n - ti * TILE), mc = min(TILE, n - tj * TILE);

        __syncwarp();
        if (lane < mc) {
            cs[wid][lane] = make_col(rec[base + tj * TILE + lane], rec_theta[base + tj * TILE + lane]);
            if (PER_EDGE) ceid[wid][lane] = rec_eid[base + tj * TILE + lane];
        }
        RowSeg rs;
        int32_t reid = 0;
        if (lane < mr) {
            rs = make_row(rec[base + ti * TILE + lane], rec_theta[base + ti * TILE + lane]);
            if (PER_EDGE) reid = rec_eid[base + ti * TILE + lane];
        }
        __syncwarp();
        if (lane >= mr) continue;

        const bool diag = ti == tj;
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
            const ColSeg c = cs[wid][jj];
            const int kind = classify_kind(rs, c);
            if (kind == PAIR_NONE) continue;
            if (kind == PAIR_COLLINEAR) {
                if (!owns_collinear(rs, c, cx, cy, k)) continue;
                ++pc.collinear;
                if (PER_EDGE) {
                    atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 2], 1ull);
                    atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)ceid[wid][jj] + 2], 1ull);
                }
                continue;
            }
            if (!owns_crossing(rs, c, x0, y0, w)) continue;
            const uint32_t qd = dev_term(rs.th, c.th, ideal);
            pc.dev += qd;
            if (kind == PAIR_PROPER) ++pc.proper; else ++pc.touching;
            if (PER_EDGE) {
                const int slot = kind == PAIR_PROPER ? 0 : 1;
                atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + slot], 1ull);
                atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)ceid[wid][jj] + slot], 1ull);
                atomicAdd((unsigned long long *)&pe.dev[reid], (unsigned long long)qd);
                atomicAdd((unsigned long long *)&pe.dev[ceid[wid][jj]], (unsigned long long)qd);
            }
        }
    }
    flush_counts(pc, acc, shu);
}

int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

void launch_grid_count(const Buffers &b, int64_t E, const GridBuffers &g, int k, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    cudaMemsetAsync(g.cell_off, 0, sizeof(uint32_t) * (C + 1), s);
    count_launches(E > 0 ? 2 : 1);
    if (E > 0) k_grid_count<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.acc, k, g.cell_off);
    launch_scan_u32(g.cell_off, g.cell_off, C, b.scan_tmp, &b.acc->records, &b.acc->eval_status, s);
    k_cell_items<<<grid_for(C, 256, 152 * 8), 256, 0, s>>>(g.cell_off, C, g.item_off, b.acc);
    launch_scan_u32(g.item_off, g.item_off, C, b.scan_tmp, &b.acc->grid_items, &b.acc->eval_status, s);
}

void launch_grid_scatter(const Buffers &b, int64_t E, const GridBuffers &g, int k, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    cudaMemsetAsync(g.cell_fill, 0, sizeof(uint32_t) * C, s);
    if (E <= 0) return;
    count_launches(1);
    k_grid_fill<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc, k, g.cell_off,
                                                           g.cell_fill, g.rec_cap, g.rec, g.rec_eid, g.rec_theta,
                                                           &b.acc->eval_status);
}

void launch_grid_pairs(const Buffers &b, const GridBuffers &g, int k, uint64_t n_items, uint32_t ideal,
                       PerEdge pe, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    if (n_items == 0) return;
    const int blocks = grid_for((int64_t)n_items, GP_WARPS, 152 * 8);
    count_launches(1);
    if (pe.counts)
        k_grid_pairs<true><<<blocks, GP_WARPS * 32, 0, s>>>(g.rec, g.rec_eid, g.rec_theta, g.cell_off, g.item_off,
                                                           C, k, b.acc, ideal, pe);
    else
        k_grid_pairs<false><<<blocks, GP_WARPS * 32, 0, s>>>(g.rec, g.rec_eid, g.rec_theta, g.cell_off,
                                                            g.item_off, C, k, b.acc, ideal, pe);
}

}  // namespace gr
