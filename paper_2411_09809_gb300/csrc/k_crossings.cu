// k_crossings.cu -- the tiled all-pairs crossing kernels (a7).
//
// Every unordered pair of compacted segments is tested once: square tiles
// (row tile bi <= column tile bj) are enumerated in lower-triangular order
// and diagonal tiles keep only column > row.
#include <math.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

namespace {

__device__ __forceinline__ void decode_tile(int64_t t, int &bi, int &bj) {
    // t = r (r + 1) / 2 + c with c <= r; (bi, bj) = (c, r)
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    bj = (int)r;
    bi = (int)(t - r * (r + 1) / 2);
}

// ----------------------------------------------------------- aggregate a7
//
// FP32 fast path with an exact fallback.  For integer coordinates below 2^16
// the orientation u x p - k (k rounded to FP32, |k| < 2^33) evaluated as
// fma(u_x, p_y, fma(-u_y, p_x, -k)) is off by at most 256 + 512 + 1024 =
// 1792 (half an ulp of k, of the inner fma result < 2^34 and of the outer one
// < 2^35).  When all four orientations of a pair exceed kOrientFilter in
// magnitude their signs are exact and none is zero, so the pair crosses
// properly iff both sign products are negative.  Any pair with a smaller
// orientation -- which includes every pair sharing an endpoint, every
// collinear and every touching pair -- is re-decided exactly in int64.
constexpr float kOrientFilter = 4096.f;

constexpr int AG_THREADS = 256;
constexpr int AG_RPT = 2;                  // rows per thread
constexpr int AG_ROWS = AG_THREADS * AG_RPT;
constexpr int AG_COLS = AG_ROWS;           // square tiles: diagonal test is local j > local i

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
    r.ax = (float)ax; r.ay = (float)ay; r.bx = (float)bx; r.by = (float)by;
    r.ux = (float)ux; r.uy = (float)uy;
    r.nk = -(float)((long long)ux * ay - (long long)uy * ax);
    r.th = th;
    return r;
}

__device__ __forceinline__ FCol make_fcol(SegRec s, uint32_t th) {
    FCol c;
    const int cx = px(s.x), cy = py(s.x), dx = px(s.y), dy = py(s.y);
    const int vx = dx - cx, vy = dy - cy;
    c.cx = (float)cx; c.cy = (float)cy; c.dx = (float)dx; c.dy = (float)dy;
    c.vx = (float)vx; c.vy = (float)vy;
    c.nk = -(float)((long long)vx * cy - (long long)vy * cx);
    c.th = th;
    return c;
}

// One block per square tile (grid-strided).  Each thread holds AG_RPT row
// segments; the columns are staged in shared memory in FP32 form (plus the
// raw records for the exact fallback) and read by broadcast.
__global__ void __launch_bounds__(AG_THREADS) k_cross_allpairs_agg(const SegRec *__restrict__ seg,
                                                                   const uint32_t *__restrict__ theta,
                                                                   DevAcc *acc, uint32_t ideal, int64_t tiles) {
    __shared__ FCol fc[AG_COLS];
    __shared__ SegRec raw[AG_COLS];
    __shared__ uint64_t shu[32];
    const int n_seg = (int)acc->n_seg;
    PairCounts pc;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int bi, bj;
        decode_tile(t, bi, bj);
        const int j0 = bj * AG_COLS;
        if (j0 >= n_seg) continue;
        const int nc = min(AG_COLS, n_seg - j0);
        __syncthreads();
        for (int c = threadIdx.x; c < nc; c += AG_THREADS) {
            const SegRec s = seg[j0 + c];
            raw[c] = s;
            fc[c] = make_fcol(s, theta[j0 + c]);
        }
        FRow rs[AG_RPT];
        SegRec rr[AG_RPT];
        bool rok[AG_RPT];
#pragma unroll
        for (int k = 0; k < AG_RPT; ++k) {
            const int i = bi * AG_ROWS + threadIdx.x + k * AG_THREADS;
            rok[k] = i < n_seg;
            rr[k] = rok[k] ? seg[i] : make_uint4(0, 0, 0, 0);
            rs[k] = make_frow(rr[k], rok[k] ? theta[i] : 0u);
        }
        __syncthreads();
        const bool diag = bi == bj;
#pragma unroll 2
        for (int jj = 0; jj < nc; ++jj) {
            const FCol c = fc[jj];
            bool unsure[AG_RPT];
            bool any_unsure = false;
#pragma unroll
            for (int k = 0; k < AG_RPT; ++k) {
                const FRow &r = rs[k];
                const float o1 = fmaf(r.ux, c.cy, fmaf(-r.uy, c.cx, r.nk));
                const float o2 = fmaf(r.ux, c.dy, fmaf(-r.uy, c.dx, r.nk));
                const float o3 = fmaf(c.vx, r.ay, fmaf(-c.vy, r.ax, c.nk));
                const float o4 = fmaf(c.vx, r.by, fmaf(-c.vy, r.bx, c.nk));
                const float mn = fminf(fminf(fabsf(o1), fabsf(o2)), fminf(fabsf(o3), fabsf(o4)));
                const bool valid = rok[k] && (!diag || jj > (int)threadIdx.x + k * AG_THREADS);
                const bool sure = mn > kOrientFilter;
                const int sx = (__float_as_int(o1) ^ __float_as_int(o2)) & (__float_as_int(o3) ^ __float_as_int(o4));
                const bool hit = valid && sure && sx < 0;
                pc.proper += hit ? 1u : 0u;
                pc.dev += hit ? dev_term(r.th, c.th, ideal) : 0u;
                unsure[k] = valid && !sure;
                any_unsure |= unsure[k];
            }
            if (__any_sync(0xffffffffu, any_unsure)) {
#pragma unroll
                for (int k = 0; k < AG_RPT; ++k) {
                    if (!unsure[k]) continue;
                    const RowSeg er = make_row(rr[k], rs[k].th);
                    const ColSeg ec = make_col(raw[jj], c.th);
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
    flush_counts(pc, acc, shu);
}

// ------------------------------------------------------------ per-edge a7
// Exact int64 classification of every pair, with per-edge tallies (atomics).
constexpr int PE_ROWS = 256;
constexpr int PE_COLS = 256;

__global__ void __launch_bounds__(PE_ROWS) k_cross_allpairs_per_edge(const SegRec *__restrict__ seg,
                                                                     const int32_t *__restrict__ seg_eid,
                                                                     const uint32_t *__restrict__ theta,
                                                                     DevAcc *acc, uint32_t ideal, PerEdge pe,
                                                                     int64_t tiles) {
    __shared__ ColSeg cs[PE_COLS];
    __shared__ int32_t ceid[PE_COLS];
    __shared__ uint64_t shu[32];
    const int n_seg = (int)acc->n_seg;
    PairCounts pc;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int bi, bj;
        decode_tile(t, bi, bj);
        const int j0 = bj * PE_COLS;
        if (j0 >= n_seg) continue;
        const int nc = min(PE_COLS, n_seg - j0);
        __syncthreads();
        if (threadIdx.x < nc) {
            cs[threadIdx.x] = make_col(seg[j0 + threadIdx.x], theta[j0 + threadIdx.x]);
            ceid[threadIdx.x] = seg_eid[j0 + threadIdx.x];
        }
        const int i = bi * PE_ROWS + threadIdx.x;
        const bool row_ok = i < n_seg;
        RowSeg rs;
        int32_t reid = 0;
        if (row_ok) {
            rs = make_row(seg[i], theta[i]);
            reid = seg_eid[i];
        }
        __syncthreads();
        if (!row_ok) continue;
        uint32_t rp = 0, rt = 0, rc = 0;
        uint64_t rdev = 0;
        for (int jj = (bi == bj) ? threadIdx.x + 1 : 0; jj < nc; ++jj) {
            const ColSeg c = cs[jj];
            const int kind = classify_kind(rs, c);
            if (kind == PAIR_NONE) continue;
            const int64_t ce = ceid[jj];
            if (kind == PAIR_COLLINEAR) {
                ++pc.collinear;
                ++rc;
                atomicAdd((unsigned long long *)&pe.counts[3 * ce + 2], 1ull);
                continue;
            }
            const uint32_t dv = dev_term(rs.th, c.th, ideal);
            pc.dev += dv;
            rdev += dv;
            if (kind == PAIR_PROPER) { ++pc.proper; ++rp; } else { ++pc.touching; ++rt; }
            atomicAdd((unsigned long long *)&pe.counts[3 * ce + (kind == PAIR_PROPER ? 0 : 1)], 1ull);
            atomicAdd((unsigned long long *)&pe.dev[ce], (unsigned long long)dv);
        }
        if (rp) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 0], (unsigned long long)rp);
        if (rt) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 1], (unsigned long long)rt);
        if (rc) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 2], (unsigned long long)rc);
        if (rdev) atomicAdd((unsigned long long *)&pe.dev[reid], (unsigned long long)rdev);
    }
    flush_counts(pc, acc, shu);
}

unsigned grid_of(int64_t tiles) {
    return (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
}

}  // namespace

void launch_crossings_allpairs(const Buffers &b, int64_t n_seg, uint32_t ideal, PerEdge pe,
                               cudaStream_t s) {
    if (n_seg < 2) return;
    count_launches(1);
    if (pe.counts) {
        const int64_t nb = (n_seg + PE_ROWS - 1) / PE_ROWS;
        const int64_t tiles = nb * (nb + 1) / 2;
        k_cross_allpairs_per_edge<<<grid_of(tiles), PE_ROWS, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc,
                                                                     ideal, pe, tiles);
    } else {
        const int64_t nb = (n_seg + AG_ROWS - 1) / AG_ROWS;
        const int64_t tiles = nb * (nb + 1) / 2;
        k_cross_allpairs_agg<<<grid_of(tiles), AG_THREADS, 0, s>>>(b.seg, b.seg_theta, b.acc, ideal, tiles);
    }
}

}  // namespace gr
