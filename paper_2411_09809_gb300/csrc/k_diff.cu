// k_diff.cu -- the differentiable form: FP32 coordinates, exact crossing
// predicates, and the adjoint kernels of E_ca, M_l and M_a.
//
// Forward (gr_diff_forward): the crossing set is decided exactly on the FP32
// inputs (each orientation through an FP32 error-bound filter, an FP64 one,
// then exact expansion arithmetic), E_c pairs are saved for the backward;
// M_l from FP64 lengths; M_a from FP64 direction angles, each vertex's
// smallest gap saved for the backward.  Backward (gr_diff_backward): with
// that crossing set and those gaps held fixed, the gradient of
// g0 * E_ca + g1 * M_l + g2 * M_a with respect to every coordinate, scattered
// with atomics into an FP32 [V][2] array.
#include <cooperative_groups.h>
#include <math.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace cg = cooperative_groups;

namespace gr {

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t ord_f(float f) {  // order-preserving float -> uint
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

// ---------------------------------------------------------- predicates
// Orientation of (p, q, r): sign of (q - p) x (r - p) for FP32 points, by the
// adaptive method of Shewchuk ("Adaptive Precision Floating-Point Arithmetic
// and Fast Robust Geometric Predicates", 1997): evaluate
//   t1 = (q_x - p_x)(r_y - p_y),  t2 = (q_y - p_y)(r_x - p_x),  d = t1 - t2
// in a floating-point format with unit roundoff e; the sign of d is the true
// sign when |d| > (3 + 16 e) e (|t1| + |t2|).  FP32 first, then FP64, then
// the exact value as a floating-point expansion.

__device__ __forceinline__ void fast_two_sum_any(double a, double b, double &s, double &t) {
    s = a + b;
    const double bb = s - a;
    t = (a - (s - bb)) + (b - bb);
}

// e (n non-overlapping components, increasing magnitude) += x; zero
// components dropped.
__device__ __forceinline__ int expansion_add(double *e, int n, double x) {
    double q = x;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        double s, t;
        fast_two_sum_any(q, e[i], s, t);
        q = s;
        if (t != 0.0) e[m++] = t;
    }
    if (q != 0.0 || m == 0) e[m++] = q;
    return m;
}

__device__ __noinline__ int orient_exact(double px, double py, double qx, double qy, double rx, double ry) {
    double a[2][2], b[2][2];  // (q - p), (r - p): [coordinate][hi, lo]
    fast_two_sum_any(qx, -px, a[0][0], a[0][1]);
    fast_two_sum_any(qy, -py, a[1][0], a[1][1]);
    fast_two_sum_any(rx, -px, b[0][0], b[0][1]);
    fast_two_sum_any(ry, -py, b[1][0], b[1][1]);
    double e[36];
    int n = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double p1 = a[0][i] * b[1][j], p1e = fma(a[0][i], b[1][j], -p1);
            const double p2 = -a[1][i] * b[0][j], p2e = fma(-a[1][i], b[0][j], -p2);
            n = expansion_add(e, n, p1e);
            n = expansion_add(e, n, p1);
            n = expansion_add(e, n, p2e);
            n = expansion_add(e, n, p2);
        }
    const double top = e[n - 1];
    return (top > 0.0) - (top < 0.0);
}

__device__ __noinline__ int orient_f64(float px, float py, float qx, float qy, float rx, float ry);

__device__ __forceinline__ int orient_f32(float px, float py, float qx, float qy, float rx, float ry) {
    const float e32 = 5.9604645e-08f;  // 2^-24
    const float t1 = (qx - px) * (ry - py), t2 = (qy - py) * (rx - px), d = t1 - t2;
    const float mag = fabsf(t1) + fabsf(t2);
    // the bound assumes no underflow: products below 2^-100 (or not finite) go on to FP64
    if (mag >= 0x1p-100f) {
        const float b32 = (3.0f + 16.0f * e32) * e32 * mag;
        if (d > b32) return 1;
        if (-d > b32) return -1;
    }
    return orient_f64(px, py, qx, qy, rx, ry);
}

// The FP64 stage and the exact fallback (out of line: rare, and their FP64
// code must not be if-converted into the FP32 callers).
__device__ __noinline__ int orient_f64(float px, float py, float qx, float qy, float rx, float ry) {
    const double e64 = 1.1102230246251565e-16;  // 2^-53
    const double T1 = ((double)qx - (double)px) * ((double)ry - (double)py);
    const double T2 = ((double)qy - (double)py) * ((double)rx - (double)px);
    const double D = T1 - T2;
    const double b64 = (3.0 + 16.0 * e64) * e64 * (fabs(T1) + fabs(T2));
    if (D > b64) return 1;
    if (-D > b64) return -1;
    return orient_exact(px, py, qx, qy, rx, ry);
}

__device__ __forceinline__ bool lex_le(float ax, float ay, float bx, float by) {
    return ax < bx || (ax == bx && ay <= by);
}

// Classification of one pair under the library's rules, exact on FP32.
__device__ __forceinline__ int classify_f32(float4 r, uint2 ri, float4 c, uint2 ci) {
    if ((ri.x == ci.x) | (ri.x == ci.y) | (ri.y == ci.x) | (ri.y == ci.y)) return PAIR_NONE;
    const int o1 = orient_f32(r.x, r.y, r.z, r.w, c.x, c.y);
    const int o2 = orient_f32(r.x, r.y, r.z, r.w, c.z, c.w);
    if (o1 * o2 > 0) return PAIR_NONE;
    const int o3 = orient_f32(c.x, c.y, c.z, c.w, r.x, r.y);
    const int o4 = orient_f32(c.x, c.y, c.z, c.w, r.z, r.w);
    if (o3 * o4 > 0) return PAIR_NONE;
    if (o1 == 0 && o2 == 0) {
        const bool ar = lex_le(r.x, r.y, r.z, r.w), ac = lex_le(c.x, c.y, c.z, c.w);
        const float elx = ar ? r.x : r.z, ely = ar ? r.y : r.w, ehx = ar ? r.z : r.x, ehy = ar ? r.w : r.y;
        const float flx = ac ? c.x : c.z, fly = ac ? c.y : c.w, fhx = ac ? c.z : c.x, fhy = ac ? c.w : c.y;
        const bool le = lex_le(flx, fly, elx, ely);  // lo = max of the minima
        const float lx = le ? elx : flx, ly = le ? ely : fly;
        const bool he = lex_le(ehx, ehy, fhx, fhy);  // hi = min of the maxima
        const float hx = he ? ehx : fhx, hy = he ? ehy : fhy;
        return lex_le(lx, ly, hx, hy) ? PAIR_COLLINEAR : PAIR_NONE;
    }
    return (o1 != 0 && o2 != 0 && o3 != 0 && o4 != 0) ? PAIR_PROPER : PAIR_TOUCHING;
}

// The FP32 filter stage of orient_f32 alone, for a line given by a point p
// and its direction u = q - p (rounded as orient_f32 rounds it): +-1 when the
// filter decides the sign, 0 when the FP64 stage would be needed.
__device__ __forceinline__ int orient_f32_filter(float ux, float uy, float px, float py, float rx, float ry) {
    const float e32 = 5.9604645e-08f;  // 2^-24
    const float t1 = ux * (ry - py), t2 = uy * (rx - px), d = t1 - t2;
    const float mag = fabsf(t1) + fabsf(t2);
    const float b32 = (3.0f + 16.0f * e32) * e32 * mag;
    return mag >= 0x1p-100f ? (d > b32 ? 1 : (-d > b32 ? -1 : 0)) : 0;
}

__device__ __noinline__ int classify_f32_slow(float4 r, uint2 ri, float4 c, uint2 ci) {
    return classify_f32(r, ri, c, ci);
}

// classify_f32 with the four orientations evaluated without branches by the
// FP32 filter (the row's direction ru given): a pair whose four signs the
// filter decides is settled here, any other goes to classify_f32.  Same
// result: a decided sign is the exact one.
__device__ __forceinline__ int classify_f32_fast(const float4 &r, float rux, float ruy, uint2 ri, const float4 &c,
                                                 uint2 ci) {
    if ((ri.x == ci.x) | (ri.x == ci.y) | (ri.y == ci.x) | (ri.y == ci.y)) return PAIR_NONE;
    const float cux = c.z - c.x, cuy = c.w - c.y;
    const int s1 = orient_f32_filter(rux, ruy, r.x, r.y, c.x, c.y);
    const int s2 = orient_f32_filter(rux, ruy, r.x, r.y, c.z, c.w);
    const int s3 = orient_f32_filter(cux, cuy, c.x, c.y, r.x, r.y);
    const int s4 = orient_f32_filter(cux, cuy, c.x, c.y, r.z, r.w);
    if (s1 * s2 > 0 || s3 * s4 > 0) return PAIR_NONE;  // one segment strictly on one side of the other's line
    if (s1 != 0 && s2 != 0 && s3 != 0 && s4 != 0) return PAIR_PROPER;
    return classify_f32_slow(r, ri, c, ci);
}

__device__ __forceinline__ void tally(int kind, uint32_t ta, uint32_t tb, uint32_t ideal, PairCounts &pc) {
    if (kind == PAIR_COLLINEAR) ++pc.collinear;
    else if (kind == PAIR_PROPER) ++pc.proper;
    else if (kind == PAIR_TOUCHING) ++pc.touching;
    if (kind == PAIR_PROPER || kind == PAIR_TOUCHING) pc.dev += dev_term(ta, tb, ideal);
}

// The sign of an E_c pair's term in d E_ca / d theta for the pair's first
// direction ta (the second gets the opposite): a_c is the acute angle
// between the lines (d = ta - tb mod pi, a_c = d or pi - d) and d|a_c -
// ideal| / d theta_a = sign(a_c - ideal) (negated when folded).  Read from the
// same integer directions the forward's terms use.
__device__ __forceinline__ int diff_sign(uint32_t ta, uint32_t tb, uint32_t ideal_u) {
    const uint32_t dd = ta - tb;
    const bool folded = dd > 0x80000000u;  // a_c = pi - d
    const uint32_t a = folded ? 0u - dd : dd;
    const int sgn = a > ideal_u ? 1 : (a < ideal_u ? -1 : 0);
    return folded ? -sgn : sgn;
}

// ------------------------------------------------------------------ gather
// Direction of the line through (dx, dy) (FP64), in units of pi / 2^32.
__device__ __forceinline__ uint32_t line_direction_d(double dx, double dy) {
    double t = atan2(dy, dx);
    if (t < 0.0) t += 3.14159265358979323846;
    return (uint32_t)(unsigned long long)rint(t * (4294967296.0 / 3.14159265358979323846));
}

// a1 for FP32 coordinates: ids and finiteness checked; seg holds the FP32
// endpoints (as bits), seg_ids the vertex ids; len2 the FP64 squared length
// (as bits) of every edge.
__global__ void __launch_bounds__(256) k_gather_f32(const float2 *__restrict__ xy, int64_t V,
                                                    const int2 *__restrict__ edges, int64_t E,
                                                    float4 *__restrict__ seg, uint2 *__restrict__ seg_ids,
                                                    int32_t *__restrict__ seg_eid, uint32_t *__restrict__ seg_theta,
                                                    int64_t *__restrict__ len2, DevAcc *acc) {
    __shared__ uint32_t h[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < E; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = base + threadIdx.x;
        bool keep = false, zero = false;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        int2 ed = make_int2(0, 0);
        double l2 = 0.0;
        if (e < E) {
            ed = edges[e];
            if (ed.x < 0 || ed.y < 0 || ed.x >= V || ed.y >= V || ed.x == ed.y) {
                atomicOr(&acc->status, ST_BAD_ID);
            } else {
                const float2 a = xy[ed.x], b = xy[ed.y];
                if (!isfinite(a.x) || !isfinite(a.y) || !isfinite(b.x) || !isfinite(b.y)) {
                    atomicOr(&acc->status, ST_BAD_COORD);
                } else if (a.x == b.x && a.y == b.y) {
                    zero = true;
                } else {
                    keep = true;
                    r = make_float4(a.x, a.y, b.x, b.y);
                    const double dx = (double)b.x - (double)a.x, dy = (double)b.y - (double)a.y;
                    l2 = dx * dx + dy * dy;
                }
            }
            len2[e] = __double_as_longlong(l2);
        }
        const unsigned mk = __ballot_sync(0xffffffffu, keep);
        const unsigned mz = __ballot_sync(0xffffffffu, zero);
        uint32_t slot = 0;
        if (lane == 0 && mk) slot = atomicAdd(&acc->n_seg, (uint32_t)__popc(mk));
        if (lane == 0 && mz) atomicAdd((unsigned long long *)&acc->zero_len, (unsigned long long)__popc(mz));
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (keep) {
            const uint32_t pos = slot + __popc(mk & lanemask_lt());
            seg[pos] = r;
            seg_ids[pos] = make_uint2((uint32_t)ed.x, (uint32_t)ed.y);
            seg_eid[pos] = (int32_t)e;
            seg_theta[pos] = line_direction_d((double)r.z - (double)r.x, (double)r.w - (double)r.y);
            // statistics for the crossing grid: major-axis length class and the bounding box
            const float m = fmaxf(fabsf(r.z - r.x), fabsf(r.w - r.y));
            const int cls = min(max(ilogbf(m) + 48, 0), 63);
            atomicAdd(&h[cls], 1u);
        }
        uint32_t mnx = keep ? min(ord_f(r.x), ord_f(r.z)) : 0xffffffffu, mny = keep ? min(ord_f(r.y), ord_f(r.w)) : 0xffffffffu;
        uint32_t mxx = keep ? max(ord_f(r.x), ord_f(r.z)) : 0u, mxy = keep ? max(ord_f(r.y), ord_f(r.w)) : 0u;
        for (int o = 16; o > 0; o >>= 1) {
            mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
            mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
            mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
            mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        }
        if (lane == 0 && mk) {
            atomicMin(&acc->f32_bounds[0], mnx);
            atomicMin(&acc->f32_bounds[1], mny);
            atomicMax(&acc->f32_bounds[2], mxx);
            atomicMax(&acc->f32_bounds[3], mxy);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (h[i]) atomicAdd(&acc->f32_hist[i], h[i]);
}

__global__ void __launch_bounds__(256) k_check_vertices_f32(const float2 *__restrict__ xy, int64_t V, DevAcc *acc) {
    bool bad = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = xy[v];
        bad |= !isfinite(p.x) || !isfinite(p.y);
    }
    if (bad) atomicOr(&acc->status, ST_BAD_COORD);
}

// ------------------------------------------------------- crossings (FP32)
constexpr int DF_ROWS = 256;
constexpr int DF_COLS = 256;

__device__ __forceinline__ void decode_tile(int64_t t, int &bi, int &bj) {
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    bj = (int)r;
    bi = (int)(t - r * (r + 1) / 2);
}

// Exclusive prefix of v over the warp; *total = the warp's sum.  Every lane
// must call it.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t *total) {
    const int lane = threadIdx.x & 31;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    *total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}


// All-pairs tiles over n FP32 segments (n = *n_p on the device): the
// compacted segments themselves, or those listed in idx.  E_c pairs
// (compacted segment indices) are appended to `pairs` (warp-aggregated), at
// most `cap` of them; the total goes to acc->records.  tiles < 0: sized on
// the device (a persistent launch).
__global__ void __launch_bounds__(DF_ROWS) k_cross_f32(const float4 *__restrict__ seg, const uint2 *__restrict__ ids,
                                                       const uint32_t *__restrict__ theta,
                                                       const uint32_t *__restrict__ idx, const uint32_t *__restrict__ n_p,
                                                       DevAcc *acc, uint32_t ideal, int64_t tiles,
                                                       int32_t *__restrict__ cnt) {
    __shared__ float4 cs[DF_COLS];
    __shared__ uint2 cid[DF_COLS];
    __shared__ uint32_t cth[DF_COLS];
    __shared__ uint32_t cix[DF_COLS];
    __shared__ int ccnt[DF_COLS];  // the columns' signed counts in this tile
    __shared__ uint64_t shu[32];
    const int n_seg = (int)*n_p;
    if (tiles < 0) {
        const int64_t nb = (n_seg + DF_ROWS - 1) / DF_ROWS;
        tiles = nb * (nb + 1) / 2;
    }
    PairCounts pc;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int bi, bj;
        decode_tile(t, bi, bj);
        const int j0 = bj * DF_COLS;
        if (j0 >= n_seg) continue;
        const int nc = min(DF_COLS, n_seg - j0);
        __syncthreads();
        if (threadIdx.x < nc) {
            const uint32_t q = idx ? idx[j0 + threadIdx.x] : (uint32_t)(j0 + threadIdx.x);
            cs[threadIdx.x] = seg[q];
            cid[threadIdx.x] = ids[q];
            cth[threadIdx.x] = theta[q];
            cix[threadIdx.x] = q;
            ccnt[threadIdx.x] = 0;
        }
        const int i = bi * DF_ROWS + threadIdx.x;
        const bool row_ok = i < n_seg;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        uint2 ri = make_uint2(0xffffffffu, 0xfffffffeu);
        uint32_t rth = 0, rix = 0;
        if (row_ok) {
            rix = idx ? idx[i] : (uint32_t)i;
            r = seg[rix];
            ri = ids[rix];
            rth = theta[rix];
        }
        const float rux = r.z - r.x, ruy = r.w - r.y;
        __syncthreads();
        const bool diag = bi == bj;
        // classify and tally; with `cnt`, each E_c pair's sign (diff_sign)
        // goes to the row's count (a register) and its column's (shared
        // memory), written once per tile
        int rsum = 0;
        for (int jj = 0; jj < nc; ++jj) {
            const bool valid = row_ok && (!diag || jj > (int)threadIdx.x);
            const int kind = valid ? classify_f32_fast(r, rux, ruy, ri, cs[jj], cid[jj]) : PAIR_NONE;
            if (kind == PAIR_NONE) continue;
            tally(kind, rth, cth[jj], ideal, pc);
            if (cnt && (kind == PAIR_PROPER || kind == PAIR_TOUCHING)) {
                const int sg = diff_sign(rth, cth[jj], ideal);
                rsum += sg;
                if (sg) atomicAdd(&ccnt[jj], -sg);
            }
        }
        if (cnt) {
            if (rsum) atomicAdd(&cnt[rix], rsum);
            __syncthreads();
            if (threadIdx.x < nc && ccnt[threadIdx.x]) atomicAdd(&cnt[cix[threadIdx.x]], ccnt[threadIdx.x]);
        }
    }
    flush_counts(pc, acc, shu);
}

// ------------------------------------------------- crossing grid (FP32)
// The crossing set on FP32 coordinates is decided exactly (classify_f32); the
// grid only chooses which pairs are tested and where each is counted.  Cells:
// a G x G grid over the segments' bounding box, cell of a coordinate
// cx(x) = clamp(floor((x - x0) * inv_w)) in FP32 with explicit rounding: a
// non-decreasing function, so the cell range of a segment's bounding box
// [cx(min x), cx(max x)] x [cy(min y), cy(max y)] holds the cell of every
// point of the segment rounded to FP32.
//   short  bounding box within 2 x 2 cells: registered in each of its (1, 2
//          or 4) cells.  Two short segments meet only in cells of both
//          boxes, a rectangle; their pair is counted in its smallest cell
//          (max of the box minima), so once.
//   long   the rest.  Its walk: for each column (or row, along its major
//          axis) the cells the segment can reach there, computed in FP64 with
//          a margin (a superset of the cells of its points).  A long x short
//          pair is tested in every walked cell holding the short one and
//          counted in the first cell of the short's box (in row-major order)
//          that the walk covers; the cell of the intersection point is one of
//          them, so the pair is counted once.
//   long x long pairs go to all-pairs tiles over the list of long segments.
struct FGrid {
    float x0, y0, inv_w;
    int G;
    double w, mx, my;  // cell side; walk margins (x, y)
};


__device__ __forceinline__ int fcell(float v, float o, float inv_w, int G) {
    const float t = __fmul_rn(__fsub_rn(v, o), inv_w);
    const int c = t < 1.0e9f ? (t > -1.0e9f ? (int)floorf(t) : 0) : G - 1;
    return min(max(c, 0), G - 1);
}

struct CellBox {
    int x0, x1, y0, y1;
};

__device__ __forceinline__ CellBox cell_box(float4 r, const FGrid &g) {
    CellBox b;
    b.x0 = fcell(fminf(r.x, r.z), g.x0, g.inv_w, g.G);
    b.x1 = fcell(fmaxf(r.x, r.z), g.x0, g.inv_w, g.G);
    b.y0 = fcell(fminf(r.y, r.w), g.y0, g.inv_w, g.G);
    b.y1 = fcell(fmaxf(r.y, r.w), g.y0, g.inv_w, g.G);
    return b;
}

__device__ __forceinline__ bool is_short_box(const CellBox &b) { return b.x1 - b.x0 <= 1 && b.y1 - b.y0 <= 1; }

// A short segment's record in a cell: its endpoints, vertex ids, direction
// and compacted index, so the pair passes read one 32-byte record instead of
// chasing an index into three arrays.
struct __align__(16) FRec {
    float4 s;
    uint2 ids;
    uint32_t th, i;
};

// The walk of a long segment: along its major axis (x when |dx| >= |dy|),
// line i of [lo, hi] covers minor cells [a, b].
struct Walk {
    bool xmajor;
    int lo, hi;
    double ax, ay, bx, by;  // endpoints, in (major, minor) order
    double slope;           // d minor / d major
    double lo_m, hi_m;      // the segment's extent along the major axis
    double o_maj, o_min;    // grid origin (major, minor)
    float o_min_f, inv_w;
    int G;
    double w, m_maj, m_min;
};

__device__ __forceinline__ Walk make_walk(float4 r, const FGrid &g) {
    Walk k;
    const double dx = (double)r.z - r.x, dy = (double)r.w - r.y;
    k.xmajor = fabs(dx) >= fabs(dy);
    const float a_maj = k.xmajor ? r.x : r.y, b_maj = k.xmajor ? r.z : r.w;
    k.ax = k.xmajor ? r.x : r.y; k.ay = k.xmajor ? r.y : r.x;
    k.bx = k.xmajor ? r.z : r.w; k.by = k.xmajor ? r.w : r.z;
    k.lo_m = fmin(k.ax, k.bx); k.hi_m = fmax(k.ax, k.bx);
    k.slope = k.bx != k.ax ? (k.by - k.ay) / (k.bx - k.ax) : 0.0;
    const float o_maj = k.xmajor ? g.x0 : g.y0;
    k.o_min_f = k.xmajor ? g.y0 : g.x0;
    k.o_maj = o_maj; k.o_min = k.o_min_f;
    k.inv_w = g.inv_w; k.G = g.G; k.w = g.w;
    k.m_maj = k.xmajor ? g.mx : g.my;
    k.m_min = k.xmajor ? g.my : g.mx;
    k.lo = fcell(fminf(a_maj, b_maj), o_maj, g.inv_w, g.G);
    k.hi = fcell(fmaxf(a_maj, b_maj), o_maj, g.inv_w, g.G);
    return k;
}

// Minor cells [a, b] of major line i of the walk (i in [lo, hi]).
__device__ __forceinline__ void walk_line(const Walk &k, int i, int &a, int &b) {
    const double u0 = fmax(k.lo_m, k.o_maj + (double)i * k.w - k.m_maj);
    const double u1 = fmin(k.hi_m, k.o_maj + (double)(i + 1) * k.w + k.m_maj);
    double v0, v1;
    if (k.bx == k.ax) {
        v0 = fmin(k.ay, k.by);
        v1 = fmax(k.ay, k.by);
    } else {
        const double p = k.ay + (u0 - k.ax) * k.slope, q = k.ay + (u1 - k.ax) * k.slope;
        v0 = fmin(p, q);
        v1 = fmax(p, q);
    }
    a = fcell((float)(v0 - k.m_min), k.o_min_f, k.inv_w, k.G);
    b = fcell((float)(v1 + k.m_min), k.o_min_f, k.inv_w, k.G);
}

__device__ __forceinline__ double ulp32(double v) {  // a unit in the last place of FP32 at |v|
    const float f = fabsf((float)v);
    return (double)(nextafterf(f, INFINITY) - f);
}

__global__ void k_f32_grid_setup(const uint32_t *__restrict__ bounds, int G, FGrid *__restrict__ g) {
    FGrid q;
    q.G = G;
    const bool any = bounds[0] <= bounds[2];
    const float x0 = any ? unord_f(bounds[0]) : 0.f, y0 = any ? unord_f(bounds[1]) : 0.f;
    const float x1 = any ? unord_f(bounds[2]) : 0.f, y1 = any ? unord_f(bounds[3]) : 0.f;
    const double span = fmax((double)x1 - x0, (double)y1 - y0);
    q.x0 = x0;
    q.y0 = y0;
    q.w = span > 0.0 ? span / G : 1.0;
    q.inv_w = span > 0.0 ? (float)(G / span) : 0.f;
    // margins: well above the FP32 rounding of the cell function (a few units
    // in the last place of the coordinates) and the FP64 evaluation of the walk
    const double ux = fmax(ulp32(x0), ulp32(x1)), uy = fmax(ulp32(y0), ulp32(y1));
    q.mx = 1e-3 * q.w + 8.0 * ux;
    q.my = 1e-3 * q.w + 8.0 * uy;
    *g = q;
}

// Short segments count their box cells; long ones go to the long list with
// the number of lines of their walk.
__global__ void __launch_bounds__(256) k_f32_grid_count(const float4 *__restrict__ seg, DevAcc *acc,
                                                        const FGrid *__restrict__ gp, uint32_t *__restrict__ cnt,
                                                        uint32_t *__restrict__ long_idx,
                                                        uint32_t *__restrict__ long_lines,
                                                        int2 *__restrict__ walk_meta) {
    const FGrid g = *gp;
    const int64_t n = acc->n_seg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = seg[i];
        const CellBox b = cell_box(r, g);
        if (is_short_box(b)) {
            for (int y = b.y0; y <= b.y1; ++y)
                for (int x = b.x0; x <= b.x1; ++x) atomicAdd(&cnt[y * g.G + x], 1u);
        } else {
            auto grp = cg::coalesced_threads();
            uint32_t base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(&acc->n_long, (uint32_t)grp.size());
            base = grp.shfl(base, 0);
            long_idx[base + grp.thread_rank()] = (uint32_t)i;
            const Walk k = make_walk(r, g);
            long_lines[base + grp.thread_rank()] = (uint32_t)(k.hi - k.lo + 1);
            walk_meta[base + grp.thread_rank()] = make_int2(k.lo, k.xmajor ? 1 : 0);
        }
    }
}

__global__ void __launch_bounds__(256) k_f32_grid_fill(const float4 *__restrict__ seg, const DevAcc *__restrict__ acc,
                                                       const FGrid *__restrict__ gp, const uint32_t *__restrict__ off,
                                                       uint32_t *__restrict__ fill, const uint2 *__restrict__ ids,
                                                       const uint32_t *__restrict__ theta, FRec *__restrict__ rec,
                                                       uint32_t *__restrict__ rec_cell) {
    const FGrid g = *gp;
    const int64_t n = acc->n_seg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = seg[i];
        const CellBox b = cell_box(r, g);
        if (!is_short_box(b)) continue;
        FRec q;
        q.s = r;
        q.ids = ids[i];
        q.th = theta[i];
        q.i = (uint32_t)i;
        for (int y = b.y0; y <= b.y1; ++y)
            for (int x = b.x0; x <= b.x1; ++x) {
                const int c = y * g.G + x;
                const uint32_t pos = off[c] + atomicAdd(&fill[c], 1u);
                rec[pos] = q;
                rec_cell[pos] = (uint32_t)c;
            }
    }
}



// Short x short: one thread per record (row), against the later records of
// its cell; a pair counts only in the smallest cell of both boxes.  Consecutive
// records belong to the same or neighbouring cells, so a warp's rows are
// short loops of similar length.  With `cnt`, each E_c pair's sign
// (diff_sign) goes to its segments' counts: the row's summed in a register,
// the column's by an atomic.  Three blocks an SM
// (at most 85 registers): more warps to hide the record loads than the
// unbounded 96 registers allow.
__global__ void __launch_bounds__(256, 3) k_f32_grid_ss(const float4 *__restrict__ seg, const uint2 *__restrict__ ids,
                                                     const uint32_t *__restrict__ theta, const FGrid *__restrict__ gp,
                                                     const uint32_t *__restrict__ off, const FRec *__restrict__ rec,
                                                     const uint32_t *__restrict__ rec_cell, DevAcc *acc,
                                                     uint32_t ideal, int32_t *__restrict__ cnt) {
    __shared__ uint64_t shu[32];
    const FGrid g = *gp;
    const int lane = threadIdx.x & 31;
    const uint32_t total = off[g.G * g.G];
    const uint32_t stride = gridDim.x * blockDim.x;
    PairCounts pc;
    uint64_t tested = 0;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const uint32_t p = base + lane;
        const bool ok = p < total;
        uint32_t ri = 0, c = 0, end = 0;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        uint2 rid = make_uint2(0, 0);
        uint32_t rth = 0;
        CellBox rb{0, 0, 0, 0};
        if (ok) {
            const FRec fr = rec[p];
            ri = fr.i;
            c = rec_cell[p];
            end = off[c + 1];
            r = fr.s;
            rid = fr.ids;
            rth = fr.th;
            rb = cell_box(r, g);
            tested += end - p - 1;
        }
        const int cxc = (int)(c % (uint32_t)g.G), cyc = (int)(c / (uint32_t)g.G);
        int rsum = 0;  // the row's signed count
        for (uint32_t q = p + 1; ok && q < end; ++q) {
            const FRec fq = rec[q];
            const int kind = classify_f32_fast(r, r.z - r.x, r.w - r.y, rid, fq.s, fq.ids);
            if (kind == PAIR_NONE) continue;
            const CellBox qb = cell_box(fq.s, g);
            if (max(rb.x0, qb.x0) != cxc || max(rb.y0, qb.y0) != cyc) continue;  // not the owner cell
            tally(kind, rth, fq.th, ideal, pc);
            if (cnt && (kind == PAIR_PROPER || kind == PAIR_TOUCHING)) {
                const int sg = diff_sign(rth, fq.th, ideal);
                rsum += sg;
                if (sg) atomicAdd(&cnt[fq.i], -sg);
            }
        }
        if (cnt && rsum) atomicAdd(&cnt[ri], rsum);
    }
    flush_counts(pc, acc, shu);
    tested = block_sum<uint64_t>(tested, shu);
    if (threadIdx.x == 0 && tested) atomic_add_u64(&acc->grid_work, tested);
}

// The minor-cell range [a, b] of every line of every walk (line u of all
// walks belongs to the long segment t with line_off[t] <= u < line_off[t + 1]),
// in FP64 once per line; lines past `cap` are left to the pair kernel.
__global__ void __launch_bounds__(256) k_f32_walk_lines(const float4 *__restrict__ seg, const FGrid *__restrict__ gp,
                                                        const uint32_t *__restrict__ long_idx,
                                                        const uint32_t *__restrict__ line_off, uint32_t line_total_at,
                                                        const DevAcc *__restrict__ acc, uint64_t cap,
                                                        int2 *__restrict__ wl) {
    // one warp per long segment: its walk is set up once per lane (the FP64
    // set-up per line, and a binary search for the line's segment, made the
    // FP64 pipe the bound), then its lines are spread over the lanes
    const FGrid g = *gp;
    const uint32_t n_long = acc->n_long;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < n_long; t += warps) {
        const uint32_t u0 = line_off[t], u1 = (uint32_t)min((uint64_t)line_off[t + 1], cap);
        if (u0 >= u1) continue;
        const Walk k = make_walk(seg[long_idx[t]], g);
        for (uint32_t u = u0 + lane; u < u1; u += 32) {
            int a, b;
            walk_line(k, k.lo + (int)(u - u0), a, b);
            wl[u] = make_int2(a, b);
        }
    }
    (void)line_total_at;
}

// Line i of a walk recomputed (kept out of line: a rare path whose FP64
// code must not be if-converted into its callers).
__device__ __noinline__ int2 line_range_slow(float4 L, FGrid g, int i) {
    const Walk k = make_walk(L, g);
    int a, b;
    walk_line(k, i, a, b);
    return make_int2(a, b);
}

// The range of line i of walk t (lo = its first line), from the table or,
// past its end, recomputed.
__device__ __forceinline__ int2 line_range(const int2 *__restrict__ wl, uint64_t cap, uint32_t off_t, int lo, int i,
                                           const float4 &L, const FGrid &g) {
    const uint64_t u = (uint64_t)off_t + (uint64_t)(i - lo);
    if (u < cap) return wl[u];
    return line_range_slow(L, g, i);
}

// A line of a walk as the lanes of k_f32_grid_ls read it: its long segment,
// the line's place in the walk and the record offset and count prefix of each
// of its first LS_CELLS cells (a line meets few cells: its minor extent is at
// most one cell plus the margins).
constexpr int LS_CELLS = 4;
struct LsLine {
    float4 L;
    uint2 lid;
    uint32_t li, lth, off_t, pre;
    int lo, hi, i, xmaj, j0, ncell;
    uint32_t cstart[LS_CELLS], cum[LS_CELLS + 1];
};

// Long x short: a warp takes 32 consecutive lines of the walks (line u
// belongs to the long segment t with line_off[t] <= u < line_off[t + 1]) and
// spreads the (line, short record) pairs of their cells over its lanes, so
// that every lane tests a pair in every round.  A pair counts only in the
// first cell of the short's box (in row-major order) that the walk covers.
// With `cnt`, each E_c pair's sign (diff_sign) goes to both segments' counts.
__global__ void __launch_bounds__(256) k_f32_grid_ls(const float4 *__restrict__ seg, const uint2 *__restrict__ ids,
                                                     const uint32_t *__restrict__ theta, const FGrid *__restrict__ gp,
                                                     const uint32_t *__restrict__ off, const FRec *__restrict__ rec,
                                                     const uint32_t *__restrict__ long_idx,
                                                     const uint32_t *__restrict__ line_off, uint32_t line_total_at,
                                                     const int2 *__restrict__ walk_meta, const int2 *__restrict__ wl,
                                                     uint64_t wl_cap, DevAcc *acc, uint32_t ideal,
                                                     int32_t *__restrict__ sign_cnt) {
    __shared__ uint64_t shu[32];
    __shared__ LsLine lines[256 / 32][32];
    const FGrid g = *gp;
    const int lane = threadIdx.x & 31;
    LsLine *wl_sh = lines[threadIdx.x >> 5];
    const uint32_t n_long = acc->n_long;
    const uint32_t total = n_long ? line_off[line_total_at] : 0u;
    const uint32_t stride = gridDim.x * blockDim.x;
    PairCounts pc;
    uint64_t tested = 0;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        // this lane's line: its long segment, the line's minor-cell range and its record count
        const uint32_t u = base + lane;
        const bool ok = u < total;
        uint32_t li = 0, off_t = 0;
        int lo = 0, hi = 0, i = 0;
        int xmaj = 1;
        float4 L = make_float4(0.f, 0.f, 0.f, 0.f);
        uint2 lid = make_uint2(0, 0);
        uint32_t lth = 0;
        int2 ab = make_int2(0, -1);
        uint32_t cnt = 0;
        LsLine &me = wl_sh[lane];
        __syncwarp();
        if (ok) {
            const uint32_t t = (uint32_t)find_segment_u32(line_off, n_long, u);
            off_t = line_off[t];
            li = long_idx[t];
            L = seg[li];
            lid = ids[li];
            lth = theta[li];
            const int2 m = walk_meta[t];
            lo = m.x;
            hi = lo + (int)(line_off[t + 1] - off_t) - 1;
            xmaj = m.y;
            i = lo + (int)(u - off_t);
            ab = line_range(wl, wl_cap, off_t, lo, i, L, g);
            me.cum[0] = 0;
            for (int j = ab.x; j <= ab.y; ++j) {
                const int c = xmaj ? j * g.G + i : i * g.G + j;
                const uint32_t c0 = off[c], n_c = off[c + 1] - c0;
                if (j - ab.x < LS_CELLS) {
                    me.cstart[j - ab.x] = c0;
                    me.cum[j - ab.x + 1] = cnt + n_c;
                }
                cnt += n_c;
            }
        }
        tested += cnt;
        uint32_t chunk_total;
        const uint32_t pre = warp_excl_scan(cnt, &chunk_total);
        if (ok) {
            me.L = L;
            me.lid = lid;
            me.li = li;
            me.lth = lth;
            me.off_t = off_t;
            me.pre = pre;
            me.lo = lo;
            me.hi = hi;
            me.i = i;
            me.xmaj = xmaj;
            me.j0 = ab.x;
            me.ncell = ab.y - ab.x + 1;
        }
        __syncwarp();
        for (uint32_t b0 = 0; b0 < chunk_total; b0 += 32) {
            const uint32_t q = b0 + lane;
            int o = 0;  // the lane whose line holds pair q
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t pp = __shfl_sync(0xffffffffu, pre, o + step);
                if (pp <= q) o += step;
            }
            if (q < chunk_total) {
                const LsLine &ln = wl_sh[o];
                const uint32_t li_o = ln.li, off_o = ln.off_t, lth_o = ln.lth;
                const int lo_o = ln.lo, hi_o = ln.hi, i_o = ln.i, xm_o = ln.xmaj;
                const float4 Lo = ln.L;
                const uint2 lid_o = ln.lid;
                // the cell and record of pair q within the line: from the
                // staged offsets, or past LS_CELLS cells from the offsets table
                uint32_t k = q - ln.pre;
                int j = ln.j0;
                uint32_t p;
                if (ln.ncell <= LS_CELLS || k < ln.cum[LS_CELLS]) {
                    int x = 0;
                    while (k >= ln.cum[x + 1]) ++x;
                    j += x;
                    p = ln.cstart[x] + (k - ln.cum[x]);
                } else {
                    k -= ln.cum[LS_CELLS];
                    j += LS_CELLS;
                    int c = 0;
                    for (;; ++j) {
                        c = xm_o ? j * g.G + i_o : i_o * g.G + j;
                        const uint32_t n_c = off[c + 1] - off[c];
                        if (k < n_c) break;
                        k -= n_c;
                    }
                    p = off[c] + k;
                }
                const int cx = xm_o ? i_o : j, cy = xm_o ? j : i_o;
                const FRec fs = rec[p];
                const float4 S = fs.s;
                const int kind = classify_f32_fast(Lo, Lo.z - Lo.x, Lo.w - Lo.y, lid_o, S, fs.ids);
                if (kind != PAIR_NONE) {
                    // owner: the first cell of the short's box (row-major) on
                    // the walk; this cell is on it, so only the cells before
                    // it matter
                    const CellBox sb = cell_box(S, g);
                    bool earlier = false;
                    for (int y = sb.y0; y <= cy && !earlier; ++y)
                        for (int x = sb.x0; x <= sb.x1; ++x) {
                            if (y == cy && x == cx) break;
                            const int l2 = xm_o ? x : y, m2 = xm_o ? y : x;
                            if (l2 < lo_o || l2 > hi_o) continue;
                            const int2 r2 = line_range(wl, wl_cap, off_o, lo_o, l2, Lo, g);
                            if (r2.x <= m2 && m2 <= r2.y) {
                                earlier = true;
                                break;
                            }
                        }
                    if (!earlier) {
                        tally(kind, lth_o, fs.th, ideal, pc);
                        if (sign_cnt && (kind == PAIR_PROPER || kind == PAIR_TOUCHING)) {
                            const int sg = diff_sign(lth_o, fs.th, ideal);
                            if (sg) {
                                atomicAdd(&sign_cnt[li_o], sg);
                                atomicAdd(&sign_cnt[fs.i], -sg);
                            }
                        }
                    }
                }
            }
        }
    }
    flush_counts(pc, acc, shu);
    tested = block_sum<uint64_t>(tested, shu);
    if (threadIdx.x == 0 && tested) atomic_add_u64(&acc->grid_work, tested);
}

// ------------------------------------------------------ min angle (FP32)
__global__ void k_degree_f32(const uint2 *__restrict__ ids, const DevAcc *__restrict__ acc, uint32_t *__restrict__ deg) {
    const int64_t n = acc->n_seg;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&deg[ids[s].x], 1u);
        atomicAdd(&deg[ids[s].y], 1u);
    }
}

// Incident directions by vertex: FP64 angle in [0, 2 pi) and the far vertex.
__global__ void k_fill_dirs_f32(const float4 *__restrict__ seg, const uint2 *__restrict__ ids,
                                const DevAcc *__restrict__ acc, const uint32_t *__restrict__ off,
                                uint32_t *__restrict__ fill, double *__restrict__ ang, int32_t *__restrict__ other) {
    const int64_t n = acc->n_seg;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = seg[s];
        const uint2 v = ids[s];
        const double dx = (double)r.z - (double)r.x, dy = (double)r.w - (double)r.y;
        double t = atan2(dy, dx);
        if (t < 0.0) t += 2.0 * M_PI;
        double tb = atan2(-dy, -dx);
        if (tb < 0.0) tb += 2.0 * M_PI;
        const uint32_t pa = off[v.x] + atomicAdd(&fill[v.x], 1u);
        ang[pa] = t;
        other[pa] = (int32_t)v.y;
        const uint32_t pb = off[v.y] + atomicAdd(&fill[v.y], 1u);
        ang[pb] = tb;
        other[pb] = (int32_t)v.x;
    }
}

// One thread per vertex (fixed vertex -> block mapping): the smallest
// counter-clockwise gap between consecutive directions (the wrap-around gap
// included); ties broken by the smaller starting angle, then the smaller far
// vertex, so the choice does not depend on storage order.  Saves the two far
// vertices bounding the gap (from i to j counter-clockwise) for the backward.
__global__ void __launch_bounds__(256) k_min_angle_f32(const uint32_t *__restrict__ off,
                                                       const double *__restrict__ ang,
                                                       const int32_t *__restrict__ other, int64_t V,
                                                       int2 *__restrict__ arg, double *__restrict__ part,
                                                       uint32_t *__restrict__ cnt) {
    __shared__ double shd[32];
    __shared__ uint64_t shu[32];
    double dsum = 0.0;
    uint32_t nv = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s0 = off[v];
        const int k = (int)(off[v + 1] - s0);
        int2 best = make_int2(-1, -1);
        if (k >= 2) {
            double gmin = 1e300, amin = 0.0;
            int omin = 0;
            for (int i = 0; i < k; ++i) {
                const double ai = ang[s0 + i];
                // successor: smallest (a_j - a_i) mod 2 pi over j != i; equal angles give 0
                double gs = 1e300;
                int os = 0x7fffffff;  // far vertex of the successor
                for (int j = 0; j < k; ++j) {
                    if (j == i) continue;
                    double g = ang[s0 + j] - ai;
                    if (g < 0.0) g += 2.0 * M_PI;
                    const int oj = other[s0 + j];
                    if (g < gs || (g == gs && oj < os)) { gs = g; os = oj; }
                }
                const int oi = other[s0 + i];
                if (gs < gmin || (gs == gmin && (ai < amin || (ai == amin && oi < omin)))) {
                    gmin = gs;
                    amin = ai;
                    omin = oi;
                    best = make_int2(oi, os);
                }
            }
            const double ideal = 2.0 * M_PI / (double)k;
            dsum += (ideal - gmin) / ideal;
            nv += 1;
        }
        arg[v] = best;
    }
    const double s = block_sum<double>(dsum, shd);
    const uint64_t c = block_sum<uint64_t>(nv, shu);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s;
        cnt[blockIdx.x] = (uint32_t)c;
    }
}

// ------------------------------------------------------------ state, out3
// Everything the backward needs, and the three forward values.
__global__ void k_diff_state(const DevAcc *__restrict__ acc, const double *__restrict__ elv_part,
                             const double *__restrict__ ma_part, const uint32_t *__restrict__ ma_cnt, int ma_blocks,
                             int64_t E, double ideal, DiffState *__restrict__ st, float *__restrict__ out3) {
    __shared__ double shd[32];
    __shared__ uint64_t shu[32];
    double sl = 0.0, sv = 0.0, ms = 0.0;
    uint64_t mn = 0;
    for (int i = threadIdx.x; i < kElvBlocks; i += blockDim.x) {
        sl += elv_part[i];
        sv += elv_part[kElvBlocks + i];
    }
    for (int i = threadIdx.x; i < ma_blocks; i += blockDim.x) {
        ms += ma_part[i];
        mn += ma_cnt[i];
    }
    sl = block_sum<double>(sl, shd);
    sv = block_sum<double>(sv, shd);
    ms = block_sum<double>(ms, shd);
    mn = block_sum<uint64_t>(mn, shu);
    if (threadIdx.x != 0) return;
    DiffState d;
    const uint64_t ec = acc->proper + acc->touching;
    const double dev = ((double)acc->dev_hi * 18446744073709551616.0 + (double)acc->dev_lo) * kAngleUnit;
    d.ec = (int64_t)ec;
    d.ideal = ideal;
    d.E_ca = ec > 0 ? 1.0 - dev / (ideal * (double)ec) : 1.0;
    d.mu = E > 0 ? sl / (double)E : 0.0;
    d.S = sv;
    d.M_l = (E > 1 && d.mu > 0.0) ? sqrt(sv / ((double)E * d.mu * d.mu)) / sqrt((double)E - 1.0) : 0.0;
    d.n_ma = (int64_t)mn;
    d.M_a = mn > 0 ? 1.0 - ms / (double)mn : 1.0;
    *st = d;
    out3[0] = (float)d.E_ca;
    out3[1] = (float)d.M_l;
    out3[2] = (float)d.M_a;
}

// ---------------------------------------------------------------- adjoint
__device__ __forceinline__ void atomic_add2(float *g, int64_t v, float x, float y) {
    atomicAdd(&g[2 * v], x);
    atomicAdd(&g[2 * v + 1], y);
}

// d E_ca: every E_c pair adds the same magnitude, scale = -gout / (ideal E_c),
// to the adjoints of its two directions with signs +-1 or 0 (diff_sign); the
// forward summed them into each segment's signed count (exact int32), so each
// segment turns scale times its count into its endpoints' gradients:
// d theta / d q = (-dy, dx) / |q - p|^2 for the vector q - p.
__global__ void __launch_bounds__(256) k_grad_theta_scatter(const float4 *__restrict__ seg,
                                                            const uint2 *__restrict__ ids,
                                                            const DevAcc *__restrict__ acc,
                                                            const DiffState *__restrict__ st,
                                                            const float *__restrict__ gout,
                                                            const int32_t *__restrict__ cnt, float *__restrict__ grad) {
    const DiffState d = *st;
    if (d.ec == 0) return;
    const double scale = -(double)gout[0] / (d.ideal * (double)d.ec);
    const int64_t n = acc->n_seg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = cnt[i];
        if (k == 0) continue;
        const double c = scale * (double)k;
        const float4 r = seg[i];
        const uint2 v = ids[i];
        const double ux = (double)r.z - r.x, uy = (double)r.w - r.y;
        const double ru = ux * ux + uy * uy;
        const float gx = (float)(c * -uy / ru), gy = (float)(c * ux / ru);
        atomic_add2(grad, v.y, gx, gy);
        atomic_add2(grad, v.x, -gx, -gy);
    }
}

// d M_l: dM_l / dl_e = M_l ((l_e - mu) / S - 1 / (N mu)), dl_e / dp_b = (p_b - p_a) / l_e.
__global__ void __launch_bounds__(256) k_grad_elv(const int2 *__restrict__ edges, const float2 *__restrict__ xy,
                                                  int64_t E, const DiffState *__restrict__ st,
                                                  const float *__restrict__ gout, float *__restrict__ grad) {
    const DiffState d = *st;
    if (!(d.S > 0.0 && d.mu > 0.0) || E < 2) return;
    const double g1 = gout[1];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int2 ed = edges[e];
        const float2 a = xy[ed.x], b = xy[ed.y];
        const double dx = (double)b.x - a.x, dy = (double)b.y - a.y;
        const double l = sqrt(dx * dx + dy * dy);
        if (l == 0.0) continue;
        const double dl = g1 * d.M_l * ((l - d.mu) / d.S - 1.0 / ((double)E * d.mu));
        const float gx = (float)(dl * dx / l), gy = (float)(dl * dy / l);
        atomic_add2(grad, ed.y, gx, gy);
        atomic_add2(grad, ed.x, -gx, -gy);
    }
}

// d M_a: dM_a / dmin_v = deg_v / (2 pi n); min_v = theta(p_j - p_v) - theta(p_i - p_v).
__global__ void __launch_bounds__(256) k_grad_min_angle(const int2 *__restrict__ arg, const uint32_t *__restrict__ off,
                                                        const float2 *__restrict__ xy, int64_t V,
                                                        const DiffState *__restrict__ st,
                                                        const float *__restrict__ gout, float *__restrict__ grad) {
    const DiffState d = *st;
    if (d.n_ma == 0) return;
    const double g2 = gout[2];
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int2 ij = arg[v];
        if (ij.x < 0) continue;
        const double c = g2 * (double)(off[v + 1] - off[v]) / (2.0 * M_PI * (double)d.n_ma);
        const float2 pv = xy[v], pi = xy[ij.x], pj = xy[ij.y];
        const double ix = (double)pi.x - pv.x, iy = (double)pi.y - pv.y;
        const double jx = (double)pj.x - pv.x, jy = (double)pj.y - pv.y;
        const double ri = ix * ix + iy * iy, rj = jx * jx + jy * jy;
        const float gjx = (float)(c * -jy / rj), gjy = (float)(c * jx / rj);
        const float gix = (float)(c * -iy / ri), giy = (float)(c * ix / ri);
        atomic_add2(grad, ij.y, gjx, gjy);
        atomic_add2(grad, ij.x, -gix, -giy);
        atomic_add2(grad, v, gix - gjx, giy - gjy);
    }
}

}  // namespace

// ------------------------------------------------------------- launchers
void launch_gather_f32(const float *xy, int64_t V, const int32_t *edges, int64_t E, Buffers &b, cudaStream_t s) {
    cudaMemsetAsync(&b.acc->f32_bounds[0], 0xff, 2 * sizeof(uint32_t), s);  // minima (the maxima start at 0)
    count_launches(V > 0 ? 1 : 0);
    if (V > 0) k_check_vertices_f32<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>((const float2 *)xy, V, b.acc);
    if (E <= 0) return;
    count_launches(1);
    k_gather_f32<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>((const float2 *)xy, V, (const int2 *)edges, E,
                                                            (float4 *)b.seg, b.seg_ids, b.seg_eid, b.seg_theta,
                                                            b.len2, b.acc);
}

void launch_crossings_f32(const Buffers &b, int64_t n_bound, uint32_t ideal, int32_t *cnt, cudaStream_t s) {
    if (n_bound < 2) return;
    const int64_t nb = (n_bound + DF_ROWS - 1) / DF_ROWS;
    const int64_t tiles = nb * (nb + 1) / 2;
    const unsigned grid = (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
    count_launches(1);
    k_cross_f32<<<grid, DF_ROWS, 0, s>>>((const float4 *)b.seg, b.seg_ids, b.seg_theta, nullptr, &b.acc->n_seg,
                                         b.acc, ideal, tiles, cnt);
}

// Lines of the walk table: up to 16 per edge (more are recomputed when needed).
uint64_t f32_walk_lines_cap(int64_t E) { return 16 * (uint64_t)E + 1024; }

size_t f32_grid_bytes(int G, int64_t E) {
    const size_t C = (size_t)G * G;
    return sizeof(FGrid) + sizeof(FRec) * 4 * (size_t)E + sizeof(uint32_t) * ((C + 1) + C + 4 * (size_t)E + 2 * (size_t)E + 1) +
           sizeof(int2) * ((size_t)E + f32_walk_lines_cap(E)) + 256 * 10;
}

void launch_crossings_f32_grid(const Buffers &b, int64_t E, int G, void *work, uint32_t ideal, int32_t *sign_cnt,
                               cudaStream_t s) {
    if (E < 2) return;
    const size_t C = (size_t)G * G;
    char *p = (char *)work;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) & ~(size_t)255;
        return q;
    };
    FGrid *g = (FGrid *)take(sizeof(FGrid));

    uint32_t *cnt = (uint32_t *)take(sizeof(uint32_t) * (C + 1));
    uint32_t *fill = (uint32_t *)take(sizeof(uint32_t) * C);
    FRec *rec = (FRec *)take(sizeof(FRec) * 4 * (size_t)E);
    uint32_t *rec_cell = (uint32_t *)take(sizeof(uint32_t) * 4 * (size_t)E);
    uint32_t *long_idx = (uint32_t *)take(sizeof(uint32_t) * (size_t)E);
    uint32_t *long_lines = (uint32_t *)take(sizeof(uint32_t) * ((size_t)E + 1));
    int2 *walk_meta = (int2 *)take(sizeof(int2) * (size_t)E);
    const uint64_t wl_cap = f32_walk_lines_cap(E);
    int2 *wl = (int2 *)take(sizeof(int2) * wl_cap);
    cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (C + 1), s);
    cudaMemsetAsync(fill, 0, sizeof(uint32_t) * C, s);
    const float4 *seg = (const float4 *)b.seg;
    const int gb = grid_for(E, 256, 152 * 8);
    count_launches(3);
    k_f32_grid_setup<<<1, 1, 0, s>>>(b.acc->f32_bounds, G, g);
    cudaMemsetAsync(long_lines, 0, sizeof(uint32_t) * ((size_t)E + 1), s);
    k_f32_grid_count<<<gb, 256, 0, s>>>(seg, b.acc, g, cnt, long_idx, long_lines, walk_meta);
    launch_scan_u32(long_lines, long_lines, E, b.scan_tmp, &b.acc->scan_sink, &b.acc->eval_status, s);
    count_launches(1);
    k_f32_walk_lines<<<152 * 8, 256, 0, s>>>(seg, g, long_idx, long_lines, (uint32_t)E, b.acc, wl_cap, wl);
    launch_scan_u32(cnt, cnt, (int64_t)C, b.scan_tmp, &b.acc->scan_sink, &b.acc->eval_status, s);
    k_f32_grid_fill<<<gb, 256, 0, s>>>(seg, b.acc, g, cnt, fill, b.seg_ids, b.seg_theta, rec, rec_cell);
    count_launches(3);
    k_f32_grid_ss<<<152 * 8, 256, 0, s>>>(seg, b.seg_ids, b.seg_theta, g, cnt, rec, rec_cell, b.acc, ideal,
                                          sign_cnt);
    k_f32_grid_ls<<<152 * 8, 256, 0, s>>>(seg, b.seg_ids, b.seg_theta, g, cnt, rec, long_idx, long_lines,
                                          (uint32_t)E, walk_meta, wl, wl_cap, b.acc, ideal, sign_cnt);
    k_cross_f32<<<152 * 8, DF_ROWS, 0, s>>>(seg, b.seg_ids, b.seg_theta, long_idx, &b.acc->n_long, b.acc, ideal, -1,
                                            sign_cnt);
}

void launch_min_angle_f32(Buffers &b, int64_t V, int64_t E, int2 *arg, cudaStream_t s) {
    if (V <= 0) return;
    cudaMemsetAsync(b.deg, 0, sizeof(uint32_t) * (V + 1), s);
    cudaMemsetAsync(b.deg_fill, 0, sizeof(uint32_t) * V, s);
    const int gb = grid_for(E, 256, 152 * 8);
    count_launches(E > 0 ? 2 : 0);
    if (E > 0) k_degree_f32<<<gb, 256, 0, s>>>(b.seg_ids, b.acc, b.deg);
    launch_scan_u32(b.deg, b.deg, V, b.scan_tmp_side, &b.acc->scan_sink, &b.acc->eval_status, s);
    if (E > 0) k_fill_dirs_f32<<<gb, 256, 0, s>>>((const float4 *)b.seg, b.seg_ids, b.acc, b.deg, b.deg_fill,
                                                  b.dir_ang, b.dir_other);
    count_launches(1);
    k_min_angle_f32<<<min_angle_blocks(V), 256, 0, s>>>(b.deg, b.dir_ang, b.dir_other, V, arg, b.ma_part, b.ma_cnt);
}

void launch_diff_state(const Buffers &b, int64_t V, int64_t E, double ideal, DiffState *st, float *out3,
                       cudaStream_t s) {
    count_launches(1);
    k_diff_state<<<1, 256, 0, s>>>(b.acc, b.elv_part, b.ma_part, b.ma_cnt, V > 0 ? min_angle_blocks(V) : 0, E, ideal,
                                   st, out3);
}

void launch_diff_backward(const Buffers &b, int64_t V, int64_t E, const int2 *arg, const DiffState *st,
                          const float *gout, const int32_t *cnt, float *grad, cudaStream_t s) {
    cudaMemsetAsync(grad, 0, sizeof(float) * 2 * V, s);
    count_launches(3);
    k_grad_theta_scatter<<<grid_for(E, 256, 152 * 8), 256, 0, s>>>((const float4 *)b.seg, b.seg_ids, b.acc, st, gout,
                                                                    cnt, grad);
    k_grad_elv<<<grid_for(E, 256, 152 * 8), 256, 0, s>>>((const int2 *)b.edges, (const float2 *)b.xy, E, st, gout,
                                                         grad);
    k_grad_min_angle<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>(arg, b.deg, (const float2 *)b.xy, V, st, gout, grad);
}

}  // namespace gr
