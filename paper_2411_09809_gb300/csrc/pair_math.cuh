// pair_math.cuh -- classification of one edge pair and its crossing-angle
// term, shared by the all-pairs and per-cell crossing kernels.
//
// Algorithm 4 decides a crossing from four orientation signs.  With
// integer coordinates in [0, 2^16) every orientation is an exact int64:
//   orient(p, q, r) = (q - p) x (r - p) = u x r - u x p,   u = q - p,
// so for a fixed segment (p, q) it is the linear form u x r - k with
// k = u x p precomputed once per segment; each orientation then costs two
// 32x32->64 multiply-adds.  Magnitudes stay below 2^35.
//
// Algorithm 5's crossing angle a_c is the acute angle between the two lines.
// Each segment carries the direction of its line, theta in [0, pi), as a
// uint32 in units of pi / 2^32; then a_c = min(d, 2^32 - d) with
// d = theta_e - theta_f (mod 2^32), and |ideal - a_c| is integer arithmetic.
#pragma once

#include "gr_internal.cuh"

namespace gr {

enum { PAIR_NONE = 0, PAIR_PROPER = 1, PAIR_TOUCHING = 2, PAIR_COLLINEAR = 3 };

// Segment held in registers by the thread that owns it.
struct RowSeg {
    int ax, ay, bx, by;
    int ux, uy;
    long long k;  // u x a
    uint32_t ida, idb;
    uint32_t th;  // line direction
};

// Segment staged in shared memory and read by every thread of a tile.
struct __align__(8) ColSeg {
    int cx, cy, dx, dy;
    int vx, vy;
    uint32_t idc, idd;
    long long k;  // v x c
    uint32_t th;
};

__device__ __forceinline__ RowSeg make_row(SegRec s, uint32_t th) {
    RowSeg r;
    r.ax = px(s.x); r.ay = py(s.x); r.bx = px(s.y); r.by = py(s.y);
    r.ux = r.bx - r.ax; r.uy = r.by - r.ay;
    r.k = (long long)r.ux * r.ay - (long long)r.uy * r.ax;
    r.ida = s.z; r.idb = s.w;
    r.th = th;
    return r;
}

__device__ __forceinline__ ColSeg make_col(SegRec s, uint32_t th) {
    ColSeg c;
    c.cx = px(s.x); c.cy = py(s.x); c.dx = px(s.y); c.dy = py(s.y);
    c.vx = c.dx - c.cx; c.vy = c.dy - c.cy;
    c.k = (long long)c.vx * c.cy - (long long)c.vy * c.cx;
    c.idc = s.z; c.idd = s.w;
    c.th = th;
    return c;
}

// Lexicographic (x, then y) key of a point; for points on one line this is a
// linear order along the line.
__device__ __forceinline__ uint32_t lex_key(int x, int y) { return (uint32_t(x) << 16) | uint32_t(y); }

// Classifies the unordered pair {r, c} under the library's reading of
// Algorithm 4: shared vertex ids never cross; a collinear pair whose extents
// meet is reported separately; otherwise the pair is in E_c when both
// orientation products are <= 0 (PAIR_PROPER when both are < 0, else
// PAIR_TOUCHING).  Exact.
__device__ __forceinline__ int classify_kind(const RowSeg &r, const ColSeg &c) {
    if ((r.ida == c.idc) | (r.ida == c.idd) | (r.idb == c.idc) | (r.idb == c.idd)) return PAIR_NONE;
    const long long o1 = (long long)r.ux * c.cy - (long long)r.uy * c.cx - r.k;  // orient(a, b, c)
    const long long o2 = (long long)r.ux * c.dy - (long long)r.uy * c.dx - r.k;  // orient(a, b, d)
    if ((o1 > 0 && o2 > 0) || (o1 < 0 && o2 < 0)) return PAIR_NONE;
    const long long o3 = (long long)c.vx * r.ay - (long long)c.vy * r.ax - c.k;  // orient(c, d, a)
    const long long o4 = (long long)c.vx * r.by - (long long)c.vy * r.bx - c.k;  // orient(c, d, b)
    if ((o3 > 0 && o4 > 0) || (o3 < 0 && o4 < 0)) return PAIR_NONE;
    if (o1 == 0 && o2 == 0) {
        // collinear (for non-zero-length segments o1 = o2 = 0 implies o3 = o4 = 0)
        const uint32_t ka = lex_key(r.ax, r.ay), kb = lex_key(r.bx, r.by);
        const uint32_t kc = lex_key(c.cx, c.cy), kd = lex_key(c.dx, c.dy);
        const uint32_t lo = max(min(ka, kb), min(kc, kd));
        const uint32_t hi = min(max(ka, kb), max(kc, kd));
        return lo <= hi ? PAIR_COLLINEAR : PAIR_NONE;
    }
    return (o1 != 0 && o2 != 0 && o3 != 0 && o4 != 0) ? PAIR_PROPER : PAIR_TOUCHING;
}

// Direction of the line through a segment with vector (dx, dy), as an angle
// in [0, pi) in units of pi / 2^32.  The vector is first turned into the
// upper half-plane (exact: the line is the same), then FP32 atan2 of the
// exactly representable integers (a few units in the last place of an angle
// below pi, i.e. below 1e-6 rad) is rounded to the nearest unit.  With t =
// m 2^(be - 150) (m the 24-bit significand, be the biased exponent),
// t 2^32 / pi = m K 2^(be - 180) for K = round(2^62 / pi); the product
// (< 2^85) is formed and rounded in 128-bit integer arithmetic, so no FP64
// instruction is needed.  Each segment's direction is computed once and
// shared by every path, so all paths derive the same crossing-angle terms.
__device__ __forceinline__ uint32_t line_direction(int dx, int dy) {
    if (dy < 0 || (dy == 0 && dx < 0)) {
        dx = -dx;
        dy = -dy;
    }
    const float t = atan2f(i2f_exact(dy), i2f_exact(dx));  // [0, pi)
    const uint32_t bits = __float_as_uint(t);
    const int be = (int)(bits >> 23);  // biased exponent; t >= 0
    if (be < 90) return 0u;            // t < 2^-37: below half a unit (and t = 0)
    const uint64_t m = (bits & 0x7fffffu) | 0x800000u;
    constexpr uint64_t K = 1467945251641000613ull;  // round(2^62 / pi)
    const int sh = 180 - be;                        // t 2^32 / pi = m K 2^(be - 180); 52 ... 90
    unsigned __int128 P = (unsigned __int128)m * K;
    P += (unsigned __int128)1 << (sh - 1);
    return (uint32_t)(uint64_t)(P >> sh);  // t <= pi - 1.5e-5 here: below 2^32
}

// |ideal - a_c| in units of pi / 2^32 for lines of directions ta and tb.
// Symmetric in (ta, tb), so every path that meets a pair derives the same
// term.  At most 2^31.
__device__ __forceinline__ uint32_t dev_term(uint32_t ta, uint32_t tb, uint32_t ideal) {
    const uint32_t d = ta - tb;
    const uint32_t a = min(d, 0u - d);  // acute angle between the lines
    return max(a, ideal) - min(a, ideal);
}

// Per-thread tallies of one crossing kernel.
struct PairCounts {
    uint32_t proper = 0, touching = 0, collinear = 0;
    uint64_t dev = 0;  // sum of |ideal - a_c|, units of pi / 2^32
};

// Block-wide reduction of the tallies and one atomic per counter.  Every
// thread of the block must call it.
__device__ __forceinline__ void flush_counts(const PairCounts &pc, DevAcc *acc, uint64_t *sh) {
    const uint64_t p = block_sum<uint64_t>(pc.proper, sh);
    const uint64_t t = block_sum<uint64_t>(pc.touching, sh);
    const uint64_t c = block_sum<uint64_t>(pc.collinear, sh);
    const uint64_t d = block_sum<uint64_t>(pc.dev, sh);
    if (threadIdx.x == 0) {
        atomic_add_u64(&acc->proper, p);
        atomic_add_u64(&acc->touching, t);
        atomic_add_u64(&acc->collinear, c);
        add_u128(&acc->dev_lo, &acc->dev_hi, d);
    }
}

}  // namespace gr
