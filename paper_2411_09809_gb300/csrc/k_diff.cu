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
#include <math.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
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
        }
    }
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

// All-pairs tiles over the compacted FP32 segments; E_c pairs (compacted
// indices) appended to `pairs` (warp-aggregated), at most `cap` of them; the
// total goes to acc->records.
__global__ void __launch_bounds__(DF_ROWS) k_cross_f32(const float4 *__restrict__ seg, const uint2 *__restrict__ ids,
                                                       const uint32_t *__restrict__ theta, DevAcc *acc, uint32_t ideal,
                                                       int64_t tiles, uint2 *__restrict__ pairs, uint64_t cap) {
    __shared__ float4 cs[DF_COLS];
    __shared__ uint2 cid[DF_COLS];
    __shared__ uint32_t cth[DF_COLS];
    __shared__ uint64_t shu[32];
    const int lane = threadIdx.x & 31;
    const int n_seg = (int)acc->n_seg;
    PairCounts pc;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int bi, bj;
        decode_tile(t, bi, bj);
        const int j0 = bj * DF_COLS;
        if (j0 >= n_seg) continue;
        const int nc = min(DF_COLS, n_seg - j0);
        __syncthreads();
        if (threadIdx.x < nc) {
            cs[threadIdx.x] = seg[j0 + threadIdx.x];
            cid[threadIdx.x] = ids[j0 + threadIdx.x];
            cth[threadIdx.x] = theta[j0 + threadIdx.x];
        }
        const int i = bi * DF_ROWS + threadIdx.x;
        const bool row_ok = i < n_seg;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        uint2 ri = make_uint2(0xffffffffu, 0xfffffffeu);
        uint32_t rth = 0;
        if (row_ok) {
            r = seg[i];
            ri = ids[i];
            rth = theta[i];
        }
        __syncthreads();
        const bool diag = bi == bj;
        for (int jj = 0; jj < nc; ++jj) {
            const bool valid = row_ok && (!diag || jj > (int)threadIdx.x);
            const int kind = valid ? classify_f32(r, ri, cs[jj], cid[jj]) : PAIR_NONE;
            const bool ec = kind == PAIR_PROPER || kind == PAIR_TOUCHING;
            if (kind == PAIR_PROPER) ++pc.proper;
            else if (kind == PAIR_TOUCHING) ++pc.touching;
            else if (kind == PAIR_COLLINEAR) ++pc.collinear;
            if (ec) pc.dev += dev_term(rth, cth[jj], ideal);
            const unsigned m = __ballot_sync(0xffffffffu, ec);
            if (m) {
                unsigned long long slot = 0;
                if (lane == 0) slot = atomicAdd((unsigned long long *)&acc->records, (unsigned long long)__popc(m));
                slot = __shfl_sync(0xffffffffu, slot, 0);
                if (ec) {
                    const uint64_t pos = slot + __popc(m & lanemask_lt());
                    if (pos < cap) pairs[pos] = make_uint2((uint32_t)i, (uint32_t)(j0 + jj));
                }
            }
        }
    }
    flush_counts(pc, acc, shu);
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
    d.pairs = acc->records;
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

// d E_ca: a_c is the acute angle between the lines of directions theta_u,
// theta_v; the fold (d = theta_u - theta_v mod pi, a_c = d or pi - d) and the
// sign of a_c - ideal are read from the same integer directions the forward
// used.  d theta / d q = (-dy, dx) / |q - p|^2 for the vector q - p.
__global__ void __launch_bounds__(256) k_grad_cross(const uint2 *__restrict__ pairs, const float4 *__restrict__ seg,
                                                    const uint2 *__restrict__ ids, const uint32_t *__restrict__ theta,
                                                    const DiffState *__restrict__ st, const float *__restrict__ gout,
                                                    uint32_t ideal_u, float *__restrict__ grad) {
    const DiffState d = *st;
    const uint64_t n = min((uint64_t)d.pairs, (uint64_t)d.ec);
    if (d.ec == 0) return;
    const double scale = -(double)gout[0] / (d.ideal * (double)d.ec);
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 pr = pairs[p];
        const float4 r = seg[pr.x], c = seg[pr.y];
        const uint2 ri = ids[pr.x], ci = ids[pr.y];
        const uint32_t dd = theta[pr.x] - theta[pr.y];
        const bool folded = dd > 0x80000000u;           // a_c = pi - d
        const uint32_t a = folded ? 0u - dd : dd;
        const double sgn = a > ideal_u ? 1.0 : (a < ideal_u ? -1.0 : 0.0);
        const double coef = scale * sgn * (folded ? -1.0 : 1.0);  // d E_ca / d theta_u
        const double ux = (double)r.z - r.x, uy = (double)r.w - r.y, vx = (double)c.z - c.x, vy = (double)c.w - c.y;
        const double ru = ux * ux + uy * uy, rv = vx * vx + vy * vy;
        const float gux = (float)(coef * -uy / ru), guy = (float)(coef * ux / ru);
        const float gvx = (float)(coef * -vy / rv), gvy = (float)(coef * vx / rv);
        atomic_add2(grad, ri.y, gux, guy);
        atomic_add2(grad, ri.x, -gux, -guy);
        atomic_add2(grad, ci.y, -gvx, -gvy);
        atomic_add2(grad, ci.x, gvx, gvy);
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
    count_launches(V > 0 ? 1 : 0);
    if (V > 0) k_check_vertices_f32<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>((const float2 *)xy, V, b.acc);
    if (E <= 0) return;
    count_launches(1);
    k_gather_f32<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>((const float2 *)xy, V, (const int2 *)edges, E,
                                                            (float4 *)b.seg, b.seg_ids, b.seg_eid, b.seg_theta,
                                                            b.len2, b.acc);
}

void launch_crossings_f32(const Buffers &b, int64_t n_bound, uint32_t ideal, uint2 *pairs, uint64_t cap,
                          cudaStream_t s) {
    if (n_bound < 2) return;
    const int64_t nb = (n_bound + DF_ROWS - 1) / DF_ROWS;
    const int64_t tiles = nb * (nb + 1) / 2;
    const unsigned grid = (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
    count_launches(1);
    k_cross_f32<<<grid, DF_ROWS, 0, s>>>((const float4 *)b.seg, b.seg_ids, b.seg_theta, b.acc, ideal, tiles, pairs,
                                         cap);
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

void launch_diff_backward(const Buffers &b, int64_t V, int64_t E, const uint2 *pairs, const int2 *arg,
                          const DiffState *st, const float *gout, uint32_t ideal_u, uint64_t n_pairs, float *grad,
                          cudaStream_t s) {
    cudaMemsetAsync(grad, 0, sizeof(float) * 2 * V, s);
    count_launches(3);
    k_grad_cross<<<grid_for((int64_t)n_pairs, 256, 152 * 16), 256, 0, s>>>(pairs, (const float4 *)b.seg, b.seg_ids,
                                                                          b.seg_theta, st, gout, ideal_u, grad);
    k_grad_elv<<<grid_for(E, 256, 152 * 8), 256, 0, s>>>((const int2 *)b.edges, (const float2 *)b.xy, E, st, gout,
                                                         grad);
    k_grad_min_angle<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>(arg, b.deg, (const float2 *)b.xy, V, st, gout, grad);
}

}  // namespace gr
