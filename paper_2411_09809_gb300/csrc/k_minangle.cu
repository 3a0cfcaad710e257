// k_minangle.cu -- minimum angle M_a (a9, Algorithm 2).
//
// The aggregateMessages step of Algorithm 2 (collect, per vertex, the angles
// of its incident edges) becomes a CSR: for a single layout, the adjacency of
// the edge list (degree count, exclusive scan, scatter of the other
// endpoints) is built once per edge list, and every evaluation writes each
// vertex's non-zero incident direction vectors into its slot range; the
// batched evaluator builds the CSR of direction vectors directly.
// GetMinAngle (sort the angles, take the smallest gap between neighbours,
// wrap-around included) becomes an exact successor search: for every
// incident direction d_i, the next direction counter-clockwise is found with
// exact integer comparisons (half plane relative to d_i, then the sign of a
// cross product), and the gap to it is the ccw angle between the two
// vectors.  The set of gaps is the set of neighbour gaps of the sorted order,
// so its minimum is GetMinAngle's result.  A vertex's d_v does not depend on
// the order its directions are stored in, and each block's partial sum covers
// a fixed set of vertices, so after a few vertices move only the blocks
// holding them or their neighbours are recomputed, with the same result as a
// full pass.
#include <math.h>

#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int MA_THREADS = 256;  // vertices in flight per block
constexpr int MA_HEAVY = 32;     // degree above which a warp shares one vertex
constexpr int MA_MAX_BLOCKS = 1024;

__global__ void k_degree(const SegRec *__restrict__ seg, const DevAcc *__restrict__ acc,
                         uint32_t *__restrict__ deg) {
    const int64_t n = acc->n_seg;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const SegRec r = seg[s];
        atomicAdd(&deg[r.z], 1u);
        atomicAdd(&deg[r.w], 1u);
    }
}

__global__ void k_fill_dirs(const SegRec *__restrict__ seg, const DevAcc *__restrict__ acc,
                            const uint32_t *__restrict__ off, uint32_t *__restrict__ fill,
                            int2 *__restrict__ dirs) {
    const int64_t n = acc->n_seg;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const SegRec r = seg[s];
        const int dx = px(r.y) - px(r.x), dy = py(r.y) - py(r.x);
        const uint32_t ia = atomicAdd(&fill[r.z], 1u);
        dirs[off[r.z] + ia] = make_int2(dx, dy);
        const uint32_t ib = atomicAdd(&fill[r.w], 1u);
        dirs[off[r.w] + ib] = make_int2(-dx, -dy);
    }
}

__device__ __forceinline__ long long cross2(int2 a, int2 b) {
    return (long long)a.x * b.y - (long long)a.y * b.x;
}
__device__ __forceinline__ long long dot2(int2 a, int2 b) {
    return (long long)a.x * b.x + (long long)a.y * b.y;
}

// Exact successor of direction di among dirs[0..k) (index i excluded): the
// direction reached first when turning counter-clockwise from di, a
// direction equal to di being reached at angle 0.
__device__ __forceinline__ int2 ccw_successor(const int2 *__restrict__ d, int k, int i, int2 di) {
    int2 db = make_int2(0, 0);
    int hb = 2;
    for (int j = 0; j < k; ++j) {
        if (j == i) continue;
        const int2 dj = d[j];
        const long long cr = cross2(di, dj), dt = dot2(di, dj);
        const int hj = (cr > 0 || (cr == 0 && dt > 0)) ? 0 : 1;  // half plane relative to di
        if (hj < hb || (hj == hb && cross2(dj, db) > 0)) {
            db = dj;
            hb = hj;
        }
    }
    return db;
}

// Exact order of directions by their angle from the positive x axis, in
// [0, 2 pi): half plane first, then the sign of the cross product.
__device__ __forceinline__ bool angle_before(int2 a, int2 b) {
    const int ha = (a.y < 0 || (a.y == 0 && a.x < 0)) ? 1 : 0;
    const int hb = (b.y < 0 || (b.y == 0 && b.x < 0)) ? 1 : 0;
    if (ha != hb) return ha < hb;
    return cross2(a, b) > 0;
}

// Candidate (gap g from direction di to bs) replaces the current one when its
// FP32 gap is smaller, or equal with di earlier in exact angular order: the
// choice does not depend on the order the directions are stored in.
__device__ __forceinline__ bool better_gap(float g, int2 di, float gmin, int2 bi) {
    return g < gmin || (g == gmin && angle_before(di, bi));
}

__device__ __forceinline__ float ccw_gap_f(int2 a, int2 b) {
    float g = atan2f(ll2f_rn(cross2(a, b)), ll2f_rn(dot2(a, b)));  // |cross|, |dot| < 2^33
    return g < 0.f ? g + 6.28318530717958647692f : g;
}

// FP64 counter-clockwise angle from a to b, in [0, 2 pi), by table-driven
// argument reduction (Tang's method): (X, Y) = (a . b, a x b) are exact; the
// FP32 atan2 picks the sector j of width w = 2 pi / kSectors nearest to the
// angle; (X, Y) is rotated back by j w with cosine and sine from an FP64
// table (built on the host); the residual angle atan(t), t = Y' / X' with
// |t| <= tan(w / 2 + 1e-6) < 0.0123, is the odd Taylor series through t^9
// (the next term is below 2^-60 of t).  Fewer FP64 instructions than a
// general atan2 and as accurate: the rotation and the series each add a few
// units in the last place.
constexpr int kSectors = 256;
constexpr double kTwoPi = 2.0 * 3.14159265358979323846;
constexpr double kSectorW = kTwoPi / kSectors;
__device__ double2 g_sector[kSectors];  // (cos, sin)(j kSectorW)

__device__ __forceinline__ double ccw_gap_d(int2 a, int2 b) {
    const long long cr = cross2(a, b), dt = dot2(a, b);
    const float g = atan2f(ll2f_rn(cr), ll2f_rn(dt));  // (-pi, pi], |cross|, |dot| < 2^33
    const int j = __float2int_rn(g * (float)(kSectors / kTwoPi)) & (kSectors - 1);
    const double2 cs = __ldg(&g_sector[j]);
    const double X = (double)dt, Y = (double)cr;
    const double x = fma(X, cs.x, Y * cs.y);     // rotation by -j w
    const double y = fma(Y, cs.x, -(X * cs.y));
    // y / x with 1 / x from the FP32 reciprocal and two Newton steps (relative
    // error 2^-24 -> 2^-48 -> a unit in the last place): fewer FP64
    // instructions than a division; x >= 0.99 |(X, Y)| >= 0.99 here
    double r = (double)__frcp_rn((float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    const double t = y * r, t2 = t * t;
    const double p = fma(fma(fma(fma(t2, 1.0 / 9.0, -1.0 / 7.0), t2, 1.0 / 5.0), t2, -1.0 / 3.0), t2, 1.0);
    double th = fma(t, p, (double)j * kSectorW);
    if (th < 0.0) th += kTwoPi;
    if (th >= kTwoPi) th -= kTwoPi;
    return th;
}

// d_v = (2 pi / k - gap) / (2 pi / k) for the smallest of the k gaps, which
// is at most 2 pi / k: a rounding below zero (a gap of exactly 2 pi / k, one
// unit in the last place off) is clamped, so d_v >= 0 always and -1 stays
// the only "not counted" mark.
__device__ __forceinline__ double dv_of_gap(double gap, int k) {
    // (ideal - gap) / ideal = 1 - gap k / (2 pi), without FP64 divisions
    // (within a few units in the last place of the quotient form)
    constexpr double kInvTwoPi = 1.0 / kTwoPi;
    return fmax(0.0, 1.0 - gap * ((double)k * kInvTwoPi));
}

// d_v of a vertex from its k incident directions d[0, k) by one thread:
// (2 pi / k - min) / (2 pi / k), or -1 when k < 2 (not counted; deg = 1 has a
// single 2 pi gap).  Gaps are compared in FP32 and the smallest is recomputed
// in FP64; the choice does not depend on the storage order.
__device__ __forceinline__ double vertex_dv(const int2 *__restrict__ d, int k) {
    if (k < 2) return -1.0;
    float gmin = 1e30f;
    int2 bi = make_int2(1, 0), bs = make_int2(1, 0);
    for (int i = 0; i < k; ++i) {
        const int2 di = d[i];
        const int2 db = ccw_successor(d, k, i, di);
        const float g = ccw_gap_f(di, db);
        if (better_gap(g, di, gmin, bi)) { gmin = g; bi = di; bs = db; }
    }
    return dv_of_gap(ccw_gap_d(bi, bs), k);
}

// The vertices [v0, v1) taken by this block: one thread per vertex, and
// vertices of degree > 32 by the whole warp after the per-thread pass.
// Accumulates d_v and the count of vertices with deg >= 2 into (dsum, nv) of
// the thread that owns the vertex (also for the warp-shared ones), so each
// thread adds its own vertices' d_v in round order; with `dv`, d_v (or -1)
// is stored per vertex as well.  `step` is the stride between this block's
// rounds of MA_THREADS vertices.
__device__ __forceinline__ void min_angle_range(const uint32_t *__restrict__ off, const uint32_t *__restrict__ nz,
                                                const int2 *__restrict__ dirs, int64_t v0, int64_t v1, int64_t step,
                                                double *__restrict__ dv, double &dsum, uint32_t &nv) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = v0; base < v1; base += step) {
        const int64_t v = base + threadIdx.x;
        int k = 0;
        uint32_t start = 0;
        if (v < v1) {
            start = off[v];
            k = (int)(nz ? nz[v] : off[v + 1] - start);
        }
        const bool heavy = k > MA_HEAVY;
        if (v < v1 && !heavy) {
            const double x = vertex_dv(dirs + start, k);
            if (dv) dv[v] = x;
            if (x >= 0.0) {
                dsum += x;
                nv += 1;
            }
        }
        // heavy vertices: the whole warp splits the directions of one vertex
        unsigned hm = __ballot_sync(0xffffffffu, heavy);
        while (hm) {
            const int src = __ffs(hm) - 1;
            hm &= hm - 1;
            const uint32_t hs = __shfl_sync(0xffffffffu, start, src);
            const int hk = __shfl_sync(0xffffffffu, k, src);
            const int2 *d = dirs + hs;
            float gmin = 1e30f;
            int2 bi = make_int2(1, 0), bs = make_int2(1, 0);
            for (int i = lane; i < hk; i += 32) {
                const int2 di = d[i];
                const int2 db = ccw_successor(d, hk, i, di);
                const float g = ccw_gap_f(di, db);
                if (better_gap(g, di, gmin, bi)) { gmin = g; bi = di; bs = db; }
            }
            // warp argmin under the same order (lanes without a candidate hold 1e30)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float og = __shfl_xor_sync(0xffffffffu, gmin, o);
                const int2 obi = make_int2(__shfl_xor_sync(0xffffffffu, bi.x, o), __shfl_xor_sync(0xffffffffu, bi.y, o));
                const int2 obs = make_int2(__shfl_xor_sync(0xffffffffu, bs.x, o), __shfl_xor_sync(0xffffffffu, bs.y, o));
                if (better_gap(og, obi, gmin, bi)) { gmin = og; bi = obi; bs = obs; }
            }
            if (lane == src) {
                const double x = dv_of_gap(ccw_gap_d(bi, bs), hk);
                if (dv) dv[v] = x;
                dsum += x;
                nv += 1;
            }
        }
    }
}

// Single layout: fixed vertex -> block mapping (vertex v in block
// (v / MA_THREADS) mod gridDim.x), so the per-block FP64 partial sums are
// deterministic.  Stores every vertex's d_v (-1: not counted) in dv.
__global__ void __launch_bounds__(MA_THREADS) k_min_angle(const uint32_t *__restrict__ off,
                                                          const uint32_t *__restrict__ nz,
                                                          const int2 *__restrict__ dirs, int64_t V,
                                                          double *__restrict__ dv, double *__restrict__ part,
                                                          uint32_t *__restrict__ cnt) {
    __shared__ double shd[32];
    __shared__ uint64_t shu[32];
    double dsum = 0.0;
    uint32_t nv = 0;
    min_angle_range(off, nz, dirs, (int64_t)blockIdx.x * MA_THREADS, V, (int64_t)gridDim.x * MA_THREADS, dv, dsum,
                    nv);
    const double s = block_sum<double>(dsum, shd);
    const uint64_t c = block_sum<uint64_t>(nv, shu);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s;
        cnt[blockIdx.x] = (uint32_t)c;
    }
}

// The partial sums of the flagged blocks again from the stored d_v, in the
// order k_min_angle adds them (each thread its own vertices by round, then
// the same block reduction), so they equal a full pass bit for bit; clears
// the flags.
__global__ void __launch_bounds__(MA_THREADS) k_min_angle_resum(const double *__restrict__ dv, int64_t V,
                                                                double *__restrict__ part,
                                                                uint32_t *__restrict__ cnt, uint32_t *flag) {
    __shared__ double shd[32];
    __shared__ uint64_t shu[32];
    if (!flag[blockIdx.x]) return;
    double dsum = 0.0;
    uint32_t nv = 0;
    for (int64_t v = (int64_t)blockIdx.x * MA_THREADS + threadIdx.x; v < V; v += (int64_t)gridDim.x * MA_THREADS) {
        const double x = dv[v];
        if (x >= 0.0) {
            dsum += x;
            nv += 1;
        }
    }
    const double s = block_sum<double>(dsum, shd);
    const uint64_t c = block_sum<uint64_t>(nv, shu);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s;
        cnt[blockIdx.x] = (uint32_t)c;
        flag[blockIdx.x] = 0u;
    }
}

__device__ __forceinline__ bool valid_edge(int2 ed, int64_t V) {
    return ed.x >= 0 && ed.y >= 0 && ed.x < V && ed.y < V && ed.x != ed.y;
}

// Adjacency of the edge list: degrees, then (after the scan) the other
// endpoint of every incident edge.  Invalid edges are left out (the gather
// reports them).
__global__ void k_adj_degree(const int2 *__restrict__ edges, int64_t E, int64_t V, uint32_t *__restrict__ deg) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int2 ed = edges[e];
        if (!valid_edge(ed, V)) continue;
        atomicAdd(&deg[ed.x], 1u);
        atomicAdd(&deg[ed.y], 1u);
    }
}

__global__ void k_adj_fill(const int2 *__restrict__ edges, int64_t E, int64_t V, const uint32_t *__restrict__ off,
                           uint32_t *__restrict__ fill, int32_t *__restrict__ adj) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int2 ed = edges[e];
        if (!valid_edge(ed, V)) continue;
        adj[off[ed.x] + atomicAdd(&fill[ed.x], 1u)] = ed.y;
        adj[off[ed.y] + atomicAdd(&fill[ed.y], 1u)] = ed.x;
    }
}

// The non-zero direction vectors from v to its neighbours, written to the
// start of v's slot range by one thread; returns how many.
__device__ __forceinline__ uint32_t vertex_dirs(const int2 *__restrict__ xy, int64_t v, uint32_t o0, uint32_t o1,
                                                const int32_t *__restrict__ adj, int2 *__restrict__ dirs) {
    const int2 p = xy[v];
    uint32_t j = o0;
    for (uint32_t q = o0; q < o1; ++q) {
        const int2 u = xy[adj[q]];
        const int dx = u.x - p.x, dy = u.y - p.y;
        if (dx | dy) dirs[j++] = make_int2(dx, dy);
    }
    return j - o0;
}

// Every vertex's non-zero directions (nz[v] of them) at the start of its
// slot range: one thread per vertex, a warp per vertex of degree > MA_HEAVY
// (ballot compaction).
__global__ void __launch_bounds__(256) k_ma_dirs(const int2 *__restrict__ xy, int64_t V,
                                                 const uint32_t *__restrict__ off, const int32_t *__restrict__ adj,
                                                 uint32_t *__restrict__ nz, int2 *__restrict__ dirs) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + threadIdx.x;
        uint32_t o0 = 0, o1 = 0;
        if (v < V) {
            o0 = off[v];
            o1 = off[v + 1];
        }
        const bool heavy = o1 - o0 > (uint32_t)MA_HEAVY;
        if (v < V && !heavy) nz[v] = vertex_dirs(xy, v, o0, o1, adj, dirs);
        unsigned hm = __ballot_sync(0xffffffffu, heavy);
        while (hm) {
            const int src = __ffs(hm) - 1;
            hm &= hm - 1;
            const int64_t hv = __shfl_sync(0xffffffffu, v, src);
            const uint32_t h0 = __shfl_sync(0xffffffffu, o0, src), h1 = __shfl_sync(0xffffffffu, o1, src);
            const int2 p = xy[hv];
            uint32_t j = h0;
            for (uint32_t q0 = h0; q0 < h1; q0 += 32) {
                const uint32_t q = q0 + lane;
                int2 dd = make_int2(0, 0);
                if (q < h1) {
                    const int2 u = xy[adj[q]];
                    dd = make_int2(u.x - p.x, u.y - p.y);
                }
                const bool keep = q < h1 && (dd.x | dd.y);
                const unsigned km = __ballot_sync(0xffffffffu, keep);
                unsigned lt;
                asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
                if (keep) dirs[j + __popc(km & lt)] = dd;
                j += __popc(km);
            }
            if (lane == 0) nz[hv] = j - h0;
        }
    }
}

// After a move: a warp per moved vertex v rewrites the directions and d_v
// of v and of each neighbour (once each: `touch` flags; one thread per
// vertex) and flags the min-angle blocks holding them (nb blocks).
__global__ void k_ma_touch(const int2 *__restrict__ xy, int64_t V, const int32_t *__restrict__ ids,
                           const int64_t *__restrict__ np, const uint32_t *__restrict__ off,
                           const int32_t *__restrict__ adj, uint32_t *__restrict__ touch, uint32_t *__restrict__ nz,
                           int2 *__restrict__ dirs, double *__restrict__ dv, uint32_t *__restrict__ flag, int nb) {
    const int lane = threadIdx.x & 31;
    const int64_t n = *np;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int32_t v = ids[i];
        if (v < 0 || v >= V) continue;  // an invalid move (reported by its validation)
        const uint32_t o0 = off[v], o1 = off[v + 1];
        for (int64_t q = (int64_t)o0 - 1 + lane; q < (int64_t)o1; q += 32) {
            const int32_t u = q < (int64_t)o0 ? v : adj[q];  // slot o0 - 1 stands for v itself
            if (atomicExch(&touch[u], 1u) != 0u) continue;
            const uint32_t k = vertex_dirs(xy, u, off[u], off[u + 1], adj, dirs);
            nz[u] = k;
            dv[u] = vertex_dv(dirs + off[u], (int)k);
            flag[(u / MA_THREADS) % nb] = 1u;
        }
    }
}

__global__ void k_ma_untouch(int64_t V, const int32_t *__restrict__ ids, const int64_t *__restrict__ np,
                             const uint32_t *__restrict__ off, const int32_t *__restrict__ adj,
                             uint32_t *__restrict__ touch) {
    const int lane = threadIdx.x & 31;
    const int64_t n = *np;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int32_t v = ids[i];
        if (v < 0 || v >= V) continue;
        const uint32_t o0 = off[v], o1 = off[v + 1];
        for (int64_t q = (int64_t)o0 - 1 + lane; q < (int64_t)o1; q += 32) touch[q < (int64_t)o0 ? v : adj[q]] = 0u;
    }
}

// Batch: one block per layout (grid-strided), M_a written per layout.
__global__ void __launch_bounds__(MA_THREADS) k_batch_min_angle(const uint32_t *__restrict__ off,
                                                                const int2 *__restrict__ dirs,
                                                                const int64_t *__restrict__ v_off, int64_t L,
                                                                gr_result *__restrict__ res) {
    __shared__ double shd[32];
    __shared__ uint64_t shu[32];
    for (int64_t l = blockIdx.x; l < L; l += gridDim.x) {
        double dsum = 0.0;
        uint32_t nv = 0;
        min_angle_range(off, nullptr, dirs, v_off[l], v_off[l + 1], MA_THREADS, nullptr, dsum, nv);
        const double s = block_sum<double>(dsum, shd);
        const uint64_t c = block_sum<uint64_t>(nv, shu);
        if (threadIdx.x == 0) {
            res[l].min_angle.sum_d = s;
            res[l].min_angle.n_vertices_counted = (int64_t)c;
            res[l].min_angle.M_a = c > 0 ? 1.0 - s / (double)c : 1.0;
        }
    }
}

int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

cudaError_t init_min_angle_table(cudaStream_t s) {
    static const struct Table {
        double2 v[kSectors];
        Table() {
            for (int j = 0; j < kSectors; ++j)
                v[j] = make_double2(cos((double)j * kSectorW), sin((double)j * kSectorW));
        }
    } table;
    return cudaMemcpyToSymbolAsync(g_sector, table.v, sizeof table.v, 0, cudaMemcpyHostToDevice, s);
}

int min_angle_blocks(int64_t V) {
    int64_t b = (V + MA_THREADS - 1) / MA_THREADS;
    if (b < 1) b = 1;
    if (b > MA_MAX_BLOCKS) b = MA_MAX_BLOCKS;
    return (int)b;
}

namespace {
// CSR of the non-zero-length incident directions of every vertex (global ids).
void build_direction_csr(Buffers &b, int64_t V, int64_t E, cudaStream_t s) {
    cudaMemsetAsync(b.deg, 0, sizeof(uint32_t) * (V + 1), s);
    cudaMemsetAsync(b.deg_fill, 0, sizeof(uint32_t) * V, s);
    const int gb = grid_for(E, 256, 152 * 8);
    count_launches(E > 0 ? 2 : 0);
    if (E > 0) k_degree<<<gb, 256, 0, s>>>(b.seg, b.acc, b.deg);
    launch_scan_u32(b.deg, b.deg, V, b.scan_tmp_side, &b.acc->scan_sink, &b.acc->eval_status, s);
    if (E > 0) k_fill_dirs<<<gb, 256, 0, s>>>(b.seg, b.acc, b.deg, b.deg_fill, b.dirs);
}
}  // namespace

void launch_adjacency(Buffers &b, int64_t V, int64_t E, cudaStream_t s) {
    if (V <= 0) return;
    cudaMemsetAsync(b.adj_off, 0, sizeof(uint32_t) * (V + 1), s);
    cudaMemsetAsync(b.deg_fill, 0, sizeof(uint32_t) * V, s);
    const int gb = grid_for(E, 256, 152 * 8);
    count_launches(E > 0 ? 2 : 0);
    if (E > 0) k_adj_degree<<<gb, 256, 0, s>>>((const int2 *)b.edges, E, V, b.adj_off);
    launch_scan_u32(b.adj_off, b.adj_off, V, b.scan_tmp, &b.acc->scan_sink, &b.acc->status, s);
    if (E > 0) k_adj_fill<<<gb, 256, 0, s>>>((const int2 *)b.edges, E, V, b.adj_off, b.deg_fill, b.adj);
}

void launch_min_angle(Buffers &b, int64_t V, int64_t E, cudaStream_t s) {
    if (V <= 0) return;
    count_launches(2);
    k_ma_dirs<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>((const int2 *)b.xy, V, b.adj_off, b.adj, b.ma_nz, b.dirs);
    k_min_angle<<<min_angle_blocks(V), MA_THREADS, 0, s>>>(b.adj_off, b.ma_nz, b.dirs, V, b.ma_dv, b.ma_part,
                                                           b.ma_cnt);
}

void launch_min_angle_moved(Buffers &b, int64_t V, const int32_t *ids, const int64_t *np, int64_t cap,
                            cudaStream_t s) {
    if (V <= 0) return;
    const int nb = min_angle_blocks(V);
    const int gw = grid_for(cap * 32, 256, 152 * 4);
    count_launches(3);
    k_ma_touch<<<gw, 256, 0, s>>>((const int2 *)b.xy, V, ids, np, b.adj_off, b.adj, b.ma_touch, b.ma_nz, b.dirs,
                                  b.ma_dv, b.ma_flag, nb);
    k_min_angle_resum<<<nb, MA_THREADS, 0, s>>>(b.ma_dv, V, b.ma_part, b.ma_cnt, b.ma_flag);
    k_ma_untouch<<<gw, 256, 0, s>>>(V, ids, np, b.adj_off, b.adj, b.ma_touch);
}

void launch_batch_min_angle(Buffers &b, const BatchView &bv, int64_t V, int64_t E, cudaStream_t s) {
    if (V <= 0 || bv.L <= 0) return;
    build_direction_csr(b, V, E, s);
    count_launches(1);
    const int blocks = (int)(bv.L < 152 * 16 ? bv.L : 152 * 16);
    k_batch_min_angle<<<blocks, MA_THREADS, 0, s>>>(b.deg, b.dirs, bv.v_off, bv.L, bv.res);
}

}  // namespace gr
