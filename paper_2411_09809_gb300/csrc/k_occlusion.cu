// k_occlusion.cu -- node occlusion N_c (a8): Algorithm 1's predicate
// ||p_v - p_u||^2 < d^2 over unordered vertex pairs, exact in int64.
#include <math.h>

#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int OC_ROWS = 256;
constexpr int OC_COLS = 256;

// All-pairs tiles, one block per (row tile, column tile) with bi <= bj in
// lower-triangular order; the diagonal tiles take only j > i.
__global__ void __launch_bounds__(OC_ROWS) k_occl_allpairs(const int2 *__restrict__ xy, int V,
                                                           long long d2, DevAcc *acc, int64_t tiles) {
    __shared__ int2 cp[OC_COLS];
    __shared__ uint64_t shu[32];
    uint32_t cnt = 0;
    uint64_t lo, hi;  // this evaluation's share of the tiles
    part_range(acc, (uint64_t)tiles, lo, hi);
    for (int64_t t = (int64_t)lo + blockIdx.x; t < (int64_t)hi; t += gridDim.x) {
        int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while (r * (r + 1) / 2 > t) --r;
        while ((r + 1) * (r + 2) / 2 <= t) ++r;
        const int bj = (int)r, bi = (int)(t - r * (r + 1) / 2);
        const int j0 = bj * OC_COLS;
        const int nc = min(OC_COLS, V - j0);
        __syncthreads();
        if (threadIdx.x < nc) cp[threadIdx.x] = xy[j0 + threadIdx.x];
        const int i = bi * OC_ROWS + threadIdx.x;
        int2 p = make_int2(0, 0);
        if (i < V) p = xy[i];
        __syncthreads();
        if (i < V) {
            const int jbeg = (bi == bj) ? threadIdx.x + 1 : 0;
#pragma unroll 8
            for (int jj = jbeg; jj < nc; ++jj) {
                const int2 q = cp[jj];
                const long long dx = p.x - q.x, dy = p.y - q.y;
                cnt += (dx * dx + dy * dy < d2) ? 1u : 0u;
            }
        }
    }
    const uint64_t s = block_sum<uint64_t>(cnt, shu);
    if (threadIdx.x == 0) atomic_add_u64(&acc->occlusion, s);
}

// ------------------------------------------------------------ occlusion grid
// Cells of side w = 2^k >= d: two vertices closer than d lie in the same or
// in 8-adjacent cells (the 2r x 2r grid of Sec. 3.2.1).  Each vertex is put
// in exactly one cell and each unordered pair of cells is visited once
// through the half stencil {E, NE, N, NW}, so no pair is seen twice and the
// paper's `distinct` step is not needed.  Vertices with a coordinate outside
// [0, 65536) (the evaluation then reports GR_ERANGE) are left out of the
// grids, so no kernel indexes a cell from them.

__device__ __forceinline__ bool in_range(int2 p) { return (unsigned)p.x < 65536u && (unsigned)p.y < 65536u; }

__global__ void __launch_bounds__(256) k_occl_count(const int2 *__restrict__ xy, int64_t V, int k,
                                                    uint32_t *__restrict__ cnt) {
    const int G = 65536 >> k;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = xy[v];
        if (!in_range(p)) continue;
        atomicAdd(&cnt[(p.y >> k) * G + (p.x >> k)], 1u);
    }
}

__global__ void __launch_bounds__(256) k_occl_fill(const int2 *__restrict__ xy, int64_t V, int k,
                                                   const uint32_t *__restrict__ off,
                                                   uint32_t *__restrict__ fill, uint32_t *__restrict__ pts) {
    const int G = 65536 >> k;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = xy[v];
        if (!in_range(p)) continue;
        const int c = (p.y >> k) * G + (p.x >> k);
        const uint32_t slot = atomicAdd(&fill[c], 1u);
        pts[off[c] + slot] = uint32_t(p.x) | (uint32_t(p.y) << 16);
    }
}

__device__ __forceinline__ uint32_t count_close(uint32_t p, const uint32_t *__restrict__ pts, uint32_t b,
                                                uint32_t e, long long d2) {
    uint32_t n = 0;
    const int x = px(p), y = py(p);
    for (uint32_t q = b; q < e; ++q) {
        const uint32_t o = pts[q];
        const long long dx = x - px(o), dy = y - py(o);
        n += (dx * dx + dy * dy < d2) ? 1u : 0u;
    }
    return n;
}

// One thread per placed vertex (off[C] of them) in cell order: later
// vertices of its own cell, then every vertex of the E, NE, N and NW cells.
__global__ void __launch_bounds__(256) k_occl_pairs(const uint32_t *__restrict__ pts,
                                                    const uint32_t *__restrict__ off, int C, int k,
                                                    long long d2, DevAcc *acc) {
    __shared__ uint64_t sh[32];
    const int G = 65536 >> k;
    const int64_t V = off[C];
    // this evaluation's share: the vertices of the cells whose first vertex
    // lies in the part's share of the placed vertices (a cell falls to one
    // part whatever order its vertices were placed in)
    uint64_t lo = 0, hi = (uint64_t)V;
    const bool part = partitioned(acc);
    if (part) part_range(acc, (uint64_t)V, lo, hi);
    uint64_t cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = pts[i];
        const int cx = px(p) >> k, cy = py(p) >> k;
        const int c = cy * G + cx;
        if (part && (off[c] < lo || off[c] >= hi)) continue;
        cnt += count_close(p, pts, (uint32_t)i + 1, off[c + 1], d2);
        if (cx + 1 < G) cnt += count_close(p, pts, off[c + 1], off[c + 2], d2);
        if (cy + 1 < G) {
            const int up = c + G;
            if (cx > 0) cnt += count_close(p, pts, off[up - 1], off[up], d2);
            cnt += count_close(p, pts, off[up], off[up + 1], d2);
            if (cx + 1 < G) cnt += count_close(p, pts, off[up + 1], off[up + 2], d2);
        }
    }
    cnt = block_sum<uint64_t>(cnt, sh);
    if (threadIdx.x == 0) atomic_add_u64(&acc->occlusion, cnt);
}

// Batch: vertex v of layout l goes to cell obase[l] + (y >> ko[l]) G_l + (x >> ko[l]).
__global__ void __launch_bounds__(256) k_batch_occl_count(const int2 *__restrict__ xy, int64_t V,
                                                          const int64_t *__restrict__ v_off, int64_t L,
                                                          const int32_t *__restrict__ ko,
                                                          const uint32_t *__restrict__ obase,
                                                          uint32_t *__restrict__ cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = find_segment(v_off, L, v);
        const int k = ko[l], G = 65536 >> k;
        const int2 p = xy[v];
        if (!in_range(p)) continue;
        atomicAdd(&cnt[obase[l] + (uint32_t)((p.y >> k) * G + (p.x >> k))], 1u);
    }
}

__global__ void __launch_bounds__(256) k_batch_occl_fill(const int2 *__restrict__ xy, int64_t V,
                                                         const int64_t *__restrict__ v_off, int64_t L,
                                                         const int32_t *__restrict__ ko,
                                                         const uint32_t *__restrict__ obase,
                                                         const uint32_t *__restrict__ off, uint32_t *__restrict__ fill,
                                                         uint32_t *__restrict__ pts, uint32_t *__restrict__ lay) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = find_segment(v_off, L, v);
        const int k = ko[l], G = 65536 >> k;
        const int2 p = xy[v];
        if (!in_range(p)) continue;
        const uint32_t c = obase[l] + (uint32_t)((p.y >> k) * G + (p.x >> k));
        const uint32_t pos = off[c] + atomicAdd(&fill[c], 1u);
        pts[pos] = uint32_t(p.x) | (uint32_t(p.y) << 16);
        lay[pos] = (uint32_t)l;
    }
}

// One thread per placed vertex (off[OC] of them) in cell order, within its
// own layout's grid.
__global__ void __launch_bounds__(256) k_batch_occl_pairs(const uint32_t *__restrict__ pts,
                                                          const uint32_t *__restrict__ lay,
                                                          const uint32_t *__restrict__ off, uint32_t OC,
                                                          const int32_t *__restrict__ ko,
                                                          const uint32_t *__restrict__ obase, long long d2,
                                                          uint64_t *__restrict__ occl) {
    const int64_t V = off[OC];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = pts[i];
        const uint32_t l = lay[i];
        const int k = ko[l], G = 65536 >> k;
        const int cx = px(p) >> k, cy = py(p) >> k;
        const uint32_t c = obase[l] + (uint32_t)(cy * G + cx);
        uint32_t cnt = count_close(p, pts, (uint32_t)i + 1, off[c + 1], d2);
        if (cx + 1 < G) cnt += count_close(p, pts, off[c + 1], off[c + 2], d2);
        if (cy + 1 < G) {
            const uint32_t up = c + (uint32_t)G;
            if (cx > 0) cnt += count_close(p, pts, off[up - 1], off[up], d2);
            cnt += count_close(p, pts, off[up], off[up + 1], d2);
            if (cx + 1 < G) cnt += count_close(p, pts, off[up + 1], off[up + 2], d2);
        }
        if (cnt) atomicAdd((unsigned long long *)&occl[l], (unsigned long long)cnt);
    }
}

int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

void launch_occlusion_grid_count(const Buffers &b, int64_t V, const GridBuffers &g, int k, cudaStream_t s) {
    const int G = 65536 >> k, C = G * G;
    cudaMemsetAsync(g.ocell_off, 0, sizeof(uint32_t) * (C + 1), s);
    count_launches(V > 0 ? 1 : 0);
    if (V > 0) k_occl_count<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>((const int2 *)b.xy, V, k, g.ocell_off);
    launch_scan_u32(g.ocell_off, g.ocell_off, C, b.scan_tmp_side, &b.acc->scan_sink, &b.acc->eval_status, s);
}

void launch_occlusion_grid_pairs(const Buffers &b, int64_t V, const GridBuffers &g, int k, int64_t d,
                                 cudaStream_t s) {
    const int G = 65536 >> k, C = G * G;
    if (V < 2 || d <= 0) return;
    cudaMemsetAsync(g.ocell_fill, 0, sizeof(uint32_t) * C, s);
    count_launches(2);
    k_occl_fill<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>((const int2 *)b.xy, V, k, g.ocell_off, g.ocell_fill,
                                                         g.opts);
    k_occl_pairs<<<grid_for(V, 256, 152 * 16), 256, 0, s>>>(g.opts, g.ocell_off, C, k, (long long)d * d, b.acc);
}

void launch_batch_occlusion(const Buffers &b, const BatchView &bv, int64_t V, const int32_t *ko,
                            const uint32_t *obase, uint32_t OC, uint32_t *ocell_off, uint32_t *ocell_fill,
                            uint32_t *opts, uint32_t *olay, int64_t d, uint64_t *occl, cudaStream_t s) {
    cudaMemsetAsync(occl, 0, sizeof(uint64_t) * bv.L, s);
    if (V < 2 || d <= 0 || OC == 0) return;
    cudaMemsetAsync(ocell_off, 0, sizeof(uint32_t) * ((size_t)OC + 1), s);
    cudaMemsetAsync(ocell_fill, 0, sizeof(uint32_t) * OC, s);
    const int g = grid_for(V, 256, 152 * 8);
    count_launches(3);
    k_batch_occl_count<<<g, 256, 0, s>>>((const int2 *)b.xy, V, bv.v_off, bv.L, ko, obase, ocell_off);
    launch_scan_u32(ocell_off, ocell_off, OC, b.scan_tmp_side, &b.acc->scan_sink, &b.acc->eval_status, s);
    k_batch_occl_fill<<<g, 256, 0, s>>>((const int2 *)b.xy, V, bv.v_off, bv.L, ko, obase, ocell_off, ocell_fill, opts,
                                        olay);
    k_batch_occl_pairs<<<grid_for(V, 256, 152 * 16), 256, 0, s>>>(opts, olay, ocell_off, OC, ko, obase,
                                                                  (long long)d * d, occl);
}

void launch_occlusion_allpairs(const Buffers &b, int64_t V, int64_t d, cudaStream_t s) {
    if (V < 2 || d <= 0) return;
    const int64_t nb = (V + OC_ROWS - 1) / OC_ROWS;
    const int64_t tiles = nb * (nb + 1) / 2;
    // any d beyond the largest possible distance counts every pair
    const long long d2 = d >= 100000 ? (long long)1e11 : (long long)d * d;
    const unsigned grid = (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
    count_launches(1);
    k_occl_allpairs<<<grid, OC_ROWS, 0, s>>>((const int2 *)b.xy, (int)V, d2, b.acc, tiles);
}

}  // namespace gr
