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
// Segments spanning more than two major lines of the grid are "long"; their
// records sit after the short ones in each cell, the pair kernel skips pairs
// of two long records, and those pairs go to the all-pairs tiles over the
// list of long segments instead (a grid cannot prune them: two long segments
// share about as many cells as there are such pairs).
#include <math.h>

#include "grid_common.cuh"

namespace gr {

namespace {

constexpr int GP_WARPS = 8;  // warps per block of the pair kernel

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Segment visited by thread slot i of n: i * (2^31 - 1) mod n, a bijection
// for n < 2^31 - 1 (2^31 - 1 is prime; larger n keep their order).  It
// spreads runs of long edges (random edges appended after the short ones,
// say) over all warps instead of leaving them to the last few, which walk
// them one by one.  The product (< 2^62) is reduced by Barrett's method with
// inv = floor((2^64 - 1) / n), set up once per block: the quotient estimate
// floor(p inv / 2^64) is at most one below floor(p / n), so one conditional
// subtraction finishes it (integer multiplies only, no 64-bit division or
// remainder per thread).
struct Spread {
    uint64_t n, m, inv;
};

__device__ __forceinline__ Spread spread_setup(int64_t n, Spread *sh) {
    if (threadIdx.x == 0) {
        Spread s{(uint64_t)n, 0, 0};
        if (n > 0 && n < 0x7fffffffll) {
            s.m = 0x7fffffffull % (uint64_t)n;
            s.inv = ~0ull / (uint64_t)n;
        }
        *sh = s;
    }
    __syncthreads();
    return *sh;
}

__device__ __forceinline__ int64_t spread_index(int64_t i, const Spread &s) {
    if (s.n >= 0x7fffffffull) return i;
    const uint64_t p = (uint64_t)i * s.m;
    uint64_t r = p - __umul64hi(p, s.inv) * s.n;
    if (r >= s.n) r -= s.n;
    return (int64_t)r;
}

// a2 -- per-cell record counts (all, and long ones); the long segments are
// appended to the long list.
__global__ void __launch_bounds__(256) k_grid_count(const SegRec *__restrict__ seg,
                                                    const int32_t *__restrict__ seg_eid,
                                                    const uint32_t *__restrict__ seg_theta, DevAcc *acc, int k,
                                                    int split, uint32_t *__restrict__ cell_cnt,
                                                    uint32_t *__restrict__ cell_nl,
                                                    SegRec *__restrict__ seg_long, uint32_t *__restrict__ theta_long,
                                                    int32_t *__restrict__ eid_long) {
    __shared__ Spread sp_sh;
    const int64_t n = acc->n_seg;
    const Spread sp = spread_setup(n, &sp_sh);
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const int64_t j = ok ? spread_index(i, sp) : 0;
        const SegRec r = ok ? seg[j] : make_uint4(0, 0, 0, 0);
        const bool lng = split && ok && is_long_seg(r, k);
        const unsigned ml = __ballot_sync(0xffffffffu, lng);
        if (ml) {
            uint32_t slot = 0;
            if (lane == 0) slot = atomicAdd(&acc->n_long, (uint32_t)__popc(ml));
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (lng) {
                const uint32_t pos = slot + __popc(ml & lanemask_lt());
                seg_long[pos] = r;
                theta_long[pos] = seg_theta[j];
                eid_long[pos] = seg_eid[j];
            }
        }
        warp_for_each_cell(r, 0, 0u, ok, k, 0u, split != 0,
                           [&](const int (&ids)[2], int nc, SegRec, int32_t, uint32_t, bool lng_cell) {
                               atomicAdd(&cell_cnt[ids[0]], 1u);
                               if (nc > 1) atomicAdd(&cell_cnt[ids[1]], 1u);
                               if (lng_cell) {
                                   atomicAdd(&cell_nl[ids[0]], 1u);
                                   if (nc > 1) atomicAdd(&cell_nl[ids[1]], 1u);
                               }
                           });
    }
}

// Work items of the pair kernel per cell (cell_item_count: short x short tile
// pairs and long x short tiles).  Also sums the candidate pairs,
// ns (ns - 1) / 2 + ns (n - ns), of all cells.
__global__ void __launch_bounds__(256) k_cell_items(const uint32_t *__restrict__ cell_off,
                                                    const uint32_t *__restrict__ cell_nl, int C,
                                                    uint32_t *__restrict__ item_cnt, DevAcc *acc) {
    __shared__ uint64_t sh[32];
    uint64_t w = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const uint64_t n = cell_off[c + 1] - cell_off[c];
        const uint64_t ns = n - cell_nl[c];
        bool tiles_over;
        const uint64_t items = cell_item_count(n, ns, &tiles_over);
        if (items > 0x7fffffffull || tiles_over) atomicOr(&acc->grid_flags, GF_ITEMS_OVERFLOW);
        item_cnt[c] = (uint32_t)min(items, (uint64_t)0x7fffffffull);
        w += ns * (ns - (ns > 0)) / 2 + ns * (n - ns);
    }
    w = block_sum<uint64_t>(w, sh);
    if (threadIdx.x == 0) atomic_add_u64(&acc->grid_work, w);
}

// Descriptor of every work item, two 16-byte words: {record offset of its
// cell, records, short records, tile word (see ItemTiles)} and {cell id}, so
// the pair kernel reads one descriptor per item instead of a chain of
// dependent loads.
__global__ void __launch_bounds__(256) k_item_descs(const uint32_t *__restrict__ item_off,
                                                    const uint32_t *__restrict__ cell_off,
                                                    const uint32_t *__restrict__ cell_nl, int C, uint64_t cap,
                                                    uint4 *__restrict__ desc, uint32_t *status) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const uint32_t q = item_off[c];
        const uint32_t e = item_off[c + 1];
        if (q == e) continue;
        if (e > cap) {
            atomicOr(status, ST_OVERFLOW);
            continue;
        }
        const uint32_t base = cell_off[c], n = cell_off[c + 1] - base, ns = n - cell_nl[c];
        cell_item_words(n, ns, q, e, [&](uint32_t i, uint32_t word) {
            desc[2 * (uint64_t)i] = make_uint4(base, n, ns, word);
            desc[2 * (uint64_t)i + 1] = make_uint4((uint32_t)c, 0u, 0u, 0u);
        });
    }
}

// a4 -- scatter of the records into their cells: segment, edge id and line
// direction go as one 32-byte record; short records fill each cell from its
// start, long ones from its end (one 64-bit counter per cell holds both
// running counts).  A batch's atomics are issued before its stores.
__global__ void __launch_bounds__(256) k_grid_fill(const SegRec *__restrict__ seg,
                                                   const int32_t *__restrict__ seg_eid,
                                                   const uint32_t *__restrict__ seg_theta,
                                                   const DevAcc *__restrict__ acc, int k, int split,
                                                   const uint32_t *__restrict__ cell_off,
                                                   unsigned long long *__restrict__ cell_fill, uint64_t cap,
                                                   GridRec *__restrict__ rec, uint32_t *status) {
    __shared__ Spread sp_sh;
    const int64_t n = acc->n_seg;
    if (acc->records > cap) {  // sized from the same counts; cannot happen unless inputs changed
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_OVERFLOW);
        return;
    }
    const Spread sp = spread_setup(n, &sp_sh);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const int64_t j = ok ? spread_index(i, sp) : 0;
        const SegRec r = ok ? seg[j] : make_uint4(0, 0, 0, 0);
        const int32_t eid = ok ? seg_eid[j] : 0;
        const uint32_t th = ok ? seg_theta[j] : 0u;
        warp_for_each_cell(r, eid, th, ok, k, 0u, split != 0,
                           [&](const int (&ids)[2], int nc, SegRec q, int32_t qe, uint32_t qt, bool lng) {
                               const unsigned long long inc = lng ? (1ull << 32) : 1ull;
                               const unsigned long long s0 = atomicAdd(&cell_fill[ids[0]], inc);
                               const unsigned long long s1 = nc > 1 ? atomicAdd(&cell_fill[ids[1]], inc) : 0ull;
                               uint32_t p0, p1 = 0;
                               if (lng) {
                                   p0 = cell_off[ids[0] + 1] - 1u - (uint32_t)(s0 >> 32);
                                   if (nc > 1) p1 = cell_off[ids[1] + 1] - 1u - (uint32_t)(s1 >> 32);
                               } else {
                                   p0 = cell_off[ids[0]] + (uint32_t)s0;
                                   if (nc > 1) p1 = cell_off[ids[1]] + (uint32_t)s1;
                               }
                               GridRec g;
                               g.s = q;
                               g.x = make_uint4((uint32_t)qe, qt, 0u, 0u);
                               rec[p0] = g;
                               if (nc > 1) rec[p1] = g;
                           });
    }
}

// a6 -- one warp per work item (cell, row tile, column tile); items in a
// warp-strided static order, the next item's descriptor prefetched.
template <bool PER_EDGE>
__global__ void __launch_bounds__(GP_WARPS * 32, 4) k_grid_pairs(const GridRec *__restrict__ rec,
                                                                 const uint4 *__restrict__ descs,
                                                                 const uint32_t *__restrict__ n_items_p,
                                                                 uint64_t rec_cap, uint64_t items_cap, int k,
                                                                 DevAcc *acc, uint32_t ideal, PerEdge pe) {
    __shared__ GSeg cs[GP_WARPS][TILE];
    __shared__ uint64_t shu[32];
    const uint32_t n_items = *n_items_p;
    if (acc->records > rec_cap || n_items > items_cap) return;  // overflow raised by the scatter or descriptors
    const int wid = threadIdx.x >> 5;
    const int G = 65536 >> k;
    const uint32_t stride = gridDim.x * GP_WARPS;
    PairCounts pc;
    uint32_t it = blockIdx.x * GP_WARPS + wid;
    uint4 next = make_uint4(0, 0, 0, 0), next_c = make_uint4(0, 0, 0, 0);
    if (it < n_items) {
        next = descs[2 * (uint64_t)it];
        next_c = descs[2 * (uint64_t)it + 1];
    }
    for (; it < n_items; it += stride) {
        const uint4 d = next, dc = next_c;
        if (it + stride < n_items) {  // prefetch the next item
            next = descs[2 * (uint64_t)(it + stride)];
            next_c = descs[2 * (uint64_t)(it + stride) + 1];
        }
        const int cell = (int)dc.x;
        grid_item<PER_EDGE>(rec + d.x, item_tiles(d.y, d.z, d.w), (cell % G) << k, (cell / G) << k, k, cs[wid],
                            ideal, pc, pe);
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

void launch_grid_count(const Buffers &b, int64_t E, const GridBuffers &g, int k, bool split, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    cudaMemsetAsync(g.cell_off, 0, sizeof(uint32_t) * (C + 1), s);
    cudaMemsetAsync(g.cell_nl, 0, sizeof(uint32_t) * C, s);
    count_launches(E > 0 ? 2 : 1);
    if (E > 0)
        k_grid_count<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc, k, split ? 1 : 0,
                                                                 g.cell_off, g.cell_nl, g.seg_long, g.theta_long,
                                                                 g.eid_long);
    launch_scan_u32(g.cell_off, g.cell_off, C, b.scan_tmp, &b.acc->records, &b.acc->eval_status, s);
    k_cell_items<<<grid_for(C, 256, 152 * 8), 256, 0, s>>>(g.cell_off, g.cell_nl, C, g.item_off, b.acc);
    launch_scan_u32(g.item_off, g.item_off, C, b.scan_tmp, &b.acc->grid_items, &b.acc->eval_status, s);
}

void launch_grid_scatter(const Buffers &b, int64_t E, const GridBuffers &g, int k, bool split, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    cudaMemsetAsync(g.cell_fill, 0, sizeof(unsigned long long) * C, s);
    count_launches(1 + (E > 0 ? 1 : 0));
    k_item_descs<<<grid_for(C, 256, 152 * 8), 256, 0, s>>>(g.item_off, g.cell_off, g.cell_nl, C, g.items_cap,
                                                           g.item_desc, &b.acc->eval_status);
    if (E <= 0) return;
    k_grid_fill<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc, k, split ? 1 : 0,
                                                           g.cell_off, g.cell_fill, g.rec_cap, g.rec,
                                                           &b.acc->eval_status);
}

void launch_grid_pairs(const Buffers &b, const GridBuffers &g, int k, uint64_t n_items_hint, uint32_t ideal,
                       PerEdge pe, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    const int blocks = n_items_hint ? grid_for((int64_t)n_items_hint, GP_WARPS, 152 * 8) : 152 * 8;
    count_launches(1);
    if (pe.counts)
        k_grid_pairs<true><<<blocks, GP_WARPS * 32, 0, s>>>(g.rec, g.item_desc, g.item_off + C, g.rec_cap,
                                                           g.items_cap, k, b.acc, ideal, pe);
    else
        k_grid_pairs<false><<<blocks, GP_WARPS * 32, 0, s>>>(g.rec, g.item_desc, g.item_off + C, g.rec_cap,
                                                            g.items_cap, k, b.acc, ideal, pe);
}

void launch_grid_long_pairs(const Buffers &b, const GridBuffers &g, int64_t n_bound, uint32_t ideal, PerEdge pe,
                            cudaStream_t s) {
    launch_crossings_allpairs_of(g.seg_long, g.eid_long, g.theta_long, &b.acc->n_long, b.acc, n_bound, ideal, pe, s);
}

}  // namespace gr
