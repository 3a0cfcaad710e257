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

#include "grid_common.cuh"

namespace gr {

namespace {

constexpr int GP_WARPS = 8;  // warps per block of the pair kernel

// a2 -- per-cell record counts.
// Segment visited by thread slot i of n: i * (2^31 - 1) mod n, a bijection
// for n < 2^31 - 1 (2^31 - 1 is prime; larger n keep their order) that spreads runs of long edges (random
// edges appended after the short ones, say) over all warps instead of
// leaving them to the last few, which walk them one by one.
__device__ __forceinline__ int64_t spread_index(int64_t i, int64_t n) {
    if (n >= 0x7fffffffll) return i;
    return (int64_t)(((uint64_t)i * (0x7fffffffull % (uint64_t)n)) % (uint64_t)n);
}

__global__ void __launch_bounds__(256) k_grid_count(const SegRec *__restrict__ seg,
                                                    const DevAcc *__restrict__ acc, int k,
                                                    uint32_t *__restrict__ cell_cnt) {
    const int64_t n = acc->n_seg;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const SegRec r = ok ? seg[spread_index(i, n)] : make_uint4(0, 0, 0, 0);
        warp_for_each_cell(r, 0, 0u, ok, k, 0u, [&](const int (&ids)[2], int nc, SegRec, int32_t, uint32_t) {
            atomicAdd(&cell_cnt[ids[0]], 1u);
            if (nc > 1) atomicAdd(&cell_cnt[ids[1]], 1u);
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

// Descriptor of every work item: {record offset of its cell, records in the
// cell, cell id, row tile << 16 | column tile}, so the pair kernel reads one
// 16-byte word per item instead of a chain of dependent loads.
__global__ void __launch_bounds__(256) k_item_descs(const uint32_t *__restrict__ item_off,
                                                    const uint32_t *__restrict__ cell_off, int C,
                                                    uint4 *__restrict__ desc) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        uint32_t q = item_off[c];
        const uint32_t e = item_off[c + 1];
        if (q == e) continue;
        const uint32_t base = cell_off[c], n = cell_off[c + 1] - base;
        const uint32_t T = (n + TILE - 1) / TILE;
        for (uint32_t tj = 0; tj < T && q < e; ++tj)
            for (uint32_t ti = 0; ti <= tj && q < e; ++ti) desc[q++] = make_uint4(base, n, (uint32_t)c, (ti << 16) | tj);
    }
}

// a4 -- scatter of the records into their cells: segment, edge id and line
// direction go as one 32-byte record to cell_off[c] + (running count of c).
// A batch's atomics are issued before its stores.
__global__ void __launch_bounds__(256) k_grid_fill(const SegRec *__restrict__ seg,
                                                   const int32_t *__restrict__ seg_eid,
                                                   const uint32_t *__restrict__ seg_theta,
                                                   const DevAcc *__restrict__ acc, int k,
                                                   const uint32_t *__restrict__ cell_off,
                                                   uint32_t *__restrict__ cell_fill, uint64_t cap,
                                                   GridRec *__restrict__ rec, uint32_t *status) {
    const int64_t n = acc->n_seg;
    if (acc->records > cap) {  // sized from the same counts; cannot happen unless inputs changed
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_OVERFLOW);
        return;
    }
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const int64_t j = ok ? spread_index(i, n) : 0;
        const SegRec r = ok ? seg[j] : make_uint4(0, 0, 0, 0);
        const int32_t eid = ok ? seg_eid[j] : 0;
        const uint32_t th = ok ? seg_theta[j] : 0u;
        warp_for_each_cell(r, eid, th, ok, k, 0u, [&](const int (&ids)[2], int nc, SegRec q, int32_t qe, uint32_t qt) {
            const uint32_t s0 = atomicAdd(&cell_fill[ids[0]], 1u);
            const uint32_t s1 = nc > 1 ? atomicAdd(&cell_fill[ids[1]], 1u) : 0u;
            const uint32_t o0 = cell_off[ids[0]];
            const uint32_t o1 = nc > 1 ? cell_off[ids[1]] : 0u;
            GridRec g;
            g.s = q;
            g.x = make_uint4((uint32_t)qe, qt, 0u, 0u);
            rec[o0 + s0] = g;
            if (nc > 1) rec[o1 + s1] = g;
        });
    }
}

// a6 -- one warp per work item (cell, row tile, column tile); items in a
// warp-strided static order, the next item's descriptor prefetched.
template <bool PER_EDGE>
__global__ void __launch_bounds__(GP_WARPS * 32, 4) k_grid_pairs(const GridRec *__restrict__ rec,
                                                                 const uint4 *__restrict__ descs, uint32_t n_items,
                                                                 int k, DevAcc *acc, uint32_t ideal, PerEdge pe) {
    __shared__ GSeg cs[GP_WARPS][TILE];
    __shared__ uint64_t shu[32];
    const int wid = threadIdx.x >> 5;
    const int G = 65536 >> k;
    const uint32_t stride = gridDim.x * GP_WARPS;
    PairCounts pc;
    uint32_t it = blockIdx.x * GP_WARPS + wid;
    uint4 next = it < n_items ? descs[it] : make_uint4(0, 0, 0, 0);
    for (; it < n_items; it += stride) {
        const uint4 d = next;
        if (it + stride < n_items) next = descs[it + stride];  // prefetch the next item
        const int cell = (int)d.z;
        grid_item<PER_EDGE>(rec + d.x, (int)d.y, (int)(d.w >> 16), (int)(d.w & 0xffffu), (cell % G) << k,
                            (cell / G) << k, k, cs[wid], ideal, pc, pe);
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
    count_launches(1 + (E > 0 ? 1 : 0));
    k_item_descs<<<grid_for(C, 256, 152 * 8), 256, 0, s>>>(g.item_off, g.cell_off, C, g.item_desc);
    if (E <= 0) return;
    k_grid_fill<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc, k, g.cell_off,
                                                           g.cell_fill, g.rec_cap, g.rec, &b.acc->eval_status);
}

void launch_grid_pairs(const Buffers &b, const GridBuffers &g, int k, uint64_t n_items, uint32_t ideal,
                       PerEdge pe, cudaStream_t s) {
    if (n_items == 0) return;
    const int blocks = grid_for((int64_t)n_items, GP_WARPS, 152 * 8);
    count_launches(1);
    if (pe.counts)
        k_grid_pairs<true><<<blocks, GP_WARPS * 32, 0, s>>>(g.rec, g.item_desc, (uint32_t)n_items, k, b.acc, ideal,
                                                           pe);
    else
        k_grid_pairs<false><<<blocks, GP_WARPS * 32, 0, s>>>(g.rec, g.item_desc, (uint32_t)n_items, k, b.acc,
                                                            ideal, pe);
}

}  // namespace gr
