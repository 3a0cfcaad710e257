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
#include <cooperative_groups.h>
#include <math.h>

#include "grid_common.cuh"

namespace gr {

namespace cg = cooperative_groups;

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

// The work items of the evaluation's part: the items of the cells whose
// first record (d.x of an item's descriptor, ascending with the item index)
// lies in the part's share of the records, so that each cell falls to one
// part whatever order its records were placed in; binary searches over the
// descriptors by thread 0, shared through `sh`.  All items when the
// evaluation is not partitioned.  Every thread of the block must call it.
__device__ __forceinline__ void part_items(const DevAcc *acc, const uint4 *__restrict__ descs, uint32_t n_items,
                                           uint32_t *sh, uint32_t &i0, uint32_t &i1) {
    if (!partitioned(acc)) {
        i0 = 0;
        i1 = n_items;
        return;
    }
    if (threadIdx.x == 0) {
        uint64_t r[2];
        part_range(acc, acc->records, r[0], r[1]);
        for (int z = 0; z < 2; ++z) {  // the first item whose cell starts at record >= r[z]
            uint32_t lo = 0, hi = n_items;
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if ((uint64_t)descs[2 * (uint64_t)mid].x < r[z]) lo = mid + 1; else hi = mid;
            }
            sh[z] = lo;
        }
    }
    __syncthreads();
    i0 = sh[0];
    i1 = sh[1];
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
// pairs and long x short tiles; rot: rot_item_count).  Also sums the candidate pairs,
// ns (ns - 1) / 2 + ns (n - ns), of all cells.
__global__ void __launch_bounds__(256) k_cell_items(const uint32_t *__restrict__ cell_off,
                                                    const uint32_t *__restrict__ cell_nl, int C, int rot,
                                                    uint32_t *__restrict__ item_cnt, DevAcc *acc) {
    __shared__ uint64_t sh[32];
    uint64_t w = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const uint64_t n = cell_off[c + 1] - cell_off[c];
        const uint64_t ns = n - cell_nl[c];
        bool tiles_over;
        const uint64_t items = rot ? rot_item_count(n, &tiles_over) : cell_item_count(n, ns, &tiles_over);
        if (items > 0x7fffffffull || tiles_over) atomicOr(&acc->grid_flags, GF_ITEMS_OVERFLOW);
        item_cnt[c] = (uint32_t)min(items, (uint64_t)0x7fffffffull);
        w += ns * (ns - (ns > 0)) / 2 + ns * (n - ns);
    }
    w = block_sum<uint64_t>(w, sh);
    if (threadIdx.x == 0) atomic_add_u64(&acc->grid_work, w);
    // the rotation kernel's queue words keep a flag in the top bit of a record index
    if (rot && blockIdx.x == 0 && threadIdx.x == 0 && acc->records >= 0x80000000ull)
        atomicOr(&acc->grid_flags, GF_ITEMS_OVERFLOW);
}

// a3 + work items in one launch, for grids of at most kOffsetsMaxCells
// cells: the exclusive scan of the per-cell record counts (in place), the
// work items per cell and their exclusive scan, the candidate-pair total and
// the overflow flags -- what the three-kernel scans and k_cell_items do.  One
// thread-block cluster of kOffsetsCluster CTAs, 16 cells a thread: each CTA
// scans its cells, publishes its two totals in shared memory, and after a
// cluster barrier reads the totals of the CTAs before it through distributed
// shared memory.  Each thread reads its cells' counts before it overwrites
// them with offsets, and no other thread touches them (in place).
constexpr int kOffsetsThreads = 512, kOffsetsPer = 16, kOffsetsCluster = 8;
constexpr int kOffsetsMaxCells = kOffsetsCluster * kOffsetsThreads * kOffsetsPer;  // 65,536

__device__ __forceinline__ void block_excl_scan2(uint64_t a, uint64_t b, uint64_t &ea, uint64_t &eb, uint64_t &ta,
                                                 uint64_t &tb, uint64_t (*sh)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += ya; ib += yb; }
    }
    if (lane == 31) { sh[0][wid] = ia; sh[1][wid] = ib; }
    __syncthreads();
    if (wid == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        const uint64_t wa = in ? sh[0][lane] : 0ull, wb = in ? sh[1][lane] : 0ull;
        uint64_t xa = wa, xb = wb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) { xa += ya; xb += yb; }
        }
        sh[0][lane] = xa - wa;  // exclusive warp offsets
        sh[1][lane] = xb - wb;
        if (lane == 31) { sh[2][0] = xa; sh[2][1] = xb; }  // totals (zeros past the last warp)
    }
    __syncthreads();
    ea = sh[0][wid] + ia - a;
    eb = sh[1][wid] + ib - b;
    ta = sh[2][0];
    tb = sh[2][1];
}

__global__ void __cluster_dims__(kOffsetsCluster, 1, 1) __launch_bounds__(kOffsetsThreads)
    k_grid_offsets(uint32_t *__restrict__ cell_off, const uint32_t *__restrict__ cell_nl, int C, int rot,
                   uint32_t *__restrict__ item_off, DevAcc *acc) {
    __shared__ uint64_t sh[3][32];
    __shared__ uint64_t cta_tot[2];
    __shared__ uint64_t base_sh[4];
    __shared__ uint64_t shw[32];
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const int c0 = (int)rank * kOffsetsThreads * kOffsetsPer + threadIdx.x * kOffsetsPer;
    // whole runs of 16 cells by 16-byte accesses (C = G^2 is a multiple of 16
    // for G >= 4); the tail of smaller grids cell by cell
    const bool full = c0 + kOffsetsPer <= C;
    uint32_t n[kOffsetsPer], it[kOffsetsPer];
    uint64_t tr = 0, ti = 0, work = 0;
    bool over = false;
#pragma unroll
    for (int q = 0; q < kOffsetsPer / 4; ++q) {
        uint32_t vn[4], vl[4];
        if (full) {
            const uint4 v = *(const uint4 *)(cell_off + c0 + 4 * q);
            const uint4 l = *(const uint4 *)(cell_nl + c0 + 4 * q);
            vn[0] = v.x; vn[1] = v.y; vn[2] = v.z; vn[3] = v.w;
            vl[0] = l.x; vl[1] = l.y; vl[2] = l.z; vl[3] = l.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + 4 * q + j;
                vn[j] = c < C ? cell_off[c] : 0u;
                vl[j] = c < C ? cell_nl[c] : 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t nn = vn[j], ns = nn - vl[j];
            bool tiles_over;
            const uint64_t items = rot ? rot_item_count(nn, &tiles_over) : cell_item_count(nn, ns, &tiles_over);
            over |= items > 0x7fffffffull || tiles_over;
            n[4 * q + j] = vn[j];
            it[4 * q + j] = (uint32_t)min(items, (uint64_t)0x7fffffffull);
            work += ns * (ns - (ns > 0)) / 2 + ns * (nn - ns);
            tr += vn[j];
            ti += it[4 * q + j];
        }
    }
    uint64_t er, ei, sr, si;
    block_excl_scan2(tr, ti, er, ei, sr, si, sh);
    if (threadIdx.x == 0) {
        cta_tot[0] = sr;
        cta_tot[1] = si;
    }
    cluster.sync();
    if (threadIdx.x == 0) {
        uint64_t br = 0, bi = 0, ar = 0, ai = 0;
        for (unsigned q = 0; q < (unsigned)kOffsetsCluster; ++q) {
            const uint64_t *t = cluster.map_shared_rank(cta_tot, q);
            const uint64_t x = t[0], y = t[1];
            if (q < rank) { br += x; bi += y; }
            ar += x;
            ai += y;
        }
        base_sh[0] = br; base_sh[1] = bi; base_sh[2] = ar; base_sh[3] = ai;
    }
    __syncthreads();
    uint64_t r = base_sh[0] + er, i = base_sh[1] + ei;
#pragma unroll
    for (int q = 0; q < kOffsetsPer / 4; ++q) {
        uint32_t o[4], oi[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            o[j] = (uint32_t)r;
            oi[j] = (uint32_t)i;
            r += n[4 * q + j];
            i += it[4 * q + j];
        }
        if (full) {
            *(uint4 *)(cell_off + c0 + 4 * q) = make_uint4(o[0], o[1], o[2], o[3]);
            *(uint4 *)(item_off + c0 + 4 * q) = make_uint4(oi[0], oi[1], oi[2], oi[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + 4 * q + j;
                if (c < C) {
                    cell_off[c] = o[j];
                    item_off[c] = oi[j];
                }
            }
        }
    }
    work = block_sum<uint64_t>(work, shw);
    const int any_over = __syncthreads_or(over ? 1 : 0);
    if (threadIdx.x == 0) {
        if (work) atomic_add_u64(&acc->grid_work, work);
        if (any_over) atomicOr(&acc->grid_flags, GF_ITEMS_OVERFLOW);
        if (rank == 0) {
            const uint64_t ar = base_sh[2], ai = base_sh[3];
            cell_off[C] = (uint32_t)ar;
            item_off[C] = (uint32_t)ai;
            acc->records = ar;
            acc->grid_items = ai;
            if (ar > 0xffffffffull || ai > 0xffffffffull) atomicOr(&acc->eval_status, ST_SCAN_OVERFLOW);
            // the rotation kernel's queue words keep a flag in the top bit of a record index
            if (rot && ar >= 0x80000000ull) atomicOr(&acc->grid_flags, GF_ITEMS_OVERFLOW);
        }
    }
    cluster.sync();  // no CTA leaves while another may still read its totals
}

// Descriptor of every work item, two 16-byte words: {record offset of its
// cell, records, short records, tile word (see ItemTiles)} and {cell id}, so
// the pair kernel reads one descriptor per item instead of a chain of
// dependent loads.
__global__ void __launch_bounds__(256) k_item_descs(const uint32_t *__restrict__ item_off,
                                                    const uint32_t *__restrict__ cell_off,
                                                    const uint32_t *__restrict__ cell_nl, int C, int rot,
                                                    uint64_t cap, uint4 *__restrict__ desc, uint32_t *status) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const uint32_t q = item_off[c];
        const uint32_t e = item_off[c + 1];
        if (q == e) continue;
        if (e > cap) {
            atomicOr(status, ST_OVERFLOW);
            continue;
        }
        const uint32_t base = cell_off[c], n = cell_off[c + 1] - base, ns = n - cell_nl[c];
        auto emit = [&](uint32_t i, uint32_t word) {
            desc[2 * (uint64_t)i] = make_uint4(base, n, ns, word);
            desc[2 * (uint64_t)i + 1] = make_uint4((uint32_t)c, 0u, 0u, 0u);
        };
        if (rot) rot_item_words(n, q, e, emit);
        else cell_item_words(n, ns, q, e, emit);
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
                               g.x = make_uint4((uint32_t)qe, qt, (uint32_t)ids[0], 0u);
                               rec[p0] = g;
                               if (nc > 1) {
                                   g.x.z = (uint32_t)ids[1];
                                   rec[p1] = g;
                               }
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
    __shared__ uint32_t part_sh[2];
    uint32_t lo, i_end;  // this evaluation's share of the items
    part_items(acc, descs, n_items, part_sh, lo, i_end);
    uint32_t it = lo + blockIdx.x * GP_WARPS + wid;
    uint4 next = make_uint4(0, 0, 0, 0), next_c = make_uint4(0, 0, 0, 0);
    if (it < i_end) {
        next = descs[2 * (uint64_t)it];
        next_c = descs[2 * (uint64_t)it + 1];
    }
    for (; it < i_end; it += stride) {
        const uint4 d = next, dc = next_c;
        if (it + stride < i_end) {  // prefetch the next item
            next = descs[2 * (uint64_t)(it + stride)];
            next_c = descs[2 * (uint64_t)(it + stride) + 1];
        }
        const int cell = (int)dc.x;
        grid_item<PER_EDGE>(rec + d.x, item_tiles(d.y, d.z, d.w), (cell % G) << k, (cell / G) << k, k, cs[wid],
                            ideal, pc, pe);
    }
    flush_counts(pc, acc, shu);
}

// The FP32 cell-relative form of every record (make_rgeo) and its FP16 form
// (make_hgeo) for the rotation kernel, in record order: coalesced reads of
// the records (their cell id in .x.z) and coalesced writes of the four
// geometry arrays.
__global__ void __launch_bounds__(256) k_rec_geo(const GridRec *__restrict__ rec, const DevAcc *__restrict__ acc,
                                                 uint64_t cap, int k, float4 *__restrict__ geo) {
    const uint64_t R = acc->records;
    if (R > cap) return;  // overflow raised by the scatter
    const int lg = 16 - k, msk = (1 << lg) - 1;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < R; p += (uint64_t)gridDim.x * blockDim.x) {
        const SegRec q = rec[p].s;
        const int id = (int)rec[p].x.z;
        float4 a, b, c;
        make_rgeo(q, (id & msk) << k, (id >> lg) << k, 1 << k, a, b, c);
        geo[p] = a;
        geo[cap + p] = b;
        geo[2 * cap + p] = c;
        reinterpret_cast<uint4 *>(geo + 3 * cap)[p] = make_hgeo(b, c, 1 << k);
    }
}

// a6, rotation form -- one warp per rotation work item (rot_item_count):
// each lane keeps one row record of the cell in registers and meets the
// item's column window, staged in shared memory, at slots l + t.  The first
// test runs in FP16 (make_hgeo) on two offsets at once: window slot u holds
// the halves of its record and of the next one interleaved, so one half2
// operation tests the pairs of offsets t and t + 1.  With the margin above
// the FP16 error (half_margin), a pair is dropped when one clipped part lies
// beyond it on one side of the other's line, and counted at once as a proper
// crossing of this cell when each part straddles the other's line by more
// than it; in the same step a pair sharing a vertex is dropped (the window
// holds both records' vertex ids) and a counted pair adds its crossing
// angle's term (from the staged directions).  The undecided rest, about 2 %
// of the pairs, are queued by per-lane rounds and settled 32 at a time by the
// whole warp (settle_pair, on the FP32 records), so the rare cases never run
// with idle lanes.  The per-edge form takes its counted pairs in the rounds
// too (their tallies are atomics on both edges).
constexpr int CP_WARPS = 8;   // warps per block
constexpr int CP_QUEUE = 64;  // queued pairs per warp: up to 31 left + 32 pushed in one round

// Settles one queued pair (row, col) of a cell of side w: shared vertex ids
// skip it; the FP32 clip test drops it, or counts it as a proper crossing of
// this cell; else the FP32 orientations decide it when they are exact or
// clear of the filter, or the exact int64 test does, and a pair in E_c
// counts if its intersection point lies in this cell (decided by the clip
// test, else by the exact test), a collinear overlap if this cell holds the
// smallest point of the overlap.
template <bool PER_EDGE>
__device__ __forceinline__ void settle_pair(const float4 *__restrict__ geo, uint64_t cap,
                                            const GridRec *__restrict__ rec, uint2 e, int w, uint32_t ideal,
                                            PairCounts &pc, PerEdge pe) {
    const uint32_t row = e.x, col = e.y;
    const uint2 rid = *(const uint2 *)&rec[row].s.z, cid = *(const uint2 *)&rec[col].s.z;
    if ((rid.x == cid.x) | (rid.x == cid.y) | (rid.y == cid.x) | (rid.y == cid.y)) return;
    const float4 rb = geo[cap + row], cb = geo[cap + col];
    const ClipTest ct = clip_test(rb, geo[2 * cap + row], fminf(rb.w, kClipExact), cb, geo[2 * cap + col]);
    if (ct.out) return;
    int kind = PAIR_PROPER;
    if (!ct.both) {
        const float4 ra = geo[row], ca = geo[col];
        const Orient4 o = orient4(ra, rb, ca, cb);
        const float F = fmaxf(rb.w, cb.w) > kClipExact ? kRotFilter : 0.f;  // a filtered record takes part
        const float mn = fminf(fminf(fabsf(o.o1), fabsf(o.o2)), fminf(fabsf(o.o3), fabsf(o.o4)));
        if ((F == 0.f || mn > F) && !(o.o1 == 0.f && o.o2 == 0.f)) {
            const float p12 = o.o1 * o.o2, p34 = o.o3 * o.o4;
            kind = (p12 <= 0.f && p34 <= 0.f) ? ((p12 < 0.f && p34 < 0.f) ? PAIR_PROPER : PAIR_TOUCHING)
                                              : PAIR_NONE;
        } else {
            kind = classify_rel(ra, ca, rid.x, rid.y, cid.x, cid.y);
        }
        if (kind == PAIR_NONE) return;
        if (kind == PAIR_COLLINEAR) {
            if (!owns_collinear_rel(ra, ca, w)) return;
            ++pc.collinear;
            if (PER_EDGE) {
                atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)(int32_t)rec[row].x.x + 2], 1ull);
                atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)(int32_t)rec[col].x.x + 2], 1ull);
            }
            return;
        }
        if (!ct.in) {
            const int iax = (int)ra.x, iay = (int)ra.y, icx = (int)ca.x, icy = (int)ca.y;
            if (!owns_crossing(iax, iay, (int)ra.z - iax, (int)ra.w - iay, icx, icy, (int)ca.z - icx,
                               (int)ca.w - icy, w))
                return;
        }
    }
    const uint2 rx = *(const uint2 *)&rec[row].x, cx = *(const uint2 *)&rec[col].x;  // edge id, direction
    const uint32_t qd = dev_term(rx.y, cx.y, ideal);
    const bool prop = kind == PAIR_PROPER;
    pc.dev += qd;
    if (prop) ++pc.proper; else ++pc.touching;
    if (PER_EDGE) {
        const int slot = prop ? 0 : 1;
        atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)(int32_t)rx.x + slot], 1ull);
        atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)(int32_t)cx.x + slot], 1ull);
        atomicAdd((unsigned long long *)&pe.dev[(int32_t)rx.x], (unsigned long long)qd);
        atomicAdd((unsigned long long *)&pe.dev[(int32_t)cx.x], (unsigned long long)qd);
    }
}

// Settles the queue's whole batches of 32 and moves the rest to its front.
template <bool PER_EDGE>
__device__ __forceinline__ void settle_queue(const float4 *__restrict__ geo, uint64_t cap,
                                             const GridRec *__restrict__ rec, uint2 *q, int &qn, int lane, int w,
                                             uint32_t ideal, PairCounts &pc, PerEdge pe) {
    if (qn < 32) return;
    __syncwarp();
    int h = 0;
    for (; h + 32 <= qn; h += 32) settle_pair<PER_EDGE>(geo, cap, rec, q[h + lane], w, ideal, pc, pe);
    const uint2 rest = lane < qn - h ? q[h + lane] : make_uint2(0u, 0u);
    __syncwarp();
    if (lane < qn - h) q[lane] = rest;
    qn -= h;
    __syncwarp();
}

__device__ __forceinline__ __half2 as_half2(uint32_t u) {
    __half2 h;
    memcpy(&h, &u, sizeof(h));
    return h;
}

// x mod n for the window's rows (x below 2 n but for the smallest cells).
__device__ __forceinline__ uint32_t wrap_row(uint32_t x, uint32_t n) {
    if (x >= n) x -= n;
    return x < n ? x : x % n;
}

// The offset of bit b of a lane's masks: bit j holds offset 2 j, bit 16 + j
// offset 2 j + 1 (the low and high halves of the j-th half2 test).
__device__ __forceinline__ int mask_offset(int b) { return b < 16 ? 2 * b : 2 * (b - 16) + 1; }

template <bool PER_EDGE>
__global__ void __launch_bounds__(CP_WARPS * 32, 4) k_cell_pairs(const float4 *__restrict__ geo,
                                                                 const GridRec *__restrict__ rec,
                                                                 const uint4 *__restrict__ descs,
                                                                 const uint32_t *__restrict__ n_items_p,
                                                                 uint64_t rec_cap, uint64_t items_cap, int k,
                                                                 float margin, DevAcc *acc, uint32_t ideal,
                                                                 PerEdge pe) {
    __shared__ uint4 win_h[CP_WARPS][2][RWIN];  // slot u: halves of records u and u + 1, interleaved
    __shared__ uint32_t win_i[CP_WARPS][RWIN];  // slot u's record
    __shared__ uint2 win_d[CP_WARPS][RWIN];     // the directions of records u and u + 1
    __shared__ uint4 win_v[CP_WARPS][RWIN];     // the vertex ids of records u and u + 1
    __shared__ uint2 win_x[CP_WARPS][PER_EDGE ? RWIN : 1];  // slot u's edge id and direction (per-edge form)
    __shared__ uint2 qbuf[CP_WARPS][CP_QUEUE];
    __shared__ uint64_t shu[32];
    __shared__ uint32_t part_sh[2];
    const uint32_t n_items = *n_items_p;
    if (acc->records > rec_cap || n_items > items_cap) return;  // overflow raised by the scatter or descriptors
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int w = 1 << k;
    const unsigned lt = lanemask_lt();
    const uint4 *__restrict__ geo_h = reinterpret_cast<const uint4 *>(geo + 3 * rec_cap);
    uint4 *wh0 = win_h[wid][0], *wh1 = win_h[wid][1];
    uint32_t *wi = win_i[wid];
    uint2 *wd = win_d[wid], *wx = win_x[wid];
    uint4 *wv = win_v[wid];
    uint2 *q = qbuf[wid];
    const __half2 hm = __half2half2(__float2half_ru(margin)), nhm = __hneg2(hm);
    int qn = 0;
    PairCounts pc;
    uint32_t lo, i_end;  // this evaluation's share of the items
    part_items(acc, descs, n_items, part_sh, lo, i_end);
    const uint32_t stride = gridDim.x * CP_WARPS;
    uint32_t it = lo + blockIdx.x * CP_WARPS + wid;
    uint4 next = it < i_end ? descs[2 * (uint64_t)it] : make_uint4(0, 0, 0, 0);
    for (; it < i_end; it += stride) {
        const uint4 d = next;
        if (it + stride < i_end) next = descs[2 * (uint64_t)(it + stride)];  // prefetch the next item
        const uint32_t base = d.x, n = d.y;
        const RotLane rl = rot_lane((int)n, d.w, lane);
        // the item's column window: stream sigma's slots hold rows
        // first + sigma RQ + x (mod n) of the cell, x < m + RQ - 1
        const int span = rl.m + RQ - 1, slots = rl.s * span;
        __syncwarp();
        for (int u = lane; u < slots; u += 32) {
            const int sig = (u >= span ? 1 : 0) + (u >= 2 * span ? 1 : 0);  // s <= 3 streams
            const uint32_t x = rl.first + (uint32_t)(sig * RQ + (u - sig * span));
            const uint32_t r0 = base + wrap_row(x, n), r1 = base + wrap_row(x + 1, n);
            const uint4 A = geo_h[r0], B = geo_h[r1];
            wh0[u] = make_uint4(__byte_perm(A.x, B.x, 0x5410), __byte_perm(A.x, B.x, 0x7632),
                                __byte_perm(A.y, B.y, 0x5410), __byte_perm(A.y, B.y, 0x7632));
            wh1[u] = make_uint4(__byte_perm(A.z, B.z, 0x5410), __byte_perm(A.z, B.z, 0x7632),
                                __byte_perm(A.w, B.w, 0x5410), 0u);
            wi[u] = r0;
            const uint2 x0 = *(const uint2 *)&rec[r0].x, v0 = *(const uint2 *)&rec[r0].s.z;
            const uint2 v1 = *(const uint2 *)&rec[r1].s.z;
            wd[u] = make_uint2(x0.y, rec[r1].x.y);
            wv[u] = make_uint4(v0.x, v0.y, v1.x, v1.y);
            if (PER_EDGE) wx[u] = x0;
        }
        const uint32_t row = base + (uint32_t)rl.i;
        const uint4 R = geo_h[row];
        const __half2 rhx = as_half2(__byte_perm(R.x, R.x, 0x1010)), rhy = as_half2(__byte_perm(R.x, R.x, 0x3232));
        const __half2 rhc = as_half2(__byte_perm(R.y, R.y, 0x1010)), r0x = as_half2(__byte_perm(R.y, R.y, 0x3232));
        const __half2 r0y = as_half2(__byte_perm(R.z, R.z, 0x1010)), r1x = as_half2(__byte_perm(R.z, R.z, 0x3232));
        const __half2 r1y = as_half2(__byte_perm(R.w, R.w, 0x1010));
        const uint2 rx = *(const uint2 *)&rec[row].x, rv = *(const uint2 *)&rec[row].s.z;
        __syncwarp();
        const int jn = (int)((__reduce_max_sync(0xffffffffu, (unsigned)rl.cnt) + 1u) >> 1);  // half2 steps
        const int ce = (rl.cnt + 1) >> 1, co = rl.cnt >> 1;  // the lane's even and odd offsets
        const uint32_t valid = ((1u << ce) - 1u) | (((1u << co) - 1u) << 16);
        uint32_t mo = 0, ms = 0;  // dropped, counted
#pragma unroll
        for (int j = 0; j < RQ / 2; ++j) {
            if (j >= jn) break;
            const int u = rl.slot + 2 * j;
            const uint4 c0 = wh0[u], c1 = wh1[u];
            const __half2 chx = as_half2(c0.x), chy = as_half2(c0.y), chc = as_half2(c0.z);
            const __half2 c0x = as_half2(c0.w), c0y = as_half2(c1.x), c1x = as_half2(c1.y), c1y = as_half2(c1.z);
            // the column's line at the row's clipped part, the row's line at the column's
            const __half2 s0 = __hfma2(chx, r0y, __hfma2(chy, r0x, chc));
            const __half2 s1 = __hfma2(chx, r1y, __hfma2(chy, r1x, chc));
            const __half2 s2 = __hfma2(rhx, c0y, __hfma2(rhy, c0x, rhc));
            const __half2 s3 = __hfma2(rhx, c1y, __hfma2(rhy, c1x, rhc));
            // t > 0: both values on one side, by t; t < 0: a strict straddle, by -t
            const __half2 t01 = __hmax2(__hmin2(s0, s1), __hneg2(__hmax2(s0, s1)));
            const __half2 t23 = __hmax2(__hmin2(s2, s3), __hneg2(__hmax2(s2, s3)));
            const __half2 tt = __hmax2_nan(t01, t23);  // NaN (a border record): undecided
            const uint32_t lo_bit = 1u << j, hi_bit = 0x10000u << j, vj = valid & (lo_bit | hi_bit);
            const uint32_t sb = __hlt2_mask(tt, nhm) & vj;  // counted
            // dropped: apart in this cell, or sharing a vertex (never counted)
            const uint4 vv = wv[u];
            const bool sh0 = (rv.x == vv.x) | (rv.x == vv.y) | (rv.y == vv.x) | (rv.y == vv.y);
            const bool sh1 = (rv.x == vv.z) | (rv.x == vv.w) | (rv.y == vv.z) | (rv.y == vv.w);
            mo |= (__hgt2_mask(tt, hm) & (lo_bit | hi_bit)) | (sh0 ? lo_bit : 0u) | (sh1 ? hi_bit : 0u);
            ms |= sb;
            if (!PER_EDGE) {  // the crossing angle's terms of the counted pairs
                const uint2 dd = wd[u];
                const uint32_t q0 = (sb & lo_bit) ? dev_term(rx.y, dd.x, ideal) : 0u;
                const uint32_t q1 = (sb & hi_bit) ? dev_term(rx.y, dd.y, ideal) : 0u;
                pc.dev += (uint64_t)q0 + q1;
            }
        }
        ms &= valid;
        uint32_t mk = ~(mo | ms) & valid;
        const int n_counted = __popc(ms);
        pc.proper += n_counted;
        if (!PER_EDGE) ms = 0;  // their terms are in
        // one pair of each kind per lane a round: a counted pair (per-edge
        // form) adds its tallies; an undecided one is queued
        uint64_t rdev = 0;
        while (__any_sync(0xffffffffu, (ms | mk) != 0)) {
            if (PER_EDGE && ms) {
                const uint2 cx = wx[rl.slot + mask_offset(__ffs(ms) - 1)];
                ms &= ms - 1;
                const uint32_t qd = dev_term(rx.y, cx.y, ideal);
                pc.dev += qd;
                if (PER_EDGE) {
                    rdev += qd;
                    atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)(int32_t)cx.x], 1ull);
                    atomicAdd((unsigned long long *)&pe.dev[(int32_t)cx.x], (unsigned long long)qd);
                }
            }
            bool push = false;
            uint2 e = make_uint2(0u, 0u);
            if (mk) {
                const int u = rl.slot + mask_offset(__ffs(mk) - 1);
                mk &= mk - 1;
                push = true;
                e = make_uint2(row, wi[u]);
            }
            const unsigned m = __ballot_sync(0xffffffffu, push);
            if (push) q[qn + __popc(m & lt)] = e;
            qn += __popc(m);
            settle_queue<PER_EDGE>(geo, rec_cap, rec, q, qn, lane, w, ideal, pc, pe);
        }
        if (PER_EDGE && n_counted) {
            atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)(int32_t)rx.x], (unsigned long long)n_counted);
            atomicAdd((unsigned long long *)&pe.dev[(int32_t)rx.x], (unsigned long long)rdev);
        }
    }
    __syncwarp();
    if (lane < qn) settle_pair<PER_EDGE>(geo, rec_cap, rec, q[lane], w, ideal, pc, pe);
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
    count_launches(E > 0 ? 1 : 0);
    if (E > 0)
        k_grid_count<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc, k, split ? 1 : 0,
                                                                 g.cell_off, g.cell_nl, g.seg_long, g.theta_long,
                                                                 g.eid_long);
    const int rot = split ? 0 : 1;  // without the split every pair of a cell is a rotation pair
    if (C <= kOffsetsMaxCells) {
        count_launches(1);
        k_grid_offsets<<<kOffsetsCluster, kOffsetsThreads, 0, s>>>(g.cell_off, g.cell_nl, C, rot, g.item_off, b.acc);
        return;
    }
    launch_scan_u32(g.cell_off, g.cell_off, C, b.scan_tmp, &b.acc->records, &b.acc->eval_status, s);
    count_launches(1);
    k_cell_items<<<grid_for(C, 256, 152 * 8), 256, 0, s>>>(g.cell_off, g.cell_nl, C, rot, g.item_off, b.acc);
    launch_scan_u32(g.item_off, g.item_off, C, b.scan_tmp, &b.acc->grid_items, &b.acc->eval_status, s);
}

void launch_grid_scatter(const Buffers &b, int64_t E, const GridBuffers &g, int k, bool split, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    cudaMemsetAsync(g.cell_fill, 0, sizeof(unsigned long long) * C, s);
    count_launches(1 + (E > 0 ? 1 : 0));
    k_item_descs<<<grid_for(C, 256, 152 * 8), 256, 0, s>>>(g.item_off, g.cell_off, g.cell_nl, C, split ? 0 : 1,
                                                           g.items_cap, g.item_desc, &b.acc->eval_status);
    if (E <= 0) return;
    k_grid_fill<<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc, k, split ? 1 : 0,
                                                           g.cell_off, g.cell_fill, g.rec_cap, g.rec,
                                                           &b.acc->eval_status);
    if (!split) {
        count_launches(1);
        k_rec_geo<<<152 * 8, 256, 0, s>>>(g.rec, b.acc, g.rec_cap, k, g.rgeo);
    }
}

void launch_grid_pairs(const Buffers &b, const GridBuffers &g, int k, bool split, uint64_t n_items_hint,
                       uint32_t ideal, PerEdge pe, cudaStream_t s) {
    const int C = (65536 >> k) * (65536 >> k);
    if (!split) {  // rotation items over every pair of each cell
        const int blocks = n_items_hint ? grid_for((int64_t)n_items_hint, CP_WARPS, 152 * 4) : 152 * 4;
        count_launches(1);
        if (pe.counts)
            k_cell_pairs<true><<<blocks, CP_WARPS * 32, 0, s>>>(g.rgeo, g.rec, g.item_desc, g.item_off + C,
                                                               g.rec_cap, g.items_cap, k, half_margin(1 << k), b.acc,
                                                               ideal, pe);
        else
            k_cell_pairs<false><<<blocks, CP_WARPS * 32, 0, s>>>(g.rgeo, g.rec, g.item_desc, g.item_off + C,
                                                                g.rec_cap, g.items_cap, k, half_margin(1 << k), b.acc,
                                                                ideal, pe);
        return;
    }
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
    // the long list is filled in the order its warps arrived: in a partitioned
    // evaluation part 0 takes all of it
    launch_crossings_allpairs_of(g.seg_long, g.eid_long, g.theta_long, &b.acc->n_long, b.acc, n_bound, ideal, pe, s,
                                 true);
}

}  // namespace gr
