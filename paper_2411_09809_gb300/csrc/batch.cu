// batch.cu -- gr_batch_*: many independent layouts evaluated together.
//
// Layouts are packed one after another (vertex and edge offsets per layout,
// edges with layout-local vertex ids).  Every step of the single-layout path
// runs once over the whole pack:
//   gather      global vertex ids, segments, directions, the layout of each
//               segment;
//   crossings   one uniform grid per layout (cell side 2^k_l, cells numbered
//               from cbase[l]), so the DDA count, scan, scatter and per-cell
//               pair kernel cover all layouts in single launches; the pair
//               kernel is persistent (one block per SM slot, each warp a
//               contiguous run of work items) and writes one partial per work
//               item, reduced per layout in a fixed order.  Pairs of two
//               long segments (spanning more than two major lines of their
//               layout's grid) skip the grid: every layout's long segments
//               are listed contiguously and one persistent kernel runs the
//               all-pairs tiles of all those lists;
//   occlusion   one grid per layout with cells of side >= d;
//   min angle, edge length variation: one block per layout.
// The cell size k_l of every layout comes from the cost model of the single
// layout (grid_cost: records, short-involved candidate pairs, cells and
// long-long pairs, from the layout's segment length histogram), shifted by a
// global offset that an autotuner picks
// by timing the crossing pipeline at creation (cached in the file named by
// GR_TUNE_CACHE, when set).  The whole evaluation is captured once into a
// CUDA graph and replayed; every kernel reads the sizes it needs from device
// memory and checks them against the buffers, so a replay after coordinates
// changed either fits or raises an overflow bit, on which the host re-plans.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "allpairs_common.cuh"
#include "grid_common.cuh"

using namespace gr;

namespace {

constexpr int BP_WARPS = 8;

struct ItemPart {
    uint32_t proper, touching, collinear, pad;
    uint64_t dev;
};

int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Gather + validation for packed layouts: edge e of layout l (found from
// e_off) has layout-local vertex ids; they become global ids v_off[l] + id.
__global__ void __launch_bounds__(256) k_batch_gather(const int2 *__restrict__ xy, const int64_t *__restrict__ v_off,
                                                      const int2 *__restrict__ edges, const int64_t *__restrict__ e_off,
                                                      int64_t L, int64_t E, SegRec *__restrict__ seg,
                                                      int32_t *__restrict__ seg_eid, uint32_t *__restrict__ seg_theta,
                                                      uint32_t *__restrict__ seg_layout, int64_t *__restrict__ len2,
                                                      DevAcc *acc) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < E; base += stride) {
        const int64_t e = base + threadIdx.x;
        bool keep = false;
        SegRec r = make_uint4(0, 0, 0, 0);
        uint32_t l = 0;
        if (e < E) {
            l = (uint32_t)find_segment(e_off, L, e);
            const int64_t v0 = v_off[l], Vl = v_off[l + 1] - v0;
            const int2 ed = edges[e];
            int64_t l2 = 0;
            if (ed.x < 0 || ed.y < 0 || ed.x >= Vl || ed.y >= Vl || ed.x == ed.y) {
                atomicOr(&acc->status, ST_BAD_ID);
            } else {
                const int64_t ga = v0 + ed.x, gb = v0 + ed.y;
                const int2 a = xy[ga], b = xy[gb];
                if ((unsigned)a.x >= 65536u || (unsigned)a.y >= 65536u || (unsigned)b.x >= 65536u ||
                    (unsigned)b.y >= 65536u) {
                    atomicOr(&acc->status, ST_BAD_COORD);
                } else {
                    const int64_t dx = b.x - a.x, dy = b.y - a.y;
                    l2 = dx * dx + dy * dy;
                    if (l2 != 0) {
                        keep = true;
                        r = make_uint4(uint32_t(a.x) | (uint32_t(a.y) << 16), uint32_t(b.x) | (uint32_t(b.y) << 16),
                                       (uint32_t)ga, (uint32_t)gb);
                    }
                }
            }
            len2[e] = l2;
        }
        const unsigned mk = __ballot_sync(0xffffffffu, keep);
        uint32_t slot = 0;
        if (lane == 0 && mk) slot = atomicAdd(&acc->n_seg, (uint32_t)__popc(mk));
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (keep) {
            const uint32_t pos = slot + __popc(mk & lanemask_lt());
            seg[pos] = r;
            seg_eid[pos] = (int32_t)e;
            seg_theta[pos] = line_direction(px(r.y) - px(r.x), py(r.y) - py(r.x));
            seg_layout[pos] = l;
        }
    }
}

// Per-layout segment counts and total L1 length, and both by major-axis
// length class [2^b, 2^(b+1)) (hn, hl1: 16 per layout), for the plan.
__global__ void __launch_bounds__(256) k_batch_stats(const SegRec *__restrict__ seg,
                                                     const uint32_t *__restrict__ seg_layout,
                                                     const DevAcc *__restrict__ acc, unsigned long long *nseg,
                                                     unsigned long long *l1, uint32_t *hn, unsigned long long *hl1) {
    const int64_t n = acc->n_seg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const SegRec r = seg[i];
        const uint32_t l = seg_layout[i];
        const int dx = abs(px(r.y) - px(r.x)), dy = abs(py(r.y) - py(r.x));
        const int b = 31 - __clz(max(dx, dy));
        atomicAdd(&nseg[l], 1ull);
        atomicAdd(&l1[l], (unsigned long long)(dx + dy));
        atomicAdd(&hn[16 * (uint64_t)l + b], 1u);
        atomicAdd(&hl1[16 * (uint64_t)l + b], (unsigned long long)(dx + dy));
    }
}

// a2 over all layouts: segment s walks layout l's grid (k_l, cells from
// cbase[l]); counts per cell (all records, long ones) and long segments per
// layout (warp-aggregated over lanes of the same layout).
__global__ void __launch_bounds__(256) k_batch_grid_count(const SegRec *__restrict__ seg,
                                                          const uint32_t *__restrict__ seg_layout,
                                                          const DevAcc *__restrict__ acc, const int32_t *__restrict__ kl,
                                                          const int32_t *__restrict__ split_l,
                                                          const uint32_t *__restrict__ cbase,
                                                          uint32_t *__restrict__ cell_cnt, uint32_t *__restrict__ cell_nl,
                                                          uint32_t *__restrict__ nlong) {
    const int64_t n = acc->n_seg;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const SegRec r = ok ? seg[i] : make_uint4(0, 0, 0, 0);
        const uint32_t l = ok ? seg_layout[i] : 0u;
        const int k = ok ? kl[l] : 16;
        const uint32_t cb = ok ? cbase[l] : 0u;
        const bool split = ok && split_l[l] != 0;
        const bool lng = split && is_long_seg(r, k);
        const unsigned ml = __ballot_sync(0xffffffffu, lng);
        if (lng) {
            const unsigned same = __match_any_sync(ml, l);
            if (lane == __ffs(same) - 1) atomicAdd(&nlong[l], (uint32_t)__popc(same));
        }
        warp_for_each_cell(r, 0, 0u, ok, k, cb, split,
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

// All-pairs tiles of every layout's long-segment list (from the scanned
// list offsets long_off): T_l (T_l + 1) / 2 with T_l = ceil(n_l / AS_ROWS)
// (the small tiles: most lists are short).
__global__ void __launch_bounds__(256) k_batch_long_tiles(const uint32_t *__restrict__ long_off, int64_t L,
                                                          uint32_t *__restrict__ tile_cnt) {
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t nl = long_off[l + 1] - long_off[l];
        const uint64_t T = (nl + AS_ROWS - 1) / AS_ROWS;
        tile_cnt[l] = nl < 2 ? 0u : (uint32_t)(T * (T + 1) / 2);
    }
}

// Work items per cell (tile pairs), and the candidate pairs of each layout.
// (Tile pairs with a short row tile, as in the single-layout grid.)
__global__ void __launch_bounds__(256) k_batch_cell_items(const uint32_t *__restrict__ cell_off,
                                                          const uint32_t *__restrict__ cell_nl, uint32_t C,
                                                          const uint32_t *__restrict__ cbase, int64_t L, int tile,
                                                          uint32_t *__restrict__ item_cnt,
                                                          unsigned long long *work, DevAcc *acc) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const uint64_t n = cell_off[c + 1] - cell_off[c];
        const uint64_t ns = n - cell_nl[c];
        bool tiles_over;
        const uint64_t items = tile == 16 ? cell_item_count<16>(n, ns, &tiles_over)
                                          : cell_item_count<32>(n, ns, &tiles_over);
        if (items > 0x7fffffffull || tiles_over) atomicOr(&acc->grid_flags, GF_ITEMS_OVERFLOW);
        item_cnt[c] = (uint32_t)min(items, (uint64_t)0x7fffffffull);
        if (items > 0) {
            const int64_t l = find_segment_u32(cbase, L, c);
            atomicAdd(&work[l], (unsigned long long)(ns * (ns - 1) / 2 + ns * (n - ns)));
        }
    }
}

// Descriptor of every work item: {record offset, records of the cell,
// layout, ti << 16 | tj} and {local cell, k, short records, 0}.
__global__ void __launch_bounds__(256) k_batch_item_descs(const uint32_t *__restrict__ item_off,
                                                          const uint32_t *__restrict__ cell_off,
                                                          const uint32_t *__restrict__ cell_nl, uint32_t C,
                                                          const uint32_t *__restrict__ cbase, int64_t L,
                                                          const int32_t *__restrict__ kl, int tile, uint64_t cap,
                                                          uint4 *__restrict__ desc, DevAcc *acc) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        uint32_t q = item_off[c];
        const uint32_t e = item_off[c + 1];
        if (q == e) continue;
        if (e > cap) {
            atomicOr(&acc->eval_status, ST_OVERFLOW);
            continue;
        }
        const int64_t l = find_segment_u32(cbase, L, c);
        const uint32_t base = cell_off[c], n = cell_off[c + 1] - base, ns = n - cell_nl[c];
        const uint4 hi = make_uint4(c - cbase[l], (uint32_t)kl[l], ns, 0u);
        auto emit = [&](uint32_t i, uint32_t word) {
            desc[2 * (uint64_t)i] = make_uint4(base, n, (uint32_t)l, word);
            desc[2 * (uint64_t)i + 1] = hi;
        };
        if (tile == 16) cell_item_words<16>(n, ns, q, e, emit);
        else cell_item_words<32>(n, ns, q, e, emit);
    }
}

// a4 over all layouts: short records from each cell's start, long ones from
// its end (one 64-bit counter per cell); every long segment is also copied
// to its layout's long list.
__global__ void __launch_bounds__(256) k_batch_grid_fill(const SegRec *__restrict__ seg,
                                                         const int32_t *__restrict__ seg_eid,
                                                         const uint32_t *__restrict__ seg_theta,
                                                         const uint32_t *__restrict__ seg_layout,
                                                         const DevAcc *__restrict__ acc, const int32_t *__restrict__ kl,
                                                         const int32_t *__restrict__ split_l,
                                                         const uint32_t *__restrict__ cbase,
                                                         const uint32_t *__restrict__ cell_off,
                                                         unsigned long long *__restrict__ cell_fill, uint64_t cap,
                                                         GridRec *__restrict__ rec,
                                                         const uint32_t *__restrict__ long_off,
                                                         uint32_t *__restrict__ long_fill,
                                                         SegRec *__restrict__ seg_long,
                                                         uint32_t *__restrict__ theta_long, uint32_t *status) {
    const int64_t n = acc->n_seg;
    if (acc->records > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_OVERFLOW);
        return;
    }
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const SegRec r = ok ? seg[i] : make_uint4(0, 0, 0, 0);
        const int32_t eid = ok ? seg_eid[i] : 0;
        const uint32_t th = ok ? seg_theta[i] : 0u;
        const uint32_t l = ok ? seg_layout[i] : 0u;
        const int k = ok ? kl[l] : 16;
        const uint32_t cb = ok ? cbase[l] : 0u;
        const bool split = ok && split_l[l] != 0;
        if (split && is_long_seg(r, k)) {
            const uint32_t pos = long_off[l] + atomicAdd(&long_fill[l], 1u);
            seg_long[pos] = r;
            theta_long[pos] = th;
        }
        warp_for_each_cell(r, eid, th, ok, k, cb, split,
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

// a6 over all layouts: persistent; warp w takes the contiguous run of items
// [w * chunk, (w + 1) * chunk), T = 32 one item at a time, T = 16 two at a
// time (one per half-warp), and writes one partial per item.  Does nothing
// when the records or work items of this evaluation outgrew their buffers
// (the scatter and the descriptors were not written; the host re-plans on the
// overflow bit).
template <int T>
__global__ void __launch_bounds__(BP_WARPS * 32, 4) k_batch_grid_pairs(const GridRec *__restrict__ rec,
                                                                       const uint4 *__restrict__ desc,
                                                                       const uint32_t *__restrict__ n_items_p,
                                                                       const DevAcc *__restrict__ acc, uint64_t rec_cap,
                                                                       uint64_t cap, uint32_t ideal,
                                                                       ItemPart *__restrict__ part) {
    constexpr int GROUPS = 32 / T;
    __shared__ GSeg cs[BP_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, grp = lane / T, loc = lane & (T - 1);
    if (acc->records > rec_cap || (uint64_t)*n_items_p > cap) return;
    const uint64_t n_items = *n_items_p;
    const uint64_t warps = (uint64_t)gridDim.x * BP_WARPS;
    const uint64_t chunk = (n_items + warps - 1) / warps;
    const uint64_t w = (uint64_t)blockIdx.x * BP_WARPS + wid;
    const uint64_t i0 = w * chunk, i1 = min(n_items, i0 + chunk);
    for (uint64_t it0 = i0; it0 < i1; it0 += GROUPS) {
        const uint64_t it = it0 + grp;
        const bool has = it < i1;
        uint4 d0 = make_uint4(0, 0, 0, 0), d1 = make_uint4(0, 0, 0, 0);
        if (has) {
            d0 = desc[2 * it];
            d1 = desc[2 * it + 1];
        }
        const int k = has ? (int)d1.y : 16, G = 65536 >> k;
        const int cell = (int)d1.x;
        ItemTiles tl = has ? item_tiles<T>(d0.y, d1.z, d0.w) : ItemTiles{0, 0, 0, 0, false};
        PairCounts pc;
        grid_item<false, T>(rec + d0.x, tl, (cell % G) << k, (cell / G) << k, k, cs[wid] + grp * T, ideal, pc,
                            PerEdge{});
        // sums over this item's T lanes
        uint32_t p = pc.proper, t = pc.touching, c = pc.collinear;
        uint64_t dv = pc.dev;
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            t += __shfl_xor_sync(0xffffffffu, t, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
            dv += __shfl_xor_sync(0xffffffffu, dv, o);
        }
        if (loc == 0 && has) {
            ItemPart ip;
            ip.proper = p; ip.touching = t; ip.collinear = c; ip.pad = 0; ip.dev = dv;
            part[it] = ip;
        }
    }
}

// The all-pairs tiles of every layout's long list (persistent, one tile per
// block at a time): tile t belongs to the layout l with tile_off[l] <= t <
// tile_off[l + 1]; its tallies are added to ll[4 l ..] (proper, touching,
// collinear, deviation sum; integers, so the order does not matter).  Does
// nothing when the records outgrew their buffer (the lists were not written).
__global__ void __launch_bounds__(AS_THREADS) k_batch_long_pairs(const SegRec *__restrict__ seg_long,
                                                                 const uint32_t *__restrict__ theta_long,
                                                                 const uint32_t *__restrict__ long_off,
                                                                 const uint32_t *__restrict__ tile_off, int64_t L,
                                                                 const DevAcc *__restrict__ acc, uint64_t rec_cap,
                                                                 uint32_t ideal, unsigned long long *__restrict__ ll) {
    __shared__ AllPairsSmem<AS_ROWS> sm;
    __shared__ uint64_t sh[32];
    if (acc->records > rec_cap) return;
    const uint32_t tiles = tile_off[L];
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t l = find_segment_u32(tile_off, L, t);
        const uint32_t o = long_off[l];
        int bi, bj;
        decode_tile((int64_t)(t - tile_off[l]), bi, bj);
        PairCounts pc;
        allpairs_tile<AS_THREADS, AS_RPT>(seg_long + o, theta_long + o, (int)(long_off[l + 1] - o), bi, bj, ideal,
                                          sm, pc);
        const uint64_t p = block_sum<uint64_t>(pc.proper, sh);
        const uint64_t q = block_sum<uint64_t>(pc.touching, sh);
        const uint64_t c = block_sum<uint64_t>(pc.collinear, sh);
        const uint64_t d = block_sum<uint64_t>(pc.dev, sh);
        if (threadIdx.x == 0) {
            if (p) atomicAdd(&ll[4 * l + 0], (unsigned long long)p);
            if (q) atomicAdd(&ll[4 * l + 1], (unsigned long long)q);
            if (c) atomicAdd(&ll[4 * l + 2], (unsigned long long)c);
            if (d) atomicAdd(&ll[4 * l + 3], (unsigned long long)d);
        }
    }
}

// Per layout: the crossing partials of its items in a fixed order and its
// long-long tallies, plus the occlusion count, into the result; metrics not
// evaluated get their defaults.
__global__ void __launch_bounds__(256) k_batch_finalize(const ItemPart *__restrict__ part,
                                                        const uint32_t *__restrict__ item_off,
                                                        const uint32_t *__restrict__ cell_off,
                                                        const uint32_t *__restrict__ cbase, const int32_t *__restrict__ kl,
                                                        const unsigned long long *__restrict__ work,
                                                        const unsigned long long *__restrict__ ll,
                                                        const uint32_t *__restrict__ long_off,
                                                        const uint64_t *__restrict__ occl, int64_t L, uint32_t metrics,
                                                        double ideal, int64_t d, uint64_t cap,
                                                        const DevAcc *__restrict__ acc,
                                                        gr_result *__restrict__ res) {
    __shared__ uint64_t sh[32];
    // a failed evaluation (invalid input, outgrown buffers) is marked by metrics = 0 in every result
    const bool failed = (acc->status | acc->eval_status) != 0 || (acc->grid_flags & GF_ITEMS_OVERFLOW) != 0;
    for (int64_t l = blockIdx.x; l < L; l += gridDim.x) {
        uint64_t p = 0, t = 0, c = 0, dv = 0;
        if (metrics & GR_METRIC_CROSSINGS) {
            const uint64_t a = min((uint64_t)item_off[cbase[l]], cap), b = min((uint64_t)item_off[cbase[l + 1]], cap);
            for (uint64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
                const ItemPart q = part[i];
                p += q.proper; t += q.touching; c += q.collinear; dv += q.dev;
            }
        }
        p = block_sum<uint64_t>(p, sh);
        t = block_sum<uint64_t>(t, sh);
        c = block_sum<uint64_t>(c, sh);
        dv = block_sum<uint64_t>(dv, sh);
        if (threadIdx.x != 0) continue;
        gr_result &r = res[l];
        r.metrics = failed ? 0u : metrics;
        if (metrics & GR_METRIC_CROSSINGS) {
            p += ll[4 * l + 0];
            t += ll[4 * l + 1];
            c += ll[4 * l + 2];
            dv += ll[4 * l + 3];
            const uint64_t nl = long_off[l + 1] - long_off[l];
            r.crossing_path = GR_PATH_GRID;
            r.cell_log2 = kl[l];
            const uint64_t ec = p + t;
            r.crossing.c.crossings = (int64_t)ec;
            r.crossing.c.proper = (int64_t)p;
            r.crossing.c.touching = (int64_t)t;
            r.crossing.c.collinear_overlaps = (int64_t)c;
            r.crossing.c.pairs_tested = (int64_t)(work[l] + nl * (nl - (nl > 0)) / 2);
            const double dev = (double)dv * kAngleUnit;
            r.crossing.angle_dev_sum = dev;
            r.crossing.ideal_rad = ideal;
            r.crossing.E_ca = ec > 0 ? 1.0 - dev / (ideal * (double)ec) : 1.0;
            r.grid_records = (int64_t)(cell_off[cbase[l + 1]] - cell_off[cbase[l]]);
        } else {
            const int64_t z = r.crossing.c.zero_length_edges;
            memset(&r.crossing, 0, sizeof(r.crossing));
            r.crossing.c.zero_length_edges = z;
            r.crossing.E_ca = 1.0;
            r.crossing_path = 0;
            r.cell_log2 = 0;
            r.grid_records = 0;
        }
        if (metrics & GR_METRIC_OCCLUSION) {
            r.occlusion_pairs = (int64_t)occl[l];
            r.occlusion_path = GR_PATH_GRID;
        } else {
            r.occlusion_pairs = 0;
            r.occlusion_path = 0;
        }
        r.occlusion_d = d;
        if (!(metrics & GR_METRIC_MIN_ANGLE)) {
            r.min_angle.M_a = 1.0;
            r.min_angle.sum_d = 0.0;
            r.min_angle.n_vertices_counted = 0;
        }
        if (!(metrics & GR_METRIC_EDGE_LENGTH)) r.M_l = 0.0;
    }
}

thread_local std::string g_batch_err;

}  // namespace

struct gr_batch {
    int64_t L = 0, V = 0, E = 0;
    cudaStream_t stream = nullptr;  // the caller's stream (may be the legacy default stream)
    cudaStream_t cap = nullptr;     // the batch's own stream: evaluations are replayed here
    cudaStream_t cs = nullptr;      // and captured here (never joined to a caller's stream)
    cudaEvent_t ev_in2 = nullptr, ev_out = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_in = nullptr, ev_fork = nullptr, ev_join = nullptr;
    int64_t graph_kernels = 0;      // kernels per replay (for the launch counter)
    gr_options opt{};
    Buffers b;
    uint32_t *seg_layout = nullptr;
    int64_t *d_voff = nullptr, *d_eoff = nullptr;
    std::vector<int64_t> v_off, e_off;
    gr_result *d_res = nullptr, *h_res = nullptr;
    DevAcc *h_acc = nullptr;
    // crossing plan
    std::vector<uint64_t> nseg_l, l1_l;
    std::vector<int32_t> k_l, split_l;
    int32_t *d_k = nullptr;
    int32_t *d_split = nullptr;  // [L] long-long pairs on the all-pairs tiles
    uint32_t *d_cbase = nullptr;
    uint32_t C = 0, C_cap = 0;
    int delta = 0;
    int tile = 32;                  // segments per tile of the pair kernel's items (16 or 32)
    unsigned long long *d_nseg = nullptr, *d_l1 = nullptr, *d_work = nullptr;
    uint32_t *d_hn = nullptr;            // [16 L] segments by major-length class
    unsigned long long *d_hl1 = nullptr; // [16 L] their L1 length
    std::vector<uint32_t> hn_l;
    std::vector<uint64_t> hl1_l;
    uint32_t *cell_off = nullptr, *cell_nl = nullptr, *item_off = nullptr;
    unsigned long long *cell_fill = nullptr;
    // long segments: per-layout lists and their all-pairs tiles
    uint32_t *long_off = nullptr;   // [L + 1] counts, then offsets
    uint32_t *long_fill = nullptr;  // [L]
    uint32_t *tile_off = nullptr;   // [L + 1] tiles, then offsets
    SegRec *seg_long = nullptr;     // [E]
    uint32_t *theta_long = nullptr; // [E]
    unsigned long long *d_ll = nullptr;  // [4 L] long-long tallies
    GridRec *rec = nullptr;
    uint64_t rec_cap = 0;
    uint4 *desc = nullptr;
    ItemPart *parts = nullptr;
    uint64_t items_cap = 0;
    // occlusion plan (per d)
    int64_t plan_d = -1;
    int32_t *d_ko = nullptr;
    uint32_t *d_obase = nullptr;
    uint32_t OC = 0, OC_cap = 0;
    uint32_t *ocell_off = nullptr, *ocell_fill = nullptr, *opts = nullptr, *olay = nullptr;
    uint64_t *occl = nullptr;
    // captured evaluation
    cudaGraphExec_t exec = nullptr;
    uint32_t g_metrics = 0, g_ideal = 0;
    int64_t g_d = -1;
};

namespace {

gr_status bfail(gr_status st, const std::string &msg) {
    set_last_error(msg.c_str());
    return st;
}

gr_status bcuda(cudaError_t e, const char *what) {
    cudaGetLastError();
    return bfail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define B_CU(call)                                        \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return bcuda(e_, #call);   \
    } while (0)

template <typename T>
gr_status balloc(T **p, size_t n) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return bcuda(e, "cudaMalloc");
    }
    return GR_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

BatchView view(const gr_batch *B) {
    BatchView v;
    v.L = B->L;
    v.v_off = B->d_voff;
    v.e_off = B->d_eoff;
    v.res = B->d_res;
    return v;
}

void drop_graph(gr_batch *B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
}

void free_batch(gr_batch *B) {
    if (!B) return;
    drop_graph(B);
    Buffers &b = B->b;
    void *ptrs[] = {b.xy, b.edges, b.seg, b.seg_eid, b.seg_theta, b.len2, b.acc, b.deg, b.deg_fill, b.dirs,
                    b.scan_tmp, b.scan_tmp_side, B->seg_layout, B->d_voff, B->d_eoff, B->d_res, B->d_k, B->d_split, B->d_cbase,
                    B->d_nseg, B->d_l1, B->d_work, B->d_hn, B->d_hl1, B->cell_off, B->cell_nl, B->item_off,
                    B->cell_fill, B->long_off, B->long_fill, B->tile_off, B->seg_long, B->theta_long, B->d_ll,
                    B->rec, B->desc, B->parts, B->d_ko, B->d_obase, B->ocell_off, B->ocell_fill, B->opts, B->olay,
                    B->occl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (B->h_res) cudaFreeHost(B->h_res);
    if (B->h_acc) cudaFreeHost(B->h_acc);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->ev_join) cudaEventDestroy(B->ev_join);
    if (B->side) cudaStreamDestroy(B->side);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->cs) cudaStreamDestroy(B->cs);
    if (B->ev_in2) cudaEventDestroy(B->ev_in2);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    delete B;
}

// Cell size of each layout: the k minimising grid_cost (the single-layout
// model; ties go to the coarser grid), shifted by the autotuned offset
// `delta`; and whether its long-long pairs go to the all-pairs tiles (the
// better form at that cell size; one launch serves every layout, so no fixed
// cost per layout).
void plan_cells(gr_batch *B) {
    B->k_l.assign(B->L, 16);
    B->split_l.assign(B->L, 0);
    uint64_t C = 0;
    for (int64_t l = 0; l < B->L; ++l) {
        const double n = (double)B->nseg_l[l], l1 = (double)B->l1_l[l];
        const uint32_t *hn = &B->hn_l[16 * l];
        const uint64_t *hl = &B->hl1_l[16 * l];
        int best = 16;
        double bestc = 1e300;
        for (int k = 16; k >= 6; --k)
            for (bool split : {false, true}) {
                const double cost = grid_cost(n, l1, hn, hl, k, split) - (split ? kSplitCost : 0.0);
                if (cost < bestc) { bestc = cost; best = k; }
            }
        B->k_l[l] = std::min(16, std::max(6, best + B->delta));
        const int k = B->k_l[l];
        B->split_l[l] = grid_cost(n, l1, hn, hl, k, true) - kSplitCost < grid_cost(n, l1, hn, hl, k, false) ? 1 : 0;
        if (B->opt.long_pairs == GR_LONG_ALLPAIRS) B->split_l[l] = 1;
        else if (B->opt.long_pairs == GR_LONG_GRID) B->split_l[l] = 0;
        C += (uint64_t)(65536 >> B->k_l[l]) * (uint64_t)(65536 >> B->k_l[l]);
    }
    // keep the scan within its 2^26-entry limit: coarsen the finest grids
    while (C > (uint64_t(1) << 26)) {
        int64_t arg = 0;
        for (int64_t l = 1; l < B->L; ++l)
            if (B->k_l[l] < B->k_l[arg]) arg = l;
        const uint64_t before = (uint64_t)(65536 >> B->k_l[arg]) * (uint64_t)(65536 >> B->k_l[arg]);
        B->k_l[arg] += 1;  // (split stays a valid choice: it only moves pairs between kernels)
        C -= before - (uint64_t)(65536 >> B->k_l[arg]) * (uint64_t)(65536 >> B->k_l[arg]);
    }
    B->C = (uint32_t)C;
}

gr_status upload_cells(gr_batch *B) {
    std::vector<uint32_t> cb(B->L + 1, 0);
    for (int64_t l = 0; l < B->L; ++l) cb[l + 1] = cb[l] + (uint32_t)((65536 >> B->k_l[l]) * (65536 >> B->k_l[l]));
    B_CU(cudaMemcpy(B->d_k, B->k_l.data(), sizeof(int32_t) * B->L, cudaMemcpyHostToDevice));
    B_CU(cudaMemcpy(B->d_split, B->split_l.data(), sizeof(int32_t) * B->L, cudaMemcpyHostToDevice));
    B_CU(cudaMemcpy(B->d_cbase, cb.data(), sizeof(uint32_t) * (B->L + 1), cudaMemcpyHostToDevice));
    gr_status st;
    if (B->C_cap < B->C) {
        if ((st = balloc(&B->cell_off, (size_t)B->C + 1)) != GR_OK) return st;
        if ((st = balloc(&B->cell_nl, (size_t)B->C)) != GR_OK) return st;
        if ((st = balloc(&B->item_off, (size_t)B->C + 1)) != GR_OK) return st;
        if ((st = balloc(&B->cell_fill, (size_t)B->C)) != GR_OK) return st;
        B->C_cap = B->C;
    }
    drop_graph(B);
    return GR_OK;
}

// The crossing binning (a2, a3) of all layouts.
void enqueue_cross_count(gr_batch *B, cudaStream_t s) {
    Buffers &b = B->b;
    cudaMemsetAsync(B->cell_off, 0, sizeof(uint32_t) * ((size_t)B->C + 1), s);
    cudaMemsetAsync(B->cell_nl, 0, sizeof(uint32_t) * (size_t)B->C, s);
    cudaMemsetAsync(B->long_off, 0, sizeof(uint32_t) * ((size_t)B->L + 1), s);
    cudaMemsetAsync(B->d_work, 0, sizeof(unsigned long long) * B->L, s);
    count_launches(4);
    k_batch_grid_count<<<grid_for(B->E, 256, 152 * 16), 256, 0, s>>>(b.seg, B->seg_layout, b.acc, B->d_k,
                                                                     B->d_split, B->d_cbase, B->cell_off,
                                                                     B->cell_nl, B->long_off);
    launch_scan_u32(B->cell_off, B->cell_off, B->C, b.scan_tmp, &b.acc->records, &b.acc->eval_status, s);
    k_batch_cell_items<<<grid_for(B->C, 256, 152 * 8), 256, 0, s>>>(B->cell_off, B->cell_nl, B->C, B->d_cbase, B->L,
                                                                    B->tile, B->item_off, B->d_work, b.acc);
    launch_scan_u32(B->item_off, B->item_off, B->C, b.scan_tmp, &b.acc->grid_items, &b.acc->eval_status, s);
    k_batch_item_descs<<<grid_for(B->C, 256, 152 * 8), 256, 0, s>>>(B->item_off, B->cell_off, B->cell_nl, B->C,
                                                                    B->d_cbase, B->L, B->d_k, B->tile, B->items_cap,
                                                                    B->desc, b.acc);
    launch_scan_u32(B->long_off, B->long_off, B->L, b.scan_tmp, &b.acc->scan_sink, &b.acc->eval_status, s);
    k_batch_long_tiles<<<grid_for(B->L, 256, 152 * 8), 256, 0, s>>>(B->long_off, B->L, B->tile_off);
    launch_scan_u32(B->tile_off, B->tile_off, B->L, b.scan_tmp, &b.acc->scan_sink, &b.acc->eval_status, s);
}

// Scatter (a4) and the per-cell pair kernel (a6) of all layouts.
void enqueue_cross_pairs(gr_batch *B, uint32_t ideal_u, cudaStream_t s) {
    Buffers &b = B->b;
    cudaMemsetAsync(B->cell_fill, 0, sizeof(unsigned long long) * B->C, s);
    cudaMemsetAsync(B->long_fill, 0, sizeof(uint32_t) * B->L, s);
    cudaMemsetAsync(B->d_ll, 0, sizeof(unsigned long long) * 4 * B->L, s);
    count_launches(3);
    k_batch_grid_fill<<<grid_for(B->E, 256, 152 * 16), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, B->seg_layout,
                                                                    b.acc, B->d_k, B->d_split, B->d_cbase,
                                                                    B->cell_off, B->cell_fill, B->rec_cap, B->rec,
                                                                    B->long_off,
                                                                    B->long_fill, B->seg_long, B->theta_long,
                                                                    &b.acc->eval_status);
    if (B->tile == 16)
        k_batch_grid_pairs<16><<<152 * 4, BP_WARPS * 32, 0, s>>>(B->rec, B->desc, B->item_off + B->C, b.acc,
                                                                 B->rec_cap, B->items_cap, ideal_u, B->parts);
    else
        k_batch_grid_pairs<32><<<152 * 4, BP_WARPS * 32, 0, s>>>(B->rec, B->desc, B->item_off + B->C, b.acc,
                                                                 B->rec_cap, B->items_cap, ideal_u, B->parts);
    k_batch_long_pairs<<<152 * 8, AS_THREADS, 0, s>>>(B->seg_long, B->theta_long, B->long_off, B->tile_off, B->L,
                                                      b.acc, B->rec_cap, ideal_u, B->d_ll);
}

// Grows the record and work-item buffers to the current sizes (read back).
gr_status size_cross_buffers(gr_batch *B, cudaStream_t s) {
    B->items_cap = 0;  // descriptors are not written while sizing
    enqueue_cross_count(B, s);
    B_CU(cudaGetLastError());
    B_CU(cudaMemcpyAsync(B->h_acc, B->b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
    B_CU(cudaStreamSynchronize(s));
    const uint64_t R = B->h_acc->records, items = B->h_acc->grid_items;
    if (B->h_acc->grid_flags & GF_ITEMS_OVERFLOW)
        return bfail(GR_ENOTSUP, "a layout has a grid cell with more than 2^31 tile pairs");
    gr_status st;
    if (B->rec_cap < R || !B->rec) {
        const uint64_t cap = R + R / 4 + 4096;
        if ((st = balloc(&B->rec, (size_t)cap)) != GR_OK) return st;
        B->rec_cap = cap;
    }
    const uint64_t icap = items + items / 4 + 4096;
    if ((st = balloc(&B->desc, 2 * (size_t)icap)) != GR_OK) return st;
    if ((st = balloc(&B->parts, (size_t)icap)) != GR_OK) return st;
    B->items_cap = icap;
    B_CU(cudaMemsetAsync((char *)B->b.acc + offsetof(DevAcc, eval_status), 0,
                         sizeof(DevAcc) - offsetof(DevAcc, eval_status), s));
    drop_graph(B);
    return GR_OK;
}

// Occlusion grids for diameter d: cell side 2^ko_l >= d and about V_l / 2 cells.
gr_status plan_occlusion(gr_batch *B, int64_t d) {
    if (B->plan_d == d) return GR_OK;
    std::vector<int32_t> ko(B->L);
    std::vector<uint32_t> ob(B->L + 1, 0);
    int kd = 6;
    while (kd < 16 && (int64_t(1) << kd) < d) ++kd;
    uint64_t OC = 0;
    for (int64_t l = 0; l < B->L; ++l) {
        const double Vl = (double)(B->v_off[l + 1] - B->v_off[l]);
        int kv = 16;
        if (Vl >= 2) kv = (int)std::lround(std::log2(65536.0 / std::sqrt(Vl / 2.0)));
        ko[l] = std::min(16, std::max(kd, std::max(6, kv)));
        OC += (uint64_t)(65536 >> ko[l]) * (uint64_t)(65536 >> ko[l]);
        ob[l + 1] = (uint32_t)OC;
    }
    if (OC > (uint64_t(1) << 26)) return bfail(GR_ENOTSUP, "occlusion grids exceed 2^26 cells");
    gr_status st;
    B_CU(cudaMemcpy(B->d_ko, ko.data(), sizeof(int32_t) * B->L, cudaMemcpyHostToDevice));
    B_CU(cudaMemcpy(B->d_obase, ob.data(), sizeof(uint32_t) * (B->L + 1), cudaMemcpyHostToDevice));
    if (B->OC_cap < OC) {
        if ((st = balloc(&B->ocell_off, (size_t)OC + 1)) != GR_OK) return st;
        if ((st = balloc(&B->ocell_fill, (size_t)OC)) != GR_OK) return st;
        B->OC_cap = (uint32_t)OC;
    }
    B->OC = (uint32_t)OC;
    B->plan_d = d;
    drop_graph(B);
    return GR_OK;
}

// One evaluation, stream-ordered on s (what the CUDA graph captures).
void enqueue_evaluate(gr_batch *B, cudaStream_t s, uint32_t metrics, double ideal, uint32_t ideal_u, int64_t d) {
    cudaStream_t t = B->side;
    Buffers &b = B->b;
    const BatchView bv = view(B);
    cudaMemsetAsync((char *)b.acc + offsetof(DevAcc, eval_status), 0, sizeof(DevAcc) - offsetof(DevAcc, eval_status), s);
    cudaEventRecord(B->ev_fork, s);
    cudaStreamWaitEvent(t, B->ev_fork, 0);
    if (metrics & GR_METRIC_EDGE_LENGTH) launch_batch_elv(b, bv, t);
    if (metrics & GR_METRIC_MIN_ANGLE) launch_batch_min_angle(b, bv, B->V, B->E, t);
    if (metrics & GR_METRIC_OCCLUSION)
        launch_batch_occlusion(b, bv, B->V, B->d_ko, B->d_obase, B->OC, B->ocell_off, B->ocell_fill, B->opts, B->olay, d,
                               B->occl, t);
    cudaEventRecord(B->ev_join, t);
    if (metrics & GR_METRIC_CROSSINGS) {
        enqueue_cross_count(B, s);
        enqueue_cross_pairs(B, ideal_u, s);
    }
    cudaStreamWaitEvent(s, B->ev_join, 0);
    count_launches(1);
    k_batch_finalize<<<grid_for(B->L, 1, 152 * 16), 256, 0, s>>>(B->parts, B->item_off, B->cell_off, B->d_cbase, B->d_k,
                                                                 B->d_work, B->d_ll, B->long_off, B->occl, B->L,
                                                                 metrics, ideal, d, B->items_cap, b.acc, B->d_res);
}

gr_status enqueue_inputs(gr_batch *B, const void *xy, const int32_t *edges) {
    cudaStream_t s = B->stream;
    Buffers &b = B->b;
    B_CU(cudaMemsetAsync(b.acc, 0, offsetof(DevAcc, eval_status), s));
    if (B->V > 0) {
        const cudaMemcpyKind k = is_device_ptr(xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        B_CU(cudaMemcpyAsync(b.xy, xy, sizeof(int32_t) * 2 * B->V, k, s));
    }
    if (B->E > 0 && edges) {
        const cudaMemcpyKind k = is_device_ptr(edges) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        B_CU(cudaMemcpyAsync(b.edges, edges, sizeof(int32_t) * 2 * B->E, k, s));
    }
    launch_check_vertices(b.xy, B->V, b, s);
    if (B->E > 0) {
        count_launches(1);
        k_batch_gather<<<grid_for(B->E, 256, 152 * 16), 256, 0, s>>>((const int2 *)b.xy, B->d_voff,
                                                                     (const int2 *)b.edges, B->d_eoff, B->L, B->E, b.seg,
                                                                     b.seg_eid, b.seg_theta, B->seg_layout, b.len2,
                                                                     b.acc);
    }
    B_CU(cudaGetLastError());
    return GR_OK;
}

gr_status status_error(uint32_t st) {
    if (st & ST_BAD_ID) return bfail(GR_EINVAL, "vertex id outside its layout or self-loop in the edge list");
    if (st & ST_BAD_COORD) return bfail(GR_ERANGE, "vertex coordinate outside [0, 65536)");
    if (st & ST_SCAN_OVERFLOW) return bfail(GR_ENOTSUP, "an offset table exceeded 2^32 entries");
    return GR_OK;
}

// Times the crossing pipeline (binning, scatter, pairs) with the current plan.
gr_status time_crossings(gr_batch *B, float *ms) {
    cudaEvent_t a, z;
    B_CU(cudaEventCreate(&a));
    B_CU(cudaEventCreate(&z));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a, B->stream);
        enqueue_cross_count(B, B->stream);
        enqueue_cross_pairs(B, 1u << 30, B->stream);
        cudaEventRecord(z, B->stream);
        cudaError_t e = cudaEventSynchronize(z);
        if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(z);
            return bcuda(e, "autotune");
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, a, z);
        best = std::min(best, t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    *ms = best;
    return GR_OK;
}

// The autotuner's key: layouts, vertices and edges, each rounded to a power
// of two, and the device's SM count.
std::string tune_key(const gr_batch *B) {
    auto lg = [](int64_t x) { int r = 0; while ((int64_t(1) << r) < x) ++r; return r; };
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    char buf[128];
    snprintf(buf, sizeof buf, "batch_tiled_L%d_V%d_E%d_sm%d", lg(B->L), lg(B->V), lg(B->E), sms);
    return buf;
}

// Cache lines: "key offset tile" (a line without the tile means 32).
bool tune_cache_lookup(const std::string &key, int *delta, int *tile) {
    const char *path = getenv("GR_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[256], k[128];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        int v = 0, t = 32;
        const int got = sscanf(line, "%127s %d %d", k, &v, &t);
        if (got >= 2 && key == k && (t == 16 || t == 32)) {
            *delta = v;
            *tile = t;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void tune_cache_store(const std::string &key, int delta, int tile) {
    const char *path = getenv("GR_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), delta, tile);
    fclose(f);
}

// A tile height fixed by the environment (GR_BATCH_TILE = 16 or 32), else 0.
int fixed_tile() {
    const char *v = getenv("GR_BATCH_TILE");
    if (!v) return 0;
    const int t = atoi(v);
    return (t == 16 || t == 32) ? t : 0;
}

gr_status apply_plan(gr_batch *B, int delta, int tile) {
    B->delta = delta;
    B->tile = tile;
    plan_cells(B);
    gr_status st = upload_cells(B);
    return st != GR_OK ? st : size_cross_buffers(B, B->stream);
}

// Picks the global cell-size offset (-1, 0, +1) and the tile height of the
// pair kernel's items (16 or 32 segments: two items per warp or one) with the
// fastest crossing pipeline, or takes them from the tune cache.
gr_status autotune(gr_batch *B) {
    const std::string key = tune_key(B);
    const int ft = fixed_tile();
    int cached = 0, ctile = 32;
    if (tune_cache_lookup(key, &cached, &ctile)) return apply_plan(B, cached, ft ? ft : ctile);
    int best_delta = 0, best_tile = 32;
    float best = 1e30f;
    for (int tile : {32, 16}) {
        if (ft && tile != ft) continue;
        for (int delta : {0, -1, 1}) {
            gr_status st = apply_plan(B, delta, tile);
            if (st != GR_OK) return st;
            float ms = 0.f;
            if ((st = time_crossings(B, &ms)) != GR_OK) return st;
            if (ms < best) {
                best = ms;
                best_delta = delta;
                best_tile = tile;
            }
        }
    }
    gr_status st = apply_plan(B, best_delta, best_tile);
    if (st == GR_OK && !ft) tune_cache_store(key, best_delta, best_tile);
    return st;
}

}  // namespace

extern "C" {

gr_status gr_batch_create(gr_batch **out, int64_t n_layouts, const int64_t *v_off, const int64_t *e_off,
                          const void *xy, gr_coord_type coord_type, const int32_t *edges, const gr_options *opt,
                          gr_stream_t stream) {
    set_last_error("");
    if (!out || !v_off || !e_off) return bfail(GR_EINVAL, "NULL argument");
    if (coord_type != GR_COORD_I32) return bfail(GR_ENOTSUP, "only GR_COORD_I32 batches are supported");
    if (n_layouts < 1 || n_layouts >= (int64_t(1) << 24)) return bfail(GR_EINVAL, "n_layouts must be in [1, 2^24)");
    std::vector<int64_t> vo(n_layouts + 1), eo(n_layouts + 1);
    {
        const cudaMemcpyKind kv = is_device_ptr(v_off) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        const cudaMemcpyKind ke = is_device_ptr(e_off) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        B_CU(cudaMemcpy(vo.data(), v_off, sizeof(int64_t) * (n_layouts + 1), kv));
        B_CU(cudaMemcpy(eo.data(), e_off, sizeof(int64_t) * (n_layouts + 1), ke));
    }
    if (vo[0] != 0 || eo[0] != 0) return bfail(GR_EINVAL, "offsets must start at 0");
    for (int64_t l = 0; l < n_layouts; ++l)
        if (vo[l + 1] < vo[l] || eo[l + 1] < eo[l]) return bfail(GR_EINVAL, "offsets must be non-decreasing");
    const int64_t V = vo[n_layouts], E = eo[n_layouts];
    if (V >= (int64_t(1) << 31) || E >= (int64_t(1) << 31)) return bfail(GR_EINVAL, "total V and E must be < 2^31");
    if ((V > 0 && !xy) || (E > 0 && !edges)) return bfail(GR_EINVAL, "NULL input pointer");
    for (int64_t l = 0; l < n_layouts; ++l)
        if (eo[l + 1] > eo[l] && vo[l + 1] - vo[l] < 2) return bfail(GR_EINVAL, "a layout with edges needs two vertices");

    gr_batch *B = new gr_batch;
    B->L = n_layouts;
    B->V = V;
    B->E = E;
    B->v_off = vo;
    B->e_off = eo;
    B->stream = (cudaStream_t)stream;
    if (opt) B->opt = *opt;
    gr_status st = GR_OK;
    Buffers &b = B->b;
#define B_TRY(x)                                 \
    do {                                         \
        if ((st = (x)) != GR_OK) {               \
            free_batch(B);                       \
            return st;                           \
        }                                        \
    } while (0)
    B_TRY(balloc(&b.xy, 2 * (size_t)V));
    B_TRY(balloc(&b.edges, 2 * (size_t)E));
    B_TRY(balloc(&b.seg, (size_t)E));
    B_TRY(balloc(&b.seg_eid, (size_t)E));
    B_TRY(balloc(&b.seg_theta, (size_t)E));
    B_TRY(balloc(&b.len2, (size_t)E));
    B_TRY(balloc(&b.acc, 1));
    B_TRY(balloc(&b.deg, (size_t)V + 1));
    B_TRY(balloc(&b.deg_fill, (size_t)V));
    B_TRY(balloc(&b.dirs, 2 * (size_t)E));
    B_TRY(balloc(&b.scan_tmp, (size_t)kScanMaxBlocks));
    B_TRY(balloc(&b.scan_tmp_side, (size_t)kScanMaxBlocks));
    B_TRY(balloc(&B->seg_layout, (size_t)E));
    B_TRY(balloc(&B->d_voff, (size_t)n_layouts + 1));
    B_TRY(balloc(&B->d_eoff, (size_t)n_layouts + 1));
    B_TRY(balloc(&B->d_res, (size_t)n_layouts));
    B_TRY(balloc(&B->d_k, (size_t)n_layouts));
    B_TRY(balloc(&B->d_split, (size_t)n_layouts));
    B_TRY(balloc(&B->d_cbase, (size_t)n_layouts + 1));
    B_TRY(balloc(&B->d_nseg, (size_t)n_layouts));
    B_TRY(balloc(&B->d_l1, (size_t)n_layouts));
    B_TRY(balloc(&B->d_work, (size_t)n_layouts));
    B_TRY(balloc(&B->d_hn, 16 * (size_t)n_layouts));
    B_TRY(balloc(&B->d_hl1, 16 * (size_t)n_layouts));
    B_TRY(balloc(&B->long_off, (size_t)n_layouts + 1));
    B_TRY(balloc(&B->long_fill, (size_t)n_layouts));
    B_TRY(balloc(&B->tile_off, (size_t)n_layouts + 1));
    B_TRY(balloc(&B->d_ll, 4 * (size_t)n_layouts));
    B_TRY(balloc(&B->seg_long, (size_t)E));
    B_TRY(balloc(&B->theta_long, (size_t)E));
    B_TRY(balloc(&B->d_ko, (size_t)n_layouts));
    B_TRY(balloc(&B->d_obase, (size_t)n_layouts + 1));
    B_TRY(balloc(&B->opts, (size_t)V));
    B_TRY(balloc(&B->olay, (size_t)V));
    B_TRY(balloc(&B->occl, (size_t)n_layouts));
#define B_CU2(call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            st = bcuda(e_, #call);                    \
            free_batch(B);                            \
            return st;                                \
        }                                             \
    } while (0)
    B_CU2(cudaMallocHost((void **)&B->h_res, sizeof(gr_result) * n_layouts));
    B_CU2(cudaMallocHost((void **)&B->h_acc, sizeof(DevAcc)));
    B_CU2(cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking));
    B_CU2(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    B_CU2(cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking));
    B_CU2(cudaEventCreateWithFlags(&B->ev_in2, cudaEventDisableTiming));
    B_CU2(cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming));
    B_CU2(cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming));
    B_CU2(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
    B_CU2(cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming));
    B_CU2(cudaMemcpy(B->d_voff, vo.data(), sizeof(int64_t) * (n_layouts + 1), cudaMemcpyHostToDevice));
    B_CU2(cudaMemcpy(B->d_eoff, eo.data(), sizeof(int64_t) * (n_layouts + 1), cudaMemcpyHostToDevice));
    B_CU2(cudaMemset(B->d_res, 0, sizeof(gr_result) * n_layouts));
    B_CU2(cudaMemset(b.acc, 0, sizeof(DevAcc)));
    B_CU2(init_min_angle_table(B->stream));
    B_TRY(enqueue_inputs(B, xy, edges));
    // validation and the per-layout statistics of the plan
    B_CU2(cudaMemsetAsync(B->d_nseg, 0, sizeof(unsigned long long) * n_layouts, B->stream));
    B_CU2(cudaMemsetAsync(B->d_l1, 0, sizeof(unsigned long long) * n_layouts, B->stream));
    B_CU2(cudaMemsetAsync(B->d_hn, 0, sizeof(uint32_t) * 16 * n_layouts, B->stream));
    B_CU2(cudaMemsetAsync(B->d_hl1, 0, sizeof(unsigned long long) * 16 * n_layouts, B->stream));
    if (E > 0) {
        count_launches(1);
        k_batch_stats<<<grid_for(E, 256, 152 * 16), 256, 0, B->stream>>>(b.seg, B->seg_layout, b.acc, B->d_nseg,
                                                                         B->d_l1, B->d_hn, B->d_hl1);
    }
    B->nseg_l.assign(n_layouts, 0);
    B->l1_l.assign(n_layouts, 0);
    B->hn_l.assign(16 * n_layouts, 0);
    B->hl1_l.assign(16 * n_layouts, 0);
    B_CU2(cudaMemcpyAsync(B->hn_l.data(), B->d_hn, sizeof(uint32_t) * 16 * n_layouts, cudaMemcpyDeviceToHost,
                          B->stream));
    B_CU2(cudaMemcpyAsync(B->hl1_l.data(), B->d_hl1, sizeof(uint64_t) * 16 * n_layouts, cudaMemcpyDeviceToHost,
                          B->stream));
    B_CU2(cudaMemcpyAsync(B->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, B->stream));
    B_CU2(cudaMemcpyAsync(B->nseg_l.data(), B->d_nseg, sizeof(uint64_t) * n_layouts, cudaMemcpyDeviceToHost, B->stream));
    B_CU2(cudaMemcpyAsync(B->l1_l.data(), B->d_l1, sizeof(uint64_t) * n_layouts, cudaMemcpyDeviceToHost, B->stream));
    B_CU2(cudaStreamSynchronize(B->stream));
    B_TRY(status_error(B->h_acc->status));
    if (B->opt.cell_log2 != 0) {
        // negative values: a fixed offset (the tile height from GR_BATCH_TILE, else 32)
        const int ft = fixed_tile();
        B_TRY(apply_plan(B, B->opt.cell_log2 < 0 ? B->opt.cell_log2 : 0, ft ? ft : 32));
    } else {
        B_TRY(autotune(B));
    }
#undef B_TRY
#undef B_CU2
    *out = B;
    return GR_OK;
}

gr_status gr_batch_update(gr_batch *B, const void *xy, const int32_t *edges) {
    set_last_error("");
    if (!B) return bfail(GR_EINVAL, "batch is NULL");
    if (B->V > 0 && !xy) return bfail(GR_EINVAL, "xy is NULL");
    return enqueue_inputs(B, xy, edges);
}

namespace {

// The graph of one evaluation with these metrics and parameters, captured on
// the batch's capture stream when it is missing or was made for others.
gr_status ensure_graph(gr_batch *B, uint32_t metrics, double ideal, uint32_t ideal_u, int64_t d) {
    if (B->exec && B->g_metrics == metrics && B->g_ideal == ideal_u && B->g_d == d) return GR_OK;
    drop_graph(B);
    cudaGraph_t graph;
    const int64_t k0 = gr_kernel_launches();
    B_CU(cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeRelaxed));
    enqueue_evaluate(B, B->cs, metrics, ideal, ideal_u, d);
    const cudaError_t ce = cudaStreamEndCapture(B->cs, &graph);
    B->graph_kernels = gr_kernel_launches() - k0;
    count_launches(-(int)B->graph_kernels);  // counted when replayed, not when captured
    if (ce != cudaSuccess) return bcuda(ce, "capturing the batch evaluation");
    const cudaError_t ie = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        B->exec = nullptr;
        return bcuda(ie, "instantiating the batch graph");
    }
    B->g_metrics = metrics;
    B->g_ideal = ideal_u;
    B->g_d = d;
    return GR_OK;
}

gr_status batch_params(const gr_params *params, double *ideal, int64_t *d, uint32_t *ideal_u) {
    *ideal = 7.0 * M_PI / 18.0;
    *d = 0;
    if (params) {
        if (params->ideal_rad > 0.0) *ideal = params->ideal_rad;
        *d = params->occlusion_d;
    }
    if (!(*ideal <= M_PI / 2 + 1e-15)) return bfail(GR_EINVAL, "ideal angle must be in (0, pi/2]");
    if (*d < 0) return bfail(GR_EINVAL, "occlusion diameter d must be >= 0");
    *ideal_u = (uint32_t)llrint(*ideal / M_PI * 4294967296.0);
    return GR_OK;
}

}  // namespace

gr_status gr_batch_evaluate_async(gr_batch *B, uint32_t metrics, const gr_params *params, gr_result *d_results,
                                  gr_stream_t stream) {
    set_last_error("");
    if (!B || !d_results) return bfail(GR_EINVAL, "NULL argument");
    if (metrics & ~GR_METRIC_ALL) return bfail(GR_EINVAL, "unknown metric bits");
    if (!is_device_ptr(d_results)) return bfail(GR_EINVAL, "d_results must be device memory");
    double ideal;
    int64_t d;
    uint32_t ideal_u;
    gr_status st = batch_params(params, &ideal, &d, &ideal_u);
    if (st != GR_OK) return st;
    if ((st = plan_occlusion(B, d)) != GR_OK) return st;
    cudaStream_t after = stream ? (cudaStream_t)stream : B->stream, c = B->cap;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (after != B->stream) B_CU(cudaStreamIsCapturing(after, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        // the caller's stream is being captured: the evaluation's steps are captured there directly
        enqueue_evaluate(B, after, metrics, ideal, ideal_u, d);
        B_CU(cudaMemcpyAsync(d_results, B->d_res, sizeof(gr_result) * B->L, cudaMemcpyDeviceToDevice, after));
        return GR_OK;
    }
    if ((st = ensure_graph(B, metrics, ideal, ideal_u, d)) != GR_OK) return st;
    // after the inputs (the batch's stream) and the caller's work, before what follows on the caller's stream
    B_CU(cudaEventRecord(B->ev_in, B->stream));
    B_CU(cudaStreamWaitEvent(c, B->ev_in, 0));
    if (after != B->stream) {
        B_CU(cudaEventRecord(B->ev_in2, after));
        B_CU(cudaStreamWaitEvent(c, B->ev_in2, 0));
    }
    B_CU(cudaGraphLaunch(B->exec, c));
    count_launches((int)B->graph_kernels);
    B_CU(cudaMemcpyAsync(d_results, B->d_res, sizeof(gr_result) * B->L, cudaMemcpyDeviceToDevice, c));
    B_CU(cudaEventRecord(B->ev_out, c));
    B_CU(cudaStreamWaitEvent(after, B->ev_out, 0));
    if (after != B->stream) B_CU(cudaStreamWaitEvent(B->stream, B->ev_out, 0));
    return GR_OK;
}

gr_status gr_batch_evaluate(gr_batch *B, uint32_t metrics, const gr_params *params, gr_result *out) {
    set_last_error("");
    if (!B || !out) return bfail(GR_EINVAL, "NULL argument");
    if (metrics & ~GR_METRIC_ALL) return bfail(GR_EINVAL, "unknown metric bits");
    double ideal = 7.0 * M_PI / 18.0;
    int64_t d = 0;
    if (params) {
        if (params->ideal_rad > 0.0) ideal = params->ideal_rad;
        d = params->occlusion_d;
    }
    if (!(ideal <= M_PI / 2 + 1e-15)) return bfail(GR_EINVAL, "ideal angle must be in (0, pi/2]");
    if (d < 0) return bfail(GR_EINVAL, "occlusion diameter d must be >= 0");
    const uint32_t ideal_u = (uint32_t)llrint(ideal / M_PI * 4294967296.0);
    gr_status st;
    if ((st = plan_occlusion(B, d)) != GR_OK) return st;
    cudaStream_t c = B->cap;
    B_CU(cudaEventRecord(B->ev_in, B->stream));  // inputs enqueued on the caller's stream come first
    B_CU(cudaStreamWaitEvent(c, B->ev_in, 0));
    for (int attempt = 0; attempt < 2; ++attempt) {
        if ((st = ensure_graph(B, metrics, ideal, ideal_u, d)) != GR_OK) return st;
        B_CU(cudaGraphLaunch(B->exec, c));
        count_launches((int)B->graph_kernels);
        B_CU(cudaMemcpyAsync(B->h_acc, B->b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, c));
        B_CU(cudaStreamSynchronize(c));
        if ((st = status_error(B->h_acc->status | B->h_acc->eval_status)) != GR_OK) return st;
        if ((B->h_acc->eval_status & ST_OVERFLOW) || (B->h_acc->grid_flags & GF_ITEMS_OVERFLOW)) {
            // the coordinates changed enough that the buffers no longer fit: re-plan
            if (attempt == 1 || (B->h_acc->grid_flags & GF_ITEMS_OVERFLOW))
                return bfail(GR_ENOMEM, "batch grid buffers overflowed after re-planning");
            if ((st = size_cross_buffers(B, c)) != GR_OK) return st;
            continue;
        }
        break;
    }
    const cudaMemcpyKind k = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    B_CU(cudaMemcpyAsync(out, B->d_res, sizeof(gr_result) * B->L, k, c));
    B_CU(cudaStreamSynchronize(c));
    return GR_OK;
}

gr_status gr_batch_tuning(const gr_batch *B, int32_t *cell_offset, int32_t *tile) {
    set_last_error("");
    if (!B || !cell_offset || !tile) return bfail(GR_EINVAL, "NULL argument");
    *cell_offset = B->delta;
    *tile = B->tile;
    return GR_OK;
}

gr_status gr_batch_destroy(gr_batch *B) {
    set_last_error("");
    if (!B) return GR_OK;
    cudaStreamSynchronize(B->stream);
    cudaStreamSynchronize(B->cap);
    free_batch(B);
    return GR_OK;
}

}  // extern "C"
