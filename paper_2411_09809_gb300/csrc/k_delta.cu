// k_delta.cu -- incremental re-evaluation after a few vertices move (the
// inner loop of layout optimisation).
//
// Only pairs that involve a moved vertex can change.  The crossing counts,
// the crossing-angle sum and the occlusion count of the previous evaluation
// are updated by
//   - the pairs {a, e} of an affected edge a (one with a moved endpoint) and
//     any edge e, classified before the move and after it (a pair of two
//     affected edges counts once, in the pass of the one with the smaller
//     index);
//   - the pairs {v, u} of a moved vertex v and any vertex u, likewise.
// Classification and angle terms are the ones of the full evaluation (exact
// int64 orientations, the same integer line directions), so the updated sums
// equal a full evaluation's bit for bit.
#include "grid_common.cuh"

namespace gr {

namespace {

constexpr int DL_COLS = 256;

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

// Marks the moved vertices; raises ST_BAD_ID for an id outside [0, V) or an
// id given twice, ST_BAD_COORD for a new coordinate outside [0, 65536).
__global__ void k_mark_moved(const int32_t *__restrict__ ids, const int2 *__restrict__ xy_new,
                             const int64_t *__restrict__ np, int64_t V, uint32_t *__restrict__ moved, DeltaAcc *d) {
    const int64_t n = *np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ids[i];
        const int2 p = xy_new[i];
        if ((unsigned)p.x >= 65536u || (unsigned)p.y >= 65536u) atomicOr(&d->status, ST_BAD_COORD);
        if (v < 0 || v >= V) {
            atomicOr(&d->status, ST_BAD_ID);
            continue;
        }
        if (atomicExch(&moved[v], 1u) != 0u) atomicOr(&d->status, ST_BAD_ID);  // given twice
    }
}

__global__ void k_unmark_moved(const int32_t *__restrict__ ids, const int64_t *__restrict__ np, int64_t V,
                               uint32_t *__restrict__ moved) {
    const int64_t n = *np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ids[i];
        if (v >= 0 && v < V) moved[v] = 0u;
    }
}

// Writes the new coordinates, unless the validation raised an error (the
// layout then stays as it was).
__global__ void k_apply_moves(const int32_t *__restrict__ ids, const int2 *__restrict__ xy_new,
                              const int64_t *__restrict__ np, const DeltaAcc *__restrict__ d, int2 *__restrict__ xy) {
    if (d->status) return;
    const int64_t n = *np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xy[ids[i]] = xy_new[i];
}

// New totals = last - before + after (the 128-bit angle sum likewise) into
// the evaluation part of the accumulators, the classified pairs as the
// grid's candidate count; nothing when the validation raised an error.
__global__ void k_delta_combine(const DeltaCounts *__restrict__ lastp, const DeltaAcc *__restrict__ d, DevAcc *acc) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || d->status || d->fallback) return;
    const DeltaCounts last = *lastp;
    const DeltaCounts k0 = d->k[0], k1 = d->k[1];
    const unsigned __int128 dev = (((unsigned __int128)last.dev_hi << 64) | last.dev_lo) -
                                  (((unsigned __int128)k0.dev_hi << 64) | k0.dev_lo) +
                                  (((unsigned __int128)k1.dev_hi << 64) | k1.dev_lo);
    acc->eval_status = 0;
    acc->grid_flags = 0;
    acc->proper = last.proper - k0.proper + k1.proper;
    acc->touching = last.touching - k0.touching + k1.touching;
    acc->collinear = last.collinear - k0.collinear + k1.collinear;
    acc->dev_lo = (uint64_t)dev;
    acc->dev_hi = (uint64_t)(dev >> 64);
    acc->occlusion = last.occlusion - k0.occlusion + k1.occlusion;
    acc->records = 0;
    acc->grid_items = 0;
    acc->grid_work = d->tested;
    acc->n_long = 0;
}

// Edges with a moved endpoint, listed (warp-aggregated append); with a dirty
// set, the ones not in it yet are added (one thread per edge, so the flag
// needs no atomic).
__global__ void __launch_bounds__(256) k_affected_edges(const int2 *__restrict__ edges, int64_t E,
                                                        const uint32_t *__restrict__ moved, uint32_t *__restrict__ list,
                                                        DeltaAcc *d, DirtySet ds) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < E; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = base + threadIdx.x;
        bool hit = false;
        if (e < E) {
            const int2 ed = edges[e];
            hit = moved[ed.x] | moved[ed.y];
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        uint32_t slot = 0;
        if (lane == 0 && m) slot = atomicAdd(&d->n_affected, (uint32_t)__popc(m));
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (hit) list[slot + __popc(m & lanemask_lt())] = (uint32_t)e;
        if (hit && ds.flag && !ds.flag[e]) {
            ds.flag[e] = 1;
            const uint32_t q = atomicAdd(ds.n, 1u);
            if (q < ds.cap) ds.list[q] = (uint32_t)e;
            else d->fallback = 1u;
        }
    }
}

__device__ __forceinline__ SegRec edge_seg(const int2 *__restrict__ xy, int2 ed) {
    const int2 a = xy[ed.x], b = xy[ed.y];
    return make_uint4(uint32_t(a.x) | (uint32_t(a.y) << 16), uint32_t(b.x) | (uint32_t(b.y) << 16), (uint32_t)ed.x,
                      (uint32_t)ed.y);
}

__device__ __forceinline__ bool zero_length(SegRec s) { return s.x == s.y; }

// Pairs {a, e}: a from the affected list (staged in shared memory with its
// bounding box), e any non-zero-length segment of the gathered array (one
// per thread; the array matches the coordinates the pass runs on).  Only
// pairs whose boxes meet (touching counts) are classified: disjoint boxes
// never cross.  Counted into d->k[which].
__global__ void __launch_bounds__(DL_COLS) k_delta_cross(const SegRec *__restrict__ seg,
                                                         const int32_t *__restrict__ seg_eid,
                                                         const uint32_t *__restrict__ seg_theta,
                                                         const DevAcc *__restrict__ acc,
                                                         const int2 *__restrict__ edges,
                                                         const int2 *__restrict__ xy,
                                                         const uint32_t *__restrict__ moved,
                                                         const uint32_t *__restrict__ list, uint32_t ideal,
                                                         DeltaAcc *d, int which) {
    __shared__ ColSeg cs[DL_COLS];
    __shared__ int4 cbox[DL_COLS];
    __shared__ uint32_t cidx[DL_COLS];
    __shared__ uint64_t shu[32];
    if (d->status | d->fallback) return;
    const uint32_t na = d->n_affected, ns = acc->n_seg;
    PairCounts pc;
    uint64_t tested = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ns; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < ns;
        RowSeg r;
        SegRec s = make_uint4(0, 0, 0, 0);
        int32_t eid = -1;
        int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
        if (ok) {
            s = seg[i];
            eid = seg_eid[i];
            r = make_row(s, seg_theta[i]);
            x0 = min(px(s.x), px(s.y));
            x1 = max(px(s.x), px(s.y));
            y0 = min(py(s.x), py(s.y));
            y1 = max(py(s.x), py(s.y));
        }
        int e_aff = -1;  // read on the first box hit
        for (uint32_t c0 = 0; c0 < na; c0 += DL_COLS) {
            const uint32_t nc = min((uint32_t)DL_COLS, na - c0);
            __syncthreads();
            if (threadIdx.x < nc) {
                const uint32_t a = list[c0 + threadIdx.x];
                const SegRec t = edge_seg(xy, edges[a]);
                const bool z = zero_length(t);
                cs[threadIdx.x] = make_col(t, z ? 0u : line_direction(px(t.y) - px(t.x), py(t.y) - py(t.x)));
                cbox[threadIdx.x] = make_int4(min(px(t.x), px(t.y)), max(px(t.x), px(t.y)), min(py(t.x), py(t.y)),
                                              max(py(t.x), py(t.y)));
                cidx[threadIdx.x] = z ? 0xffffffffu : a;  // zero-length edges never cross
            }
            __syncthreads();
            if (!ok) continue;
            for (uint32_t j = 0; j < nc; ++j) {
                const int4 bb = cbox[j];
                if (bb.y < x0 || bb.x > x1 || bb.w < y0 || bb.z > y1) continue;
                const uint32_t a = cidx[j];
                if (a == 0xffffffffu || (int32_t)a == eid) continue;
                if ((int32_t)a > eid) {  // both affected: counted in the pass of the smaller index
                    if (e_aff < 0) e_aff = (moved[s.z] | moved[s.w]) ? 1 : 0;
                    if (e_aff) continue;
                }
                ++tested;
                const int kind = classify_kind(r, cs[j]);
                if (kind == PAIR_COLLINEAR) {
                    ++pc.collinear;
                } else if (kind != PAIR_NONE) {
                    if (kind == PAIR_PROPER) ++pc.proper; else ++pc.touching;
                    pc.dev += dev_term(r.th, cs[j].th, ideal);
                }
            }
        }
    }
    const uint64_t p = block_sum<uint64_t>(pc.proper, shu);
    const uint64_t t = block_sum<uint64_t>(pc.touching, shu);
    const uint64_t c = block_sum<uint64_t>(pc.collinear, shu);
    const uint64_t v = block_sum<uint64_t>(pc.dev, shu);
    const uint64_t n = block_sum<uint64_t>(tested, shu);
    if (threadIdx.x == 0) {
        DeltaCounts &k = d->k[which];
        atomic_add_u64(&k.proper, p);
        atomic_add_u64(&k.touching, t);
        atomic_add_u64(&k.collinear, c);
        add_u128(&k.dev_lo, &k.dev_hi, v);
        atomic_add_u64(&d->tested, n);
    }
}

// One pair of the grid walk: affected segment ra against the record c of the
// cell with lower-left corner (x0, y0) and side w (both in that cell's
// coordinates).  FP32 orientations with the grid path's filter, the exact
// int64 test when inconclusive, then the owner rules: E_c pairs count in the
// cell of their intersection point, collinear overlaps in the cell of the
// overlap's smallest point.
__device__ __forceinline__ void delta_cell_pair(const GSeg &ra, const GSeg &c, int x0, int y0, int w, uint32_t ideal,
                                                PairCounts &pc) {
    if ((ra.ida == c.ida) | (ra.ida == c.idb) | (ra.idb == c.ida) | (ra.idb == c.idb)) return;
    const float o1 = fmaf(ra.ux, c.ay, fmaf(-ra.uy, c.ax, ra.nk));
    const float o2 = fmaf(ra.ux, c.by, fmaf(-ra.uy, c.bx, ra.nk));
    const float o3 = fmaf(c.ux, ra.ay, fmaf(-c.uy, ra.ax, c.nk));
    const float o4 = fmaf(c.ux, ra.by, fmaf(-c.uy, ra.bx, c.nk));
    const float mn = fminf(fminf(fabsf(o1), fabsf(o2)), fminf(fabsf(o3), fabsf(o4)));
    int kind;
    if ((ra.exact & c.exact) || mn > kOrientFilter) {
        const float p12 = o1 * o2, p34 = o3 * o4;
        if (!(p12 <= 0.f && p34 <= 0.f)) return;
        kind = (o1 == 0.f && o2 == 0.f) ? PAIR_COLLINEAR : (p12 < 0.f && p34 < 0.f) ? PAIR_PROPER : PAIR_TOUCHING;
    } else {
        kind = classify_exact(ra, c, x0, y0);
        if (kind == PAIR_NONE) return;
    }
    if (kind == PAIR_COLLINEAR) {
        // the extents must meet, and this cell must own the overlap's smallest point
        const bool ar = ra.ax < ra.bx || (ra.ax == ra.bx && ra.ay <= ra.by);
        const bool ac = c.ax < c.bx || (c.ax == c.bx && c.ay <= c.by);
        const float elx = ar ? ra.ax : ra.bx, ely = ar ? ra.ay : ra.by;
        const float ehx = ar ? ra.bx : ra.ax, ehy = ar ? ra.by : ra.ay;
        const float flx = ac ? c.ax : c.bx, fly = ac ? c.ay : c.by;
        const float fhx = ac ? c.bx : c.ax, fhy = ac ? c.by : c.ay;
        const bool lo_e = elx > flx || (elx == flx && ely >= fly);
        const float lx = lo_e ? elx : flx, ly = lo_e ? ely : fly;
        const bool hi_e = ehx < fhx || (ehx == fhx && ehy <= fhy);
        const float hx = hi_e ? ehx : fhx, hy = hi_e ? ehy : fhy;
        if (!(lx < hx || (lx == hx && ly <= hy))) return;
        if (owns_collinear(ra, c, w)) ++pc.collinear;
        return;
    }
    if (!owns_crossing_fast(ra, c, w)) return;
    pc.dev += dev_term(ra.th, c.th, ideal);
    if (kind == PAIR_PROPER) ++pc.proper; else ++pc.touching;
}

constexpr int DG_THREADS = 256;
constexpr int DG_LINES = 1024;  // major lines enumerated at a time (4 per thread)
constexpr int DG_SLICES = 8;    // blocks sharing one affected edge's records

__device__ __forceinline__ uint32_t dg_block_excl_scan(uint32_t v, uint32_t *sh, uint32_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < DG_THREADS / 32; ++w) {
            const uint32_t t = sh[w];
            sh[w] = run;
            run += t;
        }
        sh[32] = run;
    }
    __syncthreads();
    *total = sh[32];
    return sh[wid] + x - v;
}

// Pairs {a, e} of an affected edge a and a clean edge e (not moved since the
// grid was built), through the grid of the last full evaluation, which holds
// every clean edge in every cell of side 2^k its closed segment meets.
// DG_SLICES blocks share an affected edge (grid-stride over edge x slice):
// each lists the cells of the edge's current segment (DDA, up to DG_LINES
// major lines at a time) with an exclusive prefix of their record counts in
// shared memory, then its threads take the records of its slice of that
// flattened range, locating each record's cell by binary search.  Records of
// dirty edges are stale and skipped.  The owner rules count each pair in one
// cell, as in the full evaluation.
__global__ void __launch_bounds__(DG_THREADS) k_delta_grid(const int2 *__restrict__ edges,
                                                           const int2 *__restrict__ xy,
                                                           const uint32_t *__restrict__ list,
                                                           const uint8_t *__restrict__ dirty,
                                                           const uint32_t *__restrict__ cell_off,
                                                           const GridRec *__restrict__ rec, int k, uint32_t ideal,
                                                           DeltaAcc *d, int which) {
    __shared__ uint32_t cell_id[2 * DG_LINES];
    __shared__ uint32_t pre[2 * DG_LINES];
    __shared__ uint32_t scan_sh[33];
    __shared__ uint64_t shu[32];
    if (d->status | d->fallback) return;
    const uint32_t nv = d->n_affected * DG_SLICES;
    const int G = 65536 >> k, w = 1 << k;
    PairCounts pc;
    uint64_t tested = 0;
    for (uint32_t vb = blockIdx.x; vb < nv; vb += gridDim.x) {
        const uint32_t a = list[vb / DG_SLICES], slice = vb % DG_SLICES;
        const SegRec sa = edge_seg(xy, edges[a]);
        if (zero_length(sa)) continue;  // never crosses (the same edge for the whole block)
        GridRec ga;
        ga.s = sa;
        ga.x = make_uint4(a, line_direction(px(sa.y) - px(sa.x), py(sa.y) - py(sa.x)), 0u, 0u);
        const DdaSeg s = dda_norm(sa);
        const int c_last = s.x1 >> k;
        for (int cb = s.x0 >> k; cb <= c_last; cb += DG_LINES) {
            const int nl = min(DG_LINES, c_last - cb + 1);
            uint32_t cnt[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int l = 4 * threadIdx.x + q;
                int ids[2];
                const int n = l < nl ? line_cells(s, cb + l, k, G, 0u, ids) : 0;
#pragma unroll
                for (int z = 0; z < 2; ++z) {
                    uint32_t c = 0;
                    if (z < n) {
                        c = cell_off[ids[z] + 1] - cell_off[ids[z]];
                        cell_id[2 * l + z] = (uint32_t)ids[z];
                    }
                    cnt[2 * q + z] = c;
                    sum += c;
                }
            }
            uint32_t total;
            uint32_t run = dg_block_excl_scan(sum, scan_sh, &total);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                pre[8 * threadIdx.x + e] = run;
                run += cnt[e];
            }
            __syncthreads();
            const int ne = 2 * nl;
            const uint32_t per = (total + DG_SLICES - 1) / DG_SLICES;
            const uint32_t r_beg = slice * per, r_end = min(total, r_beg + per);
            for (uint32_t t = r_beg + threadIdx.x; t < r_end; t += DG_THREADS) {
                int lo = 0, hi = ne;  // the last entry with pre <= t (it has records: t < total)
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (pre[mid] <= t) lo = mid; else hi = mid;
                }
                const uint32_t cell = cell_id[lo];
                const GridRec g = rec[cell_off[cell] + (t - pre[lo])];
                if (dirty[g.x.x]) continue;
                const int x0 = (int)(cell & (uint32_t)(G - 1)) << k, y0 = (int)(cell >> (16 - k)) << k;
                ++tested;
                delta_cell_pair(make_gseg(ga, x0, y0), make_gseg(g, x0, y0), x0, y0, w, ideal, pc);
            }
            __syncthreads();  // the next chunk reuses the shared arrays
        }
    }
    const uint64_t p = block_sum<uint64_t>(pc.proper, shu);
    const uint64_t t = block_sum<uint64_t>(pc.touching, shu);
    const uint64_t cl = block_sum<uint64_t>(pc.collinear, shu);
    const uint64_t v = block_sum<uint64_t>(pc.dev, shu);
    const uint64_t n = block_sum<uint64_t>(tested, shu);
    if (threadIdx.x == 0) {
        DeltaCounts &kk = d->k[which];
        atomic_add_u64(&kk.proper, p);
        atomic_add_u64(&kk.touching, t);
        atomic_add_u64(&kk.collinear, cl);
        add_u128(&kk.dev_lo, &kk.dev_hi, v);
        atomic_add_u64(&d->tested, n);
    }
}

// Pairs {a, e} of an affected edge a and a dirty edge e (current
// coordinates), one thread per pair (grid-stride over dirty x affected; both
// lists are short and stay in cache); a pair of two affected edges once, in
// the pass of the smaller index.  Every pair is seen once: plain
// classification after a bounding-box test.
__global__ void __launch_bounds__(256) k_delta_dirty(const int2 *__restrict__ edges, const int2 *__restrict__ xy,
                                                     const uint32_t *__restrict__ moved,
                                                     const uint32_t *__restrict__ list, DirtySet ds, uint32_t ideal,
                                                     DeltaAcc *d, int which) {
    __shared__ uint64_t shu[32];
    if (d->status | d->fallback) return;
    const uint64_t na = d->n_affected, nd = min(*ds.n, ds.cap);
    PairCounts pc;
    uint64_t tested = 0;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nd * na;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t e = ds.list[p / na], a = list[p % na];
        if (a == e) continue;
        const int2 ee = edges[e], ea = edges[a];
        const SegRec se = edge_seg(xy, ee), sa = edge_seg(xy, ea);
        if (zero_length(se) || zero_length(sa)) continue;  // never cross
        if (max(px(sa.x), px(sa.y)) < min(px(se.x), px(se.y)) || min(px(sa.x), px(sa.y)) > max(px(se.x), px(se.y)) ||
            max(py(sa.x), py(sa.y)) < min(py(se.x), py(se.y)) || min(py(sa.x), py(sa.y)) > max(py(se.x), py(se.y)))
            continue;
        if (a > e && (moved[ee.x] | moved[ee.y])) continue;  // both affected: counted with the smaller index
        ++tested;
        const RowSeg r = make_row(se, line_direction(px(se.y) - px(se.x), py(se.y) - py(se.x)));
        const ColSeg c = make_col(sa, line_direction(px(sa.y) - px(sa.x), py(sa.y) - py(sa.x)));
        const int kind = classify_kind(r, c);
        if (kind == PAIR_COLLINEAR) {
            ++pc.collinear;
        } else if (kind != PAIR_NONE) {
            if (kind == PAIR_PROPER) ++pc.proper; else ++pc.touching;
            pc.dev += dev_term(r.th, c.th, ideal);
        }
    }
    const uint64_t p = block_sum<uint64_t>(pc.proper, shu);
    const uint64_t t = block_sum<uint64_t>(pc.touching, shu);
    const uint64_t cl = block_sum<uint64_t>(pc.collinear, shu);
    const uint64_t v = block_sum<uint64_t>(pc.dev, shu);
    const uint64_t n = block_sum<uint64_t>(tested, shu);
    if (threadIdx.x == 0) {
        DeltaCounts &kk = d->k[which];
        atomic_add_u64(&kk.proper, p);
        atomic_add_u64(&kk.touching, t);
        atomic_add_u64(&kk.collinear, cl);
        add_u128(&kk.dev_lo, &kk.dev_hi, v);
        atomic_add_u64(&d->tested, n);
    }
}

// Pairs {v, u}: v a moved vertex (staged), u any vertex (one per thread);
// squared distance below d2.  A pair of two moved vertices counts once.
__global__ void __launch_bounds__(DL_COLS) k_delta_occl(const int2 *__restrict__ xy, int64_t V,
                                                        const uint32_t *__restrict__ moved,
                                                        const int32_t *__restrict__ ids,
                                                        const int64_t *__restrict__ np, long long d2, DeltaAcc *d,
                                                        int which) {
    __shared__ int2 cp[DL_COLS];
    __shared__ int32_t cv[DL_COLS];
    __shared__ uint64_t shu[32];
    if (d->status | d->fallback) return;
    const int64_t n = *np;
    uint64_t cnt = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = base + threadIdx.x;
        const bool ok = u < V;
        const int2 p = ok ? xy[u] : make_int2(0, 0);
        const bool u_moved = ok && moved[u];
        for (int64_t c0 = 0; c0 < n; c0 += DL_COLS) {
            const int nc = (int)min((int64_t)DL_COLS, n - c0);
            __syncthreads();
            if (threadIdx.x < nc) {
                const int32_t v = ids[c0 + threadIdx.x];
                cv[threadIdx.x] = v;
                cp[threadIdx.x] = xy[v];
            }
            __syncthreads();
            if (!ok) continue;
            for (int j = 0; j < nc; ++j) {
                const int32_t v = cv[j];
                if (v == u || (u_moved && v > u)) continue;
                const long long dx = p.x - cp[j].x, dy = p.y - cp[j].y;
                cnt += (dx * dx + dy * dy < d2) ? 1u : 0u;
            }
        }
    }
    cnt = block_sum<uint64_t>(cnt, shu);
    if (threadIdx.x == 0) atomic_add_u64(&d->k[which].occlusion, cnt);
}

}  // namespace

void launch_delta_validate(const int32_t *ids, const int32_t *xy_new, const int64_t *np, int64_t cap, int64_t V,
                           uint32_t *moved, DeltaAcc *d, cudaStream_t s) {
    count_launches(1);
    k_mark_moved<<<grid_for(cap, 256, 152 * 4), 256, 0, s>>>(ids, (const int2 *)xy_new, np, V, moved, d);
}

void launch_delta_unmark(const int32_t *ids, const int64_t *np, int64_t cap, int64_t V, uint32_t *moved,
                         cudaStream_t s) {
    count_launches(1);
    k_unmark_moved<<<grid_for(cap, 256, 152 * 4), 256, 0, s>>>(ids, np, V, moved);
}

void launch_delta_pass(const Buffers &b, int64_t V, int64_t E, const int32_t *ids, const int64_t *np,
                       const uint32_t *moved, const uint32_t *affected, bool crossings, uint32_t ideal, bool occlusion,
                       long long d2, DeltaAcc *d, int which, cudaStream_t s) {
    if (crossings && E > 0) {
        count_launches(1);
        k_delta_cross<<<grid_for(E, DL_COLS, 152 * 8), DL_COLS, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc,
                                                                        (const int2 *)b.edges, (const int2 *)b.xy,
                                                                        moved, affected, ideal, d, which);
    }
    if (occlusion && V > 0) {
        count_launches(1);
        k_delta_occl<<<grid_for(V, DL_COLS, 152 * 8), DL_COLS, 0, s>>>((const int2 *)b.xy, V, moved, ids, np, d2, d,
                                                                       which);
    }
}

void launch_delta_affected(const Buffers &b, int64_t E, const uint32_t *moved, uint32_t *affected, DeltaAcc *d,
                           const DirtySet &ds, cudaStream_t s) {
    if (E <= 0) return;
    count_launches(1);
    k_affected_edges<<<grid_for(E, 256, 152 * 8), 256, 0, s>>>((const int2 *)b.edges, E, moved, affected, d, ds);
}

void launch_delta_grid_pass(const Buffers &b, const GridBuffers &g, int k, const uint32_t *moved,
                            const uint32_t *affected, const DirtySet &ds, uint32_t ideal, DeltaAcc *d, int which,
                            cudaStream_t s) {
    count_launches(2);
    k_delta_grid<<<152 * 4, DG_THREADS, 0, s>>>((const int2 *)b.edges, (const int2 *)b.xy, affected, ds.flag,
                                                   g.cell_off, g.rec, k, ideal, d, which);
    k_delta_dirty<<<152 * 2, 256, 0, s>>>((const int2 *)b.edges, (const int2 *)b.xy, moved, affected, ds, ideal, d,
                                          which);
}

void launch_delta_apply(const int32_t *ids, const int32_t *xy_new, const int64_t *np, int64_t cap, const DeltaAcc *d,
                        Buffers &b, cudaStream_t s) {
    count_launches(1);
    k_apply_moves<<<grid_for(cap, 256, 152 * 4), 256, 0, s>>>(ids, (const int2 *)xy_new, np, d, (int2 *)b.xy);
}

void launch_delta_combine(const DeltaCounts *last, const DeltaAcc *d, Buffers &b, cudaStream_t s) {
    count_launches(1);
    k_delta_combine<<<1, 32, 0, s>>>(last, d, b.acc);
}

}  // namespace gr
