// k_crossings.cu -- the tiled all-pairs crossing kernels (a7).
//
// Every unordered pair of compacted segments is tested once: square tiles
// (row tile bi <= column tile bj) are enumerated in lower-triangular order
// and diagonal tiles keep only column > row.
#include "allpairs_common.cuh"

namespace gr {

namespace {

// One block per square tile (grid-strided) of the n segments at seg/theta (n
// read from the device).  Each thread holds AG_RPT row segments; the columns
// are staged in shared memory in FP32 form (plus the raw records for the
// exact fallback) and read by broadcast.
template <int THREADS, int RPT>
__global__ void __launch_bounds__(THREADS) k_cross_allpairs_agg(const SegRec *__restrict__ seg,
                                                                const uint32_t *__restrict__ theta,
                                                                const uint32_t *__restrict__ n_p, DevAcc *acc,
                                                                uint32_t ideal, int64_t tiles, int part0_only) {
    __shared__ AllPairsSmem<THREADS * RPT> sm;
    __shared__ uint64_t shu[32];
    const int n = (int)*n_p;
    if (tiles < 0) {  // sized on the device: a persistent launch over all tiles of the n segments
        const int64_t nb = (n + THREADS * RPT - 1) / (THREADS * RPT);
        tiles = nb * (nb + 1) / 2;
    }
    PairCounts pc;
    uint64_t lo, hi;  // this evaluation's share of the tiles
    if (part0_only) {
        lo = 0;
        hi = (partitioned(acc) && acc->part_id != 0) ? 0 : (uint64_t)tiles;
    } else {
        part_range(acc, (uint64_t)tiles, lo, hi);
    }
    for (int64_t t = (int64_t)lo + blockIdx.x; t < (int64_t)hi; t += gridDim.x) {
        int bi, bj;
        decode_tile(t, bi, bj);
        allpairs_tile<THREADS, RPT>(seg, theta, n, bi, bj, ideal, sm, pc);
    }
    flush_counts(pc, acc, shu);
}

// Lists shorter than this take the small tiles.
constexpr int64_t kSmallTileList = 32768;

// ------------------------------------------------------------ per-edge a7
// Exact int64 classification of every pair, with per-edge tallies (atomics).
constexpr int PE_ROWS = 256;
constexpr int PE_COLS = 256;

__global__ void __launch_bounds__(PE_ROWS) k_cross_allpairs_per_edge(const SegRec *__restrict__ seg,
                                                                     const int32_t *__restrict__ seg_eid,
                                                                     const uint32_t *__restrict__ theta,
                                                                     const uint32_t *__restrict__ n_p, DevAcc *acc,
                                                                     uint32_t ideal, PerEdge pe, int64_t tiles) {
    __shared__ ColSeg cs[PE_COLS];
    __shared__ int32_t ceid[PE_COLS];
    __shared__ uint64_t shu[32];
    const int n_seg = (int)*n_p;
    PairCounts pc;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int bi, bj;
        decode_tile(t, bi, bj);
        const int j0 = bj * PE_COLS;
        if (j0 >= n_seg) continue;
        const int nc = min(PE_COLS, n_seg - j0);
        __syncthreads();
        if (threadIdx.x < nc) {
            cs[threadIdx.x] = make_col(seg[j0 + threadIdx.x], theta[j0 + threadIdx.x]);
            ceid[threadIdx.x] = seg_eid[j0 + threadIdx.x];
        }
        const int i = bi * PE_ROWS + threadIdx.x;
        const bool row_ok = i < n_seg;
        RowSeg rs;
        int32_t reid = 0;
        if (row_ok) {
            rs = make_row(seg[i], theta[i]);
            reid = seg_eid[i];
        }
        __syncthreads();
        if (!row_ok) continue;
        uint32_t rp = 0, rt = 0, rc = 0;
        uint64_t rdev = 0;
        for (int jj = (bi == bj) ? threadIdx.x + 1 : 0; jj < nc; ++jj) {
            const ColSeg c = cs[jj];
            const int kind = classify_kind(rs, c);
            if (kind == PAIR_NONE) continue;
            const int64_t ce = ceid[jj];
            if (kind == PAIR_COLLINEAR) {
                ++pc.collinear;
                ++rc;
                atomicAdd((unsigned long long *)&pe.counts[3 * ce + 2], 1ull);
                continue;
            }
            const uint32_t dv = dev_term(rs.th, c.th, ideal);
            pc.dev += dv;
            rdev += dv;
            if (kind == PAIR_PROPER) { ++pc.proper; ++rp; } else { ++pc.touching; ++rt; }
            atomicAdd((unsigned long long *)&pe.counts[3 * ce + (kind == PAIR_PROPER ? 0 : 1)], 1ull);
            atomicAdd((unsigned long long *)&pe.dev[ce], (unsigned long long)dv);
        }
        if (rp) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 0], (unsigned long long)rp);
        if (rt) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 1], (unsigned long long)rt);
        if (rc) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 2], (unsigned long long)rc);
        if (rdev) atomicAdd((unsigned long long *)&pe.dev[reid], (unsigned long long)rdev);
    }
    flush_counts(pc, acc, shu);
}

unsigned grid_of(int64_t tiles) {
    return (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
}

}  // namespace

void launch_crossings_allpairs(const Buffers &b, int64_t n_seg, uint32_t ideal, PerEdge pe,
                               cudaStream_t s) {
    launch_crossings_allpairs_of(b.seg, b.seg_eid, b.seg_theta, &b.acc->n_seg, b.acc, n_seg, ideal, pe, s);
}

void launch_crossings_allpairs_of(const SegRec *seg, const int32_t *eid, const uint32_t *theta, const uint32_t *n_p,
                                  DevAcc *acc, int64_t n_bound, uint32_t ideal, PerEdge pe, cudaStream_t s,
                                  bool part0_only) {
    const int p0 = part0_only ? 1 : 0;
    if (n_bound < 0) {  // the count is known on the device only: small tiles, persistent
        count_launches(1);
        k_cross_allpairs_agg<AS_THREADS, AS_RPT><<<152 * 8, AS_THREADS, 0, s>>>(seg, theta, n_p, acc, ideal, -1, p0);
        return;
    }
    if (n_bound < 2) return;
    count_launches(1);
    if (pe.counts) {
        const int64_t nb = (n_bound + PE_ROWS - 1) / PE_ROWS;
        const int64_t tiles = nb * (nb + 1) / 2;
        k_cross_allpairs_per_edge<<<grid_of(tiles), PE_ROWS, 0, s>>>(seg, eid, theta, n_p, acc, ideal, pe, tiles);
    } else if (n_bound < kSmallTileList) {
        const int64_t nb = (n_bound + AS_ROWS - 1) / AS_ROWS;
        const int64_t tiles = nb * (nb + 1) / 2;
        k_cross_allpairs_agg<AS_THREADS, AS_RPT><<<grid_of(tiles), AS_THREADS, 0, s>>>(seg, theta, n_p, acc, ideal,
                                                                                      tiles, p0);
    } else {
        const int64_t nb = (n_bound + AG_ROWS - 1) / AG_ROWS;
        const int64_t tiles = nb * (nb + 1) / 2;
        k_cross_allpairs_agg<AG_THREADS, AG_RPT><<<grid_of(tiles), AG_THREADS, 0, s>>>(seg, theta, n_p, acc, ideal,
                                                                                      tiles, p0);
    }
}

}  // namespace gr
