// k_crossings.cu -- edge-pair classification shared by the crossing kernels,
// and the tiled all-pairs crossing kernel (a7).
#include <math.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

namespace {

constexpr int AP_ROWS = 256;  // per-edge variant: rows per tile = threads per block
constexpr int AP_COLS = 256;  // per-edge variant: columns per tile (shared memory)

// Aggregate variant: 256 threads x 2 rows against 512 staged columns.
constexpr int AG_THREADS = 256;
constexpr int AG_RPT = 2;
constexpr int AG_ROWS = AG_THREADS * AG_RPT;
constexpr int AG_COLS = AG_ROWS;  // square tiles: the diagonal test is local j > local i
constexpr int AG_WARPS = AG_THREADS / 32;
constexpr int QCAP = 64;          // per-warp queue of E_c pairs awaiting their angle

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// a7 (aggregate counts) -- one block per square tile (bi <= bj, lower-
// triangular order, grid-strided).  Every thread holds two row segments in
// registers and walks the 512 staged columns in lock step with its warp; the
// E_c pairs a warp finds are queued in shared memory as (|u x v|, |u . v|)
// and their angles are evaluated 32 at a time, so the arctangent costs one
// lane-slot per crossing instead of stalling the whole warp on every pair
// that crosses.
__global__ void __launch_bounds__(AG_THREADS) k_cross_allpairs_agg(const SegRec *__restrict__ seg,
                                                                   DevAcc *acc, float ideal, int64_t tiles) {
    __shared__ ColSeg cs[AG_COLS];
    __shared__ float2 q[AG_WARPS][QCAP];
    __shared__ uint64_t shu[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int n_seg = (int)acc->n_seg;
    PairCounts pc;
    int qn = 0;  // warp-uniform queue length
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while (r * (r + 1) / 2 > t) --r;
        while ((r + 1) * (r + 2) / 2 <= t) ++r;
        const int bj = (int)r, bi = (int)(t - r * (r + 1) / 2);
        const int j0 = bj * AG_COLS;
        if (j0 >= n_seg) continue;
        const int nc = min(AG_COLS, n_seg - j0);
        __syncthreads();
        for (int c = threadIdx.x; c < nc; c += AG_THREADS) cs[c] = make_col(seg[j0 + c]);
        RowSeg rs[AG_RPT];
        bool rok[AG_RPT];
#pragma unroll
        for (int k = 0; k < AG_RPT; ++k) {
            const int i = bi * AG_ROWS + threadIdx.x + k * AG_THREADS;
            rok[k] = i < n_seg;
            if (rok[k]) rs[k] = make_row(seg[i]);
        }
        __syncthreads();
        const bool diag = bi == bj;
        for (int jj = 0; jj < nc; ++jj) {
            const ColSeg c = cs[jj];
#pragma unroll
            for (int k = 0; k < AG_RPT; ++k) {
                const bool valid = rok[k] && (!diag || jj > (int)threadIdx.x + k * AG_THREADS);
                const int kind = valid ? classify_kind(rs[k], c) : PAIR_NONE;
                const bool want = kind == PAIR_PROPER || kind == PAIR_TOUCHING;
                pc.proper += kind == PAIR_PROPER;
                pc.touching += kind == PAIR_TOUCHING;
                pc.collinear += kind == PAIR_COLLINEAR;
                const unsigned m = __ballot_sync(0xffffffffu, want);
                if (m) {
                    if (want) q[wid][qn + __popc(m & lt)] = cross_dot_abs(rs[k], c);
                    qn += __popc(m);
                    if (qn >= 32) {
                        __syncwarp();
                        pc.dev += dev_fixed(q[wid][lane], ideal);
                        const float2 tail = q[wid][lane + 32];
                        __syncwarp();
                        if (lane + 32 < qn) q[wid][lane] = tail;
                        qn -= 32;
                        __syncwarp();
                    }
                }
            }
        }
    }
    __syncwarp();
    if (lane < qn) pc.dev += dev_fixed(q[wid][lane], ideal);
    flush_counts(pc, acc, shu);
}

// a7 -- one block per (row tile bi, column tile bj) with bi <= bj, in
// lower-triangular enumeration order of blockIdx.x.  Each thread holds one row
// segment in registers; the column tile is staged in shared memory with its
// per-segment constants (direction v = d - c and k = v x c) precomputed, and
// every thread walks the whole column tile (broadcast reads).  Diagonal tiles
// test only j > i, so every unordered pair is tested exactly once.
template <bool PER_EDGE>
__global__ void __launch_bounds__(AP_ROWS) k_cross_allpairs(const SegRec *__restrict__ seg,
                                                            const int32_t *__restrict__ seg_eid,
                                                            DevAcc *acc, float ideal, PerEdge pe,
                                                            int64_t tiles) {
    __shared__ ColSeg cs[AP_COLS];
    __shared__ int32_t ceid[PER_EDGE ? AP_COLS : 1];
    __shared__ uint64_t shu[32];

    const int n_seg = (int)acc->n_seg;
    PairCounts pc;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // lower-triangular decode: t = r (r + 1) / 2 + c, c <= r
        int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while (r * (r + 1) / 2 > t) --r;
        while ((r + 1) * (r + 2) / 2 <= t) ++r;
        const int bj = (int)r, bi = (int)(t - r * (r + 1) / 2);
        const int j0 = bj * AP_COLS;
        if (j0 >= n_seg) continue;  // grid sized for E; compaction may have removed edges
        const int nc = min(AP_COLS, n_seg - j0);

        __syncthreads();  // the previous tile's readers are done with cs
        if (threadIdx.x < nc) {
            cs[threadIdx.x] = make_col(seg[j0 + threadIdx.x]);
            if (PER_EDGE) ceid[threadIdx.x] = seg_eid[j0 + threadIdx.x];
        }
        const int i = bi * AP_ROWS + threadIdx.x;
        const bool row_ok = i < n_seg;
        RowSeg rs;
        int32_t reid = 0;
        if (row_ok) {
            rs = make_row(seg[i]);
            if (PER_EDGE) reid = seg_eid[i];
        }
        __syncthreads();

        if (row_ok) {
            const int jbeg = (bi == bj) ? threadIdx.x + 1 : 0;
            uint32_t rp = 0, rt = 0, rc = 0;
            uint64_t rdev = 0;
#pragma unroll 4
            for (int jj = jbeg; jj < nc; ++jj) {
                const ColSeg c = cs[jj];
                float dev;
                const int k = classify(rs, c, ideal, dev);
                if (k != PAIR_NONE) {
                    uint64_t q = 0;
                    if (k == PAIR_COLLINEAR) {
                        ++pc.collinear;
                    } else {
                        q = (uint64_t)__float2ull_rn(dev * kDevScale);
                        pc.dev += q;
                        if (k == PAIR_PROPER) ++pc.proper; else ++pc.touching;
                    }
                    if (PER_EDGE) {
                        const int slot = k == PAIR_PROPER ? 0 : (k == PAIR_TOUCHING ? 1 : 2);
                        atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)ceid[jj] + slot], 1ull);
                        if (q) atomicAdd((unsigned long long *)&pe.dev[ceid[jj]], (unsigned long long)q);
                        if (slot == 0) ++rp; else if (slot == 1) ++rt; else ++rc;
                        rdev += q;
                    }
                }
            }
            if (PER_EDGE) {
                if (rp) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 0], (unsigned long long)rp);
                if (rt) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 1], (unsigned long long)rt);
                if (rc) atomicAdd((unsigned long long *)&pe.counts[3 * (int64_t)reid + 2], (unsigned long long)rc);
                if (rdev) atomicAdd((unsigned long long *)&pe.dev[reid], (unsigned long long)rdev);
            }
        }
    }
    flush_counts(pc, acc, shu);
}

}  // namespace

void launch_crossings_allpairs(const Buffers &b, int64_t n_seg, float ideal, PerEdge pe,
                               cudaStream_t s) {
    if (n_seg < 2) return;
    count_launches(1);
    if (pe.counts) {
        const int64_t nb = (n_seg + AP_ROWS - 1) / AP_ROWS;
        const int64_t tiles = nb * (nb + 1) / 2;
        const unsigned grid = (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
        k_cross_allpairs<true><<<grid, AP_ROWS, 0, s>>>(b.seg, b.seg_eid, b.acc, ideal, pe, tiles);
    } else {
        const int64_t nb = (n_seg + AG_ROWS - 1) / AG_ROWS;
        const int64_t tiles = nb * (nb + 1) / 2;
        const unsigned grid = (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
        k_cross_allpairs_agg<<<grid, AG_THREADS, 0, s>>>(b.seg, b.acc, ideal, tiles);
    }
}

}  // namespace gr
