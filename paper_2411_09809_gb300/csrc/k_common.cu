// k_common.cu -- gather + validation (a1), exclusive scan, edge length
// variation (a10) and the final reducer (a11).
#include <math.h>

#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// a1 -- one thread per edge (grid-stride, block-uniform trip count).  Reads
// the edge's vertex ids and coordinates (the D_e x D_pos join of Algorithm 4),
// checks them, stores the exact squared length of every edge and appends the
// non-zero-length ones to the compacted segment array.  Slots are reserved
// once per block and iteration (a block-wide prefix over the warps' counts),
// the L1-length and zero-length totals once per block: same-address atomics
// per warp serialised at L2 and dominated the kernel.  The order of the
// compacted array does not affect any result.  The same grid also checks
// every vertex's coordinates (isolated vertices included).
constexpr int kGatherThreads = 256, kGatherWarps = kGatherThreads / 32;

__global__ void __launch_bounds__(kGatherThreads) k_gather(const int2 *__restrict__ xy, int64_t V,
                                                           const int2 *__restrict__ edges, int64_t E,
                                                           SegRec *__restrict__ seg,
                                                           int32_t *__restrict__ seg_eid,
                                                           uint32_t *__restrict__ seg_theta,
                                                           int64_t *__restrict__ len2, DevAcc *acc) {
    __shared__ uint32_t h_n[16];
    __shared__ unsigned long long h_l1[16];
    // per-warp counts, then the warps' slots; double-buffered by iteration parity
    __shared__ uint32_t w_cnt[2][kGatherWarps];
    __shared__ unsigned long long red[kGatherWarps][2];
    if (threadIdx.x < 16) {
        h_n[threadIdx.x] = 0;
        h_l1[threadIdx.x] = 0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad_v = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
        const int2 p = xy[v];
        bad_v |= ((unsigned)p.x >= 65536u) | ((unsigned)p.y >= 65536u);
    }
    if (bad_v) atomicOr(&acc->status, ST_BAD_COORD);
    __syncthreads();
    uint64_t l1_sum = 0, zero_sum = 0;
    int par = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < E; base += stride, par ^= 1) {
        const int64_t e = base + threadIdx.x;
        bool keep = false, zero = false;
        uint32_t l1 = 0;
        SegRec r = make_uint4(0, 0, 0, 0);
        if (e < E) {
            const int2 ed = edges[e];
            int64_t l2 = 0;
            if (ed.x < 0 || ed.y < 0 || ed.x >= V || ed.y >= V || ed.x == ed.y) {
                atomicOr(&acc->status, ST_BAD_ID);
            } else {
                const int2 a = xy[ed.x], b = xy[ed.y];
                if ((unsigned)a.x >= 65536u || (unsigned)a.y >= 65536u ||
                    (unsigned)b.x >= 65536u || (unsigned)b.y >= 65536u) {
                    atomicOr(&acc->status, ST_BAD_COORD);
                } else {
                    const int64_t dx = b.x - a.x, dy = b.y - a.y;
                    l2 = dx * dx + dy * dy;
                    if (l2 != 0) {
                        keep = true;
                        l1 = (uint32_t)(abs(b.x - a.x) + abs(b.y - a.y));
                        r = make_uint4(uint32_t(a.x) | (uint32_t(a.y) << 16),
                                       uint32_t(b.x) | (uint32_t(b.y) << 16),
                                       uint32_t(ed.x), uint32_t(ed.y));
                    } else {
                        zero = true;
                    }
                }
            }
            len2[e] = l2;
        }
        l1_sum += l1;
        zero_sum += zero;
        const unsigned mk = __ballot_sync(FULL, keep);
        if (lane == 0) w_cnt[par][wid] = (uint32_t)__popc(mk);
        __syncthreads();
        if (wid == 0) {
            const uint32_t c = lane < kGatherWarps ? w_cnt[par][lane] : 0u;
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < kGatherWarps; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(FULL, incl, kGatherWarps - 1);
            uint32_t b0 = 0;
            if (lane == 0 && total) b0 = atomicAdd(&acc->n_seg, total);
            b0 = __shfl_sync(FULL, b0, 0);
            if (lane < kGatherWarps) w_cnt[par][lane] = b0 + incl - c;
        }
        __syncthreads();
        if (keep) {
            const uint32_t pos = w_cnt[par][wid] + __popc(mk & lanemask_lt());
            seg[pos] = r;
            seg_eid[pos] = (int32_t)e;
            const int dx = px(r.y) - px(r.x), dy = py(r.y) - py(r.x);
            seg_theta[pos] = line_direction(dx, dy);
        }
        // length classes, aggregated over the lanes of a warp in the same class
        const int b = keep ? 31 - __clz(max(abs(px(r.y) - px(r.x)), abs(py(r.y) - py(r.x)))) : -1;
        if (keep) {
            const unsigned same = __match_any_sync(mk, b);
            const uint32_t l1s = __reduce_add_sync(same, l1);
            if (lane == __ffs(same) - 1) {
                atomicAdd(&h_n[b], (uint32_t)__popc(same));
                atomicAdd(&h_l1[b], (unsigned long long)l1s);
            }
        }
    }
    l1_sum = warp_sum<uint64_t>(l1_sum);
    zero_sum = warp_sum<uint64_t>(zero_sum);
    if (lane == 0) {
        red[wid][0] = l1_sum;
        red[wid][1] = zero_sum;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        unsigned long long t = 0;
        for (int w = 0; w < kGatherWarps; ++w) t += red[w][threadIdx.x];
        if (t) atomicAdd(threadIdx.x == 0 ? (unsigned long long *)&acc->len_l1 : (unsigned long long *)&acc->zero_len,
                         t);
    }
    if (threadIdx.x < 16 && h_n[threadIdx.x]) {
        atomicAdd(&acc->len_hist[threadIdx.x], h_n[threadIdx.x]);
        atomicAdd((unsigned long long *)&acc->l1_hist[threadIdx.x], h_l1[threadIdx.x]);
    }
}

__global__ void __launch_bounds__(256) k_check_vertices(const int2 *__restrict__ xy, int64_t V,
                                                        DevAcc *acc) {
    bool bad = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = xy[v];
        bad |= ((unsigned)p.x >= 65536u) | ((unsigned)p.y >= 65536u);
    }
    if (bad) atomicOr(&acc->status, ST_BAD_COORD);
}

// ------------------------------------------------------------------- scan
// Three phases: per-block sums, one-block scan of the block sums, per-block
// scan + offset.  kScanItems = 1024 threads x 4 items.

__global__ void __launch_bounds__(1024) k_scan_sums(const uint32_t *__restrict__ in, int64_t n,
                                                    uint64_t *__restrict__ block_sum_out) {
    __shared__ uint64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanItems + threadIdx.x * 4;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) s += in[base + k];
    s = block_sum<uint64_t>(s, sh);
    if (threadIdx.x == 0) block_sum_out[blockIdx.x] = s;
}

// Exclusive scan of the block sums in place (one block of 1024 threads,
// 16 values per thread).
__global__ void __launch_bounds__(1024) k_scan_top(uint64_t *__restrict__ bs, int nb,
                                                   uint32_t *__restrict__ out, int64_t n,
                                                   uint64_t *total, uint32_t *status) {
    __shared__ uint64_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t v[16];
    uint64_t t = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = threadIdx.x * 16 + k;
        v[k] = i < nb ? bs[i] : 0;
        t += v[k];
    }
    // inclusive warp scan of the thread totals
    uint64_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = warp_tot[lane];
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive
    }
    __syncthreads();
    uint64_t run = warp_tot[wid] + inc - t;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = threadIdx.x * 16 + k;
        if (i < nb) bs[i] = run;
        run += v[k];
    }
    if (threadIdx.x == 1023) {
        // run now holds the grand total
        *total = run;
        if (run > 0xffffffffull) atomicOr(status, ST_SCAN_OVERFLOW);
        out[n] = (uint32_t)run;
    }
}

__global__ void __launch_bounds__(1024) k_scan_apply(const uint32_t *in, uint32_t *out, int64_t n,
                                                     const uint64_t *__restrict__ boff) {
    __shared__ uint32_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanItems + threadIdx.x * 4;
    uint32_t v[4];
    uint32_t t = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        t += v[k];
    }
    uint32_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t w = warp_tot[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = (uint32_t)boff[blockIdx.x] + warp_tot[wid] + inc - t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ------------------------------------------------------------------ ELV a10
// Pass 1: per-block FP64 sum of edge lengths l_e = sqrt(len2_e) over a fixed
// strided subset of edges (fixed order => deterministic); l_e is stored for
// pass 2, so the FP64 square root (slow on GB300) runs once per edge.
__device__ __forceinline__ double edge_length(const int64_t *__restrict__ len2, int64_t e, bool f32) {
    const int64_t q = len2[e];
    return sqrt(f32 ? __longlong_as_double(q) : (double)q);
}

__global__ void __launch_bounds__(256) k_elv_sum(const int64_t *__restrict__ len2, int64_t E,
                                                 double *__restrict__ len, double *__restrict__ part, bool f32) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)kElvBlocks * blockDim.x) {
        const double l = edge_length(len2, e, f32);
        len[e] = l;
        s += l;
    }
    s = block_sum<double>(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Pass 2: every block recomputes the mean from the pass-1 partials in the
// same fixed order, then sums (l_e - mean)^2 over its subset.
__global__ void __launch_bounds__(256) k_elv_var(const double *__restrict__ len, int64_t E,
                                                 double *__restrict__ part) {
    __shared__ double sh[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < kElvBlocks; i += blockDim.x) m += part[i];
    m = block_sum<double>(m, sh) / (double)E;
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)kElvBlocks * blockDim.x) {
        const double t = len[e] - m;
        s += t * t;
    }
    s = block_sum<double>(s, sh);
    if (threadIdx.x == 0) part[kElvBlocks + blockIdx.x] = s;
}

// ------------------------------------------------------------- finalize a11
__global__ void __launch_bounds__(256) k_finalize(const DevAcc *__restrict__ acc,
                                                  const double *__restrict__ elv_part,
                                                  const double *__restrict__ ma_part,
                                                  const uint32_t *__restrict__ ma_cnt, int ma_blocks,
                                                  uint32_t metrics, int64_t E, double ideal, int64_t d,
                                                  int32_t path, int32_t cell_log2, int32_t occl_path,
                                                  int64_t pairs_tested, gr_result *__restrict__ out) {
    __shared__ double shd[32];
    __shared__ uint64_t shu[32];
    // edge length variation (Algorithm 3)
    double sl = 0.0, sv = 0.0;
    if (metrics & GR_METRIC_EDGE_LENGTH) {
        for (int i = threadIdx.x; i < kElvBlocks; i += blockDim.x) {
            sl += elv_part[i];
            sv += elv_part[kElvBlocks + i];
        }
    }
    sl = block_sum<double>(sl, shd);
    sv = block_sum<double>(sv, shd);
    // minimum angle (Algorithm 2)
    double ms = 0.0;
    uint64_t mn = 0;
    for (int i = threadIdx.x; i < ((metrics & GR_METRIC_MIN_ANGLE) ? ma_blocks : 0); i += blockDim.x) {
        ms += ma_part[i];
        mn += ma_cnt[i];
    }
    ms = block_sum<double>(ms, shd);
    mn = block_sum<uint64_t>(mn, shu);
    if (threadIdx.x != 0) return;

    gr_result r;
    memset(&r, 0, sizeof(r));
    // a failed evaluation (invalid input, outgrown buffers) is marked by metrics = 0, so that results
    // written to device memory without a read-back can be told apart
    const bool failed = (acc->status | acc->eval_status) != 0 ||
                        (path == GR_PATH_GRID && (acc->grid_flags & GF_ITEMS_OVERFLOW) != 0);
    r.metrics = failed ? 0u : metrics;
    r.crossing_path = path;
    r.cell_log2 = cell_log2;
    r.occlusion_path = occl_path;
    // crossings (Algorithms 4 and 5)
    const uint64_t ec = acc->proper + acc->touching;
    r.crossing.c.crossings = (int64_t)ec;
    r.crossing.c.proper = (int64_t)acc->proper;
    r.crossing.c.touching = (int64_t)acc->touching;
    r.crossing.c.collinear_overlaps = (int64_t)acc->collinear;
    r.crossing.c.zero_length_edges = (int64_t)acc->zero_len;
    const uint64_t ns = acc->n_seg;
    if (pairs_tested == -2) {  // grid: candidate pairs of the cells plus the long-long pairs
        const uint64_t nl = acc->n_long;
        r.crossing.c.pairs_tested = (int64_t)(acc->grid_work + nl * (nl - (nl > 0)) / 2);
    } else {
        r.crossing.c.pairs_tested = pairs_tested >= 0 ? pairs_tested : (int64_t)(ns * (ns - (ns > 0)) / 2);
    }
    const double dev = ((double)acc->dev_hi * 18446744073709551616.0 + (double)acc->dev_lo) * kAngleUnit;
    r.crossing.angle_dev_sum = dev;
    r.crossing.ideal_rad = ideal;
    r.crossing.E_ca = ec > 0 ? 1.0 - dev / (ideal * (double)ec) : 1.0;
    r.occlusion_pairs = (int64_t)acc->occlusion;
    r.occlusion_d = d;
    r.min_angle.sum_d = ms;
    r.min_angle.n_vertices_counted = (int64_t)mn;
    r.min_angle.M_a = mn > 0 ? 1.0 - ms / (double)mn : 1.0;
    if ((metrics & GR_METRIC_EDGE_LENGTH) && E > 1) {
        const double mu = sl / (double)E;
        r.M_l = mu > 0.0 ? sqrt(sv / ((double)E * mu * mu)) / sqrt((double)E - 1.0) : 0.0;
    } else {
        r.M_l = 0.0;
    }
    r.grid_records = (int64_t)acc->records;
    *out = r;
}

__global__ void k_per_edge_export(uint64_t *dev_fixed, int64_t E) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)dev_fixed[e] * kAngleUnit;
        reinterpret_cast<double *>(dev_fixed)[e] = v;
    }
}

// a10 per layout: one block per layout (grid-strided), two passes over the
// layout's edges in a fixed order; also counts its zero-length edges.
__global__ void __launch_bounds__(256) k_batch_elv(const int64_t *__restrict__ len2,
                                                   const int64_t *__restrict__ e_off, int64_t L,
                                                   gr_result *__restrict__ res) {
    __shared__ double shd[32];
    __shared__ uint64_t shu[32];
    for (int64_t l = blockIdx.x; l < L; l += gridDim.x) {
        const int64_t e0 = e_off[l], e1 = e_off[l + 1], E = e1 - e0;
        double sl = 0.0;
        uint64_t z = 0;
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int64_t q = len2[e];
            sl += sqrt((double)q);
            z += q == 0;
        }
        sl = block_sum<double>(sl, shd);
        z = block_sum<uint64_t>(z, shu);
        const double mu = E > 0 ? sl / (double)E : 0.0;
        double sv = 0.0;
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const double t = sqrt((double)len2[e]) - mu;
            sv += t * t;
        }
        sv = block_sum<double>(sv, shd);
        if (threadIdx.x == 0) {
            res[l].M_l = (E > 1 && mu > 0.0) ? sqrt(sv / ((double)E * mu * mu)) / sqrt((double)E - 1.0) : 0.0;
            res[l].crossing.c.zero_length_edges = (int64_t)z;
        }
    }
}

// The canonical order of the compacted segments: edge order.  flags[e] = 1
// for an edge that was not kept (zero length, or invalid); after an exclusive
// scan, edge e's segment goes to e - flags[e].
__global__ void __launch_bounds__(256) k_drop_flags(const int64_t *__restrict__ len2, int64_t E,
                                                    uint32_t *__restrict__ flags) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        flags[e] = len2[e] == 0 ? 1u : 0u;
}

__global__ void __launch_bounds__(256) k_canon_scatter(const SegRec *__restrict__ seg, const int32_t *__restrict__ eid,
                                                       const uint32_t *__restrict__ theta,
                                                       const DevAcc *__restrict__ acc,
                                                       const uint32_t *__restrict__ dropped_before,
                                                       SegRec *__restrict__ tseg, int32_t *__restrict__ teid,
                                                       uint32_t *__restrict__ ttheta) {
    const int64_t n = acc->n_seg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = eid[i];
        const uint32_t p = (uint32_t)e - dropped_before[e];
        tseg[p] = seg[i];
        teid[p] = e;
        ttheta[p] = theta[i];
    }
}

int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

void launch_gather(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E, Buffers &b,
                   cudaStream_t s) {
    if (E <= 0 && V <= 0) return;
    count_launches(1);
    k_gather<<<grid_for(E > V ? E : V, kGatherThreads, 152 * 16), kGatherThreads, 0, s>>>((const int2 *)xy, V, (const int2 *)edges, E,
                                                        b.seg, b.seg_eid, b.seg_theta, b.len2, b.acc);
}

void launch_canonical_segments(Buffers &b, int64_t E, uint32_t *flags, SegRec *tmp_seg, int32_t *tmp_eid,
                               uint32_t *tmp_theta, cudaStream_t s) {
    if (E <= 0) return;
    count_launches(2);
    k_drop_flags<<<grid_for(E, 256, 152 * 8), 256, 0, s>>>(b.len2, E, flags);
    launch_scan_u32(flags, flags, E, b.scan_tmp, &b.acc->scan_sink, &b.acc->eval_status, s);
    k_canon_scatter<<<grid_for(E, 256, 152 * 8), 256, 0, s>>>(b.seg, b.seg_eid, b.seg_theta, b.acc, flags, tmp_seg,
                                                              tmp_eid, tmp_theta);
    cudaMemcpyAsync(b.seg, tmp_seg, sizeof(SegRec) * E, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(b.seg_eid, tmp_eid, sizeof(int32_t) * E, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(b.seg_theta, tmp_theta, sizeof(uint32_t) * E, cudaMemcpyDeviceToDevice, s);
}

void launch_check_vertices(const int32_t *xy, int64_t V, Buffers &b, cudaStream_t s) {
    if (V <= 0) return;
    count_launches(1);
    k_check_vertices<<<grid_for(V, 256, 152 * 8), 256, 0, s>>>((const int2 *)xy, V, b.acc);
}

void launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *block_tmp,
                     uint64_t *total, uint32_t *status, cudaStream_t s) {
    const int nb = (int)((n + kScanItems - 1) / kScanItems);
    if (nb > kScanMaxBlocks) {  // callers bound n; record it rather than overrun
        count_launches(1);
        k_scan_top<<<1, 1024, 0, s>>>(block_tmp, 0, out, 0, total, status);
        return;
    }
    count_launches(nb > 0 ? 3 : 1);
    if (nb > 0) k_scan_sums<<<nb, 1024, 0, s>>>(in, n, block_tmp);
    k_scan_top<<<1, 1024, 0, s>>>(block_tmp, nb, out, n, total, status);
    if (nb > 0) k_scan_apply<<<nb, 1024, 0, s>>>(in, out, n, block_tmp);
}

void launch_elv(const Buffers &b, int64_t E, cudaStream_t s, bool f32) {
    count_launches(2);
    k_elv_sum<<<kElvBlocks, 256, 0, s>>>(b.len2, E, b.elv_len, b.elv_part, f32);
    k_elv_var<<<kElvBlocks, 256, 0, s>>>(b.elv_len, E, b.elv_part);
}

void launch_batch_elv(const Buffers &b, const BatchView &bv, cudaStream_t s) {
    if (bv.L <= 0) return;
    count_launches(1);
    const int blocks = (int)(bv.L < 152 * 16 ? bv.L : 152 * 16);
    k_batch_elv<<<blocks, 256, 0, s>>>(b.len2, bv.e_off, bv.L, bv.res);
}

void launch_finalize(const Buffers &b, uint32_t metrics, int64_t E, double ideal, int64_t d,
                     int ma_blocks, int32_t path, int32_t cell_log2, int32_t occl_path,
                     int64_t pairs_tested, cudaStream_t s) {
    count_launches(1);
    k_finalize<<<1, 256, 0, s>>>(b.acc, b.elv_part, b.ma_part, b.ma_cnt, ma_blocks, metrics, E, ideal,
                                 d, path, cell_log2, occl_path, pairs_tested, b.result);
}

void launch_per_edge_export(uint64_t *dev_fixed, int64_t E, cudaStream_t s) {
    if (E <= 0) return;
    count_launches(1);
    k_per_edge_export<<<grid_for(E, 256, 152 * 8), 256, 0, s>>>(dev_fixed, E);
}

}  // namespace gr
