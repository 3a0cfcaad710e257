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
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
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

}  // namespace

void launch_occlusion_allpairs(const Buffers &b, int64_t V, int64_t d, cudaStream_t s) {
    if (V < 2 || d <= 0) return;
    const int64_t nb = (V + OC_ROWS - 1) / OC_ROWS;
    const int64_t tiles = nb * (nb + 1) / 2;
    // any d beyond the largest possible distance counts every pair
    const long long d2 = d >= 100000 ? (long long)1e11 : (long long)d * d;
    const unsigned grid = (unsigned)(tiles < (int64_t(1) << 30) ? tiles : (int64_t(1) << 30));
    k_occl_allpairs<<<grid, OC_ROWS, 0, s>>>((const int2 *)b.xy, (int)V, d2, b.acc, tiles);
}

}  // namespace gr
