// k_strip.cu -- the paper's approximate "enhanced" crossing and crossing-angle
// algorithms (Sec. 3.2.2-3.2.3), on the GPU.
//
// The plane is cut by the lines x = s l (vertical strips; horizontal ones
// exchange x and y).  A segment that crosses both lines of strip s gives the
// record (s, l_i, r_i, theta_i): its y at the two lines, as the exact integer
// keys floor(y * 2^30), and its line direction.  Within a strip two such
// segments cross exactly when their order reverses from the left line to the
// right one, so the strip's count is the number of inversions between the
// (l, r) order and the r order.  The paper sweeps a sorted array with a
// balanced tree (O(n log n)) and, for the angles, a 2-D segment tree over
// (r, theta) with 8 angle categories (Eq. 1, O(n log^2 n)).  Here:
//   1. span: per segment the strips it spans, as +1 / -1 marks per strip;
//   2. layout: one block turns the marks into strip sizes, record offsets and
//      tile offsets (tiles of ST_TILE records never straddle two strips);
//   3. emit: the records, scattered into their strips;
//   4. sort by (l, r) within each strip: every tile merge-sorted in shared
//      memory, then global merge levels of doubling run length;
//   5. merge sort by r within each strip (tiles, then global levels) that
//      counts, for each element of a right run, the elements of its left run
//      with a greater r -- the inverted pairs -- and adds |ideal - angle| of
//      each such pair (integer direction units, as in the exact path).
// The sum over the counted pairs is the quantity Eq. 1 computes from the
// category sums; it is formed per pair here, which costs one step per
// counted pair and needs no per-category structure.
#include "gr_internal.cuh"
#include "pair_math.cuh"

namespace gr {

namespace {

constexpr int ST_THREADS = 256;
constexpr int ST_TILE = 2048;          // records per shared-memory tile
constexpr int ST_TILE_THREADS = 512;   // threads of the tile kernel (two blocks per SM)
constexpr int ST_KEY_SHIFT = 30;
constexpr int ST_STRIP_SHIFT = 46;  // k1 = strip << 46 | l key (keys < 2^46)

// Endpoints of segment r with the strip axis first (orient 1 exchanges x and
// y), ordered so that x0 <= x1.
struct StripSeg {
    int x0, y0, x1, y1;
};

__device__ __forceinline__ StripSeg strip_seg(SegRec r, int orient) {
    int ax = px(r.x), ay = py(r.x), bx = px(r.y), by = py(r.y);
    if (orient) {
        int t = ax; ax = ay; ay = t;
        t = bx; bx = by; by = t;
    }
    if (ax > bx) {
        int t = ax; ax = bx; bx = t;
        t = ay; ay = by; by = t;
    }
    return StripSeg{ax, ay, bx, by};
}

// floor(y(X) * 2^30), x0 < x1, x0 <= X <= x1: num = y(X) dx = y0 dx + (X - x0)
// dy is an integer in [0, 2^32), so the key floor(num 2^30 / dx) is exact.
// Without a 64-bit division per record: with inv = floor(2^47 / dx) (one
// division per segment), num = q dx + r and r < dx < 2^16,
// floor(r 2^30 / dx) is floor(r 2^30 inv / 2^47) or one more (the estimate
// is low by less than r / 2^17 < 1), settled by one exact comparison.
struct KeyDiv {
    uint32_t dx;
    uint64_t inv;
};

__device__ __forceinline__ KeyDiv key_div(const StripSeg &s) {
    const uint32_t dx = (uint32_t)(s.x1 - s.x0);
    return KeyDiv{dx, (1ull << 47) / dx};
}

__device__ __forceinline__ uint64_t strip_key_fast(const StripSeg &s, const KeyDiv &kd, int X) {
    const long long dy = s.y1 - s.y0;
    const uint32_t num = (uint32_t)((long long)s.y0 * kd.dx + (long long)(X - s.x0) * dy);
    const uint32_t q = num / kd.dx, r = num - q * kd.dx;
    const uint64_t rs = (uint64_t)r << ST_KEY_SHIFT;
    uint64_t t = __umul64hi(rs, kd.inv << 17);
    if ((t + 1) * kd.dx <= rs) ++t;
    return ((uint64_t)q << ST_KEY_SHIFT) + t;
}

// Strips [s0, s1] whose two lines lie within the segment's x range (none when
// s1 < s0).
__device__ __forceinline__ void strip_range(const StripSeg &s, int l, int &s0, int &s1) {
    if (s.x0 == s.x1) {
        s0 = 1;
        s1 = 0;
        return;
    }
    s0 = (s.x0 + l - 1) / l;
    s1 = s.x1 / l - 1;
}

__global__ void __launch_bounds__(ST_THREADS) k_strip_span(const SegRec *__restrict__ seg,
                                                           const DevAcc *__restrict__ acc, int l, int orient,
                                                           uint32_t *__restrict__ mark_start,
                                                           uint32_t *__restrict__ mark_end, StripAcc *sacc) {
    __shared__ uint64_t shu[32];
    const int64_t n = acc->n_seg;
    uint64_t recs = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const StripSeg s = strip_seg(seg[i], orient);
        int s0, s1;
        strip_range(s, l, s0, s1);
        if (s1 < s0) continue;
        atomicAdd(&mark_start[s0], 1u);
        atomicAdd(&mark_end[s1 + 1], 1u);
        recs += (uint64_t)(s1 - s0 + 1);
    }
    recs = block_sum<uint64_t>(recs, shu);
    if (threadIdx.x == 0 && recs) atomic_add_u64(&sacc->records, recs);
}

// Exclusive scan over the block (1024 threads) of one value per thread.
__device__ __forceinline__ uint64_t block_excl_scan_1024(uint64_t v, uint64_t *sh, uint64_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const uint64_t w = sh[lane];
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    *total = sh[32];
    return sh[wid] + x - v;
}

// One block of 1024 threads: strip sizes n_s = sum over s' <= s of
// (starts - ends), then the record offsets (strip_off[0..ns]) and the tile
// offsets (tile_off[0..ns], ceil(n_s / ST_TILE) tiles per strip), the tile
// total and the largest strip.
__global__ void __launch_bounds__(1024) k_strip_layout(const uint32_t *__restrict__ mark_start,
                                                       const uint32_t *__restrict__ mark_end, int ns,
                                                       uint32_t *__restrict__ strip_off,
                                                       uint32_t *__restrict__ tile_off, StripAcc *sacc) {
    __shared__ uint64_t sh[33];
    const int per = (ns + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(ns, b + per);
    // pass 1: running sizes
    long long d = 0;
    for (int s = b; s < e; ++s) d += (long long)mark_start[s] - (long long)mark_end[s];
    uint64_t tot;
    const long long run0 = (long long)block_excl_scan_1024((uint64_t)d, sh, &tot);
    // pass 2: sizes -> offsets of records and tiles
    long long run = run0;
    uint64_t nrec = 0, ntile = 0;
    uint32_t mx = 0;
    for (int s = b; s < e; ++s) {
        run += (long long)mark_start[s] - (long long)mark_end[s];
        const uint64_t n = (uint64_t)run;
        nrec += n;
        ntile += (n + ST_TILE - 1) / ST_TILE;
        mx = max(mx, (uint32_t)n);
    }
    uint64_t rtot, ttot;
    uint64_t roff = block_excl_scan_1024(nrec, sh, &rtot);
    uint64_t toff = block_excl_scan_1024(ntile, sh, &ttot);
    run = run0;
    for (int s = b; s < e; ++s) {
        run += (long long)mark_start[s] - (long long)mark_end[s];
        const uint64_t n = (uint64_t)run;
        strip_off[s] = (uint32_t)roff;
        tile_off[s] = (uint32_t)toff;
        roff += n;
        toff += (n + ST_TILE - 1) / ST_TILE;
    }
    if (threadIdx.x == 1023) {
        strip_off[ns] = (uint32_t)rtot;
        tile_off[ns] = (uint32_t)ttot;
        sacc->tiles = (uint32_t)ttot;
        if (rtot > 0xffffffffull) atomicOr(&sacc->status, ST_SCAN_OVERFLOW);
    }
    // largest strip
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&sacc->max_n, mx);
}

// The records of the segments: a warp walks the union of its 32 segments'
// strip ranges in order, so that for each strip one atomic reserves the
// slots of all its lanes that span it and their records are stored side by
// side; the key at a line is computed once and serves as the right key of one
// strip and the left key of the next.
__global__ void __launch_bounds__(ST_THREADS) k_strip_emit(const SegRec *__restrict__ seg,
                                                           const uint32_t *__restrict__ seg_theta,
                                                           const DevAcc *__restrict__ acc, int l, int orient,
                                                           const uint32_t *__restrict__ strip_off,
                                                           uint32_t *__restrict__ fill, uint64_t cap,
                                                           uint64_t *__restrict__ k1, uint64_t *__restrict__ rk,
                                                           uint32_t *__restrict__ th, StripAcc *sacc) {
    const int64_t n = acc->n_seg;
    const int lane = threadIdx.x & 31;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        StripSeg s{0, 0, 0, 0};
        int s0 = 1, s1 = 0;
        uint32_t t = 0;
        if (i < n) {
            s = strip_seg(seg[i], orient);
            strip_range(s, l, s0, s1);
            t = seg_theta[i];
        }
        const bool any = s1 >= s0;
        const KeyDiv kd = any ? key_div(s) : KeyDiv{1u, 0ull};
        const int lo = __reduce_min_sync(0xffffffffu, any ? s0 : 0x7fffffff);
        const int hi = __reduce_max_sync(0xffffffffu, any ? s1 : -1);
        uint64_t kl = any ? strip_key_fast(s, kd, s0 * l) : 0ull;
        for (int q = lo; q <= hi; ++q) {
            const bool act = s0 <= q && q <= s1;
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if (!m) continue;
            uint32_t slot = 0;
            if (lane == __ffs(m) - 1) slot = atomicAdd(&fill[q], (uint32_t)__popc(m));
            slot = __shfl_sync(0xffffffffu, slot, __ffs(m) - 1);
            if (!act) continue;
            const uint64_t kr = strip_key_fast(s, kd, (q + 1) * l);
            const uint64_t pos = (uint64_t)strip_off[q] + slot + __popc(m & lt);
            if (pos < cap) {
                k1[pos] = ((uint64_t)q << ST_STRIP_SHIFT) | kl;
                rk[pos] = kr;
                th[pos] = t;
            } else {  // sized from the same count; never expected
                atomicOr(&sacc->status, ST_OVERFLOW);
            }
            kl = kr;
        }
    }
}

// Order of the (l, r) sort (k1 holds the strip above the l key), and of the r
// merge.
template <bool INV>
__device__ __forceinline__ bool key_less(uint64_t ak1, uint64_t ark, uint64_t bk1, uint64_t brk) {
    if (INV) return ark < brk;
    return ak1 < bk1 || (ak1 == bk1 && ark < brk);
}

// Position of element x of a run in the merge with its sibling run
// [sb, sb + sn) (accessed through `at`): left-run elements go before equal
// right-run ones (a stable merge).
template <bool INV, class F>
__device__ __forceinline__ uint32_t sibling_rank(uint64_t xk1, uint64_t xrk, bool left, uint32_t sn, F &&at) {
    uint32_t lo = 0, hi = sn;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        uint64_t k1, rk;
        at(mid, k1, rk);
        // left: count sibling < x; right: count sibling <= x
        const bool before = left ? key_less<INV>(k1, rk, xk1, xrk) : !key_less<INV>(xk1, xrk, k1, rk);
        if (before) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Sum of |ideal - angle| of direction xt against directions y[0, n) (shared
// memory).
__device__ __forceinline__ uint64_t dev_sum(uint32_t xt, const uint32_t *y, uint32_t n, uint32_t ideal) {
    uint64_t a = 0;
    for (uint32_t m = 0; m < n; ++m) a += dev_term(xt, y[m], ideal);
    return a;
}

struct StripTotals {
    uint64_t count = 0, dev = 0;
};

__device__ __forceinline__ void flush_strip_totals(const StripTotals &t, StripAcc *sacc, uint64_t *sh) {
    const uint64_t c = block_sum<uint64_t>(t.count, sh);
    const uint64_t d = block_sum<uint64_t>(t.dev, sh);
    if (threadIdx.x == 0) {
        if (c) atomic_add_u64(&sacc->count, c);
        if (d) add_u128(&sacc->dev_lo, &sacc->dev_hi, d);
    }
}

// One tile of at most ST_TILE records of one strip, merge-sorted in shared
// memory from runs of 1 (INV: by r, counting and summing the inverted pairs;
// else by (l, r)).
template <bool INV>
__global__ void __launch_bounds__(ST_TILE_THREADS) k_strip_tile(const uint64_t *__restrict__ k1_in,
                                                           const uint64_t *__restrict__ rk_in,
                                                           const uint32_t *__restrict__ th_in,
                                                           uint64_t *__restrict__ k1_out,
                                                           uint64_t *__restrict__ rk_out,
                                                           uint32_t *__restrict__ th_out,
                                                           const uint32_t *__restrict__ strip_off,
                                                           const uint32_t *__restrict__ tile_off, int ns,
                                                           uint32_t ideal, StripAcc *sacc) {
    extern __shared__ __align__(16) unsigned char st_smem[];
    uint64_t *ak1 = (uint64_t *)st_smem;
    uint64_t *ark = ak1 + ST_TILE;
    uint64_t *bk1 = ark + ST_TILE;
    uint64_t *brk = bk1 + ST_TILE;
    uint32_t *ath = (uint32_t *)(brk + ST_TILE);
    uint32_t *bth = ath + ST_TILE;
    __shared__ uint64_t shu[32];
    StripTotals tot;
    const uint32_t tiles = sacc->tiles;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int lo = 0, hi = ns;  // the strip s with tile_off[s] <= t < tile_off[s + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tile_off[mid] <= t) lo = mid; else hi = mid;
        }
        const uint32_t start = strip_off[lo] + (t - tile_off[lo]) * ST_TILE;
        const uint32_t n = min((uint32_t)ST_TILE, strip_off[lo + 1] - start);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += ST_TILE_THREADS) {
            ak1[i] = k1_in[start + i];
            ark[i] = rk_in[start + i];
            ath[i] = th_in[start + i];
        }
        __syncthreads();
        uint64_t *sk1 = ak1, *srk = ark, *dk1 = bk1, *drk = brk;
        uint32_t *sth = ath, *dth = bth;
        for (uint32_t w = 1; w < n; w <<= 1) {
            for (uint32_t i = threadIdx.x; i < n; i += ST_TILE_THREADS) {
                const uint32_t run = i / w, rb = run * w, sib = run ^ 1u, sb = sib * w;
                const uint32_t sn = sb < n ? min(w, n - sb) : 0u;
                const bool left = (run & 1u) == 0u;
                const uint64_t xk1 = sk1[i], xrk = srk[i];
                const uint32_t rank = sibling_rank<INV>(xk1, xrk, left, sn, [&](uint32_t m, uint64_t &k1, uint64_t &rk) {
                    k1 = sk1[sb + m];
                    rk = srk[sb + m];
                });
                const uint32_t pos = (run & ~1u) * w + (i - rb) + rank;
                dk1[pos] = xk1;
                drk[pos] = xrk;
                dth[pos] = sth[i];
                if (INV && !left) {  // left-run elements with a greater r: inverted pairs
                    tot.count += sn - rank;
                    tot.dev += dev_sum(sth[i], sth + sb + rank, sn - rank, ideal);
                }
            }
            __syncthreads();
            uint64_t *t1 = sk1; sk1 = dk1; dk1 = t1;
            t1 = srk; srk = drk; drk = t1;
            uint32_t *t2 = sth; sth = dth; dth = t2;
        }
        for (uint32_t i = threadIdx.x; i < n; i += ST_TILE_THREADS) {
            k1_out[start + i] = sk1[i];
            rk_out[start + i] = srk[i];
            th_out[start + i] = sth[i];
        }
    }
    if (INV) flush_strip_totals(tot, sacc, shu);
}

// Merge path of every chunk of a global merge level (see k_strip_merge):
// for chunk t, how many of the outputs before its start (2t) and before its
// end (2t + 1) come from the left run, one thread per entry so that the
// binary searches' global loads overlap.
template <bool INV>
__global__ void __launch_bounds__(ST_THREADS) k_strip_splits(const uint64_t *__restrict__ k1_in,
                                                             const uint64_t *__restrict__ rk_in,
                                                             const uint32_t *__restrict__ strip_off,
                                                             const uint32_t *__restrict__ tile_off, int ns,
                                                             uint32_t w, const StripAcc *__restrict__ sacc,
                                                             uint32_t *__restrict__ split) {
    const uint32_t tiles = sacc->tiles;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * tiles; q += gridDim.x * blockDim.x) {
        const uint32_t t = q >> 1;
        int lo_s = 0, hi_s = ns;
        while (hi_s - lo_s > 1) {
            const int mid = (lo_s + hi_s) >> 1;
            if (tile_off[mid] <= t) lo_s = mid; else hi_s = mid;
        }
        const uint32_t S0 = strip_off[lo_s], n = strip_off[lo_s + 1] - S0;
        const uint32_t o0 = (t - tile_off[lo_s]) * ST_TILE, o1 = min(o0 + ST_TILE, n);
        const uint32_t p0 = o0 / (2 * w) * (2 * w);
        const uint32_t la = min(w, n - p0), lb = n > p0 + w ? min(w, n - p0 - w) : 0u;
        const uint64_t *ak1 = k1_in + S0 + p0, *ark = rk_in + S0 + p0;
        const uint64_t *bk1 = ak1 + w, *brk = ark + w;
        const uint32_t k = ((q & 1u) ? o1 : o0) - p0;
        uint32_t lo = k > lb ? k - lb : 0u, hi = min(k, la);
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            const uint32_t j = k - mid - 1;
            // left[mid] goes first unless right[j] is smaller
            if (!key_less<INV>(INV ? 0ull : bk1[j], brk[j], INV ? 0ull : ak1[mid], ark[mid])) lo = mid + 1;
            else hi = mid;
        }
        split[q] = lo;
    }
}

// One global merge level: within each strip, runs of w records (w >= ST_TILE,
// a multiple of it) merged pairwise.  The output of a strip is cut into
// chunks of ST_TILE records (the tiles of the strip; a pair of runs covers
// whole chunks); each block takes a chunk, reads how many of its outputs come
// from the left run (merge path, from k_strip_splits), loads both input
// slices into shared memory (coalesced), places every
// element by a binary search in the other slice and stores the chunk
// (coalesced).  INV: a right-run element x is preceded by the left-run
// elements with a greater r: those of the chunk's left slice past x's place,
// and every left-run element after the slice (all of them follow the whole
// chunk, so their r is greater than any of its right-run elements) -- the
// latter are streamed through shared memory in batches against all of the
// chunk's right-run elements.
template <bool INV>
__global__ void __launch_bounds__(ST_TILE_THREADS) k_strip_merge(const uint64_t *__restrict__ k1_in,
                                                                 const uint64_t *__restrict__ rk_in,
                                                                 const uint32_t *__restrict__ th_in,
                                                                 uint64_t *__restrict__ k1_out,
                                                                 uint64_t *__restrict__ rk_out,
                                                                 uint32_t *__restrict__ th_out,
                                                                 const uint32_t *__restrict__ strip_off,
                                                                 const uint32_t *__restrict__ tile_off, int ns,
                                                                 uint32_t w, const uint32_t *__restrict__ split,
                                                                 uint32_t ideal, StripAcc *sacc) {
    extern __shared__ __align__(16) unsigned char st_smem[];
    uint64_t *ck1 = (uint64_t *)st_smem;   // chunk inputs: left slice, then right slice
    uint64_t *crk = ck1 + ST_TILE;
    uint64_t *ok1 = crk + ST_TILE;         // chunk outputs
    uint64_t *ork = ok1 + ST_TILE;
    uint32_t *cth = (uint32_t *)(ork + ST_TILE);
    uint32_t *oth = cth + ST_TILE;
    __shared__ uint64_t shu[32];
    StripTotals tot;
    const uint32_t tiles = sacc->tiles;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int lo_s = 0, hi_s = ns;
        while (hi_s - lo_s > 1) {
            const int mid = (lo_s + hi_s) >> 1;
            if (tile_off[mid] <= t) lo_s = mid; else hi_s = mid;
        }
        const uint32_t S0 = strip_off[lo_s], n = strip_off[lo_s + 1] - S0;
        const uint32_t o0 = (t - tile_off[lo_s]) * ST_TILE, o1 = min(o0 + ST_TILE, n);
        const uint32_t p0 = o0 / (2 * w) * (2 * w);
        const uint32_t la = min(w, n - p0), lb = n > p0 + w ? min(w, n - p0 - w) : 0u;
        const uint64_t *ak1 = k1_in + S0 + p0, *ark = rk_in + S0 + p0;
        const uint64_t *bk1 = ak1 + w, *brk = ark + w;
        const uint32_t *ath = th_in + S0 + p0, *bth = ath + w;
        if (lb == 0) {  // no right run: the chunk keeps its place
            for (uint32_t i = o0 + threadIdx.x; i < o1; i += ST_TILE_THREADS) {
                k1_out[S0 + i] = k1_in[S0 + i];
                rk_out[S0 + i] = rk_in[S0 + i];
                th_out[S0 + i] = th_in[S0 + i];
            }
            continue;
        }
        __syncthreads();  // the previous chunk is done with the shared arrays
        const uint32_t i0 = split[2 * t], i1 = split[2 * t + 1];
        const uint32_t j0 = (o0 - p0) - i0, j1 = (o1 - p0) - i1;
        const uint32_t na = i1 - i0, nb = j1 - j0;
        for (uint32_t e = threadIdx.x; e < na + nb; e += ST_TILE_THREADS) {
            if (e < na) {
                ck1[e] = INV ? 0ull : ak1[i0 + e];
                crk[e] = ark[i0 + e];
                cth[e] = ath[i0 + e];
            } else {
                ck1[e] = INV ? 0ull : bk1[j0 + e - na];
                crk[e] = brk[j0 + e - na];
                cth[e] = bth[j0 + e - na];
            }
        }
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < na + nb; e += ST_TILE_THREADS) {
            const bool left = e < na;
            const uint64_t xk1 = ck1[e], xrk = crk[e];
            const uint32_t sb = left ? na : 0u, sn = left ? nb : na;
            const uint32_t rank = sibling_rank<INV>(xk1, xrk, left, sn, [&](uint32_t m, uint64_t &k1, uint64_t &rk) {
                k1 = ck1[sb + m];
                rk = crk[sb + m];
            });
            const uint32_t pos = (left ? e : e - na) + rank;
            ok1[pos] = xk1;
            ork[pos] = xrk;
            oth[pos] = cth[e];
            if (INV && !left) {
                tot.count += la - i0 - rank;  // left elements with a greater r, in the slice and after it
                tot.dev += dev_sum(cth[e], cth + rank, na - rank, ideal);
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < na + nb; i += ST_TILE_THREADS) {
            if (!INV) k1_out[S0 + o0 + i] = ok1[i];  // (the r merge needs no l key)
            rk_out[S0 + o0 + i] = ork[i];
            th_out[S0 + o0 + i] = oth[i];
        }
        if (INV && i1 < la) {
            // left-run elements after the slice, in batches (oth is free now), against the right slice
            for (uint32_t g0 = i1; g0 < la; g0 += ST_TILE) {
                const uint32_t gn = min((uint32_t)ST_TILE, la - g0);
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < gn; i += ST_TILE_THREADS) oth[i] = ath[g0 + i];
                __syncthreads();
                for (uint32_t e = na + threadIdx.x; e < na + nb; e += ST_TILE_THREADS)
                    tot.dev += dev_sum(cth[e], oth, gn, ideal);
            }
        }
    }
    if (INV) flush_strip_totals(tot, sacc, shu);
}

int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

constexpr size_t kTileSmem = (size_t)ST_TILE * (8 + 8 + 8 + 8 + 4 + 4);  // tile and merge kernels alike

}  // namespace

int strip_count(int l) { return 65536 / l + 1; }

void launch_strip_span(const Buffers &b, int64_t E, int l, int orient, const StripBuffers &sb, cudaStream_t s) {
    count_launches(1);
    k_strip_span<<<grid_for(E, ST_THREADS, 152 * 8), ST_THREADS, 0, s>>>(b.seg, b.acc, l, orient, sb.mark_start,
                                                                        sb.mark_end, sb.acc);
    count_launches(1);
    k_strip_layout<<<1, 1024, 0, s>>>(sb.mark_start, sb.mark_end, strip_count(l), sb.strip_off, sb.tile_off,
                                      sb.acc);
}

void launch_strip_sort(const Buffers &b, int64_t E, int l, int orient, StripBuffers &sb, uint32_t max_n,
                       cudaStream_t s) {
    // (cheap, and set on every call: the current device may change between calls)
    cudaFuncSetAttribute(k_strip_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_strip_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_strip_merge<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_strip_merge<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    const int ns = strip_count(l);
    const uint64_t R = sb.records;
    sb.cur = 0;
    count_launches(1);
    k_strip_emit<<<grid_for(E, ST_THREADS, 152 * 8), ST_THREADS, 0, s>>>(b.seg, b.seg_theta, b.acc, l, orient,
                                                                        sb.strip_off, sb.fill, sb.cap, sb.k1[0],
                                                                        sb.rk[0], sb.th[0], sb.acc);
    if (R == 0) return;
    const int tb = grid_for((int64_t)sb.tiles, 1, 152 * 2);
    int cur = 0;
    count_launches(1);
    k_strip_tile<false><<<tb, ST_TILE_THREADS, kTileSmem, s>>>(sb.k1[cur], sb.rk[cur], sb.th[cur], sb.k1[cur ^ 1],
                                                          sb.rk[cur ^ 1], sb.th[cur ^ 1], sb.strip_off, sb.tile_off,
                                                          ns, 0u, sb.acc);
    cur ^= 1;
    for (uint32_t w = ST_TILE; w < max_n; w <<= 1) {
        count_launches(2);
        k_strip_splits<false><<<grid_for(2 * (int64_t)sb.tiles, ST_THREADS, 152 * 8), ST_THREADS, 0, s>>>(
            sb.k1[cur], sb.rk[cur], sb.strip_off, sb.tile_off, ns, w, sb.acc, sb.split);
        k_strip_merge<false><<<tb, ST_TILE_THREADS, kTileSmem, s>>>(sb.k1[cur], sb.rk[cur], sb.th[cur],
                                                                    sb.k1[cur ^ 1], sb.rk[cur ^ 1], sb.th[cur ^ 1],
                                                                    sb.strip_off, sb.tile_off, ns, w, sb.split, 0u, sb.acc);
        cur ^= 1;
    }
    sb.cur = cur;
}

void launch_strip_inversions(int l, StripBuffers &sb, uint32_t max_n, uint32_t ideal, cudaStream_t s) {
    const uint64_t R = sb.records;
    if (R == 0) return;
    const int ns = strip_count(l);
    const int tb = grid_for((int64_t)sb.tiles, 1, 152 * 2);
    int cur = sb.cur;
    count_launches(1);
    k_strip_tile<true><<<tb, ST_TILE_THREADS, kTileSmem, s>>>(sb.k1[cur], sb.rk[cur], sb.th[cur], sb.k1[cur ^ 1],
                                                         sb.rk[cur ^ 1], sb.th[cur ^ 1], sb.strip_off, sb.tile_off,
                                                         ns, ideal, sb.acc);
    cur ^= 1;
    for (uint32_t w = ST_TILE; w < max_n; w <<= 1) {
        count_launches(2);
        k_strip_splits<true><<<grid_for(2 * (int64_t)sb.tiles, ST_THREADS, 152 * 8), ST_THREADS, 0, s>>>(
            sb.k1[cur], sb.rk[cur], sb.strip_off, sb.tile_off, ns, w, sb.acc, sb.split);
        k_strip_merge<true><<<tb, ST_TILE_THREADS, kTileSmem, s>>>(sb.k1[cur], sb.rk[cur], sb.th[cur],
                                                                   sb.k1[cur ^ 1], sb.rk[cur ^ 1], sb.th[cur ^ 1],
                                                                   sb.strip_off, sb.tile_off, ns, w, sb.split, ideal, sb.acc);
        cur ^= 1;
    }
    sb.cur = cur;
}

}  // namespace gr
