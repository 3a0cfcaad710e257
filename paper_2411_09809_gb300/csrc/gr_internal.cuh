// gr_internal.cuh -- types and launchers shared by the translation units of
// libgr.  Not part of the public ABI (that is include/gr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gr.h"

namespace gr {

// ---------------------------------------------------------------- status bits
// Raised by device-side validation into DevAcc::status.
enum : uint32_t {
    ST_BAD_ID = 1u,       // vertex id outside [0, V) or self-loop
    ST_BAD_COORD = 2u,    // coordinate outside [0, 65536)
    ST_OVERFLOW = 4u,     // a grid record buffer was too small
    ST_SCAN_OVERFLOW = 8u // an exclusive scan total exceeded 2^32 - 1
};

// Angles are held as uint32 in units of pi / 2^32: the direction of a line
// (an angle mod pi) is a point of Z / 2^32, a difference of two directions
// wraps correctly, and the acute angle between two lines is
// min(d, 2^32 - d) <= 2^31.  Every |ideal - a_c| is an integer in these units,
// so the sums over pairs are exact, associative and independent of the
// order pairs are visited in; the quantisation of a direction is < 1e-9 rad.
constexpr double kAngleUnit = 3.14159265358979323846 / 4294967296.0;

// Device-global accumulators.  The first block is written by
// gr_layout_create / gr_layout_update; the rest is zeroed by every
// evaluation (from offsetof(DevAcc, eval_status)).
struct DevAcc {
    uint32_t status;           // ST_* bits raised by input validation
    uint32_t n_seg;            // non-zero-length segments after compaction
    uint64_t zero_len;         // zero-length edges
    uint64_t len_l1;           // sum over segments of |dx| + |dy|
    uint32_t len_hist[16];     // segments by major-axis length in [2^b, 2^(b+1))
    uint64_t l1_hist[16];      // their |dx| + |dy|
    uint32_t f32_hist[64];     // FP32 layouts: segments by major-axis length class ilogb + 48
    uint32_t f32_bounds[4];    // FP32 layouts: bounding box (order-preserving keys: min x, min y, max x, max y)
    uint32_t part_id, n_parts; // the share of the pair work an evaluation does (n_parts 0 or 1: all of it)
    // ---- per evaluation
    uint32_t eval_status;      // ST_* bits raised during an evaluation
    uint32_t grid_flags;       // GF_* bits: the grid path cannot be used
    uint64_t proper;
    uint64_t touching;
    uint64_t collinear;
    uint64_t dev_lo, dev_hi;   // 128-bit sum of |ideal - a_c| in units of pi / 2^32
    uint64_t occlusion;
    uint64_t records;          // grid (edge, cell) records
    uint64_t grid_items;       // pair-kernel work items
    uint64_t grid_work;        // candidate pairs of the grid: short-short and short-long per cell
    uint64_t scan_sink;        // totals nobody reads
    uint32_t n_long;           // long segments (their pairs go to the all-pairs tiles)
    uint32_t pad_;
};

enum : uint32_t {
    GF_ITEMS_OVERFLOW = 1u     // a cell has more than 2^31 tile pairs
};

// One compacted non-zero-length segment: endpoints packed as x | y << 16
// (coordinates are < 2^16) and the two vertex ids.
//   .x = a.x | a.y << 16, .y = b.x | b.y << 16, .z = id(a), .w = id(b)
using SegRec = uint4;

__host__ __device__ inline int px(uint32_t p) { return int(p & 0xffffu); }
__host__ __device__ inline int py(uint32_t p) { return int(p >> 16); }

// Device buffers of a layout (owned; see gr_api.cu).
struct Buffers {
    int32_t *xy = nullptr;        // [V][2]
    int32_t *edges = nullptr;     // [E][2] staging copy of host edges
    SegRec *seg = nullptr;        // [E] compacted segments
    int32_t *seg_eid = nullptr;   // [E] original edge index of seg[i]
    uint32_t *seg_theta = nullptr;// [E] line direction of seg[i] (units of pi / 2^32)
    int64_t *len2 = nullptr;      // [E] squared length of every edge
    DevAcc *acc = nullptr;        // accumulators
    double *elv_part = nullptr;   // [kElvBlocks * 2] per-block FP64 partial sums
    double *elv_len = nullptr;    // [E] l_e, written by the first ELV pass for the second
    double *ma_part = nullptr;    // [ma blocks] per-block sums of d_v
    uint32_t *ma_cnt = nullptr;   // [ma blocks] per-block vertex counts
    uint32_t *deg = nullptr;      // [V + 1] degree, then CSR offsets (scan in place)
    uint32_t *deg_fill = nullptr; // [V]
    int2 *dirs = nullptr;         // [2 E] incident directions by vertex
    uint32_t *adj_off = nullptr;  // [V + 1] single I32 layouts: adjacency offsets (per edge list)
    int32_t *adj = nullptr;       // [2 E] the other endpoint of each incident edge
    uint32_t *ma_nz = nullptr;    // [V] non-zero incident directions of each vertex (at the start of its slots)
    double *ma_dv = nullptr;      // [V] d_v of each vertex (-1: degree < 2, not counted)
    uint32_t *ma_touch = nullptr; // [V] zero between calls (incremental min angle)
    uint32_t *ma_flag = nullptr;  // [1024] min-angle blocks to recompute, zero between calls
    uint2 *seg_ids = nullptr;     // [E] FP32 layouts: vertex ids of seg[i] (seg holds the FP32 endpoints)
    double *dir_ang = nullptr;    // [2 E] FP32 layouts: incident direction angles by vertex
    int32_t *dir_other = nullptr; // [2 E] FP32 layouts: far vertex of each incident direction
    uint64_t *scan_tmp = nullptr; // [kScanMaxBlocks] block sums (crossing stream)
    uint64_t *scan_tmp_side = nullptr; // [kScanMaxBlocks] block sums (side stream)
    gr_result *result = nullptr;  // device copy of the result
};

// One (segment, cell) record of the crossing grid, 32 bytes (one sector):
// .s = the segment (as SegRec), .x = {edge id, line direction, 0, 0}.
struct __align__(32) GridRec {
    uint4 s;
    uint4 x;
};

// Buffers of the uniform grids (crossings and occlusion), grown on demand.
struct GridBuffers {
    uint32_t *cell_off = nullptr;  // [C + 1] counts, then offsets (scan in place)
    uint32_t *cell_nl = nullptr;   // [C] long records per cell
    uint32_t *item_off = nullptr;  // [C + 1] work items per cell, then offsets
    unsigned long long *cell_fill = nullptr; // [C] short (low 32 bits) and long (high) records placed
    GridRec *rec = nullptr;        // [rec_cap] records sorted by cell: short ones first, then long ones
    float4 *rgeo = nullptr;        // [4 rec_cap] the records' FP32 (make_rgeo) and FP16 (make_hgeo) forms
    uint64_t rec_cap = 0;
    uint4 *item_desc = nullptr;    // [2 items_cap] {record offset, records, short records, ti << 16 | tj}, {cell}
    uint64_t items_cap = 0;
    int cells_cap = 0;             // C the cell arrays are sized for
    SegRec *seg_long = nullptr;    // [E] the long segments, their directions and edge ids
    uint32_t *theta_long = nullptr;
    int32_t *eid_long = nullptr;
    // occlusion grid
    uint32_t *ocell_off = nullptr; // [OC + 1]
    uint32_t *ocell_fill = nullptr;// [OC]
    uint32_t *opts = nullptr;      // [V] packed points sorted by cell
    int ocells_cap = 0;
};

// Cost model of the crossing grid, in units of one pair test of the all-pairs
// tiles.  A record (two DDA walks, atomics, a scattered store) costs about
// kRecordCost, a candidate pair in a cell about kCellPairCost (lane
// efficiency, owner tests), a cell kCellCost (count, scan and work-item
// passes); measured on GB300 with the workloads of the benchmark.
constexpr double kRecordCost = 24.0;
constexpr double kCellPairCost = 3.0;
constexpr double kCellCost = 2.0;
constexpr double kSplitCost = 4e6;  // the long list and its all-pairs launch (a few microseconds)

// Estimated cost of the grid path with cells of side 2^k for n segments of
// total L1 length l1, hist_n / hist_l1 their counts and L1 lengths by
// major-axis length class [2^b, 2^(b+1)): records n + L1 / w and candidate
// pairs estimated as for evenly spread records.  With `split`, segments of
// major length >= 2w are long (length in [w, 2w): half of them) and the
// pairs of two long ones go to the all-pairs tiles (n_long^2 / 2); without,
// every pair sharing a cell is a candidate.
inline double grid_cost(double n, double l1, const uint32_t *hist_n, const uint64_t *hist_l1, int k, bool split) {
    double nl = 0.0, ll = 0.0;
    for (int b = 0; b < 16 && split; ++b) {
        const double f = b > k ? 1.0 : (b == k ? 0.5 : 0.0);
        nl += f * (double)hist_n[b];
        ll += f * (double)hist_l1[b];
    }
    const double w = double(1 << k);
    const double R_long = nl + ll / w, R_short = (n - nl) + (l1 - ll) / w;
    const double C = double(65536 >> k) * double(65536 >> k);
    const double pairs = (R_short * R_short / 2.0 + R_short * R_long) / C;
    return kRecordCost * (R_long + R_short) + kCellPairCost * pairs + kCellCost * C + nl * nl / 2.0 +
           (split ? kSplitCost : 0.0);
}

constexpr int kElvBlocks = 512;
constexpr int kScanItems = 4096;      // elements per scan block
constexpr int kScanMaxBlocks = 16384; // => up to 2^26 elements per scan

// ------------------------------------------------------------------ launchers
// All launchers enqueue on `s` and never synchronise.  Each adds the number of
// kernels it launched to the library-wide counter.
void count_launches(int n);
// Sets the message gr_last_error() returns on this host thread.
void set_last_error(const char *msg);

// a1: gathers every edge's endpoints, validates ids and every vertex's
// coordinates (vertices in no edge included), stores the squared length of
// every edge, compacts the non-zero-length segments.
void launch_gather(const int32_t *xy, int64_t V, const int32_t *edges, int64_t E,
                   Buffers &b, cudaStream_t s);
// Validates every vertex coordinate only (the batch path's gather is its own).
void launch_check_vertices(const int32_t *xy, int64_t V, Buffers &b, cudaStream_t s);

// Optional per-edge outputs of the crossing kernels (both nullable together):
// counts [E][3] (proper, touching, collinear) and integer dev sums [E] in
// units of pi / 2^32.
struct PerEdge {
    uint64_t *counts = nullptr;
    uint64_t *dev = nullptr;
};

// a7: tiled all-pairs crossing kernel over the compacted segments.
// `n_seg` is the compacted segment count (read back from the device).
// `ideal` is the ideal crossing angle in units of pi / 2^32 (<= 2^31).
// The same over an arbitrary list of n segments (n read from *n_p on the
// device, at most n_bound; n_bound < 0: unknown on the host, a persistent
// launch sized on the device, aggregate tallies only), tallies into acc.
// With `part0_only`, a partitioned evaluation leaves the whole list to part
// 0 (for lists whose order is not the same on every rank).
void launch_crossings_allpairs_of(const SegRec *seg, const int32_t *eid, const uint32_t *theta, const uint32_t *n_p,
                                  DevAcc *acc, int64_t n_bound, uint32_t ideal, PerEdge pe, cudaStream_t s,
                                  bool part0_only = false);
// Puts the compacted segments (seg, seg_eid, seg_theta) in edge order, the
// order every rank derives alike (the gather's order depends on which block
// reserved its slots first).  `flags` holds E + 1 uint32, the tmp_* arrays E
// entries each.
void launch_canonical_segments(Buffers &b, int64_t E, uint32_t *flags, SegRec *tmp_seg, int32_t *tmp_eid,
                               uint32_t *tmp_theta, cudaStream_t s);
void launch_crossings_allpairs(const Buffers &b, int64_t n_seg, uint32_t ideal, PerEdge pe,
                               cudaStream_t s);

// a2-a4: DDA count, cell offsets, work items (records -> acc->records,
// items -> acc->grid_items, candidate pairs -> acc->grid_work); the long
// segments (spanning more than two major lines of the grid) are, with
// `split`, also copied to g.seg_long / theta_long / eid_long (count ->
// acc->n_long) and their pairs with each other left out of the grid.
void launch_grid_count(const Buffers &b, int64_t E, const GridBuffers &g, int k, bool split, cudaStream_t s);
// Long-long pairs: all-pairs tiles over the long segments (at most n_bound;
// < 0: count known on the device only).
void launch_grid_long_pairs(const Buffers &b, const GridBuffers &g, int64_t n_bound, uint32_t ideal, PerEdge pe,
                            cudaStream_t s);
// a4: scatter of the records into their cells (needs rec_cap >= records).
void launch_grid_scatter(const Buffers &b, int64_t E, const GridBuffers &g, int k, bool split, cudaStream_t s);
// a6: per-cell pair kernel with the owner-cell test.  The item count is read
// on the device (item_off[C]); the kernel does nothing when the records or
// items outgrew their buffers (ST_OVERFLOW is raised by the scatter or the
// descriptor pass).  n_items_hint sizes the launch (0: unknown).
// Without `split`, the work items are rotation items over every pair of each
// cell (k_cell_pairs); with it, tile items over short x short and long x
// short pairs (k_grid_pairs).
void launch_grid_pairs(const Buffers &b, const GridBuffers &g, int k, bool split, uint64_t n_items_hint,
                       uint32_t ideal, PerEdge pe, cudaStream_t s);

// a8 occlusion grid: cell side 2^k >= d.  Count + scan, then scatter + pair
// kernel.
void launch_occlusion_grid_count(const Buffers &b, int64_t V, const GridBuffers &g, int k,
                                 cudaStream_t s);
void launch_occlusion_grid_pairs(const Buffers &b, int64_t V, const GridBuffers &g, int k, int64_t d,
                                 cudaStream_t s);

// a8: all-pairs occlusion (small V or d large).
void launch_occlusion_allpairs(const Buffers &b, int64_t V, int64_t d, cudaStream_t s);

// a9: minimum angle.
// Adjacency CSR of the edge list (b.adj_off, b.adj), once per edge list.
void launch_adjacency(Buffers &b, int64_t V, int64_t E, cudaStream_t s);
// Minimum angle of a single I32 layout (needs the adjacency): per-block
// partials into b.ma_part / b.ma_cnt.
void launch_min_angle(Buffers &b, int64_t V, int64_t E, cudaStream_t s);
// The same after vertices ids[0, n) moved (b.xy updated), when b.ma_part
// holds the partials of the layout before the move: only the blocks holding
// a moved vertex or a neighbour of one are recomputed.
void launch_min_angle_moved(Buffers &b, int64_t V, const int32_t *ids, const int64_t *np, int64_t cap,
                            cudaStream_t s);
int min_angle_blocks(int64_t V);
// Uploads the FP64 sector table of the minimum-angle kernels (cosine and
// sine of 256 evenly spaced angles) to the current device, ordered on s.
cudaError_t init_min_angle_table(cudaStream_t s);

// a10: edge length variation, two passes of deterministic FP64 partials.
// `f32`: len2 holds FP64 squared lengths (as bits) instead of int64.
void launch_elv(const Buffers &b, int64_t E, cudaStream_t s, bool f32 = false);

// Exclusive scan of n uint32 values in place into out[0..n] (out[n] = total).
// `in` and `out` may alias.  The total also goes to *total (device).
void launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *block_tmp,
                     uint64_t *total, uint32_t *status, cudaStream_t s);

// a11: folds all accumulators into b.result (device).
void launch_finalize(const Buffers &b, uint32_t metrics, int64_t E, double ideal,
                     int64_t d, int ma_blocks, int32_t path, int32_t cell_log2,
                     int32_t occl_path, int64_t pairs_tested, cudaStream_t s);

// Per-edge output conversion: integer dev sums to radians (double), in place.
void launch_per_edge_export(uint64_t *dev_fixed, int64_t E, cudaStream_t s);

// ---------------------------------------------- approximate strip algorithm
struct StripAcc {
    uint64_t records;       // (segment, strip) records
    uint64_t count;         // inverted pairs (the E_c estimate)
    uint64_t dev_lo, dev_hi;// 128-bit sum of their angle terms, units of pi / 2^32
    uint32_t tiles;         // shared-memory tiles over all strips
    uint32_t max_n;         // records of the largest strip
    uint32_t status;        // ST_* bits
    uint32_t pad_;
};
struct StripBuffers {
    uint32_t *mark_start = nullptr, *mark_end = nullptr;  // [ns + 1] segments starting / past their last strip
    uint32_t *strip_off = nullptr, *tile_off = nullptr;   // [ns + 1]
    uint32_t *fill = nullptr;                             // [ns + 1]
    int ns_cap = 0;
    uint64_t *k1[2] = {nullptr, nullptr};  // strip << 46 | key at the left line
    uint64_t *rk[2] = {nullptr, nullptr};  // key at the right line
    uint32_t *th[2] = {nullptr, nullptr};  // line direction
    uint64_t cap = 0;
    uint32_t *split = nullptr;             // [2 tiles] merge-path splits of a global merge level
    uint64_t split_cap = 0;
    StripAcc *acc = nullptr;
    uint64_t records = 0;  // host copies for the launches
    uint32_t tiles = 0;
    int cur = 0;           // which of the two record arrays holds the current order
};
int strip_count(int l);  // strips of width l covering [0, 65536): the span marks need strip_count + 1
// Marks the strips each segment spans and lays out the strips (offsets,
// tiles, records, largest strip into sb.acc).
void launch_strip_span(const Buffers &b, int64_t E, int l, int orient, const StripBuffers &sb, cudaStream_t s);
// Emits the records (sb.records of them, sb.cap >= that) and sorts each strip
// by (l, r) (max_n: records of the largest strip); sb.cur names the result.
void launch_strip_sort(const Buffers &b, int64_t E, int l, int orient, StripBuffers &sb, uint32_t max_n,
                       cudaStream_t s);
// Merge sort by r within each strip, counting the inverted pairs and their
// angle terms into sb.acc.
void launch_strip_inversions(int l, StripBuffers &sb, uint32_t max_n, uint32_t ideal, cudaStream_t s);

// ------------------------------------------------------ incremental moves
// Tallies of the pairs that involve moved vertices, before (k[0]) and after
// (k[1]) the move.
struct DeltaCounts {
    uint64_t proper, touching, collinear, dev_lo, dev_hi, occlusion;
};
// Device-resident inputs of a move, so that a captured move replays for any
// count: the number of moved vertices and the totals it updates.
struct MoveParams {
    int64_t n;
    DeltaCounts last;
};
struct DeltaAcc {
    uint32_t status;      // ST_* bits from the validation of the moves
    uint32_t n_affected;  // edges with a moved endpoint
    uint64_t tested;      // crossing pairs classified in both passes
    uint32_t fallback;    // the dirty list overflowed: the counts are incomplete (a full evaluation follows)
    uint32_t pad_;
    DeltaCounts k[2];
};

// Edges moved since the crossing grid was built ("dirty"): their grid
// records are stale, so the incremental passes take them from a list of
// their own.  dirty[e] flags membership, list[0, *n) holds them (n may pass
// cap, which raises DeltaAcc::fallback).
struct DirtySet {
    uint8_t *flag = nullptr;  // [E]
    uint32_t *list = nullptr; // [cap]
    uint32_t *n = nullptr;    // device count
    uint32_t cap = 0;
};

// Marks the moved vertices in `moved` (zero on entry), checking ids and new
// coordinates (device arrays, *np entries; grids sized for cap) into
// d->status.
void launch_delta_validate(const int32_t *ids, const int32_t *xy_new, const int64_t *np, int64_t cap, int64_t V,
                           uint32_t *moved, DeltaAcc *d, cudaStream_t s);
void launch_delta_unmark(const int32_t *ids, const int64_t *np, int64_t cap, int64_t V, uint32_t *moved,
                         cudaStream_t s);
// Lists the edges with a moved endpoint (count -> d->n_affected); with a
// dirty set (flag != nullptr), also adds the ones not yet in it.
void launch_delta_affected(const Buffers &b, int64_t E, const uint32_t *moved, uint32_t *affected, DeltaAcc *d,
                           const DirtySet &ds, cudaStream_t s);
// The crossing part of a pass through the grid of the last full evaluation
// (cell side 2^k, GridBuffers cell_off and rec as it left them): the affected
// edges against every clean edge via the cells, and against the dirty list.
void launch_delta_grid_pass(const Buffers &b, const GridBuffers &g, int k, const uint32_t *moved,
                            const uint32_t *affected, const DirtySet &ds, uint32_t ideal, DeltaAcc *d, int which,
                            cudaStream_t s);
// Tallies into d->k[which] the crossing pairs of the affected edges and the
// occlusion pairs of the moved vertices, on the coordinates in b.xy; the
// gathered segments (b.seg, b.seg_eid, b.seg_theta, b.acc->n_seg) must be
// those of the same coordinates.  Does nothing once d->status is set.
void launch_delta_pass(const Buffers &b, int64_t V, int64_t E, const int32_t *ids, const int64_t *np,
                       const uint32_t *moved, const uint32_t *affected, bool crossings, uint32_t ideal, bool occlusion,
                       long long d2, DeltaAcc *d, int which, cudaStream_t s);
// Writes the new coordinates of the moved vertices into b.xy (unless
// d->status reports an invalid move).
void launch_delta_apply(const int32_t *ids, const int32_t *xy_new, const int64_t *np, int64_t cap, const DeltaAcc *d,
                        Buffers &b, cudaStream_t s);
// The evaluation part of b.acc = *last - k[0] + k[1] (last: device memory;
// nothing when d->status reports an invalid move).
void launch_delta_combine(const DeltaCounts *last, const DeltaAcc *d, Buffers &b, cudaStream_t s);

// ------------------------------------------------------ differentiable form
// What the backward needs from the forward, on the device.
struct DiffState {
    int64_t ec;        // E_c
    double ideal;      // radians
    double E_ca;
    double mu, S, M_l; // mean length, sum (l - mu)^2, M_l
    int64_t n_ma;      // vertices counted by M_a
    double M_a;
};

// a1 for FP32 coordinates (finite values; ids checked).
void launch_gather_f32(const float *xy, int64_t V, const int32_t *edges, int64_t E, Buffers &b, cudaStream_t s);
// a7 on FP32 coordinates with exact predicates.  With `cnt` (zeroed by the
// caller, one int32 per compacted segment), every E_c pair also adds the sign
// of its crossing angle's term (diff_sign: +-1 or 0) to its first segment's
// count and subtracts it from the second's, the E_ca adjoint the backward
// scales.  The same through a G x G grid over the segments' bounding box
// (short x short pairs in cells, long x short along the long segments' walks,
// long x long on all-pairs tiles); `work` holds f32_grid_bytes(G, E) bytes.
size_t f32_grid_bytes(int G, int64_t E);
void launch_crossings_f32_grid(const Buffers &b, int64_t E, int G, void *work, uint32_t ideal, int32_t *cnt,
                               cudaStream_t s);
void launch_crossings_f32(const Buffers &b, int64_t n_bound, uint32_t ideal, int32_t *cnt, cudaStream_t s);
// a9 on FP32 coordinates; each vertex's smallest gap (far vertices) to `arg`.
void launch_min_angle_f32(Buffers &b, int64_t V, int64_t E, int2 *arg, cudaStream_t s);
// Folds the forward into `st` and the three values (E_ca, M_l, M_a) into out3.
void launch_diff_state(const Buffers &b, int64_t V, int64_t E, double ideal, DiffState *st, float *out3,
                       cudaStream_t s);
// grad[V][2] = gout[0] dE_ca + gout[1] dM_l + gout[2] dM_a (overwritten),
// from the signed counts `cnt` and the state `st` of the last forward.
void launch_diff_backward(const Buffers &b, int64_t V, int64_t E, const int2 *arg, const DiffState *st,
                          const float *gout, const int32_t *cnt, float *grad, cudaStream_t s);

// ------------------------------------------------------------------ batches
// Device view of a batch of layouts packed one after another: layout l owns
// vertices [v_off[l], v_off[l+1]) and edges [e_off[l], e_off[l+1]).
struct BatchView {
    int64_t L = 0;
    const int64_t *v_off = nullptr;  // [L + 1]
    const int64_t *e_off = nullptr;  // [L + 1]
    gr_result *res = nullptr;        // [L] per-layout results
};

// a9 per layout: CSR over all vertices (global ids), then one block per
// layout; writes res[l].min_angle.
void launch_batch_min_angle(Buffers &b, const BatchView &bv, int64_t V, int64_t E, cudaStream_t s);
// a10 per layout: one block per layout, deterministic; writes res[l].M_l and
// res[l].crossing.c.zero_length_edges.
void launch_batch_elv(const Buffers &b, const BatchView &bv, cudaStream_t s);
// a8 per layout: a grid per layout (cell side 2^ko[l] >= d, cell ids from
// obase[l]); per-layout pair counts into occl[l].
void launch_batch_occlusion(const Buffers &b, const BatchView &bv, int64_t V, const int32_t *ko,
                            const uint32_t *obase, uint32_t OC, uint32_t *ocell_off, uint32_t *ocell_fill,
                            uint32_t *opts, uint32_t *olay, int64_t d, uint64_t *occl, cudaStream_t s);

// ------------------------------------------------------------- device helpers
#ifdef __CUDACC__
// Largest i in [0, n) with off[i] <= x (off ascending, off[0] <= x): the
// segment of a packed array that holds element x; empty segments are skipped.
__device__ __forceinline__ int64_t find_segment(const int64_t *__restrict__ off, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int64_t find_segment_u32(const uint32_t *__restrict__ off, int64_t n, uint32_t x) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Exact int -> float for |x| < 2^22 without a conversion instruction: x is
// added to the bit pattern of 1.5 * 2^23 (floats in [2^23, 2^24) are the
// integers, one unit apart) and 1.5 * 2^23 subtracted again.  The 64-bit
// integer conversions run on the FP64 pipe, of which GB300 has little.
__device__ __forceinline__ float i2f_exact(int x) {
    return __int_as_float(0x4B400000 + x) - 12582912.0f;
}

// Round-to-nearest int64 -> float for |v| < 2^38 (the same value as a
// conversion instruction): the high part times 2^16 plus the low 16 bits,
// both exact, in one fused multiply-add with a single rounding.
__device__ __forceinline__ float ll2f_rn(long long v) {
    return fmaf(i2f_exact((int)(v >> 16)), 65536.0f, i2f_exact((int)(v & 0xffff)));
}

// The share [lo, hi) of `units` work units that the evaluation's part takes:
// part p of n takes floor(units p / n) up to floor(units (p + 1) / n), so the
// parts cover every unit exactly once.  The units must be enumerated in an
// order every rank derives alike from the inputs (all-pairs tiles of the
// segments in edge order, the records or points of cells in cell order).
__device__ __forceinline__ void part_range(const DevAcc *acc, uint64_t units, uint64_t &lo, uint64_t &hi) {
    const uint64_t np = acc->n_parts > 1 ? acc->n_parts : 1, p = acc->n_parts > 1 ? acc->part_id : 0;
    lo = (uint64_t)((unsigned __int128)units * p / np);
    hi = (uint64_t)((unsigned __int128)units * (p + 1) / np);
}
__device__ __forceinline__ bool partitioned(const DevAcc *acc) { return acc->n_parts > 1; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; every thread gets the result.  `sh` holds >= 32 T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (wid == 0) r = warp_sum(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

// Adds a 64-bit fixed-point partial to a 128-bit (lo, hi) accumulator.
__device__ __forceinline__ void add_u128(uint64_t *lo, uint64_t *hi, uint64_t v) {
    if (v == 0) return;
    const unsigned long long old = atomicAdd((unsigned long long *)lo, (unsigned long long)v);
    if (old + v < old) atomicAdd((unsigned long long *)hi, 1ull);
}

__device__ __forceinline__ void atomic_add_u64(uint64_t *p, uint64_t v) {
    if (v) atomicAdd((unsigned long long *)p, (unsigned long long)v);
}
#endif

}  // namespace gr
