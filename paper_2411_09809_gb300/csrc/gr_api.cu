// gr_api.cu -- the C ABI of include/gr.h: layout objects, argument checks,
// device memory, and the order in which the kernels of one evaluation are
// enqueued.
#include <cuda_runtime.h>

#include <algorithm>

#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>

#include "gr_internal.cuh"

using namespace gr;

namespace {

thread_local std::string g_err;

gr_status fail(gr_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

gr_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky launch error, if any
    return fail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define GR_CU(call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr double kDefaultIdeal = 7.0 * M_PI / 18.0;  // 70 degrees (Sec. 2.1)

// The ideal angle in the kernels' angle units (pi / 2^32), <= 2^31.
uint32_t ideal_units(double ideal) { return (uint32_t)llrint(ideal / M_PI * 4294967296.0); }

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
gr_status dalloc(T **p, size_t n) {
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    return GR_OK;
}

}  // namespace

struct gr_layout {
    int64_t V = 0, E = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;      // occlusion, min angle, ELV run here, beside the crossings
    cudaStream_t side2 = nullptr;     // a move's minimum-angle update, beside its ELV
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    cudaStream_t gstream = nullptr;   // evaluation and move graphs are replayed here
    cudaStream_t cstream = nullptr;   // and captured here (never joined to a caller's stream)
    cudaEvent_t ev_gin = nullptr, ev_gin2 = nullptr, ev_gout = nullptr;
    gr_options opt{};
    Buffers b;
    GridBuffers g;
    gr_result *h_result = nullptr;  // pinned
    DevAcc *h_acc = nullptr;        // pinned
    gr_coord_type coord = GR_COORD_I32;
    // differentiable form (FP32 layouts)
    bool part_dirty = false;        // the device accumulators hold a share (gr_evaluate_part) other than all
    bool seg_canonical = false;     // the compacted segments are in edge order (gr_evaluate_part)
    uint32_t *canon_flags = nullptr;  // [E + 1] and [E] x 3: workspace of the canonical order
    SegRec *canon_seg = nullptr;
    int32_t *canon_eid = nullptr;
    uint32_t *canon_theta = nullptr;
    bool in_part = false;           // inside gr_evaluate_part
    cudaEvent_t ev_din = nullptr, ev_dout = nullptr;  // orders the differentiable calls with the caller's stream
    int2 *arg = nullptr;            // [V] smallest gap of every vertex
    DiffState *st = nullptr;
    float *out3 = nullptr, *gout3 = nullptr;
    bool diff_ready = false;
    void *f32_work = nullptr;       // FP32 crossing grid workspace
    int32_t *theta_cnt = nullptr;   // [E] signed count of each segment's E_c pairs (the E_ca adjoint / scale)
    int f32_G = 0;                  // its grid side (0: all-pairs tiles)
    bool f32_planned = false;
    bool stats_stale = true;        // h_acc's layout part predates the last update
    // Once a synchronised evaluation has sized the grid buffers for cell size
    // fast_k (and split), later ones with the same plan run without the
    // mid-evaluation read-backs: the plan comes from the statistics read at
    // the previous evaluation's end, the kernels read the sizes on the
    // device, and an overflow re-runs the evaluation synchronised.
    bool fast_ok = false;
    int fast_k = -1;
    bool fast_split = false;
    // the last evaluation's crossing and occlusion totals, for gr_move_vertices
    struct Last {
        bool valid = false;
        uint32_t metrics = 0, ideal_u = 0;
        int64_t d = 0;
        uint64_t proper = 0, touching = 0, collinear = 0, dev_lo = 0, dev_hi = 0, occlusion = 0;
    } last;
    // incremental-move workspace
    uint32_t *moved = nullptr;      // [V] flags, zero between calls
    uint32_t *affected = nullptr;   // [E] edges with a moved endpoint
    DeltaAcc *dacc = nullptr, *h_dacc = nullptr;
    int32_t *mv_ids = nullptr, *mv_xy = nullptr;
    int64_t mv_cap = 0;
    MoveParams *mp_dev = nullptr;            // count and previous totals on the device
    void *mp_host = nullptr;                 // their pinned staging copy
    struct MoveGraph {
        bool valid = false;
        uint32_t metrics = 0;
        double ideal = 0.0;
        int64_t d = 0;
        bool use_grid = false, ma_incremental = false;
        int k = -1;
        int64_t cap = 0;
        const void *bufs[8] = {};
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0, d2h = 0;
    } mg;
    // The crossing grid left by the last full evaluation indexes the edges
    // for the incremental passes while dgrid_k >= 0 (its cell side is
    // 2^dgrid_k); edges moved since then are in the dirty set.
    // The fast-path evaluation as one CUDA graph, captured for one
    // configuration (metrics, parameters, plan, buffers) and replayed while it
    // holds.
    struct EvalGraph {
        bool valid = false;
        uint32_t metrics = 0;
        double ideal = 0.0;
        int64_t d = 0;
        bool x_on = false, grid = false, split = false, o_on = false, ogrid = false, profiling = false;
        bool readback = true;  // the graph ends with the read-back copies to pinned host memory
        int k = 0, ko = 0;
        const void *bufs[8] = {};
        uint64_t caps[3] = {};
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0, d2h = 0;
        uint32_t phases = 0;  // phases whose events the graph records
        int32_t path = 0, occl_path = 0;
        int64_t pairs_tested = -1;
    } eg;
    int dgrid_k = -1;
    DirtySet dirty;
    StripBuffers strip;             // the approximate strip algorithm's workspace
    bool dirty_any = false;         // the dirty set may be non-empty
    int64_t io_h2d = 0, io_d2h = 0; // bytes copied between host and device
    // phase timing
    bool profiling = false;
    bool capturing = false;         // an evaluation is being captured into a graph
    cudaEvent_t ev[2 * GR_NUM_PHASES] = {};
    bool pending[GR_NUM_PHASES] = {};
    double prof_ms[GR_NUM_PHASES] = {};
    int64_t prof_calls[GR_NUM_PHASES] = {};
};

namespace {

std::atomic<int64_t> g_launches{0};

void free_grid(GridBuffers &g) {
    void *ptrs[] = {g.cell_off, g.cell_nl, g.item_off, g.cell_fill, g.rec, g.rgeo, g.item_desc, g.ocell_off, g.ocell_fill,
                    g.opts, g.seg_long, g.theta_long, g.eid_long};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    g = GridBuffers{};
}

void free_layout(gr_layout *L) {
    if (!L) return;
    Buffers &b = L->b;
    void *ptrs[] = {b.xy, b.edges, b.seg, b.seg_eid, b.seg_theta, b.len2, b.acc, b.elv_part, b.elv_len, b.ma_part,
                    b.ma_cnt, b.deg, b.deg_fill, b.dirs, b.scan_tmp, b.scan_tmp_side, b.result,
                    b.seg_ids, b.dir_ang, b.dir_other, L->canon_flags, L->canon_seg,
                    L->canon_eid, L->canon_theta, L->arg, L->st, L->out3, L->gout3,
                    L->f32_work, L->theta_cnt, L->moved, L->affected, L->dacc, L->mv_ids, L->mv_xy,
                    L->dirty.flag, L->dirty.list, L->dirty.n, L->mp_dev, b.adj_off, b.adj, b.ma_nz, b.ma_dv, b.ma_touch,
                    b.ma_flag};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    free_grid(L->g);
    if (L->eg.exec) cudaGraphExecDestroy(L->eg.exec);
    {
        StripBuffers &sb = L->strip;
        void *sp[] = {sb.mark_start, sb.mark_end, sb.strip_off, sb.tile_off, sb.fill, sb.k1[0], sb.k1[1],
                      sb.rk[0], sb.rk[1], sb.th[0], sb.th[1], sb.acc, sb.split};
        for (void *p : sp)
            if (p) cudaFree(p);
    }
    for (auto &e : L->ev)
        if (e) cudaEventDestroy(e);
    if (L->ev_fork) cudaEventDestroy(L->ev_fork);
    if (L->ev_din) cudaEventDestroy(L->ev_din);
    if (L->ev_dout) cudaEventDestroy(L->ev_dout);
    if (L->ev_join) cudaEventDestroy(L->ev_join);
    if (L->ev_join2) cudaEventDestroy(L->ev_join2);
    if (L->side) cudaStreamDestroy(L->side);
    if (L->side2) cudaStreamDestroy(L->side2);
    if (L->gstream) cudaStreamDestroy(L->gstream);
    if (L->cstream) cudaStreamDestroy(L->cstream);
    if (L->ev_gin) cudaEventDestroy(L->ev_gin);
    if (L->ev_gin2) cudaEventDestroy(L->ev_gin2);
    if (L->ev_gout) cudaEventDestroy(L->ev_gout);
    if (L->h_result) cudaFreeHost(L->h_result);
    if (L->h_acc) cudaFreeHost(L->h_acc);
    if (L->h_dacc) cudaFreeHost(L->h_dacc);
    if (L->mp_host) cudaFreeHost(L->mp_host);
    if (L->mg.exec) cudaGraphExecDestroy(L->mg.exec);
    delete L;
}

constexpr int64_t kF32GridMinEdges = 2048;  // FP32 layouts: all-pairs tiles below this many edges

gr_status alloc_layout(gr_layout *L) {
    const int64_t V = L->V, E = L->E;
    Buffers &b = L->b;
    gr_status st;
#define GR_TRY(x)                   \
    if ((st = (x)) != GR_OK) return st
    GR_TRY(dalloc(&b.xy, 2 * (size_t)V));
    GR_TRY(dalloc(&b.edges, 2 * (size_t)E));
    GR_TRY(dalloc(&b.seg, (size_t)E));
    GR_TRY(dalloc(&b.seg_eid, (size_t)E));
    GR_TRY(dalloc(&b.seg_theta, (size_t)E));
    GR_TRY(dalloc(&b.len2, (size_t)E));
    GR_TRY(dalloc(&b.acc, 1));
    GR_TRY(dalloc(&b.elv_part, 2 * (size_t)kElvBlocks));
    GR_TRY(dalloc(&b.elv_len, (size_t)E));
    GR_TRY(dalloc(&b.ma_part, 1024));
    GR_TRY(dalloc(&b.ma_cnt, 1024));
    GR_TRY(dalloc(&b.deg, (size_t)V + 1));
    GR_TRY(dalloc(&b.deg_fill, (size_t)V));
    GR_TRY(dalloc(&b.dirs, 2 * (size_t)E));
    GR_TRY(dalloc(&b.scan_tmp, (size_t)kScanMaxBlocks));
    GR_TRY(dalloc(&b.scan_tmp_side, (size_t)kScanMaxBlocks));
    GR_TRY(dalloc(&b.result, 1));
    if (L->coord == GR_COORD_I32) {
        GR_TRY(dalloc(&b.adj_off, (size_t)V + 1));
        GR_TRY(dalloc(&b.adj, 2 * (size_t)E));
        GR_TRY(dalloc(&b.ma_nz, (size_t)V));
        GR_TRY(dalloc(&b.ma_dv, (size_t)V));
        GR_TRY(dalloc(&b.ma_touch, (size_t)V));
        GR_TRY(dalloc(&b.ma_flag, 1024));
        GR_CU(cudaMemsetAsync(b.ma_touch, 0, sizeof(uint32_t) * (V > 0 ? V : 1), L->stream));
        GR_CU(cudaMemsetAsync(b.ma_flag, 0, sizeof(uint32_t) * 1024, L->stream));
    }
    if (L->coord == GR_COORD_F32) {
        GR_TRY(dalloc(&b.seg_ids, (size_t)E));
        GR_TRY(dalloc(&b.dir_ang, 2 * (size_t)E));
        GR_TRY(dalloc(&b.dir_other, 2 * (size_t)E));
        GR_TRY(dalloc(&L->arg, (size_t)V));
        GR_TRY(dalloc(&L->st, 1));
        GR_TRY(dalloc(&L->out3, 3));
        GR_TRY(dalloc(&L->gout3, 3));
        GR_TRY(dalloc(&L->theta_cnt, (size_t)E));
    }
#undef GR_TRY
    GR_CU(cudaStreamCreateWithFlags(&L->side, cudaStreamNonBlocking));
    GR_CU(cudaStreamCreateWithFlags(&L->side2, cudaStreamNonBlocking));
    GR_CU(cudaStreamCreateWithFlags(&L->gstream, cudaStreamNonBlocking));
    GR_CU(cudaStreamCreateWithFlags(&L->cstream, cudaStreamNonBlocking));
    GR_CU(cudaEventCreateWithFlags(&L->ev_gin, cudaEventDisableTiming));
    GR_CU(cudaEventCreateWithFlags(&L->ev_gin2, cudaEventDisableTiming));
    GR_CU(cudaEventCreateWithFlags(&L->ev_gout, cudaEventDisableTiming));
    GR_CU(cudaEventCreateWithFlags(&L->ev_fork, cudaEventDisableTiming));
    GR_CU(cudaEventCreateWithFlags(&L->ev_join, cudaEventDisableTiming));
    GR_CU(cudaEventCreateWithFlags(&L->ev_join2, cudaEventDisableTiming));
    GR_CU(cudaMallocHost((void **)&L->h_result, sizeof(gr_result)));
    GR_CU(cudaMallocHost((void **)&L->h_acc, sizeof(DevAcc)));
    GR_CU(cudaMemsetAsync(b.acc, 0, sizeof(DevAcc), L->stream));
    return GR_OK;
}

// Grows the crossing-grid cell arrays to C cells.
gr_status ensure_cells(gr_layout *L, int C) {
    GridBuffers &g = L->g;
    gr_status st;
    if (!g.seg_long) {  // the long-segment list (at most every edge)
        if ((st = dalloc(&g.seg_long, (size_t)L->E)) != GR_OK) return st;
        if ((st = dalloc(&g.theta_long, (size_t)L->E)) != GR_OK) return st;
        if ((st = dalloc(&g.eid_long, (size_t)L->E)) != GR_OK) return st;
    }
    if (g.cells_cap >= C) return GR_OK;
    if (g.cell_off) cudaFree(g.cell_off);
    if (g.cell_nl) cudaFree(g.cell_nl);
    if (g.item_off) cudaFree(g.item_off);
    if (g.cell_fill) cudaFree(g.cell_fill);
    g.cell_off = g.cell_nl = g.item_off = nullptr;
    g.cell_fill = nullptr;
    g.cells_cap = 0;
    if ((st = dalloc(&g.cell_off, (size_t)C + 1)) != GR_OK) return st;
    if ((st = dalloc(&g.cell_nl, (size_t)C)) != GR_OK) return st;
    if ((st = dalloc(&g.item_off, (size_t)C + 1)) != GR_OK) return st;
    if ((st = dalloc(&g.cell_fill, (size_t)C)) != GR_OK) return st;
    g.cells_cap = C;
    return GR_OK;
}

gr_status ensure_records(gr_layout *L, uint64_t R, uint64_t items) {
    GridBuffers &g = L->g;
    gr_status st;
    if (g.rec_cap < R || !g.rec) {
        if (g.rec) cudaFree(g.rec);
        if (g.rgeo) cudaFree(g.rgeo);
        g.rec = nullptr;
        g.rgeo = nullptr;
        g.rec_cap = 0;
        const uint64_t cap = R + R / 4 + 1024;
        if ((st = dalloc(&g.rec, (size_t)cap)) != GR_OK) return st;
        if ((st = dalloc(&g.rgeo, 4 * (size_t)cap)) != GR_OK) return st;
        g.rec_cap = cap;
    }
    if (g.items_cap < items || !g.item_desc) {
        if (g.item_desc) cudaFree(g.item_desc);
        g.item_desc = nullptr;
        g.items_cap = 0;
        const uint64_t cap = items + items / 4 + 1024;
        if ((st = dalloc(&g.item_desc, 2 * (size_t)cap)) != GR_OK) return st;
        g.items_cap = cap;
    }
    return GR_OK;
}

gr_status ensure_ocells(gr_layout *L, int C) {
    GridBuffers &g = L->g;
    gr_status st;
    if (!g.opts && (st = dalloc(&g.opts, (size_t)L->V)) != GR_OK) return st;
    if (g.ocells_cap >= C) return GR_OK;
    if (g.ocell_off) cudaFree(g.ocell_off);
    if (g.ocell_fill) cudaFree(g.ocell_fill);
    g.ocell_off = g.ocell_fill = nullptr;
    g.ocells_cap = 0;
    if ((st = dalloc(&g.ocell_off, (size_t)C + 1)) != GR_OK) return st;
    if ((st = dalloc(&g.ocell_fill, (size_t)C)) != GR_OK) return st;
    g.ocells_cap = C;
    return GR_OK;
}

// ------------------------------------------------------------ phase timing
// Phase events; while an evaluation is being captured into a graph they are
// captured as event-record nodes, so that every replay records them.
void phase_begin(gr_layout *L, int ph, cudaStream_t s) {
    if (L->profiling)
        cudaEventRecordWithFlags(L->ev[2 * ph], s, L->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}
void phase_end(gr_layout *L, int ph, cudaStream_t s) {
    if (L->profiling) {
        cudaEventRecordWithFlags(L->ev[2 * ph + 1], s,
                                 L->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        L->pending[ph] = true;
    }
}
void phase_begin(gr_layout *L, int ph) { phase_begin(L, ph, L->stream); }
void phase_end(gr_layout *L, int ph) { phase_end(L, ph, L->stream); }
// After a stream synchronisation: folds the recorded phases into the totals.
void phase_collect(gr_layout *L) {
    if (!L->profiling) return;
    for (int ph = 0; ph < GR_NUM_PHASES; ++ph) {
        if (!L->pending[ph]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, L->ev[2 * ph], L->ev[2 * ph + 1]) == cudaSuccess) {
            L->prof_ms[ph] += ms;
            L->prof_calls[ph] += 1;
        } else {
            cudaGetLastError();
        }
        L->pending[ph] = false;
    }
}

gr_status set_profiling(gr_layout *L, bool on) {
    if (on && !L->ev[0]) {
        for (auto &e : L->ev) GR_CU(cudaEventCreate(&e));
    }
    L->profiling = on;
    return GR_OK;
}

// Copies the inputs into the layout's own buffers and runs a1 (gather and
// validation).  Stream-ordered.
gr_status enqueue_inputs(gr_layout *L, const void *xy, const int32_t *edges) {
    cudaStream_t s = L->stream;
    const int64_t V = L->V, E = L->E;
    phase_begin(L, GR_PHASE_GATHER);
    GR_CU(cudaMemsetAsync(L->b.acc, 0, offsetof(DevAcc, eval_status), s));
    if (V > 0) {
        const cudaMemcpyKind k = is_device_pointer(xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GR_CU(cudaMemcpyAsync(L->b.xy, xy, sizeof(int32_t) * 2 * V, k, s));
        if (k == cudaMemcpyHostToDevice) L->io_h2d += (int64_t)sizeof(int32_t) * 2 * V;
    }
    if (E > 0 && edges) {
        const cudaMemcpyKind k = is_device_pointer(edges) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GR_CU(cudaMemcpyAsync(L->b.edges, edges, sizeof(int32_t) * 2 * E, k, s));
        if (k == cudaMemcpyHostToDevice) L->io_h2d += (int64_t)sizeof(int32_t) * 2 * E;
    }
    if (L->coord == GR_COORD_F32) {
        launch_gather_f32((const float *)L->b.xy, V, L->b.edges, E, L->b, s);
    } else {
        launch_gather(L->b.xy, V, L->b.edges, E, L->b, s);
        if (edges) launch_adjacency(L->b, V, E, s);
    }
    L->diff_ready = false;
    L->dgrid_k = -1;
    L->seg_canonical = false;  // the gather's order depends on which block reserved its slots first
    phase_end(L, GR_PHASE_GATHER);
    GR_CU(cudaGetLastError());
    L->stats_stale = true;
    return GR_OK;
}

gr_status status_to_error(uint32_t st) {
    if (st & ST_BAD_ID) return fail(GR_EINVAL, "vertex id outside [0, V) or self-loop in the edge list");
    if (st & ST_BAD_COORD) return fail(GR_ERANGE, "vertex coordinate outside [0, 65536) (not finite for FP32 layouts)");
    if (st & ST_SCAN_OVERFLOW) return fail(GR_ENOTSUP, "an offset table exceeded 2^32 entries");
    if (st & ST_OVERFLOW) return fail(GR_ENOMEM, "grid record buffer overflow");
    return GR_OK;
}

// The share of the pair work the next evaluation does (DevAcc part_id /
// n_parts, read by the pair kernels); n_parts = 0 means all of it, the state
// every rewrite of the accumulators' first block leaves.
gr_status set_part(gr_layout *L, uint32_t part, uint32_t n_parts) {
    const uint32_t v[2] = {part, n_parts};
    GR_CU(cudaMemcpyAsync(&L->b.acc->part_id, v, sizeof v, cudaMemcpyHostToDevice, L->stream));
    L->part_dirty = n_parts > 1;
    return GR_OK;
}

// Entry points other than gr_evaluate_part evaluate all of the work.
gr_status reset_part(gr_layout *L) {
    if (!L->part_dirty || L->in_part) return GR_OK;
    return set_part(L, 0, 0);
}

gr_status read_params(const gr_params *p, double *ideal, int64_t *d) {
    *ideal = kDefaultIdeal;
    *d = 0;
    if (p) {
        if (p->ideal_rad > 0.0) *ideal = p->ideal_rad;
        *d = p->occlusion_d;
    }
    if (!(*ideal <= M_PI / 2 + 1e-15)) return fail(GR_EINVAL, "ideal angle must be in (0, pi/2]");
    if (*d < 0) return fail(GR_EINVAL, "occlusion diameter d must be >= 0");
    return GR_OK;
}

// Reads the layout part of the accumulators (compacted count, total L1
// length, validation status) once after every update.
gr_status refresh_stats(gr_layout *L) {
    if (!L->stats_stale) return GR_OK;
    GR_CU(cudaMemcpyAsync(L->h_acc, L->b.acc, offsetof(DevAcc, eval_status), cudaMemcpyDeviceToHost, L->stream));
    L->io_d2h += (int64_t)offsetof(DevAcc, eval_status);
    GR_CU(cudaStreamSynchronize(L->stream));
    L->stats_stale = false;
    return GR_OK;
}

constexpr double kGridMargin = 0.75;

struct CrossPlan {
    bool grid = false;
    bool split = false;  // long-long pairs on the all-pairs tiles
    int k = 0;
};

// Chooses the cell size with grid_cost (records, short-involved candidate
// pairs at even spread, cells, long-long pairs on the all-pairs tiles); ties
// go to the coarser grid.  Picks all-pairs unless the best grid is estimated
// at under kGridMargin of its cost (the estimate is rough where few segments
// are short and the grid is coarse).
CrossPlan plan_crossings(const gr_layout *L, const DevAcc &a) {
    CrossPlan p;
    const double n = (double)a.n_seg, l = (double)a.len_l1;
    const double allpairs = n * (n - 1) / 2;
    int best_k = 8;
    bool best_split = false;
    double best = 1e300;
    for (int k = 14; k >= 6; --k)
        for (bool split : {false, true}) {
            const double cost = grid_cost(n, l, a.len_hist, a.l1_hist, k, split);
            if (cost < best) { best = cost; best_k = k; best_split = split; }
        }
    p.k = best_k;
    p.split = best_split;
    if (L->opt.cell_log2 >= 6 && L->opt.cell_log2 <= 16) {  // a fixed cell size: the better form for it
        p.k = L->opt.cell_log2;
        p.split = grid_cost(n, l, a.len_hist, a.l1_hist, p.k, true) <
                  grid_cost(n, l, a.len_hist, a.l1_hist, p.k, false);
    }
    if (L->opt.long_pairs == GR_LONG_ALLPAIRS) p.split = true;
    else if (L->opt.long_pairs == GR_LONG_GRID) p.split = false;
    if (L->opt.crossing_path == GR_PATH_GRID) p.grid = true;
    else if (L->opt.crossing_path == GR_PATH_ALLPAIRS) p.grid = false;
    else p.grid = a.n_seg >= 2 && best < kGridMargin * allpairs;
    return p;
}

int occl_cell_log2(int64_t d) {
    int k = 6;
    while ((int64_t(1) << k) < d) ++k;
    return k;
}

// Keeps the crossing and occlusion totals of the evaluation just read back.
void remember_totals(gr_layout *L, uint32_t metrics, uint32_t ideal_u, int64_t d) {
    const DevAcc &a = *L->h_acc;
    L->last.valid = true;
    L->last.metrics = metrics;
    L->last.ideal_u = ideal_u;
    L->last.d = d;
    L->last.proper = a.proper;
    L->last.touching = a.touching;
    L->last.collinear = a.collinear;
    L->last.dev_lo = a.dev_lo;
    L->last.dev_hi = a.dev_hi;
    L->last.occlusion = a.occlusion;
}

float host_unord(uint32_t u) {
    const uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &v, sizeof f);
    return f;
}

// FP32 crossing grid, planned once from the statistics of the first
// evaluation.  For each side G (a power of two in [16, 1024]) the cost of the
// pair tests is estimated from the segments' major-axis length classes:
// segments at least a cell long count as long; short ones give about 1.5
// records each; short x short pairs R^2 / 2C at even spread; each long
// segment walks about 2 L / w + 2 cells holding R / C records each; long x
// long pairs n_long^2 / 2; plus a few units per cell and per record.
gr_status plan_f32_grid(gr_layout *L) {
    if (L->f32_planned) return GR_OK;
    L->f32_planned = true;
    const DevAcc &a = *L->h_acc;
    const uint64_t n = a.n_seg;
    if ((int64_t)n < kF32GridMinEdges || a.f32_bounds[0] > a.f32_bounds[2]) return GR_OK;
    const double span = std::max((double)host_unord(a.f32_bounds[2]) - host_unord(a.f32_bounds[0]),
                                 (double)host_unord(a.f32_bounds[3]) - host_unord(a.f32_bounds[1]));
    if (!(span > 0.0)) return GR_OK;
    int best_G = 0;
    double best = 0.5 * (double)n * (double)n;  // all-pairs tiles
    for (int G = 16; G <= 1024; G *= 2) {
        const double w = span / G, C = (double)G * G;
        double n_long = 0.0, len_long = 0.0;
        for (int b = 0; b < 64; ++b) {
            const double lo = std::ldexp(1.0, b - 48);
            if (lo >= w) {
                n_long += a.f32_hist[b];
                len_long += 1.5 * lo * a.f32_hist[b];
            }
        }
        const double R = 1.5 * ((double)n - n_long), dens = R / C;
        const double cost = R * R / (2.0 * C) + (2.0 * len_long / w + 2.0 * n_long) * dens + 0.5 * n_long * n_long +
                            4.0 * C + 8.0 * R;
        if (cost < best) { best = cost; best_G = G; }
    }
    if (best_G == 0) return GR_OK;
    L->f32_G = best_G;
    return dalloc((char **)&L->f32_work, f32_grid_bytes(best_G, L->E));
}

// The FP32 forward: E_ca and the crossing counts (with `save`, each
// segment's signed count of E_c pairs for the backward), M_l, M_a (smallest
// gaps saved), folded into L->st/out3.
gr_status forward_f32(gr_layout *L, uint32_t metrics, double ideal, bool save) {
    cudaStream_t s = L->stream;
    Buffers &b = L->b;
    const int64_t V = L->V, E = L->E;
    const uint32_t ideal_u = ideal_units(ideal);
    gr_status pst = plan_f32_grid(L);
    if (pst != GR_OK) return pst;
    int32_t *cnt = save ? L->theta_cnt : nullptr;
    GR_CU(cudaMemsetAsync((char *)b.acc + offsetof(DevAcc, eval_status), 0,
                          sizeof(DevAcc) - offsetof(DevAcc, eval_status), s));
    if (cnt) GR_CU(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (E > 0 ? E : 1), s));
    phase_begin(L, GR_PHASE_EDGE_LENGTH);
    if (metrics & GR_METRIC_EDGE_LENGTH) launch_elv(b, E, s, true);
    phase_end(L, GR_PHASE_EDGE_LENGTH);
    phase_begin(L, GR_PHASE_MIN_ANGLE);
    if (metrics & GR_METRIC_MIN_ANGLE) launch_min_angle_f32(b, V, E, L->arg, s);
    phase_end(L, GR_PHASE_MIN_ANGLE);
    phase_begin(L, GR_PHASE_CROSS_PAIRS);
    if ((metrics & GR_METRIC_CROSSINGS) && L->f32_G > 0 && L->opt.crossing_path != GR_PATH_ALLPAIRS)
        launch_crossings_f32_grid(b, E, L->f32_G, L->f32_work, ideal_u, cnt, s);
    else if (metrics & GR_METRIC_CROSSINGS)
        launch_crossings_f32(b, E, ideal_u, cnt, s);
    phase_end(L, GR_PHASE_CROSS_PAIRS);
    phase_begin(L, GR_PHASE_FINALIZE);
    if (save) launch_diff_state(b, V, E, ideal, L->st, L->out3, s);
    GR_CU(cudaGetLastError());
    GR_CU(cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
    L->io_d2h += (int64_t)sizeof(DevAcc);
    phase_end(L, GR_PHASE_FINALIZE);
    GR_CU(cudaStreamSynchronize(s));
    phase_collect(L);
    return status_to_error(L->h_acc->status | L->h_acc->eval_status);
}

gr_status evaluate_f32(gr_layout *L, uint32_t metrics, double ideal, gr_result *out) {
    if (metrics & GR_METRIC_OCCLUSION) return fail(GR_ENOTSUP, "occlusion needs GR_COORD_I32 coordinates");
    gr_status st = forward_f32(L, metrics, ideal, false);
    if (st != GR_OK) return st;
    cudaStream_t s = L->stream;
    Buffers &b = L->b;
    const bool fgrid = (metrics & GR_METRIC_CROSSINGS) && L->f32_G > 0 && L->opt.crossing_path != GR_PATH_ALLPAIRS;
    launch_finalize(b, metrics, L->E, ideal, 0, L->V > 0 ? min_angle_blocks(L->V) : 0,
                    (metrics & GR_METRIC_CROSSINGS) ? (fgrid ? GR_PATH_GRID : GR_PATH_ALLPAIRS) : 0, 0, 0,
                    fgrid ? -2 : -1, s);
    GR_CU(cudaGetLastError());
    GR_CU(cudaMemcpyAsync(L->h_result, b.result, sizeof(gr_result), cudaMemcpyDeviceToHost, s));
    L->io_d2h += (int64_t)sizeof(gr_result);
    GR_CU(cudaStreamSynchronize(s));
    *out = *L->h_result;
    out->grid_records = 0;
    return GR_OK;
}

}  // namespace

extern "C" {

const char *gr_last_error(void) { return g_err.c_str(); }

const char *gr_version(void) { return "gr 0.1 (sm_103a)"; }

gr_status gr_layout_create(gr_layout **out, const void *xy, gr_coord_type coord_type, int64_t V,
                           const int32_t *edges, int64_t E, const gr_options *opt,
                           gr_stream_t stream) {
    g_err.clear();
    if (!out) return fail(GR_EINVAL, "out is NULL");
    if (coord_type != GR_COORD_I32 && coord_type != GR_COORD_F32) return fail(GR_ENOTSUP, "unknown coordinate type");
    if (V < 0 || E < 0 || V >= (int64_t(1) << 31) || E >= (int64_t(1) << 31))
        return fail(GR_EINVAL, "V and E must be in [0, 2^31)");
    if ((V > 0 && !xy) || (E > 0 && !edges)) return fail(GR_EINVAL, "NULL input pointer");
    if (E > 0 && V < 2) return fail(GR_EINVAL, "edges need at least two vertices");
    gr_layout *L = new gr_layout;
    L->V = V;
    L->E = E;
    L->stream = (cudaStream_t)stream;
    L->coord = coord_type;
    if (opt) L->opt = *opt;
    gr_status st = alloc_layout(L);
    if (st == GR_OK) {
        const cudaError_t e = init_min_angle_table(L->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "uploading the minimum-angle table");
    }
    if (st == GR_OK && L->opt.profile) st = set_profiling(L, true);
    if (st == GR_OK) st = enqueue_inputs(L, xy, edges);
    if (st == GR_OK) {
        cudaError_t e = cudaMemcpyAsync(L->h_acc, L->b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "validating the layout");
        else st = status_to_error(L->h_acc->status);
        L->stats_stale = false;
        phase_collect(L);
    }
    if (st != GR_OK) {
        free_layout(L);
        return st;
    }
    *out = L;
    return GR_OK;
}

gr_status gr_layout_update(gr_layout *L, const void *xy, const int32_t *edges) {
    g_err.clear();
    if (!L) return fail(GR_EINVAL, "layout is NULL");
    L->last.valid = false;
    if (L->V > 0 && !xy) return fail(GR_EINVAL, "xy is NULL");
    return enqueue_inputs(L, xy, edges);
}

gr_status gr_layout_destroy(gr_layout *L) {
    g_err.clear();
    if (!L) return GR_OK;
    cudaStreamSynchronize(L->stream);
    free_layout(L);
    return GR_OK;
}

namespace {

// The end of an evaluation: one synchronisation, then the checks.  A fast
// grid evaluation whose buffers the inputs outgrew runs again, synchronised.
gr_status finish_evaluate(gr_layout *L, uint32_t metrics, const gr_params *params, double ideal, int64_t d,
                          bool fast_grid, int32_t path, int k, gr_result *out) {
    GR_CU(cudaStreamSynchronize(L->stream));
    phase_collect(L);
    L->stats_stale = false;  // the read-back holds the statistics of these inputs
    if (fast_grid && ((L->h_acc->eval_status & ST_OVERFLOW) || (L->h_acc->grid_flags & GF_ITEMS_OVERFLOW)) &&
        !(L->h_acc->status & (ST_BAD_ID | ST_BAD_COORD))) {
        L->fast_ok = false;  // the buffers did not fit these inputs: again, synchronised
        return gr_evaluate(L, metrics, params, out);
    }
    gr_status st = status_to_error(L->h_acc->status | L->h_acc->eval_status);
    if (st != GR_OK) return st;
    *out = *L->h_result;
    remember_totals(L, metrics, ideal_units(ideal), d);
    if (path == GR_PATH_GRID) L->dgrid_k = k;
    if (!L->fast_ok && path != GR_PATH_GRID) {
        // no grid buffers to size: later evaluations may take the fast path (a grid plan then
        // does not match fast_k and runs synchronised once)
        L->fast_ok = true;
        L->fast_k = -1;
        L->fast_split = false;
    }
    return GR_OK;
}

struct FastPlan {
    bool x_on = false, o_on = false, ogrid = false, graphable = false;
    int ko = 0;
    CrossPlan cp;
};

// The occlusion choice: a grid of side >= d for many vertices; all-pairs
// tiles for few, or when d is so large that the grid has at most 4 x 4 cells.
bool occlusion_grid(const gr_layout *L, int ko) {
    if (L->opt.occlusion_path == GR_PATH_GRID) return ko <= 16;
    if (L->opt.occlusion_path == GR_PATH_ALLPAIRS) return false;
    return L->V > 4096 && ko <= 14;
}

// Plan of a fast-path evaluation and its buffers.  It can run as one graph
// when no step needs a read-back: crossings absent, on all-pairs tiles, or on
// the grid plan the buffers were sized for.
gr_status plan_fast(gr_layout *L, uint32_t metrics, int64_t d, uint64_t n_seg, FastPlan *fp) {
    gr_status st;
    fp->x_on = (metrics & GR_METRIC_CROSSINGS) && n_seg >= 2;
    fp->o_on = (metrics & GR_METRIC_OCCLUSION) != 0;
    fp->ko = occl_cell_log2(d);
    fp->ogrid = fp->o_on && occlusion_grid(L, fp->ko);
    if (fp->ogrid && L->V >= 2 && d > 0) {
        const int C = (65536 >> fp->ko) * (65536 >> fp->ko);
        if ((st = ensure_ocells(L, C)) != GR_OK) return st;
    }
    if (fp->x_on) {
        fp->cp = plan_crossings(L, *L->h_acc);
        if (fp->cp.grid) {
            const int C = (65536 >> fp->cp.k) * (65536 >> fp->cp.k);
            if ((st = ensure_cells(L, C)) != GR_OK) return st;
        }
    }
    fp->graphable = !fp->x_on || !fp->cp.grid || (fp->cp.k == L->fast_k && fp->cp.split == L->fast_split);
    return GR_OK;
}

// Enqueues a fast-path evaluation (no read-back before the end): the same
// steps as the synchronised path of gr_evaluate.
void enqueue_fast(gr_layout *L, cudaStream_t s, uint32_t metrics, double ideal, int64_t d, const FastPlan &fp,
                  bool readback, int32_t *path, int32_t *occl_path, int64_t *pairs_tested) {
    cudaStream_t t = L->side;
    Buffers &b = L->b;
    const int64_t V = L->V, E = L->E;
    cudaMemsetAsync((char *)b.acc + offsetof(DevAcc, eval_status), 0, sizeof(DevAcc) - offsetof(DevAcc, eval_status),
                    s);
    cudaEventRecord(L->ev_fork, s);
    cudaStreamWaitEvent(t, L->ev_fork, 0);
    if (metrics & GR_METRIC_EDGE_LENGTH) {
        phase_begin(L, GR_PHASE_EDGE_LENGTH, t);
        launch_elv(b, E, t);
        phase_end(L, GR_PHASE_EDGE_LENGTH, t);
    }
    if (metrics & GR_METRIC_MIN_ANGLE) {
        phase_begin(L, GR_PHASE_MIN_ANGLE, t);
        launch_min_angle(b, V, E, t);
        phase_end(L, GR_PHASE_MIN_ANGLE, t);
    }
    *occl_path = 0;
    if (fp.o_on) {
        if (fp.ogrid && V >= 2 && d > 0) {
            phase_begin(L, GR_PHASE_OCCL_BIN, t);
            launch_occlusion_grid_count(b, V, L->g, fp.ko, t);
            phase_end(L, GR_PHASE_OCCL_BIN, t);
            phase_begin(L, GR_PHASE_OCCL_PAIRS, t);
            launch_occlusion_grid_pairs(b, V, L->g, fp.ko, d, t);
            phase_end(L, GR_PHASE_OCCL_PAIRS, t);
        } else {
            phase_begin(L, GR_PHASE_OCCL_PAIRS, t);
            launch_occlusion_allpairs(b, V, d, t);
            phase_end(L, GR_PHASE_OCCL_PAIRS, t);
        }
        *occl_path = fp.ogrid ? GR_PATH_GRID : GR_PATH_ALLPAIRS;
    }
    cudaEventRecord(L->ev_join, t);
    *path = 0;
    *pairs_tested = -1;
    if (fp.x_on && fp.cp.grid) {
        phase_begin(L, GR_PHASE_CROSS_BIN, s);
        launch_grid_count(b, E, L->g, fp.cp.k, fp.cp.split, s);
        phase_end(L, GR_PHASE_CROSS_BIN, s);
        phase_begin(L, GR_PHASE_CROSS_SCATTER, s);
        launch_grid_scatter(b, E, L->g, fp.cp.k, fp.cp.split, s);
        phase_end(L, GR_PHASE_CROSS_SCATTER, s);
        phase_begin(L, GR_PHASE_CROSS_PAIRS, s);
        launch_grid_pairs(b, L->g, fp.cp.k, fp.cp.split, L->g.items_cap, ideal_units(ideal), PerEdge{}, s);
        if (fp.cp.split) launch_grid_long_pairs(b, L->g, -1, ideal_units(ideal), PerEdge{}, s);
        phase_end(L, GR_PHASE_CROSS_PAIRS, s);
        *path = GR_PATH_GRID;
        *pairs_tested = -2;  // computed on the device
    } else if (fp.x_on) {
        phase_begin(L, GR_PHASE_CROSS_PAIRS, s);
        launch_crossings_allpairs(b, E, ideal_units(ideal), PerEdge{}, s);
        phase_end(L, GR_PHASE_CROSS_PAIRS, s);
        *path = GR_PATH_ALLPAIRS;
    } else if (metrics & GR_METRIC_CROSSINGS) {
        *path = GR_PATH_ALLPAIRS;
    }
    cudaStreamWaitEvent(s, L->ev_join, 0);
    phase_begin(L, GR_PHASE_FINALIZE, s);
    launch_finalize(b, metrics, E, ideal, d, V > 0 ? min_angle_blocks(V) : 0, *path,
                    *path == GR_PATH_GRID ? fp.cp.k : 0, *occl_path, *pairs_tested, s);
    if (readback) {
        cudaMemcpyAsync(L->h_result, b.result, sizeof(gr_result), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s);
        L->io_d2h += (int64_t)(sizeof(gr_result) + sizeof(DevAcc));
    }
    phase_end(L, GR_PHASE_FINALIZE, s);
}

// Replays the graph of this configuration, capturing it first when the
// configuration or a buffer changed since the last capture.
gr_status run_eval_graph(gr_layout *L, uint32_t metrics, double ideal, int64_t d, const FastPlan &fp,
                         cudaStream_t after, gr_result *d_result, bool readback) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (after != L->stream) GR_CU(cudaStreamIsCapturing(after, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        // `after` is being captured into the caller's graph: the evaluation's own steps are captured
        // there directly (the caller orders the inputs before replaying)
        int32_t path, occl_path;
        int64_t pairs_tested;
        L->capturing = true;
        enqueue_fast(L, after, metrics, ideal, d, fp, false, &path, &occl_path, &pairs_tested);
        L->capturing = false;
        if (d_result) GR_CU(cudaMemcpyAsync(d_result, L->b.result, sizeof(gr_result), cudaMemcpyDeviceToDevice, after));
        return GR_OK;
    }
    auto &g = L->eg;
    const GridBuffers &gb = L->g;
    const void *bufs[8] = {gb.cell_off, gb.cell_nl, gb.item_off, gb.cell_fill, gb.rec, gb.item_desc, gb.ocell_off,
                           gb.opts};
    const uint64_t caps[3] = {gb.rec_cap, gb.items_cap, (uint64_t)gb.cells_cap};
    const bool same = g.valid && g.metrics == metrics && g.ideal == ideal && g.d == d && g.x_on == fp.x_on &&
                      g.grid == fp.cp.grid && g.split == fp.cp.split && g.k == fp.cp.k && g.o_on == fp.o_on &&
                      g.ogrid == fp.ogrid && g.ko == fp.ko && g.profiling == L->profiling &&
                      g.readback == readback && memcmp(g.bufs, bufs, sizeof bufs) == 0 &&
                      memcmp(g.caps, caps, sizeof caps) == 0;
    // captured on a stream of its own (the caller's stream may be the legacy one, which cannot be
    // captured, or be capturing itself), replayed on another
    cudaStream_t s = L->cstream;
    if (!same) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.valid = false;
        bool pend0[GR_NUM_PHASES];
        memcpy(pend0, L->pending, sizeof pend0);
        const int64_t l0 = gr_kernel_launches(), io0 = L->io_d2h;
        GR_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        L->capturing = true;
        enqueue_fast(L, s, metrics, ideal, d, fp, readback, &g.path, &g.occl_path, &g.pairs_tested);
        L->capturing = false;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &graph);
        g.launches = gr_kernel_launches() - l0;
        count_launches((int)-g.launches);  // nothing ran yet
        g.d2h = L->io_d2h - io0;
        L->io_d2h = io0;
        g.phases = 0;
        for (int ph = 0; ph < GR_NUM_PHASES; ++ph)
            if (L->pending[ph] && !pend0[ph]) g.phases |= 1u << ph;
        memcpy(L->pending, pend0, sizeof pend0);
        if (ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ec, "capturing the evaluation");
        }
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(ei, "instantiating the evaluation graph");
        }
        g.valid = true;
        g.metrics = metrics;
        g.ideal = ideal;
        g.d = d;
        g.x_on = fp.x_on;
        g.grid = fp.cp.grid;
        g.split = fp.cp.split;
        g.k = fp.cp.k;
        g.o_on = fp.o_on;
        g.ogrid = fp.ogrid;
        g.ko = fp.ko;
        g.profiling = L->profiling;
        g.readback = readback;
        memcpy(g.bufs, bufs, sizeof bufs);
        memcpy(g.caps, caps, sizeof caps);
    }
    // after the work queued on the layout's stream (its inputs) and on `after`, and before what
    // follows on `after`
    cudaStream_t r = L->gstream;
    GR_CU(cudaEventRecord(L->ev_gin, L->stream));
    GR_CU(cudaStreamWaitEvent(r, L->ev_gin, 0));
    if (after != L->stream) {
        GR_CU(cudaEventRecord(L->ev_gin2, after));
        GR_CU(cudaStreamWaitEvent(r, L->ev_gin2, 0));
    }
    GR_CU(cudaGraphLaunch(g.exec, r));
    if (d_result) GR_CU(cudaMemcpyAsync(d_result, L->b.result, sizeof(gr_result), cudaMemcpyDeviceToDevice, r));
    GR_CU(cudaEventRecord(L->ev_gout, r));
    GR_CU(cudaStreamWaitEvent(after, L->ev_gout, 0));
    if (after != L->stream) GR_CU(cudaStreamWaitEvent(L->stream, L->ev_gout, 0));
    count_launches((int)g.launches);
    L->io_d2h += g.d2h;
    for (int ph = 0; ph < GR_NUM_PHASES; ++ph)
        if (g.phases & (1u << ph)) L->pending[ph] = true;
    return GR_OK;
}

}  // namespace

gr_status gr_evaluate(gr_layout *L, uint32_t metrics, const gr_params *params, gr_result *out) {
    g_err.clear();
    if (!L || !out) return fail(GR_EINVAL, "NULL argument");
    if (metrics & ~GR_METRIC_ALL) return fail(GR_EINVAL, "unknown metric bits");
    double ideal;
    int64_t d;
    gr_status st = read_params(params, &ideal, &d);
    if (st != GR_OK) return st;
    if ((st = reset_part(L)) != GR_OK) return st;
    cudaStream_t s = L->stream;
    Buffers &b = L->b;
    const int64_t V = L->V, E = L->E;
    // fast: plan from the statistics of the previous evaluation (the inputs'
    // validity is then checked at the end; every kernel skips invalid data)
    const bool fast = L->fast_ok && L->coord == GR_COORD_I32;
    if (!fast) {
        if ((st = refresh_stats(L)) != GR_OK) return st;
        if ((st = status_to_error(L->h_acc->status)) != GR_OK) return st;
    }
    if (L->coord == GR_COORD_F32) return evaluate_f32(L, metrics, ideal, out);
    const uint64_t n_seg = fast ? (uint64_t)E : L->h_acc->n_seg;  // (an upper bound when fast)
    L->dgrid_k = -1;  // set again below when this evaluation leaves a complete crossing grid
    if (L->dirty_any) {
        GR_CU(cudaMemsetAsync(L->dirty.flag, 0, (size_t)(E > 0 ? E : 1), s));
        GR_CU(cudaMemsetAsync(L->dirty.n, 0, sizeof(uint32_t), s));
        L->dirty_any = false;
    }
    if (fast) {
        // the plan of the fast path, and every buffer it needs, before anything is enqueued
        FastPlan fp;
        if ((st = plan_fast(L, metrics, d, n_seg, &fp)) != GR_OK) return st;
        if (fp.graphable) {
            if ((st = run_eval_graph(L, metrics, ideal, d, fp, L->stream, nullptr, true)) != GR_OK) return st;
            return finish_evaluate(L, metrics, params, ideal, d, fp.x_on && fp.cp.grid, L->eg.path, fp.cp.k, out);
        }
    }
    GR_CU(cudaMemsetAsync((char *)b.acc + offsetof(DevAcc, eval_status), 0,
                          sizeof(DevAcc) - offsetof(DevAcc, eval_status), s));

    // Occlusion, minimum angle and edge length variation depend only on the
    // inputs: they run on the side stream, beside the crossing pipeline.
    cudaStream_t t = L->side;
    GR_CU(cudaEventRecord(L->ev_fork, s));
    GR_CU(cudaStreamWaitEvent(t, L->ev_fork, 0));
    if (metrics & GR_METRIC_EDGE_LENGTH) {
        phase_begin(L, GR_PHASE_EDGE_LENGTH, t);
        launch_elv(b, E, t);
        phase_end(L, GR_PHASE_EDGE_LENGTH, t);
    }
    if (metrics & GR_METRIC_MIN_ANGLE) {
        phase_begin(L, GR_PHASE_MIN_ANGLE, t);
        launch_min_angle(b, V, E, t);
        phase_end(L, GR_PHASE_MIN_ANGLE, t);
    }
    int32_t occl_path = 0;
    if (metrics & GR_METRIC_OCCLUSION) {
        const int ko = occl_cell_log2(d);
        const bool grid = occlusion_grid(L, ko);
        if (grid && V >= 2 && d > 0) {
            const int C = (65536 >> ko) * (65536 >> ko);
            if ((st = ensure_ocells(L, C)) != GR_OK) return st;
            phase_begin(L, GR_PHASE_OCCL_BIN, t);
            launch_occlusion_grid_count(b, V, L->g, ko, t);
            phase_end(L, GR_PHASE_OCCL_BIN, t);
            phase_begin(L, GR_PHASE_OCCL_PAIRS, t);
            launch_occlusion_grid_pairs(b, V, L->g, ko, d, t);
            phase_end(L, GR_PHASE_OCCL_PAIRS, t);
        } else {
            phase_begin(L, GR_PHASE_OCCL_PAIRS, t);
            launch_occlusion_allpairs(b, V, d, t);
            phase_end(L, GR_PHASE_OCCL_PAIRS, t);
        }
        occl_path = grid ? GR_PATH_GRID : GR_PATH_ALLPAIRS;
    }
    GR_CU(cudaEventRecord(L->ev_join, t));

    // crossing binning; without the fast path the host needs its sizes
    CrossPlan cp;
    bool need_sync = false, fast_grid = false;
    if ((metrics & GR_METRIC_CROSSINGS) && n_seg >= 2) {
        cp = plan_crossings(L, *L->h_acc);
        if (cp.grid) {
            const int C = (65536 >> cp.k) * (65536 >> cp.k);
            if ((st = ensure_cells(L, C)) != GR_OK) return st;
            phase_begin(L, GR_PHASE_CROSS_BIN);
            launch_grid_count(b, E, L->g, cp.k, cp.split, s);
            phase_end(L, GR_PHASE_CROSS_BIN);
            fast_grid = fast && cp.k == L->fast_k && cp.split == L->fast_split;
            need_sync = !fast_grid;
        }
    }
    if (need_sync) {
        GR_CU(cudaGetLastError());
        GR_CU(cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
        L->io_d2h += (int64_t)sizeof(DevAcc);
        GR_CU(cudaStreamSynchronize(s));
        if ((st = status_to_error(L->h_acc->eval_status)) != GR_OK) {
            cudaStreamSynchronize(t);
            return st;
        }
    }

    int32_t path = 0;
    int64_t pairs_tested = -1;
    if (fast_grid) {
        phase_begin(L, GR_PHASE_CROSS_SCATTER);
        launch_grid_scatter(b, E, L->g, cp.k, cp.split, s);
        phase_end(L, GR_PHASE_CROSS_SCATTER);
        phase_begin(L, GR_PHASE_CROSS_PAIRS);
        launch_grid_pairs(b, L->g, cp.k, cp.split, L->g.items_cap, ideal_units(ideal), PerEdge{}, s);
        if (cp.split) launch_grid_long_pairs(b, L->g, -1, ideal_units(ideal), PerEdge{}, s);
        phase_end(L, GR_PHASE_CROSS_PAIRS);
        path = GR_PATH_GRID;
        pairs_tested = -2;  // computed on the device
    } else if ((metrics & GR_METRIC_CROSSINGS) && n_seg >= 2) {
        bool grid = cp.grid;
        const DevAcc &a = *L->h_acc;
        if (grid && (a.grid_flags & GF_ITEMS_OVERFLOW)) grid = false;
        const double nl = (double)a.n_long;
        if (grid && L->opt.crossing_path == GR_PATH_AUTO) {
            const double n = (double)n_seg;
            grid = kRecordCost * (double)a.records + kCellPairCost * (double)a.grid_work + nl * (nl - 1) / 2 <
                   kGridMargin * n * (n - 1) / 2;
        }
        if (grid) {
            if ((st = ensure_records(L, a.records, a.grid_items)) != GR_OK) return st;
            phase_begin(L, GR_PHASE_CROSS_SCATTER);
            launch_grid_scatter(b, E, L->g, cp.k, cp.split, s);
            phase_end(L, GR_PHASE_CROSS_SCATTER);
            phase_begin(L, GR_PHASE_CROSS_PAIRS);
            launch_grid_pairs(b, L->g, cp.k, cp.split, a.grid_items, ideal_units(ideal), PerEdge{}, s);
            if (cp.split) launch_grid_long_pairs(b, L->g, a.n_long, ideal_units(ideal), PerEdge{}, s);
            phase_end(L, GR_PHASE_CROSS_PAIRS);
            path = GR_PATH_GRID;
            pairs_tested = (int64_t)a.grid_work + (int64_t)a.n_long * ((int64_t)a.n_long - 1) / 2;
            L->fast_ok = true;  // buffers sized (with headroom) for this plan
            L->fast_k = cp.k;
            L->fast_split = cp.split;
        } else {
            phase_begin(L, GR_PHASE_CROSS_PAIRS);
            launch_crossings_allpairs(b, E, ideal_units(ideal), PerEdge{}, s);
            phase_end(L, GR_PHASE_CROSS_PAIRS);
            path = GR_PATH_ALLPAIRS;
        }
    } else if (metrics & GR_METRIC_CROSSINGS) {
        path = GR_PATH_ALLPAIRS;
    }
    GR_CU(cudaStreamWaitEvent(s, L->ev_join, 0));
    phase_begin(L, GR_PHASE_FINALIZE);
    launch_finalize(b, metrics, E, ideal, d, V > 0 ? min_angle_blocks(V) : 0, path,
                    path == GR_PATH_GRID ? cp.k : 0, occl_path, pairs_tested, s);
    GR_CU(cudaGetLastError());
    GR_CU(cudaMemcpyAsync(L->h_result, b.result, sizeof(gr_result), cudaMemcpyDeviceToHost, s));
    GR_CU(cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
    L->io_d2h += (int64_t)(sizeof(gr_result) + sizeof(DevAcc));
    phase_end(L, GR_PHASE_FINALIZE);
    return finish_evaluate(L, metrics, params, ideal, d, fast_grid, path, cp.k, out);
}

gr_status gr_evaluate_async(gr_layout *L, uint32_t metrics, const gr_params *params, gr_result *d_result,
                            gr_stream_t stream) {
    g_err.clear();
    if (!L || !d_result) return fail(GR_EINVAL, "NULL argument");
    if (metrics & ~GR_METRIC_ALL) return fail(GR_EINVAL, "unknown metric bits");
    if (L->coord != GR_COORD_I32) return fail(GR_ENOTSUP, "gr_evaluate_async needs a GR_COORD_I32 layout");
    if (!is_device_pointer(d_result)) return fail(GR_EINVAL, "d_result must be device memory");
    double ideal;
    int64_t d;
    gr_status st = read_params(params, &ideal, &d);
    if (st != GR_OK) return st;
    if ((st = reset_part(L)) != GR_OK) return st;
    cudaStream_t after = stream ? (cudaStream_t)stream : L->stream;
    FastPlan fp;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (L->fast_ok) {
            if ((st = plan_fast(L, metrics, d, (uint64_t)L->E, &fp)) != GR_OK) return st;
            if (fp.graphable) break;
        }
        // not planned yet, or the plan changed: one synchronised evaluation plans and sizes the buffers
        gr_result tmp;
        if ((st = gr_evaluate(L, metrics, params, &tmp)) != GR_OK) return st;
        fp.graphable = false;
    }
    if (!fp.graphable) return fail(GR_ENOTSUP, "the layout's crossing plan does not settle");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (after != L->stream) GR_CU(cudaStreamIsCapturing(after, &cap));
    if (L->dirty_any && cap == cudaStreamCaptureStatusNone) {  // (else the next synchronous evaluation does it)
        GR_CU(cudaMemsetAsync(L->dirty.flag, 0, (size_t)(L->E > 0 ? L->E : 1), L->stream));
        GR_CU(cudaMemsetAsync(L->dirty.n, 0, sizeof(uint32_t), L->stream));
        L->dirty_any = false;
    }
    // the host keeps no totals of an evaluation it does not read back
    L->last.valid = false;
    L->dgrid_k = -1;
    return run_eval_graph(L, metrics, ideal, d, fp, after, d_result, false);
}

gr_status gr_evaluate_part(gr_layout *L, uint32_t metrics, const gr_params *params, int32_t part, int32_t n_parts,
                           gr_partial *out) {
    g_err.clear();
    if (!L || !out) return fail(GR_EINVAL, "NULL argument");
    if (n_parts < 1 || part < 0 || part >= n_parts) return fail(GR_EINVAL, "part must be in [0, n_parts), n_parts >= 1");
    if (L->coord != GR_COORD_I32) return fail(GR_ENOTSUP, "gr_evaluate_part needs a GR_COORD_I32 layout");
    gr_status st;
    if (!L->seg_canonical && L->E > 0) {
        // every rank must enumerate the all-pairs tiles over the same segment order
        if (!L->canon_flags) {
            if ((st = dalloc(&L->canon_flags, (size_t)L->E + 1)) != GR_OK) return st;
            if ((st = dalloc(&L->canon_seg, (size_t)L->E)) != GR_OK) return st;
            if ((st = dalloc(&L->canon_eid, (size_t)L->E)) != GR_OK) return st;
            if ((st = dalloc(&L->canon_theta, (size_t)L->E)) != GR_OK) return st;
        }
        launch_canonical_segments(L->b, L->E, L->canon_flags, L->canon_seg, L->canon_eid, L->canon_theta, L->stream);
        GR_CU(cudaGetLastError());
    }
    L->seg_canonical = true;
    if ((st = set_part(L, (uint32_t)part, (uint32_t)n_parts)) != GR_OK) return st;
    gr_result r;
    L->in_part = true;
    st = gr_evaluate(L, metrics, params, &r);
    L->in_part = false;
    L->last.valid = false;  // a share's tallies must not seed an incremental move
    if (st != GR_OK) return st;
    const DevAcc &a = *L->h_acc;  // read back at the end of the evaluation
    memset(out, 0, sizeof *out);
    out->proper = (int64_t)a.proper;
    out->touching = (int64_t)a.touching;
    out->collinear_overlaps = (int64_t)a.collinear;
    out->occlusion_pairs = (int64_t)a.occlusion;
    // the 128-bit angle sum (dev_hi, dev_lo) as two halves that sum without overflow over many parts
    out->dev_hi32 = (int64_t)((a.dev_hi << 32) | (a.dev_lo >> 32));
    out->dev_lo32 = (int64_t)(a.dev_lo & 0xffffffffull);
    if (part == 0) {
        out->metrics = r.metrics;
        out->crossing_path = r.crossing_path;
        out->cell_log2 = r.cell_log2;
        out->occlusion_path = r.occlusion_path;
        out->zero_length_edges = r.crossing.c.zero_length_edges;
        out->pairs_tested = r.crossing.c.pairs_tested;
        out->n_vertices_counted = r.min_angle.n_vertices_counted;
        out->grid_records = r.grid_records;
        memcpy(&out->min_angle_sum_d_bits, &r.min_angle.sum_d, sizeof(double));
        memcpy(&out->M_a_bits, &r.min_angle.M_a, sizeof(double));
        memcpy(&out->M_l_bits, &r.M_l, sizeof(double));
    }
    return GR_OK;
}

gr_status gr_combine_parts(const gr_partial *sp, const gr_params *params, gr_result *out) {
    g_err.clear();
    if (!sp || !out) return fail(GR_EINVAL, "NULL argument");
    double ideal;
    int64_t d;
    gr_status st = read_params(params, &ideal, &d);
    if (st != GR_OK) return st;
    gr_result r;
    memset(&r, 0, sizeof r);
    r.metrics = (uint32_t)sp->metrics;
    r.crossing_path = (int32_t)sp->crossing_path;
    r.cell_log2 = (int32_t)sp->cell_log2;
    r.occlusion_path = (int32_t)sp->occlusion_path;
    const uint64_t ec = (uint64_t)sp->proper + (uint64_t)sp->touching;
    r.crossing.c.crossings = (int64_t)ec;
    r.crossing.c.proper = sp->proper;
    r.crossing.c.touching = sp->touching;
    r.crossing.c.collinear_overlaps = sp->collinear_overlaps;
    r.crossing.c.zero_length_edges = sp->zero_length_edges;
    r.crossing.c.pairs_tested = sp->pairs_tested;
    // the same arithmetic as the device's final reduction, on the same 128-bit sum
    const unsigned __int128 dev = ((unsigned __int128)(uint64_t)sp->dev_hi32 << 32) + (uint64_t)sp->dev_lo32;
    const uint64_t dev_hi = (uint64_t)(dev >> 64), dev_lo = (uint64_t)dev;
    const double dv = ((double)dev_hi * 18446744073709551616.0 + (double)dev_lo) * kAngleUnit;
    r.crossing.angle_dev_sum = dv;
    r.crossing.ideal_rad = ideal;
    r.crossing.E_ca = ec > 0 ? 1.0 - dv / (ideal * (double)ec) : 1.0;
    r.occlusion_pairs = sp->occlusion_pairs;
    r.occlusion_d = d;
    memcpy(&r.min_angle.sum_d, &sp->min_angle_sum_d_bits, sizeof(double));
    memcpy(&r.min_angle.M_a, &sp->M_a_bits, sizeof(double));
    r.min_angle.n_vertices_counted = sp->n_vertices_counted;
    memcpy(&r.M_l, &sp->M_l_bits, sizeof(double));
    r.grid_records = sp->grid_records;
    *out = r;
    return GR_OK;
}

gr_status gr_node_occlusion(gr_layout *L, int64_t d, int64_t *out_pairs) {
    if (!out_pairs) return fail(GR_EINVAL, "NULL argument");
    gr_params p{0.0, d};
    gr_result r;
    gr_status st = gr_evaluate(L, GR_METRIC_OCCLUSION, &p, &r);
    if (st == GR_OK) *out_pairs = r.occlusion_pairs;
    return st;
}

gr_status gr_min_angle(gr_layout *L, gr_min_angle_result *out) {
    if (!out) return fail(GR_EINVAL, "NULL argument");
    gr_result r;
    gr_status st = gr_evaluate(L, GR_METRIC_MIN_ANGLE, nullptr, &r);
    if (st == GR_OK) *out = r.min_angle;
    return st;
}

gr_status gr_edge_length_variation(gr_layout *L, double *out_M_l) {
    if (!out_M_l) return fail(GR_EINVAL, "NULL argument");
    gr_result r;
    gr_status st = gr_evaluate(L, GR_METRIC_EDGE_LENGTH, nullptr, &r);
    if (st == GR_OK) *out_M_l = r.M_l;
    return st;
}

gr_status gr_edge_crossings(gr_layout *L, gr_crossing_counts *out) {
    if (!out) return fail(GR_EINVAL, "NULL argument");
    gr_result r;
    gr_status st = gr_evaluate(L, GR_METRIC_CROSSINGS, nullptr, &r);
    if (st == GR_OK) *out = r.crossing.c;
    return st;
}

gr_status gr_crossing_angle(gr_layout *L, double ideal_rad, gr_crossing_angle_result *out) {
    if (!out) return fail(GR_EINVAL, "NULL argument");
    gr_params p{ideal_rad, 0};
    gr_result r;
    gr_status st = gr_evaluate(L, GR_METRIC_CROSSINGS, &p, &r);
    if (st == GR_OK) *out = r.crossing;
    return st;
}

namespace {

// One orientation of the strip estimate into out (synchronises twice: the
// record count sizes the buffers).
gr_status strip_one(gr_layout *L, int l, int orient, double ideal, gr_strip_result *out) {
    cudaStream_t s = L->stream;
    StripBuffers &sb = L->strip;
    const int ns = strip_count(l);
    gr_status st;
    if (sb.ns_cap < ns + 1) {
        uint32_t **arr[] = {&sb.mark_start, &sb.mark_end, &sb.strip_off, &sb.tile_off, &sb.fill};
        for (uint32_t **a : arr) {
            if (*a) cudaFree(*a);
            *a = nullptr;
        }
        sb.ns_cap = 0;
        for (uint32_t **a : arr)
            if ((st = dalloc(a, (size_t)ns + 1)) != GR_OK) return st;
        sb.ns_cap = ns + 1;
    }
    if (!sb.acc && (st = dalloc(&sb.acc, 1)) != GR_OK) return st;
    const size_t nb = sizeof(uint32_t) * ((size_t)ns + 1);
    GR_CU(cudaMemsetAsync(sb.mark_start, 0, nb, s));
    GR_CU(cudaMemsetAsync(sb.mark_end, 0, nb, s));
    GR_CU(cudaMemsetAsync(sb.fill, 0, nb, s));
    GR_CU(cudaMemsetAsync(sb.acc, 0, sizeof(StripAcc), s));
    launch_strip_span(L->b, L->E, l, orient, sb, s);
    GR_CU(cudaGetLastError());
    StripAcc h;
    GR_CU(cudaMemcpyAsync(&h, sb.acc, sizeof h, cudaMemcpyDeviceToHost, s));
    GR_CU(cudaStreamSynchronize(s));
    if (h.status) return status_to_error(h.status);
    if (h.records > sb.cap) {
        for (int i = 0; i < 2; ++i) {
            if (sb.k1[i]) cudaFree(sb.k1[i]);
            if (sb.rk[i]) cudaFree(sb.rk[i]);
            if (sb.th[i]) cudaFree(sb.th[i]);
            sb.k1[i] = sb.rk[i] = nullptr;
            sb.th[i] = nullptr;
        }
        sb.cap = 0;
        const size_t want = (size_t)h.records;
        for (int i = 0; i < 2; ++i) {
            if ((st = dalloc(&sb.k1[i], want)) != GR_OK) return st;
            if ((st = dalloc(&sb.rk[i], want)) != GR_OK) return st;
            if ((st = dalloc(&sb.th[i], want)) != GR_OK) return st;
        }
        sb.cap = h.records;
    }
    if (2ull * h.tiles > sb.split_cap) {
        if (sb.split) cudaFree(sb.split);
        sb.split = nullptr;
        sb.split_cap = 0;
        if ((st = dalloc(&sb.split, 2 * (size_t)h.tiles)) != GR_OK) return st;
        sb.split_cap = 2ull * h.tiles;
    }
    sb.records = h.records;
    sb.tiles = h.tiles;
    phase_begin(L, GR_PHASE_STRIP_SORT);
    launch_strip_sort(L->b, L->E, l, orient, sb, h.max_n, s);
    phase_end(L, GR_PHASE_STRIP_SORT);
    phase_begin(L, GR_PHASE_STRIP_COUNT);
    launch_strip_inversions(l, sb, h.max_n, ideal_units(ideal), s);
    phase_end(L, GR_PHASE_STRIP_COUNT);
    GR_CU(cudaGetLastError());
    GR_CU(cudaMemcpyAsync(&h, sb.acc, sizeof h, cudaMemcpyDeviceToHost, s));
    GR_CU(cudaStreamSynchronize(s));
    phase_collect(L);
    L->io_d2h += (int64_t)(2 * sizeof h);
    if (h.status) return status_to_error(h.status);
    const double dev = ((double)h.dev_hi * 18446744073709551616.0 + (double)h.dev_lo) * kAngleUnit;
    out->crossings = (int64_t)h.count;
    out->records = (int64_t)h.records;
    out->strips = ns;
    out->angle_dev_sum = dev;
    out->ideal_rad = ideal;
    out->E_ca = h.count > 0 ? 1.0 - dev / (ideal * (double)h.count) : 1.0;
    out->orientation = orient;
    out->strip_width = l;
    return GR_OK;
}

}  // namespace

gr_status gr_strip_crossings(gr_layout *L, int32_t strip_width, int32_t orientation, double ideal_rad,
                             gr_strip_result *out) {
    g_err.clear();
    if (!L || !out) return fail(GR_EINVAL, "NULL argument");
    if (L->coord != GR_COORD_I32) return fail(GR_ENOTSUP, "the strip estimate needs GR_COORD_I32 coordinates");
    if (strip_width < 1 || strip_width > 65535) return fail(GR_EINVAL, "strip width must be in [1, 65535]");
    if (orientation < GR_STRIP_VERTICAL || orientation > GR_STRIP_BOTH) return fail(GR_EINVAL, "bad orientation");
    gr_params p{ideal_rad, 0};
    double ideal;
    int64_t d;
    gr_status st = read_params(&p, &ideal, &d);
    if (st != GR_OK) return st;
    if ((st = refresh_stats(L)) != GR_OK) return st;
    if ((st = status_to_error(L->h_acc->status)) != GR_OK) return st;
    gr_strip_result r[2];
    const int o0 = orientation == GR_STRIP_HORIZONTAL ? 1 : 0, o1 = orientation == GR_STRIP_VERTICAL ? 0 : 1;
    for (int o = o0; o <= o1; ++o)
        if ((st = strip_one(L, strip_width, o, ideal, &r[o])) != GR_OK) return st;
    *out = (o0 != o1 && r[1].crossings > r[0].crossings) ? r[1] : r[o0];
    return GR_OK;
}

gr_status gr_crossings_per_edge(gr_layout *L, double ideal_rad, int64_t *d_counts, double *d_dev) {
    g_err.clear();
    if (!L || (L->E > 0 && (!d_counts || !d_dev))) return fail(GR_EINVAL, "NULL argument");
    if (L->coord != GR_COORD_I32) return fail(GR_ENOTSUP, "per-edge crossings need GR_COORD_I32 coordinates");
    gr_params p{ideal_rad, 0};
    double ideal;
    int64_t d;
    gr_status st = read_params(&p, &ideal, &d);
    if (st != GR_OK) return st;
    if ((st = reset_part(L)) != GR_OK) return st;
    const int64_t E = L->E;
    if (E == 0) return GR_OK;
    if (!is_device_pointer(d_counts) || !is_device_pointer(d_dev))
        return fail(GR_EINVAL, "per-edge outputs must be device memory");
    cudaStream_t s = L->stream;
    Buffers &b = L->b;
    L->dgrid_k = -1;  // the grid buffers are rebuilt below
    GR_CU(cudaMemsetAsync((char *)b.acc + offsetof(DevAcc, eval_status), 0,
                          sizeof(DevAcc) - offsetof(DevAcc, eval_status), s));
    GR_CU(cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * 3 * E, s));
    GR_CU(cudaMemsetAsync(d_dev, 0, sizeof(double) * E, s));
    PerEdge pe;
    pe.counts = (uint64_t *)d_counts;
    pe.dev = (uint64_t *)d_dev;
    gr_status st2 = refresh_stats(L);
    if (st2 != GR_OK) return st2;
    if ((st2 = status_to_error(L->h_acc->status)) != GR_OK) return st2;
    CrossPlan cp = plan_crossings(L, *L->h_acc);
    if (cp.grid && L->h_acc->n_seg >= 2) {
        const int C = (65536 >> cp.k) * (65536 >> cp.k);
        if ((st2 = ensure_cells(L, C)) != GR_OK) return st2;
        phase_begin(L, GR_PHASE_CROSS_BIN);
        launch_grid_count(b, E, L->g, cp.k, cp.split, s);
        phase_end(L, GR_PHASE_CROSS_BIN);
        GR_CU(cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
        GR_CU(cudaStreamSynchronize(s));
        if ((st2 = status_to_error(L->h_acc->eval_status)) != GR_OK) return st2;
        if (L->h_acc->grid_flags & GF_ITEMS_OVERFLOW) cp.grid = false;
    }
    if (cp.grid && L->h_acc->n_seg >= 2) {
        if ((st2 = ensure_records(L, L->h_acc->records, L->h_acc->grid_items)) != GR_OK) return st2;
        phase_begin(L, GR_PHASE_CROSS_SCATTER);
        launch_grid_scatter(b, E, L->g, cp.k, cp.split, s);
        phase_end(L, GR_PHASE_CROSS_SCATTER);
        phase_begin(L, GR_PHASE_CROSS_PAIRS);
        launch_grid_pairs(b, L->g, cp.k, cp.split, L->h_acc->grid_items, ideal_units(ideal), pe, s);
        if (cp.split) launch_grid_long_pairs(b, L->g, L->h_acc->n_long, ideal_units(ideal), pe, s);
        phase_end(L, GR_PHASE_CROSS_PAIRS);
    } else {
        phase_begin(L, GR_PHASE_CROSS_PAIRS);
        launch_crossings_allpairs(b, E, ideal_units(ideal), pe, s);
        phase_end(L, GR_PHASE_CROSS_PAIRS);
    }
    launch_per_edge_export(pe.dev, E, s);
    GR_CU(cudaGetLastError());
    GR_CU(cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
    GR_CU(cudaStreamSynchronize(s));
    phase_collect(L);
    return status_to_error(L->h_acc->status | L->h_acc->eval_status);
}

namespace {

struct MovePlan {
    uint32_t metrics;
    double ideal;
    int64_t d;
    uint32_t ideal_u;
    bool crossings, occl, use_grid, ma_incremental;
    long long d2;
};

// Enqueues an incremental move on stream s (side work on two side streams):
// validation, the before pass, the new coordinates, the regather, the after
// pass, the new totals, the other metrics and the read-back.  Every kernel
// after the validation does nothing on an invalid move.
void enqueue_move(gr_layout *L, cudaStream_t s, const MovePlan &mp) {
    Buffers &b = L->b;
    const int64_t V = L->V, E = L->E, cap = L->mv_cap;
    const int64_t *np = &L->mp_dev->n;
    cudaMemsetAsync(L->dacc, 0, sizeof(DeltaAcc), s);
    launch_delta_validate(L->mv_ids, L->mv_xy, np, cap, V, L->moved, L->dacc, s);
    if (mp.crossings)
        launch_delta_affected(b, E, L->moved, L->affected, L->dacc, mp.use_grid ? L->dirty : DirtySet{}, s);
    if (mp.use_grid)
        launch_delta_grid_pass(b, L->g, L->dgrid_k, L->moved, L->affected, L->dirty, mp.ideal_u, L->dacc, 0, s);
    launch_delta_pass(b, V, E, L->mv_ids, np, L->moved, L->affected, mp.crossings && !mp.use_grid, mp.ideal_u,
                      mp.occl, mp.d2, L->dacc, 0, s);
    launch_delta_apply(L->mv_ids, L->mv_xy, np, cap, L->dacc, b, s);
    // the moved layout's segments and statistics, then the after pass on
    // them; edge length variation and minimum angle on two side streams
    cudaMemsetAsync(b.acc, 0, offsetof(DevAcc, eval_status), s);
    launch_gather(b.xy, V, b.edges, E, b, s);
    const bool elv = (mp.metrics & GR_METRIC_EDGE_LENGTH) != 0, ma = (mp.metrics & GR_METRIC_MIN_ANGLE) != 0;
    if (elv || ma) cudaEventRecord(L->ev_fork, s);
    if (elv) {
        cudaStreamWaitEvent(L->side, L->ev_fork, 0);
        launch_elv(b, E, L->side);
        cudaEventRecord(L->ev_join, L->side);
    }
    if (ma) {
        cudaStream_t t = L->side2;
        cudaStreamWaitEvent(t, L->ev_fork, 0);
        if (mp.ma_incremental) launch_min_angle_moved(b, V, L->mv_ids, np, cap, t);
        else launch_min_angle(b, V, E, t);
        cudaEventRecord(L->ev_join2, t);
    }
    if (mp.use_grid)
        launch_delta_grid_pass(b, L->g, L->dgrid_k, L->moved, L->affected, L->dirty, mp.ideal_u, L->dacc, 1, s);
    launch_delta_pass(b, V, E, L->mv_ids, np, L->moved, L->affected, mp.crossings && !mp.use_grid, mp.ideal_u,
                      mp.occl, mp.d2, L->dacc, 1, s);
    launch_delta_unmark(L->mv_ids, np, cap, V, L->moved, s);
    launch_delta_combine(&L->mp_dev->last, L->dacc, b, s);
    if (elv) cudaStreamWaitEvent(s, L->ev_join, 0);
    if (ma) cudaStreamWaitEvent(s, L->ev_join2, 0);
    const uint32_t need = mp.metrics & (GR_METRIC_CROSSINGS | GR_METRIC_OCCLUSION);
    launch_finalize(b, mp.metrics, E, mp.ideal, mp.d, V > 0 ? min_angle_blocks(V) : 0,
                    mp.crossings ? GR_PATH_DELTA : 0, 0, (need & GR_METRIC_OCCLUSION) ? GR_PATH_DELTA : 0, -2, s);
    cudaMemcpyAsync(L->h_dacc, L->dacc, sizeof(DeltaAcc), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(L->h_result, b.result, sizeof(gr_result), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s);
    L->io_d2h += (int64_t)(sizeof(DeltaAcc) + sizeof(gr_result) + sizeof(DevAcc));
}

// Replays the captured move of this configuration (capturing it first when
// the configuration or a buffer changed), ordered after the layout's stream.
gr_status run_move_graph(gr_layout *L, const MovePlan &mp) {
    auto &g = L->mg;
    const void *bufs[8] = {L->mv_ids, L->mv_xy, L->dirty.flag, L->dirty.list, L->g.cell_off, L->g.rec, L->mp_dev,
                           L->dacc};
    const bool same = g.valid && g.metrics == mp.metrics && g.ideal == mp.ideal && g.d == mp.d &&
                      g.use_grid == mp.use_grid && g.ma_incremental == mp.ma_incremental && g.k == L->dgrid_k &&
                      g.cap == L->mv_cap && memcmp(g.bufs, bufs, sizeof bufs) == 0;
    cudaStream_t s = L->cstream;
    if (!same) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.valid = false;
        const int64_t l0 = gr_kernel_launches(), io0 = L->io_d2h;
        GR_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        enqueue_move(L, s, mp);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &graph);
        g.launches = gr_kernel_launches() - l0;
        count_launches((int)-g.launches);
        g.d2h = L->io_d2h - io0;
        L->io_d2h = io0;
        if (ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ec, "capturing the move");
        }
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(ei, "instantiating the move graph");
        }
        g.valid = true;
        g.metrics = mp.metrics;
        g.ideal = mp.ideal;
        g.d = mp.d;
        g.use_grid = mp.use_grid;
        g.ma_incremental = mp.ma_incremental;
        g.k = L->dgrid_k;
        g.cap = L->mv_cap;
        memcpy(g.bufs, bufs, sizeof bufs);
    }
    cudaStream_t r = L->gstream;
    GR_CU(cudaEventRecord(L->ev_gin, L->stream));
    GR_CU(cudaStreamWaitEvent(r, L->ev_gin, 0));
    GR_CU(cudaGraphLaunch(g.exec, r));
    GR_CU(cudaEventRecord(L->ev_gout, r));
    GR_CU(cudaStreamWaitEvent(L->stream, L->ev_gout, 0));
    count_launches((int)g.launches);
    L->io_d2h += g.d2h;
    return GR_OK;
}

}  // namespace

gr_status gr_move_vertices(gr_layout *L, int64_t n, const int32_t *ids, const int32_t *xy_new, uint32_t metrics,
                           const gr_params *params, gr_result *out) {
    g_err.clear();
    if (!L || !out) return fail(GR_EINVAL, "NULL argument");
    if (n < 0 || n > L->V) return fail(GR_EINVAL, "n must be in [0, V]");
    if (n > 0 && (!ids || !xy_new)) return fail(GR_EINVAL, "NULL ids or coordinates");
    if (metrics & ~GR_METRIC_ALL) return fail(GR_EINVAL, "unknown metric bits");
    if (L->coord != GR_COORD_I32) return fail(GR_ENOTSUP, "gr_move_vertices needs a GR_COORD_I32 layout");
    double ideal;
    int64_t d;
    gr_status st = read_params(params, &ideal, &d);
    if (st != GR_OK) return st;
    if ((st = reset_part(L)) != GR_OK) return st;
    L->seg_canonical = false;  // a move gathers the segments again
    cudaStream_t s = L->stream;
    Buffers &b = L->b;
    const int64_t V = L->V, E = L->E;
    // workspace
    if (!L->dacc) {
        if ((st = dalloc(&L->moved, (size_t)V)) != GR_OK) return st;
        if ((st = dalloc(&L->affected, (size_t)E)) != GR_OK) return st;
        if ((st = dalloc(&L->dacc, 1)) != GR_OK) return st;
        if ((st = dalloc(&L->mp_dev, 1)) != GR_OK) return st;
        GR_CU(cudaMallocHost((void **)&L->h_dacc, sizeof(DeltaAcc)));
        GR_CU(cudaMallocHost((void **)&L->mp_host, sizeof(MoveParams)));
        GR_CU(cudaMemsetAsync(L->moved, 0, sizeof(uint32_t) * (V > 0 ? V : 1), s));
    }
    if (L->mv_cap < n || !L->mv_ids) {
        if (L->mv_ids) cudaFree(L->mv_ids);
        if (L->mv_xy) cudaFree(L->mv_xy);
        L->mv_ids = L->mv_xy = nullptr;
        L->mv_cap = 0;
        const int64_t cap = std::max<int64_t>(n, 64);
        if ((st = dalloc(&L->mv_ids, (size_t)cap)) != GR_OK) return st;
        if ((st = dalloc(&L->mv_xy, 2 * (size_t)cap)) != GR_OK) return st;
        L->mv_cap = cap;
    }
    if (n > 0) {
        const cudaMemcpyKind ki = is_device_pointer(ids) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const cudaMemcpyKind kx = is_device_pointer(xy_new) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GR_CU(cudaMemcpyAsync(L->mv_ids, ids, sizeof(int32_t) * n, ki, s));
        GR_CU(cudaMemcpyAsync(L->mv_xy, xy_new, sizeof(int32_t) * 2 * n, kx, s));
        if (ki == cudaMemcpyHostToDevice) L->io_h2d += (int64_t)sizeof(int32_t) * n;
        if (kx == cudaMemcpyHostToDevice) L->io_h2d += (int64_t)sizeof(int32_t) * 2 * n;
    }
    MovePlan mp;
    mp.metrics = metrics;
    mp.ideal = ideal;
    mp.d = d;
    mp.ideal_u = ideal_units(ideal);
    const uint32_t need = metrics & (GR_METRIC_CROSSINGS | GR_METRIC_OCCLUSION);
    const bool incremental = L->last.valid && !L->stats_stale && (L->last.metrics & need) == need &&
                             L->last.ideal_u == mp.ideal_u && L->last.d == d;
    mp.crossings = (need & GR_METRIC_CROSSINGS) != 0;
    mp.occl = (need & GR_METRIC_OCCLUSION) != 0 && d > 0;
    mp.d2 = d >= 100000 ? (long long)1e11 : (long long)d * d;
    // the affected edges against the others: through the last full
    // evaluation's crossing grid when it left one, else against every segment
    mp.use_grid = incremental && mp.crossings && L->dgrid_k >= 0;
    mp.ma_incremental = (L->last.metrics & GR_METRIC_MIN_ANGLE) != 0;
    // the count and the totals the move updates (only those asked for; the
    // others stay zero, as in a full evaluation)
    MoveParams *h = (MoveParams *)L->mp_host;
    memset(h, 0, sizeof *h);
    h->n = n;
    if (mp.crossings) {
        h->last.proper = L->last.proper;
        h->last.touching = L->last.touching;
        h->last.collinear = L->last.collinear;
        h->last.dev_lo = L->last.dev_lo;
        h->last.dev_hi = L->last.dev_hi;
    }
    if (mp.occl) h->last.occlusion = L->last.occlusion;
    GR_CU(cudaMemcpyAsync(L->mp_dev, h, sizeof *h, cudaMemcpyHostToDevice, s));
    if (!incremental) {
        // validate, move, then a full evaluation
        const int64_t *np = &L->mp_dev->n;
        GR_CU(cudaMemsetAsync(L->dacc, 0, sizeof(DeltaAcc), s));
        launch_delta_validate(L->mv_ids, L->mv_xy, np, L->mv_cap, V, L->moved, L->dacc, s);
        launch_delta_apply(L->mv_ids, L->mv_xy, np, L->mv_cap, L->dacc, b, s);
        launch_delta_unmark(L->mv_ids, np, L->mv_cap, V, L->moved, s);
        GR_CU(cudaMemcpyAsync(L->h_dacc, L->dacc, sizeof(DeltaAcc), cudaMemcpyDeviceToHost, s));
        GR_CU(cudaStreamSynchronize(s));
        if (L->h_dacc->status) return status_to_error(L->h_dacc->status);
        L->last.valid = false;
        GR_CU(cudaMemsetAsync(b.acc, 0, offsetof(DevAcc, eval_status), s));
        launch_gather(b.xy, V, b.edges, E, b, s);
        GR_CU(cudaGetLastError());
        L->stats_stale = true;
        return gr_evaluate(L, metrics, params, out);
    }
    if (mp.use_grid && !L->dirty.flag) {
        L->dirty.cap = (uint32_t)std::min<int64_t>(E, std::max<int64_t>(4096, E / 32));
        if ((st = dalloc(&L->dirty.flag, (size_t)E)) != GR_OK) return st;
        if ((st = dalloc(&L->dirty.list, (size_t)L->dirty.cap)) != GR_OK) return st;
        if ((st = dalloc(&L->dirty.n, 1)) != GR_OK) return st;
        GR_CU(cudaMemsetAsync(L->dirty.flag, 0, (size_t)E, s));
        GR_CU(cudaMemsetAsync(L->dirty.n, 0, sizeof(uint32_t), s));
    }
    if (mp.use_grid) L->dirty_any = true;
    // one graph replay (one host synchronisation)
    if ((st = run_move_graph(L, mp)) != GR_OK) return st;
    GR_CU(cudaStreamSynchronize(s));
    if (L->h_dacc->status) return status_to_error(L->h_dacc->status);  // nothing moved
    L->stats_stale = false;
    if (L->h_dacc->fallback) {  // too many edges moved since the grid was built: a full evaluation rebuilds it
        L->last.valid = false;
        return gr_evaluate(L, metrics, params, out);
    }
    if ((st = status_to_error(L->h_acc->status | L->h_acc->eval_status)) != GR_OK) return st;
    *out = *L->h_result;
    remember_totals(L, metrics, mp.ideal_u, d);
    return GR_OK;
}

// The stream a differentiable call is ordered on (NULL: the layout's own) and
// whether it is being captured into a CUDA graph.
gr_status diff_stream(gr_layout *L, gr_stream_t stream, cudaStream_t *cs, bool *capturing) {
    *cs = stream ? (cudaStream_t)stream : L->stream;
    // (the legacy default stream, NULL, is never captured)
    cudaStreamCaptureStatus c1 = cudaStreamCaptureStatusNone, c2 = cudaStreamCaptureStatusNone;
    if (*cs) GR_CU(cudaStreamIsCapturing(*cs, &c1));
    if (*cs != L->stream && L->stream) GR_CU(cudaStreamIsCapturing(L->stream, &c2));
    if (c2 != cudaStreamCaptureStatusNone)
        return fail(GR_ENOTSUP, "the layout's own stream is being captured while another stream was named");
    *capturing = c1 != cudaStreamCaptureStatusNone;
    if (!L->ev_din) {
        GR_CU(cudaEventCreateWithFlags(&L->ev_din, cudaEventDisableTiming));
        GR_CU(cudaEventCreateWithFlags(&L->ev_dout, cudaEventDisableTiming));
    }
    return GR_OK;
}

gr_status gr_diff_forward(gr_layout *L, double ideal_rad, float *out3, gr_stream_t stream) {
    g_err.clear();
    if (!L || !out3) return fail(GR_EINVAL, "NULL argument");
    if (L->coord != GR_COORD_F32) return fail(GR_ENOTSUP, "gr_diff_forward needs a GR_COORD_F32 layout");
    cudaStream_t cs;
    bool capturing;
    gr_status st = diff_stream(L, stream, &cs, &capturing);
    if (st != GR_OK) return st;
    if (capturing) return fail(GR_ENOTSUP, "gr_diff_forward synchronises and cannot be captured into a graph");
    gr_params p{ideal_rad, 0};
    double ideal;
    int64_t d;
    if ((st = read_params(&p, &ideal, &d)) != GR_OK) return st;
    if (cs != L->stream) {  // after the work already queued on the caller's stream
        GR_CU(cudaEventRecord(L->ev_din, cs));
        GR_CU(cudaStreamWaitEvent(L->stream, L->ev_din, 0));
    }
    if ((st = refresh_stats(L)) != GR_OK) return st;
    if ((st = status_to_error(L->h_acc->status)) != GR_OK) return st;
    if ((st = forward_f32(L, GR_METRIC_CROSSINGS | GR_METRIC_EDGE_LENGTH | GR_METRIC_MIN_ANGLE, ideal, true)) != GR_OK)
        return st;
    const cudaMemcpyKind k = is_device_pointer(out3) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    GR_CU(cudaMemcpyAsync(out3, L->out3, sizeof(float) * 3, k, L->stream));
    if (k == cudaMemcpyDeviceToHost) L->io_d2h += (int64_t)sizeof(float) * 3;
    GR_CU(cudaStreamSynchronize(L->stream));
    L->diff_ready = true;
    return GR_OK;
}

gr_status gr_diff_backward(gr_layout *L, const float *gout3, float *d_grad_xy, gr_stream_t stream) {
    g_err.clear();
    if (!L || !gout3 || (L->V > 0 && !d_grad_xy)) return fail(GR_EINVAL, "NULL argument");
    if (L->coord != GR_COORD_F32) return fail(GR_ENOTSUP, "gr_diff_backward needs a GR_COORD_F32 layout");
    if (!L->diff_ready) return fail(GR_EINVAL, "gr_diff_backward needs a gr_diff_forward after the last update");
    if (L->V > 0 && !is_device_pointer(d_grad_xy)) return fail(GR_EINVAL, "the gradient must be device memory");
    cudaStream_t cs;
    bool capturing;
    gr_status st = diff_stream(L, stream, &cs, &capturing);
    if (st != GR_OK) return st;
    const bool host_g = !is_device_pointer(gout3);
    if (capturing) {
        // the kernels become nodes of the caller's graph; a replay reads the
        // signed counts and state of the last forward before it
        if (host_g) return fail(GR_EINVAL, "while its stream is being captured, gout3 must be device memory");
        const int64_t l0 = gr_kernel_launches();
        if (L->V > 0)
            launch_diff_backward(L->b, L->V, L->E, L->arg, L->st, gout3, L->theta_cnt, d_grad_xy, cs);
        count_launches((int)(l0 - gr_kernel_launches()));  // nothing ran yet
        GR_CU(cudaGetLastError());
        return GR_OK;
    }
    if (cs != L->stream) {
        GR_CU(cudaEventRecord(L->ev_din, cs));
        GR_CU(cudaStreamWaitEvent(L->stream, L->ev_din, 0));
    }
    const float *g = gout3;
    if (host_g) {
        GR_CU(cudaMemcpyAsync(L->gout3, gout3, sizeof(float) * 3, cudaMemcpyHostToDevice, L->stream));
        L->io_h2d += (int64_t)sizeof(float) * 3;
        g = L->gout3;
    }
    phase_begin(L, GR_PHASE_DIFF_BACKWARD);
    if (L->V > 0)
        launch_diff_backward(L->b, L->V, L->E, L->arg, L->st, g, L->theta_cnt, d_grad_xy, L->stream);
    phase_end(L, GR_PHASE_DIFF_BACKWARD);
    GR_CU(cudaGetLastError());
    if (cs != L->stream) {  // what follows on the caller's stream sees the gradient
        GR_CU(cudaEventRecord(L->ev_dout, L->stream));
        GR_CU(cudaStreamWaitEvent(cs, L->ev_dout, 0));
    }
    if (host_g) GR_CU(cudaStreamSynchronize(L->stream));  // the host buffer may go away
    return GR_OK;
}

gr_status gr_profile_enable(gr_layout *L, int enable) {
    g_err.clear();
    if (!L) return fail(GR_EINVAL, "layout is NULL");
    return set_profiling(L, enable != 0);
}

gr_status gr_profile_read(gr_layout *L, gr_profile *out, int reset) {
    g_err.clear();
    if (!L || !out) return fail(GR_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    bool pending = false;  // phases of calls that did not synchronise (gr_diff_backward)
    for (int ph = 0; ph < GR_NUM_PHASES; ++ph)
        if (L->pending[ph]) {
            cudaEventSynchronize(L->ev[2 * ph + 1]);
            pending = true;
        }
    if (pending) phase_collect(L);
    for (int ph = 0; ph < GR_NUM_PHASES; ++ph) {
        out->ms[ph] = L->prof_ms[ph];
        out->calls[ph] = L->prof_calls[ph];
        if (reset) {
            L->prof_ms[ph] = 0.0;
            L->prof_calls[ph] = 0;
        }
    }
    return GR_OK;
}

gr_status gr_io_bytes(gr_layout *L, int64_t *h2d, int64_t *d2h) {
    g_err.clear();
    if (!L || !h2d || !d2h) return fail(GR_EINVAL, "NULL argument");
    *h2d = L->io_h2d;
    *d2h = L->io_d2h;
    return GR_OK;
}

int64_t gr_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"

namespace gr {
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace gr
