// gr_api.cu -- the C ABI of include/gr.h: layout objects, argument checks,
// device memory, and the order in which the kernels of one evaluation are
// enqueued.
#include <cuda_runtime.h>

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
    gr_options opt{};
    Buffers b;
    gr_result *h_result = nullptr;  // pinned
    DevAcc *h_acc = nullptr;        // pinned
};

namespace {

void free_layout(gr_layout *L) {
    if (!L) return;
    Buffers &b = L->b;
    void *ptrs[] = {b.xy, b.edges, b.seg, b.seg_eid, b.len2, b.acc, b.elv_part, b.ma_part,
                    b.ma_cnt, b.deg, b.deg_fill, b.dirs, b.scan_tmp, b.result};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (L->h_result) cudaFreeHost(L->h_result);
    if (L->h_acc) cudaFreeHost(L->h_acc);
    delete L;
}

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
    GR_TRY(dalloc(&b.len2, (size_t)E));
    GR_TRY(dalloc(&b.acc, 1));
    GR_TRY(dalloc(&b.elv_part, 2 * (size_t)kElvBlocks));
    GR_TRY(dalloc(&b.ma_part, 1024));
    GR_TRY(dalloc(&b.ma_cnt, 1024));
    GR_TRY(dalloc(&b.deg, (size_t)V + 1));
    GR_TRY(dalloc(&b.deg_fill, (size_t)V));
    GR_TRY(dalloc(&b.dirs, 2 * (size_t)E));
    GR_TRY(dalloc(&b.scan_tmp, (size_t)kScanMaxBlocks));
    GR_TRY(dalloc(&b.result, 1));
#undef GR_TRY
    GR_CU(cudaMallocHost((void **)&L->h_result, sizeof(gr_result)));
    GR_CU(cudaMallocHost((void **)&L->h_acc, sizeof(DevAcc)));
    GR_CU(cudaMemsetAsync(b.acc, 0, sizeof(DevAcc), L->stream));
    return GR_OK;
}

// Copies the inputs into the layout's own buffers and runs a1 (gather and
// validation).  Stream-ordered.
gr_status enqueue_inputs(gr_layout *L, const void *xy, const int32_t *edges) {
    cudaStream_t s = L->stream;
    const int64_t V = L->V, E = L->E;
    GR_CU(cudaMemsetAsync(L->b.acc, 0, offsetof(DevAcc, eval_status), s));
    if (V > 0) {
        const cudaMemcpyKind k = is_device_pointer(xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GR_CU(cudaMemcpyAsync(L->b.xy, xy, sizeof(int32_t) * 2 * V, k, s));
    }
    if (E > 0 && edges) {
        const cudaMemcpyKind k = is_device_pointer(edges) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GR_CU(cudaMemcpyAsync(L->b.edges, edges, sizeof(int32_t) * 2 * E, k, s));
    }
    launch_check_vertices(L->b.xy, V, L->b, s);
    launch_gather(L->b.xy, V, L->b.edges, E, L->b, s);
    GR_CU(cudaGetLastError());
    return GR_OK;
}

gr_status status_to_error(uint32_t st) {
    if (st & ST_BAD_ID) return fail(GR_EINVAL, "vertex id outside [0, V) or self-loop in the edge list");
    if (st & ST_BAD_COORD) return fail(GR_ERANGE, "vertex coordinate outside [0, 65536)");
    if (st & ST_SCAN_OVERFLOW) return fail(GR_ENOTSUP, "an offset table exceeded 2^32 entries");
    if (st & ST_OVERFLOW) return fail(GR_ENOMEM, "grid record buffer overflow");
    return GR_OK;
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

}  // namespace

extern "C" {

const char *gr_last_error(void) { return g_err.c_str(); }

const char *gr_version(void) { return "gr 0.1 (sm_103a)"; }

gr_status gr_layout_create(gr_layout **out, const void *xy, gr_coord_type coord_type, int64_t V,
                           const int32_t *edges, int64_t E, const gr_options *opt,
                           gr_stream_t stream) {
    g_err.clear();
    if (!out) return fail(GR_EINVAL, "out is NULL");
    if (coord_type != GR_COORD_I32) return fail(GR_ENOTSUP, "only GR_COORD_I32 layouts are supported");
    if (V < 0 || E < 0 || V >= (int64_t(1) << 31) || E >= (int64_t(1) << 31))
        return fail(GR_EINVAL, "V and E must be in [0, 2^31)");
    if ((V > 0 && !xy) || (E > 0 && !edges)) return fail(GR_EINVAL, "NULL input pointer");
    if (E > 0 && V < 2) return fail(GR_EINVAL, "edges need at least two vertices");
    gr_layout *L = new gr_layout;
    L->V = V;
    L->E = E;
    L->stream = (cudaStream_t)stream;
    if (opt) L->opt = *opt;
    gr_status st = alloc_layout(L);
    if (st == GR_OK) st = enqueue_inputs(L, xy, edges);
    if (st == GR_OK) {
        cudaError_t e = cudaMemcpyAsync(L->h_acc, L->b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "validating the layout");
        else st = status_to_error(L->h_acc->status);
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

gr_status gr_evaluate(gr_layout *L, uint32_t metrics, const gr_params *params, gr_result *out) {
    g_err.clear();
    if (!L || !out) return fail(GR_EINVAL, "NULL argument");
    if (metrics & ~GR_METRIC_ALL) return fail(GR_EINVAL, "unknown metric bits");
    double ideal;
    int64_t d;
    gr_status st = read_params(params, &ideal, &d);
    if (st != GR_OK) return st;
    cudaStream_t s = L->stream;
    Buffers &b = L->b;
    const int64_t V = L->V, E = L->E;
    GR_CU(cudaMemsetAsync((char *)b.acc + offsetof(DevAcc, eval_status), 0,
                          sizeof(DevAcc) - offsetof(DevAcc, eval_status), s));
    int32_t path = 0, occl_path = 0;
    if (metrics & GR_METRIC_EDGE_LENGTH) launch_elv(b, E, s);
    if (metrics & GR_METRIC_MIN_ANGLE) launch_min_angle(b, V, E, s);
    if (metrics & GR_METRIC_OCCLUSION) {
        launch_occlusion_allpairs(b, V, d, s);
        occl_path = GR_PATH_ALLPAIRS;
    }
    if (metrics & GR_METRIC_CROSSINGS) {
        launch_crossings_allpairs(b, E, (float)ideal, PerEdge{}, s);
        path = GR_PATH_ALLPAIRS;
    }
    launch_finalize(b, metrics, E, ideal, d, V > 0 ? min_angle_blocks(V) : 0, path, 0, occl_path, -1, s);
    GR_CU(cudaGetLastError());
    GR_CU(cudaMemcpyAsync(L->h_result, b.result, sizeof(gr_result), cudaMemcpyDeviceToHost, s));
    GR_CU(cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
    GR_CU(cudaStreamSynchronize(s));
    st = status_to_error(L->h_acc->status | L->h_acc->eval_status);
    if (st != GR_OK) return st;
    *out = *L->h_result;
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

gr_status gr_crossings_per_edge(gr_layout *L, double ideal_rad, int64_t *d_counts, double *d_dev) {
    g_err.clear();
    if (!L || (L->E > 0 && (!d_counts || !d_dev))) return fail(GR_EINVAL, "NULL argument");
    gr_params p{ideal_rad, 0};
    double ideal;
    int64_t d;
    gr_status st = read_params(&p, &ideal, &d);
    if (st != GR_OK) return st;
    const int64_t E = L->E;
    if (E == 0) return GR_OK;
    if (!is_device_pointer(d_counts) || !is_device_pointer(d_dev))
        return fail(GR_EINVAL, "per-edge outputs must be device memory");
    cudaStream_t s = L->stream;
    Buffers &b = L->b;
    GR_CU(cudaMemsetAsync((char *)b.acc + offsetof(DevAcc, eval_status), 0,
                          sizeof(DevAcc) - offsetof(DevAcc, eval_status), s));
    GR_CU(cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * 3 * E, s));
    GR_CU(cudaMemsetAsync(d_dev, 0, sizeof(double) * E, s));
    PerEdge pe;
    pe.counts = (uint64_t *)d_counts;
    pe.dev = (uint64_t *)d_dev;
    launch_crossings_allpairs(b, E, (float)ideal, pe, s);
    launch_per_edge_export(pe.dev, E, s);
    GR_CU(cudaGetLastError());
    GR_CU(cudaMemcpyAsync(L->h_acc, b.acc, sizeof(DevAcc), cudaMemcpyDeviceToHost, s));
    GR_CU(cudaStreamSynchronize(s));
    return status_to_error(L->h_acc->status | L->h_acc->eval_status);
}

}  // extern "C"
