// k_noalloc.cu -- gr_crossing_angle_noalloc: crossings and crossing angle of
// one small layout using no device allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc -- a process whose device
// memory is already handed out to its own pool allocator under a fixed
// budget, or a latency-critical caller for whom cudaMalloc / cudaFree, which
// may block or synchronise the device, are not acceptable.  gr_layout_create
// allocates per layout; this entry point works entirely in a fixed scratch
// array that every GPU loading this library holds until the process exits.
//
// Scratch: the file-scope array g_noalloc_scratch below (kNoAllocMaxEdges
// compacted segments with their edge ids, line directions and squared
// lengths, plus one accumulator block and one result slot, about 1 MiB).
// Host code cannot use the array's name as a device address: every call looks
// the address up with cudaGetSymbolAddress while its device is current (a host
// call that allocates nothing), so a device reset between calls, which reloads
// the library's module at a possibly different address, cannot leave a stale
// address behind.  The first call on a device is the set-up: it also makes the
// runtime load the module there, so that first call should come before any
// stream capture on the device.
//
// Every call reuses the same array and leaves its contents behind; the
// accumulators are cleared at the start of each call.  Calls whose work
// overlaps on the GPU (other streams, other host threads) race on the array:
// issue them one after another.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>

#include "gr_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxEdges = GR_NOALLOC_MAX_EDGES;

struct NoAllocScratch {
    gr::DevAcc acc;
    gr_crossing_angle_result result;
    gr::SegRec seg[kNoAllocMaxEdges];
    int32_t seg_eid[kNoAllocMaxEdges];
    uint32_t seg_theta[kNoAllocMaxEdges];
    int64_t len2[kNoAllocMaxEdges];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

gr_status noalloc_fail(gr_status st, const std::string &msg) {
    gr::set_last_error(msg.c_str());
    return st;
}

// Folds the accumulators into the caller-visible result (one thread).
__global__ void k_noalloc_result(const gr::DevAcc *__restrict__ acc, double ideal,
                                 gr_crossing_angle_result *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    gr_crossing_angle_result r;
    memset(&r, 0, sizeof(r));
    const uint64_t ec = acc->proper + acc->touching;
    const uint64_t ns = acc->n_seg;
    r.c.crossings = (int64_t)ec;
    r.c.proper = (int64_t)acc->proper;
    r.c.touching = (int64_t)acc->touching;
    r.c.collinear_overlaps = (int64_t)acc->collinear;
    r.c.zero_length_edges = (int64_t)acc->zero_len;
    r.c.pairs_tested = (int64_t)(ns * (ns - (ns > 0)) / 2);
    const double dev = ((double)acc->dev_hi * 18446744073709551616.0 + (double)acc->dev_lo) * gr::kAngleUnit;
    r.angle_dev_sum = dev;
    r.ideal_rad = ideal;
    r.E_ca = ec > 0 ? 1.0 - dev / (ideal * (double)ec) : 1.0;
    *out = r;
}

bool is_device_memory(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device.
gr_status scratch_address(NoAllocScratch **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(GR_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    }
    *out = (NoAllocScratch *)p;
    return GR_OK;
}

}  // namespace

extern "C" {

gr_status gr_crossing_angle_noalloc(const int32_t *d_xy, int64_t V, const int32_t *d_edges, int64_t E,
                                    double ideal_rad, gr_crossing_angle_result *out, gr_stream_t stream) {
    gr::set_last_error("");
    if (!out) return noalloc_fail(GR_EINVAL, "out is NULL");
    if (V < 0 || E < 0 || V >= (int64_t(1) << 31)) return noalloc_fail(GR_EINVAL, "V and E must be >= 0, V < 2^31");
    if (E > kNoAllocMaxEdges)
        return noalloc_fail(GR_EINVAL, "E = " + std::to_string(E) + " exceeds the no-allocation limit of " +
                                           std::to_string(kNoAllocMaxEdges) + " edges");
    if ((V > 0 && !d_xy) || (E > 0 && !d_edges)) return noalloc_fail(GR_EINVAL, "NULL input pointer");
    if (E > 0 && V < 2) return noalloc_fail(GR_EINVAL, "edges need at least two vertices");
    const double ideal = ideal_rad > 0.0 ? ideal_rad : 7.0 * M_PI / 18.0;
    if (!(ideal <= M_PI / 2 + 1e-15)) return noalloc_fail(GR_EINVAL, "ideal angle must be in (0, pi/2]");
    if ((V > 0 && !is_device_memory(d_xy)) || (E > 0 && !is_device_memory(d_edges)))
        return noalloc_fail(GR_EINVAL, "inputs must be device memory");
    NoAllocScratch *sc = nullptr;
    gr_status st = scratch_address(&sc);
    if (st != GR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    gr::Buffers b;  // views into the scratch array; nothing is allocated
    b.seg = sc->seg;
    b.seg_eid = sc->seg_eid;
    b.seg_theta = sc->seg_theta;
    b.len2 = sc->len2;
    b.acc = &sc->acc;
    cudaError_t e = cudaMemsetAsync(&sc->acc, 0, sizeof(gr::DevAcc), s);
    if (e == cudaSuccess) {
        gr::launch_gather(d_xy, V, d_edges, E, b, s);
        const uint32_t ideal_u = (uint32_t)llrint(ideal / M_PI * 4294967296.0);
        gr::launch_crossings_allpairs(b, E, ideal_u, gr::PerEdge{}, s);
        gr::count_launches(1);
        k_noalloc_result<<<1, 32, 0, s>>>(&sc->acc, ideal, &sc->result);
        e = cudaGetLastError();
    }
    uint32_t status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &sc->acc.status, sizeof(status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(GR_ECUDA, std::string("gr_crossing_angle_noalloc: ") + cudaGetErrorString(e));
    }
    if (status & gr::ST_BAD_ID) return noalloc_fail(GR_EINVAL, "vertex id outside [0, V) or self-loop in the edge list");
    if (status & gr::ST_BAD_COORD) return noalloc_fail(GR_ERANGE, "vertex coordinate outside [0, 65536)");
    const cudaMemcpyKind k = is_device_memory(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    e = cudaMemcpyAsync(out, &sc->result, sizeof(gr_crossing_angle_result), k, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(GR_ECUDA, std::string("gr_crossing_angle_noalloc: ") + cudaGetErrorString(e));
    }
    return GR_OK;
}

}  // extern "C"
