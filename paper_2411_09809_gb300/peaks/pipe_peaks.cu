// pipe_peaks.cu -- measured throughput of the instruction classes the pair
// kernels are built from (integer add, logic, compare/select, integer
// multiply-add, FP32 fused multiply-add, the special-function unit, FP64
// fused multiply-add), so that roofline denominators are measured on the part
// rather than assumed.  A measurement aid loaded by bench.py; not part of
// libgr.
//
// Each kernel runs kChains independent dependency chains of one operation
// per thread for kIters iterations on every SM (8 blocks of 256 threads per
// SM); operands depend on the previous iteration and the results are
// written out, so nothing can be folded away.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256, kChains = 8, kIters = 2048;

enum Op { OP_IADD3 = 0, OP_LOP3, OP_IMNMX, OP_IMAD, OP_FFMA, OP_MUFU, OP_DFMA, OP_COUNT };

template <int OP>
__global__ void __launch_bounds__(kThreads) k_pipe(const uint32_t *__restrict__ in, uint32_t *__restrict__ out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t a = in[t & 1023], b = in[(t + 7) & 1023], c = in[(t + 13) & 1023];
    if (OP == OP_FFMA || OP == OP_MUFU) {
        float x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __uint_as_float((a + k) & 0x3f7fffffu) + 1.0f;
        const float fb = __uint_as_float((b & 0x007fffffu) | 0x3f000000u), fc = __uint_as_float(c & 0x3effffffu);
        for (int i = 0; i < kIters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (OP == OP_FFMA) x[k] = fmaf(x[k], fb, fc);
                else x[k] = rsqrtf(x[k]);
            }
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += x[k];
        out[t] = __float_as_uint(s);
    } else if (OP == OP_DFMA) {
        double x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = (double)((a + k) & 0xffff) * 1e-5 + 1.0;
        const double db = 1.0 - (double)(b & 0xff) * 1e-9, dc = (double)(c & 0xff) * 1e-9;
        for (int i = 0; i < kIters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], db, dc);
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += x[k];
        out[t] = (uint32_t)__double2hiint(s);
    } else {
        uint32_t x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = a + (uint32_t)k;
        // each chain also reads its neighbour's value, so no closed form exists
        for (int i = 0; i < kIters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                const uint32_t y = x[(k + 1) % kChains];
                if (OP == OP_IADD3) x[k] = x[k] + y + c;
                else if (OP == OP_LOP3) x[k] = (x[k] ^ y) & (c | b);   // (c | b) is loop-invariant: one LOP3
                else if (OP == OP_IMNMX) x[k] = min(x[k], y) + c;      // a compare-select and an add
                else x[k] = x[k] * y + c;                              // IMAD
            }
        }
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s ^= x[k];
        out[t] = s;
    }
}

template <int OP>
double time_op(int blocks, const uint32_t *in, uint32_t *out, cudaEvent_t e0, cudaEvent_t e1) {
    k_pipe<OP><<<blocks, kThreads>>>(in, out);  // warm-up
    cudaEventRecord(e0);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_pipe<OP><<<blocks, kThreads>>>(in, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double ops = (double)blocks * kThreads * kChains * kIters * reps;
    // operations per iteration and chain: two for the compare-select-and-add form
    return ops * (OP == OP_IMNMX ? 2.0 : 1.0) / (ms * 1e-3);
}

}  // namespace

// Measures, on the current device, the thread-operations per second of each
// class in the order IADD3, LOP3, IMNMX (+ IADD), IMAD, FFMA, MUFU (rsqrt),
// DFMA into lane_ops_per_s[0..n).  Returns the number written, or -1 on a
// CUDA error.
extern "C" int gr_peaks_measure(double *lane_ops_per_s, int n) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    const int blocks = sms * 8;
    uint32_t *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, 1024 * sizeof(uint32_t)) != cudaSuccess) return -1;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(uint32_t)) != cudaSuccess) {
        cudaFree(in);
        return -1;
    }
    cudaMemset(in, 0x5a, 1024 * sizeof(uint32_t));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double r[OP_COUNT];
    r[OP_IADD3] = time_op<OP_IADD3>(blocks, in, out, e0, e1);
    r[OP_LOP3] = time_op<OP_LOP3>(blocks, in, out, e0, e1);
    r[OP_IMNMX] = time_op<OP_IMNMX>(blocks, in, out, e0, e1);
    r[OP_IMAD] = time_op<OP_IMAD>(blocks, in, out, e0, e1);
    r[OP_FFMA] = time_op<OP_FFMA>(blocks, in, out, e0, e1);
    r[OP_MUFU] = time_op<OP_MUFU>(blocks, in, out, e0, e1);
    r[OP_DFMA] = time_op<OP_DFMA>(blocks, in, out, e0, e1);
    const cudaError_t err = cudaDeviceSynchronize();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(in);
    cudaFree(out);
    if (err != cudaSuccess) return -1;
    int w = 0;
    for (; w < n && w < OP_COUNT; ++w) lane_ops_per_s[w] = r[w];
    return w;
}
