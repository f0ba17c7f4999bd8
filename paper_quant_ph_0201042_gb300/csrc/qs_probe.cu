// Measured throughput of the fused multiply-add pipes: the denominators of
// the arithmetic rooflines (no counterpart in the paper; a measurement
// service of the library).
//
// Every thread runs eight independent FMA chains (enough to cover the
// pipes' latency) for a fixed number of iterations, on a grid of eight
// 256-thread CTAs per SM.  The rate is FMA instructions times lanes per
// second, from CUDA events around the second of two identical launches.  No
// clock or other device setting is touched.
#include "qs_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;

template <typename R>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_chains(R *__restrict__ sink, R a, R b, int iters) {
    R x0 = R(threadIdx.x), x1 = x0 + R(1), x2 = x0 + R(2), x3 = x0 + R(3);
    R x4 = x0 + R(4), x5 = x0 + R(5), x6 = x0 + R(6), x7 = x0 + R(7);
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    // one store per thread keeps the chains alive
    sink[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

template <typename R>
qs_status measure(int iters, double *per_s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return qs::cuda_fail(e, "qs_alu_peak: device");
    const int blocks = sms * 8;
    R *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(R) * size_t(blocks) * PROBE_THREADS);
    if (e != cudaSuccess) return qs::fail(QS_ENOMEM, "qs_alu_peak: sink allocation failed");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fma_chains<R><<<blocks, PROBE_THREADS>>>(sink, R(0.999), R(1e-3), iters);   // warm-up
        e = cudaEventRecord(e0);
        k_fma_chains<R><<<blocks, PROBE_THREADS>>>(sink, R(0.999), R(1e-3), iters);
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return qs::cuda_fail(e, "qs_alu_peak: timing");
    *per_s = double(blocks) * PROBE_THREADS * 8.0 * iters / (double(ms) * 1e-3);
    return QS_OK;
}

}  // namespace

extern "C" qs_status qs_alu_peak(int kind, double *fma_per_s) {
    if (!fma_per_s) return qs::fail(QS_EINVAL, "qs_alu_peak: NULL result");
    if (kind == 0) return measure<float>(8192, fma_per_s);
    if (kind == 1) return measure<double>(256, fma_per_s);
    return qs::fail(QS_EINVAL, "qs_alu_peak: kind must be 0 (single) or 1 (double)");
}
