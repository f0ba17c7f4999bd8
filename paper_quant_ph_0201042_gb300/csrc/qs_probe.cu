// Measured throughput of the fused multiply-add pipes: the denominators of
// the arithmetic rooflines (no counterpart in the paper; a measurement
// service of the library).
//
// Every thread runs sixteen independent FMA chains (enough to cover the
// pipes' latency) for a fixed number of iterations, on a grid of eight
// 256-thread CTAs per SM.  The rate is FMA instructions times lanes per
// second, from CUDA events around single launches on a stream of the probe's
// own: the best of five, after about a fifth of a second of the same
// launches, so that the SM clock has left its idle level (a process's first
// kernels otherwise run before the clock has ramped up).  No clock or other
// device setting is touched.
#include "qs_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 16;   // independent FMA chains per thread

template <typename R>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_chains(R *__restrict__ sink, R a, R b, int iters) {
    constexpr int C = CHAINS;
    R x[C];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = R(threadIdx.x) + R(c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < C; ++c) x[c] = fma(x[c], a, b);
    }
    // one store per thread keeps the chains alive
    R s = R(0);
#pragma unroll
    for (int c = 0; c < C; ++c) s += x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
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
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 0.f;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        // warm-up: launches until about 200 ms have passed (at most 4000)
        float spent = 0.f;
        for (int round = 0; round < 40 && spent < 200.f && e == cudaSuccess; ++round) {
            e = cudaEventRecord(e0, st);
            for (int k = 0; k < 100 && e == cudaSuccess; ++k) {
                k_fma_chains<R><<<blocks, PROBE_THREADS, 0, st>>>(sink, R(0.999), R(1e-3), iters);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            spent += ms;
        }
        for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, st);
            k_fma_chains<R><<<blocks, PROBE_THREADS, 0, st>>>(sink, R(0.999), R(1e-3), iters);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    if (e != cudaSuccess) return qs::cuda_fail(e, "qs_alu_peak: timing");
    if (best <= 0.f) return qs::fail(QS_ECUDA, "qs_alu_peak: no timing");
    *per_s = double(blocks) * PROBE_THREADS * double(CHAINS) * iters / (double(best) * 1e-3);
    return QS_OK;
}

}  // namespace

extern "C" qs_status qs_alu_peak(int kind, double *fma_per_s) {
    if (!fma_per_s) return qs::fail(QS_EINVAL, "qs_alu_peak: NULL result");
    if (kind == 0) return measure<float>(4096, fma_per_s);
    if (kind == 1) return measure<double>(128, fma_per_s);
    return qs::fail(QS_EINVAL, "qs_alu_peak: kind must be 0 (single) or 1 (double)");
}
