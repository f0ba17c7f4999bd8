// qs_norm_noalloc: the norm reduction without any allocation.
//
// Some callers cannot allocate device memory when they need a norm: a host
// framework that owns the whole device memory budget through its own pool,
// a latency-critical loop in which cudaMalloc/cudaFree would synchronize the
// device, or a component that is not allowed to touch the allocator at all.
// This entry point serves them: the caller passes the state and a device
// location for the result, and the partial sums live in a fixed array of
// this library's device memory (loaded with the module, held by every GPU
// that loads the library until the process exits).
//
// The reduction is a variant of the norm reduction of qs_reduce.cu with a
// different summation tree: one block per contiguous chunk of 2^16 amplitudes
// writes one double partial sum, then one block adds the partials in a fixed
// order.  The result is deterministic for a given n, but it may differ from
// qs_norm's in the last bits, because qs_norm's first level strides over the
// whole vector instead.  The scratch array holds at most 65536 partials
// (1 MiB), so states of up to 2^32 amplitudes are accepted.
//
// The array's device address is resolved once per device and cached; a
// cudaDeviceReset unloads the module, so the entry point must not be used
// across a device reset (nor may the states it reads, which the reset frees).
#include <mutex>

#include "qs_internal.cuh"

namespace {

constexpr int CHUNK_LOG = 16;                 // amplitudes per block
constexpr int THREADS = 256;
constexpr uint64_t MAX_CHUNKS = uint64_t(1) << 16;

// Scratch: one partial sum per chunk.  Every call overwrites the entries it
// reads, so nothing needs clearing; concurrent calls share it.
static __device__ __align__(256) double g_noalloc_partials[MAX_CHUNKS];

__device__ __forceinline__ double warp_add(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_add(double v) {
    __shared__ double sh[THREADS / 32];
    v = warp_add(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = l < THREADS / 32 ? sh[l] : 0.0;
        v = warp_add(v);
    }
    return v;
}

template <typename V>
__global__ void __launch_bounds__(THREADS) k_chunk_norm(const V *__restrict__ a, uint64_t N, double *__restrict__ part) {
    const uint64_t begin = uint64_t(blockIdx.x) << CHUNK_LOG;
    const uint64_t end = begin + (uint64_t(1) << CHUNK_LOG) < N ? begin + (uint64_t(1) << CHUNK_LOG) : N;
    double acc = 0.0;
    for (uint64_t i = begin + threadIdx.x; i < end; i += THREADS) {
        const double x = double(a[i].x), y = double(a[i].y);
        acc = fma(x, x, acc);
        acc = fma(y, y, acc);
    }
    acc = block_add(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(THREADS) k_sum_partials(const double *__restrict__ part, uint64_t np,
                                                          double *__restrict__ out) {
    double acc = 0.0;
    for (uint64_t k = threadIdx.x; k < np; k += THREADS) acc += part[k];
    acc = block_add(acc);
    if (threadIdx.x == 0) out[0] = acc;
}

// Device address of the scratch array, resolved once per device.
std::mutex g_mu;
double *g_addr[64] = {};

qs_status scratch_address(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev < 0 || dev >= 64) return qs::fail(QS_EUNSUPPORTED, "device index beyond 63");
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return qs::cuda_fail(e, "qs_norm_noalloc: scratch address");
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return QS_OK;
}

}  // namespace

extern "C" qs_status qs_norm_noalloc(const void *dev_state, int n, qs_dtype dt, double *dev_out, void *stream) {
    if (!dev_state || !dev_out) return qs::fail(QS_EINVAL, "qs_norm_noalloc: NULL pointer");
    if (dt != QS_C64 && dt != QS_C128) return qs::fail(QS_EINVAL, "qs_norm_noalloc: bad dtype");
    // the kernel reads float2 / double2 amplitudes and writes one double
    const uintptr_t amp_align = dt == QS_C128 ? 16 : 8;
    if (reinterpret_cast<uintptr_t>(dev_state) % amp_align)
        return qs::fail(QS_EINVAL, dt == QS_C128 ? "qs_norm_noalloc: dev_state not 16-byte aligned"
                                                 : "qs_norm_noalloc: dev_state not 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(dev_out) % 8) return qs::fail(QS_EINVAL, "qs_norm_noalloc: dev_out not 8-byte aligned");
    if (n < 1) return qs::fail(QS_ERANGE, "qs_norm_noalloc: n < 1");
    if (n > CHUNK_LOG + 16)
        return qs::fail(QS_ERANGE, "qs_norm_noalloc: n > 32 (its fixed scratch holds 65536 partial sums of "
                                   "2^16 amplitudes each)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return qs::cuda_fail(e, "qs_norm_noalloc: device");
    double *part = nullptr;
    qs_status st = scratch_address(dev, &part);
    if (st != QS_OK) return st;
    const uint64_t N = uint64_t(1) << n;
    const uint64_t chunks = (N + (uint64_t(1) << CHUNK_LOG) - 1) >> CHUNK_LOG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dt == QS_C64)
        k_chunk_norm<float2><<<unsigned(chunks), THREADS, 0, s>>>(static_cast<const float2 *>(dev_state), N, part);
    else
        k_chunk_norm<double2><<<unsigned(chunks), THREADS, 0, s>>>(static_cast<const double2 *>(dev_state), N, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return qs::cuda_fail(e, "qs_norm_noalloc: launch");
    k_sum_partials<<<1, THREADS, 0, s>>>(part, chunks, dev_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return qs::cuda_fail(e, "qs_norm_noalloc: launch");
    return QS_OK;
}
