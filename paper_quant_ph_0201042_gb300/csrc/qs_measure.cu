// Measurement gate, Sec. 2.2.3: for a random number r in [0, 1), the outcome
// is the index i with sum_{j<i} |alpha_j|^2 <= r < sum_{j<=i} |alpha_j|^2.
//
// Batched shots: (1) one block per chunk of 2^12 amplitudes sums |alpha|^2 in
// double precision; (2) one block turns the chunk sums into exclusive prefix
// sums; (3) one warp per shot binary-searches the chunk prefix for r, then
// walks its chunk 32 amplitudes at a time with a warp-wide inclusive prefix
// sum until the running sum exceeds r.  Sums are in double precision; the
// order of summation differs from a sequential cumulative sum only by
// rounding, which can move an outcome by one index when r lies within that
// rounding of a boundary.  An r at or beyond the total (rounding of a
// normalised state) gives the last index whose probability is not zero.
#include <algorithm>
#include <vector>

#include "qs_internal.cuh"

namespace qs {
namespace {

constexpr int CHUNK_LOG = 12;
constexpr int THREADS = 256;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__global__ void __launch_bounds__(THREADS) k_chunk_prob(const cplx<R> *__restrict__ a, uint64_t N,
                                                        double *__restrict__ sums) {
    __shared__ double sh[THREADS / 32];
    const uint64_t begin = uint64_t(blockIdx.x) << CHUNK_LOG;
    const uint64_t end = std::min<uint64_t>(begin + (uint64_t(1) << CHUNK_LOG), N);
    double acc = 0.0;
    for (uint64_t i = begin + threadIdx.x; i < end; i += THREADS) {
        const double x = double(a[i].x), y = double(a[i].y);
        acc = fma(x, x, fma(y, y, acc));
    }
    acc = wsum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < THREADS / 32 ? sh[threadIdx.x] : 0.0;
        v = wsum(v);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// Exclusive prefix of the chunk sums (one block; each thread a contiguous run).
__global__ void __launch_bounds__(1024) k_prefix(const double *__restrict__ sums, uint64_t C,
                                                 double *__restrict__ pre) {
    __shared__ double part[1024];
    const uint64_t per = (C + blockDim.x - 1) / blockDim.x;
    const uint64_t b = threadIdx.x * per, e = std::min<uint64_t>(b + per, C);
    double s = 0.0;
    for (uint64_t k = b; k < e; ++k) s += sums[k];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {   // prefix of the per-thread totals, in order
        double run = 0.0;
        for (unsigned t = 0; t < blockDim.x; ++t) {
            const double v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    double run = part[threadIdx.x];
    for (uint64_t k = b; k < e; ++k) {
        pre[k] = run;
        run += sums[k];
    }
}

template <typename R>
__global__ void __launch_bounds__(THREADS) k_sample(const cplx<R> *__restrict__ a, uint64_t N, uint64_t C,
                                                    const double *__restrict__ sums, const double *__restrict__ pre,
                                                    const double *__restrict__ r, uint64_t shots,
                                                    uint64_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t shot = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (shot >= shots) return;
    const double x = r[shot];
    // last chunk with pre <= x
    uint64_t lo = 0, hi = C;   // pre[lo] <= x (pre[0] = 0 <= x), answer in [lo, hi)
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (pre[mid] <= x) lo = mid; else hi = mid;
    }
    // if x is beyond this chunk's total, step back to the last chunk with mass
    uint64_t c = lo;
    double run = pre[c];
    const uint64_t begin = c << CHUNK_LOG;
    const uint64_t end = std::min<uint64_t>(begin + (uint64_t(1) << CHUNK_LOG), N);
    uint64_t found = ~uint64_t(0), last_nz = ~uint64_t(0);
    for (uint64_t base = begin; base < end; base += 32) {
        const uint64_t i = base + lane;
        double p = 0.0;
        if (i < end) {
            const double re = double(a[i].x), im = double(a[i].y);
            p = fma(re, re, im * im);
        }
        // inclusive warp prefix of p
        double inc = p;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const double upto = run + inc;               // sum_{j <= i}
        const bool hit = (i < end) && p > 0.0 && x < upto;
        const unsigned bh = __ballot_sync(0xffffffffu, hit);
        const unsigned bnz = __ballot_sync(0xffffffffu, (i < end) && p > 0.0);
        if (bnz) last_nz = base + (31 - __clz(bnz));
        if (bh) { found = base + (__ffs(bh) - 1); break; }
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) {
        if (found == ~uint64_t(0)) {
            // x at or beyond the running total: the last index with mass in this
            // or an earlier chunk
            if (last_nz == ~uint64_t(0)) {
                uint64_t cc = c;
                while (cc > 0 && sums[cc] == 0.0) --cc;
                last_nz = (cc << CHUNK_LOG) + ((uint64_t(1) << CHUNK_LOG) - 1);
                if (last_nz >= N) last_nz = N - 1;
                // walk back inside the chunk to a non-zero amplitude
                while (last_nz > (cc << CHUNK_LOG)) {
                    const double re = double(a[last_nz].x), im = double(a[last_nz].y);
                    if (re != 0.0 || im != 0.0) break;
                    --last_nz;
                }
            }
            found = last_nz;
        }
        out[shot] = found;
    }
}

template <typename R>
qs_status measure_t(qs_state *s, const double *r, size_t shots, uint64_t *out) {
    const uint64_t N = uint64_t(1) << s->n;
    const uint64_t C = (N + (uint64_t(1) << CHUNK_LOG) - 1) >> CHUNK_LOG;
    cudaStream_t st = s->stream;
    void *buf = nullptr;
    const size_t bytes = sizeof(double) * (2 * C + shots) + sizeof(uint64_t) * shots;
    cudaError_t e = cudaMallocAsync(&buf, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "measure: device allocation failed");
    }
    double *sums = static_cast<double *>(buf), *pre = sums + C, *dr = pre + C;
    uint64_t *dout = reinterpret_cast<uint64_t *>(dr + shots);
    e = cudaMemcpyAsync(dr, r, sizeof(double) * shots, cudaMemcpyHostToDevice, st);
    const cplx<R> *a = static_cast<const cplx<R> *>(s->d);
    if (e == cudaSuccess) {
        k_chunk_prob<R><<<unsigned(C), THREADS, 0, st>>>(a, N, sums);
        k_prefix<<<1, 1024, 0, st>>>(sums, C, pre);
        const uint64_t warps = shots;
        k_sample<R><<<unsigned((warps * 32 + THREADS - 1) / THREADS), THREADS, 0, st>>>(a, N, C, sums, pre, dr, shots,
                                                                                         dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "measure");
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_measure(qs_state *s, const double *r, size_t shots, uint64_t *out) {
    if (!s || (shots > 0 && (!r || !out))) return fail(QS_EINVAL, "NULL argument");
    if (shots == 0) return QS_OK;
    if (shots > (size_t(1) << 26)) return fail(QS_ERANGE, "measure: more than 2^26 shots per call");
    for (size_t k = 0; k < shots; ++k)
        if (!(r[k] >= 0.0 && r[k] < 1.0)) return fail(QS_EINVAL, "measure: r must be in [0, 1)");
    return s->dt == QS_C64 ? measure_t<float>(s, r, shots, out) : measure_t<double>(s, r, shots, out);
}
