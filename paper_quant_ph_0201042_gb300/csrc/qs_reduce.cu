// Reductions over the register in double precision: the norm (Sec. 2.1 unit
// length), the probability of one basis state or of one qubit reading 1 (the
// |0><0| term of Sec. 4.3.1, the amplitude of the marked element of Sec. 5.3),
// Pauli expectation values and inner products (the fidelity of Sec. 5.2).
//
// Two deterministic levels: RED_BLOCKS blocks each sum a fixed grid-stride
// slice of the vector, then one block sums the RED_BLOCKS partials in a fixed
// order.  The result stays on the device (s->result) and is copied to pinned
// host memory by the caller.
//
// Each thread accumulates its slice in double-single arithmetic (qs_ds.cuh):
// a product of two amplitude components is an exact pair of floats (plus the
// cross terms of their low parts for a complex128 state, whose doubles are
// split into float pairs with integer instructions), added into a float-pair
// accumulator with TwoSum.  The per-thread sums (48 significant bits) become
// doubles once, and the warp, block and final sums run in double precision.
// On this part the double-precision pipe issues about a sixty-fourth of the
// single-precision rate, so two double multiply-adds per amplitude would take
// longer than reading the amplitude from HBM.
#include "qs_ds.cuh"
#include "qs_internal.cuh"

namespace qs {

namespace {

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Block-wide sum in a fixed order; valid in thread 0.
__device__ __forceinline__ double2 block_sum(double2 v) {
    __shared__ double2 sh[32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        v = l < nw ? sh[l] : make_double2(0.0, 0.0);
        v = warp_sum(v);
    }
    return v;
}

template <typename R>
__device__ __forceinline__ double2 ld(const cplx<R> *a, uint64_t i) {
    const cplx<R> v = a[i];
    return make_double2(double(v.x), double(v.y));
}

// An amplitude as double-single components (re = rh + rl, im = ih + il).
__device__ __forceinline__ ds::camp lds(const float2 *a, uint64_t i) {
    const float2 v = a[i];
    return {v.x, 0.f, v.y, 0.f};
}
__device__ __forceinline__ ds::camp lds(const double2 *a, uint64_t i) {
    const double2 v = a[i];
    return ds::load(v.x, v.y);
}

// A float-pair accumulator: s = h + l.  LOWS: the components have low parts
// (complex128); complex64 components are single floats.
template <bool LOWS>
struct DAcc {
    float h = 0.f, l = 0.f;
    // s += sg * (a * b) for float pairs a, b (sg = +1 or -1); the product of
    // the two low parts is dropped (2^-48 of the term)
    __device__ __forceinline__ void add(float ah, float al, float bh, float bl, float sg) {
        const float p = ds::mul(sg * ah, bh);
        float e = ds::fma(sg * ah, bh, -p);
        if (LOWS) {
            e = ds::fma(sg * ah, bl, e);
            e = ds::fma(sg * al, bh, e);
        }
        float t, r;
        ds::two_sum(h, p, t, r);
        ds::fast_two_sum(t, ds::add(l, ds::add(r, e)), h, l);
    }
    __device__ __forceinline__ double value() const { return double(h) + double(l); }
};

// kind RED_NORM: sum |a_i|^2
// kind RED_PROB_BIT: sum over i with (i & arg0) != 0 of |a_i|^2
// kind RED_PAULI: sum_i conj(a[i ^ arg0]) a[i] (-1)^popcount(i & arg1)
//   (with arg0 != 0 summed over pairs, each amplitude read once)
// kind RED_INNER: sum_i conj(a_i) b_i
template <typename R, int KIND>
__global__ void __launch_bounds__(RED_THREADS) k_partial(const cplx<R> *__restrict__ a,
                                                         const cplx<R> *__restrict__ b, uint64_t N,
                                                         uint64_t arg0, uint64_t arg1,
                                                         double2 *__restrict__ partial) {
    DAcc<sizeof(R) == 8> ar, ai;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (KIND == RED_NORM || (KIND == RED_PAULI && arg0 == 0)) {
        // sum of sign * |a_i|^2 (a Pauli string of Z and I only flips nothing):
        // four amplitudes loaded ahead of their sums, for memory parallelism.
        // A Z mask within the low 32 index bits (every register up to 32
        // qubits) takes its sign from one 32-bit population count.
        const bool z32 = (arg1 >> 32) == 0;
        for (; i + 3 * stride < N; i += 4 * stride) {
            ds::camp v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = lds(a, i + u * stride);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t iu = i + u * stride;
                const int par = z32 ? __popc(uint32_t(iu) & uint32_t(arg1)) : __popcll(iu & arg1);
                const float sg = (KIND == RED_PAULI && (par & 1)) ? -1.f : 1.f;
                ar.add(v[u].rh, v[u].rl, v[u].rh, v[u].rl, sg);
                ar.add(v[u].ih, v[u].il, v[u].ih, v[u].il, sg);
            }
        }
        for (; i < N; i += stride) {
            const ds::camp v = lds(a, i);
            const float sg = (KIND == RED_PAULI && (__popcll(i & arg1) & 1)) ? -1.f : 1.f;
            ar.add(v.rh, v.rl, v.rh, v.rl, sg);
            ar.add(v.ih, v.il, v.ih, v.il, sg);
        }
    }
    if (KIND == RED_PAULI && arg0 != 0) {
        // A string with X or Y factors pairs i with j = i ^ arg0: each pair is
        // read once, from the index with the lowest flipped bit clear.  With
        // c = conj(a_j) a_i and s_i the Z sign of i, the two terms add to
        // s_i (c + sigma conj(c)), sigma = (-1)^popcount(arg0 & arg1) (the
        // sign of j relative to i): 2 s_i Re(c), or 2i s_i Im(c).
        const int b0 = __ffsll(static_cast<long long>(arg0)) - 1;
        const uint64_t low = (uint64_t(1) << b0) - 1;
        const bool odd = __popcll(arg0 & arg1) & 1;
        const bool z32 = (arg1 >> 32) == 0;
        for (uint64_t p = i; p < N / 2; p += stride) {
            const uint64_t ii = ((p & ~low) << 1) | (p & low);
            const ds::camp v = lds(a, ii), w = lds(a, ii ^ arg0);
            const int par = z32 ? __popc(uint32_t(ii) & uint32_t(arg1)) : __popcll(ii & arg1);
            const float sg = (par & 1) ? -2.f : 2.f;
            if (!odd) {
                ar.add(w.rh, w.rl, v.rh, v.rl, sg);
                ar.add(w.ih, w.il, v.ih, v.il, sg);
            } else {
                ai.add(w.rh, w.rl, v.ih, v.il, sg);
                ai.add(w.ih, w.il, v.rh, v.rl, -sg);
            }
        }
    }
    for (; KIND != RED_NORM && KIND != RED_PAULI && i < N; i += stride) {
        if (KIND == RED_PROB_BIT && !(i & arg0)) continue;
        const ds::camp v = lds(a, i);
        if (KIND == RED_PROB_BIT) {
            ar.add(v.rh, v.rl, v.rh, v.rl, 1.f);
            ar.add(v.ih, v.il, v.ih, v.il, 1.f);
        } else {  // RED_INNER: conj(v) * w
            const ds::camp w = lds(b, i);
            ar.add(v.rh, v.rl, w.rh, w.rl, 1.f);
            ar.add(v.ih, v.il, w.ih, w.il, 1.f);
            ai.add(v.rh, v.rl, w.ih, w.il, 1.f);
            ai.add(v.ih, v.il, w.rh, w.rl, -1.f);
        }
    }
    double2 acc = block_sum(make_double2(ar.value(), ai.value()));
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Sums the partials in a fixed order; multiplies by i^phase_quarter.
__global__ void __launch_bounds__(RED_THREADS) k_final(const double2 *__restrict__ partial, int np,
                                                       int phase_quarter, double2 *__restrict__ out) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        acc.x += partial[k].x;
        acc.y += partial[k].y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        double2 r = acc;
        switch (phase_quarter & 3) {
        case 1: r = make_double2(-acc.y, acc.x); break;
        case 2: r = make_double2(-acc.x, -acc.y); break;
        case 3: r = make_double2(acc.y, -acc.x); break;
        default: break;
        }
        out[0] = r;
    }
}

template <typename R>
__global__ void k_prob_index(const cplx<R> *__restrict__ a, uint64_t x, double2 *out) {
    const double2 v = ld<R>(a, x);
    out[0] = make_double2(v.x * v.x + v.y * v.y, 0.0);
}

template <typename R>
__global__ void __launch_bounds__(256) k_scale(cplx<R> *__restrict__ a, uint64_t N,
                                               const double2 *__restrict__ norm) {
    const double s = 1.0 / sqrt(norm[0].x);
    const R sr = R(s);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        cplx<R> v = a[i];
        v.x *= sr;
        v.y *= sr;
        a[i] = v;
    }
}

template <typename R>
cudaError_t reduce_t(qs_state *s, int kind, uint64_t a0, uint64_t a1, const void *other) {
    const cplx<R> *a = static_cast<const cplx<R> *>(s->d);
    const cplx<R> *b = static_cast<const cplx<R> *>(other);
    const uint64_t N = uint64_t(1) << s->n;
    double2 *part = reinterpret_cast<double2 *>(s->partial);
    double2 *res = reinterpret_cast<double2 *>(s->result);
    if (kind == RED_PROB_INDEX) {
        k_prob_index<R><<<1, 1, 0, s->stream>>>(a, a0, res);
        return cudaGetLastError();
    }
    const int quarter = kind == RED_PAULI ? int((a1 >> 62) & 3) : 0;
    const uint64_t a1m = a1 & ~(uint64_t(3) << 62);
    switch (kind) {
    case RED_NORM:
        k_partial<R, RED_NORM><<<RED_BLOCKS, RED_THREADS, 0, s->stream>>>(a, b, N, a0, a1m, part);
        break;
    case RED_PROB_BIT:
        k_partial<R, RED_PROB_BIT><<<RED_BLOCKS, RED_THREADS, 0, s->stream>>>(a, b, N, a0, a1m, part);
        break;
    case RED_PAULI:
        k_partial<R, RED_PAULI><<<RED_BLOCKS, RED_THREADS, 0, s->stream>>>(a, b, N, a0, a1m, part);
        break;
    case RED_INNER:
        k_partial<R, RED_INNER><<<RED_BLOCKS, RED_THREADS, 0, s->stream>>>(a, b, N, a0, a1m, part);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    k_final<<<1, RED_THREADS, 0, s->stream>>>(part, RED_BLOCKS, quarter, res);
    return cudaGetLastError();
}

}  // namespace

// For RED_PAULI: a0 = flip mask, a1 = sign mask with the number of Y factors
// (mod 4) in its top two bits (n <= 40 leaves them free).
cudaError_t launch_reduce(qs_state *s, int kind, uint64_t a0, uint64_t a1, const void *other) {
    return s->dt == QS_C64 ? reduce_t<float>(s, kind, a0, a1, other)
                           : reduce_t<double>(s, kind, a0, a1, other);
}

cudaError_t launch_scale(qs_state *s, const double *dev_norm) {
    const uint64_t N = uint64_t(1) << s->n;
    uint64_t blocks = (N + 255) / 256;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    const double2 *nr = reinterpret_cast<const double2 *>(dev_norm);
    if (s->dt == QS_C64)
        k_scale<float><<<unsigned(blocks), 256, 0, s->stream>>>(static_cast<float2 *>(s->d), N, nr);
    else
        k_scale<double><<<unsigned(blocks), 256, 0, s->stream>>>(static_cast<double2 *>(s->d), N, nr);
    return cudaGetLastError();
}

}  // namespace qs
