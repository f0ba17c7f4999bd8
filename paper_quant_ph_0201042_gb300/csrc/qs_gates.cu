// Unfused evolution steps: one launch per gate (quant-ph/0201042, Sec. 2.2).
//
// The paper splits X|phi> into independent block products M_k = S_k phi_k and,
// when blocks are large, into row chunks; whatever the split, the two rows j
// and j + 2^(n-i-1) of a block must be computed by the same worker so that the
// in-place update never reads a value it has already overwritten (Sec. 2.2.1).
// Here one CUDA thread owns each amplitude pair: it loads x and y, then
// stores both results.  Consecutive threads own consecutive pair indices, so
// for every target bit >= 3 a warp reads and writes contiguous runs of
// amplitudes (coalesced); for low target bits the two loads of a warp
// interleave within the same cache lines.
//
// Controlled gates (Sec. 2.2.2) enumerate only the pairs whose control bits
// hold: the pair index is expanded into an amplitude index by inserting the
// fixed bits (target and controls), so the work is 2^(n-1-#controls) pairs
// and a gate with n-1 controls (Grover's phase oracle) touches one pair.
//
// A complex128 state is updated either with double-precision instructions
// or, by default, in double-single arithmetic (qs_ds.cuh): each loaded double
// is split into two floats, the pair update runs on the single-precision pipe
// by error-free transformations, and the results are joined back into
// doubles.  On this part the double pipe is too slow for a sweep to keep up
// with HBM (8 double FMAs per amplitude); the double-single sweep is bound by
// HBM instead.
#include <algorithm>

#include "qs_ds.cuh"
#include "qs_internal.cuh"

namespace qs {

namespace {

constexpr int UNROLL = 4;
constexpr int THREADS = 256;

struct Fixed {
    uint64_t value;       // bits OR-ed into every generated index
    int32_t nfixed;       // number of fixed bit positions
    uint8_t pos[64];      // fixed positions, ascending
};

// Inserts a zero at every fixed position (ascending), turning a free-bit
// counter into an amplitude index.
__device__ __forceinline__ uint64_t deposit(uint64_t p, const Fixed &f) {
    for (int k = 0; k < f.nfixed; ++k) {
        const uint64_t low = (uint64_t(1) << f.pos[k]) - 1;
        p = ((p & ~low) << 1) | (p & low);
    }
    return p | f.value;
}

template <typename R>
struct Mat {
    cplx<R> u00, u01, u10, u11;
};

template <typename R, int CLS>
__global__ void __launch_bounds__(THREADS) k_pair(cplx<R> *__restrict__ a, uint64_t count,
                                                  uint64_t tbit, const __grid_constant__ Fixed f,
                                                  const Mat<R> m) {
    const uint64_t stride = uint64_t(gridDim.x) * THREADS;
    for (uint64_t base = uint64_t(blockIdx.x) * THREADS + threadIdx.x; base < count;
         base += stride * UNROLL) {
        uint64_t i0[UNROLL];
        cplx<R> x[UNROLL], y[UNROLL];
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            const uint64_t p = base + k * stride;
            i0[k] = p < count ? deposit(p, f) : ~uint64_t(0);
            if (p < count) {
                x[k] = a[i0[k]];
                y[k] = a[i0[k] | tbit];
            }
        }
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            if (i0[k] == ~uint64_t(0)) continue;
            cplx<R> nx, ny;
            if (CLS == GC_GEN) {
                nx = cmad2<R>(m.u00, x[k], m.u01, y[k]);
                ny = cmad2<R>(m.u10, x[k], m.u11, y[k]);
            } else if (CLS == GC_REAL) {
                nx = rmad2<R>(m.u00.x, x[k], m.u01.x, y[k]);
                ny = rmad2<R>(m.u10.x, x[k], m.u11.x, y[k]);
            } else if (CLS == GC_DIAG) {
                nx = cmul<R>(m.u00, x[k]);
                ny = cmul<R>(m.u11, y[k]);
            } else if (CLS == GC_ANTI) {
                nx = cmul<R>(m.u01, y[k]);
                ny = cmul<R>(m.u10, x[k]);
            } else {  // GC_X
                nx = y[k];
                ny = x[k];
            }
            a[i0[k]] = nx;
            a[i0[k] | tbit] = ny;
        }
    }
}

// The same pair update on a complex128 state in double-single arithmetic.
struct MatDS {
    ds::ccst u00, u01, u10, u11;
};

__device__ __forceinline__ ds::camp ld_ds(const double2 &d) { return ds::load(d.x, d.y); }
__device__ __forceinline__ double2 st_ds(const ds::camp &c) {
    return make_double2(ds::join(c.rh, c.rl), ds::join(c.ih, c.il));
}

template <int CLS>
__global__ void __launch_bounds__(THREADS) k_pair_ds(double2 *__restrict__ a, uint64_t count, uint64_t tbit,
                                                     const __grid_constant__ Fixed f, const MatDS m) {
    const uint64_t stride = uint64_t(gridDim.x) * THREADS;
    for (uint64_t base = uint64_t(blockIdx.x) * THREADS + threadIdx.x; base < count;
         base += stride * UNROLL) {
        uint64_t i0[UNROLL];
        double2 x[UNROLL], y[UNROLL];
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            const uint64_t p = base + k * stride;
            i0[k] = p < count ? deposit(p, f) : ~uint64_t(0);
            if (p < count) {
                x[k] = a[i0[k]];
                y[k] = a[i0[k] | tbit];
            }
        }
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            if (i0[k] == ~uint64_t(0)) continue;
            const ds::camp X = ld_ds(x[k]), Y = ld_ds(y[k]);
            ds::camp nx, ny;
            if (CLS == GC_GEN) {
                nx = ds::cmad2(m.u00, X, m.u01, Y);
                ny = ds::cmad2(m.u10, X, m.u11, Y);
            } else if (CLS == GC_REAL) {
                nx = ds::rmad2(m.u00, X, m.u01, Y);
                ny = ds::rmad2(m.u10, X, m.u11, Y);
            } else if (CLS == GC_DIAG) {
                nx = ds::cmul(m.u00, X);
                ny = ds::cmul(m.u11, Y);
            } else {  // GC_ANTI
                nx = ds::cmul(m.u01, Y);
                ny = ds::cmul(m.u10, X);
            }
            a[i0[k]] = st_ds(nx);
            a[i0[k] | tbit] = st_ds(ny);
        }
    }
}

// One phase on the amplitudes of one pattern (GC_PHASE): only those are read
// and written.
template <typename R>
__global__ void __launch_bounds__(THREADS) k_phase(cplx<R> *__restrict__ a, uint64_t count,
                                                   const __grid_constant__ Fixed f,
                                                   cplx<R> d) {
    const uint64_t stride = uint64_t(gridDim.x) * THREADS;
    for (uint64_t base = uint64_t(blockIdx.x) * THREADS + threadIdx.x; base < count;
         base += stride * UNROLL) {
        uint64_t i[UNROLL];
        cplx<R> x[UNROLL];
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            const uint64_t p = base + k * stride;
            i[k] = p < count ? deposit(p, f) : ~uint64_t(0);
            if (p < count) x[k] = a[i[k]];
        }
#pragma unroll
        for (int k = 0; k < UNROLL; ++k)
            if (i[k] != ~uint64_t(0)) a[i[k]] = cmul<R>(d, x[k]);
    }
}

__global__ void __launch_bounds__(THREADS) k_phase_ds(double2 *__restrict__ a, uint64_t count,
                                                      const __grid_constant__ Fixed f, ds::ccst d) {
    const uint64_t stride = uint64_t(gridDim.x) * THREADS;
    for (uint64_t base = uint64_t(blockIdx.x) * THREADS + threadIdx.x; base < count;
         base += stride * UNROLL) {
        uint64_t i[UNROLL];
        double2 x[UNROLL];
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            const uint64_t p = base + k * stride;
            i[k] = p < count ? deposit(p, f) : ~uint64_t(0);
            if (p < count) x[k] = a[i[k]];
        }
#pragma unroll
        for (int k = 0; k < UNROLL; ++k)
            if (i[k] != ~uint64_t(0)) a[i[k]] = st_ds(ds::cmul(d, ld_ds(x[k])));
    }
}

// SWAP of index bits b1 and b2: indices with (b1, b2) = (1, 0) exchange with
// (0, 1).
template <typename R>
__global__ void __launch_bounds__(THREADS) k_swap(cplx<R> *__restrict__ a, uint64_t count,
                                                  const __grid_constant__ Fixed f,
                                                  uint64_t m1, uint64_t m2) {
    const uint64_t stride = uint64_t(gridDim.x) * THREADS;
    for (uint64_t base = uint64_t(blockIdx.x) * THREADS + threadIdx.x; base < count;
         base += stride * UNROLL) {
        uint64_t i[UNROLL];
        cplx<R> x[UNROLL], y[UNROLL];
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            const uint64_t p = base + k * stride;
            i[k] = p < count ? deposit(p, f) : ~uint64_t(0);
            if (p < count) {
                x[k] = a[i[k] | m1];
                y[k] = a[i[k] | m2];
            }
        }
#pragma unroll
        for (int k = 0; k < UNROLL; ++k) {
            if (i[k] == ~uint64_t(0)) continue;
            a[i[k] | m1] = y[k];
            a[i[k] | m2] = x[k];
        }
    }
}

template <typename R>
__global__ void k_set_one(cplx<R> *a, uint64_t x) { a[x] = mk<R>(R(1), R(0)); }

unsigned grid_for(uint64_t count) {
    uint64_t b = (count + uint64_t(THREADS) * UNROLL - 1) / (uint64_t(THREADS) * UNROLL);
    const uint64_t cap = 152ull * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return unsigned(b);
}

Fixed make_fixed(std::vector<int> pos, uint64_t value) {
    Fixed f;
    f.value = value;
    std::sort(pos.begin(), pos.end());
    f.nfixed = int(pos.size());
    for (size_t k = 0; k < pos.size(); ++k) f.pos[k] = uint8_t(pos[k]);
    return f;
}

std::vector<int> bits_of(uint64_t m) {
    std::vector<int> v;
    for (int b = 0; b < 64; ++b)
        if ((m >> b) & 1) v.push_back(b);
    return v;
}

template <typename R>
Mat<R> to_mat(const double *u) {
    Mat<R> m;
    m.u00 = mk<R>(R(u[0]), R(u[1]));
    m.u01 = mk<R>(R(u[2]), R(u[3]));
    m.u10 = mk<R>(R(u[4]), R(u[5]));
    m.u11 = mk<R>(R(u[6]), R(u[7]));
    return m;
}

ds::ccst split_c(double re, double im) {
    ds::ccst c;
    ds::split_const(re, c.rh, c.rl);
    ds::split_const(im, c.ih, c.il);
    return c;
}

MatDS to_mat_ds(const double *u) {
    return {split_c(u[0], u[1]), split_c(u[2], u[3]), split_c(u[4], u[5]), split_c(u[6], u[7])};
}

// DS: complex128 arithmetic in double-single (ignored for complex64).
template <typename R>
cudaError_t launch_op_t(qs_state *s, const HostOp &op, bool DS) {
    cplx<R> *a = static_cast<cplx<R> *>(s->d);
    const int n = s->n;
    const int nctrl = __builtin_popcountll(op.cmask);
    std::vector<int> pos = bits_of(op.cmask);
    if (op.cls == GC_ID) return cudaSuccess;
    if (op.cls == GC_SWAP) {
        pos.push_back(op.bit);
        pos.push_back(op.bit2);
        const uint64_t count = uint64_t(1) << (n - 2 - nctrl);
        Fixed f = make_fixed(pos, op.cval);
        k_swap<R><<<grid_for(count), THREADS, 0, s->stream>>>(a, count, f, uint64_t(1) << op.bit,
                                                             uint64_t(1) << op.bit2);
        return cudaGetLastError();
    }
    pos.push_back(op.bit);
    if (op.cls == GC_PHASE) {
        const uint64_t count = uint64_t(1) << (n - 1 - nctrl);
        const uint64_t v = op.cval | (op.phase_on ? (uint64_t(1) << op.bit) : 0);
        Fixed f = make_fixed(pos, v);
        const double *d = op.phase_on ? &op.u[6] : &op.u[0];
        if (DS && sizeof(R) == 8)
            k_phase_ds<<<grid_for(count), THREADS, 0, s->stream>>>(reinterpret_cast<double2 *>(a), count, f,
                                                                  split_c(d[0], d[1]));
        else
            k_phase<R><<<grid_for(count), THREADS, 0, s->stream>>>(a, count, f, mk<R>(R(d[0]), R(d[1])));
        return cudaGetLastError();
    }
    const uint64_t count = uint64_t(1) << (n - 1 - nctrl);
    Fixed f = make_fixed(pos, op.cval);
    const uint64_t tbit = uint64_t(1) << op.bit;
    const unsigned g = grid_for(count);
    if (DS && sizeof(R) == 8 && op.cls != GC_X) {
        double2 *ad = reinterpret_cast<double2 *>(a);
        const MatDS md = to_mat_ds(op.u);
        switch (op.cls) {
        case GC_GEN: k_pair_ds<GC_GEN><<<g, THREADS, 0, s->stream>>>(ad, count, tbit, f, md); break;
        case GC_REAL: k_pair_ds<GC_REAL><<<g, THREADS, 0, s->stream>>>(ad, count, tbit, f, md); break;
        case GC_DIAG: k_pair_ds<GC_DIAG><<<g, THREADS, 0, s->stream>>>(ad, count, tbit, f, md); break;
        case GC_ANTI: k_pair_ds<GC_ANTI><<<g, THREADS, 0, s->stream>>>(ad, count, tbit, f, md); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    Mat<R> m = to_mat<R>(op.u);
    switch (op.cls) {
    case GC_GEN: k_pair<R, GC_GEN><<<g, THREADS, 0, s->stream>>>(a, count, tbit, f, m); break;
    case GC_REAL: k_pair<R, GC_REAL><<<g, THREADS, 0, s->stream>>>(a, count, tbit, f, m); break;
    case GC_DIAG: k_pair<R, GC_DIAG><<<g, THREADS, 0, s->stream>>>(a, count, tbit, f, m); break;
    case GC_ANTI: k_pair<R, GC_ANTI><<<g, THREADS, 0, s->stream>>>(a, count, tbit, f, m); break;
    case GC_X: k_pair<R, GC_X><<<g, THREADS, 0, s->stream>>>(a, count, tbit, f, m); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_op(qs_state *s, const HostOp &op, bool ds) {
    return s->dt == QS_C64 ? launch_op_t<float>(s, op, false) : launch_op_t<double>(s, op, ds);
}

cudaError_t launch_init_basis(qs_state *s, uint64_t x) {
    const size_t amp = s->dt == QS_C64 ? 8 : 16;
    cudaError_t e = cudaMemsetAsync(s->d, 0, amp << s->n, s->stream);
    if (e != cudaSuccess) return e;
    if (s->dt == QS_C64)
        k_set_one<float><<<1, 1, 0, s->stream>>>(static_cast<float2 *>(s->d), x);
    else
        k_set_one<double><<<1, 1, 0, s->stream>>>(static_cast<double2 *>(s->d), x);
    return cudaGetLastError();
}

}  // namespace qs
