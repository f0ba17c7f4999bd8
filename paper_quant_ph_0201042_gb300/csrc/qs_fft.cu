// Quantum Fourier transform as a black-box operator, Sec. 2.3.2:
//   beta_x = 2^{-L/2} sum_y w^{x y} alpha_y,  w = e^{2 pi i / 2^L},
// applied to the qubits q0 .. q0+L-1 (index bits [lo, hi), lo = n - q0 - L,
// hi = lo + L) by a fast Fourier transform instead of the O(L^2) gate
// circuit.  The paper uses an in-place radix-8 FFT on the CPU; here the
// transform is organised around HBM passes instead:
//
//  * Radix-2 decimation in frequency.  The stage of FFT bit b (b from hi-1
//    down to lo) combines the pair (x, y) that differs in bit b into
//    (x + y, (x - y) w_{2^{b-lo+1}}^t), t = the index bits [lo, b).  After all
//    stages position p of the range holds the output of index bitrev_L(p).
//  * The stages are grouped into passes of up to H bits (H = 8 for
//    complex64, 7 for complex128).  A pass reads each tile of 2^(5+H)
//    amplitudes (index bits 0..4, for contiguous warp accesses, plus H high
//    bits) once, runs its stages in registers (and with warp shuffles on
//    bits 0..4), and writes the tile once.  Across passes the recursion is
//    the four-step split: the sub-transform of a pass over bits [pb, pb+G)
//    is followed by the twiddle w_{2^s}^{t0 k1}, s = pb + G - lo, t0 = the
//    index bits [lo, pb), k1 = the digit the pass produced.
//  * Twiddles come from three tables built on the device per call with
//    sincospi in double precision: w_{2^13}^m (m < 2^12) for the stages of a
//    pass, and a two-level split e^{2 pi i f / 2^M} = T_hi[f >> h] T_lo[f & (2^h-1)]
//    for the pass twiddles (M = L).
//  * A last pass reverses the bit order of the range (tiled 32 x 32 through
//    shared memory when the range starts at bit 0, so that both the reads and
//    the writes are contiguous runs).
//  * Registers smaller than one tile run in a single CTA in shared memory.
//  * A complex128 state is transformed in double-single arithmetic by
//    default (qs_ds.cuh): the amplitudes are split into float pairs at the
//    load and joined at the store, the butterflies, twiddle products and
//    scale run on the single-precision pipe, and the twiddle tables hold
//    float pairs computed from double sincospi.  The kernels are written
//    once over an arithmetic type (Arith*: storage, register value and
//    twiddle types with their operations).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qs_ds.cuh"
#include "qs_internal.cuh"

namespace qs {
namespace {

constexpr int FFT_THREADS = 256;
constexpr int FFT_WB = 3;                 // warp bits (8 warps)
constexpr int TIN_LOG = 12;               // T_in[m] = w_{2^13}^m, m < 2^12
constexpr double M_PI_D = 3.14159265358979323846;

// Arithmetic types: S the amplitude in memory, V in registers, C a twiddle.
template <typename R>
struct ArithStd {                         // plain complex64 / complex128
    using S = cplx<R>;
    using V = cplx<R>;
    using C = cplx<R>;
    using Scal = R;
    static constexpr int RB = sizeof(R) == 4 ? 5 : 4;
    __device__ static V load(const S &a) { return a; }
    __device__ static S store(const V &v) { return v; }
    __device__ static V from_bits(const S &a) { return a; }   // (no intermediate format)
    __device__ static S to_bits(const V &v) { return v; }
    __device__ static V add(const V &a, const V &b) { return mk<R>(a.x + b.x, a.y + b.y); }
    __device__ static V sub(const V &a, const V &b) { return mk<R>(a.x - b.x, a.y - b.y); }
    __device__ static V mul(const C &w, const V &x) { return cmul<R>(w, x); }
    __device__ static C mulc(const C &a, const C &b) { return cmul<R>(a, b); }
    __device__ static C one() { return mk<R>(R(1), R(0)); }
    __device__ static V shfl(const V &v, int m) {
        return mk<R>(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
    }
    __device__ static V scale(const V &v, Scal s) { return mk<R>(v.x * s, v.y * s); }
    __host__ __device__ static C tw(double c, double sn) { C w; w.x = R(c); w.y = R(sn); return w; }
    static Scal scal(double v) { return R(v); }
};

struct ArithDS {                          // complex128 in double-single arithmetic
    using S = double2;
    using V = ds::camp;
    using C = ds::ccst;
    struct Scal { float h, l; };
    static constexpr int RB = 4;
    __device__ static V load(const S &a) { return ds::load(a.x, a.y); }
    __device__ static S store(const V &v) { return make_double2(ds::join(v.rh, v.rl), ds::join(v.ih, v.il)); }
    // between passes the amplitude's 16 bytes hold its float pairs as they are
    __device__ static V from_bits(const S &a) {
        V v;
        memcpy(&v, &a, sizeof(V));
        return v;
    }
    __device__ static S to_bits(const V &v) {
        S a;
        memcpy(&a, &v, sizeof(S));
        return a;
    }
    __device__ static V add(const V &a, const V &b) {
        V o;
        ds::add2(a.rh, a.rl, b.rh, b.rl, o.rh, o.rl);
        ds::add2(a.ih, a.il, b.ih, b.il, o.ih, o.il);
        return o;
    }
    __device__ static V sub(const V &a, const V &b) {
        V o;
        ds::add2(a.rh, a.rl, -b.rh, -b.rl, o.rh, o.rl);
        ds::add2(a.ih, a.il, -b.ih, -b.il, o.ih, o.il);
        return o;
    }
    __device__ static V mul(const C &w, const V &x) { return ds::cmul(w, x); }
    __device__ static C mulc(const C &a, const C &b) {
        const V p = ds::cmul(a, V{b.rh, b.rl, b.ih, b.il});
        return C{p.rh, p.rl, p.ih, p.il};
    }
    __device__ static C one() { return C{1.f, 0.f, 0.f, 0.f}; }
    __device__ static V shfl(const V &v, int m) {
        return V{__shfl_xor_sync(0xffffffffu, v.rh, m), __shfl_xor_sync(0xffffffffu, v.rl, m),
                 __shfl_xor_sync(0xffffffffu, v.ih, m), __shfl_xor_sync(0xffffffffu, v.il, m)};
    }
    __device__ static V scale(const V &v, Scal s) {
        V o;
        ds::mul1(v.rh, v.rl, s.h, s.l, o.rh, o.rl);
        ds::mul1(v.ih, v.il, s.h, s.l, o.ih, o.il);
        return o;
    }
    // the double cos / sin split into (high, low) float pairs
    __host__ __device__ static C tw(double c, double sn) {
        const float ch = float(c), sh = float(sn);
        return C{ch, float(c - double(ch)), sh, float(sn - double(sh))};
    }
    static Scal scal(double v) { Scal s; ds::split_const(v, s.h, s.l); return s; }
};

template <typename A> constexpr bool ARITH_PAIRS = false;
template <> constexpr bool ARITH_PAIRS<ArithDS> = true;

template <typename A>
struct FftPass {
    const typename A::C *tin;      // w_{2^13}^m (sign of the transform)
    const typename A::C *thi;      // e^{+-2 pi i a / 2^(M-h)}
    const typename A::C *tlo;      // e^{+-2 pi i b / 2^M}
    uint64_t tiles;          // 2^(n - K)
    int32_t M, h;            // digit-twiddle split
    int32_t lo;              // FFT range low bit
    int32_t r1, r2, r3;      // digit sizes: layout-A registers, layout-B registers, lanes
    int32_t s1, s2;          // sub-transform bits after digits 1 and 2 (top of digit - lo)
    int32_t lane_lo, lane_hi;  // lane digit: lane bits [lane_lo, lane_hi)
    typename A::Scal scale;  // 2^{-L/2} on the last pass, else 1
    bool scaled;             // this pass applies the scale
    bool in_pairs, out_pairs;  // double-single: the state between passes holds the float pairs (16 bytes
                               // per amplitude); the first pass splits the doubles, the last joins them
    uint8_t tile_pos[16];    // the K tile bit positions, ascending (0..4 first)
    uint8_t hpos[8];         // global bit of high tile bit i: FFT bits first, then spectators
    typename A::C rt[32];    // w_32^m (sign of the transform)
};

// stage twiddle w_{2^{g+1}}^t for t < 2^g (g <= 12)
template <typename A>
__device__ __forceinline__ typename A::C stage_tw(const typename A::C *__restrict__ tin, uint32_t t, int g) {
    return tin[t << (TIN_LOG - g)];
}

// e^{+-2 pi i f / 2^M} from the two-level tables
template <typename A>
__device__ __forceinline__ typename A::C big_tw(const FftPass<A> &P, uint64_t f) {
    return A::mulc(P.thi[f >> P.h], P.tlo[f & ((uint64_t(1) << P.h) - 1)]);
}

// Radix-2^D DFT (decimation in frequency) over register bits [0, D): the
// stage of bit r combines (j, j | 2^r) into (x + y, (x - y) w_{2^{r+1}}^{j mod 2^r});
// the twiddle index is known at compile time.  Register j then holds the
// digit output bitrev_D(j mod 2^D).
template <typename A, int NA, int D>
__device__ __forceinline__ void reg_dft(typename A::V (&v)[NA], const typename A::C (&rt)[32]) {
#pragma unroll
    for (int r = D - 1; r >= 0; --r) {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if ((j >> r) & 1) continue;
            const int j1 = j | (1 << r);
            const int m = (j & ((1 << r) - 1)) << (4 - r);      // w_{2^{r+1}}^t = w_32^{t 2^{4-r}}
            const typename A::V x = v[j], y = v[j1];
            v[j] = A::add(x, y);
            v[j1] = m == 0 ? A::sub(x, y) : A::mul(rt[m], A::sub(x, y));
        }
    }
}

// Twiddle of the four-step split after a digit of D register bits: register j
// (digit output k = bitrev_D(j mod 2^D)) is multiplied by w_{2^s}^{t0 k}; t0 is
// the same for all registers of the thread.  The D powers w_{2^s}^{t0 2^b}
// come from the tables, their products from a doubling tree.
template <typename A, int NA, int D>
__device__ __forceinline__ void digit_twiddle(typename A::V (&v)[NA], const FftPass<A> &P, uint64_t t0, int s) {
    if (D == 0 || t0 == 0) return;
    typename A::C w[1 << D];
    w[0] = A::one();
#pragma unroll
    for (int b = 0; b < D; ++b) {
        const typename A::C z = big_tw<A>(P, (t0 << b) << (P.M - s));
#pragma unroll
        for (int k = 0; k < (1 << b); ++k) w[k | (1 << b)] = b == 0 ? z : A::mulc(w[k], z);
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        int k = 0;
#pragma unroll
        for (int b = 0; b < D; ++b) k |= ((j >> b) & 1) << (D - 1 - b);
        if (k) v[j] = A::mul(w[k], v[j]);
    }
}

template <typename A, int NA>
__device__ __forceinline__ void digit_rt(typename A::V (&v)[NA], int D, const FftPass<A> &P, uint64_t t0, int s,
                                         const typename A::C (&rt)[32]) {
    switch (D) {
    case 1: reg_dft<A, NA, 1>(v, rt); digit_twiddle<A, NA, 1>(v, P, t0, s); break;
    case 2: reg_dft<A, NA, 2>(v, rt); digit_twiddle<A, NA, 2>(v, P, t0, s); break;
    case 3: reg_dft<A, NA, 3>(v, rt); digit_twiddle<A, NA, 3>(v, P, t0, s); break;
    case 4: reg_dft<A, NA, 4>(v, rt); digit_twiddle<A, NA, 4>(v, P, t0, s); break;
    case 5:
        if (NA >= 32) {
            reg_dft<A, NA, (NA >= 32 ? 5 : 4)>(v, rt);
            digit_twiddle<A, NA, (NA >= 32 ? 5 : 4)>(v, P, t0, s);
        }
        break;
    default: break;
    }
}

// One pass: a tile of 2^K amplitudes (index bits 0..4 in the lanes and H high
// bits) is loaded once; the pass's FFT bits form up to three digits, top
// down: the FFT high bits held in registers in layout A (high bits 3.. of the
// tile), those held in registers in layout B (high bits 0..2), and the lane
// bits of the range (only when it reaches below bit 5).  The FFT high bits
// are high tile bits 0 .. Gh-1; the spectator high bits lie above the range's
// unprocessed bits, so t0 of every digit depends on the thread alone.
template <typename A>
__global__ void __launch_bounds__(FFT_THREADS, 2) k_fft_pass(typename A::S *__restrict__ a,
                                                             const __grid_constant__ FftPass<A> P) {
    using S = typename A::S;
    using V = typename A::V;
    static_assert(sizeof(S) == sizeof(V), "the transpose buffer holds register values in place of amplitudes");
    constexpr int RB = A::RB, WB = FFT_WB, H = RB + WB, K = 5 + H, NA = 1 << RB;
    extern __shared__ __align__(16) unsigned char smraw[];
    S *sm = reinterpret_cast<S *>(smraw);      // the tiles as loaded
    V *sv = reinterpret_cast<V *>(smraw);      // the same buffer holding register values (transpose)
    const uint32_t tl = threadIdx.x, lane = tl & 31u, warp = tl >> 5;

    // layout A: register bit r <-> high bit WB + r, warp bit w <-> high bit w
    // layout B: register bit r <-> high bit r,      warp bit w <-> high bit RB + w
    uint64_t offA = lane, offB = lane;
#pragma unroll
    for (int w = 0; w < WB; ++w) {
        if ((warp >> w) & 1) {
            offA |= uint64_t(1) << P.hpos[w];
            offB |= uint64_t(1) << P.hpos[RB + w];
        }
    }
    const int lo = P.lo;
    const uint64_t m1 = (uint64_t(1) << P.s1) - 1, m2 = (uint64_t(1) << P.s2) - 1;
    const int d1b = P.s1 - P.r1, d2b = P.s2 - P.r2;     // digit bottoms relative to lo

    // Tiles are loaded with cp.async into the shared-memory transpose buffer,
    // in layout A at positions lane | warp << 5 | j << (5 + WB): each thread
    // copies the 2^RB amplitudes it will hold and later reads only those, so
    // its own wait suffices.  The copy of the next tile is issued as soon as
    // the current tile's transpose has been read, and overlaps the rest of
    // its work (digits 2 and 3, twiddles, the store).
    auto tile_base = [&](uint64_t t) {
        uint64_t b = t;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint64_t low = (uint64_t(1) << P.tile_pos[k]) - 1;
            b = ((b & ~low) << 1) | (b & low);
        }
        return b;
    };
    auto issue_tile = [&](uint64_t b) {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            uint64_t o = b | offA;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if ((j >> r) & 1) o |= uint64_t(1) << P.hpos[WB + r];
            const uint32_t sa = uint32_t(__cvta_generic_to_shared(&sm[lane | (warp << 5) | (uint32_t(j) << (5 + WB))]));
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(a + o), "n"(int(sizeof(S)))
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (blockIdx.x < P.tiles) issue_tile(tile_base(blockIdx.x));
    for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
        const uint64_t base = tile_base(tile);
        V v[NA];
        asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const S &x = sm[lane | (warp << 5) | (uint32_t(j) << (5 + WB))];
            v[j] = P.in_pairs ? A::from_bits(x) : A::load(x);
        }
        // digit 1: layout-A registers [0, r1)
        if (P.r1 > 0) {
            const uint64_t t0 = ((base | offA) >> lo) & m1 & ((uint64_t(1) << d1b) - 1);
            digit_rt<A, NA>(v, P.r1, P, t0, P.s1, P.rt);
        }
        // layout A -> B through shared memory (tile-local bit 5 + i <-> high bit i)
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NA; ++j) sv[lane | (warp << 5) | (uint32_t(j) << (5 + WB))] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NA; ++j) v[j] = sv[lane | (uint32_t(j) << 5) | (warp << (5 + RB))];
        __syncthreads();
        if (tile + gridDim.x < P.tiles) issue_tile(tile_base(tile + gridDim.x));
        // digit 2: layout-B registers [0, r2)
        if (P.r2 > 0) {
            const uint64_t t0 = ((base | offB) >> lo) & m2 & ((uint64_t(1) << d2b) - 1);
            digit_rt<A, NA>(v, P.r2, P, t0, P.s2, P.rt);
        }
        // digit 3: lane bits [lo, 5) with partners in other lanes; its t0 is 0
        if (P.r3 > 0) {
#pragma unroll
            for (int l = 4; l >= 0; --l) {
                if (l < P.lane_lo || l >= P.lane_hi) continue;
                const int g = l - P.lane_lo;
                const bool upper = (lane >> l) & 1;
                const typename A::C w = stage_tw<A>(P.tin, (lane >> P.lane_lo) & ((1u << g) - 1u), g);
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    const V o = A::shfl(v[j], 1 << l);
                    v[j] = upper ? A::mul(w, A::sub(o, v[j])) : A::add(v[j], o);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            uint64_t o = base | offB;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if ((j >> r) & 1) o |= uint64_t(1) << P.hpos[r];
            const V y = P.scaled ? A::scale(v[j], P.scale) : v[j];
            a[o] = P.out_pairs ? A::to_bits(y) : A::store(y);
        }
    }
}

// Whole register in one CTA (n below one tile): the stages in shared memory,
// then the bit reversal and the scale.
template <typename A>
__global__ void __launch_bounds__(1024) k_fft_small(typename A::S *__restrict__ a, int n, int lo, int L,
                                                    typename A::Scal scale, const typename A::C *__restrict__ tin) {
    using V = typename A::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const uint32_t N = 1u << n;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) sm[i] = A::load(a[i]);
    __syncthreads();
    for (int g = L - 1; g >= 0; --g) {
        const uint32_t bit = 1u << (lo + g);
        for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
            const uint32_t i0 = ((p >> (lo + g)) << (lo + g + 1)) | (p & (bit - 1));   // bit lo+g clear
            const uint32_t t = (i0 >> lo) & ((1u << g) - 1u);
            const V x = sm[i0], y = sm[i0 | bit];
            sm[i0] = A::add(x, y);
            sm[i0 | bit] = A::mul(stage_tw<A>(tin, t, g), A::sub(x, y));
        }
        __syncthreads();
    }
    const uint32_t field = ((1u << L) - 1u) << lo;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        const uint32_t x = (i & field) >> lo, r = __brev(x) >> (32 - L);
        const uint32_t j = (i & ~field) | (r << lo);
        a[j] = A::store(A::scale(sm[i], scale));
    }
}

// Bit reversal of the index bits [lo, lo + L), one pair per thread (the
// partner has the reversed field); contiguous when lo >= 5.
template <typename T>
__global__ void k_bitrev(T *__restrict__ a, uint64_t N, int lo, int L) {
    const uint64_t mask = ((uint64_t(1) << L) - 1) << lo;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t x = (i & mask) >> lo;
        const uint64_t r = __brevll(x) >> (64 - L);
        if (x < r) {
            const uint64_t j = (i & ~mask) | (r << lo);
            const T u = a[i], w = a[j];
            a[i] = w;
            a[j] = u;
        }
    }
}

// Bit reversal of the index bits [0, L), L >= 10, tiled: the field is
// (hi5 | m | lo5); block m and block rev(m) exchange their 32 x 32 tiles,
// each transposed and digit-reversed in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_bitrev_tiled(T *__restrict__ a, int n, int L, uint64_t blocks) {
    __shared__ T A[32][33], B[32][33];
    const int mb = L - 10;
    const uint32_t lane = threadIdx.x & 31u, row = threadIdx.x >> 5;
    for (uint64_t blk = blockIdx.x; blk < blocks; blk += gridDim.x) {
        const uint64_t m = blk & ((uint64_t(1) << mb) - 1), outer = blk >> mb;
        const uint64_t mr = mb ? (__brevll(m) >> (64 - mb)) : 0;
        if (m > mr) continue;
        const uint64_t hi = outer << L;
        const uint64_t bm = hi | (m << 5), br = hi | (mr << 5);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t rr = row + 8 * k;
            A[rr][lane] = a[bm | (uint64_t(rr) << (L - 5)) | lane];
            if (mr != m) B[rr][lane] = a[br | (uint64_t(rr) << (L - 5)) | lane];
        }
        __syncthreads();
        const uint32_t cl = __brev(lane) >> 27;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t rr = row + 8 * k, rv = __brev(rr) >> 27;
            // position (rr, lane) of the reversed block holds (rev(lane), rev(rr)) of its partner
            a[br | (uint64_t(rr) << (L - 5)) | lane] = A[cl][rv];
            if (mr != m) a[bm | (uint64_t(rr) << (L - 5)) | lane] = B[cl][rv];
        }
        __syncthreads();
    }
}

template <typename A>
__global__ void k_tw_tables(typename A::C *tin, typename A::C *thi, typename A::C *tlo, int M, int h, double sgn) {
    const uint32_t nin = 1u << TIN_LOG, nhi = 1u << (M - h), nlo = 1u << h;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nin + nhi + nlo; i += gridDim.x * blockDim.x) {
        double s, c;
        if (i < nin) {
            sincospi(double(i) / double(1u << TIN_LOG), &s, &c);       // 2 pi i m / 2^13
            tin[i] = A::tw(c, sgn * s);
        } else if (i < nin + nhi) {
            const uint32_t k = i - nin;
            sincospi(2.0 * double(k) / double(uint64_t(1) << (M - h)), &s, &c);
            thi[k] = A::tw(c, sgn * s);
        } else {
            const uint32_t k = i - nin - nhi;
            sincospi(2.0 * double(k) / double(uint64_t(1) << M), &s, &c);
            tlo[k] = A::tw(c, sgn * s);
        }
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <typename A>
cudaError_t qft_run(qs_state *s, int lo, int L, bool inverse, int64_t *launches) {
    using S = typename A::S;
    using C = typename A::C;
    constexpr int RB = A::RB, H = RB + FFT_WB, K = 5 + H;
    const int n = s->n, hi = lo + L;
    cudaStream_t st = s->stream;
    S *a = static_cast<S *>(s->d);
    const double sgn = inverse ? -1.0 : 1.0;
    const int M = L, h = (L + 1) / 2;
    const size_t nin = size_t(1) << TIN_LOG, nhi = size_t(1) << (M - h), nlo = size_t(1) << h;
    void *buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, sizeof(C) * (nin + nhi + nlo), st);
    if (e != cudaSuccess) return e;
    C *tin = static_cast<C *>(buf), *thi = tin + nin, *tlo = thi + nhi;
    k_tw_tables<A><<<64, 256, 0, st>>>(tin, thi, tlo, M, h, sgn);
    int64_t nl = 1;
    const typename A::Scal scale = A::scal(std::ldexp(1.0, -(L / 2)) * ((L & 1) ? 0.70710678118654752440 : 1.0));

    if (n < K) {
        const size_t bytes = sizeof(typename A::V) << n;
        k_fft_small<A><<<1, 1024, bytes, st>>>(a, n, lo, L, scale, tin);
        nl += 1;
    } else {
        cudaFuncSetAttribute(k_fft_pass<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(S) << K));
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fft_pass<A>, FFT_THREADS, sizeof(S) << K);
        const uint64_t tiles = uint64_t(1) << (n - K);
        const uint64_t grid = std::min<uint64_t>(tiles, uint64_t(sm_count()) * std::max(occ, 1));
        // passes, top down.  A pass takes up to H FFT bits; when the range
        // reaches below bit 5 the last pass is the low pass over [lo, pl) on
        // the tile [0, K), with pl chosen so that the bits above it split into
        // full passes.  A high pass with fewer than H FFT bits is the range's
        // lowest (pb = lo) and takes spectators from bits above it or below lo.
        std::vector<std::pair<int, int>> chunks;   // [pb, pb + G)
        int pl = lo;                                 // top of the low pass
        if (lo < 5) {
            pl = hi <= K ? hi : hi - H * ((hi - K + H - 1) / H);
        }
        for (int top = hi; top > pl;) {
            const int pb = std::max(pl, top - H);
            chunks.push_back({pb, top - pb});
            top = pb;
        }
        if (lo < 5) chunks.push_back({lo, pl - lo});
        C rt[32];
        for (int m = 0; m < 32; ++m)
            rt[m] = A::tw(std::cos(2.0 * M_PI_D * m / 32.0), sgn * std::sin(2.0 * M_PI_D * m / 32.0));
        for (const auto &c : chunks) {
            const int pb = c.first, G = c.second;
            FftPass<A> P;
            std::memset(&P, 0, sizeof P);
            P.tin = tin; P.thi = thi; P.tlo = tlo;
            P.tiles = tiles;
            P.M = M; P.h = h;
            P.lo = lo;
            P.scale = scale;
            P.scaled = pb == lo;
            // double-single passes hand the float pairs to the next pass
            P.in_pairs = ARITH_PAIRS<A> && &c != &chunks.front();
            P.out_pairs = ARITH_PAIRS<A> && &c != &chunks.back();
            for (int m = 0; m < 32; ++m) P.rt[m] = rt[m];
            std::vector<int> hb;            // FFT high bits ascending, then spectators
            int lane_bits = 0;
            if (pb < 5) {                   // low pass: tile = bits [0, K)
                for (int b = 5; b < pb + G; ++b) hb.push_back(b);
                for (int b = std::max(5, pb + G); int(hb.size()) < H; ++b) hb.push_back(b);
                lane_bits = std::min(5, pb + G) - pb;
            } else {
                for (int b = pb; b < pb + G; ++b) hb.push_back(b);
                for (int b = pb + G; int(hb.size()) < H && b < n; ++b) hb.push_back(b);
                for (int b = 5; int(hb.size()) < H && b < lo; ++b) hb.push_back(b);
            }
            if (int(hb.size()) != H) { e = cudaErrorInvalidValue; break; }
            const int Gh = pb < 5 ? std::max(0, pb + G - 5) : G;   // FFT bits among the high bits
            P.r1 = std::max(0, Gh - FFT_WB);
            P.r2 = std::min(FFT_WB, Gh);
            P.r3 = lane_bits;
            P.lane_lo = pb;
            P.lane_hi = pb + lane_bits;
            P.s1 = pb + G - lo;                  // digit 1 is the top of the pass
            P.s2 = P.s1 - P.r1;
            for (int i = 0; i < H; ++i) P.hpos[i] = uint8_t(hb[i]);
            std::vector<int> tp = {0, 1, 2, 3, 4};
            tp.insert(tp.end(), hb.begin(), hb.end());
            std::sort(tp.begin(), tp.end());
            for (int k = 0; k < K; ++k) P.tile_pos[k] = uint8_t(tp[k]);
            k_fft_pass<A><<<unsigned(grid), FFT_THREADS, sizeof(S) << K, st>>>(a, P);
            ++nl;
        }
        // bit reversal of [lo, hi)
        if (e == cudaSuccess && L > 1) {
            if (lo == 0 && L >= 10) {
                const uint64_t blocks = uint64_t(1) << (n - 10);
                const uint64_t g = std::min<uint64_t>(blocks, uint64_t(sm_count()) * 8);
                k_bitrev_tiled<S><<<unsigned(g), 256, 0, st>>>(a, n, L, blocks);
            } else {
                const uint64_t N = uint64_t(1) << n;
                const uint64_t g = std::min<uint64_t>((N + 255) / 256, uint64_t(sm_count()) * 16);
                k_bitrev<S><<<unsigned(g), 256, 0, st>>>(a, N, lo, L);
            }
            ++nl;
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFreeAsync(buf, st);
    if (launches) *launches = nl;
    return e;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_qft(qs_state *s, int q0, int L, int inverse) {
    if (!s) return fail(QS_EINVAL, "NULL state");
    if (q0 < 0 || L < 1 || q0 + L > s->n) return fail(QS_EINVAL, "qft: need 0 <= q0, 1 <= L, q0 + L <= n");
    if (L > 40) return fail(QS_ERANGE, "qft: L > 40");
    const int lo = s->n - q0 - L;
    cudaError_t e = s->dt == QS_C64 ? qft_run<ArithStd<float>>(s, lo, L, inverse != 0, nullptr)
                                    : qft_run<ArithDS>(s, lo, L, inverse != 0, nullptr);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "qft");
}
