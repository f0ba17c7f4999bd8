// Gradients of an expectation value with respect to gate angles by one
// reverse sweep over the circuit (the differentiation pattern built on the
// paper's evolution steps, Sec. 2.2).
//
// With psi_j = U_j ... U_1 |0>, E = <psi_N|O|psi_N> and lambda_j =
// (U_N ... U_{j+1})^dagger O psi_N, the derivative with respect to an angle
// of U_j is 2 Re <lambda_j| dU_j U_j^dagger |psi_j>: the 2x2 generator
// G = dU U^dagger acts on the target pair (on the pairs whose controls hold,
// for a controlled gate).  Walking j = N..1, each step computes that sum from
// the pairs of psi_j and lambda_j and, in the same pass, uncomputes both
// vectors with U_j^dagger, so no intermediate state is ever stored.  Every
// pair is handled by one thread that reads the four amplitudes before writing
// any (the in-place rule of Sec. 2.2.1).
//
// Sums: each block adds its pairs and writes one partial per angle;
// fixed-order reductions then give one sum per angle and one per parameter.
// complex128 sums in double throughout.  complex64: single precision per
// thread and across the warp; the per-step sweep then adds across threads in
// double, the fused sweep keeps a compensated (Kahan) float accumulator per
// warp over the tiles it visits and adds the warps in double.
//
// Fused sweep (default): the reverse steps are grouped into tile passes by
// the fused planner's pass formation (steps whose targets lie in a tile of
// 2^K amplitudes, controls anywhere; commuting steps may move ahead, which
// leaves every gradient term unchanged because U_k then also commutes with
// dU_j U_j^dagger).  A CTA loads the tile of psi and of lambda into shared
// memory once, runs the pass's steps on it (gradient partial, then the
// uncompute) and writes both tiles back: one HBM round trip of the two vectors
// per pass instead of per step.  Within the tile the steps run in runs on up
// to three target bits (diagonal steps join any run): each thread keeps
// octets of both vectors in registers for a whole run.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <set>
#include <string>
#include <cstdio>
#include <vector>

#include "qs_internal.cuh"

namespace qs {

namespace {

constexpr int THREADS = 256;
enum AdjClass : int32_t { AC_GEN = 0, AC_REAL = 1, AC_DIAG = 2, AC_X = 3, AC_SWAP = 4 };

struct AdjStep {
    int32_t cls;
    int32_t nang;          // angles whose derivative is accumulated (0, 1, 2)
    int32_t slot0, slot1;  // partial-sum slots of the angles
    uint64_t tbit, tbit2;  // target (and second SWAP) index bits as masks
    uint64_t cval;
    double ui[8];          // U^dagger
    double g0[8], g1[8];   // generators dU U^dagger of the angles
    uint8_t pos[64];       // fixed bit positions, ascending
    int32_t nfixed;
    int32_t pad;
};

__device__ __forceinline__ uint64_t deposit(uint64_t p, const uint8_t *pos, int nf) {
    for (int k = 0; k < nf; ++k) {
        const uint64_t low = (uint64_t(1) << pos[k]) - 1;
        p = ((p & ~low) << 1) | (p & low);
    }
    return p;
}

template <typename R>
__device__ __forceinline__ R rdot(cplx<R> a, cplx<R> b) { return a.x * b.x + a.y * b.y; }   // Re(conj(a) b)

template <typename R>
__host__ __device__ __forceinline__ cplx<R> cmat(const double *u, int k) { return mk<R>(R(u[2 * k]), R(u[2 * k + 1])); }

__device__ __forceinline__ double blk_sum(double v) {
    __shared__ double sh[THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = l < THREADS / 32 ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

// One reverse step: gradient partial sums of the step's angles from
// (psi_j, lambda_j), then psi <- U^dagger psi, lambda <- U^dagger lambda.
template <typename R>
__global__ void __launch_bounds__(THREADS) k_adj(cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam, int n,
                                                 const AdjStep *__restrict__ dp, double *__restrict__ part) {
    const AdjStep &d = *dp;
    const int nf = d.nfixed;
    const uint64_t count = uint64_t(1) << (n - nf);
    const cplx<R> u00 = cmat<R>(d.ui, 0), u01 = cmat<R>(d.ui, 1), u10 = cmat<R>(d.ui, 2), u11 = cmat<R>(d.ui, 3);
    const cplx<R> a00 = cmat<R>(d.g0, 0), a01 = cmat<R>(d.g0, 1), a10 = cmat<R>(d.g0, 2), a11 = cmat<R>(d.g0, 3);
    const cplx<R> b00 = cmat<R>(d.g1, 0), b01 = cmat<R>(d.g1, 1), b10 = cmat<R>(d.g1, 2), b11 = cmat<R>(d.g1, 3);
    R acc0 = 0, acc1 = 0;
    for (uint64_t p = uint64_t(blockIdx.x) * THREADS + threadIdx.x; p < count; p += uint64_t(gridDim.x) * THREADS) {
        const uint64_t i0 = deposit(p, d.pos, nf) | d.cval;
        if (d.cls == AC_SWAP) {
            const uint64_t ia = i0 | d.tbit, ib = i0 | d.tbit2;
            cplx<R> t = psi[ia]; psi[ia] = psi[ib]; psi[ib] = t;
            t = lam[ia]; lam[ia] = lam[ib]; lam[ib] = t;
            continue;
        }
        const uint64_t i1 = i0 | d.tbit;
        const cplx<R> px = psi[i0], py = psi[i1], lx = lam[i0], ly = lam[i1];
        if (d.nang > 0) {
            acc0 += rdot<R>(lx, cmad2<R>(a00, px, a01, py)) + rdot<R>(ly, cmad2<R>(a10, px, a11, py));
            if (d.nang > 1)
                acc1 += rdot<R>(lx, cmad2<R>(b00, px, b01, py)) + rdot<R>(ly, cmad2<R>(b10, px, b11, py));
        }
        if (d.cls == AC_X) {
            psi[i0] = py; psi[i1] = px; lam[i0] = ly; lam[i1] = lx;
        } else if (d.cls == AC_DIAG) {
            psi[i0] = cmul<R>(u00, px); psi[i1] = cmul<R>(u11, py);
            lam[i0] = cmul<R>(u00, lx); lam[i1] = cmul<R>(u11, ly);
        } else if (d.cls == AC_REAL) {
            psi[i0] = rmad2<R>(u00.x, px, u01.x, py); psi[i1] = rmad2<R>(u10.x, px, u11.x, py);
            lam[i0] = rmad2<R>(u00.x, lx, u01.x, ly); lam[i1] = rmad2<R>(u10.x, lx, u11.x, ly);
        } else {
            psi[i0] = cmad2<R>(u00, px, u01, py); psi[i1] = cmad2<R>(u10, px, u11, py);
            lam[i0] = cmad2<R>(u00, lx, u01, ly); lam[i1] = cmad2<R>(u10, lx, u11, ly);
        }
    }
    if (d.nang > 0) {
        const double s0 = blk_sum(double(acc0));
        if (threadIdx.x == 0) part[uint64_t(d.slot0) * gridDim.x + blockIdx.x] = s0;
        if (d.nang > 1) {
            const double s1 = blk_sum(double(acc1));
            if (threadIdx.x == 0) part[uint64_t(d.slot1) * gridDim.x + blockIdx.x] = s1;
        }
    }
}

// lambda = P psi for a Pauli string: (P psi)[i ^ flip] = i^ny (-1)^popcount(i & sign) psi[i]
template <typename R>
__global__ void __launch_bounds__(THREADS) k_pauli_apply(const cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam,
                                                         uint64_t N, uint64_t flip, uint64_t sign, int ny) {
    for (uint64_t i = uint64_t(blockIdx.x) * THREADS + threadIdx.x; i < N; i += uint64_t(gridDim.x) * THREADS) {
        cplx<R> v = psi[i];
        if (__popcll(i & sign) & 1) v = mk<R>(-v.x, -v.y);
        switch (ny & 3) {
        case 1: v = mk<R>(-v.y, v.x); break;
        case 2: v = mk<R>(-v.x, -v.y); break;
        case 3: v = mk<R>(v.y, -v.x); break;
        default: break;
        }
        lam[i ^ flip] = v;
    }
}

// lambda = c phi
template <typename R>
__global__ void __launch_bounds__(THREADS) k_scale_copy(const cplx<R> *__restrict__ phi, cplx<R> *__restrict__ lam,
                                                        uint64_t N, double cr, double ci) {
    const cplx<R> c = mk<R>(R(cr), R(ci));
    for (uint64_t i = uint64_t(blockIdx.x) * THREADS + threadIdx.x; i < N; i += uint64_t(gridDim.x) * THREADS)
        lam[i] = cmul<R>(c, phi[i]);
}

// Sum of each slot's block partials, in order.
__global__ void __launch_bounds__(THREADS) k_slot_sums(const double *__restrict__ part, int nblk, double *__restrict__ out) {
    double v = 0.0;
    for (int k = threadIdx.x; k < nblk; k += THREADS) v += part[uint64_t(blockIdx.x) * nblk + k];
    v = blk_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// grad[p] = 2 * sum of the slots of parameter p (slots sorted by parameter).
__global__ void k_collect(const double *__restrict__ slot_sum, const int *__restrict__ first, int n_params,
                          double *__restrict__ grad) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_params; p += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int k = first[p]; k < first[p + 1]; ++k) v += slot_sum[k];
        grad[p] = 2.0 * v;
    }
}

// 2x2 complex products (row major, re/im pairs).
void mul2(const double *a, const double *b, double *c) {
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) {
            double re = 0, im = 0;
            for (int k = 0; k < 2; ++k) {
                const double ar = a[2 * (2 * r + k)], ai = a[2 * (2 * r + k) + 1];
                const double br = b[2 * (2 * k + q)], bi = b[2 * (2 * k + q) + 1];
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            c[2 * (2 * r + q)] = re;
            c[2 * (2 * r + q) + 1] = im;
        }
}

void dagger(const double *u, double *v) {
    const double w[8] = {u[0], -u[1], u[4], -u[5], u[2], -u[3], u[6], -u[7]};
    std::memcpy(v, w, sizeof(w));
}

// Generator dU/da U^dagger of angle `which` of a gate kind at angles (a, b).
bool generator(int kind, int which, double a, double b, double *g) {
    for (int k = 0; k < 8; ++k) g[k] = 0.0;
    switch (kind) {
    case QS_GATE_RY: g[2] = -0.5; g[4] = 0.5; return true;             // -(i/2) Y
    case QS_GATE_RZ: g[1] = -0.5; g[7] = 0.5; return true;             // -(i/2) Z
    case QS_GATE_UP1: g[7] = 1.0; return true;                         // diag(0, i)
    case QS_GATE_UP2: g[1] = 1.0; return true;                         // diag(i, 0)
    case QS_GATE_UR: g[2] = -1.0; g[4] = 1.0; return true;             // -i Y
    case QS_GATE_URP1:
        if (which == 0) { g[2] = -1.0; g[4] = 1.0; return true; }      // dU_R U_R^dagger = -i Y
        {
            // U_R(a) diag(0, i) U_R(a)^dagger
            const double c = std::cos(a), s = std::sin(a);
            const double R[8] = {c, 0, -s, 0, s, 0, c, 0};
            const double D[8] = {0, 0, 0, 0, 0, 0, 0, 1};
            double Rd[8], t[8];
            dagger(R, Rd);
            mul2(R, D, t);
            mul2(t, Rd, g);
            (void)b;
            return true;
        }
    default:
        return false;
    }
}

int kind_angles(int kind) {
    switch (kind) {
    case QS_GATE_UP1: case QS_GATE_UP2: case QS_GATE_UR: case QS_GATE_RY: case QS_GATE_RZ: return 1;
    case QS_GATE_URP1: return 2;
    default: return 0;
    }
}

// ---------------------------------------------------------------------------
// Fused reverse sweep
// ---------------------------------------------------------------------------
// threads per CTA and resident CTAs per SM of the fused sweep (256 and 2
// measured fastest on the n = 26 ansatz: 186 ms, against 206 ms for 512 and
// 2 with 64 registers, 236 ms for 512 and 1)
#ifndef QS_AF_THREADS
#define QS_AF_THREADS 256
#endif
#ifndef QS_AF_MINB
#define QS_AF_MINB 2
#endif
constexpr int AF_THREADS = QS_AF_THREADS;
constexpr int AF_WARPS = AF_THREADS / 32;
// at most ADJ_MAX_OPS steps per pass (the planner counts two budget units per op)
constexpr int ADJ_MAX_OPS = 64;

template <typename R>
struct alignas(16) AdjFOp {    // one reverse step of a pass, tile-local form
    int32_t mode;              // 0 pair op, 1 C-NOT-like exchange, 2 diagonal on a tile bit, 3 diagonal on an
                               // outer bit, 4 pair op with a real matrix and real generators
    int32_t tpos;              // tile-local target bit (modes 0-2) or global target bit (mode 3)
    uint32_t cm, cv;           // controls on tile bits (tile-local positions)
    uint64_t om, ov;           // controls on outer bits (global positions)
    int32_t nang;              // generators accumulated (0, 1, 2)
    int32_t acc;               // first accumulator of this pass used by the step
    int32_t slot0, slot1;      // global partial-sum slots of the generators
    int32_t gk;                // one generator of a special form: 1 real antisymmetric [[0, -g], [g, 0]]
                               // (mode 4), 2 imaginary diagonal diag(i a, i b) (modes 2, 3); else 0
    int32_t role;              // the run role (0, 1, 2) of the target bit; 3: a diagonal whose bit is no role
    int32_t pad_[2];
    cplx<R> ui[4];             // U^dagger
    cplx<R> g0[4], g1[4];      // generators dU U^dagger
};

// A pass's steps come in runs: within a run every non-diagonal step targets
// one of at most three tile bits (the run's roles), so each thread keeps the
// same octets of psi and lambda in registers for the whole run and the tile
// goes through shared memory once per run instead of once per step.
template <typename R>
struct AdjFPass {
    const AdjFOp<R> *ops;
    uint64_t tiles;
    int32_t nops, K, nacc, nrun;
    uint8_t tile_pos[16];
    uint8_t run_len[ADJ_MAX_OPS];
    uint8_t run_bit[ADJ_MAX_OPS];
    uint8_t run_bit2[ADJ_MAX_OPS];   // tile bits of roles 1 and 2 (other tile bits where the run has
    uint8_t run_bit3[ADJ_MAX_OPS];   // fewer target bits)
    uint8_t run_pre[ADJ_MAX_OPS];    // leading exchange steps of the run, applied at its load
};

// warp sum in the state's precision; lane 0 adds it to the warp's accumulator
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ R pair_grad(const cplx<R> *g, cplx<R> px, cplx<R> py, cplx<R> lx, cplx<R> ly) {
    return rdot<R>(lx, cmad2<R>(g[0], px, g[1], py)) + rdot<R>(ly, cmad2<R>(g[2], px, g[3], py));
}

// In-place forms of the updates: every output is written by the instruction
// that reads its input for the last time, so the new value takes the old
// one's register and the branches of the step dispatch join without moves.

// x <- c x for complex c
template <typename R>
__device__ __forceinline__ void cmul_ip(cplx<R> c, cplx<R> &x) {
    const R t1 = c.y * x.y, t2 = c.y * x.x;
    x.x = fma(c.x, x.x, -t1);
    x.y = fma(c.x, x.y, t2);
}

// (x, y) <- (a x + b y, c x + d y) with real a, b, c, d
template <typename R>
__device__ __forceinline__ void rmad_ip(R a, R b, R c, R d, cplx<R> &x, cplx<R> &y) {
    const R bx = b * y.x, by = b * y.y, dx = d * y.x, dy = d * y.y;
    y.x = fma(c, x.x, dx);
    y.y = fma(c, x.y, dy);
    x.x = fma(a, x.x, bx);
    x.y = fma(a, x.y, by);
}

// (x, y) <- (u0 x + u1 y, u2 x + u3 y) with complex entries
template <typename R>
__device__ __forceinline__ void cmad_ip(cplx<R> u0, cplx<R> u1, cplx<R> u2, cplx<R> u3, cplx<R> &x, cplx<R> &y) {
    R A = u1.x * y.y, B = -u1.y * y.y, C = u2.x * x.y, D = -u2.y * x.y;
    A = fma(u1.y, y.x, A);    // new x.im: u1.re y.im + u1.im y.re
    B = fma(u1.x, y.x, B);    // new x.re: u1.re y.re - u1.im y.im
    C = fma(u2.y, x.x, C);    // new y.im: u2.re x.im + u2.im x.re
    D = fma(u2.x, x.x, D);    // new y.re: u2.re x.re - u2.im x.im
    B = fma(-u0.y, x.y, B);
    A = fma(u0.y, x.x, A);
    D = fma(-u3.y, y.y, D);
    C = fma(u3.y, y.x, C);
    x.x = fma(u0.x, x.x, B);
    x.y = fma(u0.x, x.y, A);
    y.x = fma(u3.x, y.x, D);
    y.y = fma(u3.x, y.y, C);
}

// swap x and y where p holds, by masked XOR (no register moves)
template <typename R> struct bits_t;
template <> struct bits_t<float> { using type = uint32_t; };
template <> struct bits_t<double> { using type = unsigned long long; };
template <typename R>
__device__ __forceinline__ void cswap_ip(bool p, cplx<R> &x, cplx<R> &y) {
    using B = typename bits_t<R>::type;
    const B m = p ? ~B(0) : B(0);
    B xr, xi, yr, yi;
    memcpy(&xr, &x.x, sizeof(B)); memcpy(&xi, &x.y, sizeof(B));
    memcpy(&yr, &y.x, sizeof(B)); memcpy(&yi, &y.y, sizeof(B));
    const B dr = (xr ^ yr) & m, di = (xi ^ yi) & m;
    xr ^= dr; yr ^= dr; xi ^= di; yi ^= di;
    memcpy(&x.x, &xr, sizeof(B)); memcpy(&x.y, &xi, sizeof(B));
    memcpy(&y.x, &yr, sizeof(B)); memcpy(&y.y, &yi, sizeof(B));
}

// A run acts on up to three tile bits, its roles 0, 1 and 2 (masks RA[r];
// a run with fewer target bits takes other tile bits for the spare roles).
// Each thread holds NO octets of psi and of lambda in registers: element e
// of octet o is tile index q[o] | off[e], off[e] = the OR of RA[r] over the
// set bits r of e.  A step on role RR pairs element e (bit RR clear) with
// e | 2^RR, so which registers form a pair is known at compile time.  Octets
// o >= nov hold no tile elements (the same count for every thread).

template <typename R, int NA>
__device__ __forceinline__ void diag_elem(cplx<R> d, cplx<R> g, cplx<R> h, cplx<R> &x, cplx<R> &l, R &a0, R &a1) {
    if (NA > 0) a0 += rdot<R>(l, cmul<R>(g, x));
    if (NA > 1) a1 += rdot<R>(l, cmul<R>(h, x));
    cmul_ip<R>(d, x);
    cmul_ip<R>(d, l);
}

// one imaginary diagonal generator entry i g: Re<l|i g x> = g (l.y x.x - l.x x.y)
template <typename R>
__device__ __forceinline__ void diag_elem_im(cplx<R> d, R g, cplx<R> &x, cplx<R> &l, R &a0) {
    a0 = fma(g, fma(l.y, x.x, -l.x * x.y), a0);
    cmul_ip<R>(d, x);
    cmul_ip<R>(d, l);
}

// exchange (C-NOT-like step) on role RR where the controls hold
template <typename R, int NO, int RR, bool CHK>
__device__ __forceinline__ void o_exchange(uint32_t cm, uint32_t cv, int nov, const uint32_t (&q)[NO],
                                           const uint32_t (&off)[8], cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8]) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        if (o >= nov) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e >> RR) & 1) continue;
            const int e1 = e | (1 << RR);
            const bool p = !CHK || ((q[o] | off[e]) & cm) == cv;
            cswap_ip<R>(p, ps[o][e], ps[o][e1]);
            cswap_ip<R>(p, ls[o][e], ls[o][e1]);
        }
    }
}

// complex U^dagger on role RR, NA generators accumulated
template <typename R, int NO, int RR, int NA, bool CHK>
__device__ __forceinline__ void o_pair(const AdjFOp<R> &os, int nov, const uint32_t (&q)[NO], const uint32_t (&off)[8],
                                       cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8], R &a0, R &a1) {
    const uint32_t cm = os.cm, cv = os.cv;
    const cplx<R> u0 = os.ui[0], u1 = os.ui[1], u2 = os.ui[2], u3 = os.ui[3];
    cplx<R> g[4], h[4];
    if (NA > 0) for (int k = 0; k < 4; ++k) g[k] = os.g0[k];
    if (NA > 1) for (int k = 0; k < 4; ++k) h[k] = os.g1[k];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        if (o >= nov) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e >> RR) & 1) continue;
            const int e1 = e | (1 << RR);
            if (CHK && ((q[o] | off[e]) & cm) != cv) continue;
            if (NA > 0) a0 += pair_grad<R>(g, ps[o][e], ps[o][e1], ls[o][e], ls[o][e1]);
            if (NA > 1) a1 += pair_grad<R>(h, ps[o][e], ps[o][e1], ls[o][e], ls[o][e1]);
            cmad_ip<R>(u0, u1, u2, u3, ps[o][e], ps[o][e1]);
            cmad_ip<R>(u0, u1, u2, u3, ls[o][e], ls[o][e1]);
        }
    }
}

// real U^dagger and real generators: Re<l|g x> = g Re(conj(l) x) term by term
template <typename R, int NO, int RR, int NA, bool CHK>
__device__ __forceinline__ void o_pair_real(const AdjFOp<R> &os, int nov, const uint32_t (&q)[NO],
                                            const uint32_t (&off)[8], cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8],
                                            R &a0, R &a1) {
    const uint32_t cm = os.cm, cv = os.cv;
    const R u0 = os.ui[0].x, u1 = os.ui[1].x, u2 = os.ui[2].x, u3 = os.ui[3].x;
    R g[4] = {}, h[4] = {};
    if (NA > 0) for (int k = 0; k < 4; ++k) g[k] = os.g0[k].x;
    if (NA > 1) for (int k = 0; k < 4; ++k) h[k] = os.g1[k].x;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        if (o >= nov) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e >> RR) & 1) continue;
            const int e1 = e | (1 << RR);
            if (CHK && ((q[o] | off[e]) & cm) != cv) continue;
            if (NA > 0) {
                const R xx = rdot<R>(ls[o][e], ps[o][e]), xy = rdot<R>(ls[o][e], ps[o][e1]),
                        yx = rdot<R>(ls[o][e1], ps[o][e]), yy = rdot<R>(ls[o][e1], ps[o][e1]);
                a0 += g[0] * xx + g[1] * xy + g[2] * yx + g[3] * yy;
                if (NA > 1) a1 += h[0] * xx + h[1] * xy + h[2] * yx + h[3] * yy;
            }
            rmad_ip<R>(u0, u1, u2, u3, ps[o][e], ps[o][e1]);
            rmad_ip<R>(u0, u1, u2, u3, ls[o][e], ls[o][e1]);
        }
    }
}

// one real antisymmetric generator [[0, -g], [g, 0]]:
// Re<l|G|psi> = g (Re(conj(ly) x) - Re(conj(lx) y))
template <typename R, int NO, int RR, bool CHK>
__device__ __forceinline__ void o_pair_ras(const AdjFOp<R> &os, int nov, const uint32_t (&q)[NO],
                                           const uint32_t (&off)[8], cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8],
                                           R &a0) {
    const uint32_t cm = os.cm, cv = os.cv;
    const R u0 = os.ui[0].x, u1 = os.ui[1].x, u2 = os.ui[2].x, u3 = os.ui[3].x;
    R t = R(0);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        if (o >= nov) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e >> RR) & 1) continue;
            const int e1 = e | (1 << RR);
            if (CHK && ((q[o] | off[e]) & cm) != cv) continue;
            t = fma(ls[o][e1].x, ps[o][e].x, t);
            t = fma(ls[o][e1].y, ps[o][e].y, t);
            t = fma(-ls[o][e].x, ps[o][e1].x, t);
            t = fma(-ls[o][e].y, ps[o][e1].y, t);
            rmad_ip<R>(u0, u1, u2, u3, ps[o][e], ps[o][e1]);
            rmad_ip<R>(u0, u1, u2, u3, ls[o][e], ls[o][e1]);
        }
    }
    a0 += os.g0[2].x * t;
}

// Diagonal step.  DK 0: its bit is role RR (element e takes entry 0 or 1 by
// bit RR of e); DK 1: an outer bit (one entry for the tile, chosen by the
// caller into d0); DK 2: another tile bit (one entry per octet).
template <typename R, int NO, int RR, int NA, bool CHK, int DK, bool IM>
__device__ __forceinline__ void o_diag(const AdjFOp<R> &os, bool outer_one, int nov, const uint32_t (&q)[NO],
                                       const uint32_t (&off)[8], cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8], R &a0,
                                       R &a1) {
    const uint32_t cm = os.cm, cv = os.cv;
    const int tpos = os.tpos;
    cplx<R> d0 = os.ui[0], d1 = os.ui[3];
    cplx<R> g0{}, g3{}, h0{}, h3{};
    if (NA > 0) { g0 = os.g0[0]; g3 = os.g0[3]; }
    if (NA > 1) { h0 = os.g1[0]; h3 = os.g1[3]; }
    if (DK == 1 && outer_one) { d0 = d1; g0 = g3; h0 = h3; }
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        if (o >= nov) continue;
        bool oone = false;
        if (DK == 2) oone = (q[o] >> tpos) & 1;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            bool one = false;
            if (DK == 0) one = (e >> RR) & 1;
            if (DK == 2) one = oone;
            const cplx<R> d = one ? d1 : d0;
            const cplx<R> g = one ? g3 : g0, h = one ? h3 : h0;
            if (CHK && ((q[o] | off[e]) & cm) != cv) continue;
            if (IM) diag_elem_im<R>(d, g.y, ps[o][e], ls[o][e], a0);
            else diag_elem<R, NA>(d, g, h, ps[o][e], ls[o][e], a0, a1);
        }
    }
}

// The step kinds of role RR (pair steps and diagonals on role RR's bit).
template <typename R, int NO, int RR, bool CHK>
__device__ __forceinline__ void step_role(const AdjFOp<R> &os, int nov, const uint32_t (&q)[NO],
                                          const uint32_t (&off)[8], cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8],
                                          R &a0, R &a1) {
    const int mode = os.mode, nang = os.nang;
    if (mode == 1) {
        o_exchange<R, NO, RR, CHK>(os.cm, os.cv, nov, q, off, ps, ls);
    } else if (mode == 4) {
        if (os.gk == 1) o_pair_ras<R, NO, RR, CHK>(os, nov, q, off, ps, ls, a0);
        else if (nang == 0) o_pair_real<R, NO, RR, 0, CHK>(os, nov, q, off, ps, ls, a0, a1);
        else if (nang == 1) o_pair_real<R, NO, RR, 1, CHK>(os, nov, q, off, ps, ls, a0, a1);
        else o_pair_real<R, NO, RR, 2, CHK>(os, nov, q, off, ps, ls, a0, a1);
    } else if (mode == 0) {
        if (nang == 0) o_pair<R, NO, RR, 0, CHK>(os, nov, q, off, ps, ls, a0, a1);
        else if (nang == 1) o_pair<R, NO, RR, 1, CHK>(os, nov, q, off, ps, ls, a0, a1);
        else o_pair<R, NO, RR, 2, CHK>(os, nov, q, off, ps, ls, a0, a1);
    } else {   // diagonal on this role's bit
        if (os.gk == 2) o_diag<R, NO, RR, 1, CHK, 0, true>(os, false, nov, q, off, ps, ls, a0, a1);
        else if (nang == 0) o_diag<R, NO, RR, 0, CHK, 0, false>(os, false, nov, q, off, ps, ls, a0, a1);
        else if (nang == 1) o_diag<R, NO, RR, 1, CHK, 0, false>(os, false, nov, q, off, ps, ls, a0, a1);
        else o_diag<R, NO, RR, 2, CHK, 0, false>(os, false, nov, q, off, ps, ls, a0, a1);
    }
}

// A diagonal step whose bit is not one of the run's roles: an outer bit
// (mode 3) or another tile bit (mode 2).
template <typename R, int NO, bool CHK, int DK>
__device__ __forceinline__ void step_diag_other(const AdjFOp<R> &os, bool outer_one, int nov, const uint32_t (&q)[NO],
                                                const uint32_t (&off)[8], cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8],
                                                R &a0, R &a1) {
    const int nang = os.nang;
    if (os.gk == 2) o_diag<R, NO, 0, 1, CHK, DK, true>(os, outer_one, nov, q, off, ps, ls, a0, a1);
    else if (nang == 0) o_diag<R, NO, 0, 0, CHK, DK, false>(os, outer_one, nov, q, off, ps, ls, a0, a1);
    else if (nang == 1) o_diag<R, NO, 0, 1, CHK, DK, false>(os, outer_one, nov, q, off, ps, ls, a0, a1);
    else o_diag<R, NO, 0, 2, CHK, DK, false>(os, outer_one, nov, q, off, ps, ls, a0, a1);
}

template <typename R, int NO, bool CHK>
__device__ __forceinline__ void step_octets(const AdjFOp<R> &os, uint64_t base, int nov, const uint32_t (&q)[NO],
                                            const uint32_t (&off)[8], cplx<R> (&ps)[NO][8], cplx<R> (&ls)[NO][8],
                                            R &a0, R &a1) {
    const int role = os.role;
    if (role == 0) step_role<R, NO, 0, CHK>(os, nov, q, off, ps, ls, a0, a1);
    else if (role == 1) step_role<R, NO, 1, CHK>(os, nov, q, off, ps, ls, a0, a1);
    else if (role == 2) step_role<R, NO, 2, CHK>(os, nov, q, off, ps, ls, a0, a1);
    else if (os.mode == 3) step_diag_other<R, NO, CHK, 1>(os, (base >> os.tpos) & 1, nov, q, off, ps, ls, a0, a1);
    else step_diag_other<R, NO, CHK, 2>(os, false, nov, q, off, ps, ls, a0, a1);
}

// The run's leading exchange steps as a permutation of each octet's
// places: field e (3 bits) of perm names the element whose value place e
// takes at the load.  An exchange on role RR swaps fields e and e | 2^RR
// where its controls hold on the place's index.
template <int NO, int RR>
__device__ __forceinline__ void o_pre(uint32_t cm, uint32_t cv, int nov, const uint32_t (&q)[NO],
                                      const uint32_t (&off)[8], uint32_t (&perm)[NO]) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        if (o >= nov) continue;
        uint32_t x = perm[o];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if ((e >> RR) & 1) continue;
            const int e1 = e | (1 << RR);
            const bool c = ((q[o] | off[e]) & cm) == cv;
            const uint32_t d = ((x >> (3 * e)) ^ (x >> (3 * e1))) & (c ? 7u : 0u);
            x ^= (d << (3 * e)) | (d << (3 * e1));
        }
        perm[o] = x;
    }
}

// Per-warp gradient accumulators over the tiles a CTA visits.  complex64:
// a compensated (Kahan) float sum, so the FP32 pipe does the work and the
// error does not grow with the number of tiles; complex128: double.
template <typename R>
struct Acc { double s; };
template <>
struct Acc<float> { float s, c; };

template <typename R>
__device__ __forceinline__ void acc_add(Acc<R> &a, R v) { a.s += double(v); }
template <>
__device__ __forceinline__ void acc_add<float>(Acc<float> &a, float v) {
    const float y = v - a.c;
    const float t = a.s + y;
    a.c = (t - a.s) - y;
    a.s = t;
}
template <typename R>
__device__ __forceinline__ double acc_value(const Acc<R> &a) { return a.s; }
template <>
__device__ __forceinline__ double acc_value<float>(const Acc<float> &a) { return double(a.s) - double(a.c); }

// Moves a tile of psi and lambda between HBM and shared memory (LOAD: in).
// Element e of the tile is index base | hoff[e >> 5] | (e & 31); complex64
// moves two neighbouring elements per 16-byte access.
template <typename R, bool LOAD>
__device__ __forceinline__ void tile_io(cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam, cplx<R> *sp, cplx<R> *sl,
                                        uint64_t base, const uint64_t *hoff, uint32_t T, uint32_t tid) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll 8
        for (uint32_t q = tid; q < T / 2; q += AF_THREADS) {
            const uint32_t e = 2 * q;
            const uint64_t gi = base | hoff[e >> 5] | (e & 31u);
            float4 *gp = reinterpret_cast<float4 *>(psi + gi), *gl = reinterpret_cast<float4 *>(lam + gi);
            float4 *tp = reinterpret_cast<float4 *>(sp + e), *tl = reinterpret_cast<float4 *>(sl + e);
            if (LOAD) { *tp = *gp; *tl = *gl; }
            else { *gp = *tp; *gl = *tl; }
        }
    } else {
#pragma unroll 8
        for (uint32_t e = tid; e < T; e += AF_THREADS) {
            const uint64_t gi = base | hoff[e >> 5] | (e & 31u);
            if (LOAD) { sp[e] = psi[gi]; sl[e] = lam[gi]; }
            else { psi[gi] = sp[e]; lam[gi] = sl[e]; }
        }
    }
}

// tiles of 2^12 (complex64) or 2^11 (complex128) amplitudes; pairs per thread
template <typename R>
constexpr int adj_full_k() { return sizeof(R) == 4 ? 12 : 11; }
template <typename R>
constexpr int adj_np() { return (1 << (adj_full_k<R>() - 1)) / AF_THREADS; }
// the fused sweep needs a tile of at least one octet per thread
template <typename R>
constexpr bool adj_fused_ok(int n) { return (1 << (n < adj_full_k<R>() ? n : adj_full_k<R>())) >= 8 * AF_THREADS; }

template <typename R>
__global__ void __launch_bounds__(AF_THREADS, QS_AF_MINB) k_adj_pass(cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam,
                                                            const __grid_constant__ AdjFPass<R> P,
                                                            double *__restrict__ part) {
    constexpr int NP = adj_np<R>();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int K = P.K;
    const uint32_t T = 1u << K;
    // octets per thread that hold tile elements: the tile has T / 8 octets, a
    // whole number of CTA-wide rows of them (the host guarantees at least
    // one), so the count is the same for every thread and the tests on it do
    // not diverge (a compile-time count, all octets full, let the compiler
    // schedule the run bodies into 4 KB of spills)
    constexpr int NO = NP / 4;
    const int nov = int(T / 8 / AF_THREADS);
    cplx<R> *sp = reinterpret_cast<cplx<R> *>(smraw);
    cplx<R> *sl = sp + T;
    Acc<R> *sacc = reinterpret_cast<Acc<R> *>(sl + T);                        // nacc x AF_WARPS
    AdjFOp<R> *sops = reinterpret_cast<AdjFOp<R> *>(sacc + P.nacc * AF_WARPS);   // the pass's steps
    // global offset of each value of the tile index's high K - 5 bits (the low
    // five tile bits are index bits 0..4)
    uint64_t *hoff = reinterpret_cast<uint64_t *>(sops + P.nops);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    for (int k = tid; k < P.nacc * AF_WARPS; k += AF_THREADS) sacc[k] = Acc<R>{};
    for (uint32_t h = tid; h < (T >> 5); h += AF_THREADS) {
        uint64_t o = 0;
        for (int k = 5; k < K; ++k)
            if ((h >> (k - 5)) & 1) o |= uint64_t(1) << P.tile_pos[k];
        hoff[h] = o;
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.ops);
        uint4 *dst = reinterpret_cast<uint4 *>(sops);
        const int words = P.nops * int(sizeof(AdjFOp<R>) / 16);
        for (int k = tid; k < words; k += AF_THREADS) dst[k] = src[k];
    }
    for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
        uint64_t base = tile;
        for (int k = 0; k < K; ++k) {
            const uint64_t low = (uint64_t(1) << P.tile_pos[k]) - 1;
            base = ((base & ~low) << 1) | (base & low);
        }
        __syncthreads();
        tile_io<R, true>(psi, lam, sp, sl, base, hoff, T, tid);
        __syncthreads();
        int k0 = 0;
        for (int r = 0; r < P.nrun; ++r) {
            const int len = P.run_len[r];
            const uint32_t RA0 = 1u << P.run_bit[r], RA1 = 1u << P.run_bit2[r], RA2 = 1u << P.run_bit3[r];
            // the three role bits ascending, for the octet index
            int s0 = P.run_bit[r], s1 = P.run_bit2[r], s2 = P.run_bit3[r];
            if (s0 > s1) { const int t = s0; s0 = s1; s1 = t; }
            if (s1 > s2) { const int t = s1; s1 = s2; s2 = t; }
            if (s0 > s1) { const int t = s0; s0 = s1; s1 = t; }
            uint32_t off[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) off[e] = ((e & 1) ? RA0 : 0u) | ((e & 2) ? RA1 : 0u) | ((e & 4) ? RA2 : 0u);
            uint32_t q[NO];
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                uint32_t x = tid + uint32_t(o) * AF_THREADS;
                x = ((x >> s0) << (s0 + 1)) | (x & ((1u << s0) - 1u));
                x = ((x >> s1) << (s1 + 1)) | (x & ((1u << s1) - 1u));
                x = ((x >> s2) << (s2 + 1)) | (x & ((1u << s2) - 1u));
                q[o] = x;
            }
            cplx<R> ps[NO][8], ls[NO][8];
            const int pre = P.run_pre[r];
            // the run's leading exchange steps become the choice of which
            // element loads into which place (none: place e <- element e)
            uint32_t perm[NO];
#pragma unroll
            for (int o = 0; o < NO; ++o) perm[o] = 0xFAC688u;
            for (int k = k0; k < k0 + pre; ++k) {
                const AdjFOp<R> &os = sops[k];
                if ((base & os.om) != os.ov) continue;
                if (os.role == 0) o_pre<NO, 0>(os.cm, os.cv, nov, q, off, perm);
                else if (os.role == 1) o_pre<NO, 1>(os.cm, os.cv, nov, q, off, perm);
                else o_pre<NO, 2>(os.cm, os.cv, nov, q, off, perm);
            }
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                if (o >= nov) continue;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t src = (perm[o] >> (3 * e)) & 7u;
                    const uint32_t idx = q[o] | ((src & 1u) ? RA0 : 0u) | ((src & 2u) ? RA1 : 0u) |
                                         ((src & 4u) ? RA2 : 0u);
                    ps[o][e] = sp[idx];
                    ls[o][e] = sl[idx];
                }
            }
            for (int k = k0 + pre; k < k0 + len; ++k) {
                const AdjFOp<R> &os = sops[k];
                if ((base & os.om) != os.ov) continue;            // the same for the whole tile
                const int nang = os.nang;
                R a0 = R(0), a1 = R(0);
                if (os.cm == 0) step_octets<R, NO, false>(os, base, nov, q, off, ps, ls, a0, a1);
                else step_octets<R, NO, true>(os, base, nov, q, off, ps, ls, a0, a1);
                if (nang > 0) {
                    const R s0v = warp_sum<R>(a0);
                    if (lane == 0) acc_add<R>(sacc[os.acc * AF_WARPS + warp], s0v);
                    if (nang > 1) {
                        const R s1v = warp_sum<R>(a1);
                        if (lane == 0) acc_add<R>(sacc[(os.acc + 1) * AF_WARPS + warp], s1v);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                if (o >= nov) continue;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    sp[q[o] | off[e]] = ps[o][e];
                    sl[q[o] | off[e]] = ls[o][e];
                }
            }
            k0 += len;
            __syncthreads();
        }
        tile_io<R, false>(psi, lam, sp, sl, base, hoff, T, tid);
    }
    __syncthreads();
    // one partial per generator slot and CTA
    for (int k = 0; k < P.nops; ++k) {
        const AdjFOp<R> &o = sops[k];
        for (int a = 0; a < o.nang; ++a) {
            if (tid < 32) {
                double v = lane < AF_WARPS ? acc_value<R>(sacc[(o.acc + a) * AF_WARPS + lane]) : 0.0;
#pragma unroll
                for (int q = 16; q > 0; q >>= 1) v += __shfl_xor_sync(0xffffffffu, v, q);
                if (lane == 0) part[uint64_t(a == 0 ? o.slot0 : o.slot1) * gridDim.x + blockIdx.x] = v;
            }
        }
    }
}

struct Buf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~Buf() { if (p) cudaFreeAsync(p, s); }
};

template <typename R>
size_t adj_smem(int K, int nacc, int nops) {
    return (sizeof(cplx<R>) << (K + 1)) + sizeof(Acc<R>) * AF_WARPS * size_t(nacc) + sizeof(AdjFOp<R>) * size_t(nops) +
           (sizeof(uint64_t) << (K - 5));
}

// true when the step's generators are real, as U^dagger is (mode 4)
bool real_gens(const AdjStep &d) {
    for (int e = 0; e < 4; ++e)
        if (d.g0[2 * e + 1] != 0.0 || d.g1[2 * e + 1] != 0.0) return false;
    return true;
}

// Orders a pass's steps (idx, in sweep order) into runs: the next step is the
// first ready one (every earlier step it does not commute with already
// placed) that is diagonal or targets one of the current run's bits (a run
// takes up to three target bits; a new bit joins with the first step on it);
// when none is, the run ends and the first ready step opens the next.  Two
// steps commute when every index bit they share is a control or the target
// of a diagonal step for both (the test the pass planner uses), and moving a
// step past steps it commutes with leaves every gradient term unchanged.
constexpr int RUN_BITS = 3;
struct Run {
    int len;    // steps
    int bit;    // global target bits, -1 for none (bit = -1: diagonal steps only)
    int bit2;
    int bit3;
};

void schedule_runs(const std::vector<int> &idx, const std::vector<AdjStep> &steps, const std::vector<HostOp> &hops,
                   std::vector<int> &order, std::vector<Run> &runs) {
    const size_t m = idx.size();
    std::vector<uint64_t> sup(m), dg(m);
    std::vector<char> diag(m);
    for (size_t k = 0; k < m; ++k) {
        const HostOp &o = hops[size_t(idx[k])];
        diag[k] = steps[size_t(idx[k])].cls == AC_DIAG;
        sup[k] = o.cmask | (uint64_t(1) << o.bit);
        dg[k] = o.cmask | (diag[k] ? uint64_t(1) << o.bit : 0);
    }
    std::vector<std::vector<int>> succ(m);
    std::vector<int> npred(m, 0);
    for (size_t b = 0; b < m; ++b)
        for (size_t a = 0; a < b; ++a)
            if ((sup[a] & sup[b]) & ~(dg[a] & dg[b])) { succ[a].push_back(int(b)); ++npred[b]; }
    std::set<int> ready;
    for (size_t k = 0; k < m; ++k)
        if (npred[k] == 0) ready.insert(int(k));
    order.clear();
    runs.clear();
    int cur[RUN_BITS] = {-1, -1, -1}, len = 0;
    bool lead = true;   // the run holds exchange steps only so far
    auto has = [&](int b) { return b == cur[0] || b == cur[1] || b == cur[2]; };
    auto free_slot = [&]() { return cur[RUN_BITS - 1] < 0; };
    auto fits = [&](int k) { return has(hops[size_t(idx[size_t(k)])].bit) || free_slot(); };
    while (order.size() < m) {
        int pick = -1;
        // while the run is only exchanges: another exchange on one of its
        // bits (the leading exchanges are folded into the run's load)
        if (lead)
            for (int k : ready)
                if (steps[size_t(idx[size_t(k)])].cls == AC_X && fits(k)) { pick = k; break; }
        // a step on a bit the run already has, then one that opens a bit
        if (pick < 0)
            for (int k : ready) {
                const int b = hops[size_t(idx[size_t(k)])].bit;
                if (diag[size_t(k)] || has(b)) { pick = k; break; }
            }
        if (pick < 0 && free_slot())
            for (int k : ready) { pick = k; break; }
        if (pick < 0) {
            runs.push_back({len, cur[0], cur[1], cur[2]});
            cur[0] = cur[1] = cur[2] = -1;
            len = 0;
            lead = true;
            continue;
        }
        if (steps[size_t(idx[size_t(pick)])].cls != AC_X) lead = false;
        if (!diag[size_t(pick)]) {
            const int b = hops[size_t(idx[size_t(pick)])].bit;
            if (!has(b))
                for (int r = 0; r < RUN_BITS; ++r)
                    if (cur[r] < 0) { cur[r] = b; break; }
        }
        order.push_back(idx[size_t(pick)]);
        ++len;
        ready.erase(pick);
        for (int sidx : succ[size_t(pick)])
            if (--npred[size_t(sidx)] == 0) ready.insert(sidx);
    }
    if (len > 0) runs.push_back({len, cur[0], cur[1], cur[2]});
}

// One tile pass of the fused reverse sweep, planned on the host: the tile's
// index bits (ascending), the pass's steps in sweep order, its runs (length,
// global target bit or -1 for diagonal steps only) and each run's leading
// exchange steps.
struct SweepPass {
    std::vector<int> tile;
    std::vector<int> order;
    std::vector<Run> runs;
    std::vector<int> pre;
};

// Plans the fused reverse sweep over steps[] (in forward order; run last to
// first) for tiles of 2^K amplitudes.  False if a pass's step targets a bit
// outside its tile (the pass planner never does this).
bool plan_sweep(int n, int K, const std::vector<AdjStep> &steps, const std::vector<HostOp> &hops,
                std::vector<SweepPass> &out) {
    // reverse steps as planner ops (SWAP already split into C-NOTs)
    std::vector<HostOp> rev;
    for (size_t j = steps.size(); j-- > 0;) {
        HostOp o = hops[j];
        o.step = int32_t(j);
        if (steps[j].cls == AC_DIAG) o.cls = GC_DIAG;
        else if (steps[j].cls == AC_X) o.cls = GC_X;
        else o.cls = GC_GEN;
        rev.push_back(o);
    }
    out.clear();
    for (const PassGroup &gp : group_passes(n, K - 5, 2 * ADJ_MAX_OPS, rev)) {
        SweepPass sp;
        sp.tile = {0, 1, 2, 3, 4};
        sp.tile.insert(sp.tile.end(), gp.high.begin(), gp.high.end());
        std::sort(sp.tile.begin(), sp.tile.end());
        schedule_runs(gp.idx, steps, hops, sp.order, sp.runs);
        for (int j : sp.order)
            if (steps[size_t(j)].cls != AC_DIAG &&
                std::find(sp.tile.begin(), sp.tile.end(), hops[size_t(j)].bit) == sp.tile.end())
                return false;
        for (size_t r = 0, k = 0; r < sp.runs.size(); k += size_t(sp.runs[r].len), ++r) {
            // leading exchanges on the run's bits fold into the load
            int pre = 0;
            auto on_run = [&](int b) { return b == sp.runs[r].bit || b == sp.runs[r].bit2 || b == sp.runs[r].bit3; };
            while (pre < sp.runs[r].len && steps[size_t(sp.order[k + size_t(pre)])].cls == AC_X &&
                   on_run(hops[size_t(sp.order[k + size_t(pre)])].bit))
                ++pre;
            sp.pre.push_back(pre);
        }
        out.push_back(std::move(sp));
    }
    return true;
}

// The fused reverse sweep over steps[] (in forward order; run last to first).
template <typename R>
cudaError_t fused_sweep(qs_state *s, const std::vector<AdjStep> &steps, const std::vector<HostOp> &hops,
                        cplx<R> *psi, cplx<R> *lp, double *part, int grid, int K) {
    const int n = s->n;
    cudaStream_t st = s->stream;
    std::vector<SweepPass> plan;
    if (!plan_sweep(n, K, steps, hops, plan)) return cudaErrorInvalidValue;
    std::vector<AdjFOp<R>> flat;
    std::vector<AdjFPass<R>> passes;
    std::vector<size_t> offs;
    for (const SweepPass &sp : plan) {
        int local[64];
        for (int b = 0; b < 64; ++b) local[b] = -1;
        for (int k = 0; k < K; ++k) local[sp.tile[size_t(k)]] = k;
        AdjFPass<R> P;
        std::memset(&P, 0, sizeof(P));
        P.K = K;
        P.tiles = uint64_t(1) << (n - K);
        for (int k = 0; k < K; ++k) P.tile_pos[k] = uint8_t(sp.tile[size_t(k)]);
        offs.push_back(flat.size());
        if (sp.runs.size() > size_t(ADJ_MAX_OPS)) return cudaErrorInvalidValue;
        P.nrun = int(sp.runs.size());
        // each run's three role bits (tile-local): its target bits, then the
        // highest tile bits it does not target for the spare roles
        std::vector<std::array<int, RUN_BITS>> roles(sp.runs.size());
        std::vector<int> run_of;   // run of each op, in execution order
        for (size_t r = 0; r < sp.runs.size(); ++r) {
            const int tb[RUN_BITS] = {sp.runs[r].bit, sp.runs[r].bit2, sp.runs[r].bit3};
            std::array<int, RUN_BITS> &rl = roles[r];
            uint32_t used = 0;
            for (int i = 0; i < RUN_BITS; ++i) {
                rl[size_t(i)] = tb[i] >= 0 ? local[tb[i]] : -1;
                if (rl[size_t(i)] >= 0) used |= 1u << rl[size_t(i)];
            }
            for (int i = 0, b = K - 1; i < RUN_BITS; ++i) {
                if (rl[size_t(i)] >= 0) continue;
                while (b >= 0 && ((used >> b) & 1)) --b;
                if (b < 0) return cudaErrorInvalidValue;
                rl[size_t(i)] = b;
                used |= 1u << b;
            }
            P.run_len[r] = uint8_t(sp.runs[r].len);
            P.run_bit[r] = uint8_t(rl[0]);
            P.run_bit2[r] = uint8_t(rl[1]);
            P.run_bit3[r] = uint8_t(rl[2]);
            P.run_pre[r] = uint8_t(sp.pre[r]);
            for (int i = 0; i < sp.runs[r].len; ++i) run_of.push_back(int(r));
        }
        int nacc = 0;
        for (size_t oi = 0; oi < sp.order.size(); ++oi) {
            const int j = sp.order[oi];
            const AdjStep &d = steps[size_t(j)];
            const HostOp &o = hops[size_t(j)];
            AdjFOp<R> f;
            std::memset(&f, 0, sizeof(f));
            const int b = o.bit;
            if (d.cls == AC_DIAG) {
                if (local[b] >= 0) { f.mode = 2; f.tpos = local[b]; }
                else { f.mode = 3; f.tpos = b; }
            } else {
                f.mode = d.cls == AC_X ? 1 : d.cls == AC_REAL && real_gens(d) ? 4 : 0;
                f.tpos = local[b];
            }
            for (int c = 0; c < n; ++c) {
                if (!((o.cmask >> c) & 1)) continue;
                const bool one = (o.cval >> c) & 1;
                if (local[c] >= 0) { f.cm |= 1u << local[c]; if (one) f.cv |= 1u << local[c]; }
                else { f.om |= uint64_t(1) << c; if (one) f.ov |= uint64_t(1) << c; }
            }
            // the target bit's role in the op's run; 3 for a diagonal on no role bit
            f.role = 3;
            if (f.mode != 3)
                for (int i = 0; i < RUN_BITS; ++i)
                    if (roles[size_t(run_of[oi])][size_t(i)] == f.tpos) f.role = i;
            if (f.role == 3 && f.mode != 2 && f.mode != 3) return cudaErrorInvalidValue;   // a pair step off its run
            f.nang = d.nang;
            // generator entries (re, im) at 2e, 2e + 1 for e = 0..3
            if (f.mode == 4 && d.nang == 1 && d.g0[0] == 0.0 && d.g0[6] == 0.0 && d.g0[2] == -d.g0[4]) f.gk = 1;
            if ((f.mode == 2 || f.mode == 3) && d.nang == 1 && d.g0[0] == 0.0 && d.g0[6] == 0.0) f.gk = 2;
            f.acc = nacc;
            f.slot0 = d.slot0;
            f.slot1 = d.slot1;
            nacc += d.nang;
            for (int e = 0; e < 4; ++e) {
                f.ui[e] = cmat<R>(d.ui, e);
                f.g0[e] = cmat<R>(d.g0, e);
                f.g1[e] = cmat<R>(d.g1, e);
            }
            flat.push_back(f);
        }
        P.nops = int(sp.order.size());
        P.nacc = nacc;
        passes.push_back(P);
    }
    void *dops = nullptr;
    cudaError_t e = cudaMallocAsync(&dops, sizeof(AdjFOp<R>) * std::max<size_t>(1, flat.size()), st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dops, flat.data(), sizeof(AdjFOp<R>) * flat.size(), cudaMemcpyHostToDevice, st);
    size_t smem_max = 0;
    for (const AdjFPass<R> &P : passes) smem_max = std::max(smem_max, adj_smem<R>(K, P.nacc, P.nops));
    if (smem_max > adj_smem<R>(K, 2 * ADJ_MAX_OPS, ADJ_MAX_OPS)) e = cudaErrorInvalidValue;
    for (size_t k = 0; k < passes.size() && e == cudaSuccess; ++k) {
        AdjFPass<R> P = passes[k];
        P.ops = static_cast<const AdjFOp<R> *>(dops) + offs[k];
        k_adj_pass<R><<<unsigned(grid), AF_THREADS, adj_smem<R>(K, P.nacc, P.nops), st>>>(psi, lp, P, part);
        e = cudaGetLastError();
    }
    cudaFreeAsync(dops, st);
    return e;
}

// The circuit's reverse steps in forward order: one per synthesised gate, a
// SWAP as three C-NOTs; each differentiated angle gets a partial-sum slot,
// slot_param lists (parameter, slot) in gate order.
qs_status build_steps(int n, const std::vector<qs_gate> &gg, size_t n_params, std::vector<AdjStep> &steps,
                      std::vector<HostOp> &hops, std::vector<std::pair<int, int>> &slot_param) {
    qs_status rc = QS_OK;
    for (size_t jg = 0; jg < gg.size(); ++jg) {
        HostOp og;
        rc = synthesize(n, gg[jg], og);
        if (rc != QS_OK) return rc;
        std::vector<HostOp> parts;
        if (og.cls == GC_SWAP) {
            HostOp x = og;
            x.cls = GC_X;
            x.kind = QS_GATE_X;
            for (int k = 0; k < 8; ++k) x.u[k] = 0.0;
            x.u[2] = 1.0; x.u[4] = 1.0;
            HostOp c1 = x, c2 = x;
            c1.bit = og.bit; c1.cmask = uint64_t(1) << og.bit2; c1.cval = uint64_t(1) << og.bit2;
            c2.bit = og.bit2; c2.cmask = og.cmask | (uint64_t(1) << og.bit); c2.cval = og.cval | (uint64_t(1) << og.bit);
            parts = {c1, c2, c1};
        } else {
            parts = {og};
        }
        for (const HostOp &o : parts) {
            const size_t j = steps.size();
            steps.emplace_back();
            hops.push_back(o);
            AdjStep &d = steps[j];
            std::memset(&d, 0, sizeof(d));
            std::vector<int> pos;
            for (int b = 0; b < 64; ++b)
                if ((o.cmask >> b) & 1) pos.push_back(b);
            d.cval = o.cval;
            d.tbit = uint64_t(1) << o.bit;
            if (o.cls == GC_SWAP) {
                d.cls = AC_SWAP;
                d.tbit2 = uint64_t(1) << o.bit2;
                pos.push_back(o.bit);
                pos.push_back(o.bit2);
            } else {
                pos.push_back(o.bit);
                dagger(o.u, d.ui);
                d.cls = o.cls == GC_X ? AC_X
                      : (o.cls == GC_DIAG || o.cls == GC_PHASE || o.cls == GC_ID) ? AC_DIAG
                      : o.cls == GC_REAL ? AC_REAL : AC_GEN;
            }
            std::sort(pos.begin(), pos.end());
            d.nfixed = int(pos.size());
            for (size_t k = 0; k < pos.size(); ++k) d.pos[k] = uint8_t(pos[k]);
            if (gg[jg].param >= 0) {
                const int na = kind_angles(gg[jg].kind);
                if (na == 0) return fail(QS_EUNSUPPORTED, "adjoint: a parameter on a gate kind without angles");
                for (int a = 0; a < na; ++a) {
                    const int pidx = gg[jg].param + a;
                    if (pidx >= int(n_params)) return fail(QS_EINVAL, "adjoint: parameter index beyond n_params");
                    double *g = a == 0 ? d.g0 : d.g1;
                    generator(gg[jg].kind, a, gg[jg].theta[0], gg[jg].theta[1], g);
                    const int slot = int(slot_param.size());
                    (a == 0 ? d.slot0 : d.slot1) = slot;
                    slot_param.push_back({pidx, slot});
                }
                d.nang = na;
            }
        }
    }
    return QS_OK;
}

template <typename R>
qs_status run_adjoint(qs_state *s, const std::vector<qs_gate> &gg, size_t n_params, const qs_observable &obs,
                      double *value, double *grad, bool fuse) {
    const int n = s->n;
    const uint64_t N = uint64_t(1) << n;
    cudaStream_t st = s->stream;
    // forward
    qs_status rc = qs_init_basis(s, 0);
    if (rc != QS_OK) return rc;
    rc = qs_apply_circuit(s, gg.data(), gg.size(), nullptr);
    if (rc != QS_OK) return rc;
    // value, and lambda = O psi
    Buf lam;
    lam.s = st;
    if (cudaMallocAsync(&lam.p, sizeof(cplx<R>) * N, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "adjoint: device allocation failed");
    }
    const unsigned grid = unsigned(std::min<uint64_t>((N + THREADS - 1) / THREADS, 152ull * 16));
    if (obs.kind == QS_OBS_PAULI) {
        rc = qs_expect(s, obs.pauli, value);
        if (rc != QS_OK) return rc;
        uint64_t flip = 0, sign = 0;
        int ny = 0;
        for (int q = 0; q < n; ++q) {
            const uint64_t b = uint64_t(1) << (n - 1 - q);
            if (obs.pauli[q] == 'X') flip |= b;
            else if (obs.pauli[q] == 'Y') { flip |= b; sign |= b; ++ny; }
            else if (obs.pauli[q] == 'Z') sign |= b;
        }
        k_pauli_apply<R><<<grid, THREADS, 0, st>>>(static_cast<const cplx<R> *>(s->d), static_cast<cplx<R> *>(lam.p),
                                                   N, flip, sign, ny);
    } else {
        qs_c128 c;
        rc = qs_inner(const_cast<qs_state *>(obs.ref), s, &c);
        if (rc != QS_OK) return rc;
        *value = c.re * c.re + c.im * c.im;
        k_scale_copy<R><<<grid, THREADS, 0, st>>>(static_cast<const cplx<R> *>(obs.ref->d),
                                                  static_cast<cplx<R> *>(lam.p), N, c.re, c.im);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    // steps, slots (a SWAP becomes three C-NOTs)
    std::vector<AdjStep> steps;
    std::vector<HostOp> hops;
    std::vector<std::pair<int, int>> slot_param;   // (param, slot)
    rc = build_steps(n, gg, n_params, steps, hops, slot_param);
    if (rc != QS_OK) return rc;
    const int nslot = int(slot_param.size());
    // fused sweep: tiles of 2^K amplitudes (64 KiB per vector), one CTA per
    // tile at a time, as many CTAs as fit
    const int Kf = std::min(n, adj_full_k<R>());
    const bool fused = fuse && adj_fused_ok<R>(n);
    int nblk = RED_BLOCKS;
    if (fused) {
        // the largest pass: ADJ_MAX_OPS steps with two generators each
        const size_t smem_max = adj_smem<R>(Kf, 2 * ADJ_MAX_OPS, ADJ_MAX_OPS);
        cudaFuncSetAttribute(k_adj_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_max));
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adj_pass<R>, AF_THREADS, smem_max);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        nblk = int(std::min<uint64_t>(uint64_t(1) << (n - Kf), uint64_t(std::max(sms, 1)) * std::max(occ, 1)));
    }
    Buf part, ssum, dgrad, dfirst, dsteps;
    for (Buf *b : {&part, &ssum, &dgrad, &dfirst, &dsteps}) b->s = st;
    if (cudaMallocAsync(&part.p, sizeof(double) * std::max(1, nslot) * nblk, st) != cudaSuccess ||
        cudaMallocAsync(&ssum.p, sizeof(double) * std::max(1, nslot), st) != cudaSuccess ||
        cudaMallocAsync(&dgrad.p, sizeof(double) * std::max<size_t>(1, n_params), st) != cudaSuccess ||
        cudaMallocAsync(&dfirst.p, sizeof(int) * (n_params + 1), st) != cudaSuccess ||
        cudaMallocAsync(&dsteps.p, sizeof(AdjStep) * std::max<size_t>(1, steps.size()), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "adjoint: device allocation failed");
    }
    // slots ordered by parameter (stable in gate order): CSR offsets
    std::vector<std::pair<int, int>> order = slot_param;
    std::stable_sort(order.begin(), order.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    std::vector<int> remap(nslot), first(n_params + 1, 0);
    for (int k = 0; k < nslot; ++k) remap[order[k].second] = k;
    for (const auto &sp : slot_param) first[sp.first + 1]++;
    for (size_t p = 0; p < n_params; ++p) first[p + 1] += first[p];
    for (AdjStep &d : steps) {
        if (d.nang > 0) d.slot0 = remap[d.slot0];
        if (d.nang > 1) d.slot1 = remap[d.slot1];
    }
    e = cudaMemcpyAsync(dsteps.p, steps.data(), sizeof(AdjStep) * steps.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dfirst.p, first.data(), sizeof(int) * (n_params + 1), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint upload");
    // reverse sweep
    cplx<R> *psi = static_cast<cplx<R> *>(s->d);
    cplx<R> *lp = static_cast<cplx<R> *>(lam.p);
    if (fused) {
        e = fused_sweep<R>(s, steps, hops, psi, lp, static_cast<double *>(part.p), nblk, Kf);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint fused sweep");
    } else {
        for (size_t j = steps.size(); j-- > 0;) {
            k_adj<R><<<nblk, THREADS, 0, st>>>(psi, lp, n, static_cast<const AdjStep *>(dsteps.p) + j,
                                               static_cast<double *>(part.p));
        }
    }
    if (nslot > 0) k_slot_sums<<<nslot, THREADS, 0, st>>>(static_cast<const double *>(part.p), nblk,
                                                          static_cast<double *>(ssum.p));
    if (n_params > 0)
        k_collect<<<unsigned((n_params + 255) / 256), 256, 0, st>>>(static_cast<const double *>(ssum.p),
                                                                    static_cast<const int *>(dfirst.p), int(n_params),
                                                                    static_cast<double *>(dgrad.p));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    if (n_params > 0) {
        e = cudaMemcpyAsync(grad, dgrad.p, sizeof(double) * n_params, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint results");
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint");
    return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_adjoint_grad(qs_state *s, const qs_gate *g, size_t m, const double *params, size_t n_params,
                                     const qs_observable *obs, double *value, double *grad) {
    return qs_adjoint_grad_ex(s, g, m, params, n_params, obs, value, grad, nullptr);
}

extern "C" qs_status qs_adjoint_grad_ex(qs_state *s, const qs_gate *g, size_t m, const double *params,
                                        size_t n_params, const qs_observable *obs, double *value, double *grad,
                                        const qs_exec_opts *opts) {
    const bool fuse = !(opts && opts->no_fusion);
    if (!s || !obs || !value || (m > 0 && !g) || (n_params > 0 && (!params || !grad)))
        return fail(QS_EINVAL, "NULL argument");
    if (n_params > (size_t(1) << 30)) return fail(QS_ERANGE, "too many parameters");
    if (obs->kind == QS_OBS_PAULI) {
        if (!obs->pauli || std::strlen(obs->pauli) != size_t(s->n)) return fail(QS_EINVAL, "observable: Pauli string length");
        for (int q = 0; q < s->n; ++q)
            if (!std::strchr("IXYZ", obs->pauli[q])) return fail(QS_EINVAL, "observable: Pauli characters");
    } else if (obs->kind == QS_OBS_FIDELITY) {
        if (!obs->ref || obs->ref->n != s->n || obs->ref->dt != s->dt) return fail(QS_EINVAL, "observable: reference state");
        if (obs->ref->stream != s->stream) return fail(QS_EINVAL, "observable: reference on another stream");
    } else {
        return fail(QS_EINVAL, "observable: bad kind");
    }
    std::vector<qs_gate> gg(g, g + m);
    for (qs_gate &x : gg) {
        if (x.param < 0) continue;
        const int na = kind_angles(x.kind);
        if (x.param + std::max(na, 1) > int64_t(n_params)) return fail(QS_EINVAL, "gate parameter index beyond n_params");
        for (int a = 0; a < na; ++a) x.theta[a] = params[x.param + a];
    }
    return s->dt == QS_C64 ? run_adjoint<float>(s, gg, n_params, *obs, value, grad, fuse)
                           : run_adjoint<double>(s, gg, n_params, *obs, value, grad, fuse);
}

extern "C" qs_status qs_adjoint_describe(int n, qs_dtype dt, const qs_gate *g, size_t m, char *buf, size_t len,
                                         size_t *needed) {
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_ERANGE, "n out of range");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    if (m > 0 && !g) return fail(QS_EINVAL, "NULL argument");
    std::vector<qs_gate> gg(g, g + m);
    size_t n_params = 0;
    for (const qs_gate &x : gg)
        if (x.param >= 0) n_params = std::max(n_params, size_t(x.param) + size_t(std::max(kind_angles(x.kind), 1)));
    std::vector<AdjStep> steps;
    std::vector<HostOp> hops;
    std::vector<std::pair<int, int>> slot_param;
    qs_status rc = build_steps(n, gg, n_params, steps, hops, slot_param);
    if (rc != QS_OK) return rc;
    std::string out;
    char line[640];
    for (size_t j = 0; j < steps.size(); ++j) {
        const HostOp &o = hops[j];
        const int c = steps[j].cls;
        const char *cls = c == AC_DIAG ? "diag" : c == AC_X ? "x" : c == AC_REAL ? "real" : "gen";
        std::snprintf(line, sizeof(line),
                      "step %zu cls=%s bit=%d cmask=%llx cval=%llx u=%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g\n", j,
                      cls, int(o.bit), (unsigned long long)o.cmask, (unsigned long long)o.cval, o.u[0], o.u[1], o.u[2],
                      o.u[3], o.u[4], o.u[5], o.u[6], o.u[7]);
        out += line;
    }
    if (dt == QS_C64 ? adj_fused_ok<float>(n) : adj_fused_ok<double>(n)) {
        const int K = std::min(n, dt == QS_C64 ? adj_full_k<float>() : adj_full_k<double>());
        std::vector<SweepPass> plan;
        if (!plan_sweep(n, K, steps, hops, plan)) return fail(QS_EUNSUPPORTED, "adjoint plan: a target outside its tile");
        for (size_t p = 0; p < plan.size(); ++p) {
            out += "pass " + std::to_string(p) + " tile=";
            for (size_t k = 0; k < plan[p].tile.size(); ++k) out += (k ? "," : "") + std::to_string(plan[p].tile[k]);
            out += "\n";
            size_t k = 0;
            for (size_t r = 0; r < plan[p].runs.size(); ++r) {
                out += "run bit=" + std::to_string(plan[p].runs[r].bit) + " bit2=" + std::to_string(plan[p].runs[r].bit2) +
                       " bit3=" + std::to_string(plan[p].runs[r].bit3) + " pre=" + std::to_string(plan[p].pre[r]) +
                       " steps=";
                for (int i = 0; i < plan[p].runs[r].len; ++i, ++k)
                    out += (i ? "," : "") + std::to_string(plan[p].order[k]);
                out += "\n";
            }
        }
    }
    if (needed) *needed = out.size() + 1;
    if (buf && len) {
        const size_t k = std::min(len - 1, out.size());
        std::memcpy(buf, out.data(), k);
        buf[k] = 0;
    }
    return QS_OK;
}
