// Batched noisy trajectories (quant-ph/0201042, Sec. 3 and the error
// experiments of Sec. 4.3.1, 5.2 and 5.3).
//
// The paper simulates decoherence and operational errors with pure states:
// each run draws its own errors and the results are averaged over 1000-10000
// runs.  Here all runs of a width group live side by side in device memory
// (trajectory b of a group at amplitude offset b * 2^n) and every gate step
// updates all of them in one launch:
//
//   1. k_noise draws, for every (trajectory, step), the Gaussian deviations of
//      the step's gate angles (Sec. 3.2) and synthesises that trajectory's
//      gate matrix, and draws the Pauli flips that follow the step (Sec. 3.1)
//      as X/Z index masks.  Draws come from Philox4x32-10 with counter
//      (trajectory, step, slot, stream), so every trajectory can be replayed
//      alone, in any order, with bit-identical flip decisions.
//   2. k_lists compacts, per step, the ids of the trajectories that flip.
//   3. Per step: k_gate applies each trajectory's own matrix to its amplitude
//      pairs (one thread per pair, both amplitudes read before either is
//      written, as in Sec. 2.2.1); k_flip applies the flips of the listed
//      trajectories.
//   4. The fidelity to the noiseless output |<U x0|psi>|^2 (Sec. 5.2) is the
//      probability of x0 after the inverse noiseless circuit (an echo), so no
//      reference state is stored; the probability of a marked index (Sec. 5.3)
//      is read directly.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qs_internal.cuh"

namespace qs {

namespace {

constexpr int THREADS = 256;

enum TrajClass : int32_t { TC_GEN = 0, TC_PHASE1 = 1, TC_PHASE0 = 2, TC_DIAG = 3, TC_SWAP = 4 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:
// per round the 64-bit products c0 * M0 and c2 * M1 give the new words
// (hi(c2 M1) ^ c1 ^ k0, lo(c2 M1), hi(c0 M0) ^ c3 ^ k1, lo(c0 M0)); the key
// is bumped by the two Weyl increments after each round; ten rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint64_t splitmix_final(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Standard normal deviate of angle a of step s of trajectory t (Box-Muller).
__device__ __forceinline__ double gauss(uint32_t t, uint32_t s, uint32_t a, uint32_t k0, uint32_t k1) {
    const uint4 w = philox(make_uint4(t, s, 64u + a, 1u), k0, k1);
    const uint64_t x = (uint64_t(w.x) << 32) | w.y, y = (uint64_t(w.z) << 32) | w.w;
    const double u1 = 1.0 - double(x >> 11) * 0x1.0p-53;
    const double u2 = double(y >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

// Gate matrix (row major, re/im) from kind and angles: H (Sec. 2.3.1), U_R,
// U_P1, U_P2 and their product (Sec. 3.2), Pauli matrices, RY, RZ.
__device__ void synth(int kind, double a, double b, const double *mtx, double *u) {
    for (int k = 0; k < 8; ++k) u[k] = 0.0;
    switch (kind) {
    case QS_GATE_MATRIX: for (int k = 0; k < 8; ++k) u[k] = mtx[k]; break;
    case QS_GATE_H: { const double s = 1.0 / sqrt(2.0); u[0] = s; u[2] = s; u[4] = s; u[6] = -s; break; }
    case QS_GATE_X: u[2] = 1; u[4] = 1; break;
    case QS_GATE_Y: u[3] = -1; u[5] = 1; break;
    case QS_GATE_Z: u[0] = 1; u[6] = -1; break;
    case QS_GATE_UP1: u[0] = 1; u[6] = cos(a); u[7] = sin(a); break;
    case QS_GATE_UP2: u[0] = cos(a); u[1] = sin(a); u[6] = 1; break;
    case QS_GATE_UR: u[0] = cos(a); u[2] = -sin(a); u[4] = sin(a); u[6] = cos(a); break;
    case QS_GATE_URP1: {
        const double c = cos(a), s = sin(a), cb = cos(b), sb = sin(b);
        u[0] = c; u[2] = -s * cb; u[3] = -s * sb; u[4] = s; u[6] = c * cb; u[7] = c * sb;
        break;
    }
    case QS_GATE_RY: u[0] = cos(a / 2); u[2] = -sin(a / 2); u[4] = sin(a / 2); u[6] = cos(a / 2); break;
    case QS_GATE_RZ: u[0] = cos(a / 2); u[1] = -sin(a / 2); u[6] = cos(a / 2); u[7] = sin(a / 2); break;
    default: break;
    }
}

struct StepDesc {          // one gate step of a group, as the kernels see it
    int32_t kind;
    int32_t cls;           // TrajClass
    int32_t bit, bit2;     // target (and second SWAP) index bits
    int32_t nang;          // angles deviated by operational errors
    int32_t flags;         // QS_TRAJ_NO_DEVIATION | QS_TRAJ_NO_FLIPS
    uint64_t cmask, cval;  // controls (index bits)
    double theta[2];
    double u[8];           // ideal matrix (MATRIX gates, echo steps)
    uint8_t fixed_pos[64]; // sorted fixed bit positions (controls + target[s])
    int32_t nfixed;
    int32_t pad2;
};

__device__ __forceinline__ uint64_t deposit(uint64_t p, const uint8_t *pos, int nf) {
    for (int k = 0; k < nf; ++k) {
        const uint64_t low = (uint64_t(1) << pos[k]) - 1;
        p = ((p & ~low) << 1) | (p & low);
    }
    return p;
}

// Noise of every (trajectory, step): matrix table and flip masks.
template <typename R>
__global__ void __launch_bounds__(THREADS) k_noise(const StepDesc *__restrict__ steps, int m, int n, uint32_t first,
                                                   uint32_t count, uint32_t k0, uint32_t k1, double sigma,
                                                   uint32_t thr, int mode, int every, cplx<R> *__restrict__ mtab,
                                                   uint64_t *__restrict__ ftab,
                                                   unsigned long long *__restrict__ stats) {
    const uint64_t total = uint64_t(count) * m;
    for (uint64_t it = uint64_t(blockIdx.x) * THREADS + threadIdx.x; it < total;
         it += uint64_t(gridDim.x) * THREADS) {
        const uint32_t b = uint32_t(it / m), s = uint32_t(it % m);
        const uint32_t traj = first + b;
        const StepDesc &d = steps[s];
        double ang[2] = {d.theta[0], d.theta[1]};
        if (sigma != 0.0 && !(d.flags & QS_TRAJ_NO_DEVIATION))
            for (int a = 0; a < d.nang; ++a) ang[a] += sigma * gauss(traj, s, uint32_t(a), k0, k1);
        double u[8];
        synth(d.kind, ang[0], ang[1], d.u, u);
        cplx<R> *mt = mtab + it * 4;
        for (int k = 0; k < 4; ++k) mt[k] = mk<R>(R(u[2 * k]), R(u[2 * k + 1]));
        uint64_t xm = 0, zm = 0;
        int ny = 0;
        if (thr != 0 && !(d.flags & QS_TRAJ_NO_FLIPS) && (every <= 1 || (s + 1) % uint32_t(every) == 0)) {
            for (int q = 0; q < n; ++q) {
                const uint4 w = philox(make_uint4(traj, s, uint32_t(q), 0u), k0, k1);
                if (w.x >= thr) continue;
                int kind;
                if (mode == QS_NOISE_DEPOLARIZING) kind = 1 + int((uint64_t(w.y) * 3u) >> 32);
                else kind = (w.y & 1u) ? 3 : 1;
                const uint64_t bit = uint64_t(1) << (n - 1 - q);
                if (kind == 1) xm |= bit;
                else if (kind == 2) { xm |= bit; zm |= bit; ++ny; }
                else zm |= bit;
                if (stats) {
                    atomicAdd(&stats[uint64_t(b) * 4 + (kind - 1)], 1ull);
                    atomicAdd(&stats[uint64_t(b) * 4 + 3],
                              (unsigned long long)splitmix_final((uint64_t(s) * 64u + uint64_t(q)) * 4u + uint64_t(kind)));
                }
            }
        }
        ftab[it * 2] = xm;
        ftab[it * 2 + 1] = zm | (uint64_t(ny & 3) << 62);
    }
}

// Per step, the ordered list of trajectories that flip after it (one warp per step).
__global__ void k_lists(const uint64_t *__restrict__ ftab, int m, uint32_t count, uint32_t *__restrict__ lists,
                        uint32_t *__restrict__ lens) {
    const int warps = blockDim.x / 32;
    const int s = blockIdx.x * warps + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (s >= m) return;
    uint32_t len = 0;
    for (uint32_t b0 = 0; b0 < count; b0 += 32) {
        const uint32_t b = b0 + lane;
        bool f = false;
        if (b < count) {
            const uint64_t it = uint64_t(b) * m + s;
            f = (ftab[it * 2] | (ftab[it * 2 + 1] & ~(uint64_t(3) << 62))) != 0;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, f);
        if (f) lists[uint64_t(s) * count + len + __popc(ball & ((1u << lane) - 1))] = b;
        len += __popc(ball);
    }
    if (lane == 0) lens[s] = len;
}

// One gate step on every trajectory of a group.  The matrix of trajectory b is
// mtab[(b * mstride + s) * 4 ...] (mstride 0: one matrix for all).
template <typename R>
__global__ void __launch_bounds__(THREADS) k_gate(cplx<R> *__restrict__ st, int n, uint32_t count,
                                                  const StepDesc *__restrict__ dp, const cplx<R> *__restrict__ mtab,
                                                  int s, int mstride) {
    const StepDesc &d = *dp;
    const int nf = d.nfixed;
    const uint64_t per = uint64_t(1) << (n - nf);   // items per trajectory
    const uint64_t total = per * count;
    const uint64_t N = uint64_t(1) << n;
    for (uint64_t it = uint64_t(blockIdx.x) * THREADS + threadIdx.x; it < total;
         it += uint64_t(gridDim.x) * THREADS) {
        const uint64_t b = it / per, p = it % per;
        cplx<R> *a = st + b * N;
        const cplx<R> *mt = mtab + (uint64_t(mstride) * b + s) * 4;
        const uint64_t i0 = deposit(p, d.fixed_pos, nf) | d.cval;
        if (d.cls == TC_GEN) {
            const uint64_t i1 = i0 | (uint64_t(1) << d.bit);
            const cplx<R> x = a[i0], y = a[i1];
            a[i0] = cmad2<R>(mt[0], x, mt[1], y);
            a[i1] = cmad2<R>(mt[2], x, mt[3], y);
        } else if (d.cls == TC_PHASE1) {   // only the target-1 amplitude changes
            const uint64_t i1 = i0 | (uint64_t(1) << d.bit);
            a[i1] = cmul<R>(mt[3], a[i1]);
        } else if (d.cls == TC_PHASE0) {   // only the target-0 amplitude changes
            a[i0] = cmul<R>(mt[0], a[i0]);
        } else if (d.cls == TC_DIAG) {
            const uint64_t i1 = i0 | (uint64_t(1) << d.bit);
            a[i0] = cmul<R>(mt[0], a[i0]);
            a[i1] = cmul<R>(mt[3], a[i1]);
        } else {   // TC_SWAP: (1, 0) <-> (0, 1) in bits (bit, bit2)
            const uint64_t ia = i0 | (uint64_t(1) << d.bit), ib = i0 | (uint64_t(1) << d.bit2);
            const cplx<R> x = a[ia], y = a[ib];
            a[ia] = y;
            a[ib] = x;
        }
    }
}

// The Pauli flips after step s of the listed trajectories:
// P|i> = i^ny (-1)^popcount(i & zm) |i ^ xm>.
template <typename R>
__global__ void __launch_bounds__(THREADS) k_flip(cplx<R> *__restrict__ st, int n, int m, int s, uint32_t count,
                                                  const uint64_t *__restrict__ ftab, const uint32_t *__restrict__ lists,
                                                  const uint32_t *__restrict__ lens) {
    const uint32_t L = lens[s];
    const uint64_t N = uint64_t(1) << n;
    const uint64_t total = uint64_t(L) * N;
    for (uint64_t it = uint64_t(blockIdx.x) * THREADS + threadIdx.x; it < total;
         it += uint64_t(gridDim.x) * THREADS) {
        const uint32_t b = lists[uint64_t(s) * count + it / N];
        const uint64_t j = it % N;
        const uint64_t e = (uint64_t(b) * m + s) * 2;
        const uint64_t xm = ftab[e], zw = ftab[e + 1];
        const uint64_t zm = zw & ~(uint64_t(3) << 62);
        const int ny = int(zw >> 62);
        cplx<R> *a = st + uint64_t(b) * N;
        auto phase = [&](uint64_t i, cplx<R> v) {
            if (__popcll(i & zm) & 1) v = mk<R>(-v.x, -v.y);
            switch (ny) {   // multiply by i^ny
            case 1: v = mk<R>(-v.y, v.x); break;
            case 2: v = mk<R>(-v.x, -v.y); break;
            case 3: v = mk<R>(v.y, -v.x); break;
            default: break;
            }
            return v;
        };
        const uint64_t k = j ^ xm;
        if (k < j) continue;                 // the pair is handled by its lower index
        if (k == j) { a[j] = phase(j, a[j]); continue; }
        const cplx<R> vj = a[j], vk = a[k];
        a[k] = phase(j, vj);
        a[j] = phase(k, vk);
    }
}

template <typename R>
__global__ void k_init(cplx<R> *__restrict__ st, int n, uint32_t count, const uint64_t *__restrict__ x0) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x)
        st[(uint64_t(b) << n) + x0[b]] = mk<R>(R(1), R(0));
}

template <typename R>
__global__ void k_metric(const cplx<R> *__restrict__ st, int n, uint32_t count, const uint64_t *__restrict__ idx,
                         uint64_t target, int use_idx, double *__restrict__ out) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
        const uint64_t i = use_idx ? idx[b] : target;
        const cplx<R> v = st[(uint64_t(b) << n) + i];
        const double x = double(v.x), y = double(v.y);
        out[b] = x * x + y * y;
    }
}

unsigned grid_for(uint64_t items) {
    uint64_t g = (items + THREADS - 1) / THREADS;
    return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(g, 152ull * 32)));
}

int n_angles(int kind) {
    switch (kind) {
    case QS_GATE_UP1: case QS_GATE_UP2: case QS_GATE_UR: case QS_GATE_RY: case QS_GATE_RZ: return 1;
    case QS_GATE_URP1: return 2;
    default: return 0;
    }
}

StepDesc make_step(const HostOp &o, int kind_override = -1) {
    StepDesc d;
    std::memset(&d, 0, sizeof(d));
    d.kind = kind_override >= 0 ? kind_override : o.kind;
    d.bit = o.bit;
    d.bit2 = o.bit2;
    d.cmask = o.cmask;
    d.cval = o.cval;
    d.theta[0] = o.theta[0];
    d.theta[1] = o.theta[1];
    for (int k = 0; k < 8; ++k) d.u[k] = o.u[k];
    d.nang = kind_override >= 0 ? 0 : n_angles(o.kind);
    std::vector<int> pos;
    for (int b = 0; b < 64; ++b)
        if ((o.cmask >> b) & 1) pos.push_back(b);
    if (o.cls == GC_SWAP) {
        d.cls = TC_SWAP;
        pos.push_back(o.bit);
        pos.push_back(o.bit2);
    } else {
        pos.push_back(o.bit);
        // structural class from the kind (a deviated phase stays a phase)
        const int k = d.kind;
        if (k == QS_GATE_UP1 || k == QS_GATE_Z) d.cls = TC_PHASE1;
        else if (k == QS_GATE_UP2) d.cls = TC_PHASE0;
        else if (k == QS_GATE_RZ) d.cls = TC_DIAG;
        else if (k == QS_GATE_MATRIX && (o.cls == GC_PHASE || o.cls == GC_DIAG || o.cls == GC_ID))
            d.cls = TC_DIAG;
        else d.cls = TC_GEN;
    }
    std::sort(pos.begin(), pos.end());
    d.nfixed = int(pos.size());
    for (size_t k = 0; k < pos.size(); ++k) d.fixed_pos[k] = uint8_t(pos[k]);
    return d;
}

// The inverse of a synthesised gate as an explicit matrix step (no noise).
StepDesc inverse_step(const HostOp &o) {
    HostOp inv = o;
    if (o.cls != GC_SWAP) {
        // conjugate transpose
        const double *u = o.u;
        double v[8] = {u[0], -u[1], u[4], -u[5], u[2], -u[3], u[6], -u[7]};
        for (int k = 0; k < 8; ++k) inv.u[k] = v[k];
    }
    StepDesc d = make_step(inv, QS_GATE_MATRIX);
    if (o.cls != GC_SWAP) d.cls = (o.cls == GC_PHASE || o.cls == GC_DIAG || o.cls == GC_ID) ? TC_DIAG : TC_GEN;
    return d;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, std::max<size_t>(bytes, 16)); }
};

// ---------------------------------------------------------------------------
// Fused trajectory path (complex64, n >= 10).  Flips are not applied to the
// data: each trajectory carries a Pauli frame F (psi_true = F psi_sim, F an X
// and a Z mask up to a phase, the XOR of all flips so far).  A later gate G is
// applied as F^dagger G F: its target matrix conjugated by the frame's Pauli
// on the target, its control values flipped where F has an X.  All
// trajectories then share one fused pass structure; a precompute writes each
// (trajectory, op) record, and the metric reads psi_sim at index ^ F_x.
// ---------------------------------------------------------------------------

// Frame before every step (and after the last) of every trajectory.
__global__ void k_frames(const uint64_t *__restrict__ ftab, int m, uint32_t count, uint64_t *__restrict__ fb) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
        uint64_t fx = 0, fz = 0;
        uint64_t *o = fb + uint64_t(b) * (m + 1) * 2;
        for (int s = 0; s < m; ++s) {
            o[2 * s] = fx;
            o[2 * s + 1] = fz;
            const uint64_t e = (uint64_t(b) * m + s) * 2;
            fx ^= ftab[e];
            fz ^= ftab[e + 1] & ~(uint64_t(3) << 62);
        }
        o[2 * m] = fx;
        o[2 * m + 1] = fz;
    }
}

// Per (trajectory, op) record: matrix conjugated by the frame's Pauli on the
// target (F^dagger G F with F = X^x Z^z: first swap rows and columns for X,
// then negate the off-diagonal for Z), control-value XORs where F has an X.
__global__ void __launch_bounds__(THREADS) k_optab(const TrajOpMeta *__restrict__ metas, uint32_t nmeta,
                                                   const float2 *__restrict__ mtab, int m, uint32_t count,
                                                   const uint64_t *__restrict__ fb, TrajRec *__restrict__ recs) {
    const uint64_t total = uint64_t(count) * nmeta;
    for (uint64_t it = uint64_t(blockIdx.x) * THREADS + threadIdx.x; it < total; it += uint64_t(gridDim.x) * THREADS) {
        const uint32_t b = uint32_t(it / nmeta), k = uint32_t(it % nmeta);
        const TrajOpMeta &d = metas[k];
        if (d.step < 0) continue;
        const uint64_t fx = fb[(uint64_t(b) * (m + 1) + d.step) * 2];
        const uint64_t fz = fb[(uint64_t(b) * (m + 1) + d.step) * 2 + 1];
        float2 u[4];
        if (d.msrc == 0) {
            const float2 *src = mtab + (uint64_t(b) * m + d.step) * 4;
            for (int e = 0; e < 4; ++e) u[e] = src[e];
        } else {
            for (int e = 0; e < 4; ++e) u[e] = make_float2(float(d.u[2 * e]), float(d.u[2 * e + 1]));
        }
        const bool px = (fx >> d.tbit) & 1, pz = (fz >> d.tbit) & 1;
        TrajRec r;
        if (d.diag) {
            float2 d0 = u[0], d1 = u[3];
            if (px) { const float2 t = d0; d0 = d1; d1 = t; }
            r.u[0] = d0; r.u[1] = d1; r.u[2] = make_float2(0.f, 0.f); r.u[3] = make_float2(0.f, 0.f);
        } else {
            if (px) {
                const float2 t0 = u[0], t1 = u[1];
                u[0] = u[3]; u[1] = u[2]; u[2] = t1; u[3] = t0;
            }
            if (pz) {
                u[1] = make_float2(-u[1].x, -u[1].y);
                u[2] = make_float2(-u[2].x, -u[2].y);
            }
            for (int e = 0; e < 4; ++e) r.u[e] = u[e];
        }
        const uint64_t flip = fx & d.cmask;
        uint8_t rvx = 0;
        uint16_t tvx = 0;
        for (int q = 0; q < 8; ++q)
            if (d.reg_src[q] >= 0 && ((flip >> d.reg_src[q]) & 1)) rvx |= uint8_t(1u << q);
        for (int q = 0; q < 16; ++q)
            if (d.thr_src[q] >= 0 && ((flip >> d.thr_src[q]) & 1)) tvx |= uint16_t(1u << q);
        r.ovx = flip & d.omask;
        r.tvx = tvx;
        r.rvx = rvx;
        for (int q = 0; q < 5; ++q) r.pad[q] = 0;
        recs[it] = r;
    }
}

template <typename R>
__global__ void k_metric_frame(const cplx<R> *__restrict__ st, int n, uint32_t count, const uint64_t *__restrict__ idx,
                               uint64_t target, int use_idx, const uint64_t *__restrict__ fb, int m,
                               double *__restrict__ out) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
        const uint64_t fx = fb[(uint64_t(b) * (m + 1) + m) * 2];
        const uint64_t i = (use_idx ? idx[b] : target) ^ fx;
        const cplx<R> v = st[(uint64_t(b) << n) + i];
        const double x = double(v.x), y = double(v.y);
        out[b] = x * x + y * y;
    }
}

bool diag_kind(int kind) {
    return kind == QS_GATE_UP1 || kind == QS_GATE_UP2 || kind == QS_GATE_RZ || kind == QS_GATE_Z;
}

// Op list of a group for the fused path: forward steps (noisy matrices), then
// the inverse noiseless circuit for the fidelity echo (fixed matrices, final
// frame).  SWAPs become three C-NOTs (fixed X matrices).
void traj_ops(const std::vector<HostOp> &ops, bool echo, std::vector<HostOp> &out) {
    const int m = int(ops.size());
    auto add_swap = [&](const HostOp &o, int step) {
        HostOp x{};
        x.cls = GC_GEN;
        x.kind = QS_GATE_MATRIX;
        x.param = -1;
        x.u[2] = 1.0; x.u[4] = 1.0;
        x.step = step;
        x.msrc = 1;
        HostOp c1 = x, c2 = x;
        c1.bit = o.bit; c1.cmask = uint64_t(1) << o.bit2; c1.cval = uint64_t(1) << o.bit2;
        c2.bit = o.bit2; c2.cmask = o.cmask | (uint64_t(1) << o.bit); c2.cval = o.cval | (uint64_t(1) << o.bit);
        out.push_back(c1);
        out.push_back(c2);
        out.push_back(c1);
    };
    for (int s = 0; s < m; ++s) {
        const HostOp &o = ops[s];
        if (o.cls == GC_SWAP) { add_swap(o, s); continue; }
        HostOp q = o;
        q.step = s;
        q.msrc = 0;
        const bool dg = diag_kind(o.kind) ||
                        (o.kind == QS_GATE_MATRIX && (o.cls == GC_DIAG || o.cls == GC_PHASE || o.cls == GC_ID));
        q.cls = dg ? GC_DIAG : GC_GEN;
        q.kind = QS_GATE_MATRIX;   // no Hadamard folding: the matrices differ per trajectory
        out.push_back(q);
    }
    if (!echo) return;
    for (int s = m - 1; s >= 0; --s) {
        const HostOp &o = ops[s];
        if (o.cls == GC_SWAP) { add_swap(o, m); continue; }
        HostOp q = o;
        const double *u = o.u;
        const double v[8] = {u[0], -u[1], u[4], -u[5], u[2], -u[3], u[6], -u[7]};   // U^dagger
        for (int k = 0; k < 8; ++k) q.u[k] = v[k];
        q.step = m;
        q.msrc = 1;
        const bool dg = diag_kind(o.kind) || o.cls == GC_DIAG || o.cls == GC_PHASE || o.cls == GC_ID;
        q.cls = dg ? GC_DIAG : GC_GEN;
        q.kind = QS_GATE_MATRIX;
        out.push_back(q);
    }
}

// Fusion depth of a group's fused passes, chosen by timing: every candidate
// depth runs the group's passes on a sub-batch of its own trajectories (their
// real op records), and the fastest is kept for that (width, op list, batch
// size) on this device.
uint64_t ops_hash(const std::vector<HostOp> &ops) {
    uint64_t h = 1469598103934665603ull;
    for (const HostOp &o : ops) {
        const uint64_t v[5] = {uint64_t(o.cls), uint64_t(o.bit), o.cmask, o.cval, uint64_t(o.step)};
        for (uint64_t x : v) { h ^= x; h *= 1099511628211ull; }
    }
    return h;
}

qs_status tune_depth(int n, const std::vector<HostOp> &fops, uint32_t count, int m, const float2 *mtab,
                     const uint64_t *ftab, int *out) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, uint64_t, uint32_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t sub = std::min<uint32_t>(count, n >= 18 ? 16u : 128u);
    const auto key = std::make_tuple(dev, n, ops_hash(fops), sub);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) { *out = it->second; return QS_OK; }
    }
    const int cands[3] = {120, 48, 16};
    float best_ms = 1e30f;
    int best = cands[0];
    DevBuf st, fb, meta, recs;
    const uint64_t N = uint64_t(1) << n;
    if (st.alloc(sizeof(float2) * N * sub) != cudaSuccess || fb.alloc(sizeof(uint64_t) * 2 * uint64_t(sub) * (m + 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "trajectory tuning: device allocation failed");
    }
    k_frames<<<grid_for(sub), THREADS>>>(ftab, m, sub, static_cast<uint64_t *>(fb.p));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c : cands) {
        TrajPlan *tp = nullptr;
        qs_status rc = traj_plan_build(n, fops, c, &tp);
        if (rc != QS_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
        const std::vector<TrajOpMeta> &metas = traj_plan_metas(tp);
        DevBuf dm, dr;
        if (dm.alloc(sizeof(TrajOpMeta) * metas.size()) != cudaSuccess ||
            dr.alloc(sizeof(TrajRec) * uint64_t(sub) * metas.size()) != cudaSuccess) {
            cudaGetLastError();
            traj_plan_destroy(tp);
            cudaEventDestroy(e0); cudaEventDestroy(e1);
            return fail(QS_ENOMEM, "trajectory tuning: device allocation failed");
        }
        cudaMemcpy(dm.p, metas.data(), sizeof(TrajOpMeta) * metas.size(), cudaMemcpyHostToDevice);
        k_optab<<<grid_for(uint64_t(sub) * metas.size()), THREADS>>>(
            static_cast<const TrajOpMeta *>(dm.p), uint32_t(metas.size()), mtab, m, sub,
            static_cast<const uint64_t *>(fb.p), static_cast<TrajRec *>(dr.p));
        cudaMemset(st.p, 0, sizeof(float2) * N * sub);
        float ms = 0.f;
        cudaError_t e = traj_plan_run(tp, static_cast<float2 *>(st.p), sub, static_cast<const TrajRec *>(dr.p), nullptr);
        if (e == cudaSuccess) {
            cudaEventRecord(e0);
            e = traj_plan_run(tp, static_cast<float2 *>(st.p), sub, static_cast<const TrajRec *>(dr.p), nullptr);
            cudaEventRecord(e1);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        traj_plan_destroy(tp);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0); cudaEventDestroy(e1);
            return cuda_fail(e, "trajectory tuning");
        }
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    *out = best;
    return QS_OK;
}

template <typename R>
qs_status run_group(const qs_traj_group &g, const qs_noise &nz, uint64_t seed, double *metric, uint64_t *stats,
                    int fuse_mode, int max_ops) {
    const int n = g.n;
    // fused passes for complex64 registers of 10 qubits or more
    const bool fused = fuse_mode != 0 && sizeof(R) == 4 && n >= 10;
    const int m = int(g.m);
    const uint32_t count = g.count;
    if (count == 0) return QS_OK;
    std::vector<HostOp> ops(g.m);
    for (size_t k = 0; k < g.m; ++k) {
        qs_status st = synthesize(n, g.gates[k], ops[k]);
        if (st != QS_OK) return st;
    }
    std::vector<StepDesc> steps;
    for (size_t k = 0; k < ops.size(); ++k) {
        steps.push_back(make_step(ops[k]));
        steps.back().flags = g.flags ? int32_t(g.flags[k] & 3u) : 0;
    }
    std::vector<StepDesc> echo;
    if (g.metric == QS_TRAJ_FIDELITY)
        for (size_t k = ops.size(); k-- > 0;) echo.push_back(inverse_step(ops[k]));
    // echo matrices (one per echo step, shared by all trajectories)
    std::vector<cplx<R>> echo_m(echo.size() * 4);
    for (size_t k = 0; k < echo.size(); ++k)
        for (int e = 0; e < 4; ++e) echo_m[k * 4 + e] = mk<R>(R(echo[k].u[2 * e]), R(echo[k].u[2 * e + 1]));

    const uint64_t N = uint64_t(1) << n;
    DevBuf d_st, d_steps, d_echo, d_echom, d_mtab, d_ftab, d_lists, d_lens, d_stats, d_metric, d_x0;
    cudaError_t e;
    if ((e = d_st.alloc(sizeof(cplx<R>) * N * count)) != cudaSuccess ||
        (e = d_steps.alloc(sizeof(StepDesc) * std::max<size_t>(1, steps.size()))) != cudaSuccess ||
        (e = d_echo.alloc(sizeof(StepDesc) * std::max<size_t>(1, echo.size()))) != cudaSuccess ||
        (e = d_echom.alloc(sizeof(cplx<R>) * std::max<size_t>(1, echo_m.size()))) != cudaSuccess ||
        (e = d_mtab.alloc(sizeof(cplx<R>) * 4 * uint64_t(count) * std::max(1, m))) != cudaSuccess ||
        (e = d_ftab.alloc(sizeof(uint64_t) * 2 * uint64_t(count) * std::max(1, m))) != cudaSuccess ||
        (e = d_lists.alloc(sizeof(uint32_t) * uint64_t(count) * std::max(1, m))) != cudaSuccess ||
        (e = d_lens.alloc(sizeof(uint32_t) * std::max(1, m))) != cudaSuccess ||
        (e = d_stats.alloc(sizeof(uint64_t) * 4 * count)) != cudaSuccess ||
        (e = d_metric.alloc(sizeof(double) * count)) != cudaSuccess ||
        (e = d_x0.alloc(sizeof(uint64_t) * count)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "trajectory batch: device allocation failed");
    }
    cudaStream_t sm = nullptr;
    auto ck = [&](cudaError_t r, const char *w) -> qs_status { return r == cudaSuccess ? QS_OK : cuda_fail(r, w); };
    qs_status st;
    if ((st = ck(cudaMemcpy(d_steps.p, steps.data(), sizeof(StepDesc) * steps.size(), cudaMemcpyHostToDevice), "upload")) != QS_OK) return st;
    if (!echo.empty()) {
        if ((st = ck(cudaMemcpy(d_echo.p, echo.data(), sizeof(StepDesc) * echo.size(), cudaMemcpyHostToDevice), "upload")) != QS_OK) return st;
        if ((st = ck(cudaMemcpy(d_echom.p, echo_m.data(), sizeof(cplx<R>) * echo_m.size(), cudaMemcpyHostToDevice), "upload")) != QS_OK) return st;
    }
    if ((st = ck(cudaMemcpy(d_x0.p, g.x0, sizeof(uint64_t) * count, cudaMemcpyHostToDevice), "upload")) != QS_OK) return st;
    if ((st = ck(cudaMemsetAsync(d_st.p, 0, sizeof(cplx<R>) * N * count, sm), "memset")) != QS_OK) return st;
    if ((st = ck(cudaMemsetAsync(d_stats.p, 0, sizeof(uint64_t) * 4 * count, sm), "memset")) != QS_OK) return st;
    cplx<R> *states = static_cast<cplx<R> *>(d_st.p);
    k_init<R><<<grid_for(count), THREADS, 0, sm>>>(states, n, count, static_cast<const uint64_t *>(d_x0.p));
    // flip threshold floor(p 2^32) in double, clamped
    double t = std::floor(nz.p * 4294967296.0);
    t = std::min(std::max(t, 0.0), 4294967295.0);
    const uint32_t thr = uint32_t(t);
    const uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
    if (m > 0) {
        k_noise<R><<<grid_for(uint64_t(count) * m), THREADS, 0, sm>>>(
            static_cast<const StepDesc *>(d_steps.p), m, n, g.first, count, k0, k1, nz.sigma, thr, nz.mode, nz.every,
            static_cast<cplx<R> *>(d_mtab.p), static_cast<uint64_t *>(d_ftab.p),
            reinterpret_cast<unsigned long long *>(d_stats.p));
        k_lists<<<(m + 7) / 8, 256, 0, sm>>>(static_cast<const uint64_t *>(d_ftab.p), m, count,
                                             static_cast<uint32_t *>(d_lists.p), static_cast<uint32_t *>(d_lens.p));
    }
    if ((st = ck(cudaGetLastError(), "trajectory launch")) != QS_OK) return st;
    if (fused) {
        // fused passes over all trajectories with per-trajectory op records
        std::vector<HostOp> fops;
        traj_ops(ops, g.metric == QS_TRAJ_FIDELITY, fops);
        if ((st = ck(cudaDeviceSynchronize(), "trajectory noise")) != QS_OK) return st;
        int depth = max_ops;
        if (depth <= 0) {
            st = tune_depth(n, fops, count, m, static_cast<const float2 *>(d_mtab.p),
                            static_cast<const uint64_t *>(d_ftab.p), &depth);
            if (st != QS_OK) return st;
        }
        TrajPlan *tp = nullptr;
        if ((st = traj_plan_build(n, fops, depth, &tp)) != QS_OK) return st;
        const std::vector<TrajOpMeta> &metas = traj_plan_metas(tp);
        DevBuf d_fb, d_meta, d_recs;
        if (d_fb.alloc(sizeof(uint64_t) * 2 * uint64_t(count) * (m + 1)) != cudaSuccess ||
            d_meta.alloc(sizeof(TrajOpMeta) * std::max<size_t>(1, metas.size())) != cudaSuccess ||
            d_recs.alloc(sizeof(TrajRec) * uint64_t(count) * std::max<size_t>(1, metas.size())) != cudaSuccess) {
            cudaGetLastError();
            traj_plan_destroy(tp);
            return fail(QS_ENOMEM, "trajectory batch: device allocation failed");
        }
        st = ck(cudaMemcpy(d_meta.p, metas.data(), sizeof(TrajOpMeta) * metas.size(), cudaMemcpyHostToDevice), "upload");
        if (st == QS_OK) {
            // the whole group (frames, op records, every pass, metric) as one
            // captured graph, launched once
            cudaStream_t cs = nullptr;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t e2 = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e2 == cudaSuccess) e2 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e2 == cudaSuccess) {
                k_frames<<<grid_for(count), THREADS, 0, cs>>>(static_cast<const uint64_t *>(d_ftab.p), m, count,
                                                              static_cast<uint64_t *>(d_fb.p));
                k_optab<<<grid_for(uint64_t(count) * metas.size()), THREADS, 0, cs>>>(
                    static_cast<const TrajOpMeta *>(d_meta.p), uint32_t(metas.size()),
                    reinterpret_cast<const float2 *>(d_mtab.p), m, count, static_cast<const uint64_t *>(d_fb.p),
                    static_cast<TrajRec *>(d_recs.p));
                cudaError_t e3 = traj_plan_run(tp, reinterpret_cast<float2 *>(states), count,
                                               static_cast<const TrajRec *>(d_recs.p), cs);
                k_metric_frame<R><<<grid_for(count), THREADS, 0, cs>>>(
                    states, n, count, static_cast<const uint64_t *>(d_x0.p), g.target,
                    g.metric == QS_TRAJ_FIDELITY ? 1 : 0, static_cast<const uint64_t *>(d_fb.p), m,
                    static_cast<double *>(d_metric.p));
                e2 = cudaStreamEndCapture(cs, &graph);
                if (e2 == cudaSuccess && e3 != cudaSuccess) e2 = e3;
            }
            if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(&exec, graph, 0);
            if (e2 == cudaSuccess) e2 = cudaGraphLaunch(exec, cs);
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(cs);
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (cs) cudaStreamDestroy(cs);
            st = ck(e2, "fused trajectories");
        }
        traj_plan_destroy(tp);
        if (st != QS_OK) return st;
        if ((st = ck(cudaMemcpy(metric, d_metric.p, sizeof(double) * count, cudaMemcpyDeviceToHost), "results")) != QS_OK)
            return st;
        if (stats)
            if ((st = ck(cudaMemcpy(stats, d_stats.p, sizeof(uint64_t) * 4 * count, cudaMemcpyDeviceToHost), "results")) != QS_OK)
                return st;
        return QS_OK;
    }
    const StepDesc *dsteps = static_cast<const StepDesc *>(d_steps.p);
    for (int s = 0; s < m; ++s) {
        const int free_bits = n - steps[s].nfixed;
        k_gate<R><<<grid_for((uint64_t(1) << free_bits) * count), THREADS, 0, sm>>>(
            states, n, count, dsteps + s, static_cast<const cplx<R> *>(d_mtab.p), s, m);
        if (thr != 0)
            k_flip<R><<<grid_for(N * std::min<uint64_t>(count, 64)), THREADS, 0, sm>>>(
                states, n, m, s, count, static_cast<const uint64_t *>(d_ftab.p),
                static_cast<const uint32_t *>(d_lists.p), static_cast<const uint32_t *>(d_lens.p));
    }
    const StepDesc *decho = static_cast<const StepDesc *>(d_echo.p);
    for (size_t k = 0; k < echo.size(); ++k) {
        const int free_bits = n - echo[k].nfixed;
        k_gate<R><<<grid_for((uint64_t(1) << free_bits) * count), THREADS, 0, sm>>>(
            states, n, count, decho + k, static_cast<const cplx<R> *>(d_echom.p), int(k), 0);
    }
    k_metric<R><<<grid_for(count), THREADS, 0, sm>>>(states, n, count, static_cast<const uint64_t *>(d_x0.p), g.target,
                                                     g.metric == QS_TRAJ_FIDELITY ? 1 : 0,
                                                     static_cast<double *>(d_metric.p));
    if ((st = ck(cudaGetLastError(), "trajectory launch")) != QS_OK) return st;
    if ((st = ck(cudaMemcpy(metric, d_metric.p, sizeof(double) * count, cudaMemcpyDeviceToHost), "results")) != QS_OK) return st;
    if (stats)
        if ((st = ck(cudaMemcpy(stats, d_stats.p, sizeof(uint64_t) * 4 * count, cudaMemcpyDeviceToHost), "results")) != QS_OK) return st;
    return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_run_trajectories(const qs_traj_group *groups, int n_groups, const qs_noise *noise,
                                         uint64_t seed, qs_dtype dt, const qs_traj_opts *opts, double *metric,
                                         uint64_t *stats) {
    const int fuse_mode = opts ? (opts->no_fusion ? 0 : 1) : 1;
    const int max_ops = opts ? opts->max_ops_per_pass : 0;
    if (!groups || n_groups < 0 || !noise || !metric) return fail(QS_EINVAL, "NULL argument");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    if (!(noise->p >= 0.0 && noise->p <= 1.0) || !(noise->sigma >= 0.0) || !std::isfinite(noise->sigma))
        return fail(QS_EINVAL, "noise: p must be in [0, 1] and sigma finite and >= 0");
    if (noise->mode != QS_NOISE_FLIPS && noise->mode != QS_NOISE_DEPOLARIZING) return fail(QS_EINVAL, "noise: bad mode");
    size_t off = 0;
    for (int k = 0; k < n_groups; ++k) {
        const qs_traj_group &g = groups[k];
        if (g.n < 1 || g.n > 34) return fail(QS_ERANGE, "trajectory group: n out of range [1, 34]");
        if (g.m > 0 && !g.gates) return fail(QS_EINVAL, "trajectory group: gates NULL");
        if (g.count > 0 && !g.x0) return fail(QS_EINVAL, "trajectory group: x0 NULL");
        if (g.metric != QS_TRAJ_FIDELITY && g.metric != QS_TRAJ_PROB) return fail(QS_EINVAL, "trajectory group: bad metric");
        if (g.metric == QS_TRAJ_PROB && (g.target >> g.n)) return fail(QS_ERANGE, "trajectory group: target >= 2^n");
        for (uint32_t i = 0; i < g.count; ++i)
            if (g.x0[i] >> g.n) return fail(QS_ERANGE, "trajectory group: x0 >= 2^n");
        if (g.m > (size_t(1) << 31)) return fail(QS_ERANGE, "trajectory group: too many gates");
        qs_status st = dt == QS_C64 ? run_group<float>(g, *noise, seed, metric + off, stats ? stats + 4 * off : nullptr,
                                                       fuse_mode, max_ops)
                                    : run_group<double>(g, *noise, seed, metric + off, stats ? stats + 4 * off : nullptr,
                                                        fuse_mode, max_ops);
        if (st != QS_OK) return st;
        off += g.count;
    }
    return QS_OK;
}
