// Fused circuit passes.
//
// The paper applies one gate per sweep over the register (Sec. 2.2) and
// parallelises each sweep over independent blocks M_k = S_k phi_k.  A GPU
// sweep is bound by HBM traffic, so consecutive gates are grouped into passes
// that read and write the register once:
//
//  * A pass picks a tile of K index bits: the five lowest bits (the lanes of a
//    warp, so every load and store is a contiguous run of 32 amplitudes) plus
//    H = RB + WB high bits.  One CTA owns one tile (2^K amplitudes) for each
//    assignment of the other n - K bits, which are the block index k of the
//    paper's M_k decomposition generalised to any set of fixed bits.
//  * Each thread keeps 2^RB amplitudes in registers; the RB "register bits"
//    are high tile bits chosen per phase.  Warps are told apart by the WB
//    "warp bits".  A gate whose target is a register bit is applied in
//    registers; one whose target is a lane bit exchanges partners with
//    __shfl_xor_sync; one whose target is a warp bit is preceded by a
//    transpose through shared memory that makes it a register bit.
//  * Diagonal gates (phase shifts, Z, RZ, the Grover oracle) need no tile bit:
//    the multiplier of every amplitude is known from its index.  Control bits
//    need none either: a control on a bit outside the tile is a per-CTA
//    predicate, on a lane or warp bit a per-thread predicate, on a register
//    bit a per-amplitude predicate.
//  * The in-place hazard of Sec. 2.2.1 is avoided as in the paper: the two
//    amplitudes of a pair are always combined by one thread (registers) or by
//    two lanes that exchange their old values before either writes.
//
// The host planner groups gates greedily in order; a later gate may join the
// current pass ahead of a gate that could not, when the two act on disjoint
// qubits (they commute).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>

#include "qs_internal.cuh"

namespace qs {

namespace {

constexpr int LB = 5;          // lane bits
#ifndef QS_MAX_WB
#define QS_MAX_WB 3
#endif
constexpr int MAX_WB = QS_MAX_WB;  // warp bits (2^MAX_WB warps per CTA)
constexpr int MAX_OPS = 120;   // ops per pass (shared-memory op table)
#ifndef QS_RB64
#define QS_RB64 5
#endif
#ifndef QS_WB64
#define QS_WB64 3
#endif
#ifndef QS_RB128
#define QS_RB128 4
#endif
#ifndef QS_FUSED_MINBLOCKS
#define QS_FUSED_MINBLOCKS 2
#endif
constexpr int RB64 = QS_RB64;      // complex64: 2^RB64 amplitudes per thread
constexpr int WB64 = QS_WB64;      // complex64: 2^WB64 warps per CTA
constexpr int RB128 = QS_RB128;    // complex128: 2^RB128 amplitudes per thread
// a layout packs RB + WB slots of 4 bits into 32 bits; a control mask over
// the register index is 8 bits wide
static_assert(RB64 + WB64 <= 8 && RB128 + MAX_WB <= 8, "layout does not fit 32 bits");
static_assert(RB64 <= 5 && RB128 <= 5 && MAX_WB <= 4, "register or warp bits out of range");

enum OpType : uint8_t { OP_REG = 0, OP_LANE = 1, OP_DIAG = 2, OP_XPOSE = 3 };

// Fused-only gate class: an uncontrolled Hadamard applied as the butterfly
// (x + y, x - y); the factors 1/sqrt 2 of all such gates of a pass are folded
// into one scale at the store (exact when their number is even, so a complex64
// register does not drift by the rounding of 1/sqrt 2 once per gate).
constexpr int GC_HB = 8;

template <typename R>
struct alignas(16) FOp {
    uint8_t type;      // OpType
    uint8_t cls;       // GateClass (OP_REG / OP_LANE) or GC_HB
    uint8_t tsel;      // OP_DIAG target: 0 register slot, 1 thread bit, 2 outer bit
    uint8_t tpos;      // register slot / lane bit / thread bit / outer bit
    uint8_t rmask, rval;   // control condition over the register index
    uint16_t pad0;
    uint32_t lay;          // OP_XPOSE: new layout, 4 bits per slot (register slots, then warp bits)
    uint16_t tmask, tval;  // control condition over the thread index (lane | warp << 5)
    uint64_t omask, oval;  // control condition over the index bits outside the tile
    R u[8];                // matrix, or (d0, d1) for OP_DIAG
};

template <typename R>
struct PassDesc {
    const FOp<R> *ops;     // device op table of this pass
    uint64_t tiles;        // 2^(n - K)
    int32_t K;             // tile bits
    int32_t WB;            // warp bits
    int32_t nops;
    int32_t has_xpose;
    uint32_t lay0;         // initial layout, 4 bits per slot
    R scale;               // folded Hadamard factor applied at the store (1: none)
    uint8_t tile_pos[24];  // all tile bit positions, ascending (the first five are 0..4)
    uint8_t hpos[16];      // global position of high tile bit i (= tile_pos[5 + i])
};

__device__ __forceinline__ int slot_of(uint32_t lay, int s) { return int((lay >> (4 * s)) & 15u); }

// Global offset of register index j under layout `lay`.
template <int RB>
__device__ __forceinline__ uint64_t reg_offset(int j, uint32_t lay, const uint8_t *hpos) {
    uint64_t o = 0;
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if ((j >> r) & 1) o |= uint64_t(1) << hpos[slot_of(lay, r)];
    return o;
}

// Global offset of this thread's lane and warp bits under layout `lay`.
template <int RB>
__device__ __forceinline__ uint64_t thread_offset(uint32_t lane, uint32_t warp, int WB, uint32_t lay,
                                                  const uint8_t *hpos) {
    uint64_t o = lane;
#pragma unroll
    for (int w = 0; w < MAX_WB; ++w)
        if (w < WB && ((warp >> w) & 1)) o |= uint64_t(1) << hpos[slot_of(lay, RB + w)];
    return o;
}

// Tile-local (shared memory) index of register index j of this thread.
template <int RB>
__device__ __forceinline__ uint32_t local_index(int j, uint32_t lane, uint32_t warp, int WB, uint32_t lay) {
    uint32_t o = lane;
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if ((j >> r) & 1) o |= 1u << (LB + slot_of(lay, r));
#pragma unroll
    for (int w = 0; w < MAX_WB; ++w)
        if (w < WB && ((warp >> w) & 1)) o |= 1u << (LB + slot_of(lay, RB + w));
    return o;
}

// Matrix of an op, read from shared memory with vector loads.
template <typename R> struct Mat4 { cplx<R> u00, u01, u10, u11; };

__device__ __forceinline__ Mat4<double> load_mat(const FOp<double> &op) {
    const double2 *p = reinterpret_cast<const double2 *>(&op.u[0]);
    return {p[0], p[1], p[2], p[3]};
}

template <typename R>
__device__ __forceinline__ cplx<R> sel(bool p, cplx<R> a, cplx<R> b) { return mk<R>(p ? a.x : b.x, p ? a.y : b.y); }

// General 2x2 on register slot T.  With PRED, pairs whose register bits fail
// the control condition keep their values (select, no branch); without, every
// pair is updated (the common case: no control on a register bit).
template <typename R, int RB, int T, bool PRED>
__device__ __forceinline__ void reg_gen(cplx<R> (&v)[1 << RB], const Mat4<R> &m, int rm, int rv) {
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        const cplx<R> x = v[j], y = v[j1];
        if (PRED) {
            const bool p = (j & rm) == rv;
            v[j] = sel<R>(p, cmad2<R>(m.u00, x, m.u01, y), x);
            v[j1] = sel<R>(p, cmad2<R>(m.u10, x, m.u11, y), y);
        } else {
            v[j] = cmad2<R>(m.u00, x, m.u01, y);
            v[j1] = cmad2<R>(m.u10, x, m.u11, y);
        }
    }
}

// Exchange of the pair (X, C-NOT) on register slot T; without PRED it is a
// renaming of registers.
template <typename R, int RB, int T, bool PRED>
__device__ __forceinline__ void reg_x(cplx<R> (&v)[1 << RB], int rm, int rv) {
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        const cplx<R> x = v[j], y = v[j1];
        if (PRED) {
            const bool p = (j & rm) == rv;
            v[j] = sel<R>(p, y, x);
            v[j1] = sel<R>(p, x, y);
        } else {
            v[j] = y;
            v[j1] = x;
        }
    }
}

// Uncontrolled Hadamard butterfly on register slot T (scale folded).
template <typename R, int RB, int T>
__device__ __forceinline__ void reg_hb(cplx<R> (&v)[1 << RB]) {
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        const cplx<R> x = v[j], y = v[j1];
        v[j] = mk<R>(x.x + y.x, x.y + y.y);
        v[j1] = mk<R>(x.x - y.x, x.y - y.y);
    }
}

// Diagonal gate whose target is register slot T: d0 on amplitudes with bit T
// clear, d1 on those with it set; DK = 1: d0 == 1 (skip), DK = 2: d1 == 1.
template <typename R, int RB, int T>
__device__ __forceinline__ void reg_diag(cplx<R> (&v)[1 << RB], int dk, cplx<R> d0, cplx<R> d1, int rm, int rv) {
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
        const bool hi = (j >> T) & 1;
        if ((hi && dk == 2) || (!hi && dk == 1)) continue;
        v[j] = sel<R>((j & rm) == rv, cmul<R>(hi ? d1 : d0, v[j]), v[j]);
    }
}

template <typename R, int RB, int T>
__device__ __forceinline__ void reg_op(cplx<R> (&v)[1 << RB], int cls, int rm, int rv, const FOp<R> &op) {
    if (cls == GC_HB) reg_hb<R, RB, T>(v);
    else if (cls == GC_X) {
        if (rm) reg_x<R, RB, T, true>(v, rm, rv);
        else reg_x<R, RB, T, false>(v, rm, rv);
    } else {
        const Mat4<R> m = load_mat(op);
        if (rm) reg_gen<R, RB, T, true>(v, m, rm, rv);
        else reg_gen<R, RB, T, false>(v, m, rm, rv);
    }
}

template <typename R>
__device__ __forceinline__ cplx<R> shfl(cplx<R> a, int m) {
    return mk<R>(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
}

// One CTA runs tiles blockIdx.x, blockIdx.x + gridDim.x, ... (persistent).
// Shared memory: the transpose buffer (2^K amplitudes, only when the pass
// transposes), then the op table of the pass.
template <typename R, int RB>
__global__ void __launch_bounds__(32 << QS_MAX_WB, 1) k_fused(cplx<R> *__restrict__ a, const __grid_constant__ PassDesc<R> P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int NA = 1 << RB;
    const int K = P.K, WB = P.WB, nops = P.nops;
    cplx<R> *sm = reinterpret_cast<cplx<R> *>(smraw);
    FOp<R> *sops = reinterpret_cast<FOp<R> *>(smraw + (P.has_xpose ? (size_t(sizeof(cplx<R>)) << K) : 0));
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.ops);
        uint4 *dst = reinterpret_cast<uint4 *>(sops);
        const int words = nops * int(sizeof(FOp<R>) / 16);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
        __syncthreads();
    }
    const uint32_t tl = threadIdx.x;            // lane | warp << 5
    const uint32_t lane = tl & 31u, warp = tl >> 5;

    for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
        // tile base: the tile index with zeros inserted at every tile position
        uint64_t base = tile;
        for (int k = 0; k < K; ++k) {
            const uint64_t low = (uint64_t(1) << P.tile_pos[k]) - 1;
            base = ((base & ~low) << 1) | (base & low);
        }
        uint32_t lay = P.lay0;
        cplx<R> v[NA];
        {
            const cplx<R> *src = a + (base | thread_offset<RB>(lane, warp, WB, lay, P.hpos));
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = src[reg_offset<RB>(j, lay, P.hpos)];
        }
        for (int k = 0; k < nops; ++k) {
            const FOp<R> &op = sops[k];
            const uint4 hd = *reinterpret_cast<const uint4 *>(&op);
            const int type = hd.x & 0xff, cls = (hd.x >> 8) & 0xff, tsel = (hd.x >> 16) & 0xff,
                      tpos = hd.x >> 24;
            const int rm = hd.y & 0xff, rv = (hd.y >> 8) & 0xff;
            const uint32_t tm = hd.w & 0xffff, tv = hd.w >> 16;
            if (type == OP_XPOSE) {
                // write with the current layout, read back with the new one
#pragma unroll
                for (int j = 0; j < NA; ++j) sm[local_index<RB>(j, lane, warp, WB, lay)] = v[j];
                __syncthreads();
                lay = hd.z;
#pragma unroll
                for (int j = 0; j < NA; ++j) v[j] = sm[local_index<RB>(j, lane, warp, WB, lay)];
                __syncthreads();
                continue;
            }
            const bool ok = ((tl & tm) == tv) && ((base & op.omask) == op.oval);
            if (type == OP_REG) {
                if (!ok) continue;
                if (tpos == 0) reg_op<R, RB, 0>(v, cls, rm, rv, op);
                else if (tpos == 1) reg_op<R, RB, 1>(v, cls, rm, rv, op);
                else if (tpos == 2) reg_op<R, RB, 2>(v, cls, rm, rv, op);
                else if (tpos == 3) reg_op<R, RB, 3>(v, cls, rm, rv, op);
                else reg_op<R, RB, (RB > 4 ? 4 : 0)>(v, cls, rm, rv, op);
            } else if (type == OP_LANE) {
                // partners sit in the lane that differs in bit tpos; both lanes
                // exchange their old values before either writes
                const int m = 1 << tpos;
                const bool hi = (lane >> tpos) & 1;
                if (cls == GC_HB) {
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const cplx<R> o = shfl<R>(v[j], m);
                        v[j] = hi ? mk<R>(o.x - v[j].x, o.y - v[j].y) : mk<R>(v[j].x + o.x, v[j].y + o.y);
                    }
                } else if (cls == GC_X) {
                    if (rm == 0) {
#pragma unroll
                        for (int j = 0; j < NA; ++j) {
                            const cplx<R> o = shfl<R>(v[j], m);
                            v[j] = sel<R>(ok, o, v[j]);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NA; ++j) {
                            if ((j & rm) != rv) continue;   // uniform across the warp
                            const cplx<R> o = shfl<R>(v[j], m);
                            v[j] = sel<R>(ok, o, v[j]);
                        }
                    }
                } else {
                    const Mat4<R> mt = load_mat(op);
                    // coefficients on my own amplitude and on the partner's
                    const cplx<R> cs = hi ? mt.u11 : mt.u00, co = hi ? mt.u10 : mt.u01;
                    if (rm == 0 && __all_sync(0xffffffffu, ok)) {
#pragma unroll
                        for (int j = 0; j < NA; ++j) {
                            const cplx<R> o = shfl<R>(v[j], m);
                            v[j] = cmad2<R>(cs, v[j], co, o);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NA; ++j) {
                            if ((j & rm) != rv) continue;   // uniform across the warp
                            const cplx<R> o = shfl<R>(v[j], m);
                            v[j] = sel<R>(ok, cmad2<R>(cs, v[j], co, o), v[j]);
                        }
                    }
                }
            } else {  // OP_DIAG
                if (!ok) continue;
                const Mat4<R> mt = load_mat(op);   // (d0, d1) in the first two entries
                const cplx<R> d0 = mt.u00, d1 = mt.u01;
                if (tsel == 0) {
                    if (tpos == 0) reg_diag<R, RB, 0>(v, cls, d0, d1, rm, rv);
                    else if (tpos == 1) reg_diag<R, RB, 1>(v, cls, d0, d1, rm, rv);
                    else if (tpos == 2) reg_diag<R, RB, 2>(v, cls, d0, d1, rm, rv);
                    else if (tpos == 3) reg_diag<R, RB, 3>(v, cls, d0, d1, rm, rv);
                    else reg_diag<R, RB, (RB > 4 ? 4 : 0)>(v, cls, d0, d1, rm, rv);
                } else {
                    const uint64_t word = tsel == 1 ? uint64_t(tl) : base;
                    const cplx<R> d = ((word >> tpos) & 1) ? d1 : d0;
#pragma unroll
                    for (int j = 0; j < NA; ++j) v[j] = sel<R>((j & rm) == rv, cmul<R>(d, v[j]), v[j]);
                }
            }
        }
        if (P.scale != R(1)) {
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = mk<R>(v[j].x * P.scale, v[j].y * P.scale);
        }
        // store with the final layout
        cplx<R> *dst = a + (base | thread_offset<RB>(lane, warp, WB, lay, P.hpos));
#pragma unroll
        for (int j = 0; j < NA; ++j) dst[reg_offset<RB>(j, lay, P.hpos)] = v[j];
    }
}

// ---------------------------------------------------------------------------
// Complex64 pass kernel.
//
// Each thread keeps 32 amplitudes (register index j, 5 register bits) as
// (re, im) pairs and updates them with scalar FFMA (packing two amplitudes
// per FFMA2 costs more in register moves than it saves in issue slots).
//
// Exchanges (X, C-NOT) on a register slot whose condition is uniform across
// the warp move no data: each thread keeps a mask xm such that physical
// register index p holds the amplitude of logical register index p ^ xm.
// Later gates read their matrix in swapped roles (X U X) where xm has their
// slot, control predicates and diagonal selectors use the logical index
// p ^ xm, and transposes and the store put physical p at the place of p ^ xm.
//
// Every layout-dependent offset (global offsets of register indices and warp
// bits at the load and at the store, the read pattern of each transpose) is
// computed on the host when the plan is built, so the kernel does no bit
// scattering.
// ---------------------------------------------------------------------------

// One op of the complex64 kernel (112 bytes).
struct alignas(16) POp {
    uint8_t type, cls, tsel, tpos;
    uint8_t rmask, rval;
    uint8_t fast;          // state-vector fast paths: 1 uncontrolled general gate on a register slot,
                           // 2 X deferred into the index mask, 3 uncontrolled general gate on a lane bit,
                           // 4 / 5 as 1 / 3 for a real matrix (RY, U_R, ...), 6 / 7 an uncontrolled
                           // Hadamard butterfly on a register slot / lane bit
    uint8_t pad0;
    uint32_t pad1;
    uint16_t tmask, tval;
    uint64_t omask, oval;
    // OP_REG / OP_LANE: u00, u01, u10, u11 in c[0..3]; OP_DIAG: d0, d1 in c[0..1]
    // OP_XPOSE: 32 uint16 read offsets (old tile order) of the new register
    //           indices in c[0..7], then the old tile-order bit of each new
    //           warp bit (bytes) in c[8..9]
    float2 c[10];
};
static_assert(sizeof(POp) == 112, "POp layout");

struct PassC64 {
    const POp *ops;
    uint64_t tiles;
    int32_t K, WB, nops, has_xpose;
    int32_t has_hb, pad_hb;            // an op takes a Hadamard fast path (fast 6 or 7)
    float scale;
    int32_t n;                         // qubits (trajectory mode: state stride 2^n)
    // trajectory mode: per-(trajectory, op) records; trajectory b's record of
    // op k of this pass is recs[b * rec_stride + rec_off + k]
    const TrajRec *recs;
    uint64_t tiles_per_traj;
    uint32_t rec_stride, rec_off;
    uint8_t tile_pos[24];
    uint64_t ld_reg[32], ld_warp[4];   // global offsets of register index j / warp bit w (first layout)
    uint64_t st_reg[32], st_warp[4];   // the same for the last layout (store)
};

__device__ __forceinline__ bool lpred(int j, uint32_t xm, int rm, int rv) {
    return ((uint32_t(j) ^ xm) & uint32_t(rm)) == uint32_t(rv);
}

// (x, y) <- (u00 x + u01 y, u10 x + u11 y) in place.  The four output chains
// run in lockstep and each ends on the input it replaces (x.re, x.im, y.re,
// y.im last read by the chain that overwrites it), so the results land in
// the registers of the inputs: no register moves where the op dispatch
// branches join again.
__device__ __forceinline__ void pair_inplace(float2 &x, float2 &y, const Mat4<float> &m) {
    float A = m.u01.x * y.y, B = -m.u01.y * y.y, C = m.u10.x * x.y, D = -m.u10.y * x.y;
    A = fmaf(m.u01.y, y.x, A);    // nx.im: u01.re y.im + u01.im y.re
    B = fmaf(m.u01.x, y.x, B);    // nx.re: u01.re y.re - u01.im y.im
    C = fmaf(m.u10.y, x.x, C);    // ny.im: u10.re x.im + u10.im x.re
    D = fmaf(m.u10.x, x.x, D);    // ny.re: u10.re x.re - u10.im x.im
    B = fmaf(-m.u00.y, x.y, B);
    A = fmaf(m.u00.y, x.x, A);
    D = fmaf(-m.u11.y, y.y, D);
    C = fmaf(m.u11.y, y.x, C);
    x.x = fmaf(m.u00.x, x.x, B);
    x.y = fmaf(m.u00.x, x.y, A);
    y.x = fmaf(m.u11.x, y.x, D);
    y.y = fmaf(m.u11.x, y.y, C);
}

// (x, y) <- (a x + b y, c x + d y) for a real matrix [[a, b], [c, d]]:
// four multiply-adds per amplitude instead of eight
template <int T, int NA>
__device__ __forceinline__ void s_real(float2 (&v)[NA], float a, float b, float c, float d, uint32_t xm) {
    if ((xm >> T) & 1) {   // deferred exchange on this slot: X U X
        float t = a; a = d; d = t;
        t = b; b = c; c = t;
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        const float2 x = v[j], y = v[j1];
        v[j] = make_float2(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y));
        v[j1] = make_float2(fmaf(c, x.x, d * y.x), fmaf(c, x.y, d * y.y));
    }
}

template <int T, bool PRED, int NA>
__device__ __forceinline__ void s_gen(float2 (&v)[NA], Mat4<float> m, uint32_t xm, int rm, int rv) {
    if ((xm >> T) & 1) {
        float2 t = m.u00; m.u00 = m.u11; m.u11 = t;
        t = m.u01; m.u01 = m.u10; m.u10 = t;
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        if (PRED) {
            const float2 x = v[j], y = v[j1];
            const float2 nx = cmad2<float>(m.u00, x, m.u01, y), ny = cmad2<float>(m.u10, x, m.u11, y);
            const bool p = lpred(j, xm, rm, rv);
            v[j] = p ? nx : x;
            v[j1] = p ? ny : y;
        } else {
            pair_inplace(v[j], v[j1], m);
        }
    }
}

template <int T, int NA>
__device__ __forceinline__ void s_xdata(float2 (&v)[NA], uint32_t xm, int rm, int rv, bool ok) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        const bool p = ok && lpred(j, xm, rm, rv);
        const float2 x = v[j], y = v[j1];
        v[j] = p ? y : x;
        v[j1] = p ? x : y;
    }
}

template <int T, int NA>
__device__ __forceinline__ void s_hb(float2 (&v)[NA], uint32_t xm) {
    // the deferred-exchange bit of the slot is the same across the warp: a
    // branch, not a select per amplitude
    // In place: the difference overwrites one input, and the sum is formed
    // from it as 2 x - (x - y) (one rounding of the exact 2 x minus the
    // rounded difference), so each output lands in an input's register and
    // no register copies are needed where the op dispatch rejoins.
    if ((xm >> T) & 1) {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if ((j >> T) & 1) continue;
            const int j1 = j | (1 << T);
            v[j].x = v[j1].x - v[j].x;
            v[j].y = v[j1].y - v[j].y;
            v[j1].x = fmaf(2.f, v[j1].x, -v[j].x);
            v[j1].y = fmaf(2.f, v[j1].y, -v[j].y);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if ((j >> T) & 1) continue;
            const int j1 = j | (1 << T);
            v[j1].x = v[j].x - v[j1].x;
            v[j1].y = v[j].y - v[j1].y;
            v[j].x = fmaf(2.f, v[j].x, -v[j1].x);
            v[j].y = fmaf(2.f, v[j].y, -v[j1].y);
        }
    }
}

// LEAN: the per-register entry chosen at compile time after a warp-uniform
// swap, and no control test without controls (the state-vector passes);
// else the compact form (one loop, a select and a test per register), which
// the trajectory passes, whose diagonals mostly carry controls, run faster
// (4096 trajectories: 0.293 against 0.306 s)
template <int T, int NA, bool LEAN>
__device__ __forceinline__ void s_diag(float2 (&v)[NA], float2 d0, float2 d1, uint32_t xm, int rm, int rv) {
    if (!LEAN) {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const uint32_t l = uint32_t(j) ^ xm;
            const float2 d = ((l >> T) & 1) ? d1 : d0;
            if ((l & uint32_t(rm)) == uint32_t(rv)) v[j] = cmul<float>(d, v[j]);
        }
        return;
    }
    // register j holds logical index j ^ xm: its entry is d0 or d1 by bit T
    // of j, the two swapped where xm has bit T (the same across the warp, so
    // a branch here and a compile-time choice per register)
    if ((xm >> T) & 1) {
        const float2 t = d0;
        d0 = d1;
        d1 = t;
    }
    if (rm == 0) {
#pragma unroll
        for (int j = 0; j < NA; ++j) v[j] = cmul<float>(((j >> T) & 1) ? d1 : d0, v[j]);
    } else {
#pragma unroll
        for (int j = 0; j < NA; ++j)
            if (lpred(j, xm, rm, rv)) v[j] = cmul<float>(((j >> T) & 1) ? d1 : d0, v[j]);
    }
}

// Diagonal on register slot T with one entry exactly 1: only the amplitudes
// whose physical bit T equals BIT change (the caller turns the logical side
// into the physical one with bit T of xm).
template <int T, int NA, int BIT>
__device__ __forceinline__ void s_diag_half(float2 (&v)[NA], float2 d, uint32_t xm, int rm, int rv) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if (((j >> T) & 1) != BIT) continue;
        if (lpred(j, xm, rm, rv)) v[j] = cmul<float>(d, v[j]);
    }
}

// d0 == 1 exactly: the logical-one side changes; d1 == 1: the logical-zero
// side; otherwise both (s_diag).
template <int T, int NA, bool LEAN>
__device__ __forceinline__ void s_diag_any(float2 (&v)[NA], float2 d0, float2 d1, uint32_t xm, int rm, int rv) {
    const bool id0 = d0.x == 1.f && d0.y == 0.f, id1 = d1.x == 1.f && d1.y == 0.f;
    const uint32_t xt = (xm >> T) & 1u;
    if (id0) {
        if (xt) s_diag_half<T, NA, 0>(v, d1, xm, rm, rv);
        else s_diag_half<T, NA, 1>(v, d1, xm, rm, rv);
    } else if (id1) {
        if (xt) s_diag_half<T, NA, 1>(v, d0, xm, rm, rv);
        else s_diag_half<T, NA, 0>(v, d0, xm, rm, rv);
    } else {
        s_diag<T, NA, LEAN>(v, d0, d1, xm, rm, rv);
    }
}

template <int T, int NA>
__device__ __forceinline__ void s_reg_op(float2 (&v)[NA], int cls, uint32_t &xm, bool ok, int rm, int rv, bool lanectl,
                                         const Mat4<float> &m) {
    if (cls == GC_X) {
        if (rm == 0 && !lanectl) { xm ^= ok ? (1u << T) : 0u; return; }
        s_xdata<T, NA>(v, xm, rm, rv, ok);
        return;
    }
    if (!ok) return;
    if (cls == GC_HB) { s_hb<T, NA>(v, xm); return; }
    if (rm) s_gen<T, true, NA>(v, m, xm, rm, rv);
    else s_gen<T, false, NA>(v, m, xm, rm, rv);
}

// TRAJ: trajectory mode.  Tiles run over (trajectory, tile of its state);
// each op takes its matrix and the XOR of its control values from the
// trajectory's records, loaded into shared memory when the tile's trajectory
// changes.
// HBF: the pass has uncontrolled Hadamard butterflies with fast paths (fast
// codes 6 and 7).  Passes without them run an instantiation without those
// branches, whose code and register allocation are those of the plain
// dispatch (the random-circuit passes measured 1.2% slower with them).
template <bool TRAJ, bool HBF>
__global__ void __launch_bounds__(32 << QS_WB64, QS_FUSED_MINBLOCKS) k_fused_c64(float2 *__restrict__ a0,
                                                                       const __grid_constant__ PassC64 P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int K = P.K, WB = P.WB, nops = P.nops;
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    POp *sops = reinterpret_cast<POp *>(smraw + (P.has_xpose ? (size_t(8) << K) : 0));
    TrajRec *srec = reinterpret_cast<TrajRec *>(reinterpret_cast<unsigned char *>(sops) + size_t(nops) * sizeof(POp));
    uint64_t cur_b = ~uint64_t(0);
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.ops);
        uint4 *dst = reinterpret_cast<uint4 *>(sops);
        const int words = nops * int(sizeof(POp) / 16);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
        __syncthreads();
    }
    const uint32_t tl = threadIdx.x;
    const uint32_t lane = tl & 31u, warp = tl >> 5;
    const int stride = 32 << WB;
    uint64_t ld_t = lane, st_t = lane;
#pragma unroll
    for (int w = 0; w < WB64; ++w)
        if ((warp >> w) & 1) { ld_t += P.ld_warp[w]; st_t += P.st_warp[w]; }

    // trajectory mode walks a contiguous range of tiles per CTA, so that the
    // tiles of one trajectory share one load of its op records
    uint64_t t_begin = blockIdx.x, t_end = P.tiles, t_step = gridDim.x;
    if (TRAJ) {
        const uint64_t per = (P.tiles + gridDim.x - 1) / gridDim.x;
        t_begin = uint64_t(blockIdx.x) * per;
        t_end = t_begin + per < P.tiles ? t_begin + per : P.tiles;
        t_step = 1;
    }
    for (uint64_t tile = t_begin; tile < t_end; tile += t_step) {
        float2 *a = a0;
        uint64_t base = tile;
        if (TRAJ) {
            const uint64_t b = tile / P.tiles_per_traj;
            base = tile - b * P.tiles_per_traj;
            a = a0 + (b << P.n);
            if (b != cur_b) {   // this trajectory's op records
                __syncthreads();
                const uint4 *src = reinterpret_cast<const uint4 *>(P.recs + b * P.rec_stride + P.rec_off);
                uint4 *dst = reinterpret_cast<uint4 *>(srec);
                const int words = nops * int(sizeof(TrajRec) / 16);
                for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
                __syncthreads();
                cur_b = b;
            }
        }
        for (int k = 0; k < K; ++k) {
            const uint64_t low = (uint64_t(1) << P.tile_pos[k]) - 1;
            base = ((base & ~low) << 1) | (base & low);
        }
        uint32_t xm = 0;
        constexpr int NA = 1 << RB64;
        float2 v[NA];
        {
            const float2 *src = a + (base | ld_t);
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = src[P.ld_reg[j]];
        }
        for (int k = 0; k < nops; ++k) {
            const POp &op = sops[k];
            const uint4 *q = reinterpret_cast<const uint4 *>(&op);
            const uint4 hd = q[0];
            // trajectory mode: an uncontrolled op's matrix is the trajectory's
            // record; the deferred C-NOT path is skipped there (its control
            // values change with the trajectory's Pauli frame)
            int fast = int((hd.y >> 16) & 0xff);
            if (TRAJ && (fast == 2 || fast >= 6)) fast = 0;
            if (TRAJ && fast >= 4) fast = fast == 4 ? 1 : 3;   // a trajectory's matrix need not be real
            if (fast) {
                // the common cases without the general dispatch: no predicate
                // work and no class tests
                const int tp = hd.x >> 24;
                if (fast == 2) {
                    const uint4 oc = q[1];
                    const uint64_t omask = uint64_t(oc.x) | (uint64_t(oc.y) << 32);
                    const uint64_t oval = uint64_t(oc.z) | (uint64_t(oc.w) << 32);
                    const bool ok = ((tl & (hd.w & 0xffff)) == (hd.w >> 16)) && ((base & omask) == oval);
                    xm ^= ok ? (1u << tp) : 0u;
                    continue;
                }
                if (HBF && fast == 6) {   // Hadamard butterfly on a register slot (factor folded into the pass scale)
                    if (tp == 0) s_hb<0, NA>(v, xm);
                    else if (tp == 1) s_hb<1, NA>(v, xm);
                    else if (tp == 2) s_hb<2, NA>(v, xm);
                    else if (tp == 3) s_hb<3, NA>(v, xm);
                    else s_hb<(RB64 > 4 ? 4 : 0), NA>(v, xm);
                    continue;
                }
                if (HBF && fast == 7) {   // Hadamard butterfly on a lane bit: low lane v + o, high lane o - v
                    const int m = 1 << tp;
                    const float sg = ((lane >> tp) & 1) ? -1.f : 1.f;
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const float2 o = shfl<float>(v[j], m);
                        v[j] = make_float2(fmaf(sg, v[j].x, o.x), fmaf(sg, v[j].y, o.y));
                    }
                    continue;
                }
                const float4 *cs4 = TRAJ ? reinterpret_cast<const float4 *>(srec[k].u) : reinterpret_cast<const float4 *>(q) + 2;
                const float4 f0 = cs4[0], f1 = cs4[1];
                const Mat4<float> mf = {make_float2(f0.x, f0.y), make_float2(f0.z, f0.w), make_float2(f1.x, f1.y),
                                        make_float2(f1.z, f1.w)};
                if (fast == 1) {
                    if (tp == 0) s_gen<0, false, NA>(v, mf, xm, 0, 0);
                    else if (tp == 1) s_gen<1, false, NA>(v, mf, xm, 0, 0);
                    else if (tp == 2) s_gen<2, false, NA>(v, mf, xm, 0, 0);
                    else if (tp == 3) s_gen<3, false, NA>(v, mf, xm, 0, 0);
                    else s_gen<(RB64 > 4 ? 4 : 0), false, NA>(v, mf, xm, 0, 0);
                } else if (fast == 4) {
                    const float a = f0.x, b = f0.z, c = f1.x, d = f1.z;
                    if (tp == 0) s_real<0, NA>(v, a, b, c, d, xm);
                    else if (tp == 1) s_real<1, NA>(v, a, b, c, d, xm);
                    else if (tp == 2) s_real<2, NA>(v, a, b, c, d, xm);
                    else if (tp == 3) s_real<3, NA>(v, a, b, c, d, xm);
                    else s_real<(RB64 > 4 ? 4 : 0), NA>(v, a, b, c, d, xm);
                } else if (fast == 5) {
                    const int m = 1 << tp;
                    const bool hi = (lane >> tp) & 1;
                    const float cs = hi ? f1.z : f0.x, co = hi ? f1.x : f0.z;
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const float2 o = shfl<float>(v[j], m);
                        v[j] = make_float2(fmaf(cs, v[j].x, co * o.x), fmaf(cs, v[j].y, co * o.y));
                    }
                } else {
                    const int m = 1 << tp;
                    const bool hi = (lane >> tp) & 1;
                    const float2 cs = hi ? mf.u11 : mf.u00, co = hi ? mf.u10 : mf.u01;
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const float2 o = shfl<float>(v[j], m);
                        v[j] = cmad2<float>(cs, v[j], co, o);
                    }
                }
                continue;
            }
            const uint4 oc = q[1];
            const int type = hd.x & 0xff, cls = (hd.x >> 8) & 0xff, tsel = (hd.x >> 16) & 0xff,
                      tpos = hd.x >> 24;
            const int rm = hd.y & 0xff, rv = (hd.y >> 8) & 0xff;
            const uint32_t tm = hd.w & 0xffff, tv = hd.w >> 16;
            if (type == OP_XPOSE) {
                const uint32_t cw = (xm * uint32_t(stride)) | tl;
#pragma unroll
                for (int j = 0; j < NA; ++j) sm[uint32_t(j * stride) ^ cw] = v[j];
                const uint4 *rt = reinterpret_cast<const uint4 *>(op.c);
                uint32_t rd[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 w4 = rt[q];
                    rd[4 * q] = w4.x; rd[4 * q + 1] = w4.y; rd[4 * q + 2] = w4.z; rd[4 * q + 3] = w4.w;
                }
                const uint4 ow4 = rt[4];
                uint32_t cth = lane;
#pragma unroll
                for (int w = 0; w < WB64; ++w)
                    if (w < WB && ((warp >> w) & 1)) cth |= 1u << ((ow4.x >> (8 * w)) & 0xff);
                __syncthreads();
                xm = 0;
#pragma unroll
                for (int j = 0; j < NA; ++j) v[j] = sm[((rd[j >> 1] >> (16 * (j & 1))) & 0xffff) ^ cth];
                __syncthreads();
                continue;
            }
            const uint64_t omask = uint64_t(oc.x) | (uint64_t(oc.y) << 32);
            uint64_t oval = uint64_t(oc.z) | (uint64_t(oc.w) << 32);
            float4 c0 = reinterpret_cast<const float4 *>(q)[2], c1 = reinterpret_cast<const float4 *>(q)[3];
            uint32_t tvv = tv;
            int rv2 = rv;
            if (TRAJ) {
                const TrajRec &tr = srec[k];
                c0 = reinterpret_cast<const float4 *>(tr.u)[0];
                c1 = reinterpret_cast<const float4 *>(tr.u)[1];
                oval ^= tr.ovx;
                tvv ^= tr.tvx;
                rv2 ^= tr.rvx;
            }
            const bool ok = ((tl & tm) == tvv) && ((base & omask) == oval);
            const Mat4<float> mt = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                                    make_float2(c1.z, c1.w)};
            if (type == OP_REG) {
                const bool lc = (tm & 31u) != 0;
                if (tpos == 0) s_reg_op<0, NA>(v, cls, xm, ok, rm, rv2, lc, mt);
                else if (tpos == 1) s_reg_op<1, NA>(v, cls, xm, ok, rm, rv2, lc, mt);
                else if (tpos == 2) s_reg_op<2, NA>(v, cls, xm, ok, rm, rv2, lc, mt);
                else if (tpos == 3) s_reg_op<3, NA>(v, cls, xm, ok, rm, rv2, lc, mt);
                else s_reg_op<(RB64 > 4 ? 4 : 0), NA>(v, cls, xm, ok, rm, rv2, lc, mt);
            } else if (type == OP_LANE) {
                const int m = 1 << tpos;
                const bool hi = (lane >> tpos) & 1;
                if (cls == GC_HB) {
                    // low lane: v + o; high lane: o - v, i.e. o + sg v with sg = -1
                    const float sg = hi ? -1.f : 1.f;
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const float2 o = shfl<float>(v[j], m);
                        v[j] = make_float2(fmaf(sg, v[j].x, o.x), fmaf(sg, v[j].y, o.y));
                    }
                } else if (cls == GC_X) {
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const float2 o = shfl<float>(v[j], m);
                        if (ok && lpred(j, xm, rm, rv2)) v[j] = o;
                    }
                } else {
                    const float2 cs = hi ? mt.u11 : mt.u00, co = hi ? mt.u10 : mt.u01;
                    if (rm == 0 && __all_sync(0xffffffffu, ok)) {
#pragma unroll
                        for (int j = 0; j < NA; ++j) {
                            const float2 o = shfl<float>(v[j], m);
                            v[j] = cmad2<float>(cs, v[j], co, o);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NA; ++j) {
                            const float2 o = shfl<float>(v[j], m);
                            if (ok && lpred(j, xm, rm, rv2)) v[j] = cmad2<float>(cs, v[j], co, o);
                        }
                    }
                }
            } else {  // OP_DIAG
                if (!ok) continue;
                const float2 d0 = mt.u00, d1 = mt.u01;
                if (tsel == 0) {
                    if (tpos == 0) s_diag_any<0, NA, !TRAJ>(v, d0, d1, xm, rm, rv2);
                    else if (tpos == 1) s_diag_any<1, NA, !TRAJ>(v, d0, d1, xm, rm, rv2);
                    else if (tpos == 2) s_diag_any<2, NA, !TRAJ>(v, d0, d1, xm, rm, rv2);
                    else if (tpos == 3) s_diag_any<3, NA, !TRAJ>(v, d0, d1, xm, rm, rv2);
                    else s_diag_any<(RB64 > 4 ? 4 : 0), NA, !TRAJ>(v, d0, d1, xm, rm, rv2);
                } else {
                    const uint64_t word = tsel == 1 ? uint64_t(tl) : base;
                    const float2 d = ((word >> tpos) & 1) ? d1 : d0;
                    if (d.x == 1.f && d.y == 0.f) continue;   // this thread's entry is exactly 1
                    if (!TRAJ && rm == 0) {
#pragma unroll
                        for (int j = 0; j < NA; ++j) v[j] = cmul<float>(d, v[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < NA; ++j)
                            if (lpred(j, xm, rm, rv2)) v[j] = cmul<float>(d, v[j]);
                    }
                }
            }
        }
        if (P.scale != 1.f) {
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = make_float2(v[j].x * P.scale, v[j].y * P.scale);
        }
        float2 *dst = a + (base | st_t);
        if (xm == 0) {
#pragma unroll
            for (int j = 0; j < NA; ++j) dst[P.st_reg[j]] = v[j];
        } else {
            uint64_t xg = 0;
#pragma unroll
            for (int r = 0; r < RB64; ++r)
                if ((xm >> r) & 1) xg |= P.st_reg[1 << r];
#pragma unroll
            for (int j = 0; j < NA; ++j) dst[P.st_reg[j] ^ xg] = v[j];
        }
    }
}

// The pass kernel of each precision.
template <typename R, int RB> struct PassKernel;
template <> struct PassKernel<double, RB128> {
    static void *ptr() { return reinterpret_cast<void *>(&k_fused<double, RB128>); }
    static void launch(unsigned g, unsigned b, size_t sm, cudaStream_t st, double2 *a, const PassDesc<double> &D) {
        k_fused<double, RB128><<<g, b, sm, st>>>(a, D);
    }
};

// ---------------------------------------------------------------------------
// Host planner
// ---------------------------------------------------------------------------

bool is_diag(int cls) { return cls == GC_DIAG || cls == GC_PHASE; }

uint64_t support(const HostOp &o) {
    uint64_t s = o.cmask | (uint64_t(1) << o.bit);
    if (o.cls == GC_SWAP) s |= uint64_t(1) << o.bit2;
    return s;
}

// SWAP (with optional controls C) as C-NOTs: CX(b->a), CX(C+a -> b), CX(b->a).
void expand_swaps(const std::vector<HostOp> &in, std::vector<HostOp> &out) {
    for (const HostOp &o : in) {
        if (o.cls == GC_ID) continue;
        if (o.cls != GC_SWAP) { out.push_back(o); continue; }
        HostOp x{};
        x.cls = GC_X;
        x.param = -1;
        x.kind = QS_GATE_X;
        x.u[2] = 1.0; x.u[4] = 1.0;
        HostOp c1 = x, c2 = x;
        c1.bit = o.bit; c1.cmask = uint64_t(1) << o.bit2; c1.cval = uint64_t(1) << o.bit2;
        c2.bit = o.bit2; c2.cmask = o.cmask | (uint64_t(1) << o.bit);
        c2.cval = o.cval | (uint64_t(1) << o.bit);
        out.push_back(c1);
        out.push_back(c2);
        out.push_back(c1);
    }
}

struct PlannedPass {
    std::vector<int> high;          // high tile bits, ascending
    std::vector<HostOp> ops;        // ops in execution order
};

}  // namespace

struct Plan {
    int n = 0;
    qs_dtype dt = QS_C64;
    bool fused = false;
    bool unfused_ds = false;                 // unfused mode: complex128 gates in double-single arithmetic
    DsPlan *dsp = nullptr;                   // complex128 passes in double-single arithmetic (qs_fused_ds.cu)
    std::vector<HostOp> ops;                 // unfused mode
    std::vector<PassDesc<float>> pf;         // fused passes, complex64
    std::vector<PassDesc<double>> pd;        // fused passes, complex128
    std::vector<std::vector<FOp<float>>> of; // op tables of the passes (host)
    std::vector<PassC64> pc;                 // complex64 kernel descriptors
    std::vector<std::vector<POp>> pco;       // complex64 kernel op tables (host)
    std::vector<std::vector<FOp<double>>> od;
    void *dev_ops = nullptr;                 // all op tables (device), owned
    bool temp = false;                       // stream-ordered table (one-shot plan)
    cudaStream_t free_stream = nullptr;
    int64_t n_gates = 0;
    std::vector<HostOp> ex;                  // fused mode: the ops planned (SWAPs as C-NOTs); step = index
    std::vector<std::vector<int>> order;     // fused mode: each pass's ops (indices into ex) in execution order
    int RB = 0;
    int grid = 0;                            // persistent grid size
    // per-launch timing (qs_plan_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev;             // begin/end pairs
    size_t ev_used = 0;

    ~Plan() {
        if (dsp) ds_plan_destroy(dsp);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (dev_ops) {
            if (temp) cudaFreeAsync(dev_ops, free_stream);
            else cudaFree(dev_ops);
        }
    }
    // records the begin (end = false) or end event of a launch
    cudaError_t mark(cudaStream_t st, bool end) {
        if (!timing) return cudaSuccess;
        if (ev_used == ev.size()) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
            ev.push_back(e);
        }
        (void)end;
        return cudaEventRecord(ev[ev_used++], st);
    }
};

namespace {

uint32_t pack_layout(const std::vector<int> &regs, const std::vector<int> &warps) {
    uint32_t lay = 0;
    int s = 0;
    for (int r : regs) lay |= uint32_t(r) << (4 * s++);
    for (int w : warps) lay |= uint32_t(w) << (4 * s++);
    return lay;
}

// Reorders the ops of a pass within their commutation freedom so that ops
// whose target is already a register slot run before a transpose is needed.
// Two ops commute when every index bit they share is one on which both act
// diagonally (a control bit, or the target of a diagonal gate): both are then
// block diagonal over the shared bits and act on disjoint bits otherwise.
// List scheduling: the lowest ready op (all non-commuting predecessors done)
// that needs no transpose runs next; when there is none, the register set
// becomes the slots the ready ops need (then the rest in order).
std::vector<HostOp> schedule_pass(const std::vector<HostOp> &ops, const std::map<int, int> &hidx, int RB, int H) {
    const size_t m = ops.size();
    std::vector<uint64_t> sup(m), dg(m);
    std::vector<int> need(m, -1);
    for (size_t k = 0; k < m; ++k) {
        const HostOp &o = ops[k];
        sup[k] = support(o);
        dg[k] = o.cmask | (is_diag(o.cls) ? uint64_t(1) << o.bit : 0);
        if (!is_diag(o.cls) && o.bit >= LB) need[k] = hidx.at(o.bit);
    }
    std::vector<std::vector<int>> succ(m);
    std::vector<int> npred(m, 0);
    for (size_t b = 0; b < m; ++b)
        for (size_t a = 0; a < b; ++a)
            if ((sup[a] & sup[b]) & ~(dg[a] & dg[b])) { succ[a].push_back(int(b)); ++npred[b]; }
    std::set<int> ready;
    for (size_t k = 0; k < m; ++k)
        if (npred[k] == 0) ready.insert(int(k));
    std::vector<char> done(m, 0);
    auto fill = [&](std::vector<int> regs) {
        for (int k : ready)
            if (int(regs.size()) < RB && need[k] >= 0 && std::find(regs.begin(), regs.end(), need[k]) == regs.end())
                regs.push_back(need[k]);
        for (size_t k = 0; k < m && int(regs.size()) < RB; ++k)
            if (!done[k] && need[k] >= 0 && std::find(regs.begin(), regs.end(), need[k]) == regs.end())
                regs.push_back(need[k]);
        for (int i = 0; i < H && int(regs.size()) < RB; ++i)
            if (std::find(regs.begin(), regs.end(), i) == regs.end()) regs.push_back(i);
        return regs;
    };
    std::vector<int> regs = fill({});
    std::vector<HostOp> out;
    out.reserve(m);
    while (out.size() < m) {
        int pick = -1;
        for (int k : ready)
            if (need[k] < 0 || std::find(regs.begin(), regs.end(), need[k]) != regs.end()) { pick = k; break; }
        if (pick < 0) {
            regs = fill({});
            pick = *ready.begin();
        }
        out.push_back(ops[size_t(pick)]);
        done[size_t(pick)] = 1;
        ready.erase(pick);
        for (int sidx : succ[size_t(pick)])
            if (--npred[size_t(sidx)] == 0) ready.insert(sidx);
    }
    return out;
}

template <typename R>
qs_status resolve_pass(int n, int RB, int WB, const PlannedPass &pp, PassDesc<R> &D,
                       std::vector<FOp<R>> &ops_out, std::vector<TrajOpMeta> *metas = nullptr,
                       std::vector<int> *order = nullptr) {
    const int H = RB + WB;
    std::memset(&D, 0, sizeof(D));
    D.K = LB + H;
    D.WB = WB;
    for (int k = 0; k < LB; ++k) D.tile_pos[k] = uint8_t(k);
    for (int i = 0; i < H; ++i) {
        D.tile_pos[LB + i] = uint8_t(pp.high[i]);
        D.hpos[i] = uint8_t(pp.high[i]);
    }
    std::map<int, int> hidx;   // global bit -> high index
    for (int i = 0; i < H; ++i) hidx[pp.high[i]] = i;
    // state-vector plans run the pass's ops in a transpose-saving order; the
    // trajectory mode keeps program order (its per-step Pauli frames follow it)
    const std::vector<HostOp> sched = metas ? pp.ops : schedule_pass(pp.ops, hidx, RB, H);
    const std::vector<HostOp> &ops = sched;
    if (order) {
        order->clear();
        for (const HostOp &o : ops) order->push_back(o.step);
    }

    // register-slot demand sequence: high index needed as a register bit by op k
    const size_t m = ops.size();
    std::vector<int> need(m, -1);
    for (size_t k = 0; k < m; ++k) {
        const HostOp &o = ops[k];
        if (!is_diag(o.cls) && o.bit >= LB) need[k] = hidx.at(o.bit);
    }
    // choose the register set at position k: the RB distinct bits needed
    // soonest from k on, then fill with the lowest remaining
    auto choose = [&](size_t from, std::vector<int> keep_first) {
        std::vector<int> regs = keep_first;
        for (size_t k = from; k < m && int(regs.size()) < RB; ++k)
            if (need[k] >= 0 && std::find(regs.begin(), regs.end(), need[k]) == regs.end())
                regs.push_back(need[k]);
        for (int i = 0; i < H && int(regs.size()) < RB; ++i)
            if (std::find(regs.begin(), regs.end(), i) == regs.end()) regs.push_back(i);
        return regs;
    };
    std::vector<int> regs = choose(0, {});
    auto warps_of = [&](const std::vector<int> &rg) {
        std::vector<int> w;
        for (int i = 0; i < H; ++i)
            if (std::find(rg.begin(), rg.end(), i) == rg.end()) w.push_back(i);
        return w;
    };
    std::vector<int> warps = warps_of(regs);
    D.lay0 = pack_layout(regs, warps);

    ops_out.clear();
    if (metas) metas->clear();
    int n_hb = 0;
    TrajOpMeta cur_meta{};
    auto push = [&](const FOp<R> &f) -> bool {
        if (int(ops_out.size()) >= MAX_OPS) return false;
        ops_out.push_back(f);
        if (metas) {
            TrajOpMeta m = cur_meta;
            if (f.type == OP_XPOSE) m.step = -1;
            metas->push_back(m);
        }
        return true;
    };
    for (size_t k = 0; k < m; ++k) {
        const HostOp &o = ops[k];
        if (need[k] >= 0 && std::find(regs.begin(), regs.end(), need[k]) == regs.end()) {
            // transpose: keep the slots still in demand soonest, in place
            std::vector<int> want = choose(k, {});
            std::vector<int> nr(RB, -1);
            std::vector<bool> used(want.size(), false);
            for (int r = 0; r < RB; ++r)
                for (size_t q = 0; q < want.size(); ++q)
                    if (!used[q] && want[q] == regs[r]) { nr[r] = want[q]; used[q] = true; }
            size_t q = 0;
            for (int r = 0; r < RB; ++r) {
                if (nr[r] >= 0) continue;
                while (used[q]) ++q;
                nr[r] = want[q];
                used[q] = true;
            }
            regs = nr;
            warps = warps_of(regs);
            FOp<R> x{};
            x.type = OP_XPOSE;
            x.lay = pack_layout(regs, warps);
            D.has_xpose = 1;
            if (!push(x)) return QS_EUNSUPPORTED;
        }
        FOp<R> f{};
        cur_meta = TrajOpMeta{};
        cur_meta.step = o.step;
        cur_meta.msrc = o.msrc;
        cur_meta.tbit = o.bit;
        cur_meta.diag = is_diag(o.cls) ? 1 : 0;
        cur_meta.cmask = o.cmask;
        for (int k2 = 0; k2 < 8; ++k2) cur_meta.u[k2] = o.u[k2];
        for (int k2 = 0; k2 < 8; ++k2) cur_meta.reg_src[k2] = -1;
        for (int k2 = 0; k2 < 16; ++k2) cur_meta.thr_src[k2] = -1;
        // controls
        for (int b = 0; b < n; ++b) {
            if (!((o.cmask >> b) & 1)) continue;
            const int val = int((o.cval >> b) & 1);
            if (b < LB) {
                f.tmask |= uint16_t(1u << b);
                if (val) f.tval |= uint16_t(1u << b);
                cur_meta.thr_src[b] = int8_t(b);
            } else if (hidx.count(b)) {
                const int i = hidx[b];
                auto it = std::find(regs.begin(), regs.end(), i);
                if (it != regs.end()) {
                    const int r = int(it - regs.begin());
                    f.rmask |= uint8_t(1u << r);
                    if (val) f.rval |= uint8_t(1u << r);
                    cur_meta.reg_src[r] = int8_t(b);
                } else {
                    const int w = int(std::find(warps.begin(), warps.end(), i) - warps.begin());
                    f.tmask |= uint16_t(1u << (LB + w));
                    if (val) f.tval |= uint16_t(1u << (LB + w));
                    cur_meta.thr_src[LB + w] = int8_t(b);
                }
            } else {
                f.omask |= uint64_t(1) << b;
                if (val) f.oval |= uint64_t(1) << b;
            }
        }
        cur_meta.omask = f.omask;
        if (is_diag(o.cls)) {
            f.type = OP_DIAG;
            // (d0, d1)
            double d0r = o.u[0], d0i = o.u[1], d1r = o.u[6], d1i = o.u[7];
            if (o.cls == GC_PHASE) {
                if (o.phase_on) { d0r = 1; d0i = 0; } else { d1r = 1; d1i = 0; }
            }
            f.u[0] = R(d0r); f.u[1] = R(d0i); f.u[2] = R(d1r); f.u[3] = R(d1i);
            // which side is the identity: 1 = d0 == 1, 2 = d1 == 1, 0 = neither
            f.cls = uint8_t(o.cls == GC_PHASE ? (o.phase_on ? 1 : 2) : 0);
            const int b = o.bit;
            if (b < LB) { f.tsel = 1; f.tpos = uint8_t(b); }
            else if (hidx.count(b)) {
                const int i = hidx[b];
                auto it = std::find(regs.begin(), regs.end(), i);
                if (it != regs.end()) { f.tsel = 0; f.tpos = uint8_t(it - regs.begin()); }
                else {
                    const int w = int(std::find(warps.begin(), warps.end(), i) - warps.begin());
                    f.tsel = 1; f.tpos = uint8_t(LB + w);
                }
            } else { f.tsel = 2; f.tpos = uint8_t(b); }
        } else {
            f.cls = uint8_t(o.cls == GC_X ? GC_X : GC_GEN);
            if (o.kind == QS_GATE_H && o.cmask == 0) {
                f.cls = uint8_t(GC_HB);
                ++n_hb;
            }
            for (int k2 = 0; k2 < 8; ++k2) f.u[k2] = R(o.u[k2]);
            if (o.bit < LB) { f.type = OP_LANE; f.tpos = uint8_t(o.bit); }
            else {
                f.type = OP_REG;
                f.tpos = uint8_t(std::find(regs.begin(), regs.end(), hidx.at(o.bit)) - regs.begin());
            }
        }
        if (!push(f)) return QS_EUNSUPPORTED;
    }
    D.nops = int(ops_out.size());
    // (1/sqrt 2)^n_hb: an exact power of two when n_hb is even
    double sc = std::ldexp(1.0, -(n_hb / 2));
    if (n_hb & 1) sc *= 1.0 / std::sqrt(2.0);
    D.scale = R(sc);
    return QS_OK;
}

// Greedy pass formation.  Ops deferred by one pass are carried (in order)
// ahead of the not yet scanned ops; the scan of a pass stops when every qubit
// is blocked, the pass is full, or a lookahead window is exhausted, so the
// planning time is linear in the circuit length.
std::vector<PlannedPass> form_passes(int n, int H, int max_ops, const std::vector<HostOp> &ops) {
    std::vector<PlannedPass> passes;
    std::vector<HostOp> carry;
    size_t cursor = 0;
    const uint64_t all = n >= 64 ? ~uint64_t(0) : (uint64_t(1) << n) - 1;
    while (!carry.empty() || cursor < ops.size()) {
        PlannedPass pp;
        std::set<int> S;
        std::vector<HostOp> blocked;
        uint64_t blocked_support = 0;
        int budget = max_ops;
        size_t scanned = 0;
        // returns false (op not consumed) when the scan must stop
        auto visit = [&](const HostOp &o) -> bool {
            if ((blocked_support & all) == all || budget <= 1 || scanned > 8192) return false;
            ++scanned;
            const uint64_t sup = support(o);
            bool take = !(sup & blocked_support);
            if (take && !is_diag(o.cls) && o.bit >= LB && !S.count(o.bit)) {
                if (int(S.size()) < H) S.insert(o.bit);
                else take = false;
            }
            if (take) {
                pp.ops.push_back(o);
                budget -= 2;   // room for a transpose per op at worst
            } else {
                blocked.push_back(o);
                blocked_support |= sup;
            }
            return true;
        };
        bool stop = false;
        for (const HostOp &o : carry) {
            if (!stop && visit(o)) continue;
            stop = true;
            blocked.push_back(o);
        }
        while (!stop && cursor < ops.size()) {
            if (!visit(ops[cursor])) break;
            ++cursor;
        }
        // fill the tile with further high bits
        for (int b = LB; b < n && int(S.size()) < H; ++b) S.insert(b);
        pp.high.assign(S.begin(), S.end());
        passes.push_back(std::move(pp));
        carry.swap(blocked);
    }
    return passes;
}

}  // namespace

void expand_swap_ops(const std::vector<HostOp> &in, std::vector<HostOp> &out) { expand_swaps(in, out); }

cudaError_t plan_mark(Plan *p, cudaStream_t st, bool end) { return p ? p->mark(st, end) : cudaSuccess; }

std::vector<PassGroup> group_passes(int n, int H, int max_ops, const std::vector<HostOp> &ops) {
    std::vector<PlannedPass> pp = form_passes(n, H, max_ops, ops);
    std::vector<PassGroup> out(pp.size());
    for (size_t k = 0; k < pp.size(); ++k) {
        out[k].high = pp[k].high;
        for (const HostOp &o : pp[k].ops) out[k].idx.push_back(o.step);
    }
    return out;
}

namespace {

template <typename R, int RB>
qs_status build_fused(Plan *P, const std::vector<HostOp> &ops, int max_ops,
                      std::vector<PassDesc<R>> &out, std::vector<std::vector<FOp<R>>> &tables) {
    const int n = P->n;
    const int WB = std::min(sizeof(R) == 4 ? WB64 : MAX_WB, n - LB - RB);
    const int H = RB + WB;
    std::vector<HostOp> ex;
    expand_swaps(ops, ex);
    for (size_t i = 0; i < ex.size(); ++i) ex[i].step = int32_t(i);
    std::vector<PlannedPass> passes = form_passes(n, H, max_ops, ex);
    out.resize(passes.size());
    tables.resize(passes.size());
    P->order.assign(passes.size(), {});
    size_t total = 0;
    for (size_t k = 0; k < passes.size(); ++k) {
        qs_status st = resolve_pass<R>(n, RB, WB, passes[k], out[k], tables[k], nullptr, &P->order[k]);
        if (st != QS_OK) return st;
        out[k].tiles = uint64_t(1) << (n - out[k].K);
        total += tables[k].size();
    }
    (void)total;
    P->ex = std::move(ex);
    return QS_OK;
}

// Uploads the op tables of all passes on first use (planning itself needs no
// GPU) and sizes the persistent grid.  A temporary plan (one qs_apply_circuit
// call) takes stream-ordered memory that is released on the same stream.
template <typename R, int RB>
cudaError_t ensure_device(Plan *P, std::vector<PassDesc<R>> &passes,
                          const std::vector<std::vector<FOp<R>>> &tables, cudaStream_t st) {
    if (P->dev_ops || passes.empty()) return cudaSuccess;
    std::vector<FOp<R>> flat;
    std::vector<size_t> offs;
    for (auto &t : tables) {
        offs.push_back(flat.size());
        flat.insert(flat.end(), t.begin(), t.end());
    }
    const size_t bytes = flat.size() * sizeof(FOp<R>);
    cudaError_t e;
    if (P->temp) {
        e = cudaMallocAsync(&P->dev_ops, bytes, st);
        if (e != cudaSuccess) return e;
        P->free_stream = st;
        e = cudaMemcpyAsync(P->dev_ops, flat.data(), bytes, cudaMemcpyHostToDevice, st);
    } else {
        e = cudaMalloc(&P->dev_ops, bytes);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(P->dev_ops, flat.data(), bytes, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return e;
    for (size_t k = 0; k < passes.size(); ++k)
        passes[k].ops = static_cast<const FOp<R> *>(P->dev_ops) + offs[k];
    // persistent grid: resident CTAs per SM x SMs (queried once per device)
    static int grid_cache[2][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int &g = grid_cache[sizeof(R) == 8 ? 1 : 0][dev & 63];
    if (g == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t smem_max = (size_t(1) << (LB + RB + MAX_WB)) * sizeof(cplx<R>) + MAX_OPS * sizeof(FOp<R>);
        e = cudaFuncSetAttribute(PassKernel<R, RB>::ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_max));
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, PassKernel<R, RB>::ptr(), 32 << MAX_WB, smem_max);
        if (e != cudaSuccess) return e;
        g = std::max(1, sms * std::max(1, per_sm));
    }
    P->grid = g;
    return cudaSuccess;
}

template <typename R, int RB>
cudaError_t run_passes(qs_state *s, const std::vector<PassDesc<R>> &passes, Plan *P) {
    for (const PassDesc<R> &D : passes) {
        const size_t smem = (D.has_xpose ? (size_t(1) << D.K) * sizeof(cplx<R>) : 0) +
                            size_t(D.nops) * sizeof(FOp<R>);
        const uint64_t grid = std::min<uint64_t>(D.tiles, uint64_t(P->grid));
        cudaError_t e = P->mark(s->stream, false);
        if (e != cudaSuccess) return e;
        PassKernel<R, RB>::launch(unsigned(grid), 32u << D.WB, smem, s->stream, static_cast<cplx<R> *>(s->d), D);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = P->mark(s->stream, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

namespace {

int lay_slot(uint32_t lay, int s) { return int((lay >> (4 * s)) & 15u); }

// Complex64 kernel descriptor and op table from a planned pass: coefficient
// vectors for FFMA2, global offsets of the first and last layouts, and the
// read pattern of every transpose.
void convert_c64(const PassDesc<float> &D, const std::vector<FOp<float>> &ops, PassC64 &out, std::vector<POp> &pops) {
    constexpr int RB = RB64;
    std::memset(&out, 0, sizeof(out));
    out.tiles = D.tiles;
    out.K = D.K;
    out.WB = D.WB;
    out.nops = D.nops;
    out.has_xpose = D.has_xpose;
    out.has_hb = 0;
    out.pad_hb = 0;
    out.scale = D.scale;
    std::memcpy(out.tile_pos, D.tile_pos, sizeof(out.tile_pos));
    const int WB = D.WB;
    auto offsets = [&](uint32_t lay, uint64_t *reg, uint64_t *warp) {
        for (int j = 0; j < 32; ++j) {
            uint64_t o = 0;
            for (int r = 0; r < RB; ++r)
                if ((j >> r) & 1) o |= uint64_t(1) << D.hpos[lay_slot(lay, r)];
            reg[j] = o;
        }
        for (int w = 0; w < 4; ++w) warp[w] = w < WB ? uint64_t(1) << D.hpos[lay_slot(lay, RB + w)] : 0;
    };
    uint32_t lay = D.lay0;
    offsets(lay, out.ld_reg, out.ld_warp);
    pops.assign(ops.size(), POp{});
    for (size_t k = 0; k < ops.size(); ++k) {
        const FOp<float> &f = ops[k];
        POp &q = pops[k];
        q.type = f.type; q.cls = f.cls; q.tsel = f.tsel; q.tpos = f.tpos;
        q.rmask = f.rmask; q.rval = f.rval; q.tmask = f.tmask; q.tval = f.tval;
        q.omask = f.omask; q.oval = f.oval;
        q.fast = 0;
        if (f.type == OP_REG && f.cls != GC_X && f.cls != GC_HB && f.rmask == 0 && f.tmask == 0 && f.omask == 0)
            q.fast = 1;
        else if (f.type == OP_REG && f.cls == GC_X && f.rmask == 0 && (f.tmask & 31u) == 0)
            q.fast = 2;
        else if (f.type == OP_LANE && f.cls != GC_X && f.cls != GC_HB && f.rmask == 0 && f.tmask == 0 &&
                 f.omask == 0)
            q.fast = 3;
        if ((q.fast == 1 || q.fast == 3) && f.u[1] == 0 && f.u[3] == 0 && f.u[5] == 0 && f.u[7] == 0)
            q.fast = uint8_t(q.fast == 1 ? 4 : 5);   // real matrix
        if (f.cls == GC_HB && f.rmask == 0 && f.tmask == 0 && f.omask == 0) {
            if (f.type == OP_REG) q.fast = 6;
            else if (f.type == OP_LANE) q.fast = 7;
            if (q.fast >= 6) out.has_hb = 1;
        }
        if (f.type == OP_XPOSE) {
            // position of each high tile bit in the old tile order
            // (register index bits above the warp bits, warp bits above the lanes)
            int oldpos[16];
            for (int r = 0; r < RB; ++r) oldpos[lay_slot(lay, r)] = LB + WB + r;
            for (int w = 0; w < WB; ++w) oldpos[lay_slot(lay, RB + w)] = LB + w;
            const uint32_t nl = f.lay;
            uint16_t rd[32];
            for (int j = 0; j < 32; ++j) {
                uint32_t o = 0;
                for (int r = 0; r < RB; ++r)
                    if ((j >> r) & 1) o |= 1u << oldpos[lay_slot(nl, r)];
                rd[j] = uint16_t(o);
            }
            std::memcpy(&q.c[0], rd, sizeof(rd));
            uint8_t ow[16] = {0};
            for (int w = 0; w < WB; ++w) ow[w] = uint8_t(oldpos[lay_slot(nl, RB + w)]);
            std::memcpy(&q.c[8], ow, sizeof(ow));
            lay = nl;
        } else if (f.type == OP_DIAG) {
            q.c[0] = make_float2(f.u[0], f.u[1]);
            q.c[1] = make_float2(f.u[2], f.u[3]);
        } else {
            for (int e = 0; e < 4; ++e) q.c[e] = make_float2(f.u[2 * e], f.u[2 * e + 1]);
        }
    }
    offsets(lay, out.st_reg, out.st_warp);
}

cudaError_t ensure_device_c64(Plan *P, cudaStream_t st) {
    if (P->dev_ops || P->pc.empty()) return cudaSuccess;
    std::vector<POp> flat;
    std::vector<size_t> offs;
    for (auto &t : P->pco) {
        offs.push_back(flat.size());
        flat.insert(flat.end(), t.begin(), t.end());
    }
    const size_t bytes = flat.size() * sizeof(POp);
    cudaError_t e;
    if (P->temp) {
        e = cudaMallocAsync(&P->dev_ops, bytes, st);
        if (e != cudaSuccess) return e;
        P->free_stream = st;
        e = cudaMemcpyAsync(P->dev_ops, flat.data(), bytes, cudaMemcpyHostToDevice, st);
    } else {
        e = cudaMalloc(&P->dev_ops, bytes);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(P->dev_ops, flat.data(), bytes, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return e;
    for (size_t k = 0; k < P->pc.size(); ++k) P->pc[k].ops = static_cast<const POp *>(P->dev_ops) + offs[k];
    static int grid_cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int &g = grid_cache[dev & 63];
    if (g == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t smem_max = (size_t(8) << (LB + RB64 + WB64)) + MAX_OPS * sizeof(POp);
        e = cudaFuncSetAttribute(k_fused_c64<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_max));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_c64<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_max));
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_c64<false, false>, 32 << WB64, smem_max);
        if (e != cudaSuccess) return e;
        g = std::max(1, sms * std::max(1, per_sm));
    }
    P->grid = g;
    return cudaSuccess;
}

cudaError_t run_passes_c64(qs_state *s, Plan *P) {
    for (const PassC64 &D : P->pc) {
        const size_t smem = (D.has_xpose ? (size_t(8) << D.K) : 0) + size_t(D.nops) * sizeof(POp);
        const uint64_t grid = std::min<uint64_t>(D.tiles, uint64_t(P->grid));
        cudaError_t e = P->mark(s->stream, false);
        if (e != cudaSuccess) return e;
        if (D.has_hb)
            k_fused_c64<false, true><<<unsigned(grid), 32u << D.WB, smem, s->stream>>>(static_cast<float2 *>(s->d), D);
        else
            k_fused_c64<false, false><<<unsigned(grid), 32u << D.WB, smem, s->stream>>>(static_cast<float2 *>(s->d), D);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = P->mark(s->stream, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

qs_status plan_build(int n, qs_dtype dt, const std::vector<HostOp> &ops, const qs_exec_opts &o, Plan **out,
                     bool temp) {
    Plan *P = new Plan();
    P->temp = temp;
    P->n = n;
    P->dt = dt;
    P->n_gates = int64_t(ops.size());
    P->RB = dt == QS_C64 ? RB64 : RB128;
    const int max_ops = o.max_ops_per_pass > 0 ? std::max(4, std::min(o.max_ops_per_pass, MAX_OPS)) : MAX_OPS;
    P->fused = !o.no_fusion && n >= LB + P->RB;
    // complex128: double-single passes (registers of at least a tile) unless
    // the caller asks for double-precision instructions
    const bool ds = dt == QS_C128 && o.c128_arith != QS_ARITH_F64 && n >= ds_min_qubits();
    if (!P->fused) {
        P->ops = ops;
        P->unfused_ds = dt == QS_C128 && o.c128_arith != QS_ARITH_F64;
    } else if (ds) {
        qs_status st = ds_plan_build(n, ops, o.max_ops_per_pass, temp, &P->dsp);
        if (st != QS_OK) {
            delete P;
            return st;
        }
    } else {
        qs_status st = dt == QS_C64 ? build_fused<float, RB64>(P, ops, max_ops, P->pf, P->of)
                                    : build_fused<double, RB128>(P, ops, max_ops, P->pd, P->od);
        if (st == QS_OK && dt == QS_C64) {
            P->pc.resize(P->pf.size());
            P->pco.resize(P->pf.size());
            for (size_t k = 0; k < P->pf.size(); ++k) convert_c64(P->pf[k], P->of[k], P->pc[k], P->pco[k]);
        }
        if (st != QS_OK) {
            delete P;
            if (st == QS_EUNSUPPORTED) return fail(st, "fusion planner: pass too large");
            return st;
        }
    }
    *out = P;
    return QS_OK;
}

qs_status plan_run(qs_state *s, Plan *p) {
    cudaError_t e = cudaSuccess;
    if (!p->fused) {
        for (const HostOp &o : p->ops) {
            if (o.cls == GC_ID) continue;
            e = p->mark(s->stream, false);
            if (e == cudaSuccess) e = launch_op(s, o, p->unfused_ds);
            if (e == cudaSuccess) e = p->mark(s->stream, true);
            if (e != cudaSuccess) break;
        }
    } else if (p->dsp) {
        e = ds_plan_run(p->dsp, static_cast<double2 *>(s->d), s->stream, p);
    } else if (s->dt == QS_C64) {
        e = ensure_device_c64(p, s->stream);
        if (e == cudaSuccess) e = run_passes_c64(s, p);
    } else {
        e = ensure_device<double, RB128>(p, p->pd, p->od, s->stream);
        if (e == cudaSuccess) e = run_passes<double, RB128>(s, p->pd, p);
    }
    if (e != cudaSuccess) return cuda_fail(e, "circuit launch");
    return QS_OK;
}

void plan_destroy(Plan *p) { delete p; }

void plan_counts(const Plan *p, int64_t *launches, int64_t *gates) {
    if (launches) {
        if (!p->fused) {
            int64_t c = 0;
            for (const HostOp &o : p->ops) c += o.cls == GC_ID ? 0 : 1;
            *launches = c;
        } else {
            *launches = p->dsp ? ds_plan_launches(p->dsp) : int64_t(p->dt == QS_C64 ? p->pf.size() : p->pd.size());
        }
    }
    if (gates) *gates = p->n_gates;
}

qs_status plan_set_timing(Plan *p, bool on) {
    p->timing = on;
    return QS_OK;
}

qs_status plan_timing(Plan *p, double *ms, int64_t *launches) {
    double sum = 0.0;
    for (size_t k = 0; k + 1 < p->ev_used; k += 2) {
        cudaError_t e = cudaEventSynchronize(p->ev[k + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "timing");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p->ev[k], p->ev[k + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "timing");
        sum += double(t);
    }
    if (ms) *ms = sum;
    if (launches) *launches = int64_t(p->ev_used / 2);
    p->ev_used = 0;
    return QS_OK;
}

namespace {
template <typename R>
void describe_passes(const std::vector<PassDesc<R>> &passes, const std::vector<std::vector<FOp<R>>> &tables,
                     const std::vector<std::vector<int>> &order, std::string &out) {
    for (size_t k = 0; k < passes.size(); ++k) {
        const PassDesc<R> &D = passes[k];
        // register ops: general (uncontrolled / register-controlled), Hadamard
        // butterflies, X deferred into the index mask / X moving data; lane ops
        int rg = 0, rgc = 0, rhb = 0, rxd = 0, rx = 0, lg = 0, lx = 0, diag = 0, xp = 0;
        for (const FOp<R> &f : tables[k]) {
            if (f.type == OP_XPOSE) ++xp;
            else if (f.type == OP_DIAG) ++diag;
            else if (f.type == OP_LANE) (f.cls == GC_X ? lx : lg)++;
            else if (f.cls == GC_X) ((f.rmask == 0 && (f.tmask & 31u) == 0) ? rxd : rx)++;
            else if (f.cls == GC_HB) ++rhb;
            else (f.rmask ? rgc : rg)++;
        }
        char line[320];
        std::string bits;
        for (int i = 0; i < D.K; ++i) bits += (i ? "," : "") + std::to_string(int(D.tile_pos[i]));
        std::snprintf(line, sizeof(line),
                      "pass %zu: K=%d WB=%d reg(gen=%d gen_ctl=%d hb=%d x_deferred=%d x_moved=%d) "
                      "lane(gen=%d x=%d) diag=%d xpose=%d bits=[%s]\n",
                      k, D.K, D.WB, rg, rgc, rhb, rxd, rx, lg, lx, diag, xp, bits.c_str());
        out += line;
        if (k < order.size()) {
            out += "  order=";
            for (size_t i = 0; i < order[k].size(); ++i) out += (i ? "," : "") + std::to_string(order[k][i]);
            out += "\n";
        }
    }
}
}  // namespace

std::string plan_describe(const Plan *p) {
    std::string out;
    char head[160];
    std::snprintf(head, sizeof(head), "plan: n=%d dtype=%s gates=%lld fused=%d arith=%s\n", p->n,
                  p->dt == QS_C64 ? "c64" : "c128", (long long)p->n_gates, int(p->fused),
                  p->dt == QS_C64 ? "f32" : (p->dsp ? "double-single" : "f64"));
    out += head;
    if (!p->fused) return out;
    if (p->dsp) return out + ds_plan_describe(p->dsp);
    if (p->dt == QS_C64) describe_passes<float>(p->pf, p->of, p->order, out);
    else describe_passes<double>(p->pd, p->od, p->order, out);
    // the planned ops (forward matrices, (re, im) row-major)
    char line[640];
    for (size_t i = 0; i < p->ex.size(); ++i) {
        const HostOp &o = p->ex[i];
        std::snprintf(line, sizeof(line),
                      "op %zu bit=%d cmask=%llx cval=%llx u=%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g\n", i,
                      int(o.bit), (unsigned long long)o.cmask, (unsigned long long)o.cval, o.u[0], o.u[1], o.u[2],
                      o.u[3], o.u[4], o.u[5], o.u[6], o.u[7]);
        out += line;
    }
    return out;
}

int plan_n(const Plan *p) { return p->n; }
qs_dtype plan_dtype(const Plan *p) { return p->dt; }

// ---------------------------------------------------------------------------
// Trajectory mode: a plan over one group's op list (SWAP-free, classes fixed
// by the caller), executed on all trajectories of the group at once.
// ---------------------------------------------------------------------------
struct TrajPlan {
    int n = 0;
    std::vector<PassC64> pc;
    std::vector<std::vector<POp>> tables;
    std::vector<TrajOpMeta> metas;
    void *dev_ops = nullptr;
    int grid = 0;
    ~TrajPlan() {
        if (dev_ops) cudaFree(dev_ops);
    }
};

qs_status traj_plan_build(int n, const std::vector<HostOp> &ops, int max_ops, TrajPlan **out) {
    if (n < LB + RB64) return fail(QS_EUNSUPPORTED, "trajectory passes need n >= 10");
    TrajPlan *T = new TrajPlan();
    T->n = n;
    const int WB = std::min(WB64, n - LB - RB64);
    const int H = RB64 + WB;
    max_ops = std::max(4, std::min(max_ops > 0 ? max_ops : MAX_OPS, MAX_OPS));
    std::vector<PlannedPass> passes = form_passes(n, H, max_ops, ops);
    for (const PlannedPass &pp : passes) {
        PassDesc<float> D;
        std::vector<FOp<float>> f;
        std::vector<TrajOpMeta> m;
        qs_status st = resolve_pass<float>(n, RB64, WB, pp, D, f, &m);
        if (st != QS_OK) { delete T; return fail(st, "trajectory planner: pass too large"); }
        D.tiles = uint64_t(1) << (n - D.K);
        PassC64 c;
        std::vector<POp> pops;
        convert_c64(D, f, c, pops);
        c.n = n;
        c.rec_off = uint32_t(T->metas.size());
        c.tiles_per_traj = D.tiles;
        T->metas.insert(T->metas.end(), m.begin(), m.end());
        T->pc.push_back(c);
        T->tables.push_back(std::move(pops));
    }
    for (PassC64 &c : T->pc) c.rec_stride = uint32_t(T->metas.size());
    // op tables on the device
    std::vector<POp> flat;
    std::vector<size_t> offs;
    for (auto &t : T->tables) {
        offs.push_back(flat.size());
        flat.insert(flat.end(), t.begin(), t.end());
    }
    if (!flat.empty()) {
        if (cudaMalloc(&T->dev_ops, flat.size() * sizeof(POp)) != cudaSuccess) {
            cudaGetLastError();
            delete T;
            return fail(QS_ENOMEM, "trajectory planner: device allocation failed");
        }
        cudaError_t e = cudaMemcpy(T->dev_ops, flat.data(), flat.size() * sizeof(POp), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { delete T; return cuda_fail(e, "trajectory planner upload"); }
        for (size_t k = 0; k < T->pc.size(); ++k) T->pc[k].ops = static_cast<const POp *>(T->dev_ops) + offs[k];
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem_max = (size_t(8) << (LB + RB64 + WB64)) + MAX_OPS * (sizeof(POp) + sizeof(TrajRec));
    cudaError_t e = cudaFuncSetAttribute(k_fused_c64<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_max));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_c64<true, false>, 32 << WB64, smem_max);
    if (e != cudaSuccess) { delete T; return cuda_fail(e, "trajectory planner: kernel attributes"); }
    T->grid = std::max(1, sms * std::max(1, per_sm));
    *out = T;
    return QS_OK;
}

const std::vector<TrajOpMeta> &traj_plan_metas(const TrajPlan *p) { return p->metas; }
int64_t traj_plan_launches(const TrajPlan *p) { return int64_t(p->pc.size()); }

cudaError_t traj_plan_run(TrajPlan *T, float2 *states, uint32_t count, const TrajRec *recs, cudaStream_t st) {
    for (const PassC64 &c0 : T->pc) {
        PassC64 D = c0;
        D.recs = recs;
        D.tiles = D.tiles_per_traj * count;
        const size_t smem = (D.has_xpose ? (size_t(8) << D.K) : 0) + size_t(D.nops) * (sizeof(POp) + sizeof(TrajRec));
        const uint64_t grid = std::min<uint64_t>(D.tiles, uint64_t(T->grid));
        k_fused_c64<true, false><<<unsigned(grid), 32u << D.WB, smem, st>>>(states, D);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void traj_plan_destroy(TrajPlan *p) { delete p; }

}  // namespace qs
