// Fused passes over a complex128 state in double-single arithmetic.
//
// A pass groups consecutive gates whose targets lie in a tile of 2^12
// amplitudes (the five lowest index bits, so that global loads and stores are
// contiguous 512-byte rows, plus seven higher bits chosen per pass) and
// applies all of them to the tile in shared memory: one HBM read and one
// write of the state per pass.  The tile is the paper's block M_k (Sec.
// 2.2.1) generalised to any set of fixed index bits.
//
// Number format: the state is complex128 in memory (the paper's double
// precision, Sec. 2.1) before and after a plan runs.  The first pass of a
// plan splits each amplitude into two float pairs (re = rh + rl, im = ih +
// il, 48 significant bits) with integer instructions, the gates run in
// double-single arithmetic (qs_ds.cuh: exact products and sums of the high
// parts by error-free transformations, low parts in single precision) on the
// single-precision pipe, and the last pass joins the pairs back into
// doubles; between the passes of the plan the state holds the float pairs
// (16 bytes per amplitude, like the complex128).  Gate matrices come from
// the plan's double-precision matrices, split on the host.
//
// The tile lives in shared memory (16 bytes per amplitude, float4), not in
// registers: a gate is a loop over the thread's pairs with the target bit a
// runtime value, one loop per op type, so the code does not multiply with
// the target bits and any tile bit can be a target without a transpose.
// Per op:
//   * general or real 2x2 on tile bit t (Sec. 2.2.1: x' = u11 x + u12 y,
//     y' = u21 x + u22 y), with controls as a predicate on the pair's index
//     (tile bits) or on the tile's position (other bits), Sec. 2.2.2;
//   * an uncontrolled Hadamard as the butterfly (x + y, x - y), the factors
//     1/sqrt 2 of a pass folded into one scale at the store;
//   * a diagonal gate on the amplitudes it changes (only one side of the
//     target when the other entry is exactly 1);
//   * a C-NOT without controls on tile bits moves no data: the tile keeps an
//     XOR mask, and logical index i sits at place i ^ mask.
// 256 threads per CTA, three CTAs per SM (shared memory), so that one CTA's
// HBM phase overlaps the others' arithmetic.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "qs_ds.cuh"
#include "qs_internal.cuh"

namespace qs {

namespace {

constexpr int LB = 5;                   // lane bits (contiguous rows of 32 amplitudes)
#ifndef QS_DS_K
#define QS_DS_K 12
#endif
#ifndef QS_DS_THREADS
#define QS_DS_THREADS 256
#endif
#ifndef QS_DS_MINBLOCKS
#define QS_DS_MINBLOCKS 3
#endif
// pairs of an op per loop iteration: the eight pairs of a thread fully
// unrolled measured fastest (n = 30 random circuit: 4.82 s per step, against
// 4.86 s for two and 4.97 s for one; one loop per op type in every case)
#ifndef QS_DS_UNROLL
#define QS_DS_UNROLL 8
#endif
constexpr int DK = QS_DS_K;             // tile bits
constexpr int DH = DK - LB;             // high tile bits
constexpr int DT = 1 << DK;             // amplitudes per tile
constexpr int DTHREADS = QS_DS_THREADS;
constexpr int DMAX_OPS = 80;            // ops per pass
constexpr int DMINBLOCKS = QS_DS_MINBLOCKS;
constexpr int DUNROLL = QS_DS_UNROLL;     // pairs per loop iteration

enum DsType : uint8_t { D_GEN = 0, D_REAL = 1, D_HB = 2, D_X = 3, D_DIAG = 4 };

// One op (96 bytes).
struct alignas(16) SOp {
    uint8_t type;       // DsType
    uint8_t tbit;       // tile-local target bit; D_DIAG with the target outside the tile: 0xff
    uint8_t one;        // D_DIAG: 1 d0 == 1 (only target-1 amplitudes change), 2 d1 == 1, 0 neither
    uint8_t obit;       // D_DIAG with the target outside the tile: its index bit
    uint32_t tmask, tval;   // control condition over the tile-local (logical) index
    uint32_t pad;
    uint64_t omask, oval;   // control condition over the index bits outside the tile
    float c[16];        // u00, u01, u10, u11 as (re_h, re_l, im_h, im_l); D_DIAG: d0, d1
};
static_assert(sizeof(SOp) == 96, "SOp layout");

struct DsPass {
    const SOp *ops;
    uint64_t tiles;
    int32_t nops;
    float scale_h, scale_l;     // folded Hadamard factor
    // between the passes of one plan the state holds each amplitude as its
    // float pairs (rh, rl, ih, il: 16 bytes, the size of the complex128): the
    // first pass splits the doubles, the last joins them back
    uint8_t in_pairs, out_pairs;
    uint8_t pad[2];
    uint8_t tile_pos[DK];       // ascending; the first LB are 0 .. LB-1
};

using ds::camp;
using ds::ccst;

__device__ __forceinline__ ccst cst(const float *c) { return {c[0], c[1], c[2], c[3]}; }
__device__ __forceinline__ camp ld(const float4 &f) { return {f.x, f.y, f.z, f.w}; }
__device__ __forceinline__ float4 st(const camp &a) { return make_float4(a.rh, a.rl, a.ih, a.il); }

// A 2x2 op (general, real or Hadamard butterfly) on the pair (x, y).
__device__ __forceinline__ void pair_op(int type, const ccst &u00, const ccst &u01, const ccst &u10, const ccst &u11,
                                        camp &x, camp &y) {
    if (type == D_HB) {
        ds::butterfly(x, y);
    } else if (type == D_REAL) {
        const camp nx = ds::rmad2(u00, x, u01, y), ny = ds::rmad2(u10, x, u11, y);
        x = nx;
        y = ny;
    } else {
        const camp nx = ds::cmad2(u00, x, u01, y), ny = ds::cmad2(u10, x, u11, y);
        x = nx;
        y = ny;
    }
}

// logical index of pair p with a zero inserted at bit t
__device__ __forceinline__ uint32_t pair_index(uint32_t p, int t) {
    return ((p >> t) << (t + 1)) | (p & ((1u << t) - 1u));
}

// One 2x2 op of type TY on the thread's pairs whose controls hold (CTL:
// the op has controls on tile bits).  The thread's pair j is p = tid + j *
// DTHREADS; with the zero inserted at bit t its index is the index of pair
// tid ORed with that of j * DTHREADS (the two have no bit in common), so the
// eight indices cost one OR each.
template <int TY, bool CTL>
__device__ __forceinline__ void pairs_loop(float4 *amp, int t, uint32_t tm, uint32_t tv, uint32_t xm, const float *c,
                                           int tid) {
    ccst u00{}, u01{}, u10{}, u11{};
    if (TY == D_GEN || TY == D_REAL) { u00 = cst(c); u01 = cst(c + 4); u10 = cst(c + 8); u11 = cst(c + 12); }
    static_assert(DT / 2 / DTHREADS == 8, "eight pairs per thread");
    const uint32_t ib = pair_index(uint32_t(tid), t), tb = 1u << t;
    const uint32_t o1 = pair_index(DTHREADS, t), o2 = pair_index(2 * DTHREADS, t), o4 = pair_index(4 * DTHREADS, t);
#pragma unroll DUNROLL
    for (int j = 0; j < DT / 2 / DTHREADS; ++j) {
        const uint32_t i0 = ib | ((j & 1) ? o1 : 0u) | ((j & 2) ? o2 : 0u) | ((j & 4) ? o4 : 0u);
        if (CTL && (i0 & tm) != tv) continue;
        const uint32_t q0 = i0 ^ xm, q1 = q0 ^ tb;
        camp x = ld(amp[q0]), y = ld(amp[q1]);
        if (TY == D_X) {
            amp[q0] = st(y);
            amp[q1] = st(x);
            continue;
        }
        pair_op(TY, u00, u01, u10, u11, x, y);
        amp[q0] = st(x);
        amp[q1] = st(y);
    }
}

__global__ void __launch_bounds__(DTHREADS, DMINBLOCKS) k_fused_ds(double2 *__restrict__ a,
                                                                const __grid_constant__ DsPass P) {
    extern __shared__ __align__(16) float4 smem[];
    float4 *amp = smem;                                            // DT amplitudes
    SOp *ops = reinterpret_cast<SOp *>(smem + DT);                 // P.nops ops
    uint64_t *rowoff = reinterpret_cast<uint64_t *>(ops + P.nops); // 2^DH row offsets
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.ops);
        uint4 *dst = reinterpret_cast<uint4 *>(ops);
        for (int k = tid; k < P.nops * int(sizeof(SOp) / 16); k += DTHREADS) dst[k] = src[k];
        for (int r = tid; r < (1 << DH); r += DTHREADS) {
            uint64_t o = 0;
            for (int h = 0; h < DH; ++h)
                if ((r >> h) & 1) o |= uint64_t(1) << P.tile_pos[LB + h];
            rowoff[r] = o;
        }
        __syncthreads();
    }
    for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
        uint64_t base = tile;
        for (int k = 0; k < DK; ++k) {
            const uint64_t low = (uint64_t(1) << P.tile_pos[k]) - 1;
            base = ((base & ~low) << 1) | (base & low);
        }
        // load: warp w reads rows w, w + 8, ... (512 contiguous bytes each)
#pragma unroll 4
        for (int r = warp; r < (1 << DH); r += DTHREADS / 32) {
            const uint64_t gi = base | rowoff[r] | uint64_t(lane);
            if (P.in_pairs) {
                amp[(r << LB) | lane] = reinterpret_cast<const float4 *>(a)[gi];
            } else {
                const double2 d = a[gi];
                amp[(r << LB) | lane] = st(ds::load(d.x, d.y));
            }
        }
        __syncthreads();
        uint32_t xm = 0;   // logical index i sits at amp[i ^ xm]
        for (int k = 0; k < P.nops; ++k) {
            const SOp &o = ops[k];
            if ((base & o.omask) != o.oval) continue;   // the same for the whole tile
            const int type = o.type;
            const uint32_t tm = o.tmask, tv = o.tval;
            if (type == D_X && tm == 0) {                // relabel, no data moves
                xm ^= 1u << o.tbit;
                continue;
            }
            if (type == D_DIAG) {
                const ccst d0 = cst(o.c), d1 = cst(o.c + 4);
                if (o.tbit == 0xff) {
                    const ccst d = ((base >> o.obit) & 1) ? d1 : d0;
                    if (!(d.rh == 1.f && d.rl == 0.f && d.ih == 0.f && d.il == 0.f)) {
                        for (uint32_t i = tid; i < uint32_t(DT); i += DTHREADS)
                            if ((i & tm) == tv) amp[i ^ xm] = st(ds::cmul(d, ld(amp[i ^ xm])));
                    }
                } else {
                    const int t = o.tbit;
                    const int one = o.one;
                    for (uint32_t p = tid; p < uint32_t(DT / 2); p += DTHREADS) {
                        const uint32_t i0 = pair_index(p, t), i1 = i0 | (1u << t);
                        if (one != 1 && (i0 & tm) == tv) amp[i0 ^ xm] = st(ds::cmul(d0, ld(amp[i0 ^ xm])));
                        if (one != 2 && (i1 & tm) == tv) amp[i1 ^ xm] = st(ds::cmul(d1, ld(amp[i1 ^ xm])));
                    }
                }
            } else {
                if (tm == 0) {
                    if (type == D_GEN) pairs_loop<D_GEN, false>(amp, o.tbit, tm, tv, xm, o.c, tid);
                    else if (type == D_REAL) pairs_loop<D_REAL, false>(amp, o.tbit, tm, tv, xm, o.c, tid);
                    else pairs_loop<D_HB, false>(amp, o.tbit, tm, tv, xm, o.c, tid);   // (D_X without controls relabels)
                } else {
                    if (type == D_GEN) pairs_loop<D_GEN, true>(amp, o.tbit, tm, tv, xm, o.c, tid);
                    else if (type == D_REAL) pairs_loop<D_REAL, true>(amp, o.tbit, tm, tv, xm, o.c, tid);
                    else if (type == D_HB) pairs_loop<D_HB, true>(amp, o.tbit, tm, tv, xm, o.c, tid);
                    else pairs_loop<D_X, true>(amp, o.tbit, tm, tv, xm, o.c, tid);
                }
            }
            __syncthreads();
        }
        // store (with the folded Hadamard factor)
        const bool scale = P.scale_h != 1.f || P.scale_l != 0.f;
#pragma unroll 4
        for (int r = warp; r < (1 << DH); r += DTHREADS / 32) {
            camp x = ld(amp[((uint32_t(r) << LB) | uint32_t(lane)) ^ xm]);
            if (scale) {
                ds::mul1(x.rh, x.rl, P.scale_h, P.scale_l, x.rh, x.rl);
                ds::mul1(x.ih, x.il, P.scale_h, P.scale_l, x.ih, x.il);
            }
            const uint64_t gi = base | rowoff[r] | uint64_t(lane);
            if (P.out_pairs) reinterpret_cast<float4 *>(a)[gi] = st(x);
            else a[gi] = make_double2(ds::join(x.rh, x.rl), ds::join(x.ih, x.il));
        }
        __syncthreads();
    }
}

size_t ds_smem(int nops) { return size_t(DT) * 16 + size_t(nops) * sizeof(SOp) + (size_t(8) << DH); }

bool diag_cls(int cls) { return cls == GC_DIAG || cls == GC_PHASE; }

}  // namespace

struct DsPlan {
    int n = 0;
    std::vector<DsPass> passes;
    std::vector<std::vector<SOp>> tables;
    std::vector<std::vector<int>> order;    // per pass: indices into ex, in execution order
    std::vector<HostOp> ex;                 // the planned ops (SWAPs as three C-NOTs)
    void *dev = nullptr;
    bool temp = false;
    cudaStream_t free_stream = nullptr;
    int grid = 0;
    ~DsPlan() {
        if (dev) {
            if (temp) cudaFreeAsync(dev, free_stream);
            else cudaFree(dev);
        }
    }
};

qs_status ds_plan_build(int n, const std::vector<HostOp> &ops, int max_ops, bool temp, DsPlan **out) {
    if (n < DK) return fail(QS_EUNSUPPORTED, "double-single passes need n >= the tile bits");
    DsPlan *P = new DsPlan();
    P->n = n;
    P->temp = temp;
    expand_swap_ops(ops, P->ex);
    for (size_t i = 0; i < P->ex.size(); ++i) P->ex[i].step = int32_t(i);
    max_ops = std::max(4, std::min(max_ops > 0 ? max_ops : 2 * DMAX_OPS, 2 * DMAX_OPS));
    for (const PassGroup &gp : group_passes(n, DH, max_ops, P->ex)) {
        DsPass D;
        std::memset(&D, 0, sizeof(D));
        for (int k = 0; k < LB; ++k) D.tile_pos[k] = uint8_t(k);
        int local[64];
        for (int b = 0; b < 64; ++b) local[b] = -1;
        for (int k = 0; k < LB; ++k) local[k] = k;
        for (int h = 0; h < DH; ++h) {
            D.tile_pos[LB + h] = uint8_t(gp.high[size_t(h)]);
            local[gp.high[size_t(h)]] = LB + h;
        }
        std::vector<SOp> tab;
        int n_hb = 0;
        for (int idx : gp.idx) {
            const HostOp &o = P->ex[size_t(idx)];
            SOp s;
            std::memset(&s, 0, sizeof(s));
            for (int b = 0; b < n; ++b) {
                if (!((o.cmask >> b) & 1)) continue;
                const uint64_t v = (o.cval >> b) & 1;
                if (local[b] >= 0) {
                    s.tmask |= 1u << local[b];
                    s.tval |= uint32_t(v) << local[b];
                } else {
                    s.omask |= uint64_t(1) << b;
                    s.oval |= v << b;
                }
            }
            auto put = [&](int e, double re, double im) {
                ds::split_const(re, s.c[4 * e], s.c[4 * e + 1]);
                ds::split_const(im, s.c[4 * e + 2], s.c[4 * e + 3]);
            };
            if (diag_cls(o.cls)) {
                s.type = D_DIAG;
                double d0r = o.u[0], d0i = o.u[1], d1r = o.u[6], d1i = o.u[7];
                if (o.cls == GC_PHASE) {
                    if (o.phase_on) { d0r = 1; d0i = 0; } else { d1r = 1; d1i = 0; }
                }
                put(0, d0r, d0i);
                put(1, d1r, d1i);
                s.one = uint8_t((d0r == 1 && d0i == 0) ? 1 : (d1r == 1 && d1i == 0) ? 2 : 0);
                if (local[o.bit] >= 0) s.tbit = uint8_t(local[o.bit]);
                else { s.tbit = 0xff; s.obit = uint8_t(o.bit); }
            } else {
                if (local[o.bit] < 0) { delete P; return fail(QS_EUNSUPPORTED, "planner: target outside the tile"); }
                s.tbit = uint8_t(local[o.bit]);
                const bool real = o.u[1] == 0 && o.u[3] == 0 && o.u[5] == 0 && o.u[7] == 0;
                if (o.cls == GC_X) s.type = D_X;
                else if (o.kind == QS_GATE_H && o.cmask == 0) { s.type = D_HB; ++n_hb; }
                else s.type = real ? D_REAL : D_GEN;
                for (int e = 0; e < 4; ++e) put(e, o.u[2 * e], o.u[2 * e + 1]);
            }
            tab.push_back(s);
        }
        if (int(tab.size()) > DMAX_OPS) { delete P; return fail(QS_EUNSUPPORTED, "planner: pass too large"); }
        double sc = std::ldexp(1.0, -(n_hb / 2));
        if (n_hb & 1) sc *= 1.0 / std::sqrt(2.0);
        ds::split_const(sc, D.scale_h, D.scale_l);
        D.nops = int32_t(tab.size());
        D.tiles = uint64_t(1) << (n - DK);
        P->passes.push_back(D);
        P->tables.push_back(std::move(tab));
        P->order.push_back(gp.idx);
    }
    for (size_t k = 0; k < P->passes.size(); ++k) {
        P->passes[k].in_pairs = uint8_t(k > 0);
        P->passes[k].out_pairs = uint8_t(k + 1 < P->passes.size());
    }
    *out = P;
    return QS_OK;
}

// Uploads the op tables on first use and sizes the grid.
static cudaError_t ds_ensure_device(DsPlan *P, cudaStream_t st) {
    if (P->dev || P->passes.empty()) return cudaSuccess;
    std::vector<SOp> flat;
    std::vector<size_t> offs;
    for (auto &t : P->tables) {
        offs.push_back(flat.size());
        flat.insert(flat.end(), t.begin(), t.end());
    }
    const size_t bytes = std::max<size_t>(1, flat.size()) * sizeof(SOp);
    cudaError_t e;
    if (P->temp) {
        e = cudaMallocAsync(&P->dev, bytes, st);
        if (e != cudaSuccess) return e;
        P->free_stream = st;
        e = cudaMemcpyAsync(P->dev, flat.data(), flat.size() * sizeof(SOp), cudaMemcpyHostToDevice, st);
    } else {
        e = cudaMalloc(&P->dev, bytes);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(P->dev, flat.data(), flat.size() * sizeof(SOp), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return e;
    for (size_t k = 0; k < P->passes.size(); ++k) P->passes[k].ops = static_cast<const SOp *>(P->dev) + offs[k];
    static int grid_cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int &g = grid_cache[dev & 63];
    if (g == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t smax = ds_smem(DMAX_OPS);
        e = cudaFuncSetAttribute(k_fused_ds, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smax));
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_ds, DTHREADS, smax);
        if (e != cudaSuccess) return e;
        g = std::max(1, sms * std::max(1, per_sm));
    }
    P->grid = g;
    return cudaSuccess;
}

cudaError_t ds_plan_run(DsPlan *P, double2 *state, cudaStream_t st, Plan *timing) {
    cudaError_t e = ds_ensure_device(P, st);
    if (e != cudaSuccess) return e;
    for (const DsPass &D : P->passes) {
        const uint64_t grid = std::min<uint64_t>(D.tiles, uint64_t(P->grid));
        e = plan_mark(timing, st, false);
        if (e != cudaSuccess) return e;
        k_fused_ds<<<unsigned(grid), DTHREADS, ds_smem(D.nops), st>>>(state, D);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = plan_mark(timing, st, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int64_t ds_plan_launches(const DsPlan *P) { return int64_t(P->passes.size()); }

int ds_min_qubits() { return DK; }

std::string ds_plan_describe(const DsPlan *P) {
    std::string out;
    char line[640];
    for (size_t k = 0; k < P->passes.size(); ++k) {
        const DsPass &D = P->passes[k];
        int cnt[5] = {0, 0, 0, 0, 0}, xdef = 0;
        for (const SOp &s : P->tables[k]) {
            if (s.type == D_X && s.tmask == 0) ++xdef;
            else ++cnt[s.type];
        }
        std::string bits;
        for (int i = 0; i < DK; ++i) bits += (i ? "," : "") + std::to_string(int(D.tile_pos[i]));
        std::snprintf(line, sizeof(line),
                      "pass %zu: K=%d double-single gen=%d real=%d hb=%d x_deferred=%d x_moved=%d diag=%d bits=[%s]\n",
                      k, DK, cnt[D_GEN], cnt[D_REAL], cnt[D_HB], xdef, cnt[D_X], cnt[D_DIAG], bits.c_str());
        out += line;
        out += "  order=";
        for (size_t i = 0; i < P->order[k].size(); ++i) out += (i ? "," : "") + std::to_string(P->order[k][i]);
        out += "\n";
    }
    for (size_t i = 0; i < P->ex.size(); ++i) {
        const HostOp &o = P->ex[i];
        std::snprintf(line, sizeof(line),
                      "op %zu bit=%d cmask=%llx cval=%llx u=%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g\n", i,
                      int(o.bit), (unsigned long long)o.cmask, (unsigned long long)o.cval, o.u[0], o.u[1], o.u[2],
                      o.u[3], o.u[4], o.u[5], o.u[6], o.u[7]);
        out += line;
    }
    return out;
}

void ds_plan_destroy(DsPlan *P) { delete P; }

}  // namespace qs
