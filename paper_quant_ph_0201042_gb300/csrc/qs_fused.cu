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
#include <cstring>
#include <map>
#include <set>

#include "qs_internal.cuh"

namespace qs {

namespace {

constexpr int LB = 5;          // lane bits
constexpr int MAX_WB = 3;      // warp bits (8 warps)
constexpr int MAX_OPS = 120;   // ops per pass (kernel parameter space)

enum OpType : uint8_t { OP_REG = 0, OP_LANE = 1, OP_DIAG = 2, OP_XPOSE = 3 };

template <typename R>
struct FOp {
    uint8_t type;      // OpType
    uint8_t cls;       // GateClass (OP_REG / OP_LANE)
    uint8_t tsel;      // OP_DIAG target: 0 register slot, 1 thread bit, 2 outer bit
    uint8_t tpos;      // register slot / lane bit / thread bit / outer bit
    uint8_t rmask, rval;   // control condition over the register index
    uint8_t tmask, tval;   // control condition over the thread index (lane | warp << 5)
    uint8_t lay[8];        // OP_XPOSE: new high-bit index of each register slot, then warp bit
    uint64_t omask, oval;  // control condition over the index bits outside the tile
    R u[8];                // matrix, or (d0, d1) for OP_DIAG
};

template <typename R>
struct PassDesc {
    int32_t K;             // tile bits
    int32_t WB;            // warp bits
    int32_t nops;
    int32_t pad;
    uint8_t tile_pos[24];  // all tile bit positions, ascending (the first five are 0..4)
    uint8_t hpos[16];      // global position of high tile bit i (= tile_pos[5 + i])
    uint8_t lay0[8];       // initial layout (register slots, then warp bits)
    FOp<R> ops[MAX_OPS];
};

// Global index offset of register index j given the register-slot bit values.
template <int RB>
__device__ __forceinline__ uint64_t reg_offset(int j, const uint64_t (&rpos)[RB]) {
    uint64_t o = 0;
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if ((j >> r) & 1) o |= rpos[r];
    return o;
}

template <int RB>
__device__ __forceinline__ uint32_t reg_local(int j, const uint32_t (&lpos)[RB]) {
    uint32_t o = 0;
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if ((j >> r) & 1) o |= lpos[r];
    return o;
}

template <typename R, int RB, int T>
__device__ __forceinline__ void apply_reg(cplx<R> (&v)[1 << RB], const FOp<R> &op, bool ok) {
    const cplx<R> u00 = mk<R>(op.u[0], op.u[1]), u01 = mk<R>(op.u[2], op.u[3]);
    const cplx<R> u10 = mk<R>(op.u[4], op.u[5]), u11 = mk<R>(op.u[6], op.u[7]);
    const int cls = op.cls;
    const int rm = op.rmask, rv = op.rval;
#pragma unroll
    for (int j = 0; j < (1 << RB); ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        if (!(ok && ((j & rm) == rv))) continue;
        const cplx<R> x = v[j], y = v[j1];
        if (cls == GC_GEN) {
            v[j] = cmad2<R>(u00, x, u01, y);
            v[j1] = cmad2<R>(u10, x, u11, y);
        } else if (cls == GC_REAL) {
            v[j] = rmad2<R>(u00.x, x, u01.x, y);
            v[j1] = rmad2<R>(u10.x, x, u11.x, y);
        } else if (cls == GC_ANTI) {
            v[j] = cmul<R>(u01, y);
            v[j1] = cmul<R>(u10, x);
        } else {  // GC_X
            v[j] = y;
            v[j1] = x;
        }
    }
}

template <typename R>
__device__ __forceinline__ cplx<R> shfl(cplx<R> a, int m) {
    return mk<R>(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
}

template <typename R, int RB>
__global__ void __launch_bounds__(256) k_fused(cplx<R> *__restrict__ a, const __grid_constant__ PassDesc<R> P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<R> *sm = reinterpret_cast<cplx<R> *>(smraw);
    constexpr int NA = 1 << RB;
    const int K = P.K, WB = P.WB;
    const uint32_t tl = threadIdx.x;            // lane | warp << 5
    const uint32_t lane = tl & 31u, warp = tl >> 5;

    // tile base: the block index with zeros inserted at every tile position
    uint64_t base = blockIdx.x;
    for (int k = 0; k < K; ++k) {
        const uint64_t low = (uint64_t(1) << P.tile_pos[k]) - 1;
        base = ((base & ~low) << 1) | (base & low);
    }

    // layout: high-bit index of each register slot and warp bit
    int rh[RB], wh[MAX_WB];
#pragma unroll
    for (int r = 0; r < RB; ++r) rh[r] = P.lay0[r];
#pragma unroll
    for (int w = 0; w < MAX_WB; ++w) wh[w] = w < WB ? P.lay0[RB + w] : 0;

    uint64_t rpos[RB];
    uint64_t toff = lane;
#pragma unroll
    for (int r = 0; r < RB; ++r) rpos[r] = uint64_t(1) << P.hpos[rh[r]];
#pragma unroll
    for (int w = 0; w < MAX_WB; ++w)
        if (w < WB && ((warp >> w) & 1)) toff |= uint64_t(1) << P.hpos[wh[w]];

    cplx<R> v[NA];
    const cplx<R> *src = a + (base | toff);
#pragma unroll
    for (int j = 0; j < NA; ++j) v[j] = src[reg_offset<RB>(j, rpos)];

    for (int k = 0; k < P.nops; ++k) {
        const FOp<R> &op = P.ops[k];
        const int type = op.type;
        if (type == OP_XPOSE) {
            // write with the current layout, read back with the new one
            uint32_t lpos[RB];
            uint32_t tloc = lane;
#pragma unroll
            for (int r = 0; r < RB; ++r) lpos[r] = 1u << (LB + rh[r]);
#pragma unroll
            for (int w = 0; w < MAX_WB; ++w)
                if (w < WB && ((warp >> w) & 1)) tloc |= 1u << (LB + wh[w]);
#pragma unroll
            for (int j = 0; j < NA; ++j) sm[tloc | reg_local<RB>(j, lpos)] = v[j];
            __syncthreads();
#pragma unroll
            for (int r = 0; r < RB; ++r) rh[r] = op.lay[r];
#pragma unroll
            for (int w = 0; w < MAX_WB; ++w) wh[w] = w < WB ? op.lay[RB + w] : 0;
            tloc = lane;
#pragma unroll
            for (int r = 0; r < RB; ++r) lpos[r] = 1u << (LB + rh[r]);
#pragma unroll
            for (int w = 0; w < MAX_WB; ++w)
                if (w < WB && ((warp >> w) & 1)) tloc |= 1u << (LB + wh[w]);
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = sm[tloc | reg_local<RB>(j, lpos)];
            __syncthreads();
            continue;
        }
        const bool ok = ((tl & op.tmask) == op.tval) && ((base & op.omask) == op.oval);
        if (type == OP_REG) {
            switch (op.tpos) {
            case 0: apply_reg<R, RB, 0>(v, op, ok); break;
            case 1: apply_reg<R, RB, 1>(v, op, ok); break;
            case 2: apply_reg<R, RB, 2>(v, op, ok); break;
            case 3: apply_reg<R, RB, 3>(v, op, ok); break;
            default: if (RB > 4) apply_reg<R, RB, (RB > 4 ? 4 : 0)>(v, op, ok); break;
            }
        } else if (type == OP_LANE) {
            const int m = 1 << op.tpos;
            const bool hi = (lane >> op.tpos) & 1;
            const cplx<R> u00 = mk<R>(op.u[0], op.u[1]), u01 = mk<R>(op.u[2], op.u[3]);
            const cplx<R> u10 = mk<R>(op.u[4], op.u[5]), u11 = mk<R>(op.u[6], op.u[7]);
            // the coefficient on my own amplitude and on the partner's
            const cplx<R> cs = hi ? u11 : u00, co = hi ? u10 : u01;
            const int cls = op.cls;
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                if ((j & op.rmask) != op.rval) continue;   // uniform across the warp
                const cplx<R> o = shfl<R>(v[j], m);
                if (!ok) continue;
                if (cls == GC_GEN) v[j] = cmad2<R>(cs, v[j], co, o);
                else if (cls == GC_REAL) v[j] = rmad2<R>(cs.x, v[j], co.x, o);
                else if (cls == GC_ANTI) v[j] = cmul<R>(co, o);
                else v[j] = o;
            }
        } else {  // OP_DIAG
            const cplx<R> d0 = mk<R>(op.u[0], op.u[1]), d1 = mk<R>(op.u[2], op.u[3]);
            if (op.tsel == 0) {
#pragma unroll
                for (int j = 0; j < NA; ++j)
                    if (ok && ((j & op.rmask) == op.rval)) v[j] = cmul<R>(((j >> op.tpos) & 1) ? d1 : d0, v[j]);
            } else {
                const uint64_t word = op.tsel == 1 ? uint64_t(tl) : base;
                const cplx<R> d = ((word >> op.tpos) & 1) ? d1 : d0;
#pragma unroll
                for (int j = 0; j < NA; ++j)
                    if (ok && ((j & op.rmask) == op.rval)) v[j] = cmul<R>(d, v[j]);
            }
        }
    }

    // store with the final layout
#pragma unroll
    for (int r = 0; r < RB; ++r) rpos[r] = uint64_t(1) << P.hpos[rh[r]];
    toff = lane;
#pragma unroll
    for (int w = 0; w < MAX_WB; ++w)
        if (w < WB && ((warp >> w) & 1)) toff |= uint64_t(1) << P.hpos[wh[w]];
    cplx<R> *dst = a + (base | toff);
#pragma unroll
    for (int j = 0; j < NA; ++j) dst[reg_offset<RB>(j, rpos)] = v[j];
}

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
    std::vector<HostOp> ops;                 // unfused mode
    std::vector<PassDesc<float>> pf;         // fused passes, complex64
    std::vector<PassDesc<double>> pd;        // fused passes, complex128
    int64_t n_gates = 0;
    int RB = 0;
    // per-launch timing (qs_plan_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev;             // begin/end pairs
    size_t ev_used = 0;

    ~Plan() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
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

template <typename R>
qs_status resolve_pass(int n, int RB, int WB, const PlannedPass &pp, PassDesc<R> &D) {
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

    // register-slot demand sequence: high index needed as a register bit by op k
    const size_t m = pp.ops.size();
    std::vector<int> need(m, -1);
    for (size_t k = 0; k < m; ++k) {
        const HostOp &o = pp.ops[k];
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
    for (int r = 0; r < RB; ++r) D.lay0[r] = uint8_t(regs[r]);
    for (int w = 0; w < WB; ++w) D.lay0[RB + w] = uint8_t(warps[w]);

    int nops = 0;
    auto push = [&](const FOp<R> &f) -> bool {
        if (nops >= MAX_OPS) return false;
        D.ops[nops++] = f;
        return true;
    };
    for (size_t k = 0; k < m; ++k) {
        const HostOp &o = pp.ops[k];
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
            for (int r = 0; r < RB; ++r) x.lay[r] = uint8_t(regs[r]);
            for (int w = 0; w < WB; ++w) x.lay[RB + w] = uint8_t(warps[w]);
            if (!push(x)) return QS_EUNSUPPORTED;
        }
        FOp<R> f{};
        // controls
        for (int b = 0; b < n; ++b) {
            if (!((o.cmask >> b) & 1)) continue;
            const int val = int((o.cval >> b) & 1);
            if (b < LB) {
                f.tmask |= uint8_t(1u << b);
                if (val) f.tval |= uint8_t(1u << b);
            } else if (hidx.count(b)) {
                const int i = hidx[b];
                auto it = std::find(regs.begin(), regs.end(), i);
                if (it != regs.end()) {
                    const int r = int(it - regs.begin());
                    f.rmask |= uint8_t(1u << r);
                    if (val) f.rval |= uint8_t(1u << r);
                } else {
                    const int w = int(std::find(warps.begin(), warps.end(), i) - warps.begin());
                    f.tmask |= uint8_t(1u << (LB + w));
                    if (val) f.tval |= uint8_t(1u << (LB + w));
                }
            } else {
                f.omask |= uint64_t(1) << b;
                if (val) f.oval |= uint64_t(1) << b;
            }
        }
        if (is_diag(o.cls)) {
            f.type = OP_DIAG;
            // (d0, d1)
            double d0r = o.u[0], d0i = o.u[1], d1r = o.u[6], d1i = o.u[7];
            if (o.cls == GC_PHASE) {
                if (o.phase_on) { d0r = 1; d0i = 0; } else { d1r = 1; d1i = 0; }
            }
            f.u[0] = R(d0r); f.u[1] = R(d0i); f.u[2] = R(d1r); f.u[3] = R(d1i);
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
            f.cls = uint8_t(o.cls);
            for (int k2 = 0; k2 < 8; ++k2) f.u[k2] = R(o.u[k2]);
            if (o.bit < LB) { f.type = OP_LANE; f.tpos = uint8_t(o.bit); }
            else {
                f.type = OP_REG;
                f.tpos = uint8_t(std::find(regs.begin(), regs.end(), hidx.at(o.bit)) - regs.begin());
            }
        }
        if (!push(f)) return QS_EUNSUPPORTED;
    }
    D.nops = nops;
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

template <typename R>
qs_status build_fused(Plan *P, int RB, const std::vector<HostOp> &ops, int max_ops,
                      std::vector<PassDesc<R>> &out) {
    const int n = P->n;
    const int WB = std::min(MAX_WB, n - LB - RB);
    const int H = RB + WB;
    std::vector<HostOp> ex;
    expand_swaps(ops, ex);
    std::vector<PlannedPass> passes = form_passes(n, H, max_ops, ex);
    out.resize(passes.size());
    for (size_t k = 0; k < passes.size(); ++k) {
        qs_status st = resolve_pass<R>(n, RB, WB, passes[k], out[k]);
        if (st != QS_OK) return st;
    }
    return QS_OK;
}

template <typename R, int RB>
cudaError_t run_passes(qs_state *s, const std::vector<PassDesc<R>> &passes, Plan *P) {
    static bool attr_done[8] = {false};
    const int n = s->n;
    for (const PassDesc<R> &D : passes) {
        const uint64_t tiles = uint64_t(1) << (n - D.K);
        bool any_x = false;
        for (int k = 0; k < D.nops; ++k) any_x |= D.ops[k].type == OP_XPOSE;
        const size_t smem = any_x ? (size_t(1) << D.K) * sizeof(cplx<R>) : 0;
        int dev = 0;
        cudaGetDevice(&dev);
        if (smem > 48 * 1024 && !attr_done[dev & 7]) {
            cudaError_t e = cudaFuncSetAttribute(k_fused<R, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int((size_t(1) << (LB + RB + MAX_WB)) * sizeof(cplx<R>)));
            if (e != cudaSuccess) return e;
            attr_done[dev & 7] = true;
        }
        cudaError_t e = P->mark(s->stream, false);
        if (e != cudaSuccess) return e;
        k_fused<R, RB><<<unsigned(tiles), 32u << D.WB, smem, s->stream>>>(static_cast<cplx<R> *>(s->d), D);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = P->mark(s->stream, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

constexpr int RB64 = 5;    // complex64: 32 amplitudes per thread
constexpr int RB128 = 4;   // complex128: 16 amplitudes per thread

}  // namespace

qs_status plan_build(int n, qs_dtype dt, const std::vector<HostOp> &ops, const qs_exec_opts &o, Plan **out) {
    Plan *P = new Plan();
    P->n = n;
    P->dt = dt;
    P->n_gates = int64_t(ops.size());
    P->RB = dt == QS_C64 ? RB64 : RB128;
    const int max_ops = o.max_ops_per_pass > 0 ? std::max(4, std::min(o.max_ops_per_pass, MAX_OPS)) : MAX_OPS;
    P->fused = !o.no_fusion && n >= LB + P->RB;
    if (!P->fused) {
        P->ops = ops;
    } else {
        qs_status st = dt == QS_C64 ? build_fused<float>(P, RB64, ops, max_ops, P->pf)
                                    : build_fused<double>(P, RB128, ops, max_ops, P->pd);
        if (st != QS_OK) { delete P; return fail(st, "fusion planner: pass too large"); }
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
            if (e == cudaSuccess) e = launch_op(s, o);
            if (e == cudaSuccess) e = p->mark(s->stream, true);
            if (e != cudaSuccess) break;
        }
    } else if (s->dt == QS_C64) {
        e = run_passes<float, RB64>(s, p->pf, p);
    } else {
        e = run_passes<double, RB128>(s, p->pd, p);
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
            *launches = int64_t(p->dt == QS_C64 ? p->pf.size() : p->pd.size());
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

int plan_n(const Plan *p) { return p->n; }
qs_dtype plan_dtype(const Plan *p) { return p->dt; }

}  // namespace qs
