// A register partitioned over ranks (one GPU each).
//
// The paper parallelises a gate on qubit i by splitting the overall matrix
// into independent blocks M_k = S_k phi_k, one group of blocks per processor
// (Sec. 2.2.1).  Across GPUs the same split becomes a partition of the
// amplitude index: with 2^g ranks, the g most significant index bits
// (qubits 0 .. g-1, "global" qubits) name the rank, and rank r holds the
// 2^(n-g) amplitudes whose top g bits equal r.  A gate is local to every
// rank when its target is a local qubit; controls on global qubits are
// per-rank predicates, and a diagonal gate on a global qubit multiplies each
// rank's slice by one of its two entries.  A non-diagonal gate on a global
// qubit needs the pairs (i0, i0 + 2^(n-1-q)) on one rank: before it, the
// global qubit exchanges places with a local one (a qubit swap), which moves
// half of every slice to the partner rank r ^ (bit of the global qubit) and
// brings the partner's half back (the half-slice exchange).
//
// qs_shard_plan rewrites a circuit into physical qubit numbering:
//   * an uncontrolled SWAP of the circuit relabels qubits and moves no data;
//     a controlled SWAP becomes three C-NOTs;
//   * before a non-diagonal gate on a global qubit, a SWAP(global, local)
//     exchange is emitted; the local qubit given up is the one whose next
//     non-diagonal use lies furthest ahead (Belady's rule), so that few
//     exchanges are needed;
//   * every other gate keeps its kind and angles, with its qubits renamed.
// qs_shard_localize turns a stretch of that list between two exchanges into
// one rank's gates on its 2^(n-g)-amplitude slice.  qs_shard_pack / unpack
// move a half slice to and from a contiguous device buffer for the exchange
// (the transport, NCCL or another, is the caller's).
#include <algorithm>
#include <cstring>
#include <limits>
#include <vector>

#include "qs_internal.cuh"

namespace qs {
namespace {

qs_gate cnot(int control, int target, uint64_t extra_mask, uint64_t extra_val) {
    qs_gate x;
    std::memset(&x, 0, sizeof(x));
    x.kind = QS_GATE_X;
    x.t = target;
    x.t2 = -1;
    x.param = -1;
    x.ctrl_mask = extra_mask | (uint64_t(1) << control);
    x.ctrl_val = extra_val | (uint64_t(1) << control);
    return x;
}

// Qubits of a gate renamed by map[old] = new (target, second SWAP qubit,
// controls and their values).
qs_gate rename(const qs_gate &g, const std::vector<int> &map) {
    qs_gate o = g;
    o.t = map[size_t(g.t)];
    if (g.kind == QS_GATE_SWAP) o.t2 = map[size_t(g.t2)];
    o.ctrl_mask = 0;
    o.ctrl_val = 0;
    for (size_t q = 0; q < map.size(); ++q) {
        if ((g.ctrl_mask >> q) & 1) {
            o.ctrl_mask |= uint64_t(1) << map[q];
            if ((g.ctrl_val >> q) & 1) o.ctrl_val |= uint64_t(1) << map[q];
        }
    }
    return o;
}

__global__ void k_pack(const uint8_t *__restrict__ a, uint8_t *__restrict__ buf, uint64_t half, int bit, uint64_t val,
                       int amp_bytes, bool unpack) {
    // element i of the buffer <-> the amplitude whose index is i with `val`
    // inserted at index bit `bit`
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < half;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t low = i & ((uint64_t(1) << bit) - 1);
        const uint64_t idx = ((i >> bit) << (bit + 1)) | (val << bit) | low;
        if (amp_bytes == 16) {
            const double2 *src = reinterpret_cast<const double2 *>(unpack ? buf : a);
            double2 *dst = reinterpret_cast<double2 *>(unpack ? const_cast<uint8_t *>(a) : buf);
            if (unpack) dst[idx] = src[i];
            else dst[i] = src[idx];
        } else {
            const float2 *src = reinterpret_cast<const float2 *>(unpack ? buf : a);
            float2 *dst = reinterpret_cast<float2 *>(unpack ? const_cast<uint8_t *>(a) : buf);
            if (unpack) dst[idx] = src[i];
            else dst[i] = src[idx];
        }
    }
}

qs_status pack_common(qs_state *s, int q, int value, void *buf, bool unpack) {
    if (!s || !buf) return fail(QS_EINVAL, "NULL argument");
    if (q < 0 || q >= s->n) return fail(QS_EINVAL, "qubit out of range");
    if (value != 0 && value != 1) return fail(QS_EINVAL, "value must be 0 or 1");
    const int amp = s->dt == QS_C128 ? 16 : 8;
    if (reinterpret_cast<uintptr_t>(buf) % amp) return fail(QS_EINVAL, "buffer not aligned to an amplitude");
    const uint64_t half = uint64_t(1) << (s->n - 1);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, unpack ? "shard unpack: device" : "shard pack: device");
    const uint64_t blocks = std::min<uint64_t>((half + 255) / 256, uint64_t(std::max(1, sms)) * 8);
    k_pack<<<unsigned(blocks), 256, 0, s->stream>>>(static_cast<const uint8_t *>(s->d), static_cast<uint8_t *>(buf),
                                                    half, s->n - 1 - q, uint64_t(value), amp, unpack);
    e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : cuda_fail(e, unpack ? "shard unpack" : "shard pack");
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_shard_plan(int n, int g, const qs_gate *gates, size_t m, qs_gate *out, size_t max_out,
                                   size_t *n_out, int32_t *final_pos) {
    if (!n_out || (m > 0 && !gates)) return fail(QS_EINVAL, "NULL argument");
    if (n < 2 || n > QS_MAX_QUBITS) return fail(QS_ERANGE, "n out of range");
    if (g < 0 || g > n - 2) return fail(QS_ERANGE, "g must leave at least two local qubits");
    // 1. circuit in "data qubits": uncontrolled SWAPs relabel, controlled
    //    SWAPs become three C-NOTs (CX(b->a), CX(C, a -> b), CX(b->a))
    std::vector<int> lab(static_cast<size_t>(n));          // logical qubit -> data qubit
    for (int q = 0; q < n; ++q) lab[size_t(q)] = q;
    std::vector<qs_gate> dg;
    std::vector<char> diag;
    for (size_t k = 0; k < m; ++k) {
        HostOp op;
        if (synthesize(n, gates[k], op) != QS_OK) {
            return fail(QS_EINVAL, "gate " + std::to_string(k) + ": invalid");
        }
        const qs_gate &x = gates[k];
        if (x.kind == QS_GATE_SWAP && x.ctrl_mask == 0) {
            std::swap(lab[size_t(x.t)], lab[size_t(x.t2)]);
            continue;
        }
        if (x.kind == QS_GATE_SWAP) {
            const qs_gate c1 = cnot(x.t2, x.t, 0, 0), c2 = cnot(x.t, x.t2, x.ctrl_mask, x.ctrl_val);
            for (const qs_gate &c : {c1, c2, c1}) {
                dg.push_back(rename(c, lab));
                diag.push_back(0);
            }
            continue;
        }
        dg.push_back(rename(x, lab));
        diag.push_back(op.cls == GC_DIAG || op.cls == GC_PHASE || op.cls == GC_ID ? 1 : 0);
    }
    // 2. next non-diagonal use of each data qubit, for Belady's choice
    const size_t M = dg.size();
    const int64_t NEVER = std::numeric_limits<int64_t>::max();
    std::vector<std::vector<int64_t>> uses(static_cast<size_t>(n));
    for (size_t k = 0; k < M; ++k)
        if (!diag[k]) uses[size_t(dg[k].t)].push_back(int64_t(k));
    std::vector<size_t> cursor(size_t(n), 0);
    auto next_use = [&](int d, size_t k) {
        std::vector<int64_t> &u = uses[size_t(d)];
        size_t &c = cursor[size_t(d)];
        while (c < u.size() && u[c] < int64_t(k)) ++c;
        return c < u.size() ? u[c] : NEVER;
    };
    // 3. placement: data qubit d sits at physical qubit pos[d]
    std::vector<int> pos(static_cast<size_t>(n)), at(static_cast<size_t>(n));
    for (int q = 0; q < n; ++q) pos[size_t(q)] = at[size_t(q)] = q;
    size_t cnt = 0;
    auto emit = [&](const qs_gate &x) {
        if (out && cnt < max_out) out[cnt] = x;
        ++cnt;
    };
    for (size_t k = 0; k < M; ++k) {
        const qs_gate &x = dg[k];
        if (!diag[k] && pos[size_t(x.t)] < g) {
            // bring the target to a local place: give up the local qubit used
            // furthest ahead, preferring one that is not a control of x
            int best = -1;
            int64_t best_use = -1;
            bool best_ctl = true;
            for (int p = g; p < n; ++p) {
                const int d = at[size_t(p)];
                const bool ctl = (x.ctrl_mask >> d) & 1;
                const int64_t u = next_use(d, k);
                if (best < 0 || (best_ctl && !ctl) || (ctl == best_ctl && u > best_use)) {
                    best = p;
                    best_use = u;
                    best_ctl = ctl;
                }
            }
            const int pg = pos[size_t(x.t)];
            qs_gate sw;
            std::memset(&sw, 0, sizeof(sw));
            sw.kind = QS_GATE_SWAP;
            sw.t = pg;
            sw.t2 = best;
            sw.param = -1;
            emit(sw);
            const int dl = at[size_t(best)];
            std::swap(pos[size_t(x.t)], pos[size_t(dl)]);
            at[size_t(pg)] = dl;
            at[size_t(best)] = x.t;
        }
        emit(rename(x, pos));
    }
    *n_out = cnt;
    if (final_pos)
        for (int q = 0; q < n; ++q) final_pos[q] = pos[size_t(lab[size_t(q)])];
    if (out && cnt > max_out) return fail(QS_ERANGE, "output array too small (see *n_out)");
    return QS_OK;
}

extern "C" qs_status qs_shard_localize(int n, int g, uint32_t rank, const qs_gate *in, size_t m, qs_gate *out,
                                       size_t max_out, size_t *n_out) {
    if (!n_out || (m > 0 && !in)) return fail(QS_EINVAL, "NULL argument");
    if (n < 2 || n > QS_MAX_QUBITS) return fail(QS_ERANGE, "n out of range");
    if (g < 0 || g > n - 2) return fail(QS_ERANGE, "g must leave at least two local qubits");
    if (g < 32 && rank >> g) return fail(QS_ERANGE, "rank >= 2^g");
    const int nl = n - g;
    const uint64_t gmask = (uint64_t(1) << g) - 1;   // global qubits 0 .. g-1
    size_t cnt = 0;
    auto rbit = [&](int q) { return uint64_t((rank >> (g - 1 - q)) & 1u); };
    for (size_t k = 0; k < m; ++k) {
        const qs_gate &x = in[k];
        HostOp op;
        if (synthesize(n, x, op) != QS_OK) return fail(QS_EINVAL, "gate " + std::to_string(k) + ": invalid");
        if (x.kind == QS_GATE_SWAP && (x.t < g || x.t2 < g))
            return fail(QS_EINVAL, "gate " + std::to_string(k) + ": an exchange (SWAP with a global qubit)");
        // controls on global qubits: this rank's bits decide
        bool holds = true;
        for (int q = 0; q < g; ++q)
            if ((x.ctrl_mask >> q) & 1) holds = holds && rbit(q) == ((x.ctrl_val >> q) & 1);
        if (!holds) continue;
        qs_gate o = x;
        o.ctrl_mask = (x.ctrl_mask & ~gmask) >> g;
        o.ctrl_val = (x.ctrl_val & x.ctrl_mask & ~gmask) >> g;
        if (x.t >= g) {
            o.t = x.t - g;
            if (x.kind == QS_GATE_SWAP) o.t2 = x.t2 - g;
        } else {
            // target global: only a diagonal gate; this rank's entry scales
            // every amplitude of the slice that meets the local controls
            if (!(op.cls == GC_DIAG || op.cls == GC_PHASE || op.cls == GC_ID))
                return fail(QS_EINVAL, "gate " + std::to_string(k) + ": non-diagonal gate on a global qubit");
            const double dr = rbit(x.t) ? op.u[6] : op.u[0], di = rbit(x.t) ? op.u[7] : op.u[1];
            if (dr == 1.0 && di == 0.0) continue;
            // a local qubit that is not a control carries diag(d, d); if every
            // local qubit is a control, the last control carries the entry on
            // its required value only
            int tq = -1;
            for (int q = nl - 1; q >= 0 && tq < 0; --q)
                if (!((o.ctrl_mask >> q) & 1)) tq = q;
            std::memset(o.u, 0, sizeof(o.u));
            o.kind = QS_GATE_MATRIX;
            o.t2 = -1;
            o.param = -1;
            if (tq >= 0) {
                o.t = tq;
                o.u[0] = {dr, di};
                o.u[3] = {dr, di};
            } else {
                tq = nl - 1;
                const bool v1 = (o.ctrl_val >> tq) & 1;
                o.ctrl_mask &= ~(uint64_t(1) << tq);
                o.ctrl_val &= ~(uint64_t(1) << tq);
                o.t = tq;
                o.u[0] = v1 ? qs_c128{1.0, 0.0} : qs_c128{dr, di};
                o.u[3] = v1 ? qs_c128{dr, di} : qs_c128{1.0, 0.0};
            }
        }
        if (out && cnt < max_out) out[cnt] = o;
        ++cnt;
    }
    *n_out = cnt;
    if (out && cnt > max_out) return fail(QS_ERANGE, "output array too small (see *n_out)");
    return QS_OK;
}

extern "C" qs_status qs_shard_pack(qs_state *s, int q, int value, void *dev_buf) {
    return pack_common(s, q, value, dev_buf, false);
}

extern "C" qs_status qs_shard_unpack(qs_state *s, int q, int value, const void *dev_buf) {
    return pack_common(s, q, value, const_cast<void *>(dev_buf), true);
}
