// C ABI of libqsim (declared in include/qsim.h): argument validation, gate
// synthesis, state lifetime, and the host side of every call.  All arithmetic
// on the register runs in the kernels of qs_gates.cu, qs_fused.cu and
// qs_reduce.cu; nothing here touches amplitudes on the host.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qs_internal.cuh"

namespace qs {

namespace {
thread_local std::string g_err;

size_t amp_size(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

bool finite8(const double *u) {
    for (int k = 0; k < 8; ++k)
        if (!std::isfinite(u[k])) return false;
    return true;
}
}  // namespace

qs_status fail(qs_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

qs_status cuda_fail(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return QS_ECUDA;
}

// Matrix of a gate from its kind and angles (Sec. 2.3.1 H, Sec. 3.2 U_R,
// U_P1, U_P2 and their products, Pauli matrices), then its class.
qs_status synthesize(int n, const qs_gate &g, HostOp &op) {
    std::memset(&op, 0, sizeof(op));
    op.param = g.param;
    op.kind = g.kind;
    op.theta[0] = g.theta[0];
    op.theta[1] = g.theta[1];
    if (g.t < 0 || g.t >= n) return fail(QS_EINVAL, "target qubit out of range");
    if (n < 64 && (g.ctrl_mask >> n) != 0) return fail(QS_EINVAL, "control qubit out of range");
    if ((g.ctrl_mask >> g.t) & 1) return fail(QS_EINVAL, "target qubit is also a control");
    // index-bit form (qubit q is index bit n-1-q)
    for (int q = 0; q < n; ++q) {
        if ((g.ctrl_mask >> q) & 1) {
            op.cmask |= uint64_t(1) << (n - 1 - q);
            if ((g.ctrl_val >> q) & 1) op.cval |= uint64_t(1) << (n - 1 - q);
        }
    }
    op.bit = n - 1 - g.t;
    op.bit2 = -1;
    if (g.kind == QS_GATE_SWAP) {
        if (g.t2 < 0 || g.t2 >= n || g.t2 == g.t) return fail(QS_EINVAL, "bad second SWAP qubit");
        if ((g.ctrl_mask >> g.t2) & 1) return fail(QS_EINVAL, "SWAP qubit is also a control");
        op.cls = GC_SWAP;
        op.bit2 = n - 1 - g.t2;
        return QS_OK;
    }
    double *u = op.u;
    const double a = g.theta[0], b = g.theta[1];
    const double s2 = 1.0 / std::sqrt(2.0);
    auto set = [&](double r0, double i0, double r1, double i1, double r2, double i2, double r3, double i3) {
        u[0] = r0; u[1] = i0; u[2] = r1; u[3] = i1; u[4] = r2; u[5] = i2; u[6] = r3; u[7] = i3;
    };
    switch (g.kind) {
    case QS_GATE_MATRIX:
        for (int k = 0; k < 4; ++k) { u[2 * k] = g.u[k].re; u[2 * k + 1] = g.u[k].im; }
        break;
    case QS_GATE_H: set(s2, 0, s2, 0, s2, 0, -s2, 0); break;
    case QS_GATE_X: set(0, 0, 1, 0, 1, 0, 0, 0); break;
    case QS_GATE_Y: set(0, 0, 0, -1, 0, 1, 0, 0); break;
    case QS_GATE_Z: set(1, 0, 0, 0, 0, 0, -1, 0); break;
    case QS_GATE_UP1: set(1, 0, 0, 0, 0, 0, std::cos(a), std::sin(a)); break;
    case QS_GATE_UP2: set(std::cos(a), std::sin(a), 0, 0, 0, 0, 1, 0); break;
    case QS_GATE_UR: set(std::cos(a), 0, -std::sin(a), 0, std::sin(a), 0, std::cos(a), 0); break;
    case QS_GATE_URP1: {
        // [[c, -s], [s, c]] diag(1, e^{i b}) = [[c, -s e^{ib}], [s, c e^{ib}]]
        const double c = std::cos(a), s = std::sin(a), cb = std::cos(b), sb = std::sin(b);
        set(c, 0, -s * cb, -s * sb, s, 0, c * cb, c * sb);
        break;
    }
    case QS_GATE_RY: set(std::cos(a / 2), 0, -std::sin(a / 2), 0, std::sin(a / 2), 0, std::cos(a / 2), 0); break;
    case QS_GATE_RZ: set(std::cos(a / 2), -std::sin(a / 2), 0, 0, 0, 0, std::cos(a / 2), std::sin(a / 2)); break;
    default:
        return fail(QS_EINVAL, "unknown gate kind");
    }
    if (!finite8(u)) return fail(QS_EINVAL, "gate matrix is not finite");
    // classification
    const bool off0 = u[2] == 0 && u[3] == 0 && u[4] == 0 && u[5] == 0;
    const bool dia0 = u[0] == 0 && u[1] == 0 && u[6] == 0 && u[7] == 0;
    const bool real = u[1] == 0 && u[3] == 0 && u[5] == 0 && u[7] == 0;
    if (off0) {
        const bool one0 = u[0] == 1 && u[1] == 0, one1 = u[6] == 1 && u[7] == 0;
        if (one0 && one1) op.cls = GC_ID;
        else if (one0) { op.cls = GC_PHASE; op.phase_on = 1; }
        else if (one1) { op.cls = GC_PHASE; op.phase_on = 0; }
        else op.cls = GC_DIAG;
    } else if (dia0) {
        op.cls = (u[2] == 1 && u[3] == 0 && u[4] == 1 && u[5] == 0) ? GC_X : GC_ANTI;
    } else {
        op.cls = real ? GC_REAL : GC_GEN;
    }
    return QS_OK;
}

static qs_status synth_all(int n, const qs_gate *g, size_t m, std::vector<HostOp> &ops) {
    ops.resize(m);
    for (size_t k = 0; k < m; ++k) {
        qs_status st = synthesize(n, g[k], ops[k]);
        if (st != QS_OK) {
            g_err = "gate " + std::to_string(k) + ": " + g_err;
            return st;
        }
    }
    return QS_OK;
}

}  // namespace qs

using namespace qs;

static qs_status state_scratch(qs_state *s) {
    cudaError_t e = cudaMalloc(&s->partial, sizeof(double) * 4 * RED_BLOCKS);
    if (e != cudaSuccess) return fail(QS_ENOMEM, "scratch allocation failed");
    e = cudaMalloc(&s->result, sizeof(double) * 4);
    if (e != cudaSuccess) return fail(QS_ENOMEM, "scratch allocation failed");
    e = cudaMallocHost(&s->host_result, sizeof(double) * 4);
    if (e != cudaSuccess) return fail(QS_ENOMEM, "pinned allocation failed");
    return QS_OK;
}

static void state_release(qs_state *s) {
    if (s->partial) cudaFree(s->partial);
    if (s->result) cudaFree(s->result);
    if (s->host_result) cudaFreeHost(s->host_result);
    if (s->owned && s->d) cudaFree(s->d);
    delete s;
}

extern "C" {

const char *qs_last_error(void) { return g_err.c_str(); }

qs_status qs_alloc(int n, qs_dtype dt, qs_state **out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_ERANGE, "n out of range");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    qs_state *s = new qs_state();
    s->n = n;
    s->dt = dt;
    s->owned = true;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaMalloc(&s->d, amp_size(dt) << n);
    if (e != cudaSuccess) {
        s->d = nullptr;
        cudaGetLastError();
        state_release(s);
        return fail(QS_ENOMEM, "device allocation of the state failed");
    }
    qs_status st = state_scratch(s);
    if (st != QS_OK) { state_release(s); return st; }
    e = launch_init_basis(s, 0);
    if (e != cudaSuccess) { state_release(s); return cuda_fail(e, "init"); }
    *out = s;
    return QS_OK;
}

qs_status qs_wrap(void *dev_ptr, int n, qs_dtype dt, qs_state **out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_ERANGE, "n out of range");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 15)) return fail(QS_EINVAL, "pointer NULL or not 16-byte aligned");
    qs_state *s = new qs_state();
    s->n = n;
    s->dt = dt;
    s->d = dev_ptr;
    s->owned = false;
    cudaGetDevice(&s->device);
    qs_status st = state_scratch(s);
    if (st != QS_OK) { state_release(s); return st; }
    *out = s;
    return QS_OK;
}

qs_status qs_free(qs_state *s) {
    if (!s) return QS_OK;
    cudaStreamSynchronize(s->stream);
    state_release(s);
    return QS_OK;
}

qs_status qs_set_stream(qs_state *s, void *stream) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    s->stream = static_cast<cudaStream_t>(stream);
    return QS_OK;
}

qs_status qs_info(const qs_state *s, void **dev_ptr, int *n, qs_dtype *dt) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    if (dev_ptr) *dev_ptr = s->d;
    if (n) *n = s->n;
    if (dt) *dt = s->dt;
    return QS_OK;
}

qs_status qs_init_basis(qs_state *s, uint64_t x) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    if (x >> s->n) return fail(QS_ERANGE, "basis index >= 2^n");
    cudaError_t e = launch_init_basis(s, x);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "init_basis");
}

qs_status qs_apply_gate(qs_state *s, const qs_gate *g) {
    if (!s || !g) return fail(QS_EINVAL, "NULL argument");
    HostOp op;
    qs_status st = synthesize(s->n, *g, op);
    if (st != QS_OK) return st;
    cudaError_t e = launch_op(s, op, true);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "gate launch");
}

static qs_gate matrix_gate(int t, uint64_t cmask, uint64_t cval, const qs_c128 U[4]) {
    qs_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = QS_GATE_MATRIX;
    g.t = t;
    g.t2 = -1;
    g.param = -1;
    g.ctrl_mask = cmask;
    g.ctrl_val = cval & cmask;
    for (int k = 0; k < 4; ++k) g.u[k] = U[k];
    return g;
}

qs_status qs_apply_1q(qs_state *s, int q, const qs_c128 U[4]) {
    if (!s || !U) return fail(QS_EINVAL, "NULL argument");
    qs_gate g = matrix_gate(q, 0, 0, U);
    return qs_apply_gate(s, &g);
}

qs_status qs_apply_ctrl(qs_state *s, int c, int t, const qs_c128 U[4]) {
    if (!s || !U) return fail(QS_EINVAL, "NULL argument");
    if (c < 0 || c >= s->n) return fail(QS_EINVAL, "control qubit out of range");
    if (c == t) return fail(QS_EINVAL, "control equals target");
    qs_gate g = matrix_gate(t, uint64_t(1) << c, uint64_t(1) << c, U);
    return qs_apply_gate(s, &g);
}

qs_status qs_apply_mctrl(qs_state *s, uint64_t ctrl_mask, uint64_t ctrl_val, int t, const qs_c128 U[4]) {
    if (!s || !U) return fail(QS_EINVAL, "NULL argument");
    qs_gate g = matrix_gate(t, ctrl_mask, ctrl_val, U);
    return qs_apply_gate(s, &g);
}

qs_status qs_apply_swap(qs_state *s, int a, int b) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    qs_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = QS_GATE_SWAP;
    g.t = a;
    g.t2 = b;
    g.param = -1;
    return qs_apply_gate(s, &g);
}

static qs_status plan_create(int n, qs_dtype dt, const qs_gate *g, size_t m, const qs_exec_opts *opts,
                             qs_plan **out, bool temp) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_ERANGE, "n out of range");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    if (m > 0 && !g) return fail(QS_EINVAL, "gates NULL");
    std::vector<HostOp> ops;
    qs_status st = synth_all(n, g, m, ops);
    if (st != QS_OK) return st;
    qs_exec_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    Plan *p = nullptr;
    st = plan_build(n, dt, ops, o, &p, temp);
    if (st != QS_OK) return st;
    *out = reinterpret_cast<qs_plan *>(p);
    return QS_OK;
}

qs_status qs_plan_create(int n, qs_dtype dt, const qs_gate *g, size_t m, const qs_exec_opts *opts, qs_plan **out) {
    return plan_create(n, dt, g, m, opts, out, false);
}

qs_status qs_plan_execute(qs_state *s, const qs_plan *plan) {
    if (!s || !plan) return fail(QS_EINVAL, "NULL argument");
    Plan *p = reinterpret_cast<Plan *>(const_cast<qs_plan *>(plan));
    if (plan_n(p) != s->n || plan_dtype(p) != s->dt) return fail(QS_EINVAL, "plan does not match the state");
    return plan_run(s, p);
}

qs_status qs_plan_describe(const qs_plan *plan, char *buf, size_t len, size_t *needed) {
    if (!plan) return fail(QS_EINVAL, "plan is NULL");
    const std::string d = plan_describe(reinterpret_cast<const Plan *>(plan));
    if (needed) *needed = d.size() + 1;
    if (buf && len) {
        const size_t k = std::min(len - 1, d.size());
        std::memcpy(buf, d.data(), k);
        buf[k] = 0;
    }
    return QS_OK;
}

qs_status qs_plan_set_timing(qs_plan *plan, int enable) {
    if (!plan) return fail(QS_EINVAL, "plan is NULL");
    return plan_set_timing(reinterpret_cast<Plan *>(plan), enable != 0);
}

qs_status qs_plan_timing(qs_plan *plan, double *kernel_ms, int64_t *n_launches) {
    if (!plan) return fail(QS_EINVAL, "plan is NULL");
    return plan_timing(reinterpret_cast<Plan *>(plan), kernel_ms, n_launches);
}

qs_status qs_plan_info(const qs_plan *plan, int64_t *n_launches, int64_t *n_gates) {
    if (!plan) return fail(QS_EINVAL, "plan is NULL");
    plan_counts(reinterpret_cast<const Plan *>(plan), n_launches, n_gates);
    return QS_OK;
}

qs_status qs_plan_free(qs_plan *plan) {
    if (plan) plan_destroy(reinterpret_cast<Plan *>(plan));
    return QS_OK;
}

qs_status qs_apply_circuit(qs_state *s, const qs_gate *g, size_t m, const qs_exec_opts *opts) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    qs_plan *p = nullptr;
    qs_status st = plan_create(s->n, s->dt, g, m, opts, &p, true);
    if (st != QS_OK) return st;
    st = qs_plan_execute(s, p);
    qs_plan_free(p);   // its gate table is released in stream order
    return st;
}

// Runs a reduction and copies its (re, im) result to the host.
static qs_status reduce_to_host(qs_state *s, int kind, uint64_t a0, uint64_t a1, const void *other,
                                double *re, double *im) {
    cudaError_t e = launch_reduce(s, kind, a0, a1, other);
    if (e != cudaSuccess) return cuda_fail(e, "reduction launch");
    e = cudaMemcpyAsync(s->host_result, s->result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduction copy");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduction");
    if (re) *re = s->host_result[0];
    if (im) *im = s->host_result[1];
    return QS_OK;
}

qs_status qs_prob(qs_state *s, uint64_t index, double *out) {
    if (!s || !out) return fail(QS_EINVAL, "NULL argument");
    if (index >> s->n) return fail(QS_ERANGE, "index >= 2^n");
    return reduce_to_host(s, RED_PROB_INDEX, index, 0, nullptr, out, nullptr);
}

qs_status qs_prob_qubit(qs_state *s, int q, double *p1) {
    if (!s || !p1) return fail(QS_EINVAL, "NULL argument");
    if (q < 0 || q >= s->n) return fail(QS_EINVAL, "qubit out of range");
    return reduce_to_host(s, RED_PROB_BIT, uint64_t(1) << (s->n - 1 - q), 0, nullptr, p1, nullptr);
}

qs_status qs_expect(qs_state *s, const char *pauli, double *out) {
    if (!s || !pauli || !out) return fail(QS_EINVAL, "NULL argument");
    if (std::strlen(pauli) != size_t(s->n)) return fail(QS_EINVAL, "Pauli string length must equal n");
    uint64_t flip = 0, sign = 0;
    int ny = 0;
    for (int q = 0; q < s->n; ++q) {
        const uint64_t b = uint64_t(1) << (s->n - 1 - q);
        switch (pauli[q]) {
        case 'I': break;
        case 'X': flip |= b; break;
        case 'Y': flip |= b; sign |= b; ++ny; break;
        case 'Z': sign |= b; break;
        default: return fail(QS_EINVAL, "Pauli string characters must be I, X, Y or Z");
        }
    }
    // P|i> = i^{#Y} (-1)^{popcount(i & sign)} |i ^ flip>
    const uint64_t a1 = sign | (uint64_t(ny & 3) << 62);
    return reduce_to_host(s, RED_PAULI, flip, a1, nullptr, out, nullptr);
}

qs_status qs_inner(qs_state *a, qs_state *b, qs_c128 *out) {
    if (!a || !b || !out) return fail(QS_EINVAL, "NULL argument");
    if (a->n != b->n || a->dt != b->dt) return fail(QS_EINVAL, "states differ in size or dtype");
    if (a->device != b->device) return fail(QS_EINVAL, "states are on different devices");
    if (a->stream != b->stream) return fail(QS_EINVAL, "states are on different streams");
    return reduce_to_host(a, RED_INNER, 0, 0, b->d, &out->re, &out->im);
}

qs_status qs_norm(qs_state *s, double *out) {
    if (!s || !out) return fail(QS_EINVAL, "NULL argument");
    return reduce_to_host(s, RED_NORM, 0, 0, nullptr, out, nullptr);
}

qs_status qs_renormalize(qs_state *s) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    cudaError_t e = launch_reduce(s, RED_NORM, 0, 0, nullptr);
    if (e == cudaSuccess) e = launch_scale(s, s->result);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "renormalize");
}

qs_status qs_copy_out(qs_state *s, void *host, size_t bytes) {
    if (!s || !host) return fail(QS_EINVAL, "NULL argument");
    if (bytes != (amp_size(s->dt) << s->n)) return fail(QS_ERANGE, "byte count does not match the state");
    cudaError_t e = cudaMemcpyAsync(host, s->d, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "copy_out");
}

qs_status qs_copy_out_async(qs_state *s, void *host, size_t bytes) {
    if (!s || !host) return fail(QS_EINVAL, "NULL argument");
    if (bytes != (amp_size(s->dt) << s->n)) return fail(QS_ERANGE, "byte count does not match the state");
    const cudaError_t e = cudaMemcpyAsync(host, s->d, bytes, cudaMemcpyDeviceToHost, s->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "copy_out_async");
}

qs_status qs_sync(qs_state *s) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    const cudaError_t e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "sync");
}

qs_status qs_copy_in(qs_state *s, const void *host, size_t bytes) {
    if (!s || !host) return fail(QS_EINVAL, "NULL argument");
    if (bytes != (amp_size(s->dt) << s->n)) return fail(QS_ERANGE, "byte count does not match the state");
    cudaError_t e = cudaMemcpyAsync(s->d, host, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "copy_in");
}

}  // extern "C"
