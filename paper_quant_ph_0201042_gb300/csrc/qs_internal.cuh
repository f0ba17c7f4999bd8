// Internal definitions shared by the translation units of libqsim.
//
// Vocabulary (quant-ph/0201042, Sec. 2.2): a gate on qubit q acts on index
// bit b = n-1-q (qubit 0 is the most significant bit); the partner stride is
// 2^b.  Control conditions are kept as (mask, value) pairs over index bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qsim.h"

namespace qs {

// ---------------------------------------------------------------------------
// Complex helpers (interleaved re, im)
// ---------------------------------------------------------------------------
template <typename R> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename R> using cplx = typename cplx_t<R>::type;

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R re, R im) { cplx<R> c; c.x = re; c.y = im; return c; }

// a*x + b*y with complex a, b, x, y (8 real multiply-adds)
template <typename R>
__device__ __forceinline__ cplx<R> cmad2(cplx<R> a, cplx<R> x, cplx<R> b, cplx<R> y) {
    R re = a.x * x.x;
    re = fma(-a.y, x.y, re);
    re = fma(b.x, y.x, re);
    re = fma(-b.y, y.y, re);
    R im = a.x * x.y;
    im = fma(a.y, x.x, im);
    im = fma(b.x, y.y, im);
    im = fma(b.y, y.x, im);
    return mk<R>(re, im);
}

template <typename R>
__device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> x) {
    return mk<R>(fma(a.x, x.x, -a.y * x.y), fma(a.x, x.y, a.y * x.x));
}

// a*x + b*y with real a, b (4 real multiply-adds)
template <typename R>
__device__ __forceinline__ cplx<R> rmad2(R a, cplx<R> x, R b, cplx<R> y) {
    return mk<R>(fma(a, x.x, b * y.x), fma(a, x.y, b * y.y));
}

// ---------------------------------------------------------------------------
// Gate classes chosen on the host from the synthesised matrix
// ---------------------------------------------------------------------------
enum GateClass : int32_t {
    GC_GEN = 0,     // general complex 2x2
    GC_REAL = 1,    // real 2x2 (H, U_R, RY)
    GC_DIAG = 2,    // diag(d0, d1)
    GC_ANTI = 3,    // [[0, u12], [u21, 0]]
    GC_X = 4,       // [[0, 1], [1, 0]]: pure exchange (NOT, C-NOT)
    GC_PHASE = 5,   // one pattern of the target multiplied by a phase: diag(1, d1) or diag(d0, 1)
    GC_ID = 6,      // identity (skipped)
    GC_SWAP = 7     // exchange of two index bits
};

// A gate after host-side synthesis, in index-bit form.
struct HostOp {
    int32_t cls;
    int32_t bit;          // target index bit
    int32_t bit2;         // second bit (SWAP)
    int32_t phase_on;     // GC_PHASE: value of the target bit that gets the phase
    uint64_t cmask;       // control mask over index bits
    uint64_t cval;        // control values over index bits
    double u[8];          // matrix (re, im) x 4, row major
    int32_t param;        // parameter index or -1 (differentiation)
    int32_t kind;         // original qs_gate_kind
    double theta[2];
    int32_t step;         // trajectory mode: gate step whose noisy matrix and frame the op uses
    int32_t msrc;         // trajectory mode: 0 noisy matrix of `step`, 1 the fixed matrix u
};

// Trajectory mode of the fused complex64 pass (qs_fused.cu / qs_traj.cu):
// every trajectory of a group shares the pass structure; what differs per
// trajectory is each op's matrix and control values, written per
// (trajectory, op) into a TrajRec by a precompute kernel from TrajOpMeta.
struct TrajOpMeta {
    int32_t step;          // -1: a transpose (no record)
    int32_t msrc;          // 0: the trajectory's noisy matrix of `step`; 1: the fixed matrix u
    int32_t tbit;          // target index bit
    int32_t diag;          // 1: diagonal op (u[0..1] = d0, u[6..7] = d1)
    uint64_t cmask;        // control mask over index bits
    uint64_t omask;        // the controls outside the tile
    int8_t reg_src[8];     // index bit of the register-slot control r (or -1)
    int8_t thr_src[16];    // index bit of the thread-bit control t (or -1)
    double u[8];           // fixed matrix (msrc = 1)
};

struct TrajRec {           // per (trajectory, op): 48 bytes
    float2 u[4];           // matrix (diagonal ops: d0 in u[0], d1 in u[1])
    uint64_t ovx;          // XOR on the outer-bit control values
    uint16_t tvx;          // XOR on the thread-bit control values
    uint8_t rvx;           // XOR on the register-slot control values
    uint8_t pad[5];
};

// Per-state scratch for reductions.
constexpr int RED_BLOCKS = 1216;   // 152 SMs x 8
constexpr int RED_THREADS = 256;

}  // namespace qs

struct qs_state {
    int n = 0;
    qs_dtype dt = QS_C64;
    void *d = nullptr;          // amplitudes
    bool owned = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    double *partial = nullptr;  // RED_BLOCKS x 4 doubles (device)
    double *result = nullptr;   // 4 doubles (device)
    double *host_result = nullptr;  // 4 doubles (pinned host)
};

namespace qs {

// Thread-local error message handling (qsim_api.cu).
qs_status fail(qs_status st, const std::string &msg);
qs_status cuda_fail(cudaError_t e, const char *where);

// Host-side synthesis and classification (qs_api.cu).
qs_status synthesize(int n, const qs_gate &g, HostOp &op);

// Unfused kernels (qs_gates.cu).
// One unfused gate launch; ds: a complex128 state in double-single arithmetic
// (else double-precision instructions).
cudaError_t launch_op(qs_state *s, const HostOp &op, bool ds);
cudaError_t launch_init_basis(qs_state *s, uint64_t x);

// Reductions (qs_reduce.cu). Results are written to s->result on the device.
enum RedKind { RED_NORM = 0, RED_PROB_BIT = 1, RED_PAULI = 2, RED_INNER = 3, RED_PROB_INDEX = 4 };
cudaError_t launch_reduce(qs_state *s, int kind, uint64_t a0, uint64_t a1, const void *other);
cudaError_t launch_scale(qs_state *s, const double *dev_norm);

// Fused circuits (qs_fused.cu).
struct Plan;
qs_status plan_build(int n, qs_dtype dt, const std::vector<HostOp> &ops, const qs_exec_opts &o, Plan **out,
                     bool temp);
qs_status plan_run(qs_state *s, Plan *p);
qs_status plan_set_timing(Plan *p, bool on);
qs_status plan_timing(Plan *p, double *ms, int64_t *launches);
void plan_destroy(Plan *p);
void plan_counts(const Plan *p, int64_t *launches, int64_t *gates);
int plan_n(const Plan *p);

struct TrajPlan;
qs_status traj_plan_build(int n, const std::vector<HostOp> &ops, int max_ops, TrajPlan **out);
const std::vector<TrajOpMeta> &traj_plan_metas(const TrajPlan *p);
int64_t traj_plan_launches(const TrajPlan *p);
cudaError_t traj_plan_run(TrajPlan *p, float2 *states, uint32_t count, const TrajRec *recs, cudaStream_t st);
void traj_plan_destroy(TrajPlan *p);
std::string plan_describe(const Plan *p);

// The fused planner's greedy pass formation, for other fused kernels: per
// pass, its high tile bits (ascending; the five lowest index bits are always
// in the tile) and the ops it runs, as their HostOp::step values, in order.
// An op needs its target among the tile bits unless it is diagonal; controls
// may be anywhere.  Ops move ahead of others only where they commute.
struct PassGroup {
    std::vector<int> high;
    std::vector<int> idx;
};
std::vector<PassGroup> group_passes(int n, int H, int max_ops, const std::vector<HostOp> &ops);
qs_dtype plan_dtype(const Plan *p);
// A SWAP (with optional controls C) as C-NOTs CX(b->a), CX(C + a -> b), CX(b->a);
// identity ops dropped.
void expand_swap_ops(const std::vector<HostOp> &in, std::vector<HostOp> &out);
// Records a timing event around a launch when the plan's per-launch timing
// is on (qs_plan_set_timing); a no-op otherwise or for a NULL plan.
cudaError_t plan_mark(Plan *p, cudaStream_t st, bool end);

// Double-single fused passes over a complex128 state (qs_fused_ds.cu).
struct DsPlan;
qs_status ds_plan_build(int n, const std::vector<HostOp> &ops, int max_ops, bool temp, DsPlan **out);
cudaError_t ds_plan_run(DsPlan *p, double2 *state, cudaStream_t st, Plan *timing);
int64_t ds_plan_launches(const DsPlan *p);
int ds_min_qubits();   // registers smaller than the tile use the double-instruction passes
std::string ds_plan_describe(const DsPlan *p);
void ds_plan_destroy(DsPlan *p);

}  // namespace qs
