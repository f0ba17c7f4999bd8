/*
 * qsim.h -- C ABI of the GB300 state-vector simulator.
 *
 * The method is that of Niwa, Matsumoto and Imai, "General-Purpose Parallel
 * Simulator for Quantum Computing" (quant-ph/0201042):
 *   - Sec. 2.1: an n-qubit register is a vector of 2^n complex amplitudes;
 *   - Sec. 2.2.1: a single-qubit gate U on qubit q updates the amplitude
 *     pairs (x, y) = (alpha[i0], alpha[i0 + s]), s = 2^(n-1-q), bit n-1-q of
 *     i0 clear, as x' = u11 x + u12 y, y' = u21 x + u22 y; qubit 0 is the most
 *     significant bit of the index;
 *   - Sec. 2.2.2: a controlled gate updates only the pairs whose control bits
 *     hold ("many controlled bit cases" and the f-controlled gate are the
 *     same rule with more control bits);
 *   - Sec. 3: decoherence (Pauli flips) and operational errors (Gaussian
 *     deviations of gate angles), simulated as pure-state trajectories.
 *
 * Conventions for every call:
 *   - Qubit indices are in [0, n); qubit q is index bit n-1-q.  Control masks
 *     are in qubit order: bit q of ctrl_mask set means qubit q is a control,
 *     and bit q of ctrl_val is the value it must hold.
 *   - Gate matrices cross the ABI in double precision (qs_c128), row major
 *     u11, u12, u21, u22, whatever the dtype of the state; a complex64 state
 *     is updated in single precision with the matrix rounded to single.
 *   - Amplitudes are stored interleaved (re, im): 8 bytes each for QS_C64,
 *     16 bytes each for QS_C128, amplitude i at byte offset i * size.
 *   - Calls that modify a state are asynchronous on the state's stream (the
 *     legacy default stream until qs_set_stream).  Calls that return a number
 *     to the host (qs_prob, qs_norm, ...) synchronise that stream.
 *   - Every call returns a qs_status; QS_OK is 0.  On failure the state is
 *     left as it was when the error is detected on the host (argument
 *     errors), and qs_last_error() returns a message for the calling thread.
 *     No C++ exception crosses this boundary.
 *   - The library does not fall back to any CPU computation: every gate and
 *     every reduction runs in the library's CUDA kernels.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QS_OK = 0,
    QS_EINVAL = 1,        /* bad argument (qubit out of range, target among controls, ...) */
    QS_ERANGE = 2,        /* size out of range (n > QS_MAX_QUBITS, index >= 2^n, bytes mismatch) */
    QS_ENOMEM = 3,        /* device or pinned host allocation failed */
    QS_ECUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    QS_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    QS_EUNSUPPORTED = 6   /* valid request this build does not implement */
} qs_status;

typedef enum { QS_C64 = 1, QS_C128 = 2 } qs_dtype;

#define QS_MAX_QUBITS 40

typedef struct { double re, im; } qs_c128;

typedef struct qs_state qs_state;   /* opaque; created by qs_alloc / qs_wrap, released by qs_free */
typedef struct qs_plan qs_plan;     /* opaque compiled circuit; released by qs_plan_free */

/* Gate kinds.  Angles are in radians.  Paper references: H (Sec. 2.3.1),
 * U_R, U_P1, U_P2 (Sec. 3.2), Pauli X, Y, Z (Sec. 3.1). */
typedef enum {
    QS_GATE_MATRIX = 0,  /* explicit u[0..3] */
    QS_GATE_H = 1,       /* (1/sqrt 2) [[1, 1], [1, -1]] */
    QS_GATE_X = 2,       /* NOT; with one control: C-NOT */
    QS_GATE_Y = 3,
    QS_GATE_Z = 4,
    QS_GATE_UP1 = 5,     /* U_P1(theta[0]) = diag(1, e^{i phi}); controlled: the phase shift R_k */
    QS_GATE_UP2 = 6,     /* U_P2(theta[0]) = diag(e^{i phi}, 1) */
    QS_GATE_UR = 7,      /* U_R(theta[0]) = [[cos, -sin], [sin, cos]] */
    QS_GATE_URP1 = 8,    /* U_R(theta[0]) U_P1(theta[1]); H = URP1(pi/4, pi), NOT = URP1(pi/2, pi) */
    QS_GATE_RY = 9,      /* exp(-i theta[0] Y / 2) */
    QS_GATE_RZ = 10,     /* exp(-i theta[0] Z / 2) */
    QS_GATE_SWAP = 11    /* exchange qubits t and t2 */
} qs_gate_kind;

/* One gate of a circuit (112 bytes). */
typedef struct {
    int32_t kind;        /* qs_gate_kind */
    int32_t t;           /* target qubit */
    int32_t t2;          /* second qubit of QS_GATE_SWAP, otherwise ignored (set -1) */
    int32_t param;       /* index of theta[0] in a parameter vector for differentiation,
                            -1 if the gate is not differentiated; URP1 also uses param+1 */
    uint64_t ctrl_mask;  /* qubit-order control mask; must not contain t (or t2) */
    uint64_t ctrl_val;   /* required control values (bits outside ctrl_mask ignored) */
    double theta[2];     /* angles of the kind */
    qs_c128 u[4];        /* matrix of QS_GATE_MATRIX, row major; ignored otherwise */
} qs_gate;

/* Execution options of qs_apply_circuit / qs_plan_create.  A zeroed struct
 * (or NULL) selects the defaults. */
typedef struct {
    int32_t no_fusion;       /* 1: one unfused pair-sweep launch per gate (the plain
                                per-gate path); 0: fuse runs of gates into tile passes */
    int32_t max_ops_per_pass;/* 0: default */
    int32_t c128_arith;      /* arithmetic of the passes or per-gate sweeps over a
                                complex128 state: QS_ARITH_DEFAULT (0) or QS_ARITH_DS:
                                double-single (each double split into two floats carrying
                                48 significant bits; products and sums by error-free
                                transformations on the single-precision pipe; the state
                                stays complex128 in memory); QS_ARITH_F64:
                                double-precision instructions.  Fused double-single passes
                                need n >= 12 (2^12-amplitude tiles), else the passes use
                                doubles; the per-gate sweeps have no minimum. */
    int32_t reserved[5];
} qs_exec_opts;

enum { QS_ARITH_DEFAULT = 0, QS_ARITH_F64 = 1, QS_ARITH_DS = 2 };

/* --------------------------------------------------------------------- */
/* State lifetime                                                          */
/* --------------------------------------------------------------------- */

/* Allocates a 2^n-amplitude state on the current CUDA device, owned by the
 * library (freed by qs_free), and initialises it to |0...0>.
 * Errors: QS_ERANGE if n < 1 or n > QS_MAX_QUBITS, QS_EINVAL for a bad
 * dtype or NULL out, QS_ENOMEM if the device allocation fails. */
qs_status qs_alloc(int n, qs_dtype dt, qs_state **out);

/* Wraps caller-owned device memory (e.g. a torch tensor) of 2^n amplitudes
 * of dtype dt as a state.  The memory must stay valid until qs_free, which
 * never frees it; it must be 16-byte aligned.  Contents are not modified.
 * Errors: as qs_alloc, QS_EINVAL for a NULL or misaligned pointer. */
qs_status qs_wrap(void *dev_ptr, int n, qs_dtype dt, qs_state **out);

/* Releases the state (and, for qs_alloc states, its device memory) after
 * synchronising its stream.  NULL is accepted. */
qs_status qs_free(qs_state *s);

/* All later operations on s are enqueued on `stream` (a cudaStream_t; NULL
 * selects the legacy default stream). */
qs_status qs_set_stream(qs_state *s, void *stream);

/* Device pointer, qubit count and dtype of a state (any out may be NULL). */
qs_status qs_info(const qs_state *s, void **dev_ptr, int *n, qs_dtype *dt);

/* --------------------------------------------------------------------- */
/* Evolution steps, Sec. 2.2                                               */
/* --------------------------------------------------------------------- */

/* The single-gate calls below launch one pair sweep per gate.  A complex128
 * state is updated in double-single arithmetic: each amplitude's doubles are
 * split into float pairs carrying 48 significant bits, the update runs on the
 * single-precision pipe by error-free products and sums, and the results are
 * joined back into doubles (a relative error of a few 2^-48 per gate, against
 * 2^-53 for double-precision instructions).  qs_apply_circuit with
 * no_fusion = 1 and c128_arith = QS_ARITH_F64 runs the same sweeps with
 * double-precision instructions. */

/* |x>: amplitude x set to 1, all others to 0.  QS_ERANGE if x >= 2^n. */
qs_status qs_init_basis(qs_state *s, uint64_t x);

/* Single-qubit gate U on qubit q (Sec. 2.2.1): every pair (i0, i0 + 2^(n-1-q))
 * is updated in place by one thread that reads both amplitudes before it
 * writes either.  QS_EINVAL if q is out of range or U is NULL. */
qs_status qs_apply_1q(qs_state *s, int q, const qs_c128 U[4]);

/* Controlled gate (Sec. 2.2.2): U on target t for the pairs whose control
 * qubit c is 1.  QS_EINVAL if c == t or either is out of range. */
qs_status qs_apply_ctrl(qs_state *s, int c, int t, const qs_c128 U[4]);

/* Many-control gate (Sec. 2.2.2, also the f-controlled gate with f an index
 * predicate): U on target t for the pairs whose control qubits (ctrl_mask)
 * hold the values ctrl_val.  Only the matching pairs are visited, so a gate
 * with n-1 controls touches two amplitudes.  QS_EINVAL if ctrl_mask contains
 * t or a qubit >= n. */
qs_status qs_apply_mctrl(qs_state *s, uint64_t ctrl_mask, uint64_t ctrl_val, int t,
                         const qs_c128 U[4]);

/* SWAP of qubits a and b (a != b). */
qs_status qs_apply_swap(qs_state *s, int a, int b);

/* One gate of any kind, unfused. */
qs_status qs_apply_gate(qs_state *s, const qs_gate *g);

/* Applies the m gates in order.  With fusion (the default) consecutive gates
 * are grouped into passes that each read and write the state once: a pass
 * keeps a tile of 2^k amplitudes (the low index bits plus a chosen set of
 * high bits) in registers and shared memory and applies every gate of the
 * group to it.  Gates are validated and copied before the call returns. */
qs_status qs_apply_circuit(qs_state *s, const qs_gate *g, size_t m, const qs_exec_opts *opts);

/* Compiles a circuit for n qubits and dtype dt once (validation, fusion
 * planning, gate tables uploaded to the device) so that it can be executed
 * many times.  The plan is bound to the device that was current. */
qs_status qs_plan_create(int n, qs_dtype dt, const qs_gate *g, size_t m,
                         const qs_exec_opts *opts, qs_plan **out);

/* Executes a plan on a state of matching n and dtype, on the state's stream.
 * QS_EINVAL on a size or dtype mismatch. */
qs_status qs_plan_execute(qs_state *s, const qs_plan *p);

/* Number of kernel launches one execution makes and the number of gates;
 * either pointer may be NULL. */
qs_status qs_plan_info(const qs_plan *p, int64_t *n_launches, int64_t *n_gates);

qs_status qs_plan_free(qs_plan *p);

/* Writes a human-readable description of the plan into buf (NUL-terminated,
 * truncated to len bytes); *needed (may be NULL) receives the full length + 1.
 * Fused plans: one line per pass (tile bits, op counts by kind, transposes),
 * each followed by "  order=<i,...>", the pass's ops in execution order as
 * indices into the planned op list; then one line per planned op (a SWAP
 * appears as three C-NOTs):
 *   op <i> bit=<index bit> cmask=<hex> cval=<hex> u=<8 numbers, (re, im) row-major> */
qs_status qs_plan_describe(const qs_plan *p, char *buf, size_t len, size_t *needed);

/* Per-launch timing of plan executions, for roofline measurement.  While
 * enabled, qs_plan_execute records a CUDA event pair on the state's stream
 * around every kernel launch it makes; qs_plan_timing waits for the recorded
 * events, returns the summed device time (ms) and the number of timed
 * launches since the previous read, and clears them.  Disabled by default;
 * enabling allocates the events lazily (QS_ECUDA if that fails).  Not
 * thread-safe with respect to concurrent executions of the same plan. */
qs_status qs_plan_set_timing(qs_plan *p, int enable);
qs_status qs_plan_timing(qs_plan *p, double *kernel_ms, int64_t *n_launches);

/* --------------------------------------------------------------------- */
/* Reductions, accumulated in double precision for both dtypes             */
/* --------------------------------------------------------------------- */

/* |alpha_index|^2.  QS_ERANGE if index >= 2^n. */
qs_status qs_prob(qs_state *s, uint64_t index, double *out);

/* Probability that qubit q reads 1. */
qs_status qs_prob_qubit(qs_state *s, int q, double *p1);

/* <psi| P |psi> for the Pauli string P: exactly n characters from
 * {'I','X','Y','Z'}, character q acting on qubit q.  QS_EINVAL otherwise. */
qs_status qs_expect(qs_state *s, const char *pauli, double *out);

/* <a|b> = sum_i conj(a_i) b_i.  a and b must have the same n and dtype, live
 * on the same device and use the same stream.  QS_EINVAL otherwise, before
 * anything is launched. */
qs_status qs_inner(qs_state *a, qs_state *b, qs_c128 *out);

/* sum_i |alpha_i|^2. */
qs_status qs_norm(qs_state *s, double *out);

/* Divides the state by the square root of its (double precision) norm. */
qs_status qs_renormalize(qs_state *s);

/* Measurement gate (Sec. 2.2.3), one outcome per random number: out[k] is the
 * index i with sum_{j<i} |alpha_j|^2 <= r[k] < sum_{j<=i} |alpha_j|^2, sums
 * in double precision (chunked; a sequential sum can differ from it by
 * rounding, which matters only when r[k] lies within that rounding of a
 * boundary).  An r at or beyond the total (rounding) gives the last index
 * with non-zero probability.  r: `shots` host doubles in [0, 1), else
 * QS_EINVAL; out: `shots` host indices.  The state is not collapsed.
 * At most 2^26 shots per call (QS_ERANGE).  Synchronous. */
qs_status qs_measure(qs_state *s, const double *r, size_t shots, uint64_t *out);

/* Quantum Fourier transform as a black-box operator (Sec. 2.3.2: the paper
 * replaces the QFT circuit by a classical FFT when the circuit is taken to be
 * error free): on the L qubits q0 .. q0+L-1, qubit q0 the most significant of
 * that register and the other qubits spectators,
 *     beta_x = 2^{-L/2} sum_y w^{x y} alpha_y,  w = e^{2 pi i / 2^L}
 * (inverse != 0: w = e^{-2 pi i / 2^L}, the adjoint).  With q0 = 0, L = n it
 * equals the QFT circuit of Sec. 2.3.2 including its final qubit reversal.
 * In place, in the state's precision (twiddles from double-precision
 * tables).  Needs 0 <= q0, 1 <= L, q0 + L <= n, else QS_EINVAL.
 * Asynchronous on the state's stream; allocates a small twiddle table
 * (2^12 + 2^ceil(L/2) + 2^floor(L/2) complex entries) with the stream-ordered
 * allocator for the duration of the call (QS_ECUDA if that fails). */
qs_status qs_qft(qs_state *s, int q0, int L, int inverse);

/* Norm of a state without any allocation, for callers that cannot allocate
 * device memory at the point they need it (a framework that owns the whole
 * device memory budget through its own pool, a latency-critical loop in which
 * cudaMalloc/cudaFree would synchronize the device, a component that may not
 * call the allocator at all).  The paper has no counterpart: this is a
 * service of the library, not a step of the method.
 *
 * dev_state: 2^n amplitudes of dtype dt in device memory (16-byte aligned
 * for QS_C128, 8-byte for QS_C64); dev_out: one 8-byte aligned double in
 * device memory that receives sum_i |alpha_i|^2.  Errors, detected before
 * anything is launched: QS_EINVAL for a NULL or misaligned pointer or a bad
 * dtype, QS_ERANGE for n < 1 or n > 32.
 * The call is enqueued on `stream` (NULL: legacy default stream) and returns
 * without waiting.  It calls no cudaMalloc, cudaFree or other allocating
 * routine: its partial sums (one per 2^16 amplitudes) live in a fixed
 * 1 MiB array of this library's device memory, which every GPU that loads
 * the library holds until the process exits.  Limit: n <= 32; larger n
 * returns QS_ERANGE.  The first call on a device resolves the array's
 * address (cudaGetSymbolAddress) with that device current, so make it before
 * any stream capture.  All calls share the array: calls that overlap on the
 * GPU (different streams, no ordering between them) race and may return
 * wrong sums; order them on one stream or with events.  The sum is
 * deterministic for a given n but may differ from qs_norm's in the last bits
 * (the two reductions add in different orders).  The cached array address
 * does not survive cudaDeviceReset: do not use the entry point across one. */
qs_status qs_norm_noalloc(const void *dev_state, int n, qs_dtype dt, double *dev_out, void *stream);

/* --------------------------------------------------------------------- */
/* Noisy trajectories, Sec. 3 (error model) and Sec. 4.3.1 / 5.2 / 5.3     */
/* (pure-state Monte Carlo: each run draws its own errors; the paper       */
/* averages 1000-10000 runs)                                                */
/* --------------------------------------------------------------------- */

/* Error model of a batch.
 *   p      probability of a flip per qubit per noisy step (Sec. 3.1)
 *   sigma  standard deviation (rad) of the Gaussian deviation added to every
 *          gate angle (Sec. 3.2); gates without angles (MATRIX, SWAP, H, X,
 *          Y, Z) are not deviated: write H as URP1(pi/4, pi) and NOT as
 *          URP1(pi/2, pi) to deviate them as the paper does
 *   mode   QS_NOISE_FLIPS: a flip is X or Z with equal probability;
 *          QS_NOISE_DEPOLARIZING: X, Y or Z with equal probability (the
 *          depolarizing channel of Sec. 3.1)
 *   every  flips are drawn after gate step s when (s + 1) % every == 0
 *          (1: after every gate; n: once per Hadamard layer of n gates) */
typedef struct {
    double p;
    double sigma;
    int32_t mode;
    int32_t every;
} qs_noise;

enum { QS_NOISE_FLIPS = 0, QS_NOISE_DEPOLARIZING = 1 };

/* Execution options of qs_run_trajectories (NULL: defaults).
 *   no_fusion         1: one launch per gate step with the flips applied to
 *                     the states (the plain batched path); 0 (default): for
 *                     complex64 groups of 10 qubits or more, fused passes over
 *                     all trajectories, the flips carried as a Pauli frame per
 *                     trajectory and folded into the later gates
 *   max_ops_per_pass  fusion depth of the fused path; 0: chosen by timing a
 *                     few candidate depths on a small batch (cached per shape) */
typedef struct {
    int32_t no_fusion;
    int32_t max_ops_per_pass;
    int32_t reserved[6];
} qs_traj_opts;
enum { QS_TRAJ_FIDELITY = 0, QS_TRAJ_PROB = 1 };

/* A group of trajectories that run the same circuit on the same width.
 *   metric  QS_TRAJ_FIDELITY: |<U x0 | psi>|^2, the fidelity to the noiseless
 *           output of the same circuit (Sec. 5.2); QS_TRAJ_PROB: |<target|psi>|^2
 *           (the amplitude of the marked element, Sec. 5.3)
 *   first   id of the group's first trajectory; trajectory first + i draws
 *           from the Philox4x32-10 stream with counter word 0 = first + i
 *   x0      initial basis index of each of the `count` trajectories
 *   flags   NULL, or one byte per gate: QS_TRAJ_NO_DEVIATION (its angles are
 *           not deviated), QS_TRAJ_NO_FLIPS (no flips are drawn after it).
 *           A noiseless state preparation is a prefix of gates with both
 *           flags; the QFT experiment of Sec. 5.2 (decoherence after each
 *           phase shift R_d only) sets QS_TRAJ_NO_FLIPS on the other gates.
 *           Flags change no counter: the draws of the other gates are the
 *           same as without them. */
enum { QS_TRAJ_NO_DEVIATION = 1, QS_TRAJ_NO_FLIPS = 2 };
typedef struct {
    int32_t n;
    int32_t metric;
    uint64_t target;
    const qs_gate *gates;
    size_t m;
    uint32_t first;
    uint32_t count;
    const uint64_t *x0;
    const uint8_t *flags;
} qs_traj_group;

/* Runs every trajectory of every group on the current device and writes the
 * metric of trajectory k of group g to metric[offset_g + k], offset_g being
 * the sum of the counts of the groups before g.  Random draws (Philox4x32-10,
 * key = seed, counter (trajectory, step, slot, stream)):
 *   flip on qubit q after step s: block (traj, s, q, 0); flip iff word 0 <
 *     floor(p 2^32); kind from word 1 (flips mode: X if even, Z if odd;
 *     depolarizing: (word1 * 3) >> 32 = 0, 1, 2 for X, Y, Z);
 *   deviation of angle a of step s: block (traj, s, 64 + a, 1); Box-Muller
 *     g = sqrt(-2 ln u1) cos(2 pi u2) with u1 = 1 - (w0:w1 >> 11) 2^-53 and
 *     u2 = (w2:w3 >> 11) 2^-53.
 * stats (may be NULL) receives 4 words per trajectory: the numbers of X, Y and
 * Z flips and the sum (mod 2^64) over flip events of the SplitMix64 finalizer
 * of (s * 64 + q) * 4 + kind (kind 1, 2, 3 = X, Y, Z).  dt selects the state
 * precision; draws and gate synthesis are in double precision.  Synchronous
 * (returns when the results are on the host).  Device memory: the states of
 * all trajectories of the largest group (count x 2^n amplitudes) plus
 * per-step tables; QS_ENOMEM if it cannot be allocated.  opts (may be NULL)
 * selects the fused or the plain path and the fusion depth. */
qs_status qs_run_trajectories(const qs_traj_group *groups, int n_groups, const qs_noise *noise, uint64_t seed,
                              qs_dtype dt, const qs_traj_opts *opts, double *metric, uint64_t *stats);

/* --------------------------------------------------------------------- */
/* Gradients by the adjoint (reverse) sweep                                */
/* --------------------------------------------------------------------- */

enum { QS_OBS_PAULI = 0, QS_OBS_FIDELITY = 1 };

/* Cost whose gradient is taken.
 *   QS_OBS_PAULI     E = <psi| P |psi> for the Pauli string `pauli` (n
 *                    characters from I, X, Y, Z, character q on qubit q)
 *   QS_OBS_FIDELITY  E = |<phi|psi>|^2 with phi the state `ref` (same n and
 *                    dtype as the workspace, on the same stream) */
typedef struct {
    int32_t kind;
    int32_t pad;
    const char *pauli;
    const qs_state *ref;
} qs_observable;

/* Runs the circuit g[0..m-1] from |0...0> on the workspace s, with every gate
 * whose `param` is >= 0 taking theta[0] = params[param] (and, for URP1,
 * theta[1] = params[param + 1]); writes E to *value and dE/dparams to
 * grad[0..n_params-1] (parameters no gate uses get 0).  The gradient comes
 * from one reverse sweep: with lambda = O psi (or phi <phi|psi>), each
 * parameterised gate U_j contributes 2 Re <lambda_j| (dU_j U_j^dagger) |psi_j>,
 * then psi and lambda are uncomputed with U_j^dagger, so no intermediate
 * state is stored.  A deviated angle theta + x has the same derivative with
 * respect to x as with respect to theta.  Differentiable kinds: RY, RZ, UR,
 * UP1, UP2, URP1 (QS_EUNSUPPORTED for a parameter on another kind).  On
 * return the workspace holds the uncomputed state (close to |0...0>).  Uses
 * one extra state-sized buffer and per-gate partial sums.  Synchronous. */
qs_status qs_adjoint_grad(qs_state *s, const qs_gate *g, size_t m, const double *params, size_t n_params,
                          const qs_observable *obs, double *value, double *grad);

/* qs_adjoint_grad with execution options (NULL: defaults).  By default the
 * reverse sweep is fused: consecutive steps whose targets lie in a tile of
 * 2^12 (complex64) / 2^11 (complex128) amplitudes run tile by tile with psi
 * and lambda in shared memory (one HBM round trip of both vectors per group
 * of steps); opts->no_fusion = 1 runs one sweep of both vectors per step.
 * Registers of fewer than 6 qubits always use the per-step sweep.  The two
 * paths give the same gradient up to rounding (the order of the partial sums
 * differs). */
qs_status qs_adjoint_grad_ex(qs_state *s, const qs_gate *g, size_t m, const double *params, size_t n_params,
                             const qs_observable *obs, double *value, double *grad, const qs_exec_opts *opts);

/* Host-side plan of the fused reverse sweep that qs_adjoint_grad would run for
 * this circuit on an n-qubit state of dtype dt.  It needs no GPU and uses the
 * gates' own angles (theta).  Writes text into buf (NUL-terminated, truncated
 * to len bytes); *needed (may be NULL) receives the full length + 1.  Lines:
 *   step <j> cls=<gen|real|diag|x> bit=<index bit> cmask=<hex> cval=<hex> u=<8 numbers>
 *     one per reverse step in forward order (a SWAP gives three C-NOT steps);
 *     u is the step's forward matrix, (re, im) row-major
 *   pass <p> tile=<index bits of the tile, ascending>
 *   run bit=<index bit, or -1 for diagonal steps only> pre=<k> steps=<j,...>
 *     the pass's runs in sweep order; the first k steps of a run are exchanges
 * No pass lines for n < 6 (the per-step sweep runs there).
 * Errors: QS_ERANGE for n out of range, QS_EINVAL for a bad dtype or NULL
 * gates with m > 0, QS_EUNSUPPORTED for a gate the adjoint cannot take. */
qs_status qs_adjoint_describe(int n, qs_dtype dt, const qs_gate *g, size_t m, char *buf, size_t len, size_t *needed);

/* --------------------------------------------------------------------- */
/* A register partitioned over 2^g ranks (Sec. 2.2.1: the overall matrix    */
/* splits into independent blocks M_k = S_k phi_k, spread here over GPUs)   */
/* --------------------------------------------------------------------- */

/* Partition: qubits 0 .. g-1 (the g most significant index bits) are
 * "global" and name the rank; rank r holds the 2^(n-g) amplitudes whose top
 * g bits equal r, as a state of n-g qubits (its qubit j is qubit g+j of the
 * register).
 *
 * qs_shard_plan rewrites gates g[0..m-1] (qubits of the register) into the
 * physical numbering of the partition: an uncontrolled SWAP of the circuit
 * renames qubits (no data moves), a controlled SWAP becomes three C-NOTs,
 * and before every non-diagonal gate whose target sits on a global qubit an
 * exchange is inserted: an uncontrolled QS_GATE_SWAP with t < g <= t2, which
 * swaps the global qubit t with the local qubit t2 (the local qubit chosen
 * is the one whose next non-diagonal use lies furthest ahead).  Every other
 * output gate has the input's kind, angles and matrix with its qubits
 * renamed; its controls may be global, and its target is global only for a
 * diagonal gate.  final_pos (n entries, may be NULL) receives the physical
 * qubit of each logical qubit after the last gate.  out may be NULL (count
 * only); *n_out receives the number of output gates, and QS_ERANGE is
 * returned if it exceeds max_out.  Needs n - g >= 2 (QS_ERANGE), valid gates
 * (QS_EINVAL).  Host only: no GPU needed.
 *
 * An exchange SWAP(t, t2) on rank r, with b = bit (g-1-t) of r and partner
 * r ^ (1 << (g-1-t)): the rank sends the half of its slice whose local qubit
 * t2-g equals 1-b and receives the partner's half (whose local qubit equals
 * b on the partner) into the same places, i.e. qs_shard_pack(s, t2-g, 1-b,
 * send), transport, qs_shard_unpack(s, t2-g, 1-b, recv).
 *
 * qs_shard_localize converts physical gates without exchanges (a stretch
 * between two of them) into rank `rank`'s gates on its (n-g)-qubit slice:
 * gates whose global controls this rank does not meet are dropped, global
 * controls it meets are removed, a diagonal gate on a global qubit becomes
 * the scalar (its entry for this rank's bit) on the slice's amplitudes that
 * meet the local controls (a QS_GATE_MATRIX diag(d, d), or diag on a control
 * qubit if every local qubit is a control); entries exactly 1 are dropped.
 * QS_EINVAL for an exchange or a non-diagonal gate on a global qubit.
 * Output sizing as for qs_shard_plan.  Host only. */
qs_status qs_shard_plan(int n, int g, const qs_gate *gates, size_t m, qs_gate *out, size_t max_out, size_t *n_out,
                        int32_t *final_pos);
qs_status qs_shard_localize(int n, int g, uint32_t rank, const qs_gate *in, size_t m, qs_gate *out, size_t max_out,
                            size_t *n_out);

/* Copies the 2^(n-1) amplitudes of s whose qubit q equals value (0 or 1), in
 * index order, into the device buffer dev_buf (qs_shard_pack), or writes
 * them back from it (qs_shard_unpack); asynchronous on the state's stream.
 * dev_buf must hold 2^(n-1) amplitudes of the state's dtype and be aligned
 * to one amplitude (QS_EINVAL otherwise, and for q out of range). */
qs_status qs_shard_pack(qs_state *s, int q, int value, void *dev_buf);
qs_status qs_shard_unpack(qs_state *s, int q, int value, const void *dev_buf);

/* --------------------------------------------------------------------- */
/* Host copies (checkpoint / restore)                                      */
/* --------------------------------------------------------------------- */

/* Copies the whole state to / from host memory (pinned or pageable).  bytes
 * must equal 2^n times the amplitude size, else QS_ERANGE.  Synchronous. */
qs_status qs_copy_out(qs_state *s, void *host, size_t bytes);
qs_status qs_copy_in(qs_state *s, const void *host, size_t bytes);

/* Enqueues the copy of the whole state to host memory on the state's stream
 * and returns without waiting: the host buffer holds the state once qs_sync(s)
 * (or a synchronisation of that stream) returns, and must stay valid until
 * then.  With page-locked (pinned) host memory the copy overlaps work on other
 * streams; pageable memory makes it synchronous.  bytes as for qs_copy_out
 * (QS_ERANGE otherwise); QS_EINVAL for NULL arguments. */
qs_status qs_copy_out_async(qs_state *s, void *host, size_t bytes);

/* Waits for all work enqueued on the state's stream; QS_ECUDA with the
 * message of an asynchronous failure. */
qs_status qs_sync(qs_state *s);

/* --------------------------------------------------------------------- */
/* Measurement service (no counterpart in the paper)                       */
/* --------------------------------------------------------------------- */

/* Measured rate of fused multiply-add instructions on the current device,
 * in lane operations per second (kind 0: single precision, kind 1: double
 * precision): a kernel of sixteen independent FMA chains per thread on eight
 * 256-thread CTAs per SM on a stream of its own, the best of five launches
 * timed with CUDA events after about 200 ms of the same launches (so that
 * the SM clock has left its idle level).  These are the denominators of the
 * arithmetic rooflines.  Synchronous; allocates and frees a small sink
 * buffer and a stream.  Changes no device setting. */
qs_status qs_alu_peak(int kind, double *fma_per_s);

/* Thread-local message describing the last failure of this thread. */
const char *qs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
