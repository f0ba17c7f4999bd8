/*
 * qs_oracle.c -- plain complex128 CPU oracle for the state-vector method of
 * Niwa, Matsumoto and Imai, "General-Purpose Parallel Simulator for Quantum
 * Computing" (quant-ph/0201042).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Everything here is the plain definition, written for a reader checking it
 * against the paper by eye:
 *   - the register is 2^n complex amplitudes in double precision (Sec. 2.1);
 *   - qubit 0 is the most significant bit of the amplitude index (Sec. 2.2.1),
 *     so qubit q is index bit n-1-q;
 *   - a gate is applied row by row from the definition of the overall matrix:
 *     row j of X has two non-zeros (the block S_k of the "Total unitary
 *     matrix" figure, Sec. 2.2.1), and row j of CTX is row j of X when the
 *     control bits of j hold and the identity row otherwise (Sec. 2.2.2).
 *     Every new amplitude is computed from a copy of the old vector
 *     (out-of-place), so the in-place ordering hazard described in
 *     Sec. 2.2.1 cannot occur here by construction;
 *   - gates are synthesised from the rotation U_R and phase shifts U_P1,
 *     U_P2 of Sec. 3.2, the Hadamard matrix of Sec. 2.3.1 and the Pauli
 *     matrices of Sec. 3.1;
 *   - noisy trajectories follow the error model of Sec. 3 (depolarizing or
 *     bit/phase flips after a gate step, Gaussian deviations of gate angles),
 *     with the flips applied to the state physically, after the gate;
 *   - random draws come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), implemented here
 *     from that paper's definition.
 *
 * Pins (tests/test_oracle_*.py): dense Kronecker-product matrices for n<=8,
 * the closed-form QFT of a basis state, the Hadamard transform formula,
 * Grover's closed-form state, the one-qubit density-matrix recursions of
 * Sec. 4.3.1, curand's host Philox generator, parameter-shift vs central
 * finite differences.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Gate description (the oracle's own; the CUDA library has a separate one).  */
/* ------------------------------------------------------------------------- */
enum {
    OR_MATRIX = 0, /* explicit 2x2 matrix m[] (row major, re/im interleaved) */
    OR_H = 1,      /* Hadamard, Sec. 2.3.1 */
    OR_X = 2,      /* sigma_x */
    OR_Y = 3,      /* sigma_y */
    OR_Z = 4,      /* sigma_z */
    OR_UP1 = 5,    /* U_P1(angle0) = diag(1, e^{i phi}), Sec. 3.2 */
    OR_UP2 = 6,    /* U_P2(angle0) = diag(e^{i phi}, 1), Sec. 3.2 */
    OR_UR = 7,     /* U_R(angle0) = [[cos, -sin], [sin, cos]], Sec. 3.2 */
    OR_URP1 = 8,   /* U_R(angle0) U_P1(angle1): the paper's synthesis of H and NOT */
    OR_RY = 9,     /* exp(-i angle0 Y / 2) */
    OR_RZ = 10,    /* exp(-i angle0 Z / 2) */
    OR_SWAP = 11   /* exchange qubits target and target2 */
};

typedef struct {
    int32_t kind;
    int32_t target;
    int32_t target2;
    int32_t param;          /* index of angle0 in a parameter vector, -1 if none */
    uint64_t ctrl_mask;     /* bit q set: qubit q is a control */
    uint64_t ctrl_val;      /* required value of each control qubit */
    double angle[2];
    double m[8];            /* OR_MATRIX: u11, u12, u21, u22 as (re, im) */
} or_gate;

/* Number of angles a gate kind carries (the angles an operational error
 * perturbs, Sec. 3.2). */
int or_gate_n_angles(int kind)
{
    switch (kind) {
    case OR_UP1: case OR_UP2: case OR_UR: case OR_RY: case OR_RZ: return 1;
    case OR_URP1: return 2;
    default: return 0;
    }
}

/* 2x2 matrix of a gate from its kind and angles, row major u11 u12 u21 u22. */
static void gate_matrix(int kind, const double *a, const double *m, cplx U[4])
{
    const double s = 1.0 / sqrt(2.0);
    switch (kind) {
    case OR_MATRIX:
        for (int k = 0; k < 4; k++) U[k] = m[2 * k] + I * m[2 * k + 1];
        break;
    case OR_H:   /* (1/sqrt 2) [[1, 1], [1, -1]] */
        U[0] = s; U[1] = s; U[2] = s; U[3] = -s;
        break;
    case OR_X:
        U[0] = 0; U[1] = 1; U[2] = 1; U[3] = 0;
        break;
    case OR_Y:
        U[0] = 0; U[1] = -I; U[2] = I; U[3] = 0;
        break;
    case OR_Z:
        U[0] = 1; U[1] = 0; U[2] = 0; U[3] = -1;
        break;
    case OR_UP1:
        U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(I * a[0]);
        break;
    case OR_UP2:
        U[0] = cexp(I * a[0]); U[1] = 0; U[2] = 0; U[3] = 1;
        break;
    case OR_UR:
        U[0] = cos(a[0]); U[1] = -sin(a[0]); U[2] = sin(a[0]); U[3] = cos(a[0]);
        break;
    case OR_URP1: {
        /* product of U_R(theta) and U_P1(phi): multiply the two matrices */
        cplx R[4] = { cos(a[0]), -sin(a[0]), sin(a[0]), cos(a[0]) };
        cplx P[4] = { 1, 0, 0, cexp(I * a[1]) };
        U[0] = R[0] * P[0] + R[1] * P[2];
        U[1] = R[0] * P[1] + R[1] * P[3];
        U[2] = R[2] * P[0] + R[3] * P[2];
        U[3] = R[2] * P[1] + R[3] * P[3];
        break;
    }
    case OR_RY:  /* cos(t/2) I - i sin(t/2) Y */
        U[0] = cos(a[0] / 2); U[1] = -sin(a[0] / 2);
        U[2] = sin(a[0] / 2); U[3] = cos(a[0] / 2);
        break;
    case OR_RZ:  /* diag(e^{-i t/2}, e^{i t/2}) */
        U[0] = cexp(-I * a[0] / 2); U[1] = 0; U[2] = 0; U[3] = cexp(I * a[0] / 2);
        break;
    default:
        U[0] = U[1] = U[2] = U[3] = NAN;
    }
}

/* Exported for tests: matrix of a gate as 8 doubles. */
void or_gate_matrix(int kind, const double *angle, const double *m, double *out8)
{
    cplx U[4];
    gate_matrix(kind, angle, m, U);
    for (int k = 0; k < 4; k++) { out8[2 * k] = creal(U[k]); out8[2 * k + 1] = cimag(U[k]); }
}

/* Index bit of qubit q (qubit 0 = most significant, Sec. 2.2.1). */
static inline uint64_t qbit(int n, int q) { return (uint64_t)1 << (n - 1 - q); }

/* Control mask/value in index-bit form. */
static void ctrl_bits(int n, uint64_t qmask, uint64_t qval, uint64_t *cm, uint64_t *cv)
{
    *cm = 0; *cv = 0;
    for (int q = 0; q < n; q++) {
        if ((qmask >> q) & 1) {
            *cm |= qbit(n, q);
            if ((qval >> q) & 1) *cv |= qbit(n, q);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Evolution step, Sec. 2.2.1 / 2.2.2.                                        */
/* ------------------------------------------------------------------------- */

/* psi <- CTX psi, where X = I x..x U (on qubit t) x..x I and row j of CTX is
 * row j of X if every control bit of j holds, else row j of the identity.
 * Row j of X: with b the index bit of qubit t, the two non-zeros of row j sit
 * at columns j0 = j with bit b cleared and j1 = j with bit b set, and carry
 * (u11, u12) when bit b of j is 0, (u21, u22) when it is 1. */
static void apply_ctrl_u(cplx *psi, int n, int t, uint64_t cmask, uint64_t cval,
                         const cplx U[4])
{
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t b = qbit(n, t);
    cplx *old = (cplx *)malloc(N * sizeof(cplx));
    memcpy(old, psi, N * sizeof(cplx));
#pragma omp parallel for schedule(static)
    for (int64_t jj = 0; jj < (int64_t)N; jj++) {
        uint64_t j = (uint64_t)jj;
        if ((j & cmask) != cval) continue;          /* identity row */
        uint64_t j0 = j & ~b, j1 = j | b;
        if ((j & b) == 0) psi[j] = U[0] * old[j0] + U[1] * old[j1];
        else              psi[j] = U[2] * old[j0] + U[3] * old[j1];
    }
    free(old);
}

/* SWAP of qubits a and b: new amplitude j is the old amplitude at j with the
 * two index bits exchanged. */
static void apply_swap(cplx *psi, int n, int a, int b2, uint64_t cmask, uint64_t cval)
{
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t ba = qbit(n, a), bb = qbit(n, b2);
    cplx *old = (cplx *)malloc(N * sizeof(cplx));
    memcpy(old, psi, N * sizeof(cplx));
#pragma omp parallel for schedule(static)
    for (int64_t jj = 0; jj < (int64_t)N; jj++) {
        uint64_t j = (uint64_t)jj;
        if ((j & cmask) != cval) continue;
        uint64_t src = j & ~(ba | bb);
        if (j & ba) src |= bb;
        if (j & bb) src |= ba;
        psi[j] = old[src];
    }
    free(old);
}

static int gate_valid(int n, const or_gate *g)
{
    if (g->target < 0 || g->target >= n) return 0;
    if (g->kind == OR_SWAP) {
        if (g->target2 < 0 || g->target2 >= n || g->target2 == g->target) return 0;
        if ((g->ctrl_mask >> g->target2) & 1) return 0;
    }
    if ((g->ctrl_mask >> g->target) & 1) return 0;
    if (n < 64 && (g->ctrl_mask >> n) != 0) return 0;
    return 1;
}

/* Apply one gate whose angles are given separately (so a caller can perturb
 * them, Sec. 3.2).  Returns 0 on success, -1 on an invalid gate. */
static int apply_gate_angles(cplx *psi, int n, const or_gate *g, const double *angle)
{
    if (!gate_valid(n, g)) return -1;
    uint64_t cm, cv;
    ctrl_bits(n, g->ctrl_mask, g->ctrl_val, &cm, &cv);
    if (g->kind == OR_SWAP) { apply_swap(psi, n, g->target, g->target2, cm, cv); return 0; }
    cplx U[4];
    gate_matrix(g->kind, angle, g->m, U);
    apply_ctrl_u(psi, n, g->target, cm, cv, U);
    return 0;
}

/* psi is 2^n interleaved (re, im) doubles. */
int or_apply_gate(double *psi, int n, const or_gate *g)
{
    return apply_gate_angles((cplx *)psi, n, g, g->angle);
}

int or_apply_circuit(double *psi, int n, const or_gate *g, int64_t m)
{
    for (int64_t k = 0; k < m; k++)
        if (or_apply_gate(psi, n, &g[k]) != 0) return -1;
    return 0;
}

/* Basis state |x>. */
void or_init_basis(double *psi, int n, uint64_t x)
{
    const uint64_t N = (uint64_t)1 << n;
    memset(psi, 0, N * 2 * sizeof(double));
    psi[2 * x] = 1.0;
}

/* ------------------------------------------------------------------------- */
/* Reductions (plain sums in double precision).                               */
/* ------------------------------------------------------------------------- */

/* sum_i |alpha_i|^2  (the unit-length condition of Sec. 2.1) */
double or_norm2(const double *psi, int n)
{
    const cplx *a = (const cplx *)psi;
    const uint64_t N = (uint64_t)1 << n;
    double s = 0.0;
    for (uint64_t i = 0; i < N; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* |alpha_index|^2 */
double or_prob(const double *psi, int n, uint64_t index)
{
    (void)n;
    return psi[2 * index] * psi[2 * index] + psi[2 * index + 1] * psi[2 * index + 1];
}

/* probability that qubit q reads 1 */
double or_prob_qubit(const double *psi, int n, int q)
{
    const uint64_t N = (uint64_t)1 << n, b = qbit(n, q);
    double s = 0.0;
    for (uint64_t i = 0; i < N; i++)
        if (i & b) s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    return s;
}

/* <a|b> = sum_i conj(a_i) b_i, result as (re, im) */
void or_inner(const double *a, const double *b, int n, double *out2)
{
    const cplx *x = (const cplx *)a, *y = (const cplx *)b;
    const uint64_t N = (uint64_t)1 << n;
    cplx s = 0.0;
    for (uint64_t i = 0; i < N; i++) s += conj(x[i]) * y[i];
    out2[0] = creal(s); out2[1] = cimag(s);
}

/* <psi| P |psi> for a Pauli string P (one character per qubit, qubit 0
 * first, each of 'I','X','Y','Z'): apply P to a copy with the gate routine
 * above, then take the inner product. */
double or_expect_pauli(const double *psi, int n, const char *pauli)
{
    const uint64_t N = (uint64_t)1 << n;
    double *phi = (double *)malloc(N * 2 * sizeof(double));
    memcpy(phi, psi, N * 2 * sizeof(double));
    for (int q = 0; q < n; q++) {
        or_gate g;
        memset(&g, 0, sizeof g);
        g.target = q; g.target2 = -1; g.param = -1;
        switch (pauli[q]) {
        case 'X': g.kind = OR_X; break;
        case 'Y': g.kind = OR_Y; break;
        case 'Z': g.kind = OR_Z; break;
        default: continue;
        }
        or_apply_gate(phi, n, &g);
    }
    double r[2];
    or_inner(psi, phi, n, r);
    free(phi);
    return r[0];
}

/* ------------------------------------------------------------------------- */
/* Measurement gate, Sec. 2.2.3: the i with                                    */
/*   sum_{j<i} |alpha_j|^2 <= r < sum_{j<=i} |alpha_j|^2.                      */
/* ------------------------------------------------------------------------- */
uint64_t or_measure(const double *psi, int n, double r)
{
    const uint64_t N = (uint64_t)1 << n;
    double c = 0.0;
    uint64_t last = 0;
    for (uint64_t i = 0; i < N; i++) {
        double p = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
        double next = c + p;
        if (c <= r && r < next) return i;
        if (p > 0.0) last = i;
        c = next;
    }
    /* r at or beyond the rounded total: no interval contains it; the outcome
     * is the last index whose interval is not empty */
    return last;
}

/* ------------------------------------------------------------------------- */
/* Quantum Fourier transform as a black-box operator, Sec. 2.3.2:              */
/*   beta_x = 2^{-L/2} sum_y w^{x y} alpha_y,  w = e^{2 pi i / 2^L}            */
/* on the L qubits q0 .. q0+L-1 (qubit q0 the most significant of that         */
/* register; the other qubits are spectators), written as the plain double     */
/* sum (O(2^n 2^L), no fast transform).  inverse != 0 uses w^{-1}.  The         */
/* exponent x*y is reduced modulo 2^L in integers before the angle is formed.  */
/* ------------------------------------------------------------------------- */
int or_qft_dft(double *psi, int n, int q0, int L, int inverse)
{
    if (n < 1 || n > 30 || q0 < 0 || L < 1 || q0 + L > n) return -1;
    const uint64_t N = (uint64_t)1 << n, M = (uint64_t)1 << L;
    const int lo = n - q0 - L;                 /* index bit of the least significant qubit */
    const uint64_t field = (M - 1) << lo;
    const double sgn = inverse ? -1.0 : 1.0, scale = 1.0 / sqrt((double)M);
    cplx *a = (cplx *)psi;
    cplx *out = (cplx *)calloc(N, sizeof(cplx));
    cplx *w = (cplx *)malloc(M * sizeof(cplx));   /* w^e, e < 2^L */
    if (!out || !w) { free(out); free(w); return -1; }
    for (uint64_t e = 0; e < M; e++) w[e] = cexp(I * (sgn * 2.0 * M_PI * (double)e / (double)M));
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < (int64_t)N; ii++) {   /* output index i = (rest, x) */
        const uint64_t i = (uint64_t)ii;
        const uint64_t x = (i & field) >> lo, rest = i & ~field;
        cplx s = 0.0;
        for (uint64_t y = 0; y < M; y++) s += w[(x * y) & (M - 1)] * a[rest | (y << lo)];
        out[i] = s * scale;
    }
    free(w);
    memcpy(a, out, N * sizeof(cplx));
    free(out);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11).  Counter (c0..c3), key (k0, k1).     */
/* One round: multiply c0 and c2 by the two round multipliers into 64-bit      */
/* products; the new words are (hi(c2*M1) ^ c1 ^ k0, lo(c2*M1),               */
/* hi(c0*M0) ^ c3 ^ k1, lo(c0*M0)); then the key is bumped by the two Weyl    */
/* constants.  Ten rounds.                                                     */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Noisy trajectories, Sec. 3 (error model) and Sec. 4.3.1 / 5.2 / 5.3        */
/* (pure-state Monte Carlo: one run with its own random draws, averaged over  */
/* many runs).                                                                 */
/*                                                                             */
/* Draws (the counter layout, identical on every implementation):             */
/*   key = (seed low word, seed high word)                                    */
/*   flip after gate step s on qubit q : block (traj, s, q, 0)                */
/*       flip  iff word0 < floor(p * 2^32)                                    */
/*       kind  flips mode: X if word1 is even, Z if odd                       */
/*             depolarizing mode: (word1 * 3) >> 32 = 0,1,2 -> X, Y, Z        */
/*   deviation of angle a of gate step s : block (traj, s, 64 + a, 1)         */
/*       u1 = 1 - ((word0:word1) >> 11) 2^-53  in (0, 1]                      */
/*       u2 =     ((word2:word3) >> 11) 2^-53  in [0, 1)                      */
/*       g  = sqrt(-2 ln u1) cos(2 pi u2)       (Box-Muller)                  */
/*       angle a of the gate is replaced by angle + sigma * g                 */
/* ------------------------------------------------------------------------- */
enum { OR_NOISE_FLIPS = 0, OR_NOISE_DEPOLARIZING = 1 };

typedef struct {
    double p;          /* flip probability per qubit per noisy step */
    double sigma;      /* standard deviation of the angle deviations (rad) */
    int32_t mode;      /* OR_NOISE_FLIPS or OR_NOISE_DEPOLARIZING */
    int32_t every;     /* decoherence after gate step s iff (s + 1) % every == 0;
                          1 = after every gate, n = once per Hadamard layer */
} or_noise;

uint32_t or_flip_threshold(double p)
{
    double t = floor(p * 4294967296.0);
    if (t < 0) t = 0;
    if (t > 4294967295.0) t = 4294967295.0;
    return (uint32_t)t;
}

double or_gauss(uint64_t seed, uint32_t traj, uint32_t step, uint32_t a)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { traj, step, 64u + a, 1u };
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    uint64_t x = ((uint64_t)w[0] << 32) | w[1];
    uint64_t y = ((uint64_t)w[2] << 32) | w[3];
    double u1 = 1.0 - (double)(x >> 11) * 0x1.0p-53;
    double u2 = (double)(y >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* SplitMix64 finalizer (S. Vigna, "SplitMix64", public domain): a bijective
 * 64-bit mixing function, used to fingerprint flip events. */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Runs trajectory `traj` of the noisy circuit from basis state x0; the final
 * state is left in psi.  Statistics: stats[0] = number of X flips,
 * stats[1] = Y flips, stats[2] = Z flips, stats[3] = fingerprint of the flip
 * events: the sum (mod 2^64) of mix64((s * 64 + q) * 4 + kind) over events
 * (kind 1 = X, 2 = Y, 3 = Z), which does not depend on their order. */
/* flags (may be NULL): per gate, bit 0 = its angles are not deviated, bit 1 =
 * no flips are drawn after it (a noiseless preparation; decoherence only
 * after chosen gates, as the phase shifts R_d of the QFT experiment of
 * Sec. 5.2).  The draws of the other gates keep their counters. */
int or_run_trajectory(double *psi_out, int n, const or_gate *g, int64_t m,
                      const or_noise *noise, uint64_t seed, uint32_t traj,
                      uint64_t x0, uint64_t *stats, const uint8_t *flags)
{
    cplx *psi = (cplx *)psi_out;
    or_init_basis(psi_out, n, x0);
    const uint32_t T = or_flip_threshold(noise->p);
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    stats[0] = stats[1] = stats[2] = stats[3] = 0;
    for (int64_t s = 0; s < m; s++) {
        /* the gate, with its angles deviated (Sec. 3.2) */
        double ang[2] = { g[s].angle[0], g[s].angle[1] };
        int na = or_gate_n_angles(g[s].kind);
        const int fl = flags ? flags[s] : 0;
        if (noise->sigma != 0.0 && !(fl & 1))
            for (int a = 0; a < na; a++)
                ang[a] += noise->sigma * or_gauss(seed, traj, (uint32_t)s, (uint32_t)a);
        if (apply_gate_angles(psi, n, &g[s], ang) != 0) return -1;
        /* then decoherence on every qubit (Sec. 3.1) */
        if (T == 0 || (fl & 2)) continue;
        if (noise->every > 1 && (s + 1) % noise->every != 0) continue;
        for (int q = 0; q < n; q++) {
            uint32_t ctr[4] = { traj, (uint32_t)s, (uint32_t)q, 0u };
            uint32_t w[4];
            or_philox4x32_10(ctr, key, w);
            if (w[0] >= T) continue;
            int kind;
            if (noise->mode == OR_NOISE_DEPOLARIZING)
                kind = 1 + (int)(((uint64_t)w[1] * 3u) >> 32);
            else
                kind = (w[1] & 1u) ? 3 : 1;
            or_gate e;
            memset(&e, 0, sizeof e);
            e.kind = kind == 1 ? OR_X : kind == 2 ? OR_Y : OR_Z;
            e.target = q; e.target2 = -1; e.param = -1;
            apply_gate_angles(psi, n, &e, e.angle);
            stats[kind - 1] += 1;
            stats[3] += mix64(((uint64_t)s * 64u + (uint64_t)q) * 4u + (uint64_t)kind);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradients of an expectation value with respect to gate angles.            */
/* The oracle's gradient is the parameter-shift rule, exact for gates of the  */
/* form exp(-i a r P) with P a Pauli operator (E is then a trigonometric      */
/* polynomial of degree one in 2ra), and central finite differences for the   */
/* check.                                                                      */
/* The cost E is either <psi|Pauli|psi> or the fidelity |<phi|psi>|^2.        */
/* ------------------------------------------------------------------------- */
static double cost_eval(int n, const or_gate *g, int64_t m, const double *params,
                        const char *pauli, const double *ref, double *work)
{
    or_init_basis(work, n, 0);
    for (int64_t k = 0; k < m; k++) {
        double ang[2] = { g[k].angle[0], g[k].angle[1] };
        if (g[k].param >= 0) {
            ang[0] = params[g[k].param];
            if (or_gate_n_angles(g[k].kind) == 2) ang[1] = params[g[k].param + 1];
        }
        if (apply_gate_angles((cplx *)work, n, &g[k], ang) != 0) return NAN;
    }
    if (ref) {
        double z[2];
        or_inner(ref, work, n, z);
        return z[0] * z[0] + z[1] * z[1];
    }
    return or_expect_pauli(work, n, pauli);
}

/* E(params) for the circuit started from |0...0>; ref == NULL selects the
 * Pauli observable, otherwise the fidelity to the state ref. */
double or_cost(int n, const or_gate *g, int64_t m, const double *params,
               const char *pauli, const double *ref)
{
    const uint64_t N = (uint64_t)1 << n;
    double *work = (double *)malloc(N * 2 * sizeof(double));
    double e = cost_eval(n, g, m, params, pauli, ref, work);
    free(work);
    return e;
}

/* Eigenvalue magnitude r of the generator of angle a of a gate kind, where the
 * gate is exp(-i a r P) up to a global phase with P a Pauli operator:
 * RY, RZ, U_P1, U_P2 have r = 1/2 and U_R(theta) = exp(-i theta Y) has r = 1.
 * Returns 0 for angles that have no shift rule here. */
static double shift_r(int kind, int which)
{
    switch (kind) {
    case OR_RY: case OR_RZ: case OR_UP1: case OR_UP2: return 0.5;
    case OR_UR: return 1.0;
    case OR_URP1: return which == 0 ? 1.0 : 0.5;
    default: return 0.0;
    }
}

/* Frequencies of E as a function of one gate's angle a.  With generator
 * eigenvalues {-r, r} (uncontrolled rotation, or a phase shift, whose
 * eigenvalues {0, 2r} differ by 2r) E has the single frequency 2r; a
 * controlled rotation (RY, RZ, U_R, the U_R angle of URP1) has the generator
 * eigenvalues {-r, 0, r} and E the frequencies r and 2r. */
static int three_eigenvalues(const or_gate *g, int which)
{
    if (g->ctrl_mask == 0) return 0;
    switch (g->kind) {
    case OR_RY: case OR_RZ: case OR_UR: return 1;
    case OR_URP1: return which == 0;
    default: return 0;
    }
}

/* grad[k] for k < n_params: the sum over the gate occurrences that use
 * parameter k of the derivative with respect to that occurrence's angle
 * alone (its angle is moved, the other occurrences keep theirs).
 * method 0, parameter shift with s = r a, D(t) = E(a + t/r) - E(a - t/r):
 *     single frequency 2r:   dE/da = r D(pi/4)
 *     frequencies r and 2r:  dE/da = r [(1/2 - sqrt(2)/2) D(pi/2) + D(pi/4)]
 *     (the second is exact for both: matching the sin-coefficients of
 *      the two frequencies gives the two weights);
 * method 1, central finite differences [E(a + h) - E(a - h)] / (2h).
 * Returns -1 for a parameter index beyond n_params. */
/* E with angle `which` of gate k moved to base[which] + t (the gate is given
 * explicit angles, so other gates on the same parameter keep theirs). */
static double eval_moved(int n, or_gate *gg, int64_t k, int64_t m, const double *params, const double base[2],
                         int which, double t, const char *pauli, const double *ref, double *work)
{
    gg[k].param = -1;
    gg[k].angle[0] = base[0] + (which == 0 ? t : 0.0);
    gg[k].angle[1] = base[1] + (which == 1 ? t : 0.0);
    return cost_eval(n, gg, m, params, pauli, ref, work);
}

int or_gradient(int n, const or_gate *g, int64_t m, const double *params, int64_t n_params,
                const char *pauli, const double *ref, int method, double h, double *grad)
{
    const uint64_t N = (uint64_t)1 << n;
    or_gate *gg = (or_gate *)malloc((size_t)(m > 0 ? m : 1) * sizeof(or_gate));
    double *work = (double *)malloc(N * 2 * sizeof(double));
    int bad = 0;
    memcpy(gg, g, (size_t)m * sizeof(or_gate));
    for (int64_t k = 0; k < n_params; k++) grad[k] = 0.0;
    for (int64_t k = 0; k < m && !bad; k++) {
        if (g[k].param < 0) continue;
        const int na = or_gate_n_angles(g[k].kind);
        if (g[k].param + na > n_params) { bad = 1; break; }
        const double base[2] = { params[g[k].param], na > 1 ? params[g[k].param + 1] : 0.0 };
        for (int a = 0; a < na; a++) {
            const double r = shift_r(g[k].kind, a);
            double dE;
            if (method == 0) {
                const double d1 = M_PI / (4 * r), d2 = M_PI / (2 * r);
                const double D1 = eval_moved(n, gg, k, m, params, base, a, d1, pauli, ref, work) -
                                  eval_moved(n, gg, k, m, params, base, a, -d1, pauli, ref, work);
                if (three_eigenvalues(&g[k], a)) {
                    const double D2 = eval_moved(n, gg, k, m, params, base, a, d2, pauli, ref, work) -
                                      eval_moved(n, gg, k, m, params, base, a, -d2, pauli, ref, work);
                    dE = r * ((0.5 - 0.5 * sqrt(2.0)) * D2 + D1);
                } else {
                    dE = r * D1;
                }
            } else {
                dE = (eval_moved(n, gg, k, m, params, base, a, h, pauli, ref, work) -
                      eval_moved(n, gg, k, m, params, base, a, -h, pauli, ref, work)) / (2 * h);
            }
            gg[k] = g[k];
            grad[g[k].param + a] += dE;
        }
    }
    free(gg);
    free(work);
    return bad ? -1 : 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
