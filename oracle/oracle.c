/*
 * Reference oracle: a plain, slow, per-gate complex128 state-vector simulator
 * with adjoint-method gradients.
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it. It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Everything follows the paper's definitions literally, one gate at a time:
 *
 *  - State representation (Sec. 3.1): psi in C^{2^n}, amplitude a_x with
 *    x = sum_i x_i 2^i, so qubit i is bit i of the index.
 *  - Single-qubit gate (Sec. 3.1): every pair (a_{..0_t..}, a_{..1_t..}) is
 *    multiplied by the 2x2 matrix u.
 *  - CZ (Sec. 3.1): amplitudes whose control and target bits are both 1 are
 *    negated. CNOT (Sec. 3.1): the pair with control bit 1 is swapped.
 *  - Rotation gates (Sec. 3.3, gradient step): u(t) = cos(t/2) I - i sin(t/2) P
 *    and du/dt = -1/2 sin(t/2) I - i 1/2 cos(t/2) P, with P in {X, Y, Z}.
 *  - Expectation (Eq. 1): E = <psi_M| O |psi_M>, O a Pauli string applied
 *    qubit by qubit as 2x2 matrices.
 *  - Adjoint seed (Eq. 4, with the chain rule for a general loss):
 *    lambda_M = 2 (dL/dE) O psi_M.
 *  - Adjoint update (Eq. 2): lambda_{j-1} = U_j^dagger lambda_j.
 *  - Gradient (Eq. 3): dL/dtheta_j = Re <lambda_j| dU_j/dtheta_j |psi_{j-1}>.
 *
 * The oracle never reverses a gate to recover psi_{j-1}: it takes psi_{j-1}
 * from stored states. To bound memory it keeps the input state of every block
 * of `block` consecutive gates and, walking the blocks backwards, re-runs each
 * block forward from its stored input, keeping every intermediate state of
 * that block (gradient checkpointing, Sec. 3.4). block >= M keeps all states.
 *
 * Parallelism: OpenMP over samples when there are at least as many samples
 * as threads; otherwise the samples run one after another and every loop over
 * the 2^n amplitudes is split across the threads instead (the arithmetic per
 * amplitude is unchanged; only the order of the final sums in <a|b> differs).
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

/* 1 while the amplitude loops run in parallel (fewer samples than threads). */
static int amp_par = 0;

/* Amplitude loops shorter than this stay on one thread (below 2^17 complex128
 * amplitudes, 2 MiB, the fork and join per gate cost more than the loop). */
#define OR_PAR_MIN_DIM ((uint64_t)1 << 17)

/* The parallel clause of an amplitude loop over `dim` entries. */
#define OR_AMP_PAR(dim) if (amp_par && (dim) >= OR_PAR_MIN_DIM) schedule(static)

/* Gate kinds understood by the oracle. */
enum { OR_RX = 0, OR_RY = 1, OR_RZ = 2, OR_CZ = 3, OR_CNOT = 4 };

/* Pauli letters of an observable, one per qubit. */
enum { OR_I = 0, OR_X = 1, OR_Y = 2, OR_Z = 3 };

/* One gate: kind, qubits (q1 used by two-qubit gates: q0 = control,
 * q1 = target), index into theta (-1 for constant gates). */
typedef struct {
    int32_t kind;
    int32_t q0;
    int32_t q1;
    int32_t param;
} or_gate;

/* ---- 2x2 matrices (Sec. 3.3, definition of u and du/dtheta) ------------ */

static void pauli_matrix(int letter, cplx m[2][2]) {
    m[0][0] = 0; m[0][1] = 0; m[1][0] = 0; m[1][1] = 0;
    switch (letter) {
    case OR_I: m[0][0] = 1; m[1][1] = 1; break;
    case OR_X: m[0][1] = 1; m[1][0] = 1; break;
    case OR_Y: m[0][1] = -I; m[1][0] = I; break;
    case OR_Z: m[0][0] = 1; m[1][1] = -1; break;
    }
}

static int rotation_letter(int kind) {
    return kind == OR_RX ? OR_X : kind == OR_RY ? OR_Y : OR_Z;
}

/* u(t) = cos(t/2) I - i sin(t/2) P */
static void rotation_matrix(int kind, double t, cplx u[2][2]) {
    cplx p[2][2];
    pauli_matrix(rotation_letter(kind), p);
    double c = cos(t / 2.0), s = sin(t / 2.0);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k)
            u[r][k] = (r == k ? c : 0.0) - I * s * p[r][k];
}

/* du/dt = -1/2 sin(t/2) I - i 1/2 cos(t/2) P */
static void rotation_derivative(int kind, double t, cplx du[2][2]) {
    cplx p[2][2];
    pauli_matrix(rotation_letter(kind), p);
    double c = cos(t / 2.0), s = sin(t / 2.0);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k)
            du[r][k] = (r == k ? -0.5 * s : 0.0) - I * 0.5 * c * p[r][k];
}

static void dagger(cplx u[2][2], cplx ud[2][2]) {
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k) ud[r][k] = conj(u[k][r]);
}

/* ---- gate application on a state (Sec. 3.1) ----------------------------- */

/* For every index pair differing only in bit t:
 * (a0', a1') = u (a0, a1). */
static void apply_1q(cplx *psi, int n, int t, cplx u[2][2]) {
    const uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << t;
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim)
#endif
    for (uint64_t x = 0; x < dim; ++x) {
        if (x & bit) continue;
        cplx a0 = psi[x], a1 = psi[x | bit];
        psi[x] = u[0][0] * a0 + u[0][1] * a1;
        psi[x | bit] = u[1][0] * a0 + u[1][1] * a1;
    }
}

/* CZ: negate a_x when bits c and t of x are both 1. */
static void apply_cz(cplx *psi, int n, int c, int t) {
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t bc = (uint64_t)1 << c, bt = (uint64_t)1 << t;
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim)
#endif
    for (uint64_t x = 0; x < dim; ++x)
        if ((x & bc) && (x & bt)) psi[x] = -psi[x];
}

/* CNOT: swap a_{..1_c..0_t..} and a_{..1_c..1_t..}. */
static void apply_cnot(cplx *psi, int n, int c, int t) {
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t bc = (uint64_t)1 << c, bt = (uint64_t)1 << t;
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim)
#endif
    for (uint64_t x = 0; x < dim; ++x) {
        if (!(x & bc) || (x & bt)) continue;
        cplx tmp = psi[x];
        psi[x] = psi[x | bt];
        psi[x | bt] = tmp;
    }
}

/* Apply gate g (or its adjoint when adj != 0). */
static void apply_gate(cplx *psi, int n, const or_gate *g, const double *theta,
                       int adj) {
    if (g->kind == OR_CZ) { apply_cz(psi, n, g->q0, g->q1); return; }
    if (g->kind == OR_CNOT) { apply_cnot(psi, n, g->q0, g->q1); return; }
    cplx u[2][2], ud[2][2];
    rotation_matrix(g->kind, theta[g->param], u);
    if (adj) { dagger(u, ud); apply_1q(psi, n, g->q0, ud); }
    else apply_1q(psi, n, g->q0, u);
}

/* dst = src over 2^n amplitudes. */
static void copy_state(cplx *dst, const cplx *src, int n) {
    const uint64_t dim = (uint64_t)1 << n;
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim)
#endif
    for (uint64_t x = 0; x < dim; ++x) dst[x] = src[x];
}

/* O psi for a Pauli string, applied one qubit at a time. */
static void apply_pauli(cplx *out, const cplx *psi, int n, const int32_t *letters) {
    copy_state(out, psi, n);
    for (int q = 0; q < n; ++q) {
        if (letters[q] == OR_I) continue;
        cplx p[2][2];
        pauli_matrix(letters[q], p);
        apply_1q(out, n, q, p);
    }
}

/* <a|b> = sum_x conj(a_x) b_x */
static cplx inner(const cplx *a, const cplx *b, int n) {
    const uint64_t dim = (uint64_t)1 << n;
    double sr = 0, si = 0;
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim) reduction(+ : sr, si)
#endif
    for (uint64_t x = 0; x < dim; ++x) {
        const cplx t = conj(a[x]) * b[x];
        sr += creal(t);
        si += cimag(t);
    }
    return sr + I * si;
}

/* Initial state. When init_state is non-null it is copied (interleaved
 * re/im doubles); otherwise |0...0> is encoded by RY(x_q) on each qubit q
 * (data encoding: one RY(x_q) per qubit, applied gate by gate). */
static void prepare(cplx *psi, int n, const double *xrow, const double *init_state) {
    const uint64_t dim = (uint64_t)1 << n;
    if (init_state) {
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim)
#endif
        for (uint64_t x = 0; x < dim; ++x)
            psi[x] = init_state[2 * x] + I * init_state[2 * x + 1];
        return;
    }
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim)
#endif
    for (uint64_t x = 0; x < dim; ++x) psi[x] = 0;
    psi[0] = 1;
    for (int q = 0; q < n; ++q) {
        cplx u[2][2];
        rotation_matrix(OR_RY, xrow[q], u);
        apply_1q(psi, n, q, u);
    }
}

/* ---- public entry points ------------------------------------------------ */

/* Thread count for this call (n_threads > 0 sets it) and where the threads
 * go: over samples when there are at least as many samples as threads,
 * else over the amplitudes of one sample at a time. */
static void set_parallelism(int B, int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    amp_par = B < omp_get_max_threads();
#else
    (void)B;
    (void)n_threads;
    amp_par = 0;
#endif
}

/* Final state of one sample: psi_out gets 2*2^n doubles (re, im interleaved).
 * x: [n] encoding angles (ignored when init_state is given). */
int oracle_final_state(int n, const or_gate *gates, int n_gates, const double *theta,
                       const double *x, const double *init_state, double *psi_out) {
    const uint64_t dim = (uint64_t)1 << n;
    cplx *psi = malloc(dim * sizeof(cplx));
    if (!psi) return -1;
    set_parallelism(1, 0);
    prepare(psi, n, x, init_state);
    for (int j = 0; j < n_gates; ++j) apply_gate(psi, n, &gates[j], theta, 0);
    for (uint64_t k = 0; k < dim; ++k) {
        psi_out[2 * k] = creal(psi[k]);
        psi_out[2 * k + 1] = cimag(psi[k]);
    }
    free(psi);
    return 0;
}

/* Expectations E_b = <psi_M|O|psi_M> (Eq. 1) for B samples.
 * x: [B][n]; init_states: [B][2^n][2] or null; letters: [n] Pauli letters. */
int oracle_expectation(int n, const or_gate *gates, int n_gates, const double *theta,
                       int B, const double *x, const double *init_states,
                       const int32_t *letters, double *E_out, int n_threads) {
    const uint64_t dim = (uint64_t)1 << n;
    int fail = 0;
    set_parallelism(B, n_threads);
#ifdef _OPENMP
#pragma omp parallel for if (!amp_par) schedule(dynamic, 1) reduction(| : fail)
#endif
    for (int b = 0; b < B; ++b) {
        cplx *psi = malloc(dim * sizeof(cplx));
        cplx *opsi = malloc(dim * sizeof(cplx));
        if (!psi || !opsi) { free(psi); free(opsi); fail |= 1; continue; }
        prepare(psi, n, x ? x + (size_t)b * n : 0,
                init_states ? init_states + (size_t)b * 2 * dim : 0);
        for (int j = 0; j < n_gates; ++j) apply_gate(psi, n, &gates[j], theta, 0);
        apply_pauli(opsi, psi, n, letters);
        E_out[b] = creal(inner(psi, opsi, n));
        free(psi);
        free(opsi);
    }
    return fail ? -1 : 0;
}

/* Adjoint-method gradients (Sec. 2.2).
 *
 * dLdE: [B] values dL/dE_b (the chain-rule factor in the seed of Eq. 4).
 * grad_out: [n_params] (sum over samples) when per_sample == 0, else
 *           [B][n_params]. E_out: [B] (may be null).
 * block: number of gates per recompute block (>= n_gates stores all states).
 */
int oracle_gradient(int n, const or_gate *gates, int n_gates, const double *theta,
                    int n_params, int B, const double *x, const double *init_states,
                    const int32_t *letters, const double *dLdE, int per_sample,
                    int block, double *grad_out, double *E_out, int n_threads) {
    const uint64_t dim = (uint64_t)1 << n;
    if (block < 1) block = 1;
    if (block > n_gates) block = n_gates > 0 ? n_gates : 1;
    const int n_blocks = n_gates > 0 ? (n_gates + block - 1) / block : 0;
    double *per = calloc((size_t)B * (n_params > 0 ? n_params : 1), sizeof(double));
    if (!per) return -1;
    int fail = 0;
    set_parallelism(B, n_threads);
#ifdef _OPENMP
#pragma omp parallel for if (!amp_par) schedule(dynamic, 1) reduction(| : fail)
#endif
    for (int b = 0; b < B; ++b) {
        /* block inputs: state before gate k*block, k = 0..n_blocks-1 */
        cplx *ckpt = malloc((size_t)(n_blocks > 0 ? n_blocks : 1) * dim * sizeof(cplx));
        /* states inside the active block: psi before each of its gates */
        cplx *inside = malloc((size_t)block * dim * sizeof(cplx));
        cplx *psi = malloc(dim * sizeof(cplx));
        cplx *lam = malloc(dim * sizeof(cplx));
        cplx *tmp = malloc(dim * sizeof(cplx));
        if (!ckpt || !inside || !psi || !lam || !tmp) {
            free(ckpt); free(inside); free(psi); free(lam); free(tmp);
            fail |= 1;
            continue;
        }
        double *g = per + (size_t)b * n_params;

        /* forward pass, keeping each block's input state */
        prepare(psi, n, x ? x + (size_t)b * n : 0,
                init_states ? init_states + (size_t)b * 2 * dim : 0);
        for (int j = 0; j < n_gates; ++j) {
            if (j % block == 0) copy_state(ckpt + (size_t)(j / block) * dim, psi, n);
            apply_gate(psi, n, &gates[j], theta, 0);
        }
        /* E (Eq. 1) and seed lambda_M = 2 (dL/dE) O psi_M (Eq. 4) */
        apply_pauli(tmp, psi, n, letters);
        if (E_out) E_out[b] = creal(inner(psi, tmp, n));
        const double seed = 2.0 * dLdE[b];
#ifdef _OPENMP
#pragma omp parallel for OR_AMP_PAR(dim)
#endif
        for (uint64_t k = 0; k < dim; ++k) lam[k] = seed * tmp[k];

        /* backward pass, block by block in reverse */
        for (int k = n_blocks - 1; k >= 0; --k) {
            const int j0 = k * block;
            const int j1 = (j0 + block < n_gates) ? j0 + block : n_gates;
            /* recompute psi_{j-1} for every gate of the block from its input */
            copy_state(psi, ckpt + (size_t)k * dim, n);
            for (int j = j0; j < j1; ++j) {
                copy_state(inside + (size_t)(j - j0) * dim, psi, n);
                apply_gate(psi, n, &gates[j], theta, 0);
            }
            for (int j = j1 - 1; j >= j0; --j) {
                const or_gate *gt = &gates[j];
                const cplx *psi_prev = inside + (size_t)(j - j0) * dim;
                if (gt->param >= 0 && gt->kind <= OR_RZ) {
                    /* Eq. 3: Re <lambda_j| dU_j |psi_{j-1}> */
                    cplx du[2][2];
                    rotation_derivative(gt->kind, theta[gt->param], du);
                    copy_state(tmp, psi_prev, n);
                    apply_1q(tmp, n, gt->q0, du);
                    g[gt->param] += creal(inner(lam, tmp, n));
                }
                /* Eq. 2: lambda_{j-1} = U_j^dagger lambda_j */
                apply_gate(lam, n, gt, theta, 1);
            }
        }
        free(ckpt); free(inside); free(psi); free(lam); free(tmp);
    }
    if (!fail) {
        if (per_sample) {
            memcpy(grad_out, per, (size_t)B * n_params * sizeof(double));
        } else {
            for (int p = 0; p < n_params; ++p) {
                double s = 0;
                for (int b = 0; b < B; ++b) s += per[(size_t)b * n_params + p];
                grad_out[p] = s;
            }
        }
    }
    free(per);
    return fail ? -1 : 0;
}

/* Threads OpenMP would use (for reporting the CPU-baseline core count). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
