/*
 * tqd_oracle.c -- plain, slow, gate-by-gate complex128 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library; it has its own gate matrices, its own index loops and uses
 * C99 `double complex` throughout.
 *
 * What it computes (the definitions, written out):
 *   - gate application Y = M x_Q X (contraction of the gate's ordered qubit
 *     set Q with the unitary M; notation of Sec. 2.2, applied as in
 *     Algorithm 1: gather the 2^k amplitudes addressed by Q, multiply by M,
 *     scatter back);
 *   - the circuit state psi_L = G_L ... G_1 e_j  (Sec. 2.2.1, Sec. 4.1);
 *   - Pauli-sum expectation E = sum_j c_j psi^* P_j psi, P_j applied as a
 *     product of single-qubit Pauli matrices (Sec. 2.2.1, measurement);
 *   - dE/dtheta by the parameter-shift rule, independent of any adjoint;
 *   - dE/dtheta by a stored-activation reverse pass: every intermediate state
 *     is kept and the gradient of a unitary layer y = U x is taken as in the
 *     first form of Sec. 4.4 (d_x = U^dagger d_y, d_U = d_y x^T, chained to
 *     the angle through the analytic derivative dU/dtheta).
 *
 * Qubit i is bit i of the flat index.  For a k-qubit gate with wires
 * (w_0, ..., w_{k-1}), w_0 is the most significant bit of the local index.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum {
    O_H = 0, O_X, O_Y, O_Z, O_S, O_T,
    O_RX, O_RY, O_RZ, O_PHASE,
    O_CNOT, O_CZ, O_CPHASE, O_SWAP,
    O_UNITARY1, O_UNITARY2, O_NKINDS
};

typedef struct {
    int32_t kind;
    int32_t nwires;
    int32_t wires[3];
    int32_t param;   /* index into the parameter vector, -1 = fixed angle */
    double angle;    /* used when param < 0 */
    int32_t mat;     /* UNITARY1/2: offset (complex entries) into the matrix table */
    int32_t pad;
} orc_gate;

static const double ORC_PI = 3.14159265358979323846;

static int gate_arity(int kind) {
    switch (kind) {
    case O_CNOT: case O_CZ: case O_CPHASE: case O_SWAP: case O_UNITARY2: return 2;
    default: return 1;
    }
}

static int gate_is_parametric(int kind) {
    return kind == O_RX || kind == O_RY || kind == O_RZ || kind == O_PHASE || kind == O_CPHASE;
}

/* The unitary of one gate, row-major, dimension 2^arity.
 * Rotations R_P(t) = exp(-i t P / 2) = cos(t/2) I - i sin(t/2) P. */
static void gate_matrix(int kind, double t, const cplx *table, int mat, cplx *M) {
    const double c = cos(0.5 * t), s = sin(0.5 * t);
    const double r = 1.0 / sqrt(2.0);
    int d = 1 << gate_arity(kind);
    for (int i = 0; i < d * d; ++i) M[i] = 0;
    switch (kind) {
    case O_H:  M[0] = r; M[1] = r; M[2] = r; M[3] = -r; break;
    case O_X:  M[1] = 1; M[2] = 1; break;
    case O_Y:  M[1] = -I; M[2] = I; break;
    case O_Z:  M[0] = 1; M[3] = -1; break;
    case O_S:  M[0] = 1; M[3] = I; break;
    case O_T:  M[0] = 1; M[3] = cexp(I * ORC_PI / 4.0); break;
    case O_RX: M[0] = c; M[1] = -I * s; M[2] = -I * s; M[3] = c; break;
    case O_RY: M[0] = c; M[1] = -s; M[2] = s; M[3] = c; break;
    case O_RZ: M[0] = cexp(-0.5 * I * t); M[3] = cexp(0.5 * I * t); break;
    case O_PHASE: M[0] = 1; M[3] = cexp(I * t); break;
    /* two-qubit gates: local index = 2*bit(w0) + bit(w1) */
    case O_CNOT: M[0] = 1; M[5] = 1; M[11] = 1; M[14] = 1; break;
    case O_CZ: M[0] = 1; M[5] = 1; M[10] = 1; M[15] = -1; break;
    case O_CPHASE: M[0] = 1; M[5] = 1; M[10] = 1; M[15] = cexp(I * t); break;
    case O_SWAP: M[0] = 1; M[6] = 1; M[9] = 1; M[15] = 1; break;
    case O_UNITARY1: for (int i = 0; i < 4; ++i) M[i] = table[mat + i]; break;
    case O_UNITARY2: for (int i = 0; i < 16; ++i) M[i] = table[mat + i]; break;
    default: break;
    }
}

/* d/dt of the unitary above (only for the parametric kinds). */
static void gate_matrix_deriv(int kind, double t, cplx *D) {
    const double c = cos(0.5 * t), s = sin(0.5 * t);
    int d = 1 << gate_arity(kind);
    for (int i = 0; i < d * d; ++i) D[i] = 0;
    switch (kind) {
    case O_RX: D[0] = -0.5 * s; D[1] = -0.5 * I * c; D[2] = -0.5 * I * c; D[3] = -0.5 * s; break;
    case O_RY: D[0] = -0.5 * s; D[1] = -0.5 * c; D[2] = 0.5 * c; D[3] = -0.5 * s; break;
    case O_RZ: D[0] = -0.5 * I * cexp(-0.5 * I * t); D[3] = 0.5 * I * cexp(0.5 * I * t); break;
    case O_PHASE: D[3] = I * cexp(I * t); break;
    case O_CPHASE: D[15] = I * cexp(I * t); break;
    default: break;
    }
}

static void dagger(const cplx *M, int d, cplx *Md) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Md[i * d + j] = conj(M[j * d + i]);
}

/* Y = M x_Q X over the whole state: for every index b whose wire bits are all
 * zero, gather the 2^k amplitudes b + (bits of l on the wires), multiply by M,
 * scatter back. */
static void apply_matrix(int n, cplx *psi, int k, const int32_t *wires, const cplx *M) {
    const uint64_t N = (uint64_t)1 << n;
    const int d = 1 << k;
    uint64_t wmask = 0;
    for (int i = 0; i < k; ++i) wmask |= (uint64_t)1 << wires[i];
    uint64_t offs[8];
    for (int l = 0; l < d; ++l) {
        uint64_t o = 0;
        for (int i = 0; i < k; ++i)
            if ((l >> (k - 1 - i)) & 1) o |= (uint64_t)1 << wires[i];
        offs[l] = o;
    }
    cplx v[8], w[8];
    for (uint64_t b = 0; b < N; ++b) {
        if (b & wmask) continue;
        for (int l = 0; l < d; ++l) v[l] = psi[b | offs[l]];
        for (int r = 0; r < d; ++r) {
            cplx acc = 0;
            for (int c = 0; c < d; ++c) acc += M[r * d + c] * v[c];
            w[r] = acc;
        }
        for (int l = 0; l < d; ++l) psi[b | offs[l]] = w[l];
    }
}

static double gate_angle(const orc_gate *g, const double *params) {
    return g->param >= 0 ? params[g->param] : g->angle;
}

static void apply_gate_angle(int n, cplx *psi, const orc_gate *g, double t, const cplx *table,
                             int adjoint) {
    cplx M[16], Md[16];
    gate_matrix(g->kind, t, table, g->mat, M);
    int k = gate_arity(g->kind);
    if (adjoint) {
        dagger(M, 1 << k, Md);
        apply_matrix(n, psi, k, g->wires, Md);
    } else {
        apply_matrix(n, psi, k, g->wires, M);
    }
}

/* ---------------------------------------------------------------- exported */

int orc_version(void) { return 1; }

void orc_basis_state(int n, uint64_t j, cplx *psi) {
    const uint64_t N = (uint64_t)1 << n;
    for (uint64_t b = 0; b < N; ++b) psi[b] = 0;
    psi[j] = 1;
}

/* Apply one gate (adjoint != 0 applies its conjugate transpose). */
void orc_apply_gate(int n, cplx *psi, const orc_gate *g, const double *params, const cplx *table,
                    int adjoint) {
    apply_gate_angle(n, psi, g, gate_angle(g, params), table, adjoint);
}

/* Apply gates[first..last) in order, or their adjoints in reverse order. */
void orc_apply_gates(int n, cplx *psi, const orc_gate *gates, int first, int last,
                     const double *params, const cplx *table, int adjoint) {
    if (!adjoint) {
        for (int g = first; g < last; ++g) orc_apply_gate(n, psi, &gates[g], params, table, 0);
    } else {
        for (int g = last - 1; g >= first; --g) orc_apply_gate(n, psi, &gates[g], params, table, 1);
    }
}

/* psi_L = G_L ... G_1 e_init  with per-gate angles (angles[g] used for every
 * parametric gate; non-parametric gates ignore it). */
static void run_angles(int n, const orc_gate *gates, int ng, const double *angles,
                       const cplx *table, uint64_t init, cplx *psi) {
    orc_basis_state(n, init, psi);
    for (int g = 0; g < ng; ++g) apply_gate_angle(n, psi, &gates[g], angles[g], table, 0);
}

static void gate_angles(const orc_gate *gates, int ng, const double *params, double *angles) {
    for (int g = 0; g < ng; ++g) angles[g] = gate_angle(&gates[g], params);
}

void orc_run(int n, const orc_gate *gates, int ng, const double *params, const cplx *table,
             uint64_t init, cplx *psi) {
    double *angles = (double *)malloc(sizeof(double) * (ng > 0 ? ng : 1));
    gate_angles(gates, ng, params, angles);
    run_angles(n, gates, ng, angles, table, init, psi);
    free(angles);
}

/* Single-qubit Pauli matrices, op codes 1 = X, 2 = Y, 3 = Z. */
static void pauli_matrix(int op, cplx *P) {
    P[0] = P[1] = P[2] = P[3] = 0;
    if (op == 1) { P[1] = 1; P[2] = 1; }
    if (op == 2) { P[1] = -I; P[2] = I; }
    if (op == 3) { P[0] = 1; P[3] = -1; }
}

/* phi = P_j psi, with P_j = tensor product of the term's single-qubit Paulis;
 * ops is the term's row of n op codes (0 = I). */
static void apply_pauli_word(int n, const int8_t *ops, cplx *phi) {
    cplx P[4];
    for (int q = 0; q < n; ++q) {
        if (ops[q] == 0) continue;
        pauli_matrix(ops[q], P);
        int32_t w = q;
        apply_matrix(n, phi, 1, &w, P);
    }
}

static cplx inner(int n, const cplx *a, const cplx *b) {
    const uint64_t N = (uint64_t)1 << n;
    cplx acc = 0;
    for (uint64_t i = 0; i < N; ++i) acc += conj(a[i]) * b[i];
    return acc;
}

/* E = sum_j c_j <psi|P_j|psi>; per-term values <psi|P_j|psi> (without c_j)
 * go to out_terms when it is not NULL. */
double orc_expval(int n, const cplx *psi, int nterms, const int8_t *ops, const double *coeffs,
                  double *out_terms) {
    const uint64_t N = (uint64_t)1 << n;
    cplx *phi = (cplx *)malloc(sizeof(cplx) * N);
    double total = 0;
    for (int j = 0; j < nterms; ++j) {
        memcpy(phi, psi, sizeof(cplx) * N);
        apply_pauli_word(n, ops + (size_t)j * n, phi);
        double e = creal(inner(n, psi, phi));
        if (out_terms) out_terms[j] = e;
        total += coeffs[j] * e;
    }
    free(phi);
    return total;
}

/* out = H psi = sum_j c_j P_j psi. */
void orc_apply_observable(int n, const cplx *psi, int nterms, const int8_t *ops,
                          const double *coeffs, cplx *out) {
    const uint64_t N = (uint64_t)1 << n;
    cplx *phi = (cplx *)malloc(sizeof(cplx) * N);
    for (uint64_t b = 0; b < N; ++b) out[b] = 0;
    for (int j = 0; j < nterms; ++j) {
        memcpy(phi, psi, sizeof(cplx) * N);
        apply_pauli_word(n, ops + (size_t)j * n, phi);
        for (uint64_t b = 0; b < N; ++b) out[b] += coeffs[j] * phi[b];
    }
    free(phi);
}

/* Gradient by the parameter-shift rule.  Every parametric gate used here has
 * a generator with two eigenvalues half a unit apart from its mean, so
 * dE/dt = (E(t + pi/2) - E(t - pi/2)) / 2 exactly.  A parameter read by
 * several gates gets the sum over its gates (chain rule).  Parallel over
 * gates when built with OpenMP; contributions are summed in gate order. */
void orc_grad_param_shift(int n, const orc_gate *gates, int ng, const double *params, int nparams,
                          const cplx *table, uint64_t init, int nterms, const int8_t *ops,
                          const double *coeffs, double *grad) {
    const uint64_t N = (uint64_t)1 << n;
    double *contrib = (double *)calloc(ng > 0 ? ng : 1, sizeof(double));
    double *base = (double *)malloc(sizeof(double) * (ng > 0 ? ng : 1));
    gate_angles(gates, ng, params, base);
#pragma omp parallel
    {
        cplx *psi = (cplx *)malloc(sizeof(cplx) * N);
        double *angles = (double *)malloc(sizeof(double) * (ng > 0 ? ng : 1));
        memcpy(angles, base, sizeof(double) * ng);
#pragma omp for schedule(dynamic, 1)
        for (int g = 0; g < ng; ++g) {
            if (gates[g].param < 0 || !gate_is_parametric(gates[g].kind)) continue;
            angles[g] = base[g] + 0.5 * ORC_PI;
            run_angles(n, gates, ng, angles, table, init, psi);
            double ep = orc_expval(n, psi, nterms, ops, coeffs, NULL);
            angles[g] = base[g] - 0.5 * ORC_PI;
            run_angles(n, gates, ng, angles, table, init, psi);
            double em = orc_expval(n, psi, nterms, ops, coeffs, NULL);
            angles[g] = base[g];
            contrib[g] = 0.5 * (ep - em);
        }
        free(angles);
        free(psi);
    }
    for (int k = 0; k < nparams; ++k) grad[k] = 0;
    for (int g = 0; g < ng; ++g)
        if (gates[g].param >= 0) grad[gates[g].param] += contrib[g];
    free(base);
    free(contrib);
}

/* Gradient by a stored-activation reverse pass (first form of Sec. 4.4):
 * keep x_g = psi before gate g for every g; with the adjoint state
 * l_{g+1} = dE/d(psi after g)^* (l_L = H psi_L), the layer y = U x gives
 * dE/dt = 2 Re <l_{g+1}| dU/dt x_g> and l_g = U^dagger l_{g+1}.
 * Memory: (ng + 1) states, so only for small n. Returns E. */
double orc_grad_stored(int n, const orc_gate *gates, int ng, const double *params, int nparams,
                       const cplx *table, uint64_t init, int nterms, const int8_t *ops,
                       const double *coeffs, double *grad) {
    const uint64_t N = (uint64_t)1 << n;
    cplx *xs = (cplx *)malloc(sizeof(cplx) * N * (size_t)(ng + 1));
    cplx *lam = (cplx *)malloc(sizeof(cplx) * N);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * N);
    orc_basis_state(n, init, xs);
    for (int g = 0; g < ng; ++g) {
        memcpy(xs + (size_t)(g + 1) * N, xs + (size_t)g * N, sizeof(cplx) * N);
        orc_apply_gate(n, xs + (size_t)(g + 1) * N, &gates[g], params, table, 0);
    }
    const cplx *psiL = xs + (size_t)ng * N;
    double E = orc_expval(n, psiL, nterms, ops, coeffs, NULL);
    orc_apply_observable(n, psiL, nterms, ops, coeffs, lam);
    for (int k = 0; k < nparams; ++k) grad[k] = 0;
    for (int g = ng - 1; g >= 0; --g) {
        const orc_gate *gg = &gates[g];
        if (gg->param >= 0 && gate_is_parametric(gg->kind)) {
            cplx D[16];
            gate_matrix_deriv(gg->kind, gate_angle(gg, params), D);
            memcpy(tmp, xs + (size_t)g * N, sizeof(cplx) * N);
            apply_matrix(n, tmp, gate_arity(gg->kind), gg->wires, D);
            grad[gg->param] += 2.0 * creal(inner(n, lam, tmp));
        }
        orc_apply_gate(n, lam, gg, params, table, 1);
    }
    free(tmp);
    free(lam);
    free(xs);
    return E;
}

/* sum_b |psi_b|^2 */
double orc_norm2(int n, const cplx *psi) { return creal(inner(n, psi, psi)); }

/* The full 2^n x 2^n matrix of one gate, column by column (apply the gate to
 * every basis vector).  Used by the dense cross-checks for small n. */
void orc_gate_dense(int n, const orc_gate *g, const double *params, const cplx *table, cplx *U) {
    const uint64_t N = (uint64_t)1 << n;
    cplx *col = (cplx *)malloc(sizeof(cplx) * N);
    for (uint64_t j = 0; j < N; ++j) {
        orc_basis_state(n, j, col);
        orc_apply_gate(n, col, g, params, table, 0);
        for (uint64_t i = 0; i < N; ++i) U[i * N + j] = col[i];
    }
    free(col);
}
