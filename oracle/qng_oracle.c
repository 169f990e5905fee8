/*
 * CPU oracle for the quantum natural gradient (T. Jones, "Efficient classical calculation of
 * the Quantum Natural Gradient", arXiv:2011.02991).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may call this file; only the
 * tests, the package's smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Plain, slow, complex128 (C99 double complex) code that follows the definitions:
 *   - psi(theta) = U_P ... U_1 |in> with |in> = |0...0> (Sec. 2, definition of U and psi);
 *   - |d_i psi> built explicitly, one state per parameter, by replacing gate i with its
 *     derivative (Appendix A, Alg. 7 "compute each derivative state independently");
 *   - G_ij = <d_i psi|d_j psi> - <d_i psi|psi><psi|d_j psi> (Eq. 4, the quantum geometric tensor);
 *   - <E> = sum_k c_k <psi|sigma_k|psi> and d<E>/d theta_i = 2 Re <psi|H|d_i psi> (Eq. 2 with
 *     the product rule; the paper gives no gradient algorithm).
 * Gate matrices are the textbook ones written entry by entry; derivatives are the entry-wise
 * derivatives of those matrices. Generalised rotations (Sec. 2's remark on multi-qubit and
 * controlled Pauli-string rotations): CR_sigma = |0><0|_c (x) 1 + |1><1|_c (x) R_sigma, and
 * R_S = exp(-i theta S / 2) = cos(theta/2) 1 - i sin(theta/2) S for a Pauli string S, optionally
 * controlled; their derivatives are written from the same closed forms. Pauli strings are applied one single-qubit Pauli matrix at a
 * time. None of this shares code with the CUDA path.
 *
 * It also holds literal CPU transcriptions of the paper's recurrences (Alg. 1 and Appendix A's
 * Alg. 3, 6 and 8), written from the steps of those algorithms with operation counters, so the
 * tests can check them against the definition and against Table 1.
 *
 * Readings where the paper is silent (stated again in the design notes):
 *   - R_sigma(theta) = exp(-i theta sigma / 2) (textbook sign; the paper writes exp(+i ...)).
 *   - Fixed gates between parametric gates k-1 and k belong to U_k = R_k F_k; fixed gates after
 *     the last parametric gate form W, which is part of psi but cancels in G.
 *   - Qubit q is bit q of the amplitude index.
 *
 * Complex arrays cross this interface as interleaved (re, im) doubles, the numpy complex128 layout.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { K_RX = 0, K_RY = 1, K_RZ = 2, K_CZ = 3, K_CNOT = 4, K_X = 5, K_Y = 6, K_Z = 7, K_H = 8,
       K_CRX = 9, K_CRY = 10, K_CRZ = 11, K_RP = 12, K_CRP = 13 };

/* One gate: kind, qubits, parameter index (-1 for fixed gates) and, for K_RP / K_CRP, the Pauli
 * string S as (xmask, zmask): bit q of xmask/zmask = X/Z part on qubit q, both = Y. */
typedef struct {
    int32_t kind, q0, q1, param;
    uint64_t xmask, zmask;
} ogate_t;

/* ------------------------------------------------------------------------------------ */
/* primitives: "apply gate", "clone state", "inner product" (Appendix A, the three operations) */

static void apply_1q(cplx *psi, int n, int q, cplx m00, cplx m01, cplx m10, cplx m11) {
    const int64_t N = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (int64_t k = 0; k < N; ++k) {
        if (k & bit) continue;
        cplx a = psi[k], b = psi[k | bit];
        psi[k] = m00 * a + m01 * b;
        psi[k | bit] = m10 * a + m11 * b;
    }
}

static void apply_cz(cplx *psi, int n, int q0, int q1) {
    const int64_t N = (int64_t)1 << n;
    const int64_t m = ((int64_t)1 << q0) | ((int64_t)1 << q1);
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (int64_t k = 0; k < N; ++k)
        if ((k & m) == m) psi[k] = -psi[k];
}

static void apply_cnot(cplx *psi, int n, int control, int target) {
    const int64_t N = (int64_t)1 << n;
    const int64_t c = (int64_t)1 << control, t = (int64_t)1 << target;
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (int64_t k = 0; k < N; ++k) {
        if ((k & c) && !(k & t)) {
            cplx tmp = psi[k];
            psi[k] = psi[k | t];
            psi[k | t] = tmp;
        }
    }
}

/* A 2x2 matrix on qubit t, only on the amplitudes whose control qubit c is 1. With zero_rest the
 * amplitudes whose control is 0 are set to 0 (the derivative of the identity part). */
static void apply_c1q(cplx *psi, int n, int c, int t, cplx m00, cplx m01, cplx m10, cplx m11, int zero_rest) {
    const int64_t N = (int64_t)1 << n;
    const int64_t cb = (int64_t)1 << c, tb = (int64_t)1 << t;
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (int64_t k = 0; k < N; ++k) {
        if (k & tb) continue;
        if (!(k & cb)) {
            if (zero_rest) { psi[k] = 0; psi[k | tb] = 0; }
            continue;
        }
        cplx a = psi[k], b = psi[k | tb];
        psi[k] = m00 * a + m01 * b;
        psi[k | tb] = m10 * a + m11 * b;
    }
}

static void clone_state(cplx *dst, const cplx *src, int n) {
    memcpy(dst, src, sizeof(cplx) * ((size_t)1 << n));
}

static cplx inner(const cplx *a, const cplx *b, int n) { /* <a|b> */
    const int64_t N = (int64_t)1 << n;
    double re = 0.0, im = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : re, im) if (N >= 65536)
    for (int64_t k = 0; k < N; ++k) {
        cplx t = conj(a[k]) * b[k];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

static void zero_state(cplx *psi, int n) {
    memset(psi, 0, sizeof(cplx) * ((size_t)1 << n));
    psi[0] = 1.0;
}

static void apply_pauli_string(cplx *out, const cplx *psi, int n, uint64_t xm, uint64_t zm);

/*
 * exp(-i theta S / 2) = cos(theta/2) 1 - i sin(theta/2) S for a Pauli string S (S^2 = 1), on the
 * amplitudes whose control qubit (ctrl >= 0) is 1; the others keep their value for the gate and
 * its adjoint and become 0 for the derivatives. With c = cos(theta/2), s = sin(theta/2):
 *   mode 0: c psi - i s S psi        mode 1 (adjoint): c psi + i s S psi
 *   mode 2: -(s/2) psi - (i c/2) S psi   (d/dtheta)   mode 3: -(s/2) psi + (i c/2) S psi
 * S does not act on the control qubit, so S maps the control-1 subspace onto itself.
 */
static void apply_pauli_rotation(cplx *psi, int n, int ctrl, uint64_t xm, uint64_t zm, double theta, int mode) {
    const int64_t N = (int64_t)1 << n;
    const double c = cos(0.5 * theta), s = sin(0.5 * theta);
    cplx *sp = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    if (!sp) return;
    apply_pauli_string(sp, psi, n, xm, zm);
    cplx a, b;
    switch (mode) {
    case 0: a = c; b = -I * s; break;
    case 1: a = c; b = I * s; break;
    case 2: a = -0.5 * s; b = -0.5 * I * c; break;
    default: a = -0.5 * s; b = 0.5 * I * c; break;
    }
    const int64_t cb = ctrl >= 0 ? (int64_t)1 << ctrl : 0;
    for (int64_t k = 0; k < N; ++k) {
        if (cb && !(k & cb)) {
            if (mode >= 2) psi[k] = 0;
            continue;
        }
        psi[k] = a * psi[k] + b * sp[k];
    }
    free(sp);
}

/* mode: 0 = the gate, 1 = its adjoint, 2 = d/dtheta of the gate, 3 = adjoint of the derivative */
static void apply_gate_mode(cplx *psi, int n, const ogate_t *g, double theta, int mode) {
    const int kind = g->kind, q0 = g->q0, q1 = g->q1;
    const double c = cos(0.5 * theta), s = sin(0.5 * theta);
    cplx m00, m01, m10, m11;
    int controlled = 0, target = q0;
    switch (kind) {
    case K_RP: apply_pauli_rotation(psi, n, -1, g->xmask, g->zmask, theta, mode); return;
    case K_CRP: apply_pauli_rotation(psi, n, q0, g->xmask, g->zmask, theta, mode); return;
    case K_CRX: case K_CRY: case K_CRZ: {
        /* |0><0|_c (x) 1 + |1><1|_c (x) R_sigma(theta): R_sigma's matrix (as below) on the target,
           where the control is 1; its derivative is |1><1|_c (x) dR_sigma/dtheta */
        const int axis = kind - K_CRX + K_RX;
        const double cc = c, ss = s;
        cplx t[4];
        if (axis == K_RX) {
            if (mode < 2) { t[0] = cc; t[1] = -I * ss; t[2] = -I * ss; t[3] = cc; }
            else          { t[0] = -0.5 * ss; t[1] = -0.5 * I * cc; t[2] = -0.5 * I * cc; t[3] = -0.5 * ss; }
        } else if (axis == K_RY) {
            if (mode < 2) { t[0] = cc; t[1] = -ss; t[2] = ss; t[3] = cc; }
            else          { t[0] = -0.5 * ss; t[1] = -0.5 * cc; t[2] = 0.5 * cc; t[3] = -0.5 * ss; }
        } else {
            if (mode < 2) { t[0] = cc - I * ss; t[1] = 0; t[2] = 0; t[3] = cc + I * ss; }
            else          { t[0] = -0.5 * I * (cc - I * ss); t[1] = 0; t[2] = 0; t[3] = 0.5 * I * (cc + I * ss); }
        }
        m00 = t[0]; m01 = t[1]; m10 = t[2]; m11 = t[3];
        controlled = 1;
        target = q1;
        break;
    }
    case K_RX: /* exp(-i t X/2) = [[c, -i s], [-i s, c]] */
        if (mode < 2) { m00 = c; m01 = -I * s; m10 = -I * s; m11 = c; }
        else          { m00 = -0.5 * s; m01 = -0.5 * I * c; m10 = -0.5 * I * c; m11 = -0.5 * s; }
        break;
    case K_RY: /* exp(-i t Y/2) = [[c, -s], [s, c]] */
        if (mode < 2) { m00 = c; m01 = -s; m10 = s; m11 = c; }
        else          { m00 = -0.5 * s; m01 = -0.5 * c; m10 = 0.5 * c; m11 = -0.5 * s; }
        break;
    case K_RZ: /* exp(-i t Z/2) = diag(e^{-i t/2}, e^{+i t/2}) */
        if (mode < 2) { m00 = c - I * s; m01 = 0; m10 = 0; m11 = c + I * s; }
        else          { m00 = -0.5 * I * (c - I * s); m01 = 0; m10 = 0; m11 = 0.5 * I * (c + I * s); }
        break;
    case K_X: m00 = 0; m01 = 1; m10 = 1; m11 = 0; break;
    case K_Y: m00 = 0; m01 = -I; m10 = I; m11 = 0; break;
    case K_Z: m00 = 1; m01 = 0; m10 = 0; m11 = -1; break;
    case K_H: m00 = sqrt(0.5); m01 = sqrt(0.5); m10 = sqrt(0.5); m11 = -sqrt(0.5); break;
    case K_CZ: apply_cz(psi, n, q0, q1); return;            /* self-adjoint */
    case K_CNOT: apply_cnot(psi, n, q0, q1); return;        /* self-adjoint */
    default: return;
    }
    if (mode == 1 || mode == 3) { /* conjugate transpose */
        cplx t = m01;
        m00 = conj(m00); m11 = conj(m11); m01 = conj(m10); m10 = conj(t);
    }
    if (controlled) apply_c1q(psi, n, q0, target, m00, m01, m10, m11, mode >= 2);
    else apply_1q(psi, n, target, m00, m01, m10, m11);
}

static int is_rot(int kind) { return (kind >= K_RX && kind <= K_RZ) || (kind >= K_CRX && kind <= K_CRP); }

/* ------------------------------------------------------------------------------------ */
/* exported single operations (for the gate-level pins) */

/* Apply one gate (mode as above) to psi (interleaved complex, 2^n entries). */
int oracle_apply_gate(int n, double *psi, int kind, int q0, int q1, uint64_t xmask, uint64_t zmask, double theta,
                      int mode) {
    const ogate_t g = {kind, q0, q1, -1, xmask, zmask};
    apply_gate_mode((cplx *)psi, n, &g, theta, mode);
    return 0;
}

/* out = sigma psi for one Pauli string, one single-qubit Pauli matrix per qubit. */
static void apply_pauli_string(cplx *out, const cplx *psi, int n, uint64_t xm, uint64_t zm) {
    clone_state(out, psi, n);
    for (int q = 0; q < n; ++q) {
        int x = (int)((xm >> q) & 1u), z = (int)((zm >> q) & 1u);
        ogate_t g = {-1, q, -1, -1, 0, 0};
        if (x && z) g.kind = K_Y;
        else if (x) g.kind = K_X;
        else if (z) g.kind = K_Z;
        else continue;
        apply_gate_mode(out, n, &g, 0.0, 0);
    }
}

int oracle_apply_pauli(int n, const double *psi, double *out, uint64_t xmask, uint64_t zmask) {
    apply_pauli_string((cplx *)out, (const cplx *)psi, n, xmask, zmask);
    return 0;
}

/* out = H psi = sum_k c_k sigma_k psi */
static int hamiltonian_apply(cplx *out, const cplx *psi, int n, int T, const double *coeff,
                             const uint64_t *xm, const uint64_t *zm) {
    const int64_t N = (int64_t)1 << n;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    if (!tmp) return -1;
    memset(out, 0, sizeof(cplx) * (size_t)N);
    for (int k = 0; k < T; ++k) {
        apply_pauli_string(tmp, psi, n, xm[k], zm[k]);
#pragma omp parallel for schedule(static) if (N >= 65536)
        for (int64_t a = 0; a < N; ++a) out[a] += coeff[k] * tmp[a];
    }
    free(tmp);
    return 0;
}

int oracle_hamiltonian_apply(int n, const double *psi, double *out, int T, const double *coeff,
                             const uint64_t *xm, const uint64_t *zm) {
    return hamiltonian_apply((cplx *)out, (const cplx *)psi, n, T, coeff, xm, zm);
}

/* ------------------------------------------------------------------------------------ */
/* circuit-level definitions */

/* psi = W U_P ... U_1 |0>: every gate of the list in order (Sec. 2). */
static void run_circuit(cplx *psi, int n, const ogate_t *gates, int G, const double *theta, int deriv_param) {
    zero_state(psi, n);
    for (int k = 0; k < G; ++k) {
        const ogate_t *g = gates + k;
        if (is_rot(g->kind)) {
            const int mode = (g->param == deriv_param) ? 2 : 0;
            apply_gate_mode(psi, n, g, theta[g->param], mode);
        } else {
            apply_gate_mode(psi, n, g, 0.0, 0);
        }
    }
}

int oracle_state(int n, const ogate_t *gates, int G, const double *theta, double *psi_out) {
    run_circuit((cplx *)psi_out, n, gates, G, theta, -1);
    return 0;
}

/* |d_p psi>: the circuit with parametric gate p replaced by its derivative (Alg. 7). */
int oracle_deriv_state(int n, const ogate_t *gates, int G, const double *theta, int p, double *out) {
    run_circuit((cplx *)out, n, gates, G, theta, p);
    return 0;
}

/*
 * Quantum geometric tensor restricted to the parameter subset idx[0..m-1] (m = P for all of it).
 *   G_out (m x m, row-major, complex): G_ab = <d_{idx a} psi|d_{idx b} psi> - T_a^* T_b   (Eq. 4)
 *   T_out (m, complex):               T_a = <psi|d_{idx a} psi>                          (Sec. 2)
 *   psi_out (optional, 2^n complex):  the circuit state
 * Every derivative state is built from |0> on its own, so memory is (m + 1) states.
 */
int oracle_qgt(int n, const ogate_t *gates, int G, const double *theta, const int32_t *idx, int m,
               double *G_out, double *T_out, double *psi_out) {
    const size_t N = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * N);
    cplx *d = (cplx *)malloc(sizeof(cplx) * N * (size_t)m);
    if (!psi || !d) { free(psi); free(d); return -1; }
    run_circuit(psi, n, gates, G, theta, -1);
    /* Below 2^16 amplitudes the primitives run on one thread, so the independent derivative states
     * and entries are spread over the threads instead; every entry is computed the same way. */
#pragma omp parallel for schedule(dynamic) if (N < 65536)
    for (int a = 0; a < m; ++a) run_circuit(d + (size_t)a * N, n, gates, G, theta, idx[a]);
    cplx *T = (cplx *)T_out;
    cplx *Gm = (cplx *)G_out;
#pragma omp parallel for schedule(static) if (N < 65536)
    for (int a = 0; a < m; ++a) T[a] = inner(psi, d + (size_t)a * N, n);
#pragma omp parallel for schedule(dynamic) if (N < 65536)
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b)
            Gm[(size_t)a * m + b] = inner(d + (size_t)a * N, d + (size_t)b * N, n) - conj(T[a]) * T[b];
    if (psi_out) clone_state((cplx *)psi_out, psi, n);
    free(psi);
    free(d);
    return 0;
}

/* <E> = sum_k c_k <psi|sigma_k|psi> for the circuit state (Eq. 2's objective). */
int oracle_energy(int n, const ogate_t *gates, int G, const double *theta, int T, const double *coeff,
                  const uint64_t *xm, const uint64_t *zm, double *E_out) {
    const size_t N = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * N);
    cplx *hpsi = (cplx *)malloc(sizeof(cplx) * N);
    if (!psi || !hpsi) { free(psi); free(hpsi); return -1; }
    run_circuit(psi, n, gates, G, theta, -1);
    int rc = hamiltonian_apply(hpsi, psi, n, T, coeff, xm, zm);
    *E_out = creal(inner(psi, hpsi, n));
    free(psi);
    free(hpsi);
    return rc;
}

/* d<E>/d theta_{idx a} = 2 Re <psi|H|d_{idx a} psi> for a = 0..m-1 (product rule on Eq. 2). */
int oracle_gradient(int n, const ogate_t *gates, int G, const double *theta, int T, const double *coeff,
                    const uint64_t *xm, const uint64_t *zm, const int32_t *idx, int m, double *grad_out,
                    double *E_out) {
    const size_t N = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * N);
    cplx *hpsi = (cplx *)malloc(sizeof(cplx) * N);
    if (!psi || !hpsi) { free(psi); free(hpsi); return -1; }
    run_circuit(psi, n, gates, G, theta, -1);
    int rc = hamiltonian_apply(hpsi, psi, n, T, coeff, xm, zm);
    if (E_out) *E_out = creal(inner(psi, hpsi, n));
    int bad = 0;
    /* one derivative state per parameter, on one thread each below 2^16 amplitudes (see oracle_qgt) */
#pragma omp parallel if (N < 65536) reduction(| : bad)
    {
        cplx *d = (cplx *)malloc(sizeof(cplx) * N);
        if (!d) bad = 1;
#pragma omp for schedule(dynamic)
        for (int a = 0; a < m; ++a) {
            if (!d) continue;
            run_circuit(d, n, gates, G, theta, idx[a]);
            grad_out[a] = 2.0 * creal(inner(hpsi, d, n));
        }
        free(d);
    }
    free(psi);
    free(hpsi);
    return bad ? -1 : rc;
}

/* ------------------------------------------------------------------------------------ */
/* literal recurrences with operation counters (Alg. 1; Appendix A Alg. 3, 6, 8)          */
/*
 * The circuit's fixed gates are folded into the parametric ones: U_k applies the fixed gates
 * that precede rotation k, then the rotation; U_k^dagger undoes both in reverse; dU_k applies
 * the fixed gates, then the rotation's derivative. Each U_k, U_k^dagger, dU_k or dU_k^dagger
 * counts as ONE gate operation, each register copy as one clone, each <a|b> as one inner
 * product. counts = {gates, clones, inner products}.
 */
typedef struct {
    int n, G, P;
    const ogate_t *gates;
    const double *theta;
    int32_t *first; /* first[k] = index in gates[] of the first fixed gate belonging to U_k */
    int32_t *rot;   /* rot[k] = index in gates[] of rotation k */
    int64_t counts[3];
} circ_t;

static int circ_init(circ_t *c, int n, const ogate_t *gates, int G, const double *theta) {
    c->n = n; c->G = G; c->gates = gates; c->theta = theta;
    c->counts[0] = c->counts[1] = c->counts[2] = 0;
    int P = 0;
    for (int k = 0; k < G; ++k) P += is_rot(gates[k].kind);
    c->P = P;
    c->first = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P + 1));
    c->rot = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P + 1));
    if (!c->first || !c->rot) return -1;
    int p = 0, start = 0;
    for (int k = 0; k < G; ++k) {
        if (is_rot(gates[k].kind)) { c->first[p] = start; c->rot[p] = k; ++p; start = k + 1; }
    }
    return 0;
}

static void circ_free(circ_t *c) { free(c->first); free(c->rot); }

/* k is 0-based here: U_{k+1} in the paper's 1-based notation. mode: 0 U, 1 U^dag, 2 dU, 3 dU^dag */
static void op_U(circ_t *c, cplx *psi, int k, int mode) {
    const ogate_t *rg = c->gates + c->rot[k];
    const double th = c->theta[rg->param];
    c->counts[0]++;
    if (mode == 0 || mode == 2) {
        for (int f = c->first[k]; f < c->rot[k]; ++f) apply_gate_mode(psi, c->n, c->gates + f, 0.0, 0);
        apply_gate_mode(psi, c->n, rg, th, mode == 0 ? 0 : 2);
    } else {
        apply_gate_mode(psi, c->n, rg, th, mode == 1 ? 1 : 3);
        for (int f = c->rot[k] - 1; f >= c->first[k]; --f) apply_gate_mode(psi, c->n, c->gates + f, 0.0, 1);
    }
}

static void op_clone(circ_t *c, cplx *dst, const cplx *src) { c->counts[1]++; clone_state(dst, src, c->n); }
static cplx op_inner(circ_t *c, const cplx *a, const cplx *b) { c->counts[2]++; return inner(a, b, c->n); }
static void op_clone_in(circ_t *c, cplx *dst) { c->counts[1]++; zero_state(dst, c->n); }

/*
 * Algorithm 1 (Sec. 3), five registers chi, psi, phi, lambda, mu.
 * Outputs L (P x P complex, the i <= j triangle filled, the rest zero), T (P complex) and
 * counts. With skip_diag = 1 the diagonal is taken a priori as 1/4 (Eq. L_diag_when_single_pauli)
 * instead of <phi|phi>. psi_out (optional) receives register psi = U_P ... U_1 |in>.
 */
static int alg1_impl(int n, const ogate_t *gates, int G, const double *theta, int skip_diag, const uint8_t *want,
                     double *L_out, double *T_out, int64_t *counts, double *psi_out);

int oracle_alg1(int n, const ogate_t *gates, int G, const double *theta, int skip_diag, double *L_out,
                double *T_out, int64_t *counts, double *psi_out) {
    return alg1_impl(n, gates, G, theta, skip_diag, NULL, L_out, T_out, counts, psi_out);
}

/*
 * Algorithm 1 for a subset of its columns (Sec. 3: the inner loop over i for column j reads only
 * psi = psi_{j-1} and the gate list, so columns may be computed apart and gathered). want[j] != 0
 * (j = 0..P-1, the paper's j + 1) selects the columns whose inner loop runs; register psi still
 * advances through every gate. Column j's entries L_ij (i <= j) and T_j are written for the
 * selected columns only; the others are left zero. With every column selected this is Algorithm 1
 * exactly as oracle_alg1 runs it, operation for operation.
 */
int oracle_alg1_columns(int n, const ogate_t *gates, int G, const double *theta, const uint8_t *want,
                        double *L_out, double *T_out) {
    return alg1_impl(n, gates, G, theta, 1, want, L_out, T_out, NULL, NULL);
}

static int alg1_impl(int n, const ogate_t *gates, int G, const double *theta, int skip_diag, const uint8_t *want,
                     double *L_out, double *T_out, int64_t *counts, double *psi_out) {
    circ_t c;
    if (circ_init(&c, n, gates, G, theta)) { circ_free(&c); return -1; }
    const int P = c.P;
    const size_t N = (size_t)1 << n;
    cplx *chi = malloc(sizeof(cplx) * N), *psi = malloc(sizeof(cplx) * N), *phi = malloc(sizeof(cplx) * N),
         *lam = malloc(sizeof(cplx) * N), *mu = malloc(sizeof(cplx) * N);
    if (!chi || !psi || !phi || !lam || !mu) { free(chi); free(psi); free(phi); free(lam); free(mu); circ_free(&c); return -1; }
    cplx *L = (cplx *)L_out, *T = (cplx *)T_out;
    memset(L, 0, sizeof(cplx) * (size_t)P * (size_t)P);
    if (want) memset(T, 0, sizeof(cplx) * (size_t)P);
    if (P > 0) {
        op_clone_in(&c, chi);                 /* chi := |in>            */
        op_U(&c, chi, 0, 0);                  /* chi <- U_1             */
        op_clone(&c, psi, chi);               /* psi := chi             */
        if (!want || want[0]) {
            op_clone_in(&c, phi);             /* phi := |in>            */
            op_U(&c, phi, 0, 2);              /* phi <- dU_1            */
            T[0] = op_inner(&c, chi, phi);    /* T_1 = <chi|phi>        */
            L[0] = skip_diag ? 0.25 : op_inner(&c, phi, phi);
        }
        for (int j = 1; j < P; ++j) {         /* paper's j = 2..P       */
            if (want && !want[j]) {           /* another rank's column: */
                op_U(&c, psi, j, 0);          /* psi <- U_j only        */
                continue;
            }
            op_clone(&c, lam, psi);           /* lambda := psi          */
            op_clone(&c, phi, psi);           /* phi := psi             */
            op_U(&c, phi, j, 2);              /* phi <- dU_j            */
            L[(size_t)j * P + j] = skip_diag ? 0.25 : op_inner(&c, phi, phi);
            for (int i = j - 1; i >= 0; --i) {/* paper's i = j-1..1     */
                op_U(&c, phi, i + 1, 1);      /* phi <- U_{i+1}^dag     */
                op_U(&c, lam, i, 1);          /* lambda <- U_i^dag      */
                op_clone(&c, mu, lam);        /* mu := lambda           */
                op_U(&c, mu, i, 2);           /* mu <- dU_i             */
                L[(size_t)i * P + j] = op_inner(&c, mu, phi);
            }
            T[j] = op_inner(&c, chi, phi);    /* T_j = <chi|phi>        */
            op_U(&c, psi, j, 0);              /* psi <- U_j             */
        }
    }
    if (counts) { counts[0] = c.counts[0]; counts[1] = c.counts[1]; counts[2] = c.counts[2]; }
    if (psi_out && P > 0) clone_state((cplx *)psi_out, psi, n);
    free(chi); free(psi); free(phi); free(lam); free(mu);
    circ_free(&c);
    return 0;
}

/*
 * Appendix A, Alg. 3: every L_{i<=j} on its own, one register, gates after j eliminated.
 * L_ij = <in|phi> after phi := |in>, U_1..U_{j-1}, dU_j, U_j^dag..U_{i+1}^dag, dU_i^dag,
 * U_{i-1}^dag..U_1^dag.
 */
int oracle_alg3(int n, const ogate_t *gates, int G, const double *theta, double *L_out, int64_t *counts) {
    circ_t c;
    if (circ_init(&c, n, gates, G, theta)) { circ_free(&c); return -1; }
    const int P = c.P;
    const size_t N = (size_t)1 << n;
    cplx *phi = malloc(sizeof(cplx) * N), *in = malloc(sizeof(cplx) * N);
    if (!phi || !in) { free(phi); free(in); circ_free(&c); return -1; }
    zero_state(in, n);
    cplx *L = (cplx *)L_out;
    memset(L, 0, sizeof(cplx) * (size_t)P * (size_t)P);
    for (int j = 0; j < P; ++j) {
        for (int i = 0; i <= j; ++i) {
            op_clone_in(&c, phi);
            for (int k = 0; k < j; ++k) op_U(&c, phi, k, 0);
            op_U(&c, phi, j, 2);
            for (int k = j; k > i; --k) op_U(&c, phi, k, 1);
            op_U(&c, phi, i, 3);
            for (int k = i - 1; k >= 0; --k) op_U(&c, phi, k, 1);
            L[(size_t)i * P + j] = op_inner(&c, in, phi);
        }
    }
    if (counts) { counts[0] = c.counts[0]; counts[1] = c.counts[1]; counts[2] = c.counts[2]; }
    free(phi); free(in);
    circ_free(&c);
    return 0;
}

/*
 * Appendix A, Alg. 6: rolling suffix (psi), infix (phi) and prefix (mu), plus lambda.
 * skip_last = 1 omits the update phi <- U_1^dag at i = 1, whose result is never read; Table 1's
 * gate count for this algorithm assumes it is omitted.
 */
int oracle_alg6(int n, const ogate_t *gates, int G, const double *theta, int skip_last, double *L_out,
                int64_t *counts) {
    circ_t c;
    if (circ_init(&c, n, gates, G, theta)) { circ_free(&c); return -1; }
    const int P = c.P;
    const size_t N = (size_t)1 << n;
    cplx *psi = malloc(sizeof(cplx) * N), *phi = malloc(sizeof(cplx) * N), *lam = malloc(sizeof(cplx) * N),
         *mu = malloc(sizeof(cplx) * N);
    if (!psi || !phi || !lam || !mu) { free(psi); free(phi); free(lam); free(mu); circ_free(&c); return -1; }
    cplx *L = (cplx *)L_out;
    memset(L, 0, sizeof(cplx) * (size_t)P * (size_t)P);
    op_clone_in(&c, psi);
    for (int j = 0; j < P; ++j) {
        op_clone(&c, mu, psi);
        op_clone(&c, phi, psi);
        op_U(&c, phi, j, 2);
        for (int i = j; i >= 0; --i) {
            op_clone(&c, lam, phi);
            op_U(&c, lam, i, 3);
            L[(size_t)i * P + j] = op_inner(&c, mu, lam);
            if (!(skip_last && i == 0)) op_U(&c, phi, i, 1);
            if (i > 0) op_U(&c, mu, i - 1, 1);
        }
        op_U(&c, psi, j, 0);
    }
    if (counts) { counts[0] = c.counts[0]; counts[1] = c.counts[1]; counts[2] = c.counts[2]; }
    free(psi); free(phi); free(lam); free(mu);
    circ_free(&c);
    return 0;
}

/*
 * Appendix A, Alg. 8: every derivative state in its own register, from a rolling suffix;
 * then L_ij = <phi_i|phi_j> for i <= j. (P + 1 registers.)
 */
int oracle_alg8(int n, const ogate_t *gates, int G, const double *theta, double *L_out, int64_t *counts) {
    circ_t c;
    if (circ_init(&c, n, gates, G, theta)) { circ_free(&c); return -1; }
    const int P = c.P;
    const size_t N = (size_t)1 << n;
    cplx *psi = malloc(sizeof(cplx) * N), *d = malloc(sizeof(cplx) * N * (size_t)(P > 0 ? P : 1));
    if (!psi || !d) { free(psi); free(d); circ_free(&c); return -1; }
    cplx *L = (cplx *)L_out;
    memset(L, 0, sizeof(cplx) * (size_t)P * (size_t)P);
    op_clone_in(&c, psi);
    for (int i = 0; i < P; ++i) {
        cplx *di = d + (size_t)i * N;
        op_clone(&c, di, psi);
        op_U(&c, di, i, 2);
        for (int k = i + 1; k < P; ++k) op_U(&c, di, k, 0);
        op_U(&c, psi, i, 0);
    }
    for (int j = 0; j < P; ++j)
        for (int i = 0; i <= j; ++i) L[(size_t)i * P + j] = op_inner(&c, d + (size_t)i * N, d + (size_t)j * N);
    if (counts) { counts[0] = c.counts[0]; counts[1] = c.counts[1]; counts[2] = c.counts[2]; }
    free(psi); free(d);
    circ_free(&c);
    return 0;
}

/* Number of OpenMP threads the oracle's loops use (1 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
void oracle_set_num_threads(int t) { if (t > 0) omp_set_num_threads(t); }
#else
int oracle_num_threads(void) { return 1; }
void oracle_set_num_threads(int t) { (void)t; }
#endif

/*
 * Everything a QNG step needs, restricted to the parameter subset idx[0..m-1], in one sweep of
 * derivative states (for large states where the full set is out of reach):
 *   G_out (m x m complex, Eq. 4), T_out (m complex), grad_out (m, 2 Re <psi|H|d psi>), E_out.
 * Memory: m + 2 states.
 */
int oracle_sampled(int n, const ogate_t *gates, int G, const double *theta, int T, const double *coeff,
                   const uint64_t *xm, const uint64_t *zm, const int32_t *idx, int m, double *G_out, double *T_out,
                   double *grad_out, double *E_out) {
    const size_t N = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * N);
    cplx *hpsi = (cplx *)malloc(sizeof(cplx) * N);
    cplx *d = (cplx *)malloc(sizeof(cplx) * N * (size_t)(m > 0 ? m : 1));
    if (!psi || !hpsi || !d) { free(psi); free(hpsi); free(d); return -1; }
    run_circuit(psi, n, gates, G, theta, -1);
    int rc = hamiltonian_apply(hpsi, psi, n, T, coeff, xm, zm);
    *E_out = creal(inner(psi, hpsi, n));
    cplx *Tc = (cplx *)T_out, *Gc = (cplx *)G_out;
#pragma omp parallel for schedule(dynamic) if (N < 65536)
    for (int a = 0; a < m; ++a) {
        cplx *da = d + (size_t)a * N;
        run_circuit(da, n, gates, G, theta, idx[a]);
        Tc[a] = inner(psi, da, n);
        grad_out[a] = 2.0 * creal(inner(hpsi, da, n));
    }
#pragma omp parallel for schedule(dynamic) if (N < 65536)
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b)
            Gc[(size_t)a * m + b] = inner(d + (size_t)a * N, d + (size_t)b * N, n) - conj(Tc[a]) * Tc[b];
    free(psi);
    free(hpsi);
    free(d);
    return rc;
}
