/*
 * CPU oracle for the statevector hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header or table with the CUDA
 * path; it is the plain definition, written for a reader to check by eye:
 *
 *   - psi starts at e_0 (psi_0 = 1) and every gate of the list is applied
 *     to the 2^n complex128 amplitudes one at a time, in list order
 *     (full-circuit statevector simulation, Sec. III-B; the paper hands
 *     this work to Qiskit Aer, Listing 3).
 *   - index bit q of an amplitude is qubit q (little-endian, as in the
 *     Statevector.probabilities call of Listings 2 and 3).
 *   - probabilities p_i = |psi_i|^2 (Listing 3), norm = sum_i p_i summed with
 *     Neumaier's compensated summation (Neumaier 1974).
 *
 * Gate matrices (the paper is silent on them; it uses Qiskit 1.0.2, Sec. V-A,
 * whose conventions are followed, global phases included):
 *   H = [[1,1],[1,-1]]/sqrt2, X, Y = [[0,-i],[i,0]], Z = diag(1,-1),
 *   S = diag(1,i), T = diag(1,e^{i pi/4}),
 *   RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]],
 *   RZ(t) = diag(e^{-it/2}, e^{it/2}),          c = cos t/2, s = sin t/2
 *   U3(t,p,l) = [[c, -e^{il} s], [e^{ip} s, e^{i(p+l)} c]],
 *   two-qubit gates act on the local index b(q0) + 2*b(q1):
 *   CX (q0 = control, q1 = target), CZ = diag(1,1,1,-1),
 *   RZZ(t) = diag(e^{-it/2}, e^{it/2}, e^{it/2}, e^{-it/2}), SWAP.
 *
 * Parity pins (tests marked "not gpu"): a numpy dense-unitary brute force for
 * n <= 8, textbook gate identities, and closed forms (GHZ, QFT of a basis
 * state, U U^dagger = I, norm 1).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double OR_PI = 3.14159265358979323846264338327950288;

/* Same memory layout as the gate records the tests pass in. */
typedef struct {
    int32_t op, q0, q1;
    double theta, phi, lam;
} or_gate;

enum { OR_H, OR_X, OR_Y, OR_Z, OR_S, OR_T, OR_RX, OR_RY, OR_RZ, OR_U3,
       OR_CX, OR_CZ, OR_RZZ, OR_SWAP, OR_NOPS };

/* Number of qubits the gate acts on, 0 for an unknown opcode. */
int oracle_gate_arity(int op)
{
    if (op < 0 || op >= OR_NOPS) return 0;
    return op >= OR_CX ? 2 : 1;
}

/* Row-major 2x2 (arity 1) or 4x4 (arity 2) matrix of a gate, as interleaved
 * (re, im) doubles.  Returns the arity, or 0 for an unknown opcode. */
int oracle_gate_matrix(const or_gate* g, double* out)
{
    cplx m[16];
    int k = oracle_gate_arity(g->op);
    if (k == 0) return 0;
    for (int i = 0; i < 16; i++) m[i] = 0;
    const double r2 = 1.0 / sqrt(2.0);
    const double c = cos(g->theta / 2), s = sin(g->theta / 2);
    switch (g->op) {
    case OR_H:  m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; break;
    case OR_X:  m[1] = 1; m[2] = 1; break;
    case OR_Y:  m[1] = -I; m[2] = I; break;
    case OR_Z:  m[0] = 1; m[3] = -1; break;
    case OR_S:  m[0] = 1; m[3] = I; break;
    case OR_T:  m[0] = 1; m[3] = cexp(I * OR_PI / 4); break;
    case OR_RX: m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    case OR_RY: m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
    case OR_RZ: m[0] = cexp(-I * g->theta / 2); m[3] = cexp(I * g->theta / 2); break;
    case OR_U3:
        m[0] = c;
        m[1] = -cexp(I * g->lam) * s;
        m[2] = cexp(I * g->phi) * s;
        m[3] = cexp(I * (g->phi + g->lam)) * c;
        break;
    /* 4x4, row r / column col = local index b(q0) + 2*b(q1) */
    case OR_CX:   /* flips b(q1) when b(q0) = 1: 1 <-> 3 */
        m[0 * 4 + 0] = 1; m[3 * 4 + 1] = 1; m[2 * 4 + 2] = 1; m[1 * 4 + 3] = 1; break;
    case OR_CZ:
        m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1; break;
    case OR_RZZ: {
        cplx a = cexp(-I * g->theta / 2), b = cexp(I * g->theta / 2);
        m[0] = a; m[5] = b; m[10] = b; m[15] = a; break;
    }
    case OR_SWAP: /* 1 <-> 2 */
        m[0] = 1; m[2 * 4 + 1] = 1; m[1 * 4 + 2] = 1; m[15] = 1; break;
    }
    int dim = 1 << k;
    for (int i = 0; i < dim * dim; i++) {
        out[2 * i] = creal(m[i]);
        out[2 * i + 1] = cimag(m[i]);
    }
    return k;
}

/* Checks a gate list against an n-qubit register: known opcode, qubits in
 * range, distinct operands for two-qubit gates.  Returns the index of the
 * first bad gate, or -1 when all are valid. */
long oracle_validate(int n, const or_gate* g, size_t ng)
{
    for (size_t t = 0; t < ng; t++) {
        int k = oracle_gate_arity(g[t].op);
        if (k == 0) return (long)t;
        if (g[t].q0 < 0 || g[t].q0 >= n) return (long)t;
        if (k == 2 && (g[t].q1 < 0 || g[t].q1 >= n || g[t].q1 == g[t].q0)) return (long)t;
    }
    return -1;
}

/* psi <- e_basis. */
void oracle_init(int n, double* psi_ri, uint64_t basis)
{
    size_t dim = (size_t)1 << n;
    memset(psi_ri, 0, dim * 2 * sizeof(double));
    psi_ri[2 * basis] = 1.0;
}

static void apply_1q(int n, cplx* psi, int q, const cplx u[4])
{
    const size_t dim = (size_t)1 << n, bit = (size_t)1 << q;
    #pragma omp parallel for schedule(static)
    for (size_t i = 0; i < dim; i++) {
        if (i & bit) continue;
        size_t j = i | bit;
        cplx a0 = psi[i], a1 = psi[j];
        psi[i] = u[0] * a0 + u[1] * a1;
        psi[j] = u[2] * a0 + u[3] * a1;
    }
}

static void apply_2q(int n, cplx* psi, int q0, int q1, const cplx u[16])
{
    const size_t dim = (size_t)1 << n, b0 = (size_t)1 << q0, b1 = (size_t)1 << q1;
    #pragma omp parallel for schedule(static)
    for (size_t i = 0; i < dim; i++) {
        if ((i & b0) || (i & b1)) continue;
        size_t idx[4] = { i, i | b0, i | b1, i | b0 | b1 };  /* local index b(q0) + 2 b(q1) */
        cplx a[4], r[4];
        for (int k = 0; k < 4; k++) a[k] = psi[idx[k]];
        for (int row = 0; row < 4; row++) {
            r[row] = 0;
            for (int col = 0; col < 4; col++) r[row] += u[row * 4 + col] * a[col];
        }
        for (int k = 0; k < 4; k++) psi[idx[k]] = r[k];
    }
}

/* Applies the gates one by one, in list order, to psi (interleaved complex128,
 * 2^n entries).  Returns 0, or -1 - t when gate t is invalid (psi then holds
 * the result of gates 0..t-1). */
long oracle_apply(int n, double* psi_ri, const or_gate* g, size_t ng)
{
    cplx* psi = (cplx*)psi_ri;
    for (size_t t = 0; t < ng; t++) {
        if (oracle_validate(n, &g[t], 1) >= 0) return -1 - (long)t;
        double mr[32];
        cplx u[16];
        int k = oracle_gate_matrix(&g[t], mr);
        for (int i = 0; i < (1 << (2 * k)); i++) u[i] = mr[2 * i] + I * mr[2 * i + 1];
        if (k == 1) apply_1q(n, psi, g[t].q0, u);
        else apply_2q(n, psi, g[t].q0, g[t].q1, u);
    }
    return 0;
}

/* Simulates the circuit from |0...0>: init then apply. */
long oracle_run(int n, double* psi_ri, const or_gate* g, size_t ng)
{
    oracle_init(n, psi_ri, 0);
    return oracle_apply(n, psi_ri, g, ng);
}

/* p_i = re^2 + im^2. */
void oracle_probabilities(int n, const double* psi_ri, double* p)
{
    size_t dim = (size_t)1 << n;
    #pragma omp parallel for schedule(static)
    for (size_t i = 0; i < dim; i++)
        p[i] = psi_ri[2 * i] * psi_ri[2 * i] + psi_ri[2 * i + 1] * psi_ri[2 * i + 1];
}

/* Neumaier compensated sum of the probabilities. */
double oracle_norm(int n, const double* psi_ri)
{
    size_t dim = (size_t)1 << n;
    double s = 0.0, comp = 0.0;
    for (size_t i = 0; i < dim; i++) {
        double x = psi_ri[2 * i] * psi_ri[2 * i] + psi_ri[2 * i + 1] * psi_ri[2 * i + 1];
        double t = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - t) + x;
        else comp += (x - t) + s;
        s = t;
    }
    return s + comp;
}

/* Marginal distribution over the qubits set in mask: out[k] = sum of p_i over
 * all i whose mask bits, packed in ascending qubit order, equal k. */
void oracle_marginal(int n, const double* psi_ri, uint64_t mask, double* out)
{
    size_t dim = (size_t)1 << n;
    int m = 0;
    for (int q = 0; q < n; q++) if ((mask >> q) & 1) m++;
    memset(out, 0, ((size_t)1 << m) * sizeof(double));
    for (size_t i = 0; i < dim; i++) {
        size_t k = 0;
        int pos = 0;
        for (int q = 0; q < n; q++)
            if ((mask >> q) & 1) { k |= ((i >> q) & 1) << pos; pos++; }
        out[k] += psi_ri[2 * i] * psi_ri[2 * i] + psi_ri[2 * i + 1] * psi_ri[2 * i + 1];
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
