/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously correct complex128 state-vector routines used to
 * check the CUDA path.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the simulator itself never does.
 *
 * Conventions (Sec. 2.1 of the paper: amplitude index bits are the qubit
 * values, qubit 1 <-> least-significant bit; Pauli matrices as printed
 * there; Y = iXZ as in Sec. 2.4):
 *   - a Pauli string is (x, z) with per-qubit factor X^x Z^z and an extra
 *     i for every qubit where x = z = 1, so that the operator is
 *     P = i^{|x & z|} X^x Z^z, Hermitian, with Y on x = z = 1;
 *   - (P psi)[y] = i^{|x&z|} (-1)^{|z & (y ^ x)|} psi[y ^ x]
 *     because Z^z multiplies |w> by (-1)^{|z&w|} and X^x maps |w> to |w^x>.
 *   - exp(-i theta P) = cos(theta) I - i sin(theta) P since P^2 = I.
 *
 * The Trotter product of Eq. (trotter_decomp) is applied one term at a
 * time, in the order given by an explicit list of (term, angle) pairs that
 * the caller builds (group order, input order inside each group).
 *
 * The state is an array of 2^n interleaved (re, im) doubles.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int popc64(uint64_t v)
{
    int c = 0;
    while (v) { v &= v - 1; c++; }
    return c;
}

/* i^k for k mod 4, as (re, im) */
static void ipow(int k, double *re, double *im)
{
    switch (k & 3) {
    case 0: *re = 1; *im = 0; break;
    case 1: *re = 0; *im = 1; break;
    case 2: *re = -1; *im = 0; break;
    default: *re = 0; *im = -1; break;
    }
}

/* Phase factor ph(y) with (P psi)[y] = ph(y) psi[y ^ x]. */
static void pauli_phase(uint64_t x, uint64_t z, uint64_t y, double *re, double *im)
{
    int k = popc64(x & z) + 2 * (popc64(z & (y ^ x)) & 1);
    ipow(k, re, im);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* out = P psi (out must not alias psi). */
void oracle_apply_pauli(int n, const double *psi, double *out, uint64_t x, uint64_t z)
{
    int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < N; y++) {
        double pr, pi;
        pauli_phase(x, z, (uint64_t)y, &pr, &pi);
        int64_t s = (int64_t)((uint64_t)y ^ x);
        double ar = psi[2 * s], ai = psi[2 * s + 1];
        out[2 * y] = pr * ar - pi * ai;
        out[2 * y + 1] = pr * ai + pi * ar;
    }
}

/* psi <- exp(-i theta P) psi, in place, pair by pair. */
void oracle_apply_rotation(int n, double *psi, uint64_t x, uint64_t z, double theta)
{
    int64_t N = (int64_t)1 << n;
    double c = cos(theta), s = sin(theta);
    if (x == 0) {
        /* diagonal: P|y> = (-1)^{|z&y|} |y> */
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < N; y++) {
            double sg = (popc64(z & (uint64_t)y) & 1) ? -1.0 : 1.0;
            /* (c - i s sg) * psi */
            double ar = psi[2 * y], ai = psi[2 * y + 1];
            psi[2 * y] = c * ar + s * sg * ai;
            psi[2 * y + 1] = c * ai - s * sg * ar;
        }
        return;
    }
    uint64_t low = x & (~x + 1);  /* lowest set bit: pairs (y, y^x) with y bit clear */
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < N; y++) {
        if ((uint64_t)y & low) continue;
        int64_t w = (int64_t)((uint64_t)y ^ x);
        double ar = psi[2 * y], ai = psi[2 * y + 1];
        double br = psi[2 * w], bi = psi[2 * w + 1];
        double p1r, p1i, p2r, p2i;
        pauli_phase(x, z, (uint64_t)y, &p1r, &p1i);   /* (P psi)[y] = p1 * b */
        pauli_phase(x, z, (uint64_t)w, &p2r, &p2i);   /* (P psi)[w] = p2 * a */
        double qyr = p1r * br - p1i * bi, qyi = p1r * bi + p1i * br;
        double qwr = p2r * ar - p2i * ai, qwi = p2r * ai + p2i * ar;
        /* new = c*psi - i*s*(P psi);  -i*(u+iv) = v - i u */
        psi[2 * y] = c * ar + s * qyi;
        psi[2 * y + 1] = c * ai - s * qyr;
        psi[2 * w] = c * br + s * qwi;
        psi[2 * w + 1] = c * bi - s * qwr;
    }
}

/* Apply the listed rotations exp(-i angle[k] P_{term[k]}) for k = 0..L-1,
 * `reps` times over. */
void oracle_apply_sequence(int n, double *psi, const uint64_t *x, const uint64_t *z,
                           int64_t L, const int64_t *term, const double *angle,
                           int64_t reps)
{
    for (int64_t r = 0; r < reps; r++)
        for (int64_t k = 0; k < L; k++)
            oracle_apply_rotation(n, psi, x[term[k]], z[term[k]], angle[k]);
}

/* <psi| sum_k oc_k P_k |psi>  (real part; the imaginary part vanishes for
 * Hermitian P_k up to rounding). */
double oracle_expect(int n, const double *psi, int64_t mo, const uint64_t *ox,
                     const uint64_t *oz, const double *oc)
{
    int64_t N = (int64_t)1 << n;
    double total = 0.0;
    for (int64_t k = 0; k < mo; k++) {
        double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+:acc)
        for (int64_t y = 0; y < N; y++) {
            double pr, pi;
            pauli_phase(ox[k], oz[k], (uint64_t)y, &pr, &pi);
            int64_t s = (int64_t)((uint64_t)y ^ ox[k]);
            double br = psi[2 * s], bi = psi[2 * s + 1];
            double qr = pr * br - pi * bi, qi = pr * bi + pi * br;
            double ar = psi[2 * y], ai = psi[2 * y + 1];
            acc += ar * qr + ai * qi;      /* Re(conj(a) * q) */
        }
        total += oc[k] * acc;
    }
    return total;
}

/* Gradient of f = <psi_T| O |psi_T> with psi_T = prod_k exp(-i a_k P_{t_k}) psi_0
 * (the listed sequence repeated `reps` times) with respect to the Hamiltonian
 * coefficients c_j, where a_k = c_{t_k} * dtk[k].
 *
 * Reverse sweep over single rotations: with phi_l the state after
 * rotation l and lambda_l = U_{l+1}^dag ... U_L^dag O psi_T,
 *     d f / d a_l = 2 Im <lambda_l| P_l |phi_l>,
 * and d f / d c_j = sum over l with t_l = j of dtk[l] * d f / d a_l.
 * psi0 is left untouched; grad has m entries; the return value is f. */
double oracle_grad(int n, const double *psi0, int64_t m, const uint64_t *x,
                   const uint64_t *z, const double *c, int64_t L, const int64_t *term,
                   const double *dtk, int64_t reps, int64_t mo, const uint64_t *ox,
                   const uint64_t *oz, const double *oc, double *grad)
{
    int64_t N = (int64_t)1 << n;
    size_t bytes = (size_t)N * 2 * sizeof(double);
    double *phi = (double *)malloc(bytes);
    double *lam = (double *)malloc(bytes);
    double *tmp = (double *)malloc(bytes);
    memcpy(phi, psi0, bytes);
    for (int64_t r = 0; r < reps; r++)
        for (int64_t k = 0; k < L; k++)
            oracle_apply_rotation(n, phi, x[term[k]], z[term[k]], c[term[k]] * dtk[k]);
    double f = oracle_expect(n, phi, mo, ox, oz, oc);
    /* lam = O phi */
    memset(lam, 0, bytes);
    for (int64_t k = 0; k < mo; k++) {
        oracle_apply_pauli(n, phi, tmp, ox[k], oz[k]);
        for (int64_t y = 0; y < 2 * N; y++) lam[y] += oc[k] * tmp[y];
    }
    for (int64_t j = 0; j < m; j++) grad[j] = 0.0;
    for (int64_t r = reps - 1; r >= 0; r--) {
        for (int64_t k = L - 1; k >= 0; k--) {
            int64_t j = term[k];
            /* 2 Im <lam| P |phi> */
            oracle_apply_pauli(n, phi, tmp, x[j], z[j]);
            double im = 0.0;
#pragma omp parallel for schedule(static) reduction(+:im)
            for (int64_t y = 0; y < N; y++) {
                double ar = lam[2 * y], ai = lam[2 * y + 1];
                double br = tmp[2 * y], bi = tmp[2 * y + 1];
                im += ar * bi - ai * br;       /* Im(conj(a) * b) */
            }
            grad[j] += 2.0 * im * dtk[k];
            double a = c[j] * dtk[k];
            oracle_apply_rotation(n, phi, x[j], z[j], -a);
            oracle_apply_rotation(n, lam, x[j], z[j], -a);
        }
    }
    free(phi); free(lam); free(tmp);
    return f;
}
