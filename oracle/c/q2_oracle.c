/*
 * Plain C restatement of the oracle's state-vector definitions (test
 * infrastructure only: used by the tests, the golden-value script and the
 * CPU-baseline timing; never by the library's compute path).
 *
 * Double precision complex, one amplitude loop per operation, OpenMP over
 * the amplitude index.  No blocking, fusion or reordering.
 *
 *   (P psi)[i] = i^{|x&z|} (-1)^{|(i^x)&z|} psi[i^x]      Pauli string (x, z)
 *   exp(-i phi/2 P) psi = cos(phi/2) psi - i sin(phi/2) P psi   (product
 *                         formula after Eq. ucc)
 *   E = sum_t c_t <psi|P_t|psi>                            Eq. qubit-ham-detail
 *   g_k = Im <lambda_k|P_k|psi_k>                          Algorithm 1
 *
 * States are interleaved (re, im) double arrays of 2^n complex entries.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static cplx ipow(int k)
{
    switch (k & 3) {
    case 0: return 1.0;
    case 1: return I;
    case 2: return -1.0;
    default: return -I;
    }
}

static int parity64(uint64_t v) { return __builtin_parityll(v); }
static int popcount64(uint64_t v) { return __builtin_popcountll(v); }

int q2o_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void q2o_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* out = P psi */
static void pauli_apply(int n, const cplx *psi, cplx *out, uint64_t x, uint64_t z)
{
    const int64_t dim = (int64_t)1 << n;
    const cplx ph = ipow(popcount64(x & z));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) {
        uint64_t src = (uint64_t)i ^ x;
        double s = parity64(src & z) ? -1.0 : 1.0;
        out[i] = ph * s * psi[src];
    }
}

/* psi <- exp(-i phi/2 P) psi, out of place through tmp */
static void rotation_apply(int n, cplx *psi, cplx *tmp, uint64_t x, uint64_t z, double phi)
{
    const int64_t dim = (int64_t)1 << n;
    pauli_apply(n, psi, tmp, x, z);
    const double c = cos(0.5 * phi), s = sin(0.5 * phi);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i)
        psi[i] = c * psi[i] - I * s * tmp[i];
}

void q2o_hf_state(int n, int n_elec, double *psi)
{
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(double) * 2 * (size_t)dim);
    psi[2 * (((int64_t)1 << n_elec) - 1)] = 1.0;
}

int q2o_apply_rotations(int n, double *psi_d, int64_t n_rot, const uint64_t *x,
                        const uint64_t *z, const double *phi)
{
    cplx *psi = (cplx *)psi_d;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * ((size_t)1 << n));
    if (!tmp) return 1;
    for (int64_t k = 0; k < n_rot; ++k)
        rotation_apply(n, psi, tmp, x[k], z[k], phi[k]);
    free(tmp);
    return 0;
}

/* E = sum_t c_t Re <psi|P_t psi>; also <psi|psi> */
int q2o_expectation(int n, const double *psi_d, int64_t n_terms, const uint64_t *x,
                    const uint64_t *z, const double *c, double *e_out, double *norm_out)
{
    const cplx *psi = (const cplx *)psi_d;
    const int64_t dim = (int64_t)1 << n;
    double e = 0.0;
    for (int64_t t = 0; t < n_terms; ++t) {
        const cplx ph = ipow(popcount64(x[t] & z[t]));
        double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
        for (int64_t i = 0; i < dim; ++i) {
            uint64_t src = (uint64_t)i ^ x[t];
            double s = parity64(src & z[t]) ? -1.0 : 1.0;
            acc += creal(conj(psi[i]) * ph * s * psi[src]);
        }
        e += c[t] * acc;
    }
    double nrm = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : nrm)
    for (int64_t i = 0; i < dim; ++i)
        nrm += creal(conj(psi[i]) * psi[i]);
    *e_out = e;
    if (norm_out) *norm_out = nrm;
    return 0;
}

/* lam = H psi */
int q2o_apply_hamiltonian(int n, const double *psi_d, double *lam_d, int64_t n_terms,
                          const uint64_t *x, const uint64_t *z, const double *c)
{
    const cplx *psi = (const cplx *)psi_d;
    cplx *lam = (cplx *)lam_d;
    const int64_t dim = (int64_t)1 << n;
    memset(lam, 0, sizeof(cplx) * (size_t)dim);
    for (int64_t t = 0; t < n_terms; ++t) {
        const cplx ph = ipow(popcount64(x[t] & z[t]));
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < dim; ++i) {
            uint64_t src = (uint64_t)i ^ x[t];
            double s = parity64(src & z[t]) ? -1.0 : 1.0;
            lam[i] += c[t] * ph * s * psi[src];
        }
    }
    return 0;
}

/* Algorithm 1 (reverse mode), gradient per rotation angle.  Returns E. */
int q2o_energy_grad(int n, int n_elec, int64_t n_rot, const uint64_t *rx, const uint64_t *rz,
                    const double *phi, int64_t n_terms, const uint64_t *hx, const uint64_t *hz,
                    const double *hc, double *e_out, double *g_out)
{
    const int64_t dim = (int64_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *lam = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    if (!psi || !lam || !tmp) { free(psi); free(lam); free(tmp); return 1; }
    q2o_hf_state(n, n_elec, (double *)psi);
    for (int64_t k = 0; k < n_rot; ++k)
        rotation_apply(n, psi, tmp, rx[k], rz[k], phi[k]);
    q2o_apply_hamiltonian(n, (const double *)psi, (double *)lam, n_terms, hx, hz, hc);
    double e = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : e)
    for (int64_t i = 0; i < dim; ++i)
        e += creal(conj(psi[i]) * lam[i]);
    for (int64_t k = n_rot - 1; k >= 0; --k) {
        pauli_apply(n, psi, tmp, rx[k], rz[k]);
        double gi = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : gi)
        for (int64_t i = 0; i < dim; ++i)
            gi += cimag(conj(lam[i]) * tmp[i]);
        g_out[k] = gi;
        rotation_apply(n, psi, tmp, rx[k], rz[k], -phi[k]);
        rotation_apply(n, lam, tmp, rx[k], rz[k], -phi[k]);
    }
    *e_out = e;
    free(psi);
    free(lam);
    free(tmp);
    return 0;
}
