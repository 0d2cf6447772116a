/* FP64 CPU oracle of the QAOA MaxCut energy and adjoint gradient
 * (TEST INFRASTRUCTURE: only tests/, the smoke check and the benchmark's CPU
 * baseline load it; the CUDA library shares no code with it).
 *
 * A plain C restatement of the QuPack QAOA evaluation (§6.2) with the ansatz
 * of §5.2: start from |+>^n; layer l applies the cost layer
 * exp(-i gs gamma_l C) with C(x) = sum over edges (a, b) of z_a z_b,
 * z_q = 1 - 2 x_q, then RX(beta_l) = exp(-i beta_l X / 2) on every qubit
 * (§2.3.3).  E = <psi|C|psi>.  The gradient is the adjoint method (§4.1, §7.2):
 * lam = C psi, then going back through the layers,
 *   dE/dbeta_l  = sum_q Im <lam|X_q|psi>   (taken after the mixer of layer l;
 *                                          X_q commutes with every RX of it),
 *   undo the mixer on psi and lam,
 *   dE/dgamma_l = 2 gs Im <lam|C|psi>,
 *   undo the cost layer on psi and lam.
 * One loop per gate over the whole state, FP64 complex, in the paper's
 * order; loops over amplitudes run under OpenMP when it is enabled (the
 * paper's own CPU runs use OpenMP), with the thread count given by the
 * caller.  Sums reduce per thread, so results do not depend on the thread
 * count beyond rounding.
 *
 * Parity pins (tests/test_qaoa_c_oracle.py): the K5 depth-10 expectation and
 * 20 gradients printed in §6.2.2; gamma = 0 (E = 0 and dE/dbeta = 0 for
 * every beta, since RX^n leaves |+>^n unchanged up to a phase); central finite
 * differences of E at random angles. */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* C(x) for every basis state x (little endian: qubit q is bit q of x). */
static void cost_values(int n, const int* edges, int n_edges, double* C) {
  const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; ++x) {
    int s = 0;
    for (int e = 0; e < n_edges; ++e) {
      const int za = ((x >> edges[2 * e]) & 1) ? -1 : 1;
      const int zb = ((x >> edges[2 * e + 1]) & 1) ? -1 : 1;
      s += za * zb;
    }
    C[x] = (double)s;
  }
}

/* v <- [[c, -i s], [-i s, c]] v on qubit q (RX(theta), c = cos theta/2, s = sin theta/2). */
static void apply_rx(cplx* v, int n, int q, double c, double s) {
  const int64_t half = (int64_t)1 << (n - 1), bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < half; ++k) {
    const int64_t i0 = ((k >> q) << (q + 1)) | (k & (bit - 1)), i1 = i0 | bit;
    const cplx a0 = v[i0], a1 = v[i1];
    v[i0] = c * a0 - I * s * a1;
    v[i1] = c * a1 - I * s * a0;
  }
}

/* v <- exp(-i t C) v */
static void apply_cost(cplx* v, const double* C, int n, double t) {
  const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; ++x) v[x] *= cexp(-I * t * C[x]);
}

/* Im <lam|X_q|psi> = Im sum_x conj(lam[x]) psi[x ^ 2^q] */
static double im_lam_x_psi(const cplx* lam, const cplx* psi, int n, int q) {
  const int64_t N = (int64_t)1 << n, bit = (int64_t)1 << q;
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
  for (int64_t x = 0; x < N; ++x) acc += cimag(conj(lam[x]) * psi[x ^ bit]);
  return acc;
}

/* Im <lam|C|psi> */
static double im_lam_c_psi(const cplx* lam, const cplx* psi, const double* C, int n) {
  const int64_t N = (int64_t)1 << n;
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
  for (int64_t x = 0; x < N; ++x) acc += C[x] * cimag(conj(lam[x]) * psi[x]);
  return acc;
}

/* Energy and gradients of one evaluation.  edges: int[2 n_edges]; gamma, beta,
 * dgamma, dbeta: double[p].  threads <= 0: the OpenMP default.  Returns 0, or
 * -1 on bad arguments or a failed allocation. */
int qaoa_oracle_eval(int n, const int* edges, int n_edges, int p, const double* gamma, const double* beta,
                     double gs, int threads, double* energy, double* dgamma, double* dbeta) {
  if (n < 1 || n > 34 || p < 1 || n_edges < 0 || !edges || !gamma || !beta || !energy || !dgamma || !dbeta)
    return -1;
  for (int e = 0; e < 2 * n_edges; ++e)
    if (edges[e] < 0 || edges[e] >= n) return -1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  const int64_t N = (int64_t)1 << n;
  double* C = (double*)malloc(sizeof(double) * (size_t)N);
  cplx* psi = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  cplx* lam = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  if (!C || !psi || !lam) {
    free(C);
    free(psi);
    free(lam);
    return -1;
  }
  cost_values(n, edges, n_edges, C);
  const double amp = pow(2.0, -0.5 * n);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; ++x) psi[x] = amp;
  for (int l = 0; l < p; ++l) {  // forward: cost layer, then the mixer
    apply_cost(psi, C, n, gs * gamma[l]);
    const double c = cos(0.5 * beta[l]), s = sin(0.5 * beta[l]);
    for (int q = 0; q < n; ++q) apply_rx(psi, n, q, c, s);
  }
  double E = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : E)
  for (int64_t x = 0; x < N; ++x) {
    const double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    E += C[x] * pr;
    lam[x] = C[x] * psi[x];
  }
  *energy = E;
  for (int l = p - 1; l >= 0; --l) {  // reverse sweep
    double gb = 0.0;
    for (int q = 0; q < n; ++q) gb += im_lam_x_psi(lam, psi, n, q);
    dbeta[l] = gb;
    const double c = cos(0.5 * beta[l]), s = -sin(0.5 * beta[l]);  // RX(beta)^dagger = RX(-beta)
    for (int q = 0; q < n; ++q) {
      apply_rx(psi, n, q, c, s);
      apply_rx(lam, n, q, c, s);
    }
    dgamma[l] = 2.0 * gs * im_lam_c_psi(lam, psi, C, n);
    apply_cost(psi, C, n, -gs * gamma[l]);
    apply_cost(lam, C, n, -gs * gamma[l]);
  }
  free(C);
  free(psi);
  free(lam);
  return 0;
}

/* Threads an evaluation would use with threads <= 0 (1 without OpenMP). */
int qaoa_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
