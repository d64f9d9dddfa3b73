/*
 * Plain FP64 CPU oracle, complex potentials (TEST INFRASTRUCTURE ONLY; see
 * fdtd_oracle.c for the conventions: padded (N+2)^3 fields with a zero
 * shell, x fastest, interior site (i, j, k) at ((i, j, k) - (N+1)/2) a).
 *
 * The paper names complex potentials as a further application of the
 * method (Sec. VIII).  With V = V_R + i V_I the wavefunction is complex and
 * the update of Eq. updateeq keeps its form with complex coefficients
 *     A = (1 - dtau V / 2) / (1 + dtau V / 2),   B = 1 / (1 + dtau V / 2),
 *     Psi(tau + dtau) = A Psi + (B dtau / 2m) sum_i (D . PsiHat)_i .
 * A complex field is held as two real padded arrays (re, im).  The energy
 * is the Rayleigh quotient with the Hermitian inner product,
 *     E = sum conj(psi) [ -(1/2m) sum_i (D . PsiHat)_i + V psi ] / sum |psi|^2,
 * whose imaginary part is <V_I> (the kinetic part is real for the real
 * symmetric lattice Laplacian).  Renormalisation divides by
 * sqrt(sum |psi|^2 a^3); the symmetry masks act on both parts.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PIDX(n, i, j, k) \
  ((((size_t)(k)) * (size_t)((n) + 2) + (size_t)(j)) * (size_t)((n) + 2) + (size_t)(i))
#define DIDX(n, i, j, k) \
  ((((size_t)(k) - 1) * (size_t)(n) + ((size_t)(j) - 1)) * (size_t)(n) + ((size_t)(i) - 1))

int oracle_impose_parity(int n, int mask, double* psi);  /* fdtd_oracle.c (Sec. IV) */

/* sum_i (D . PsiHat)_i at an interior site of one real padded field (zero shell) */
static double lap_at(int n, double a, const double* p, int i, int j, int k) {
  double c = p[PIDX(n, i, j, k)];
  double dxx = (p[PIDX(n, i - 1, j, k)] - 2.0 * c + p[PIDX(n, i + 1, j, k)]) / (a * a);
  double dyy = (p[PIDX(n, i, j - 1, k)] - 2.0 * c + p[PIDX(n, i, j + 1, k)]) / (a * a);
  double dzz = (p[PIDX(n, i, j, k - 1)] - 2.0 * c + p[PIDX(n, i, j, k + 1)]) / (a * a);
  return dxx + dyy + dzz;
}

/* One update (Eq. updateeq, complex A and B).  v_re, v_im: dense N^3. */
void oracle_cstep(int n, double a, double dtau, double mass, const double* v_re, const double* v_im,
                  const double* in_re, const double* in_im, double* out_re, double* out_im) {
  size_t cells = (size_t)(n + 2) * (n + 2) * (n + 2);
  memset(out_re, 0, sizeof(double) * cells);
  memset(out_im, 0, sizeof(double) * cells);
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        double complex vv = v_re[DIDX(n, i, j, k)] + I * v_im[DIDX(n, i, j, k)];
        double complex A = (1.0 - 0.5 * dtau * vv) / (1.0 + 0.5 * dtau * vv);
        double complex B = 1.0 / (1.0 + 0.5 * dtau * vv);
        double complex psi = in_re[PIDX(n, i, j, k)] + I * in_im[PIDX(n, i, j, k)];
        double complex lap = lap_at(n, a, in_re, i, j, k) + I * lap_at(n, a, in_im, i, j, k);
        double complex r = A * psi + B * dtau / (2.0 * mass) * lap;
        out_re[PIDX(n, i, j, k)] = creal(r);
        out_im[PIDX(n, i, j, k)] = cimag(r);
      }
}

/* Lattice sums with the Hermitian inner product:
 *   out[0] = S0 = sum |psi|^2
 *   out[1], out[2] = Re, Im of SH = sum conj(psi) [ -(1/2m) sum_i (D . PsiHat)_i + V psi ]
 *   out[3] = Sr = sum r^2 |psi|^2
 *   out[4], out[5] = Re, Im of SV = sum V |psi|^2
 * so that E = SH / S0, <r^2> = Sr / S0, <V> = SV / S0.  Planes are summed
 * in increasing k (the result does not depend on the thread count). */
void oracle_cobservables(int n, double a, double mass, const double* v_re, const double* v_im, const double* p_re,
                         const double* p_im, double out[6]) {
  double* plane = (double*)calloc((size_t)6 * (n + 1), sizeof(double));
  double half = 0.5 * (double)(n + 1);
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= n; ++k) {
    double s[6] = {0, 0, 0, 0, 0, 0};
    double z = ((double)k - half) * a;
    for (int j = 1; j <= n; ++j) {
      double y = ((double)j - half) * a;
      for (int i = 1; i <= n; ++i) {
        double x = ((double)i - half) * a;
        double complex psi = p_re[PIDX(n, i, j, k)] + I * p_im[PIDX(n, i, j, k)];
        double complex vv = v_re[DIDX(n, i, j, k)] + I * v_im[DIDX(n, i, j, k)];
        double complex lap = lap_at(n, a, p_re, i, j, k) + I * lap_at(n, a, p_im, i, j, k);
        double m2 = creal(psi) * creal(psi) + cimag(psi) * cimag(psi);
        double complex h = conj(psi) * (-lap / (2.0 * mass) + vv * psi);
        s[0] += m2;
        s[1] += creal(h);
        s[2] += cimag(h);
        s[3] += (x * x + y * y + z * z) * m2;
        s[4] += creal(vv) * m2;
        s[5] += cimag(vv) * m2;
      }
    }
    for (int q = 0; q < 6; ++q) plane[6 * k + q] = s[q];
  }
  for (int q = 0; q < 6; ++q) out[q] = 0.0;
  for (int k = 1; k <= n; ++k)
    for (int q = 0; q < 6; ++q) out[q] += plane[6 * k + q];
  free(plane);
}

/* Evolution with checks, as oracle_evolve (Secs. III-V) for a complex
 * field: at t = 0, check_every, ... and t = max_steps the sums, E and
 * E_b = E - v_inf, renormalisation by 1 / sqrt(S0 a^3), the symmetry mask on
 * both parts, and the convergence test |E_b - E_b,prev| <= tol (x |E_b| if
 * relative), |.| the complex modulus.  psi (re, im padded) is updated in
 * place; tmp_re, tmp_im are padded work fields.
 * rec[0..9]: Re E, Im E, Re E_b, S0 (before scaling), <r^2>, Re <V>,
 * Im <V>, |dE_b| (or -1), steps, converged.  Returns the number of checks,
 * or -1 on bad arguments. */
int64_t oracle_cevolve(int n, double a, double dtau, double mass, const double* v_re, const double* v_im,
                       double* p_re, double* p_im, double* tmp_re, double* tmp_im, int64_t max_steps,
                       int64_t check_every, double tol, int tol_relative, int mask, double v_inf, double* rec) {
  if (n < 1 || check_every < 1 || max_steps < 0) return -1;
  size_t bytes = sizeof(double) * (size_t)(n + 2) * (n + 2) * (n + 2);
  double complex prev = 0.0;
  int have_prev = 0, converged = 0;
  int64_t nchecks = 0, t = 0;
  double last_delta = -1.0;
  for (t = 0;; ++t) {
    if (t % check_every == 0 || t == max_steps) {
      double s[6];
      oracle_cobservables(n, a, mass, v_re, v_im, p_re, p_im, s);
      double complex e = (s[1] + I * s[2]) / s[0];
      double complex eb = e - v_inf;
      ++nchecks;
      rec[0] = creal(e);
      rec[1] = cimag(e);
      rec[2] = creal(eb);
      rec[3] = s[0];
      rec[4] = s[3] / s[0];
      rec[5] = s[4] / s[0];
      rec[6] = s[5] / s[0];
      double sc = 1.0 / sqrt(s[0] * a * a * a);
      for (size_t q = 0; q < bytes / sizeof(double); ++q) {
        p_re[q] *= sc;
        p_im[q] *= sc;
      }
      if (mask) {
        oracle_impose_parity(n, mask, p_re);
        oracle_impose_parity(n, mask, p_im);
      }
      if (have_prev) {
        last_delta = cabs(eb - prev);
        double thr = tol * (tol_relative ? cabs(eb) : 1.0);
        if (tol > 0 && last_delta <= thr) {
          converged = 1;
          break;
        }
      }
      prev = eb;
      have_prev = 1;
    }
    if (t == max_steps) break;
    oracle_cstep(n, a, dtau, mass, v_re, v_im, p_re, p_im, tmp_re, tmp_im);
    memcpy(p_re, tmp_re, bytes);
    memcpy(p_im, tmp_im, bytes);
  }
  rec[7] = last_delta;
  rec[8] = (double)t;
  rec[9] = (double)converged;
  return nchecks;
}
