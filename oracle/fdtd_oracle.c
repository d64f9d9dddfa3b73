/*
 * Plain FP64 CPU oracle for the imaginary-time FDTD solver of the 3-D
 * Schroedinger equation (Strickland & Yager-Elorriaga, "A Parallel Algorithm
 * for Solving the 3d Schroedinger Equation").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header or constant table with the
 * CUDA library; the two agree only through the paper's equations and through
 * the published SplitMix64 definition of the random initial condition.
 *
 * Storage follows the paper (Sec. V): every field psi is held on the padded
 * lattice of (N+2)^3 sites, index (i, j, k) with x = i fastest, and the
 * padding shell i, j, k in {0, N+1} holds the boundary value psi = 0
 * (Sec. III: "The boundary values of the wavefunction are set to zero").
 * The paper notes that other boundary conditions are easily implemented
 * (Sec. III); oracle_set_boundary(1) selects periodic ones, under which a
 * neighbour index 0 stands for N and N+1 for 1 (the shell is not read).
 * The potential V is passed densely on the N^3 interior sites, x fastest.
 * Interior site (i, j, k), 1 <= i, j, k <= N, sits at
 *     x = (i - (N+1)/2) a,   y = (j - (N+1)/2) a,   z = (k - (N+1)/2) a,
 * so the box spans L = N a and its centre is not a lattice site for even N.
 *
 * Floating point: compiled with -ffp-contract=off so that x86-64 and aarch64
 * hosts give identical results.  Sums over the lattice are taken per z-plane
 * and then over planes in increasing k, so the result does not depend on the
 * number of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PIDX(n, i, j, k) \
  ((((size_t)(k)) * (size_t)((n) + 2) + (size_t)(j)) * (size_t)((n) + 2) + (size_t)(i))
#define DIDX(n, i, j, k) \
  ((((size_t)(k) - 1) * (size_t)(n) + ((size_t)(j) - 1)) * (size_t)(n) + ((size_t)(i) - 1))

/* ------------------------------------------------------------------------ */
/* Random initial condition (Sec. III: "choosing a random 3d wavefunction as */
/* the initial condition ... Gaussian distributed random numbers with an     */
/* amplitude of one").                                                        */
/*                                                                            */
/* Generator: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  The state       */
/* advances by the odd constant gamma = 0x9E3779B97F4A7C15 and every output   */
/* is the state passed through the 64-bit finaliser with multipliers          */
/* 0xBF58476D1CE4E5B9, 0x94D049BB133111EB and shifts 30, 27, 31.  Output      */
/* number d (d = 0, 1, ...) of the stream seeded with s is therefore          */
/*     mix(s + (d + 1) * gamma)  (mod 2^64).                                  */
/* Lattice number `lat` draws from outputs d = lat * 2^42 + (draw index), and */
/* the interior site with dense index n = ((k-1) N + (j-1)) N + (i-1) uses    */
/* draw index n (uniform) or draws 2n and 2n+1 (Gaussian, Box-Muller).        */
/* ------------------------------------------------------------------------ */
static const uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t oracle_splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t oracle_splitmix64_output(uint64_t seed, uint64_t d) {
  return oracle_splitmix64_mix(seed + (d + 1) * SM64_GAMMA);
}

/* top 53 bits -> double in [0, 1) */
static double u01_from_bits(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

double oracle_draw_uniform(uint64_t seed, uint64_t lat, uint64_t n) {
  uint64_t d = (lat << 42) + n;
  return 2.0 * u01_from_bits(oracle_splitmix64_output(seed, d)) - 1.0;
}

double oracle_draw_gaussian(uint64_t seed, uint64_t lat, uint64_t n) {
  uint64_t d = (lat << 42) + 2 * n;
  double u1 = u01_from_bits(oracle_splitmix64_output(seed, d));
  double u2 = u01_from_bits(oracle_splitmix64_output(seed, d + 1));
  /* Box & Muller (1958): sqrt(-2 ln U1) cos(2 pi U2) with U1 in (0, 1] */
  double r = sqrt(-2.0 * log(1.0 - u1));
  return r * cos(2.0 * M_PI * u2);
}

/* dist: 0 = uniform in [-1, 1), 1 = standard Gaussian.  Fills the interior
 * of the padded field and zeroes the padding. */
void oracle_init_random(int n, uint64_t seed, uint64_t lat, int dist, double* psi) {
  memset(psi, 0, sizeof(double) * (size_t)(n + 2) * (n + 2) * (n + 2));
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        uint64_t lin = DIDX(n, i, j, k);
        psi[PIDX(n, i, j, k)] =
            dist == 1 ? oracle_draw_gaussian(seed, lat, lin) : oracle_draw_uniform(seed, lat, lin);
      }
}

/* ------------------------------------------------------------------------ */
/* Symmetrisation S_i and antisymmetrisation A_i about the plane x_i = 0      */
/* (Sec. IV): copy one half of the lattice onto the other, flipping the sign  */
/* for A_i.  The mirror of index m is N+1-m (x -> -x).  The source half is    */
/* the one with the lower index; for odd N the central plane is its own       */
/* mirror and A_i sets it to zero.                                             */
/* mask: two bits per axis (x: bits 0-1, y: 2-3, z: 4-5); 0 none, 1 S, 2 A.    */
/* Axes are applied one after another in the order x, y, z.                    */
/* Returns 0, or -1 for an invalid mask.                                       */
/* ------------------------------------------------------------------------ */
int oracle_impose_parity(int n, int mask, double* psi) {
  if (mask < 0 || mask >= 64) return -1;
  for (int axis = 0; axis < 3; ++axis) {
    int mode = (mask >> (2 * axis)) & 3;
    if (mode == 3) return -1;
  }
  for (int axis = 0; axis < 3; ++axis) {
    int mode = (mask >> (2 * axis)) & 3;
    if (mode == 0) continue;
    double sgn = (mode == 2) ? -1.0 : 1.0;
    for (int k = 1; k <= n; ++k)
      for (int j = 1; j <= n; ++j)
        for (int i = 1; i <= n; ++i) {
          int m = axis == 0 ? i : (axis == 1 ? j : k);
          int mm = n + 1 - m;
          if (m > mm) {
            int si = axis == 0 ? mm : i, sj = axis == 1 ? mm : j, sk = axis == 2 ? mm : k;
            psi[PIDX(n, i, j, k)] = sgn * psi[PIDX(n, si, sj, sk)];
          } else if (m == mm && mode == 2) {
            psi[PIDX(n, i, j, k)] = 0.0;
          }
        }
  }
  return 0;
}

/* Transpose of the linear map applied by oracle_impose_parity (used by the
 * adjoint).  The forward map is P = Pz Py Px; its transpose is applied here
 * as Px^T Py^T Pz^T, i.e. axes in the order z, y, x.  For one axis the
 * forward map sends value(lower m) to itself and to sgn * value(mirror);
 * its transpose adds sgn * lambda(upper) onto lambda(lower) and zeroes the
 * upper half (and the central plane for A). */
int oracle_impose_parity_adjoint(int n, int mask, double* lam) {
  if (mask < 0 || mask >= 64) return -1;
  for (int axis = 0; axis < 3; ++axis)
    if (((mask >> (2 * axis)) & 3) == 3) return -1;
  for (int axis = 2; axis >= 0; --axis) {
    int mode = (mask >> (2 * axis)) & 3;
    if (mode == 0) continue;
    double sgn = (mode == 2) ? -1.0 : 1.0;
    for (int k = 1; k <= n; ++k)
      for (int j = 1; j <= n; ++j)
        for (int i = 1; i <= n; ++i) {
          int m = axis == 0 ? i : (axis == 1 ? j : k);
          int mm = n + 1 - m;
          if (m > mm) {
            int si = axis == 0 ? mm : i, sj = axis == 1 ? mm : j, sk = axis == 2 ? mm : k;
            lam[PIDX(n, si, sj, sk)] += sgn * lam[PIDX(n, i, j, k)];
            lam[PIDX(n, i, j, k)] = 0.0;
          } else if (m == mm && mode == 2) {
            lam[PIDX(n, i, j, k)] = 0.0;
          }
        }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Update equation (Sec. III, Eq. updateeq):                                  */
/*   Psi(tau + dtau) = A Psi + (B dtau / 2m) sum_{i=1..3} (D . PsiHat)_i       */
/* with D = [1, -2, 1] / a^2 along each axis and                               */
/*   A = (1 - dtau V / 2) / (1 + dtau V / 2),   B = 1 / (1 + dtau V / 2).      */
/* psi_in and psi_out are distinct padded fields (Jacobi update); the         */
/* padding of psi_out is set to zero.                                          */
/* ------------------------------------------------------------------------ */
/* Boundary: 0 = the zero shell of Sec. III, 1 = periodic (index 0 is N,
 * index N+1 is 1 along every axis). */
static int g_periodic = 0;
void oracle_set_boundary(int periodic) { g_periodic = periodic ? 1 : 0; }

/* neighbour index along one axis: i in [0, N+1] */
static int nb(int n, int i) {
  if (!g_periodic) return i;
  return i < 1 ? i + n : (i > n ? i - n : i);
}

static double second_differences(int n, double a, const double* p, int i, int j, int k) {
  double c = p[PIDX(n, i, j, k)];
  double dxx = (p[PIDX(n, nb(n, i - 1), j, k)] - 2.0 * c + p[PIDX(n, nb(n, i + 1), j, k)]) / (a * a);
  double dyy = (p[PIDX(n, i, nb(n, j - 1), k)] - 2.0 * c + p[PIDX(n, i, nb(n, j + 1), k)]) / (a * a);
  double dzz = (p[PIDX(n, i, j, nb(n, k - 1))] - 2.0 * c + p[PIDX(n, i, j, nb(n, k + 1))]) / (a * a);
  return dxx + dyy + dzz;
}

void oracle_step(int n, double a, double dtau, double mass, const double* v, const double* psi_in,
                 double* psi_out) {
  memset(psi_out, 0, sizeof(double) * (size_t)(n + 2) * (n + 2) * (n + 2));
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        double vv = v[DIDX(n, i, j, k)];
        double A = (1.0 - 0.5 * dtau * vv) / (1.0 + 0.5 * dtau * vv);
        double B = 1.0 / (1.0 + 0.5 * dtau * vv);
        double lap = second_differences(n, a, psi_in, i, j, k);
        psi_out[PIDX(n, i, j, k)] = A * psi_in[PIDX(n, i, j, k)] + B * dtau / (2.0 * mass) * lap;
      }
}

/* ------------------------------------------------------------------------ */
/* Lattice sums (Sec. III, Eq. energysum, with the sign of the Hamiltonian    */
/* H = -nabla^2 / 2m + V of Sec. II):                                          */
/*   out[0] = S0 = sum psi^2                                                   */
/*   out[1] = SH = sum psi [ -(1/2m) sum_i (D . PsiHat)_i + V psi ]            */
/*   out[2] = Sr = sum r^2 psi^2,   r measured from the lattice centre         */
/*   out[3] = SV = sum V psi^2                                                 */
/* so that E = SH / S0 and <r^2> = Sr / S0.                                    */
/* ------------------------------------------------------------------------ */
void oracle_observables(int n, double a, double mass, const double* v, const double* psi,
                        double out[4]) {
  double* plane = (double*)calloc((size_t)4 * (n + 1), sizeof(double));
  double half = 0.5 * (double)(n + 1);
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= n; ++k) {
    double s0 = 0, sh = 0, sr = 0, sv = 0;
    double z = ((double)k - half) * a;
    for (int j = 1; j <= n; ++j) {
      double y = ((double)j - half) * a;
      for (int i = 1; i <= n; ++i) {
        double x = ((double)i - half) * a;
        double c = psi[PIDX(n, i, j, k)];
        double vv = v[DIDX(n, i, j, k)];
        double lap = second_differences(n, a, psi, i, j, k);
        s0 += c * c;
        sh += c * (-lap / (2.0 * mass) + vv * c);
        sr += (x * x + y * y + z * z) * c * c;
        sv += vv * c * c;
      }
    }
    plane[4 * k + 0] = s0;
    plane[4 * k + 1] = sh;
    plane[4 * k + 2] = sr;
    plane[4 * k + 3] = sv;
  }
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (int k = 1; k <= n; ++k)
    for (int q = 0; q < 4; ++q) out[q] += plane[4 * k + q];
  free(plane);
}

/* psi <- s psi on the interior (renormalisation, Sec. III). */
void oracle_scale(int n, double s, double* psi) {
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) psi[PIDX(n, i, j, k)] *= s;
}

/* ------------------------------------------------------------------------ */
/* Evolution with periodic checks (Sec. III renormalisation; Sec. IV          */
/* periodic re-imposition of the symmetry; Sec. V convergence test on the     */
/* binding energy every `check_every` steps).                                  */
/*                                                                            */
/* At every step index t that is a multiple of check_every, and at t =        */
/* max_steps, before the step from t:                                          */
/*   1. S0, SH, Sr, SV on psi_t;  E = SH/S0, E_b = E - v_inf (Eq.              */
/*      bindingenergy with constant V_inf), <r^2> = Sr/S0;                     */
/*   2. psi_t <- psi_t / sqrt(S0 a^3), so that sum psi^2 a^3 = 1;              */
/*   3. the symmetry mask is imposed again (if non-zero);                      */
/*   4. converged if a previous check exists and                               */
/*      |E_b - E_b,prev| <= tol * (tol_relative ? |E_b| : 1).                  */
/* tol <= 0 never converges (fixed number of steps).                          */
/*                                                                            */
/* psi (padded) is updated in place; tmp is a padded work field.              */
/* rec[0..7] receives, from the last check: E, E_b, S0 (before scaling),      */
/* <r^2>, <V>, |E_b - E_b,prev| (or -1), steps, converged.                    */
/* hist (optional, 4 doubles per check: t, E, <r^2>, S0) up to hist_cap rows. */
/* Returns the number of checks, or -1 on bad arguments.                      */
/* ------------------------------------------------------------------------ */
int64_t oracle_evolve(int n, double a, double dtau, double mass, const double* v, double* psi,
                      double* tmp, int64_t max_steps, int64_t check_every, double tol,
                      int tol_relative, int mask, double v_inf, double* rec, double* hist,
                      int64_t hist_cap) {
  if (n < 1 || check_every < 1 || max_steps < 0) return -1;
  size_t bytes = sizeof(double) * (size_t)(n + 2) * (n + 2) * (n + 2);
  double prev_eb = 0.0;
  int have_prev = 0, converged = 0;
  int64_t nchecks = 0, t = 0;
  double last_delta = -1.0;
  for (t = 0;; ++t) {
    if (t % check_every == 0 || t == max_steps) {
      double s[4];
      oracle_observables(n, a, mass, v, psi, s);
      double e = s[1] / s[0];
      double eb = e - v_inf;
      double r2 = s[2] / s[0];
      if (hist && nchecks < hist_cap) {
        hist[4 * nchecks + 0] = (double)t;
        hist[4 * nchecks + 1] = e;
        hist[4 * nchecks + 2] = r2;
        hist[4 * nchecks + 3] = s[0];
      }
      ++nchecks;
      rec[0] = e;
      rec[1] = eb;
      rec[2] = s[0];
      rec[3] = r2;
      rec[4] = s[3] / s[0];
      oracle_scale(n, 1.0 / sqrt(s[0] * a * a * a), psi);
      if (mask) oracle_impose_parity(n, mask, psi);
      if (have_prev) {
        last_delta = fabs(eb - prev_eb);
        double thr = tol * (tol_relative ? fabs(eb) : 1.0);
        if (tol > 0 && last_delta <= thr) {
          converged = 1;
          break;
        }
      }
      prev_eb = eb;
      have_prev = 1;
    }
    if (t == max_steps) break;
    oracle_step(n, a, dtau, mass, v, psi, tmp);
    memcpy(psi, tmp, bytes);
  }
  rec[5] = last_delta;
  rec[6] = (double)t;
  rec[7] = (double)converged;
  return nchecks;
}

/* ------------------------------------------------------------------------ */
/* Multi-resolution transfer (Sec. VI; Sec. VII.G "sampling/spreading out"):  */
/* trilinear interpolation from an Nc^3 lattice to an Nf^3 = (2 Nc)^3 lattice */
/* of the same box length L.                                                   */
/* Fine site j sits at x = (j - (2Nc+1)/2) a/2 with a the coarse spacing; in  */
/* coarse index units that is xi = x/a + (Nc+1)/2 = j/2 + 1/4.  The value is   */
/* interpolated linearly along each axis between coarse indices floor(xi) and */
/* floor(xi)+1, where the coarse padding (index 0 and Nc+1) holds zero, or,  */
/* with periodic boundaries, index 0 stands for Nc and Nc+1 for 1.             */
/* ------------------------------------------------------------------------ */
void oracle_upsample(int nc, const double* psi_c, double* psi_f) {
  int nf = 2 * nc;
  memset(psi_f, 0, sizeof(double) * (size_t)(nf + 2) * (nf + 2) * (nf + 2));
  for (int k = 1; k <= nf; ++k)
    for (int j = 1; j <= nf; ++j)
      for (int i = 1; i <= nf; ++i) {
        double xi[3] = {0.5 * i + 0.25, 0.5 * j + 0.25, 0.5 * k + 0.25};
        int lo[3];
        double w1[3];
        for (int d = 0; d < 3; ++d) {
          lo[d] = (int)floor(xi[d]);
          w1[d] = xi[d] - (double)lo[d];
        }
        double acc = 0.0;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              double w = (dx ? w1[0] : 1.0 - w1[0]) * (dy ? w1[1] : 1.0 - w1[1]) *
                         (dz ? w1[2] : 1.0 - w1[2]);
              acc += w * psi_c[PIDX(nc, nb(nc, lo[0] + dx), nb(nc, lo[1] + dy), nb(nc, lo[2] + dz))];
            }
        psi_f[PIDX(nf, i, j, k)] = acc;
      }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of one update step.  The update is linear in Psi:                   */
/*   Psi' = M Psi,   M = diag(A) + (dtau / 2m) diag(B) Lap,                    */
/* with Lap the sum of second differences (symmetric for zero and for        */
/* periodic boundaries), so                                                    */
/*   M^T lambda = A lambda + (dtau / 2m) Lap (B lambda).                       */
/* ------------------------------------------------------------------------ */
void oracle_adjoint_step(int n, double a, double dtau, double mass, const double* v,
                         const double* lam_in, double* lam_out) {
  size_t np = (size_t)(n + 2) * (n + 2) * (n + 2);
  double* u = (double*)calloc(np, sizeof(double));
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        double vv = v[DIDX(n, i, j, k)];
        double B = 1.0 / (1.0 + 0.5 * dtau * vv);
        u[PIDX(n, i, j, k)] = B * lam_in[PIDX(n, i, j, k)];
      }
  memset(lam_out, 0, sizeof(double) * np);
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        double vv = v[DIDX(n, i, j, k)];
        double A = (1.0 - 0.5 * dtau * vv) / (1.0 + 0.5 * dtau * vv);
        double lap = second_differences(n, a, u, i, j, k);
        lam_out[PIDX(n, i, j, k)] = A * lam_in[PIDX(n, i, j, k)] + dtau / (2.0 * mass) * lap;
      }
  free(u);
}

/* Derivative of one update step with respect to the potential at each site:
 * with h = dtau V / 2,  dA/dV = -dtau / (1+h)^2,  dB/dV = -(dtau/2) / (1+h)^2,
 * so  g_V(s) += lambda'(s) [ dA/dV Psi(s) + dB/dV (dtau / 2m) Lap Psi(s) ].
 * gv is dense N^3. */
void oracle_grad_v_accum(int n, double a, double dtau, double mass, const double* v,
                         const double* psi, const double* lam_next, double* gv) {
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        double vv = v[DIDX(n, i, j, k)];
        double h = 0.5 * dtau * vv;
        double dA = -dtau / ((1.0 + h) * (1.0 + h));
        double dB = -0.5 * dtau / ((1.0 + h) * (1.0 + h));
        double lap = second_differences(n, a, psi, i, j, k);
        gv[DIDX(n, i, j, k)] +=
            lam_next[PIDX(n, i, j, k)] * (dA * psi[PIDX(n, i, j, k)] + dB * dtau / (2.0 * mass) * lap);
      }
}

/* ------------------------------------------------------------------------ */
/* Gradient of  loss = wE * E[psi_T] + wr * <r^2>[psi_T]  with respect to V,  */
/* through T unrolled steps started from the fixed padded field psi0.         */
/* The forward pass is oracle_evolve with tol = 0: a check (renormalisation   */
/* and, if mask != 0, the symmetry projection) at every multiple of           */
/* check_every below T, and the loss is taken on psi_T as the step produced   */
/* it (the observables that oracle_evolve reports at its final check).        */
/* The renormalisation factors are held constant: E and <r^2> are homogeneous */
/* of degree 0 in psi, so their derivative along psi itself vanishes and the  */
/* factors contribute nothing.  At T:                                         */
/*   dE/dpsi = 2 (H psi - E psi) / S0,  d<r^2>/dpsi = 2 (r^2 - <r^2>) psi / S0 */
/*   direct dE/dV(s) = psi(s)^2 / S0.                                          */
/* Every intermediate field is stored (no checkpointing).                     */
/* gv (dense N^3) is overwritten; obs[0..3] = E, <r^2>, S0, loss at T.        */
/* Returns 0, or -1 on bad arguments or if the trajectory cannot be held.     */
/* ------------------------------------------------------------------------ */
int oracle_backward(int n, double a, double dtau, double mass, const double* v,
                    const double* psi0, int64_t T, int64_t check_every, int mask, double w_e,
                    double w_r, double* gv, double* obs) {
  if (n < 1 || T < 0 || check_every < 1) return -1;
  size_t np = (size_t)(n + 2) * (n + 2) * (n + 2);
  size_t nd = (size_t)n * n * n;
  double* traj = (double*)malloc(sizeof(double) * np * (size_t)(T + 1));
  double* scale = (double*)calloc((size_t)(T + 1), sizeof(double));
  double* lam = (double*)calloc(np, sizeof(double));
  double* lam2 = (double*)calloc(np, sizeof(double));
  if (!traj || !scale || !lam || !lam2) {
    free(traj); free(scale); free(lam); free(lam2);
    return -1;
  }
  /* forward; traj[t] (t < T) holds psi_t after its check, traj[T] the raw psi_T */
  memcpy(traj, psi0, sizeof(double) * np);
  for (int64_t t = 0; t < T; ++t) {
    double* cur = traj + np * (size_t)t;
    if (t % check_every == 0) {
      double s[4];
      oracle_observables(n, a, mass, v, cur, s);
      scale[t] = 1.0 / sqrt(s[0] * a * a * a);
      oracle_scale(n, scale[t], cur);
      if (mask) oracle_impose_parity(n, mask, cur);
    }
    oracle_step(n, a, dtau, mass, v, cur, cur + np);
  }
  double* psiT = traj + np * (size_t)T;
  double f[4];
  oracle_observables(n, a, mass, v, psiT, f);
  double e = f[1] / f[0], r2 = f[2] / f[0];
  obs[0] = e;
  obs[1] = r2;
  obs[2] = f[0];
  obs[3] = w_e * e + w_r * r2;
  double half = 0.5 * (double)(n + 1);
  memset(gv, 0, sizeof(double) * nd);
  for (int k = 1; k <= n; ++k)
    for (int j = 1; j <= n; ++j)
      for (int i = 1; i <= n; ++i) {
        double x = ((double)i - half) * a, y = ((double)j - half) * a, z = ((double)k - half) * a;
        double c = psiT[PIDX(n, i, j, k)];
        double vv = v[DIDX(n, i, j, k)];
        double hpsi = -second_differences(n, a, psiT, i, j, k) / (2.0 * mass) + vv * c;
        lam[PIDX(n, i, j, k)] = w_e * 2.0 * (hpsi - e * c) / f[0] +
                                w_r * 2.0 * ((x * x + y * y + z * z) - r2) * c / f[0];
        gv[DIDX(n, i, j, k)] = w_e * c * c / f[0];
      }
  /* walk back: psi_t = M psi_{t-1}, where psi_{t-1} is taken after its check */
  for (int64_t t = T; t >= 1; --t) {
    double* prev = traj + np * (size_t)(t - 1);
    oracle_grad_v_accum(n, a, dtau, mass, v, prev, lam, gv);
    oracle_adjoint_step(n, a, dtau, mass, v, lam, lam2);
    memcpy(lam, lam2, sizeof(double) * np);
    if ((t - 1) % check_every == 0) {
      /* the check applied psi <- P(s psi); its transpose is lam <- s P^T lam */
      if (mask) oracle_impose_parity_adjoint(n, mask, lam);
      oracle_scale(n, scale[t - 1], lam);
    }
  }
  free(traj); free(scale); free(lam); free(lam2);
  return 0;
}
