/*
 * FP64 CPU oracle for the far-field, spectrally resolved Lienard-Wiechert
 * radiation sum over macro-particles with the general form-factor formalism
 * of Pausch et al., "Quantitatively consistent computation of coherent and
 * incoherent radiation in particle-in-cell codes - a general form factor
 * formalism for macro-particles" (NIM A, 2018).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * definition that the CUDA library is checked against. Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it; the library
 * never calls it, and it shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes, for every accumulate call (time t, step dt, particle
 * arrays), every requested bin (direction n, frequency omega) and every
 * particle k, in that loop order (calls -> particles), in FP64 with
 * Neumaier-compensated sums:
 *
 *   A_k   = n x [(n - beta_k) x betadot_k] / (1 - beta_k . n)^2      (Eq. 1)
 *   phi_k = omega (t - n . r_k / c)                                  (Eq. 1)
 *   U += w_k dt A_k e^{i phi_k}              coherent accumulator
 *   V += sqrt(w_k) dt A_k e^{i phi_k}        incoherent accumulator
 *   P += F_k(omega) dt A_k e^{i phi_k}       the paper's literal in-situ sum
 *          with F_k = sqrt(w_k + (w_k^2 - w_k) f(omega)^2)     (Eq. 13 with Eq. 12)
 *
 * and at readout, with K0 = q_e^2 / (16 pi^3 eps0 c)                 (Eq. 1, 2)
 *
 *   I_coh   = K0 f^2 |U|^2
 *   I_inc   = K0 (1 - f^2) |V|^2
 *   I_tot   = I_coh + I_inc
 *   I_paper = K0 |P|^2
 *
 * f(omega) is the amplitude form factor of Table 1 normalised to f(0) = 1.
 * Readings of the paper taken here (where it is garbled or silent):
 *  - the prefactor of the discretised sum (Eq. 13, Sec. 3.3) is read as
 *    squared, (dt q_e)^2 / (16 pi^3 eps0 c), as Eq. 1 and Eq. 2 force when the
 *    time integral inside |.|^2 becomes a sum; dt is folded into the
 *    accumulated weight, so the readout uses K0;
 *  - the dimensionful prefactors Delta/c and sigma^2/c^2 of Table 1 are
 *    dropped, so that rho integrates to one and f(0) = 1 (needed for the
 *    point-charge limit of Sec. 3.2 to give N^2);
 *  - sinc(x) = sin(x)/x, argument omega Delta / (2c) (Table 1);
 *  - the form factor depends on omega only (Table 1 as printed, which takes
 *    n along one axis without loss of generality, Sec. 3.2); with the 3-D flag
 *    the box shapes are axis-aligned products rho(x) rho(y) rho(z) and f
 *    depends on the direction too (oracle_form_factor_dir);
 *  - "incoherent" is weighted by w (1 - f^2), "coherent" by w^2 f^2: per
 *    macro-particle the same total as Eq. 12, N + (N^2 - N) f^2, with the
 *    inter-particle incoherence kept out of the incoherent part at low omega.
 *
 * Parity pins: the tests pin every function here to closed forms, limits
 * and brute force (circular-orbit harmonics, the integration-by-parts
 * identity of the amplitude, N^2 / N scaling, form-factor limits, Monte-Carlo
 * electrons drawn from the macro-particle shape, quadrature of Table 1).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define ORC_C 299792458.0           /* speed of light, m/s (exact) */
#define ORC_QE 1.602176634e-19      /* elementary charge, C (exact) */
#define ORC_EPS0 8.8541878128e-12   /* vacuum permittivity, F/m (CODATA 2018) */
#define ORC_PI 3.14159265358979323846

enum { ORC_FF_POINT = 0, ORC_FF_CIC = 1, ORC_FF_TSC = 2, ORC_FF_QSC = 3, ORC_FF_GAUSS = 4 };

/* Number of doubles per bin in the accumulator arrays: U, V, P, each a
 * complex 3-vector stored as (x.re, x.im, y.re, y.im, z.re, z.im). */
#define ORC_PER_BIN 18

/* K0 = q_e^2 / (16 pi^3 eps0 c): the prefactor of Eq. 1 for one electron. */
double oracle_k0(void) {
  return ORC_QE * ORC_QE / (16.0 * ORC_PI * ORC_PI * ORC_PI * ORC_EPS0 * ORC_C);
}

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* Amplitude form factor f(omega), Table 1 with f(0) = 1:
 *   point: 1; CIC: sinc(x); TSC: sinc(x)^2; QSC: sinc(x)^3, x = omega Delta/(2c);
 *   Gauss: exp(-omega^2 sigma^2 / (2 c^2)), so f^2 = exp(-omega^2 sigma^2 / c^2).
 * width is Delta for CIC/TSC/QSC and sigma for Gauss, in metres.
 * Returns NaN for an unknown kind. */
double oracle_form_factor(int kind, double width, double omega) {
  const double x = omega * width / (2.0 * ORC_C);
  switch (kind) {
    case ORC_FF_POINT: return 1.0;
    case ORC_FF_CIC: return sinc(x);
    case ORC_FF_TSC: return sinc(x) * sinc(x);
    case ORC_FF_QSC: return sinc(x) * sinc(x) * sinc(x);
    case ORC_FF_GAUSS: {
      const double s = omega * width / ORC_C;
      return exp(-0.5 * s * s);
    }
    default: return NAN;
  }
}

/* Bit of ff_flags: box shapes (CIC/TSC/QSC) taken as the 3-D product
 * rho(x) rho(y) rho(z) of the 1-D shape along the coordinate axes (Sec. 3.1, 3.2:
 * the charge distribution factorises per axis), so that for a direction n the
 * phase factor of the offsets is the product over axes,
 *   f(n, omega) = prod_d f_1(omega n_d),   f_1 as Table 1 with omega n_d.
 * Without the bit (and always for the isotropic Gaussian) f depends on omega
 * only: Table 1 as printed, n along one axis. */
#define ORC_FF_3D 1

double oracle_form_factor_dir(int kind, int flags, double width, double omega, const double n[3]) {
  if (!(flags & ORC_FF_3D) || kind == ORC_FF_POINT || kind == ORC_FF_GAUSS)
    return oracle_form_factor(kind, width, omega);
  double f = 1.0;
  for (int d = 0; d < 3; ++d) f *= oracle_form_factor(kind, width, omega * n[d]);
  return f;
}

/* Neumaier's compensated summation: s + c carries the running sum. */
static void nadd(double* s, double* c, double x) {
  const double t = *s + x;
  if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
  else *c += (x - t) + *s;
  *s = t;
}

static void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* A = n x [(n - beta) x betadot] / (1 - beta . n)^2, the radiation amplitude
 * of Eq. 1, written out directly. */
void oracle_amplitude(const double n[3], const double beta[3], const double bdot[3], double A[3]) {
  const double u[3] = {n[0] - beta[0], n[1] - beta[1], n[2] - beta[2]};
  double c[3], m[3];
  cross(u, bdot, c);
  cross(n, c, m);
  const double d = 1.0 - (beta[0] * n[0] + beta[1] * n[1] + beta[2] * n[2]);
  const double d2 = d * d;
  A[0] = m[0] / d2;
  A[1] = m[1] / d2;
  A[2] = m[2] / d2;
}

/* One accumulate call: adds the contribution of N particles at time t with
 * step dt to every bin b = (bin_omega[b], bin_dir[3b..3b+2]).
 *   r, beta, beta_dot: SoA [3][N] (x block, y block, z block), metres / 1 / 1/s
 *   w: [N] electrons per macro-particle (> 0)
 *   ff_kind, ff_flags, ff_width: the shape used for the paper's literal sum P
 *   acc, comp: [n_bins][18] running sums and their Neumaier compensation
 * Layout per bin: U (6 doubles), V (6), P (6), each (x,y,z) x (re,im).
 * Bins are independent and processed in parallel; within a bin the particle
 * order is fixed, so the result does not depend on the thread count. */
void oracle_accumulate(int64_t n_bins, const double* bin_omega, const double* bin_dir,
                       int64_t N, const double* r, const double* beta, const double* beta_dot,
                       const double* w, double t, double dt, int ff_kind, int ff_flags,
                       double ff_width, double* acc, double* comp) {
  int64_t b;
#pragma omp parallel for schedule(dynamic, 1)
  for (b = 0; b < n_bins; ++b) {
    const double omega = bin_omega[b];
    const double* n = bin_dir + 3 * b;
    const double f = oracle_form_factor_dir(ff_kind, ff_flags, ff_width, omega, n);
    double* s = acc + ORC_PER_BIN * b;
    double* c = comp + ORC_PER_BIN * b;
    for (int64_t k = 0; k < N; ++k) {
      const double rk[3] = {r[k], r[N + k], r[2 * N + k]};
      const double bk[3] = {beta[k], beta[N + k], beta[2 * N + k]};
      const double dk[3] = {beta_dot[k], beta_dot[N + k], beta_dot[2 * N + k]};
      double A[3];
      oracle_amplitude(n, bk, dk, A);
      const double phi = omega * (t - (n[0] * rk[0] + n[1] * rk[1] + n[2] * rk[2]) / ORC_C);
      const double cph = cos(phi), sph = sin(phi);
      const double wk = w[k];
      const double weight[3] = {wk * dt, sqrt(wk) * dt, sqrt(wk + (wk * wk - wk) * f * f) * dt};
      for (int a = 0; a < 3; ++a) {
        for (int d = 0; d < 3; ++d) {
          nadd(&s[6 * a + 2 * d], &c[6 * a + 2 * d], weight[a] * A[d] * cph);
          nadd(&s[6 * a + 2 * d + 1], &c[6 * a + 2 * d + 1], weight[a] * A[d] * sph);
        }
      }
    }
  }
}

/* Test-only: per-particle time integrals a_k = sum_t dt A_k e^{i phi_k}
 * (no weight), so that the exact expected incoherent part
 * K0 (1 - f^2) sum_k w_k |a_k|^2 can be formed. a: [N][n_bins][6],
 * accumulated in plain FP64 (tiny cases only). */
void oracle_accumulate_particles(int64_t n_bins, const double* bin_omega, const double* bin_dir,
                                 int64_t N, const double* r, const double* beta,
                                 const double* beta_dot, double t, double dt, double* a) {
  int64_t b;
#pragma omp parallel for schedule(dynamic, 1)
  for (b = 0; b < n_bins; ++b) {
    const double omega = bin_omega[b];
    const double* n = bin_dir + 3 * b;
    for (int64_t k = 0; k < N; ++k) {
      const double rk[3] = {r[k], r[N + k], r[2 * N + k]};
      const double bk[3] = {beta[k], beta[N + k], beta[2 * N + k]};
      const double dk[3] = {beta_dot[k], beta_dot[N + k], beta_dot[2 * N + k]};
      double A[3];
      oracle_amplitude(n, bk, dk, A);
      const double phi = omega * (t - (n[0] * rk[0] + n[1] * rk[1] + n[2] * rk[2]) / ORC_C);
      double* ak = a + 6 * (k * n_bins + b);
      for (int d = 0; d < 3; ++d) {
        ak[2 * d] += dt * A[d] * cos(phi);
        ak[2 * d + 1] += dt * A[d] * sin(phi);
      }
    }
  }
}

/* Readout of the spectra d^2I/dOmega domega for every bin (J s / sr per rad/s
 * in SI): coherent K0 f^2 |U|^2, incoherent K0 (1 - f^2) |V|^2, total their
 * sum, and the paper's literal K0 |P|^2. f is taken for (ff_kind, ff_flags,
 * ff_width) and the bin's direction; any output pointer may be NULL. */
void oracle_readout(int64_t n_bins, const double* bin_omega, const double* bin_dir,
                    const double* acc, const double* comp, int ff_kind, int ff_flags,
                    double ff_width, double* coh, double* inc, double* tot, double* paper) {
  const double k0 = oracle_k0();
  for (int64_t b = 0; b < n_bins; ++b) {
    const double f =
        oracle_form_factor_dir(ff_kind, ff_flags, ff_width, bin_omega[b], bin_dir + 3 * b);
    double m2[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < 6; ++j) {
        const double v = acc[ORC_PER_BIN * b + 6 * a + j] + comp[ORC_PER_BIN * b + 6 * a + j];
        m2[a] += v * v;
      }
    const double ic = k0 * f * f * m2[0];
    const double ii = k0 * (1.0 - f * f) * m2[1];
    if (coh) coh[b] = ic;
    if (inc) inc[b] = ii;
    if (tot) tot[b] = ic + ii;
    if (paper) paper[b] = k0 * m2[2];
  }
}

/* Number of threads the parallel loops above use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
