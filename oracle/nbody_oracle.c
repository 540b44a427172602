/*
 * nbody_oracle.c -- plain FP64 CPU oracle of the differentiable direct-sum
 * N-body method of "Differentiable N-body code for Galactic Dynamics
 * Odisseo" (arXiv 2511.22468).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is built into its own shared library
 * (liborc) and is called only by the test-suite, by the package smoke check
 * and by the CPU-baseline leg of the benchmark.  The product (CUDA) path
 * neither links nor calls it, and it shares no source with that path.
 *
 * What it computes, each routine the textbook definition written out with
 * plain loops in FP64 (OpenMP only splits independent output rows):
 *   - softened direct pairwise gravity (paper Sec. 1, "N-body codes": exact
 *     pairwise forces with softening, no tree or multipole), Plummer
 *     softening a_i = -G sum_{j!=i} m_j (x_i-x_j) (|x_i-x_j|^2+eps^2)^-3/2;
 *   - the NFW halo, Miyamoto-Nagai disk and power-law bulge of
 *     MWPotential2014 (Sec. 2.2.1):
 *     potential, acceleration and the Jacobian of the acceleration;
 *   - the second-order Velocity-Verlet (kick-drift-kick) integrator with a
 *     fixed number of steps (Sec. 2.2.1);
 *   - its discrete adjoint: reverse-mode gradients of a function of the
 *     final state with respect to the initial state, the time step, the
 *     particle masses and the two potential masses (Sec. 2, end-to-end
 *     differentiability; Sec. 2.2.1 / Fig. 2 parameter vector).
 * The adjoint takes the forward sub-steps (kick, drift, kick) one at a time
 * in reverse order; it does not merge the two half kicks that meet at a
 * step boundary, and it builds every pair Jacobian block explicitly.
 *
 * Harmonic test force: ext bit 2 adds a = -omega2 * x.  It is not part of
 * the method; it gives the integrator and its adjoint a closed form.
 *
 * Layout: positions, velocities, accelerations are AoS, x[3*i + d].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NFW 1u
#define ORC_MN 2u
#define ORC_HARM 4u
#define ORC_BULGE 8u

typedef struct orc_params {
  double G;      /* gravitational constant */
  double eps;    /* Plummer softening length, >= 0 */
  int32_t pair;  /* 1: include the softened pair sum */
  uint32_t ext;  /* ORC_NFW | ORC_MN | ORC_HARM */
  double nfw_M;  /* NFW scale mass 4 pi rho_0 r_s^3 */
  double nfw_rs; /* NFW scale radius */
  double mn_M;   /* Miyamoto-Nagai disk mass */
  double mn_a;   /* MN scale length */
  double mn_b;   /* MN scale height */
  double omega2; /* harmonic test force */
  double bulge_M;     /* bulge total mass */
  double bulge_alpha; /* bulge inner power-law slope, 0 <= alpha < 3 */
  double bulge_rc;    /* bulge cut-off radius */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Pair gravity                                                              */
/* ------------------------------------------------------------------------ */

/* a_i for i = rows[r] (or r when rows == NULL), r < nrows; sum over j != i in
 * increasing j.  out[3*r + d]. */
void orc_pair_accel(int64_t n, const double *x, const double *m, double G,
                    double eps, const int64_t *rows, int64_t nrows,
                    double *out) {
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows ? rows[r] : r;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dx = x[3 * i + 0] - x[3 * j + 0];
      const double dy = x[3 * i + 1] - x[3 * j + 1];
      const double dz = x[3 * i + 2] - x[3 * j + 2];
      const double s2 = dx * dx + dy * dy + dz * dz + e2;
      const double s3 = s2 * sqrt(s2);
      const double f = G * m[j] / s3;
      ax -= f * dx;
      ay -= f * dy;
      az -= f * dz;
    }
    out[3 * r + 0] = ax;
    out[3 * r + 1] = ay;
    out[3 * r + 2] = az;
  }
}

/* W = -G sum_{i<j} m_i m_j / sqrt(|x_i-x_j|^2 + eps^2).  Row sums are formed
 * in parallel and added in row order, so the result does not depend on the
 * thread count. */
double orc_pair_potential(int64_t n, const double *x, const double *m, double G,
                          double eps) {
  const double e2 = eps * eps;
  double *row = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!row) return NAN;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < n; ++i) {
    double w = 0.0;
    for (int64_t j = i + 1; j < n; ++j) {
      const double dx = x[3 * i + 0] - x[3 * j + 0];
      const double dy = x[3 * i + 1] - x[3 * j + 1];
      const double dz = x[3 * i + 2] - x[3 * j + 2];
      w -= G * m[i] * m[j] / sqrt(dx * dx + dy * dy + dz * dz + e2);
    }
    row[i] = w;
  }
  double W = 0.0;
  for (int64_t i = 0; i < n; ++i) W += row[i];
  free(row);
  return W;
}

/* d a_i / d x_i contribution of particle j (written B):
 *   a_i gets -G m_j (x_i - x_j) s^-3, s^2 = |x_i - x_j|^2 + eps^2, so
 *   B = -G m_j [ s^-3 I - 3 s^-5 (x_i - x_j)(x_i - x_j)^T ].
 * d a_i / d x_j from the same term is -B. */
static void pair_jac_block(const double *xi, const double *xj, double mj,
                           double G, double e2, double B[9]) {
  const double r[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
  const double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + e2;
  const double s = sqrt(s2);
  const double s3 = s2 * s, s5 = s3 * s2;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      B[3 * a + b] =
          -G * mj * ((a == b ? 1.0 / s3 : 0.0) - 3.0 * r[a] * r[b] / s5);
}

/* g_k = sum_i (d a_i / d x_k)^T lam_i for k = rows[r] (or r).  Chain rule
 * in gather form: the first loop is a_k's dependence on its own position,
 * the second the dependence of every other a_i on x_k. */
void orc_pair_vjp(int64_t n, const double *x, const double *m, double G,
                  double eps, const double *lam, const int64_t *rows,
                  int64_t nrows, double *out) {
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t k = rows ? rows[r] : r;
    double g[3] = {0.0, 0.0, 0.0};
    double B[9];
    for (int64_t j = 0; j < n; ++j) { /* d a_k / d x_k */
      if (j == k) continue;
      pair_jac_block(&x[3 * k], &x[3 * j], m[j], G, e2, B);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) g[b] += B[3 * a + b] * lam[3 * k + a];
    }
    for (int64_t i = 0; i < n; ++i) { /* d a_i / d x_k = -B(x_i, x_k, m_k) */
      if (i == k) continue;
      pair_jac_block(&x[3 * i], &x[3 * k], m[k], G, e2, B);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) g[b] -= B[3 * a + b] * lam[3 * i + a];
    }
    out[3 * r + 0] = g[0];
    out[3 * r + 1] = g[1];
    out[3 * r + 2] = g[2];
  }
}

/* mbar_j = sum_{i != j} lam_i . d a_i / d m_j, d a_i / d m_j =
 * -G (x_i - x_j) s_ij^-3, for the rows j listed in rows (all j when rows is
 * NULL; out[r] belongs to rows[r]). */
void orc_pair_mass_vjp(int64_t n, const double *x, double G, double eps,
                       const double *lam, const int64_t *rows, int64_t nrows,
                       double *out) {
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t j = rows ? rows[r] : r;
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (i == j) continue;
      const double dx = x[3 * i + 0] - x[3 * j + 0];
      const double dy = x[3 * i + 1] - x[3 * j + 1];
      const double dz = x[3 * i + 2] - x[3 * j + 2];
      const double s2 = dx * dx + dy * dy + dz * dz + e2;
      const double s3 = s2 * sqrt(s2);
      acc -= G * (lam[3 * i + 0] * dx + lam[3 * i + 1] * dy +
                  lam[3 * i + 2] * dz) / s3;
    }
    out[r] = acc;
  }
}

/* ------------------------------------------------------------------------ */
/* External potentials (MWPotential2014 halo and disk, Sec. 2.2.1)          */
/* ------------------------------------------------------------------------ */

/* NFW, per unit G*M:  Phi = -ln(1 + r/r_s) / r.
 * a = -f(r) x with f(r) = ln(1+r/r_s)/r^3 - 1/(r^2 (r + r_s)).
 * For r < 1e-4 r_s the two terms cancel; f is then its Taylor series
 * 1/(2 r_s^2 r) - 2/(3 r_s^3) + 3 r/(4 r_s^4) - 4 r^2/(5 r_s^5). */
static double nfw_f(double r, double rs) {
  const double u = r / rs;
  if (u < 1e-4) {
    const double rs2 = rs * rs, rs3 = rs2 * rs;
    return 1.0 / (2.0 * rs2 * r) - 2.0 / (3.0 * rs3) +
           3.0 * r / (4.0 * rs3 * rs) - 4.0 * r * r / (5.0 * rs3 * rs2);
  }
  return log1p(u) / (r * r * r) - 1.0 / (r * r * (r + rs));
}

/* f'(r) = 1/(r^3 (r+r_s)) - 3 ln(1+r/r_s)/r^4 + (3 r + 2 r_s)/(r^3 (r+r_s)^2) */
static double nfw_fprime(double r, double rs) {
  const double r3 = r * r * r;
  return 1.0 / (r3 * (r + rs)) - 3.0 * log1p(r / rs) / (r3 * r) +
         (3.0 * r + 2.0 * rs) / (r3 * (r + rs) * (r + rs));
}

/* unit-mass (G*M = 1) NFW acceleration */
static void nfw_unit_accel(double rs, const double *p, double *a) {
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (r == 0.0) {
    a[0] = a[1] = a[2] = 0.0;
    return;
  }
  const double f = nfw_f(r, rs);
  a[0] = -f * p[0];
  a[1] = -f * p[1];
  a[2] = -f * p[2];
}

static double nfw_unit_potential(double rs, const double *p) {
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (r == 0.0) return -1.0 / rs;
  return -log1p(r / rs) / r;
}

/* d a / d x per unit G*M:  -[ f I + f'(r) x x^T / r ] */
static void nfw_unit_jac(double rs, const double *p, double J[9]) {
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  const double f = nfw_f(r, rs), fp = nfw_fprime(r, rs);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      J[3 * a + b] = -((a == b ? f : 0.0) + fp * p[a] * p[b] / r);
}

/* d(unit NFW acceleration)/d r_s.  From f above,
 * df/dr_s = -(1/r^3) (r/r_s^2)/(1 + r/r_s) + 1/(r^2 (r+r_s)^2)
 *         = -1/(r_s r (r + r_s)^2),
 * so d a/d r_s = x / (r_s r (r + r_s)^2) (zero at r = 0). */
static void nfw_unit_drs(double rs, const double *p, double *g) {
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (r == 0.0) {
    g[0] = g[1] = g[2] = 0.0;
    return;
  }
  const double c = 1.0 / (rs * r * (r + rs) * (r + rs));
  for (int d = 0; d < 3; ++d) g[d] = c * p[d];
}

/* Miyamoto-Nagai, per unit G*M:  Phi = -1/S, S^2 = R^2 + (a + B)^2,
 * B = sqrt(z^2 + b^2), R^2 = x^2 + y^2.
 * a_x = -x/S^3, a_y = -y/S^3, a_z = -z (a + B) / (B S^3). */
static void mn_unit_accel(double ma, double mb, const double *p, double *a) {
  const double B = sqrt(p[2] * p[2] + mb * mb);
  const double S2 = p[0] * p[0] + p[1] * p[1] + (ma + B) * (ma + B);
  const double S3 = S2 * sqrt(S2);
  a[0] = -p[0] / S3;
  a[1] = -p[1] / S3;
  a[2] = -p[2] * (ma + B) / (B * S3);
}

static double mn_unit_potential(double ma, double mb, const double *p) {
  const double B = sqrt(p[2] * p[2] + mb * mb);
  return -1.0 / sqrt(p[0] * p[0] + p[1] * p[1] + (ma + B) * (ma + B));
}

/* d a / d x per unit G*M.  With q = (x, y, z (a+B)/B):
 *   d a_x/dx = -(1/S^3 - 3 x^2/S^5),  d a_x/dy = 3 x y / S^5,
 *   d a_x/dz = 3 x z (a+B) / (B S^5) (and y alike),
 *   d a_z/dz = -[(1 + a b^2/B^3)/S^3 - 3 z^2 (a+B)^2 / (B^2 S^5)]. */
static void mn_unit_jac(double ma, double mb, const double *p, double J[9]) {
  const double x = p[0], y = p[1], z = p[2];
  const double B = sqrt(z * z + mb * mb);
  const double S2 = x * x + y * y + (ma + B) * (ma + B);
  const double S = sqrt(S2), S3 = S2 * S, S5 = S3 * S2;
  const double q = z * (ma + B) / B; /* d S^2/dz / 2 */
  J[0] = -(1.0 / S3 - 3.0 * x * x / S5);
  J[1] = 3.0 * x * y / S5;
  J[2] = 3.0 * x * q / S5;
  J[3] = J[1];
  J[4] = -(1.0 / S3 - 3.0 * y * y / S5);
  J[5] = 3.0 * y * q / S5;
  J[6] = J[2];
  J[7] = J[5];
  J[8] = -((1.0 + ma * mb * mb / (B * B * B)) / S3 - 3.0 * q * q / S5);
}

/* Power-law bulge with an exponential cut-off, the bulge of MWPotential2014
 * (Sec. 2.2.1): rho(r) = rho_0 (r/r_1)^-alpha exp(-(r/r_c)^2), normalised by
 * its total mass M_b = 2 pi rho_0 r_1^alpha r_c^(3-alpha) Gamma(s),
 * s = (3 - alpha)/2, so 4 pi rho_0 r_1^alpha = 2 M_b / (r_c^(3-alpha) Gamma(s)).
 * Everything follows from the density by its definitions:
 *   M(<r) = int_0^r 4 pi r'^2 rho dr'; with r' = r t^(1/(3-alpha))
 *         = 4 pi rho_0 r_1^alpha r^(3-alpha)/(3-alpha)
 *           int_0^1 exp(-(r/r_c)^2 t^(2/(3-alpha))) dt,
 *   a = -G M(<r) x / r^3,  M'(r) = 4 pi r^2 rho(r),
 *   Phi = -G M(<r)/r - G int_r^inf 4 pi r' rho(r') dr'; with
 *         r' = r + r_c w/(1-w) the tail becomes an integral over [0, 1).
 * Integrals by adaptive Simpson quadrature (relative tolerance 1e-15). */
static double simpson_rec(double (*f)(double, const double *), const double *c,
                          double a, double b, double fa, double fm, double fb,
                          double whole, double tol, int depth) {
  const double m = 0.5 * (a + b);
  const double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  const double flm = f(lm, c), frm = f(rm, c);
  const double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
  const double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  const double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * tol) return left + right + delta / 15.0;
  return simpson_rec(f, c, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
         simpson_rec(f, c, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

static double simpson(double (*f)(double, const double *), const double *c, double a,
                      double b, double rtol) {
  const double fa = f(a, c), fb = f(b, c), fm = f(0.5 * (a + b), c);
  const double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
  /* a first pass fixes the scale of the absolute tolerance */
  const double rough = simpson_rec(f, c, a, b, fa, fm, fb, whole, 1e-6 * fabs(whole) + 1e-300, 30);
  return simpson_rec(f, c, a, b, fa, fm, fb, whole, rtol * fabs(rough) + 1e-300, 50);
}

/* c = {u = (r/r_c)^2, 2/(3-alpha)} */
static double bulge_inner(double t, const double *c) {
  return exp(-c[0] * pow(t, c[1]));
}

/* c = {r, r_c, alpha} ; integrand of int_r^inf r'^(1-alpha) exp(-(r'/r_c)^2) dr' */
static double bulge_tail(double w, const double *c) {
  if (w >= 1.0) return 0.0;
  const double rp = c[0] + c[1] * w / (1.0 - w);
  const double x = rp / c[1];
  return pow(rp, 1.0 - c[2]) * exp(-x * x) * c[1] / ((1.0 - w) * (1.0 - w));
}

static double bulge_4pi_rho0r1a(double Mb, double alpha, double rc) {
  const double s = 0.5 * (3.0 - alpha);
  return 2.0 * Mb / (pow(rc, 3.0 - alpha) * tgamma(s));
}

/* enclosed mass M(<r) */
static double bulge_mass(double Mb, double alpha, double rc, double r) {
  if (r <= 0.0) return 0.0;
  const double c[2] = {(r / rc) * (r / rc), 2.0 / (3.0 - alpha)};
  return bulge_4pi_rho0r1a(Mb, alpha, rc) * pow(r, 3.0 - alpha) / (3.0 - alpha) *
         simpson(bulge_inner, c, 0.0, 1.0, 1e-15);
}

/* unit-G acceleration of the bulge */
static void bulge_accel(double Mb, double alpha, double rc, const double *p, double *a) {
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (r == 0.0) {
    a[0] = a[1] = a[2] = 0.0;
    return;
  }
  const double f = bulge_mass(Mb, alpha, rc, r) / (r * r * r);
  for (int d = 0; d < 3; ++d) a[d] = -f * p[d];
}

static double bulge_potential(double Mb, double alpha, double rc, const double *p) {
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  const double c[3] = {r, rc, alpha};
  const double tail = bulge_4pi_rho0r1a(Mb, alpha, rc) * simpson(bulge_tail, c, 0.0, 1.0, 1e-15);
  return (r > 0.0 ? -bulge_mass(Mb, alpha, rc, r) / r : 0.0) - tail;
}

/* d a / d x per unit G: -[ f I + (f'/r) x x^T ], f = M/r^3,
 * f' = M'(r)/r^3 - 3 M/r^4, M'(r) = 4 pi rho_0 r_1^alpha r^(2-alpha) exp(-(r/r_c)^2) */
static void bulge_jac(double Mb, double alpha, double rc, const double *p, double J[9]) {
  const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  const double M = bulge_mass(Mb, alpha, rc, r);
  const double Mp = bulge_4pi_rho0r1a(Mb, alpha, rc) * pow(r, 2.0 - alpha) *
                    exp(-(r / rc) * (r / rc));
  const double f = M / (r * r * r);
  const double fp = Mp / (r * r * r) - 3.0 * M / (r * r * r * r);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) J[3 * a + b] = -((a == b ? f : 0.0) + fp * p[a] * p[b] / r);
}

/* enclosed mass, exported for the quadrature's pins */
double orc_bulge_mass(double Mb, double alpha, double rc, double r) {
  return bulge_mass(Mb, alpha, rc, r);
}

/* Derivatives of the unit MN acceleration with respect to its shape
 * parameters.  With dS^2/da = 2 (a+B), dB/db = b/B, dS^2/db = 2 (a+B) b/B:
 *   d a_x/da = 3 x (a+B)/S^5,            (y alike)
 *   d a_z/da = -(z/B) [1/S^3 - 3 (a+B)^2/S^5],
 *   d a_x/db = 3 x (a+B) (b/B)/S^5,      (y alike)
 *   d a_z/db = z b [a/(B^3 S^3) + 3 (a+B)^2/(B^2 S^5)]. */
static void mn_unit_dab(double ma, double mb, const double *p, double *ga,
                        double *gb) {
  const double x = p[0], y = p[1], z = p[2];
  const double B = sqrt(z * z + mb * mb);
  const double aB = ma + B;
  const double S2 = x * x + y * y + aB * aB;
  const double S = sqrt(S2), S3 = S2 * S, S5 = S3 * S2;
  ga[0] = 3.0 * x * aB / S5;
  ga[1] = 3.0 * y * aB / S5;
  ga[2] = -(z / B) * (1.0 / S3 - 3.0 * aB * aB / S5);
  gb[0] = ga[0] * mb / B;
  gb[1] = ga[1] * mb / B;
  gb[2] = z * mb * (ma / (B * B * B * S3) + 3.0 * aB * aB / (B * B * S5));
}

/* Components of the external acceleration at one point.  parts[0..2] = NFW,
 * parts[3..5] = MN, parts[6..8] = harmonic; each is the full acceleration
 * (G*M included) of that component, zero when the component is off. */
void orc_ext_accel_parts(const orc_params *p, const double *x3, double *parts) {
  memset(parts, 0, 12 * sizeof(double));
  double u[3];
  if (p->ext & ORC_NFW) {
    nfw_unit_accel(p->nfw_rs, x3, u);
    for (int d = 0; d < 3; ++d) parts[d] = p->G * p->nfw_M * u[d];
  }
  if (p->ext & ORC_MN) {
    mn_unit_accel(p->mn_a, p->mn_b, x3, u);
    for (int d = 0; d < 3; ++d) parts[3 + d] = p->G * p->mn_M * u[d];
  }
  if (p->ext & ORC_HARM)
    for (int d = 0; d < 3; ++d) parts[6 + d] = -p->omega2 * x3[d];
  if (p->ext & ORC_BULGE) {
    bulge_accel(p->bulge_M, p->bulge_alpha, p->bulge_rc, x3, u);
    for (int d = 0; d < 3; ++d) parts[9 + d] = p->G * u[d];
  }
}

void orc_ext_accel(const orc_params *p, const double *x3, double *a3) {
  double parts[12];
  orc_ext_accel_parts(p, x3, parts);
  for (int d = 0; d < 3; ++d) a3[d] = parts[d] + parts[3 + d] + parts[6 + d] + parts[9 + d];
}

double orc_ext_potential(const orc_params *p, const double *x3) {
  double phi = 0.0;
  if (p->ext & ORC_NFW) phi += p->G * p->nfw_M * nfw_unit_potential(p->nfw_rs, x3);
  if (p->ext & ORC_MN) phi += p->G * p->mn_M * mn_unit_potential(p->mn_a, p->mn_b, x3);
  if (p->ext & ORC_HARM)
    phi += 0.5 * p->omega2 * (x3[0] * x3[0] + x3[1] * x3[1] + x3[2] * x3[2]);
  if (p->ext & ORC_BULGE)
    phi += p->G * bulge_potential(p->bulge_M, p->bulge_alpha, p->bulge_rc, x3);
  return phi;
}

/* J[3*a + b] = d a_a / d x_b of the whole external acceleration */
void orc_ext_jac(const orc_params *p, const double *x3, double *J) {
  double Ju[9];
  memset(J, 0, 9 * sizeof(double));
  if (p->ext & ORC_NFW) {
    nfw_unit_jac(p->nfw_rs, x3, Ju);
    for (int k = 0; k < 9; ++k) J[k] += p->G * p->nfw_M * Ju[k];
  }
  if (p->ext & ORC_MN) {
    mn_unit_jac(p->mn_a, p->mn_b, x3, Ju);
    for (int k = 0; k < 9; ++k) J[k] += p->G * p->mn_M * Ju[k];
  }
  if (p->ext & ORC_HARM)
    for (int d = 0; d < 3; ++d) J[4 * d] -= p->omega2;
  if (p->ext & ORC_BULGE) {
    bulge_jac(p->bulge_M, p->bulge_alpha, p->bulge_rc, x3, Ju);
    for (int k = 0; k < 9; ++k) J[k] += p->G * Ju[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Total acceleration, integrator, diagnostics                              */
/* ------------------------------------------------------------------------ */

void orc_accel(const orc_params *p, int64_t n, const double *x,
               const double *m, double *a) {
  if (p->pair)
    orc_pair_accel(n, x, m, p->G, p->eps, NULL, n, a);
  else
    memset(a, 0, (size_t)(3 * n) * sizeof(double));
  if (p->ext) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double ae[3];
      orc_ext_accel(p, &x[3 * i], ae);
      for (int d = 0; d < 3; ++d) a[3 * i + d] += ae[d];
    }
  }
}

/* Velocity-Verlet / kick-drift-kick, nsteps steps of dt, in place.
 *   v_{s+1/2} = v_s + (dt/2) a(x_s)
 *   x_{s+1}   = x_s + dt v_{s+1/2}
 *   v_{s+1}   = v_{s+1/2} + (dt/2) a(x_{s+1})
 * traj_x (optional) receives x_0..x_nsteps, traj_vh v_{1/2}..v_{nsteps-1/2}.
 * Returns 0, or -2 on allocation failure. */
int orc_integrate(const orc_params *p, int64_t n, double *x, double *v,
                  const double *m, double dt, int64_t nsteps, double *traj_x,
                  double *traj_vh) {
  const size_t n3 = (size_t)(3 * n);
  double *a = (double *)malloc((n3 ? n3 : 1) * sizeof(double));
  if (!a) return -2;
  orc_accel(p, n, x, m, a);
  if (traj_x) memcpy(traj_x, x, n3 * sizeof(double));
  for (int64_t s = 0; s < nsteps; ++s) {
    for (size_t k = 0; k < n3; ++k) v[k] += 0.5 * dt * a[k];
    for (size_t k = 0; k < n3; ++k) x[k] += dt * v[k];
    if (traj_vh) memcpy(&traj_vh[(size_t)s * n3], v, n3 * sizeof(double));
    orc_accel(p, n, x, m, a);
    for (size_t k = 0; k < n3; ++k) v[k] += 0.5 * dt * a[k];
    if (traj_x) memcpy(&traj_x[(size_t)(s + 1) * n3], x, n3 * sizeof(double));
  }
  free(a);
  return 0;
}

/* out = {K, W_pair, W_ext, P_x, P_y, P_z}:
 * K = sum m v^2 / 2, W_ext = sum m Phi_ext(x), P = sum m v. */
void orc_energy(const orc_params *p, int64_t n, const double *x,
                const double *v, const double *m, double *out) {
  double K = 0.0, We = 0.0, P[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) {
    const double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                      v[3 * i + 2] * v[3 * i + 2];
    K += 0.5 * m[i] * v2;
    if (p->ext) We += m[i] * orc_ext_potential(p, &x[3 * i]);
    for (int d = 0; d < 3; ++d) P[d] += m[i] * v[3 * i + d];
  }
  out[0] = K;
  out[1] = p->pair ? orc_pair_potential(n, x, m, p->G, p->eps) : 0.0;
  out[2] = We;
  out[3] = P[0];
  out[4] = P[1];
  out[5] = P[2];
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of orc_integrate                                        */
/* ------------------------------------------------------------------------ */

/* Adjoint of one half kick v' = v + c a(X), c = dt/2, given lam = vbar':
 *   xbar += c (da/dx)^T lam,  mbar += c (da/dm)^T lam,
 *   dt_bar += (dc/ddt) lam . a(X) = lam . a(X) / 2,
 *   Mbar_NFW += c lam . da/dM_NFW, Mbar_MN += c lam . da/dM_MN,
 *   and for the shape parameters r_s, a_MN, b_MN likewise
 *   (pbar[3..5] += c lam . da/dtheta). */
static void kick_adjoint(const orc_params *p, int64_t n, const double *X,
                         const double *m, double c, const double *lam,
                         double *xbar, double *mbar, double *pbar,
                         double *work_a, double *work_g, double *work_m) {
  orc_accel(p, n, X, m, work_a);
  double hb = 0.0;
  for (int64_t k = 0; k < 3 * n; ++k) hb += lam[k] * work_a[k];
  pbar[0] += 0.5 * hb;

  if (p->pair) {
    orc_pair_vjp(n, X, m, p->G, p->eps, lam, NULL, n, work_g);
    for (int64_t k = 0; k < 3 * n; ++k) xbar[k] += c * work_g[k];
    if (mbar) {
      orc_pair_mass_vjp(n, X, p->G, p->eps, lam, NULL, n, work_m);
      for (int64_t j = 0; j < n; ++j) mbar[j] += c * work_m[j];
    }
  }
  if (p->ext) {
    double sn = 0.0, sm = 0.0, srs = 0.0, sa = 0.0, sb = 0.0, sbm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double J[9], u[3];
      orc_ext_jac(p, &X[3 * i], J);
      for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += J[3 * a + b] * lam[3 * i + a];
        xbar[3 * i + b] += c * s;
      }
      const double *l = &lam[3 * i];
      if (p->ext & ORC_NFW) {
        nfw_unit_accel(p->nfw_rs, &X[3 * i], u);
        sn += p->G * (l[0] * u[0] + l[1] * u[1] + l[2] * u[2]);
        nfw_unit_drs(p->nfw_rs, &X[3 * i], u);
        srs += p->G * p->nfw_M * (l[0] * u[0] + l[1] * u[1] + l[2] * u[2]);
      }
      if (p->ext & ORC_BULGE) {
        bulge_accel(1.0, p->bulge_alpha, p->bulge_rc, &X[3 * i], u);
        sbm += p->G * (l[0] * u[0] + l[1] * u[1] + l[2] * u[2]);
      }
      if (p->ext & ORC_MN) {
        double ga[3], gb[3];
        mn_unit_accel(p->mn_a, p->mn_b, &X[3 * i], u);
        sm += p->G * (l[0] * u[0] + l[1] * u[1] + l[2] * u[2]);
        mn_unit_dab(p->mn_a, p->mn_b, &X[3 * i], ga, gb);
        sa += p->G * p->mn_M * (l[0] * ga[0] + l[1] * ga[1] + l[2] * ga[2]);
        sb += p->G * p->mn_M * (l[0] * gb[0] + l[1] * gb[1] + l[2] * gb[2]);
      }
    }
    pbar[1] += c * sn;
    pbar[2] += c * sm;
    pbar[3] += c * srs;
    pbar[4] += c * sa;
    pbar[5] += c * sb;
    pbar[6] += c * sbm;
  }
}

/* Reverse-mode gradient of L(x_T, v_T) through orc_integrate from (x0, v0):
 * inputs xbar = dL/dx_T, vbar = dL/dv_T; outputs dL/dx0, dL/dv0, dL/dm
 * (mbar, optional) and pbar = {dL/ddt, dL/dM_NFW, dL/dM_MN, dL/dr_s,
 * dL/da_MN, dL/db_MN, dL/dM_bulge}.
 * The forward trajectory is recomputed and kept in full.
 * Returns 0, or -2 on allocation failure. */
int orc_vjp(const orc_params *p, int64_t n, const double *x0, const double *v0,
            const double *m, double dt, int64_t nsteps, const double *xbar_T,
            const double *vbar_T, double *x0bar, double *v0bar, double *mbar,
            double *pbar) {
  const size_t n3 = (size_t)(3 * n);
  double *X = (double *)malloc((size_t)(nsteps + 1) * n3 * sizeof(double));
  double *VH = (double *)malloc((size_t)(nsteps > 0 ? nsteps : 1) * n3 * sizeof(double));
  double *x = (double *)malloc(n3 * sizeof(double));
  double *v = (double *)malloc(n3 * sizeof(double));
  double *wa = (double *)malloc(n3 * sizeof(double));
  double *wg = (double *)malloc(n3 * sizeof(double));
  double *wm = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  int rc = 0;
  if (!X || !VH || !x || !v || !wa || !wg || !wm) {
    rc = -2;
    goto done;
  }
  memcpy(x, x0, n3 * sizeof(double));
  memcpy(v, v0, n3 * sizeof(double));
  rc = orc_integrate(p, n, x, v, m, dt, nsteps, X, VH);
  if (rc) goto done;

  memcpy(x0bar, xbar_T, n3 * sizeof(double)); /* running xbar */
  memcpy(v0bar, vbar_T, n3 * sizeof(double)); /* running vbar */
  if (mbar) memset(mbar, 0, (size_t)n * sizeof(double));
  for (int k = 0; k < 7; ++k) pbar[k] = 0.0;
  for (int64_t s = nsteps - 1; s >= 0; --s) {
    const double *Xs1 = &X[(size_t)(s + 1) * n3];
    const double *Xs = &X[(size_t)s * n3];
    const double *vh = &VH[(size_t)s * n3];
    /* closing kick of step s: v_{s+1} = v_{s+1/2} + (dt/2) a(x_{s+1}) */
    kick_adjoint(p, n, Xs1, m, 0.5 * dt, v0bar, x0bar, mbar, pbar, wa, wg, wm);
    /* drift: x_{s+1} = x_s + dt v_{s+1/2} */
    for (size_t k = 0; k < n3; ++k) pbar[0] += x0bar[k] * vh[k];
    for (size_t k = 0; k < n3; ++k) v0bar[k] += dt * x0bar[k];
    /* opening kick of step s: v_{s+1/2} = v_s + (dt/2) a(x_s) */
    kick_adjoint(p, n, Xs, m, 0.5 * dt, v0bar, x0bar, mbar, pbar, wa, wg, wm);
  }
done:
  free(X);
  free(VH);
  free(x);
  free(v);
  free(wa);
  free(wg);
  free(wm);
  return rc;
}
