// ext_potential.cuh -- FP64 device functions of the external potential:
// MWPotential2014's NFW halo, Miyamoto-Nagai disk and bulge (paper
// Sec. 2.2.1),
//   NFW  Phi = -G M ln(1 + r/r_s) / r,
//   MN   Phi = -G M / sqrt(R^2 + (a + sqrt(z^2 + b^2))^2),
//   bulge rho = rho_0 (r/r_1)^-alpha exp(-(r/r_c)^2) with total mass M_b:
//        M(<r) = M_b P(s, r^2/r_c^2), s = (3 - alpha)/2, a = -G M(<r) x / r^3,
//        Phi = -G M_b [P(s, u)/r + Gamma(s - 1/2, u) / (r_c Gamma(s))],
// their accelerations (per unit G M and full) and the Jacobian-vector
// product of the acceleration.  Shared by the integrator, the adjoint and
// the single-orbit kernels.
#pragma once

#include "nbody_internal.cuh"

namespace nb {

// Unit-mass (G M = 1) accelerations of the halo and the disk.
struct ExtUnit {
  double n[3];
  double d[3];
  double b[3];
};

// Incomplete gamma functions, each with a bounded number of terms:
//   gamma(s, u) = e^-u u^s sum_{n>=0} u^n / (s (s+1) ... (s+n))   (u < s+1;
//                 the power series, Abramowitz & Stegun 6.5.29),
//   Gamma(s, u) = e^-u u^s / K,  K = b_0 + a_1 / (b_1 + a_2 / (b_2 + ...)),
//                 b_k = u + 2k + 1 - s, a_k = -k (k - s)   (u >= s+1; the
//                 Legendre continued fraction, A&S 6.5.31, in its even form).
// lnpre = s ln u - u.
static __device__ __forceinline__ double igamma_lower_series(double s, double u,
                                                             double lnpre) {
  double ap = s, term = 1.0 / s, sum = term;
  for (int k = 0; k < 400; ++k) {
    ap += 1.0;
    term *= u / ap;
    sum += term;
    if (fabs(term) < fabs(sum) * 1e-17) break;
  }
  return sum * exp(lnpre);
}

// K by its convergents K_k = P_k / Q_k and the three-term recurrences
// P_k = b_k P_{k-1} + a_k P_{k-2}, Q_k = b_k Q_{k-1} + a_k Q_{k-2}
// (P_{-1} = 1, Q_{-1} = 0, P_0 = b_0, Q_0 = 1), both pairs divided by Q_k
// after every step so that Q_k = 1 and K_k = P_k stay in range; stops when
// two convergents agree to 1e-16.
static __device__ __forceinline__ double igamma_upper_cf(double s, double u, double lnpre) {
  double p_prev = 1.0, q_prev = 0.0;  // P_{k-1}, Q_{k-1} (scaled)
  double p = u + 1.0 - s, q = 1.0;    // P_k, Q_k
  for (int k = 1; k < 400; ++k) {
    const double a = -(double)k * ((double)k - s);
    const double b = u + (double)(2 * k + 1) - s;
    const double p_new = b * p + a * p_prev;
    const double q_new = b * q + a * q_prev;
    const double inv = 1.0 / q_new;
    p_prev = p * inv;
    q_prev = q * inv;
    const double k_old = p / q;
    p = p_new * inv;
    q = 1.0;
    if (fabs(p - k_old) <= 1e-16 * fabs(p)) break;
  }
  return exp(lnpre) / p;
}

// regularised lower incomplete gamma P(s, u); 1 beyond u = 60, where
// 1 - P < 1e-26
static __device__ __forceinline__ double bulge_P(const DevParams& P, double u) {
  if (u <= 0.0) return 0.0;
  if (u > 60.0) return 1.0;
  const double s = P.bulge_s;
  const double lnpre = s * log(u) - u;
  return u < s + 1.0 ? igamma_lower_series(s, u, lnpre) * P.bulge_igs
                     : 1.0 - igamma_upper_cf(s, u, lnpre) * P.bulge_igs;
}

// upper incomplete gamma Gamma(s - 1/2, u) (not regularised), 0 < s - 1/2 <= 1
static __device__ __forceinline__ double bulge_upper(const DevParams& P, double u) {
  const double sh = P.bulge_s - 0.5;
  if (u <= 0.0) return P.bulge_gsh;
  const double lnpre = sh * log(u) - u;
  return u < sh + 1.0 ? P.bulge_gsh - igamma_lower_series(sh, u, lnpre)
                      : igamma_upper_cf(sh, u, lnpre);
}

static __device__ __forceinline__ double nfw_f(double r, double rs) {
  // a_NFW = -G M f(r) x, f(r) = ln(1 + r/r_s)/r^3 - 1/(r^2 (r + r_s));
  // below r = 1e-4 r_s the two terms cancel and the Taylor series is used.
  const double u = r / rs;
  if (u < 1e-4) {
    const double rs2 = rs * rs, rs3 = rs2 * rs;
    return (0.5 / rs2) / r - (2.0 / 3.0) / rs3 + (0.75 / (rs3 * rs)) * r -
           (0.8 / (rs3 * rs2)) * r * r;
  }
  return (log1p(u) / r - 1.0 / (r + rs)) / (r * r);
}

static __device__ __forceinline__ double nfw_fprime_over_r(double r, double rs) {
  // f'(r)/r with f' = 1/(r^3 (r+r_s)) - 3 ln(1+r/r_s)/r^4
  //                   + (3 r + 2 r_s)/(r^3 (r+r_s)^2)
  const double u = r / rs;
  if (u < 1e-4) {
    const double rs2 = rs * rs, rs4 = rs2 * rs2;
    return (-0.5 / rs2) / (r * r * r) + (0.75 / rs4) / r - 1.6 / (rs4 * rs);
  }
  const double rp = r + rs;
  const double r3 = r * r * r;
  return (1.0 / (r3 * rp) - 3.0 * log1p(u) / (r3 * r) +
          (3.0 * r + 2.0 * rs) / (r3 * rp * rp)) / r;
}

// FP64 reciprocal square root by Newton-Raphson refinement of the FP32 MUFU
// approximation: y <- y + y (1 - v y^2) / 2 squares the relative error
// (about 2^-22 after the seed, 2^-44 after one step, FP64 rounding after
// two).  It gives 1/r and, with one multiply, r, for less than the cost of
// the correctly rounded square root and division (measured on GB300: 4.0
// against 3.3 + 2.4 time units of a dependent FP64 FMA chain's 1.0).
// Arguments outside the FP32 normal range take the exact expression.
static __device__ __forceinline__ double rsqrt_nr(double v) {
  if (!(v > 1e-30 && v < 1e30)) return 1.0 / sqrt(v);
  float s;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"((float)v));
  double y = (double)s;
  double e = fma(-v * y, y, 1.0);
  y = fma(0.5 * y, e, y);
  e = fma(-v * y, y, 1.0);
  return fma(0.5 * y, e, y);
}

// Unit accelerations of the forward integration, with 1/r, 1/B and 1/S from
// rsqrt_nr: NFW f = (ln(1 + r/r_s)/r - 1/(r + r_s)) / r^2 (the Taylor
// series of nfw_f below r = 1e-4 r_s); MN 1/S^3 and z (a + B)/B.
static __device__ __forceinline__ void ext_unit(const DevParams& P, double x,
                                         double y, double z, ExtUnit& e) {
  e.n[0] = e.n[1] = e.n[2] = 0.0;
  e.d[0] = e.d[1] = e.d[2] = 0.0;
  if (P.ext & NBODY_EXT_NFW) {
    const double r2 = x * x + y * y + z * z;
    if (r2 > 0.0) {
      const double ir = rsqrt_nr(r2);
      const double r = r2 * ir;
      const double u = r / P.nfw_rs;
      const double f = u < 1e-4 ? nfw_f(r, P.nfw_rs)
                                : (log1p(u) * ir - 1.0 / (r + P.nfw_rs)) * (ir * ir);
      e.n[0] = -f * x;
      e.n[1] = -f * y;
      e.n[2] = -f * z;
    }
  }
  if (P.ext & NBODY_EXT_MN) {
    const double B2 = z * z + P.mn_b * P.mn_b;
    const double iB = B2 > 0.0 ? rsqrt_nr(B2) : 0.0;
    const double aB = P.mn_a + B2 * iB;
    const double iS = rsqrt_nr(x * x + y * y + aB * aB);
    const double iS3 = iS * iS * iS;
    e.d[0] = -x * iS3;
    e.d[1] = -y * iS3;
    e.d[2] = -z * aB * iB * iS3;
  }
  e.b[0] = e.b[1] = e.b[2] = 0.0;
  if (P.ext & NBODY_EXT_BULGE) {
    const double r2 = x * x + y * y + z * z;
    if (r2 > 0.0) {
      const double ir = rsqrt_nr(r2);
      const double f = bulge_P(P, r2 * P.bulge_irc2) * (ir * ir * ir);
      e.b[0] = -f * x;
      e.b[1] = -f * y;
      e.b[2] = -f * z;
    }
  }
}

// full external acceleration (G M included) at one point
static __device__ __forceinline__ void ext_accel(const DevParams& P, double x, double y,
                                          double z, double a[3]) {
  ExtUnit e;
  ext_unit(P, x, y, z, e);
#pragma unroll
  for (int d = 0; d < 3; ++d) a[d] = P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d];
}

// (d a_ext / d x) l, full accelerations (G M included); the Jacobian is
// symmetric so this is also J^T l.
static __device__ __forceinline__ void ext_jvp(const DevParams& P, double x, double y,
                                        double z, const double l[3],
                                        double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (P.ext & NBODY_EXT_NFW) {
    const double r = sqrt(x * x + y * y + z * z);
    if (r > 0.0) {
      // J = -G M [ f I + (f'/r) x x^T ]
      const double f = nfw_f(r, P.nfw_rs);
      const double g = nfw_fprime_over_r(r, P.nfw_rs);
      const double xl = x * l[0] + y * l[1] + z * l[2];
      out[0] -= P.nfw_GM * (f * l[0] + g * xl * x);
      out[1] -= P.nfw_GM * (f * l[1] + g * xl * y);
      out[2] -= P.nfw_GM * (f * l[2] + g * xl * z);
    }
  }
  if (P.ext & NBODY_EXT_MN) {
    // a = -G M q / S^3 with q = (x, y, z (a+B)/B), S^2 = R^2 + (a+B)^2:
    // J = -G M [ dq/dx / S^3 - 3 q q^T / S^5 ],
    // dq/dx = diag(1, 1, 1 + a b^2 / B^3)
    const double b2 = P.mn_b * P.mn_b;
    const double B = sqrt(z * z + b2);
    const double aB = P.mn_a + B;
    const double S2 = x * x + y * y + aB * aB;
    const double iS = 1.0 / sqrt(S2);
    const double iS3 = iS * iS * iS;
    const double iS5 = iS3 * iS * iS;
    const double q2 = z * aB / B;
    const double ql = x * l[0] + y * l[1] + q2 * l[2];
    const double dz = 1.0 + P.mn_a * b2 / (B * B * B);
    out[0] -= P.mn_GM * (l[0] * iS3 - 3.0 * x * ql * iS5);
    out[1] -= P.mn_GM * (l[1] * iS3 - 3.0 * y * ql * iS5);
    out[2] -= P.mn_GM * (dz * l[2] * iS3 - 3.0 * q2 * ql * iS5);
  }
  if (P.ext & NBODY_EXT_BULGE) {
    // J = -G M_b [ f I + (f'/r) x x^T ], f = P(s,u)/r^3, u = r^2/r_c^2,
    // f'/r = (2/r_c^2) P'(u)/r^3 - 3 P/r^5, P'(u) = u^(s-1) e^-u / Gamma(s)
    const double r2 = x * x + y * y + z * z;
    if (r2 > 0.0) {
      const double u = r2 * P.bulge_irc2;
      const double ir = 1.0 / sqrt(r2);
      const double ir3 = ir * ir * ir;
      const double Pu = bulge_P(P, u);
      const double dP = u > 700.0 ? 0.0 : exp((P.bulge_s - 1.0) * log(u) - u) * P.bulge_igs;
      const double f = Pu * ir3;
      const double g = 2.0 * P.bulge_irc2 * dP * ir3 - 3.0 * Pu * ir3 * ir * ir;
      const double xl = x * l[0] + y * l[1] + z * l[2];
      out[0] -= P.bulge_GM * (f * l[0] + g * xl * x);
      out[1] -= P.bulge_GM * (f * l[1] + g * xl * y);
      out[2] -= P.bulge_GM * (f * l[2] + g * xl * z);
    }
  }
}

// l . d a_ext / d theta for the shape parameters theta = (r_s, a_MN, b_MN),
// full accelerations (G M included):
//   NFW: d a / d r_s = G M x / (r_s r (r + r_s)^2);
//   MN, with S^2 = R^2 + (a+B)^2, B = sqrt(z^2 + b^2):
//     d a_{x,y} / d a = 3 G M {x,y} (a+B) / S^5,
//     d a_z / d a     = -G M (z/B) [1/S^3 - 3 (a+B)^2/S^5],
//     d a_{x,y} / d b = (b/B) d a_{x,y} / d a,
//     d a_z / d b     = G M z b [a/(B^3 S^3) + 3 (a+B)^2/(B^2 S^5)].
static __device__ __forceinline__ void ext_shape_vjp(const DevParams& P, double x,
                                              double y, double z, const double l[3],
                                              double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (P.ext & NBODY_EXT_NFW) {
    const double r = sqrt(x * x + y * y + z * z);
    if (r > 0.0) {
      const double rp = r + P.nfw_rs;
      out[0] = P.nfw_GM * (x * l[0] + y * l[1] + z * l[2]) / (P.nfw_rs * r * rp * rp);
    }
  }
  if (P.ext & NBODY_EXT_MN) {
    const double b = P.mn_b;
    const double B = sqrt(z * z + b * b);
    const double aB = P.mn_a + B;
    const double S2 = x * x + y * y + aB * aB;
    const double iS = 1.0 / sqrt(S2);
    const double iS3 = iS * iS * iS;
    const double iS5 = iS3 * iS * iS;
    const double xy = x * l[0] + y * l[1];
    const double iB = 1.0 / B;
    const double da_z = -(z * iB) * (iS3 - 3.0 * aB * aB * iS5);
    const double db_z = z * b * (P.mn_a * iB * iB * iB * iS3 + 3.0 * aB * aB * iB * iB * iS5);
    const double da_xy = 3.0 * aB * iS5 * xy;
    out[1] = P.mn_GM * (da_xy + da_z * l[2]);
    out[2] = P.mn_GM * (da_xy * b * iB + db_z * l[2]);
  }
}

// Everything the adjoint of a kick needs of the external field at one
// point, with the square roots, the logarithm and the incomplete gamma
// function taken once: for cotangents l,
//   jl = (d a_ext / d x) l                           (as ext_jvp),
//   ln = l . e.n, lm = l . e.d, lb = l . e.b          (unit accelerations, as ext_unit),
//   sh = l . d a_ext / d (r_s, a_MN, b_MN)            (as ext_shape_vjp; SHAPE only).
struct ExtAdj {
  double jl[3];
  double ln, lm, lb;
  double sh[3];
};

template <bool SHAPE>
static __device__ __forceinline__ void ext_adjoint(const DevParams& P, double x, double y,
                                                   double z, const double l[3], ExtAdj& o) {
  o.jl[0] = o.jl[1] = o.jl[2] = 0.0;
  o.ln = o.lm = o.lb = 0.0;
  o.sh[0] = o.sh[1] = o.sh[2] = 0.0;
  const double xl = x * l[0] + y * l[1] + z * l[2];
  const double r2 = x * x + y * y + z * z;
  if ((P.ext & NBODY_EXT_NFW) && r2 > 0.0) {
    // a = -G M f(r) x; J = -G M [f I + (f'/r) x x^T] (nfw_f, nfw_fprime_over_r)
    const double rs = P.nfw_rs;
    const double ir = rsqrt_nr(r2);
    const double r = r2 * ir;
    const double u = r / rs;
    const double irp = 1.0 / (r + rs);
    double f, g;
    if (u < 1e-4) {
      f = nfw_f(r, rs);
      g = nfw_fprime_over_r(r, rs);
    } else {
      const double L = log1p(u);
      const double ir2 = ir * ir, ir3 = ir2 * ir;
      f = (L * ir - irp) * ir2;
      g = (ir3 * irp - 3.0 * L * ir2 * ir2 + (3.0 * r + 2.0 * rs) * ir3 * irp * irp) * ir;
    }
    o.ln = -f * xl;
    o.jl[0] -= P.nfw_GM * (f * l[0] + g * xl * x);
    o.jl[1] -= P.nfw_GM * (f * l[1] + g * xl * y);
    o.jl[2] -= P.nfw_GM * (f * l[2] + g * xl * z);
    if (SHAPE) o.sh[0] = P.nfw_GM * xl * ir * irp * irp / rs;  // G M x.l / (r_s r (r+r_s)^2)
  }
  if (P.ext & NBODY_EXT_MN) {
    // a = -G M q / S^3, q = (x, y, z (a+B)/B); J and the shape terms as in
    // ext_jvp and ext_shape_vjp
    const double b = P.mn_b;
    const double B2 = z * z + b * b;
    const double iB = B2 > 0.0 ? rsqrt_nr(B2) : 0.0;
    const double B = B2 * iB;
    const double aB = P.mn_a + B;
    const double iS = rsqrt_nr(x * x + y * y + aB * aB);
    const double iS2 = iS * iS, iS3 = iS2 * iS, iS5 = iS3 * iS2;
    const double q2 = z * aB * iB;
    const double xy = x * l[0] + y * l[1];
    const double ql = xy + q2 * l[2];
    o.lm = -ql * iS3;
    const double dz = 1.0 + P.mn_a * b * b * iB * iB * iB;
    o.jl[0] -= P.mn_GM * (l[0] * iS3 - 3.0 * x * ql * iS5);
    o.jl[1] -= P.mn_GM * (l[1] * iS3 - 3.0 * y * ql * iS5);
    o.jl[2] -= P.mn_GM * (dz * l[2] * iS3 - 3.0 * q2 * ql * iS5);
    if (SHAPE) {
      const double da_z = -(z * iB) * (iS3 - 3.0 * aB * aB * iS5);
      const double db_z = z * b * (P.mn_a * iB * iB * iB * iS3 + 3.0 * aB * aB * iB * iB * iS5);
      const double da_xy = 3.0 * aB * iS5 * xy;
      o.sh[1] = P.mn_GM * (da_xy + da_z * l[2]);
      o.sh[2] = P.mn_GM * (da_xy * b * iB + db_z * l[2]);
    }
  }
  if ((P.ext & NBODY_EXT_BULGE) && r2 > 0.0) {
    // a = -G M_b P(s, u) x / r^3, u = r^2 / r_c^2; J as in ext_jvp
    const double u = r2 * P.bulge_irc2;
    const double ir = rsqrt_nr(r2);
    const double ir3 = ir * ir * ir;
    const double Pu = bulge_P(P, u);
    const double dP = u > 700.0 ? 0.0 : exp((P.bulge_s - 1.0) * log(u) - u) * P.bulge_igs;
    const double f = Pu * ir3;
    const double g = 2.0 * P.bulge_irc2 * dP * ir3 - 3.0 * Pu * ir3 * ir * ir;
    o.lb = -f * xl;
    o.jl[0] -= P.bulge_GM * (f * l[0] + g * xl * x);
    o.jl[1] -= P.bulge_GM * (f * l[1] + g * xl * y);
    o.jl[2] -= P.bulge_GM * (f * l[2] + g * xl * z);
  }
}

static __device__ __forceinline__ double ext_potential(const DevParams& P, double x,
                                                double y, double z) {
  double phi = 0.0;
  if (P.ext & NBODY_EXT_NFW) {
    const double r = sqrt(x * x + y * y + z * z);
    phi -= P.nfw_GM * (r > 0.0 ? log1p(r / P.nfw_rs) / r : 1.0 / P.nfw_rs);
  }
  if (P.ext & NBODY_EXT_MN) {
    const double B = sqrt(z * z + P.mn_b * P.mn_b);
    const double aB = P.mn_a + B;
    phi -= P.mn_GM / sqrt(x * x + y * y + aB * aB);
  }
  if (P.ext & NBODY_EXT_BULGE) {
    const double r2 = x * x + y * y + z * z;
    const double u = r2 * P.bulge_irc2;
    const double inner = r2 > 0.0 ? bulge_P(P, u) / sqrt(r2) : 0.0;
    phi -= P.bulge_GM * (inner + bulge_upper(P, u) * P.bulge_irc * P.bulge_igs);
  }
  return phi;
}


}  // namespace nb
