// orbitfit.cu -- orbit fitting of the progenitor and the Fisher matrix
// (paper Sec. 2.2.2).  A single particle is integrated from its present-day
// phase-space point forward and backward in the NFW + Miyamoto-Nagai field
// with kick-drift-kick steps, projected onto the stream frame (phi1, phi2,
// mu_phi1 cos phi2, mu_phi2, v_h), interpolated along phi1 at the observed
// points and compared by chi^2 = sum (model - obs)^2 / sigma^2.  The five
// parameters are theta = (M_NFW, r_s, M_MN, a_MN, b_MN), handled as
// xi = ln theta.
//
// GPU form: one thread per parameter vector.  The orbit, the projection and
// the interpolation run in forward-mode dual numbers over the five xi, so
// every evaluation returns chi^2, its exact gradient and the Gauss-Newton
// matrix sum_r (dr/dxi)(dr/dxi)^T (one half of the Gauss-Newton Hessian of
// chi^2), accumulated while the orbit streams past the sorted observations.
// Levenberg-Marquardt runs whole inside a group of 16 lanes, 8 per half of
// the arc, each lane carrying one derivative direction (1000 random starts
// are 16000 threads); every loop has a fixed bound.
//
// The arc: from t = 0 forward while phi1 stays in the window and keeps
// increasing, and backward (step -dt) while it stays in the window and keeps
// decreasing, at most t_max each way; an observation beyond the arc's end
// takes the end point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "dual.cuh"
#include "nbody_internal.cuh"

namespace nb {
namespace {

constexpr int kP = 5;  // parameters
using D5 = Dual<kP>;
using H5 = HDual<kP>;  // second order, for the exact Hessian
using D1 = Dual<1>;    // one derivative direction per lane (lane-parallel fits)

template <class T>
__device__ __forceinline__ T cst(double c);
template <>
__device__ __forceinline__ D5 cst<D5>(double c) {
  return dconst<kP>(c);
}
template <>
__device__ __forceinline__ H5 cst<H5>(double c) {
  return hconst<kP>(c);
}
template <>
__device__ __forceinline__ D1 cst<D1>(double c) {
  return dconst<1>(c);
}

constexpr double kMasYr = 206.26480624709636;        // 1 rad/Myr in mas/yr
constexpr double kKms = 1.0227121650537077e-3;       // 1 km/s in kpc/Myr

struct FitCfg {
  double G;
  double X0[3], V0[3];
  double xo[3], vo[3];
  double e1[3], e2[3], nv[3];
  double lo, hi;   // phi1 window
  double dt;
  int64_t nmax;    // steps per direction
  double isig[4];  // 1 / sigma of (phi2, mu1, mu2, v_h)
};

struct Acc {  // running chi^2, gradient (d chi^2 / d xi), Gauss-Newton matrix
  double chi2;
  double g[kP];
  double A[kP][kP];
};

struct AccH : Acc {  // and the exact Hessian d^2 chi^2 / d xi^2
  double H[kP][kP];
};

// Lane-parallel accumulation: 8 lanes per half-arc, lane `dir` carries the
// derivative along xi_dir (lanes 5..7 repeat direction 4); the lanes of a
// half see the same values, so they take the same branches.  Row `dir` of
// the Gauss-Newton matrix gathers the other directions by shuffles.
struct AccL {
  double chi2;
  double g;         // d chi^2 / d xi_dir
  double A[kP];     // row dir of sum (dr/dxi)(dr/dxi)^T
  unsigned mask;    // the 8 lanes of this half
  int base;         // lane of direction 0 of this half
  int dir;
};

// NFW + MN acceleration in duals; th = (M_NFW, r_s, M_MN, a, b)
template <class T>
__device__ void field(const FitCfg& c, const T x[3], const T th[kP], T a[3]) {
  const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const T r = dsqrt(r2);
  const T u = r / th[1];
  T f;
  if (u.v < 1e-4) {
    // Taylor series of the NFW f(r) below r = 1e-4 r_s
    const T rs = th[1];
    const T rs2 = rs * rs, rs3 = rs2 * rs;
    f = cst<T>(0.5) / (rs2 * r) - cst<T>(2.0 / 3.0) / rs3 + cst<T>(0.75) * r / (rs3 * rs) -
        cst<T>(0.8) * r2 / (rs3 * rs2);
  } else {
    f = (dlog1p(u) / r - cst<T>(1.0) / (r + th[1])) / r2;
  }
  const T gmn = c.G * th[0];
  const T B = dsqrt(x[2] * x[2] + th[4] * th[4]);
  const T aB = th[3] + B;
  const T S2 = x[0] * x[0] + x[1] * x[1] + aB * aB;
  const T iS3 = cst<T>(1.0) / (S2 * dsqrt(S2));
  const T gmd = c.G * th[2];
  const T kn = gmn * f, kd = gmd * iS3;
  a[0] = -(kn * x[0]) - kd * x[0];
  a[1] = -(kn * x[1]) - kd * x[1];
  a[2] = -(kn * x[2]) - kd * x[2] * aB / B;
}

// (phi1, phi2, mu1 [mas/yr], mu2 [mas/yr], v_h [km/s])
template <class T>
__device__ void observe(const FitCfg& c, const T x[3], const T v[3], T q[5]) {
  T d[3], w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d[k] = x[k] - c.xo[k];
    w[k] = v[k] - c.vo[k];
  }
  const T d1 = c.e1[0] * d[0] + c.e1[1] * d[1] + c.e1[2] * d[2];
  const T d2 = c.e2[0] * d[0] + c.e2[1] * d[1] + c.e2[2] * d[2];
  const T d3 = c.nv[0] * d[0] + c.nv[1] * d[1] + c.nv[2] * d[2];
  const T w1 = c.e1[0] * w[0] + c.e1[1] * w[1] + c.e1[2] * w[2];
  const T w2 = c.e2[0] * w[0] + c.e2[1] * w[1] + c.e2[2] * w[2];
  const T w3 = c.nv[0] * w[0] + c.nv[1] * w[1] + c.nv[2] * w[2];
  const T rho2 = d1 * d1 + d2 * d2;
  const T D2 = rho2 + d3 * d3;
  const T D = dsqrt(D2);
  const T rho = dsqrt(rho2);
  q[0] = datan2(d2, d1);
  q[1] = dasin(d3 / D);
  q[2] = kMasYr * ((d1 * w2 - d2 * w1) / (rho * D));
  q[3] = kMasYr * ((rho * w3 - d3 * (d1 * w1 + d2 * w2) / rho) / D2);
  q[4] = (1.0 / kKms) * ((d1 * w1 + d2 * w2 + d3 * w3) / D);
}

// residuals of observation j against model q (4 duals) into the running sums
__device__ void add_obs(const FitCfg& c, const double* ob, const D5 q[4], Acc& s) {
  D5 r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = c.isig[k] * (q[k] - ob[1 + k]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s.chi2 += r[k].v * r[k].v;
#pragma unroll
    for (int a = 0; a < kP; ++a) {
      s.g[a] += 2.0 * r[k].v * r[k].d[a];
#pragma unroll
      for (int b = 0; b < kP; ++b) s.A[a][b] += r[k].d[a] * r[k].d[b];
    }
  }
}

// the same with second derivatives: d^2 chi^2 = 2 sum (r_a r_b + r r_ab)
__device__ void add_obs(const FitCfg& c, const double* ob, const H5 q[4], AccH& s) {
  H5 r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = c.isig[k] * (q[k] - ob[1 + k]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s.chi2 += r[k].v * r[k].v;
    int p = 0;
#pragma unroll
    for (int a = 0; a < kP; ++a) {
      s.g[a] += 2.0 * r[k].v * r[k].d[a];
#pragma unroll
      for (int b = 0; b < kP; ++b) s.A[a][b] += r[k].d[a] * r[k].d[b];
#pragma unroll
      for (int b = a; b < kP; ++b, ++p) {
        const double hab = 2.0 * (r[k].d[a] * r[k].d[b] + r[k].v * r[k].h[p]);
        s.H[a][b] += hab;
        if (b != a) s.H[b][a] += hab;
      }
    }
  }
}

__device__ void add_obs(const FitCfg& c, const double* ob, const D1 q[4], AccL& s) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const D1 r = c.isig[k] * (q[k] - ob[1 + k]);
    s.chi2 += r.v * r.v;
    s.g += 2.0 * r.v * r.d[0];
#pragma unroll
    for (int b = 0; b < kP; ++b) {
      const double rb = __shfl_sync(s.mask, r.d[0], s.base + b);
      s.A[b] += r.d[0] * rb;
    }
  }
}

// linear interpolation of (phi2, mu1, mu2, v_h) at phi1 = p between two
// arc points
template <class T>
__device__ void interp(const T qa[5], const T qb[5], double p, T out[4]) {
  const T w = (p - qa[0]) / (qb[0] - qa[0]);
#pragma unroll
  for (int k = 0; k < 4; ++k) out[k] = qa[1 + k] + w * (qb[1 + k] - qa[1 + k]);
}

// One half of the arc (sign = +1 forward, -1 backward) with the observations
// of that side: obs sorted by phi1; forward side j = jb, jb+1, .. n-1;
// backward side j = jb, jb-1, .. 0.  arc_out (values, may be NULL) receives
// the points, the count returned.
template <class T, class S>
__device__ int64_t half_arc(const FitCfg& c, const T th[kP], double sign, const double* obs,
                            int n_obs, int jb, S& s, double* arc_out) {
  T x[3], v[3], a[3], q[5], qp[5];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    x[k] = cst<T>(c.X0[k]);
    v[k] = cst<T>(c.V0[k]);
  }
  observe(c, x, v, q);
  int64_t npts = 1;
  if (arc_out)
    for (int k = 0; k < 5; ++k) arc_out[k] = q[k].v;
  int j = jb;
  const int dj = sign > 0 ? 1 : -1;
  field(c, x, th, a);
  const double h = sign * c.dt;
  for (int64_t step = 0; step < c.nmax; ++step) {
#pragma unroll
    for (int k = 0; k < 5; ++k) qp[k] = q[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] = v[k] + (0.5 * h) * a[k];
      x[k] = x[k] + h * v[k];
    }
    field(c, x, th, a);
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = v[k] + (0.5 * h) * a[k];
    observe(c, x, v, q);
    if (!(q[0].v >= c.lo && q[0].v <= c.hi) || !(sign * (q[0].v - qp[0].v) > 0.0)) {
#pragma unroll
      for (int k = 0; k < 5; ++k) q[k] = qp[k];  // the arc ends at the previous point
      break;
    }
    // observations between the previous and this point
    while (j >= 0 && j < n_obs && sign * (obs[5 * j] - q[0].v) < 0.0) {
      T m[4];
      interp(qp, q, obs[5 * j], m);
      add_obs(c, obs + 5 * j, m, s);
      j += dj;
    }
    if (arc_out)
      for (int k = 0; k < 5; ++k) arc_out[5 * npts + k] = q[k].v;
    ++npts;
  }
  // observations beyond the arc's end take the end point
  while (j >= 0 && j < n_obs) {
    T m[4] = {q[1], q[2], q[3], q[4]};
    add_obs(c, obs + 5 * j, m, s);
    j += dj;
  }
  return npts;
}

__device__ void evaluate(const FitCfg& c, const double* obs, int n_obs, int split,
                         const double xi[kP], Acc& s) {
  D5 th[kP];
#pragma unroll
  for (int k = 0; k < kP; ++k) {
    const double t = exp(xi[k]);
    th[k] = dconst<kP>(t);
    th[k].d[k] = t;  // d theta / d xi
  }
  s.chi2 = 0.0;
#pragma unroll
  for (int a = 0; a < kP; ++a) {
    s.g[a] = 0.0;
#pragma unroll
    for (int b = 0; b < kP; ++b) s.A[a][b] = 0.0;
  }
  half_arc(c, th, 1.0, obs, n_obs, split, s, nullptr);
  half_arc(c, th, -1.0, obs, n_obs, split - 1, s, nullptr);
}

__global__ void k_fit_eval(FitCfg c, const double* __restrict__ obs, int n_obs, int split,
                           const double* __restrict__ xi, int count, double* __restrict__ chi2,
                           double* __restrict__ grad, double* __restrict__ gn) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double z[kP];
  for (int k = 0; k < kP; ++k) z[k] = xi[kP * t + k];
  Acc s;
  evaluate(c, obs, n_obs, split, z, s);
  chi2[t] = s.chi2;
  if (grad)
    for (int k = 0; k < kP; ++k) grad[kP * t + k] = s.g[k];
  if (gn)
    for (int a = 0; a < kP; ++a)
      for (int b = 0; b < kP; ++b) gn[kP * kP * t + kP * a + b] = s.A[a][b];
}

// chi^2, gradient, Gauss-Newton matrix and exact Hessian (second-order
// duals; d theta / d xi = d^2 theta / d xi^2 = theta)
__global__ void k_fit_hess(FitCfg c, const double* __restrict__ obs, int n_obs, int split,
                           const double* __restrict__ xi, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  H5 th[kP];
  for (int k = 0; k < kP; ++k) {
    const double t = exp(xi[k]);
    th[k] = hconst<kP>(t);
    th[k].d[k] = t;
    int p = 0;  // index of (k, k) in the upper triangle
    for (int i = 0; i < k; ++i) p += kP - i;
    th[k].h[p] = t;
  }
  AccH s;
  s.chi2 = 0.0;
  for (int a = 0; a < kP; ++a) {
    s.g[a] = 0.0;
    for (int b = 0; b < kP; ++b) s.A[a][b] = s.H[a][b] = 0.0;
  }
  half_arc(c, th, 1.0, obs, n_obs, split, s, nullptr);
  half_arc(c, th, -1.0, obs, n_obs, split - 1, s, nullptr);
  out[0] = s.chi2;
  for (int a = 0; a < kP; ++a) {
    out[1 + a] = s.g[a];
    for (int b = 0; b < kP; ++b) {
      out[1 + kP + kP * a + b] = s.A[a][b];
      out[1 + kP + kP * kP + kP * a + b] = s.H[a][b];
    }
  }
}

// solve (A + lam diag(A)) x = b by Cholesky; false if not positive definite
__device__ bool damped_solve(const double A[kP][kP], double lam, const double b[kP],
                             double x[kP]) {
  double L[kP][kP];
  double dmax = 0.0;
  for (int k = 0; k < kP; ++k) dmax = fmax(dmax, A[k][k]);
  for (int i = 0; i < kP; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[i][j];
      if (i == j) s += lam * A[i][i] + 1e-14 * dmax;
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  double y[kP];
  for (int i = 0; i < kP; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = kP - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < kP; ++k) s -= L[k][i] * x[k];
    x[i] = s / L[i][i];
  }
  return true;
}

// One lane group (16 lanes: 8 per half-arc) evaluates chi^2, its gradient
// and the Gauss-Newton matrix at xi; every lane of the group ends with the
// same full results (sums combined in the same order everywhere).
__device__ void evaluate_lanes(const FitCfg& c, const double* obs, int n_obs, int split,
                               const double xi[kP], int glane, unsigned gmask, Acc& out) {
  const int half = glane >> 3;
  const int dir = min(glane & 7, kP - 1);
  const int lane = threadIdx.x & 31;
  const int gbase = lane - glane;  // first lane of the group
  AccL s;
  s.chi2 = 0.0;
  s.g = 0.0;
  for (int b = 0; b < kP; ++b) s.A[b] = 0.0;
  s.base = gbase + 8 * half;
  s.mask = 0xFFu << s.base;
  s.dir = dir;
  D1 th[kP];
  for (int k = 0; k < kP; ++k) {
    const double t = exp(xi[k]);
    th[k] = dconst<1>(t);
    if (k == dir) th[k].d[0] = t;
  }
  if (half == 0)
    half_arc(c, th, 1.0, obs, n_obs, split, s, nullptr);
  else
    half_arc(c, th, -1.0, obs, n_obs, split - 1, s, nullptr);
  // both halves: partner lane glane ^ 8 holds the other half's sums
  double chi2 = s.chi2, g = s.g, A[kP];
  const double co = __shfl_xor_sync(gmask, chi2, 8);
  const double go = __shfl_xor_sync(gmask, g, 8);
  out.chi2 = half == 0 ? chi2 + co : co + chi2;
  g = half == 0 ? g + go : go + g;
  for (int b = 0; b < kP; ++b) {
    const double ao = __shfl_xor_sync(gmask, s.A[b], 8);
    A[b] = half == 0 ? s.A[b] + ao : ao + s.A[b];
  }
  // every lane gathers all rows from the group's first five lanes
  for (int a = 0; a < kP; ++a) {
    out.g[a] = __shfl_sync(gmask, g, gbase + a);
    for (int b = 0; b < kP; ++b) out.A[a][b] = __shfl_sync(gmask, A[b], gbase + a);
  }
}

// Levenberg-Marquardt from each start, one start per 16-lane group (the
// lanes share the work of every evaluation and take identical decisions):
// minimise chi^2(xi) with the step (A + lam diag A) delta = -g/2, A the
// Gauss-Newton matrix and g = d chi^2 / d xi
__global__ void __launch_bounds__(128)
    k_fit_lm_lanes(FitCfg c, const double* __restrict__ obs, int n_obs, int split,
                   const double* __restrict__ xi0, int count, int max_iter,
                   const double* __restrict__ bounds, double* __restrict__ xi_out,
                   double* __restrict__ chi2_out, int* __restrict__ iters_out) {
  const int lane = threadIdx.x & 31;
  const int glane = lane & 15;
  const unsigned gmask = 0xFFFFu << (lane & 16);
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;  // start
  if (t >= count) return;  // whole groups leave together (count is per group)
  double xi[kP], xn[kP], delta[kP], rhs[kP];
  for (int k = 0; k < kP; ++k) xi[k] = xi0[kP * t + k];
  Acc cur, trial;
  evaluate_lanes(c, obs, n_obs, split, xi, glane, gmask, cur);
  double lam = 1e-3;
  int it = 0;
  for (; it < max_iter; ++it) {
    for (int k = 0; k < kP; ++k) rhs[k] = -0.5 * cur.g[k];
    if (!damped_solve(cur.A, lam, rhs, delta)) {
      lam *= 10.0;
      if (lam > 1e12) break;
      continue;
    }
    double pred = 0.0;
    for (int k = 0; k < kP; ++k) pred -= 0.5 * cur.g[k] * delta[k];
    if (lam <= 1e-3 && pred < 1e-6) break;
    for (int k = 0; k < kP; ++k) {
      xn[k] = xi[k] + delta[k];
      if (bounds) xn[k] = fmin(fmax(xn[k], bounds[k]), bounds[kP + k]);
    }
    evaluate_lanes(c, obs, n_obs, split, xn, glane, gmask, trial);
    if (isfinite(trial.chi2) && trial.chi2 < cur.chi2) {
      const double drop = cur.chi2 - trial.chi2;
      for (int k = 0; k < kP; ++k) xi[k] = xn[k];
      cur = trial;
      lam = fmax(lam * 0.1, 1e-12);
      if (drop <= 1e-10 * cur.chi2 + 1e-300) break;
    } else {
      lam *= 10.0;
      if (lam > 1e12) break;
    }
  }
  if (glane == 0) {
    for (int k = 0; k < kP; ++k) xi_out[kP * t + k] = xi[k];
    chi2_out[t] = cur.chi2;
    iters_out[t] = it;
  }
}

// the model arc at one parameter vector (values only): forward and backward
// halves, each starting at t = 0
__global__ void k_fit_arc(FitCfg c, const double* __restrict__ xi, double* __restrict__ fwd,
                          double* __restrict__ bwd, int64_t* __restrict__ counts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  D5 th[kP];
  for (int k = 0; k < kP; ++k) th[k] = dconst<kP>(exp(xi[k]));
  Acc s;
  s.chi2 = 0.0;
  counts[0] = half_arc(c, th, 1.0, nullptr, 0, 0, s, fwd);
  counts[1] = half_arc(c, th, -1.0, nullptr, 0, -1, s, bwd);
}

void unit(const double* a, double* o) {
  const double r = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  for (int k = 0; k < 3; ++k) o[k] = a[k] / r;
}

void cross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

}  // namespace
}  // namespace nb

struct nbody_orbitfit {
  cudaStream_t s = nullptr;
  nb::FitCfg c{};
  int n_obs = 0, split = 0;
  double* obs = nullptr;  // sorted by phi1, [n_obs][5]
};

namespace {

int fit_alloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 8) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return NBODY_ENOMEM;
  }
  return NBODY_OK;
}

bool valid_theta(const double* th, int64_t count) {
  for (int64_t i = 0; i < count * nb::kP; ++i)
    if (!(th[i] > 0.0) || !std::isfinite(th[i])) return false;
  return true;
}

// xi = ln theta for count vectors, on the device
int upload_xi(nbody_orbitfit* h, const double* theta, int64_t count, double** dxi) {
  std::vector<double> xi((size_t)count * nb::kP);
  for (size_t i = 0; i < xi.size(); ++i) xi[i] = std::log(theta[i]);
  int rc = fit_alloc((void**)dxi, xi.size() * sizeof(double));
  if (rc) return rc;
  if (cudaMemcpyAsync(*dxi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice,
                      h->s) != cudaSuccess ||
      cudaStreamSynchronize(h->s) != cudaSuccess) {
    cudaFree(*dxi);
    *dxi = nullptr;
    return NBODY_ECUDA;
  }
  return NBODY_OK;
}

}  // namespace

extern "C" {

int nbody_orbitfit_create(nbody_orbitfit** out, const nbody_orbitfit_cfg* cfg, int64_t n_obs,
                          const double* obs, void* cuda_stream) {
  if (!out) return NBODY_EINVAL;
  *out = nullptr;
  if (!cfg || n_obs < 1 || n_obs > (1 << 20) || !obs) return NBODY_EINVAL;
  if (!(cfg->dt > 0.0) || !(cfg->t_max >= cfg->dt) || !(cfg->phi1_hi > cfg->phi1_lo) ||
      !(cfg->phi1_lo < 0.0 && cfg->phi1_hi > 0.0))
    return NBODY_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (!(cfg->sigma[k] > 0.0)) return NBODY_EINVAL;
  int dev = 0, maj = 0, min = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev) ||
      cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev)) {
    cudaGetLastError();
    return NBODY_ENODEV;
  }
  if (maj != 10 || min != 3) return NBODY_ENODEV;
  nb::FitCfg c{};
  c.G = cfg->G;
  double d[3], pole[3];
  for (int k = 0; k < 3; ++k) {
    c.X0[k] = cfg->X0[k];
    c.V0[k] = cfg->V0[k];
    c.xo[k] = cfg->observer[k];
    c.vo[k] = cfg->observer_vel[k];
    d[k] = cfg->X0[k] - cfg->observer[k];
  }
  nb::cross(d, cfg->V0, pole);
  if (!(pole[0] * pole[0] + pole[1] * pole[1] + pole[2] * pole[2] > 0.0)) return NBODY_EINVAL;
  nb::unit(d, c.e1);
  nb::unit(pole, c.nv);
  nb::cross(c.nv, c.e1, c.e2);
  c.lo = cfg->phi1_lo;
  c.hi = cfg->phi1_hi;
  c.dt = cfg->dt;
  c.nmax = (int64_t)std::llround(cfg->t_max / cfg->dt);
  for (int k = 0; k < 4; ++k) c.isig[k] = 1.0 / cfg->sigma[k];
  // observations sorted by phi1; split = first with phi1 >= 0 (forward side)
  std::vector<double> o(obs, obs + 5 * n_obs);
  std::vector<int> idx((size_t)n_obs);
  for (int i = 0; i < n_obs; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int a, int b) { return o[5 * a] < o[5 * b]; });
  std::vector<double> so((size_t)5 * n_obs);
  int split = (int)n_obs;
  for (int i = 0; i < n_obs; ++i) {
    for (int k = 0; k < 5; ++k) so[5 * i + k] = o[5 * idx[i] + k];
    if (!std::isfinite(so[5 * i])) return NBODY_EINVAL;
    if (split == (int)n_obs && so[5 * i] >= 0.0) split = i;
  }
  nbody_orbitfit* h = new (std::nothrow) nbody_orbitfit();
  if (!h) return NBODY_ENOMEM;
  h->s = (cudaStream_t)cuda_stream;
  h->c = c;
  h->n_obs = (int)n_obs;
  h->split = split;
  int rc = fit_alloc((void**)&h->obs, so.size() * sizeof(double));
  if (!rc && (cudaMemcpyAsync(h->obs, so.data(), so.size() * sizeof(double),
                              cudaMemcpyHostToDevice, h->s) != cudaSuccess ||
              cudaStreamSynchronize(h->s) != cudaSuccess))
    rc = NBODY_ECUDA;
  if (rc) {
    if (h->obs) cudaFree(h->obs);
    delete h;
    return rc;
  }
  *out = h;
  return NBODY_OK;
}

int nbody_orbitfit_eval(nbody_orbitfit* h, int64_t count, const double* theta, double* chi2,
                        double* grad, double* gn) {
  if (!h || count < 1 || count > (1 << 24) || !theta || !chi2) return NBODY_EINVAL;
  if (!valid_theta(theta, count)) return NBODY_EINVAL;
  double *dxi = nullptr, *dc = nullptr, *dg = nullptr, *da = nullptr;
  int rc = upload_xi(h, theta, count, &dxi);
  if (!rc) rc = fit_alloc((void**)&dc, (size_t)count * sizeof(double));
  if (!rc && grad) rc = fit_alloc((void**)&dg, (size_t)count * nb::kP * sizeof(double));
  if (!rc && gn) rc = fit_alloc((void**)&da, (size_t)count * 25 * sizeof(double));
  if (!rc) {
    nb::k_fit_eval<<<(unsigned)((count + 63) / 64), 64, 0, h->s>>>(
        h->c, h->obs, h->n_obs, h->split, dxi, (int)count, dc, dg, da);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  if (!rc && (cudaMemcpyAsync(chi2, dc, (size_t)count * sizeof(double), cudaMemcpyDefault,
                              h->s) ||
              (grad && cudaMemcpyAsync(grad, dg, (size_t)count * nb::kP * sizeof(double),
                                       cudaMemcpyDefault, h->s)) ||
              (gn && cudaMemcpyAsync(gn, da, (size_t)count * 25 * sizeof(double),
                                     cudaMemcpyDefault, h->s))))
    rc = NBODY_ECUDA;
  if (cudaStreamSynchronize(h->s) != cudaSuccess) rc = NBODY_ECUDA;
  if (dxi) cudaFree(dxi);
  if (dc) cudaFree(dc);
  if (dg) cudaFree(dg);
  if (da) cudaFree(da);
  return rc;
}

int nbody_orbitfit_lm(nbody_orbitfit* h, int64_t count, const double* theta0, int max_iter,
                      const double* theta_lo, const double* theta_hi, double* theta_out,
                      double* chi2_out, int* iters_out) {
  if (!h || count < 1 || count > (1 << 24) || !theta0 || !theta_out || !chi2_out ||
      max_iter < 1 || max_iter > 10000)
    return NBODY_EINVAL;
  if (!valid_theta(theta0, count)) return NBODY_EINVAL;
  if ((theta_lo == nullptr) != (theta_hi == nullptr)) return NBODY_EINVAL;
  double box[2 * nb::kP];
  if (theta_lo) {
    if (!valid_theta(theta_lo, 1) || !valid_theta(theta_hi, 1)) return NBODY_EINVAL;
    for (int k = 0; k < nb::kP; ++k) {
      if (!(theta_hi[k] >= theta_lo[k])) return NBODY_EINVAL;
      box[k] = std::log(theta_lo[k]);
      box[nb::kP + k] = std::log(theta_hi[k]);
    }
  }
  double *dxi = nullptr, *dxo = nullptr, *dc = nullptr, *dbox = nullptr;
  int* dit = nullptr;
  int rc = upload_xi(h, theta0, count, &dxi);
  if (!rc && theta_lo) {
    rc = fit_alloc((void**)&dbox, sizeof(box));
    if (!rc && (cudaMemcpyAsync(dbox, box, sizeof(box), cudaMemcpyHostToDevice, h->s) ||
                cudaStreamSynchronize(h->s)))
      rc = NBODY_ECUDA;
  }
  if (!rc) rc = fit_alloc((void**)&dxo, (size_t)count * nb::kP * sizeof(double));
  if (!rc) rc = fit_alloc((void**)&dc, (size_t)count * sizeof(double));
  if (!rc) rc = fit_alloc((void**)&dit, (size_t)count * sizeof(int));
  std::vector<double> xo((size_t)count * nb::kP);
  std::vector<int> its((size_t)count);
  if (!rc) {
    // 16 lanes per start, 8 starts per block of 128 threads
    nb::k_fit_lm_lanes<<<(unsigned)((count + 7) / 8), 128, 0, h->s>>>(
        h->c, h->obs, h->n_obs, h->split, dxi, (int)count, max_iter, dbox, dxo, dc, dit);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  if (!rc && (cudaMemcpyAsync(xo.data(), dxo, xo.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, h->s) ||
              cudaMemcpyAsync(chi2_out, dc, (size_t)count * sizeof(double), cudaMemcpyDefault,
                              h->s) ||
              cudaMemcpyAsync(its.data(), dit, its.size() * sizeof(int), cudaMemcpyDeviceToHost,
                              h->s)))
    rc = NBODY_ECUDA;
  if (cudaStreamSynchronize(h->s) != cudaSuccess) rc = NBODY_ECUDA;
  if (dxi) cudaFree(dxi);
  if (dxo) cudaFree(dxo);
  if (dc) cudaFree(dc);
  if (dit) cudaFree(dit);
  if (dbox) cudaFree(dbox);
  if (rc) return rc;
  for (size_t i = 0; i < xo.size(); ++i) theta_out[i] = std::exp(xo[i]);
  if (iters_out)
    for (int64_t i = 0; i < count; ++i) iters_out[i] = its[i];
  return NBODY_OK;
}

int nbody_orbitfit_fisher(nbody_orbitfit* h, const double* theta, double F[25],
                          double F_gn[25]) {
  if (!h || !theta || !F) return NBODY_EINVAL;
  if (!valid_theta(theta, 1)) return NBODY_EINVAL;
  const int nout = 1 + nb::kP + 2 * nb::kP * nb::kP;
  double *dxi = nullptr, *dout = nullptr;
  int rc = upload_xi(h, theta, 1, &dxi);
  if (!rc) rc = fit_alloc((void**)&dout, nout * sizeof(double));
  std::vector<double> o(nout);
  if (!rc) {
    nb::k_fit_hess<<<1, 32, 0, h->s>>>(h->c, h->obs, h->n_obs, h->split, dxi, dout);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  if (!rc && cudaMemcpyAsync(o.data(), dout, nout * sizeof(double), cudaMemcpyDeviceToHost,
                             h->s) != cudaSuccess)
    rc = NBODY_ECUDA;
  if (cudaStreamSynchronize(h->s) != cudaSuccess) rc = NBODY_ECUDA;
  if (dxi) cudaFree(dxi);
  if (dout) cudaFree(dout);
  if (rc) return rc;
  for (int q = 0; q < 25; ++q) {
    F[q] = 0.5 * o[1 + nb::kP + 25 + q];  // (1/2) d^2 chi^2 / d xi^2
    if (F_gn) F_gn[q] = o[1 + nb::kP + q];
  }
  return NBODY_OK;
}

int nbody_orbitfit_arc(nbody_orbitfit* h, const double* theta, int64_t max_pts, double* arc,
                       int64_t* n_pts) {
  if (!h || !theta || !arc || !n_pts || max_pts < 1) return NBODY_EINVAL;
  if (!valid_theta(theta, 1)) return NBODY_EINVAL;
  const int64_t cap = h->c.nmax + 1;
  double *dxi = nullptr, *fwd = nullptr, *bwd = nullptr;
  int64_t* cnt = nullptr;
  int rc = upload_xi(h, theta, 1, &dxi);
  if (!rc) rc = fit_alloc((void**)&fwd, (size_t)cap * 5 * sizeof(double));
  if (!rc) rc = fit_alloc((void**)&bwd, (size_t)cap * 5 * sizeof(double));
  if (!rc) rc = fit_alloc((void**)&cnt, 2 * sizeof(int64_t));
  std::vector<double> hf((size_t)cap * 5), hb((size_t)cap * 5);
  int64_t hc[2] = {0, 0};
  if (!rc) {
    nb::k_fit_arc<<<1, 32, 0, h->s>>>(h->c, dxi, fwd, bwd, cnt);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  if (!rc && (cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, h->s) ||
              cudaMemcpyAsync(hf.data(), fwd, hf.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, h->s) ||
              cudaMemcpyAsync(hb.data(), bwd, hb.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, h->s)))
    rc = NBODY_ECUDA;
  if (cudaStreamSynchronize(h->s) != cudaSuccess) rc = NBODY_ECUDA;
  if (dxi) cudaFree(dxi);
  if (fwd) cudaFree(fwd);
  if (bwd) cudaFree(bwd);
  if (cnt) cudaFree(cnt);
  if (rc) return rc;
  // increasing phi1: the backward half reversed, then the forward half
  const int64_t total = hc[1] + hc[0] - 1;
  *n_pts = total;
  if (total > max_pts) return NBODY_ESIZE;
  int64_t w = 0;
  for (int64_t i = hc[1] - 1; i >= 1; --i, ++w)
    for (int k = 0; k < 5; ++k) arc[5 * w + k] = hb[5 * i + k];
  for (int64_t i = 0; i < hc[0]; ++i, ++w)
    for (int k = 0; k < 5; ++k) arc[5 * w + k] = hf[5 * i + k];
  return NBODY_OK;
}

void nbody_orbitfit_destroy(nbody_orbitfit* h) {
  if (!h) return;
  cudaStreamSynchronize(h->s);
  if (h->obs) cudaFree(h->obs);
  delete h;
}

}  // extern "C"
