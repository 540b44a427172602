// stream.cu -- the mock-stream pipeline of the paper's inference (Fig. 2,
// Sec. 2.2.1) and its discrete adjoint (Sec. 2), on the GPU:
//
//   backward orbit of the progenitor centre (1 particle, NFW + MN)  k_orbit
//   Plummer scale-and-shift to the recovered phase-space point      k_ic
//   n-body forward run (pair forces + potential, KDK)               nbody_integrate
//   projection to (phi1, phi2), soft 2-D histogram, squared error   k_head_weights,
//                                                                   k_hist, k_loss
// and in reverse: k_head_vjp -> nbody_vjp -> k_ic_vjp -> k_orbit_vjp ->
// k_theta_bar.  All arithmetic is FP64 (the n-body pair sums are the FP32
// kernels behind nbody_integrate / nbody_vjp); every reduction has a fixed
// order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "block_reduce.cuh"
#include "ext_potential.cuh"
#include "nbody_internal.cuh"

namespace {

using nb::DevParams;
using nb::ExtUnit;

constexpr int kMaxBins = 64;

struct HeadGeom {
  double obs[3], e1[3], e2[3], nv[3];
  double lo1, h1, lo2, h2;  // bin edges lo + b h
  int nb1, nb2;
};

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ------------------------------------------------------------------ orbit
// single particle, external potential only: v += dt/2 a; x += dt v;
// v += dt/2 a.  Stores x_0..x_n and the half-step velocities.
__global__ void k_orbit(DevParams P, double X0, double X1, double X2,
                        double V0, double V1, double V2, int64_t ns,
                        double* __restrict__ ox, double* __restrict__ ovh,
                        double* __restrict__ g6) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double x[3] = {X0, X1, X2}, v[3] = {V0, V1, V2};
  ExtUnit e;
  nb::ext_unit(P, x[0], x[1], x[2], e);
  for (int d = 0; d < 3; ++d) ox[d] = x[d];
  for (int64_t k = 0; k < ns; ++k) {
    for (int d = 0; d < 3; ++d) {
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
      ovh[3 * k + d] = v[d];
      x[d] += P.dt * v[d];
      ox[3 * (k + 1) + d] = x[d];
    }
    nb::ext_unit(P, x[0], x[1], x[2], e);
    for (int d = 0; d < 3; ++d)
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
  }
  for (int d = 0; d < 3; ++d) {
    g6[d] = x[d];
    g6[3 + d] = v[d];
  }
}

// Backward orbits of many parameter vectors at once, one thread each (the
// arithmetic of k_orbit without the stored trajectory): theta_b = (t_end,
// M_prog, M_NFW, M_MN) -> g6[b] = (X, V) after ns steps of -t_end/ns.
__global__ void k_orbit_batch(DevParams P0, double X0, double X1, double X2, double V0,
                              double V1, double V2, int64_t ns,
                              const double* __restrict__ theta, int64_t count,
                              double* __restrict__ g6) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  DevParams P = P0;
  P.dt = -theta[4 * b] / (double)ns;
  P.nfw_GM = P0.G * theta[4 * b + 2];
  P.mn_GM = P0.G * theta[4 * b + 3];
  double x[3] = {X0, X1, X2}, v[3] = {V0, V1, V2};
  ExtUnit e;
  nb::ext_unit(P, x[0], x[1], x[2], e);
  for (int64_t k = 0; k < ns; ++k) {
    for (int d = 0; d < 3; ++d) {
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
      x[d] += P.dt * v[d];
    }
    nb::ext_unit(P, x[0], x[1], x[2], e);
    for (int d = 0; d < 3; ++d)
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
  }
  for (int d = 0; d < 3; ++d) {
    g6[6 * b + d] = x[d];
    g6[6 * b + 3 + d] = v[d];
  }
}

// Plummer spheres of many parameter vectors: member b's particle i is
// column b n + i of x0, v0 (3 x count n) and element b n + i of m.
__global__ void k_ic_batch(const double* __restrict__ xh, const double* __restrict__ vh,
                           const double* __restrict__ g6, const double* __restrict__ theta,
                           double a, double G, int64_t n, int64_t count,
                           double* __restrict__ x0, double* __restrict__ v0,
                           double* __restrict__ m) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n * count) return;
  const int64_t b = k / n, i = k - b * n, ld = n * count;
  const double M = theta[4 * b + 1];
  const double vscale = sqrt(G * M / a);
  for (int d = 0; d < 3; ++d) {
    x0[d * ld + k] = a * xh[d * n + i] + g6[6 * b + d];
    v0[d * ld + k] = vscale * vh[d * n + i] + g6[6 * b + 3 + d];
  }
  m[k] = M / (double)n;
}

// adjoint of one half kick v' = v + (dt/2) a(x) with cotangent vb = vbar'
__device__ __forceinline__ void orbit_kick_adj(const DevParams& P,
                                               const double* x,
                                               const double* vb, double* xb,
                                               double* acc3) {
  ExtUnit e;
  nb::ext_unit(P, x[0], x[1], x[2], e);
  double jl[3];
  nb::ext_jvp(P, x[0], x[1], x[2], vb, jl);
  double ln = 0.0, lm = 0.0;
  for (int d = 0; d < 3; ++d) {
    xb[d] += 0.5 * P.dt * jl[d];
    ln += vb[d] * e.n[d];
    lm += vb[d] * e.d[d];
  }
  acc3[0] += 0.5 * (P.nfw_GM * ln + P.mn_GM * lm);  // d/d dt
  acc3[1] += 0.5 * P.dt * P.G * ln;                  // d/d M_NFW
  acc3[2] += 0.5 * P.dt * P.G * lm;                  // d/d M_MN
}

// reverse of k_orbit from cotangents (Xbar, Vbar) of its final state:
// out = { dL/d dt_orbit, dL/d M_NFW, dL/d M_MN } (orbit part)
__global__ void k_orbit_vjp(DevParams P, const double* __restrict__ ox,
                            const double* __restrict__ ovh, int64_t ns,
                            const double* __restrict__ cot,
                            double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double xb[3] = {cot[0], cot[1], cot[2]};
  double vb[3] = {cot[3], cot[4], cot[5]};
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t k = ns - 1; k >= 0; --k) {
    orbit_kick_adj(P, &ox[3 * (k + 1)], vb, xb, acc);  // closing kick
    for (int d = 0; d < 3; ++d) acc[0] += xb[d] * ovh[3 * k + d];
    for (int d = 0; d < 3; ++d) vb[d] += P.dt * xb[d];   // drift
    orbit_kick_adj(P, &ox[3 * k], vb, xb, acc);         // opening kick
  }
  out[0] = acc[0];
  out[1] = acc[1];
  out[2] = acc[2];
}

// ---------------------------------------------------------- Plummer shift
__global__ void k_ic(const double* __restrict__ xh, const double* __restrict__ vh,
                     const double* __restrict__ g6, double a, double vscale,
                     double mass, int64_t n, double* __restrict__ x0,
                     double* __restrict__ v0, double* __restrict__ m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < 3; ++d) {
    x0[d * n + i] = a * xh[d * n + i] + g6[d];
    v0[d * n + i] = vscale * vh[d * n + i] + g6[3 + d];
  }
  m[i] = mass;
}

// sums of x0bar, v0bar and of v0bar . vhat
__global__ void __launch_bounds__(256)
    k_ic_vjp(const double* __restrict__ x0b, const double* __restrict__ v0b,
             const double* __restrict__ vh, int64_t n, double* __restrict__ blk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double val[7] = {0, 0, 0, 0, 0, 0, 0};
  if (i < n) {
    for (int d = 0; d < 3; ++d) {
      val[d] = x0b[d * n + i];
      val[3 + d] = v0b[d * n + i];
      val[6] += v0b[d * n + i] * vh[d * n + i];
    }
  }
  nb::block_accumulate<7>(val, blk);
}

// ------------------------------------------------------------------- head
__global__ void k_head_weights(HeadGeom g, const double* __restrict__ x,
                               int64_t n, double* __restrict__ phi,
                               double* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = x[k * n + i] - g.obs[k];
  const double p1 = dot3(d, g.e1), p2 = dot3(d, g.e2), p3 = dot3(d, g.nv);
  const double r = sqrt(dot3(d, d));
  const double f1 = atan2(p2, p1);
  const double f2 = asin(p3 / r);
  phi[i] = f1;
  phi[n + i] = f2;
  const int nbt = g.nb1 + g.nb2;
  const double s1 = 0.5 * g.h1, s2 = 0.5 * g.h2;
  double c_prev = normcdf((g.lo1 - f1) / s1);
  for (int b = 0; b < g.nb1; ++b) {
    const double c = normcdf((g.lo1 + (b + 1) * g.h1 - f1) / s1);
    w[i * nbt + b] = c - c_prev;
    c_prev = c;
  }
  c_prev = normcdf((g.lo2 - f2) / s2);
  for (int b = 0; b < g.nb2; ++b) {
    const double c = normcdf((g.lo2 + (b + 1) * g.h2 - f2) / s2);
    w[i * nbt + g.nb1 + b] = c - c_prev;
    c_prev = c;
  }
}

// rho[b1][b2] = (1/n) sum_i w1[i][b1] w2[i][b2]; one block per b1
__global__ void __launch_bounds__(256)
    k_hist(const double* __restrict__ w, int64_t n, int nb1, int nb2,
           double* __restrict__ rho) {
  __shared__ double sh[8][32];
  const int b1 = blockIdx.x;
  const int nbt = nb1 + nb2;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nb2; c0 += 32) {
    double acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) {
      const double w1 = w[i * nbt + b1];
      const double* w2 = &w[i * nbt + nb1 + c0];
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (c0 + k < nb2) acc[k] += w1 * w2[k];
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      double v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[wp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32 && c0 + (int)threadIdx.x < nb2) {
      double s = 0.0;
      for (int q = 0; q < 8; ++q) s += sh[q][threadIdx.x];
      rho[b1 * nb2 + c0 + threadIdx.x] = s / (double)n;
    }
    __syncthreads();
  }
}

// L = mean (rho - t)^2 and rbar = dL/drho (one block of 256)
__global__ void __launch_bounds__(256)
    k_loss(const double* __restrict__ rho, const double* __restrict__ t, int nb,
           double* __restrict__ loss, double* __restrict__ rbar) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) {
    const double d = rho[b] - t[b];
    s += d * d;
    rbar[b] = 2.0 * d / (double)nb;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = sh[0] / (double)nb;
}

__device__ __forceinline__ double npdf(double z) {
  return 0.3989422804014327 * exp(-0.5 * z * z);
}

// per particle: phi-bar from rbar, then x-bar through the projection
__global__ void __launch_bounds__(256)
    k_head_vjp(HeadGeom g, const double* __restrict__ x,
               const double* __restrict__ phi, const double* __restrict__ w,
               const double* __restrict__ rbar, int64_t n,
               double* __restrict__ xbar) {
  __shared__ double sr[kMaxBins * kMaxBins];
  const int nb1 = g.nb1, nb2 = g.nb2, nbt = nb1 + nb2;
  for (int k = threadIdx.x; k < nb1 * nb2; k += blockDim.x) sr[k] = rbar[k];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double f1 = phi[i], f2 = phi[n + i];
  const double s1 = 0.5 * g.h1, s2 = 0.5 * g.h2;
  const double* wi = &w[i * nbt];
  // g1 = (1/n) sum_b1 dw1[b1] sum_b2 rbar[b1][b2] w2[b2],
  // dw1[b] = -(pdf(z_{b+1}) - pdf(z_b)) / s1
  double g1 = 0.0;
  double p_prev = npdf((g.lo1 - f1) / s1);
  for (int b1 = 0; b1 < nb1; ++b1) {
    const double p = npdf((g.lo1 + (b1 + 1) * g.h1 - f1) / s1);
    const double dw = -(p - p_prev) / s1;
    p_prev = p;
    double t = 0.0;
    for (int b2 = 0; b2 < nb2; ++b2) t += sr[b1 * nb2 + b2] * wi[nb1 + b2];
    g1 += dw * t;
  }
  double g2 = 0.0;
  p_prev = npdf((g.lo2 - f2) / s2);
  for (int b2 = 0; b2 < nb2; ++b2) {
    const double p = npdf((g.lo2 + (b2 + 1) * g.h2 - f2) / s2);
    const double dw = -(p - p_prev) / s2;
    p_prev = p;
    double t = 0.0;
    for (int b1 = 0; b1 < nb1; ++b1) t += sr[b1 * nb2 + b2] * wi[b1];
    g2 += dw * t;
  }
  g1 /= (double)n;
  g2 /= (double)n;
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = x[k * n + i] - g.obs[k];
  const double p1 = dot3(d, g.e1), p2 = dot3(d, g.e2), p3 = dot3(d, g.nv);
  const double q2 = p1 * p1 + p2 * p2;
  const double r2 = dot3(d, d);
  const double den = r2 * sqrt(r2 - p3 * p3);
  for (int k = 0; k < 3; ++k) {
    const double dphi1 = (p1 * g.e2[k] - p2 * g.e1[k]) / q2;
    const double dphi2 = (g.nv[k] * r2 - p3 * d[k]) / den;
    xbar[k * n + i] = g1 * dphi1 + g2 * dphi2;
  }
}

__global__ void k_theta_bar(double tb0, double tb1, double tb2, double tb3,
                            int64_t ns, double G, double a, double M,
                            const double* __restrict__ red,
                            const double* __restrict__ orb,
                            double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // t_end: dt = t/n in the n-body run, dt_b = -t/n in the orbit
  out[0] = tb0 / (double)ns - orb[0] / (double)ns;
  // M_Plummer: v = sqrt(G M / a) vhat + V and m_j = M / n
  out[1] = 0.5 * sqrt(G / (a * M)) * red[6] + tb1 / M;
  out[2] = tb2 + orb[1];
  out[3] = tb3 + orb[2];
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------- batched pipeline
// orbit parameters of member b: theta_b = (t_end, M_prog, M_NFW, M_MN)
__device__ __forceinline__ DevParams member_orbit_params(const DevParams& P0,
                                                         const double* theta, int64_t ns) {
  DevParams P = P0;
  P.dt = -theta[0] / (double)ns;
  P.nfw_GM = P0.G * theta[2];
  P.mn_GM = P0.G * theta[3];
  return P;
}

// backward orbits of every member, one thread each, with the trajectory
// stored (the arithmetic of k_orbit): member b's x_0..x_ns at
// ox + b 3 (ns + 1), half-step velocities at ovh + b 3 ns, end point g6[b]
__global__ void k_orbit_batch_tape(DevParams P0, double X0, double X1, double X2, double V0,
                                   double V1, double V2, int64_t ns,
                                   const double* __restrict__ theta, int64_t count,
                                   double* __restrict__ ox, double* __restrict__ ovh,
                                   double* __restrict__ g6) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const DevParams P = member_orbit_params(P0, theta + 4 * b, ns);
  double* xo = ox + b * 3 * (ns + 1);
  double* vo = ovh + b * 3 * ns;
  double x[3] = {X0, X1, X2}, v[3] = {V0, V1, V2};
  ExtUnit e;
  nb::ext_unit(P, x[0], x[1], x[2], e);
  for (int d = 0; d < 3; ++d) xo[d] = x[d];
  for (int64_t k = 0; k < ns; ++k) {
    for (int d = 0; d < 3; ++d) {
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
      vo[3 * k + d] = v[d];
      x[d] += P.dt * v[d];
      xo[3 * (k + 1) + d] = x[d];
    }
    nb::ext_unit(P, x[0], x[1], x[2], e);
    for (int d = 0; d < 3; ++d)
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
  }
  for (int d = 0; d < 3; ++d) {
    g6[6 * b + d] = x[d];
    g6[6 * b + 3 + d] = v[d];
  }
}

// per member b (one block each): sums of x0bar, v0bar and of v0bar . vhat
// over its particles (columns b n .. of 3 x count n) into red[b][0..6]
__global__ void __launch_bounds__(256)
    k_ic_vjp_batch(const double* __restrict__ x0b, const double* __restrict__ v0b,
                   const double* __restrict__ vh, int64_t n, int64_t count,
                   double* __restrict__ red) {
  const int64_t b = blockIdx.x, ld = n * count;
  double val[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      val[d] += x0b[d * ld + b * n + i];
      val[3 + d] += v0b[d * ld + b * n + i];
      val[6] += v0b[d * ld + b * n + i] * vh[d * n + i];
    }
  nb::block_accumulate<7>(val, red);
}

// reverse of every member's backward orbit (the arithmetic of k_orbit_vjp)
// from the cotangents red[b][0..5] of its end point: orb[b] = (dL/d dt_orbit,
// dL/dM_NFW, dL/dM_MN), orbit part
__global__ void k_orbit_vjp_batch(DevParams P0, const double* __restrict__ ox,
                                  const double* __restrict__ ovh, int64_t ns,
                                  const double* __restrict__ theta, int64_t count,
                                  const double* __restrict__ red, double* __restrict__ orb) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const DevParams P = member_orbit_params(P0, theta + 4 * b, ns);
  const double* xo = ox + b * 3 * (ns + 1);
  const double* vo = ovh + b * 3 * ns;
  const double* cot = red + 7 * b;
  double xb[3] = {cot[0], cot[1], cot[2]};
  double vb[3] = {cot[3], cot[4], cot[5]};
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t k = ns - 1; k >= 0; --k) {
    orbit_kick_adj(P, &xo[3 * (k + 1)], vb, xb, acc);  // closing kick
    for (int d = 0; d < 3; ++d) acc[0] += xb[d] * vo[3 * k + d];
    for (int d = 0; d < 3; ++d) vb[d] += P.dt * xb[d];  // drift
    orbit_kick_adj(P, &xo[3 * k], vb, xb, acc);        // opening kick
  }
  for (int q = 0; q < 3; ++q) orb[3 * b + q] = acc[q];
}

// dL/dtheta of every member (the arithmetic of k_theta_bar) from its n-body
// parameter gradient tb[b][0..3] (dt, mass scale, M_NFW, M_MN), its
// initial-state sums red[b] and its orbit part orb[b]
// (every component is the sum of two separately computed parts, kept in
// parts[b][0..3] and parts[b][4..7]: the n-body run's and the backward
// orbit's for t_end, M_NFW and M_MN; the velocity scaling's and the masses'
// for M_Plummer)
__global__ void k_theta_bar_batch(const double* __restrict__ tb, int64_t ns, double G,
                                  double a, const double* __restrict__ theta, int64_t count,
                                  const double* __restrict__ red,
                                  const double* __restrict__ orb, double* __restrict__ out,
                                  double* __restrict__ parts) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const double* t = tb + 8 * b;
  const double M = theta[4 * b + 1];
  const double p1[4] = {t[0] / (double)ns, 0.5 * sqrt(G / (a * M)) * red[7 * b + 6], t[2],
                        t[3]};
  const double p2[4] = {-orb[3 * b] / (double)ns, t[1] / M, orb[3 * b + 1], orb[3 * b + 2]};
  for (int q = 0; q < 4; ++q) {
    out[4 * b + q] = p1[q] + p2[q];
    parts[8 * b + q] = p1[q];
    parts[8 * b + 4 + q] = p2[q];
  }
}

// members whose loss or gradient is not finite (their run left the finite
// range): loss +inf and gradient NaN, the other members untouched
__global__ void k_mark_failed_batch(double* __restrict__ loss, double* __restrict__ out,
                                    int64_t count, unsigned* __restrict__ nmark) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  bool bad = !isfinite(loss[b]);
  if (out)
    for (int q = 0; q < 4; ++q) bad |= !isfinite(out[4 * b + q]);
  if (!bad) return;
  atomicAdd(nmark, 1u);
  loss[b] = INFINITY;
  if (out)
    for (int q = 0; q < 4; ++q) out[4 * b + q] = NAN;
}

}  // namespace

struct nbody_stream {
  nbody_stream_cfg cfg{};
  cudaStream_t s = nullptr;
  int64_t n = 0, nb = 0;
  nbody_ctx* ctx = nullptr;
  HeadGeom geom{};
  double *xhat = nullptr, *vhat = nullptr;
  double *x0 = nullptr, *v0 = nullptr, *m = nullptr, *xT = nullptr;
  double *ox = nullptr, *ovh = nullptr, *g6 = nullptr;
  double *phi = nullptr, *w = nullptr;
  double *rho = nullptr, *target = nullptr, *rbar = nullptr, *loss = nullptr;
  double *xbar = nullptr, *x0bar = nullptr, *v0bar = nullptr;
  double *vT = nullptr, *vbar = nullptr;  // the point-cloud (MMD) head
  nbody_mmd* mmd = nullptr;               // set: the loss is MMD^2 to a cloud
  double *blk = nullptr, *red = nullptr, *orb = nullptr, *tbar = nullptr;
  int nblk = 0;
  double theta[4] = {0, 0, 0, 0};
  bool have_forward = false;
};

// The pipeline for `count` parameter vectors at once (the gradient
// refinement of many grid points or bootstrap realisations, Sec. 2.2.1):
// one batch context of count members of n particles, each member scored by
// MMD^2 against its own target cloud.
struct nbody_stream_batch {
  nbody_stream_cfg cfg{};
  cudaStream_t s = nullptr;
  int64_t n = 0, count = 0;
  nbody_ctx* ctx = nullptr;   // batch of count members, trajectories recorded
  nbody_mmd* mmd = nullptr;   // one target per member
  bool tuned = false;
  double *xhat = nullptr, *vhat = nullptr, *theta = nullptr;
  double *x0 = nullptr, *v0 = nullptr, *m = nullptr, *xT = nullptr, *vT = nullptr;
  double *xbar = nullptr, *vbar = nullptr, *x0bar = nullptr, *v0bar = nullptr;
  double *ox = nullptr, *ovh = nullptr, *g6 = nullptr;
  double *loss = nullptr, *tb = nullptr, *red = nullptr, *orb = nullptr, *out = nullptr;
  unsigned* nmark = nullptr;  // members marked failed by the last call
  double* parts = nullptr;    // [count][8] the gradient's two parts per component
  bool have_parts = false;
};

namespace {

#define SCK(call)                              \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return NBODY_ECUDA; \
  } while (0)

template <class T>
int salloc(T** p, size_t count) {
  if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return NBODY_ENOMEM;
  }
  return NBODY_OK;
}

template <class T>
void sfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_stream(nbody_stream* s) {
  if (s->ctx) nbody_destroy(s->ctx);
  s->ctx = nullptr;
  if (s->mmd) nbody_mmd_destroy(s->mmd);
  s->mmd = nullptr;
  sfree(s->vT); sfree(s->vbar);
  sfree(s->xhat); sfree(s->vhat); sfree(s->x0); sfree(s->v0); sfree(s->m);
  sfree(s->xT); sfree(s->ox); sfree(s->ovh); sfree(s->g6); sfree(s->phi);
  sfree(s->w); sfree(s->rho); sfree(s->target); sfree(s->rbar); sfree(s->loss);
  sfree(s->xbar); sfree(s->x0bar); sfree(s->v0bar); sfree(s->blk); sfree(s->red);
  sfree(s->orb); sfree(s->tbar);
}

void free_stream_batch(nbody_stream_batch* s) {
  if (s->ctx) nbody_destroy(s->ctx);
  if (s->mmd) nbody_mmd_destroy(s->mmd);
  for (double** p : {&s->xhat, &s->vhat, &s->theta, &s->x0, &s->v0, &s->m, &s->xT, &s->vT,
                     &s->xbar, &s->vbar, &s->x0bar, &s->v0bar, &s->ox, &s->ovh, &s->g6,
                     &s->loss, &s->tb, &s->red, &s->orb, &s->out})
    sfree(*p);
  sfree(s->nmark);
  sfree(s->parts);
}

void unit3(const double* a, double* out) {
  const double r = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  for (int k = 0; k < 3; ++k) out[k] = a[k] / r;
}

void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

DevParams orbit_params(const nbody_stream* s) {
  DevParams P{};
  P.G = s->cfg.G;
  P.dt = -s->theta[0] / (double)s->cfg.n_steps;
  P.ext = NBODY_EXT_NFW | NBODY_EXT_MN;
  P.nfw_GM = s->cfg.G * s->theta[2];
  P.nfw_rs = s->cfg.nfw_rs;
  P.mn_GM = s->cfg.G * s->theta[3];
  P.mn_a = s->cfg.mn_a;
  P.mn_b = s->cfg.mn_b;
  return P;
}

}  // namespace

extern "C" {

int nbody_stream_create(nbody_stream** out, const nbody_stream_cfg* cfg,
                        const double* xhat, const double* vhat,
                        void* cuda_stream) {
  if (!out || !cfg || !xhat || !vhat) return NBODY_EINVAL;
  *out = nullptr;
  const nbody_stream_cfg& c = *cfg;
  if (c.n < 1 || c.n_steps < 1 || c.checkpoint_every < 1 || !(c.eps > 0.0) ||
      !(c.a_prog > 0.0) || !(c.nfw_rs > 0.0) || c.mn_a < 0.0 || c.mn_b < 0.0 ||
      c.nb1 < 1 || c.nb2 < 1 || c.nb1 > kMaxBins || c.nb2 > kMaxBins ||
      !(c.phi1_hi > c.phi1_lo) || !(c.phi2_hi > c.phi2_lo))
    return NBODY_EINVAL;
  double d[3] = {c.X0[0] - c.observer[0], c.X0[1] - c.observer[1],
                 c.X0[2] - c.observer[2]};
  double pole[3];
  cross3(d, c.V0, pole);
  if (!(pole[0] * pole[0] + pole[1] * pole[1] + pole[2] * pole[2] > 0.0))
    return NBODY_EINVAL;
  nbody_stream* s = new (std::nothrow) nbody_stream();
  if (!s) return NBODY_ENOMEM;
  s->cfg = c;
  s->s = (cudaStream_t)cuda_stream;
  s->n = c.n;
  s->nb = (int64_t)c.nb1 * c.nb2;
  HeadGeom& g = s->geom;
  for (int k = 0; k < 3; ++k) g.obs[k] = c.observer[k];
  unit3(d, g.e1);
  unit3(pole, g.nv);
  cross3(g.nv, g.e1, g.e2);
  g.lo1 = c.phi1_lo;
  g.h1 = (c.phi1_hi - c.phi1_lo) / c.nb1;
  g.lo2 = c.phi2_lo;
  g.h2 = (c.phi2_hi - c.phi2_lo) / c.nb2;
  g.nb1 = c.nb1;
  g.nb2 = c.nb2;

  nbody_params p{};
  p.G = c.G;
  p.eps = c.eps;
  p.dt = 1.0;
  p.checkpoint_every = c.checkpoint_every;
  p.ext_flags = NBODY_EXT_NFW | NBODY_EXT_MN;
  p.center_mode = NBODY_CENTER_GUIDE;
  p.nfw_M = 0.0;
  p.nfw_rs = c.nfw_rs;
  p.mn_a = c.mn_a;
  p.mn_b = c.mn_b;
  int rc = nbody_create(&s->ctx, c.n, &p, cuda_stream);
  const size_t n3 = (size_t)3 * c.n;
  const size_t ns = (size_t)c.n_steps;
  s->nblk = (int)blocks_for(c.n, 256);
  if (rc || (rc = salloc(&s->xhat, n3)) || (rc = salloc(&s->vhat, n3)) ||
      (rc = salloc(&s->x0, n3)) || (rc = salloc(&s->v0, n3)) ||
      (rc = salloc(&s->m, (size_t)c.n)) || (rc = salloc(&s->xT, n3)) ||
      (rc = salloc(&s->vT, n3)) || (rc = salloc(&s->vbar, n3)) ||
      (rc = salloc(&s->ox, 3 * (ns + 1))) || (rc = salloc(&s->ovh, 3 * ns)) ||
      (rc = salloc(&s->g6, 6)) || (rc = salloc(&s->phi, 2 * (size_t)c.n)) ||
      (rc = salloc(&s->w, (size_t)c.n * (c.nb1 + c.nb2))) ||
      (rc = salloc(&s->rho, (size_t)s->nb)) || (rc = salloc(&s->target, (size_t)s->nb)) ||
      (rc = salloc(&s->rbar, (size_t)s->nb)) || (rc = salloc(&s->loss, 1)) ||
      (rc = salloc(&s->xbar, n3)) || (rc = salloc(&s->x0bar, n3)) ||
      (rc = salloc(&s->v0bar, n3)) || (rc = salloc(&s->blk, (size_t)s->nblk * 7)) ||
      (rc = salloc(&s->red, 8)) || (rc = salloc(&s->orb, 3)) ||
      (rc = salloc(&s->tbar, 4))) {
    free_stream(s);
    delete s;
    return rc ? rc : NBODY_ENOMEM;
  }
  if (cudaMemcpyAsync(s->xhat, xhat, n3 * sizeof(double), cudaMemcpyDefault, s->s) ||
      cudaMemcpyAsync(s->vhat, vhat, n3 * sizeof(double), cudaMemcpyDefault, s->s) ||
      cudaMemsetAsync(s->target, 0, (size_t)s->nb * sizeof(double), s->s) ||
      cudaStreamSynchronize(s->s)) {
    free_stream(s);
    delete s;
    return NBODY_ECUDA;
  }
  *out = s;
  return NBODY_OK;
}

int nbody_stream_initial_state(nbody_stream* s, const double theta[4], double* x0,
                               double* v0, double* m, double com[6]) {
  if (!s || !theta || !x0 || !v0 || !m) return NBODY_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (!(theta[k] > 0.0) || !std::isfinite(theta[k])) return NBODY_EINVAL;
  // the orbit helpers read s->theta; keep the recorded forward unchanged
  double keep[4];
  for (int k = 0; k < 4; ++k) {
    keep[k] = s->theta[k];
    s->theta[k] = theta[k];
  }
  const nbody_stream_cfg& c = s->cfg;
  const DevParams P = orbit_params(s);
  for (int k = 0; k < 4; ++k) s->theta[k] = keep[k];
  const int64_t n = s->n;
  // private orbit buffers would be wasteful: the orbit of this call goes to
  // the pipeline's own buffers only when no forward is recorded
  double* ox = s->ox;
  double* ovh = s->ovh;
  double* g6 = s->g6;
  double* tmp = nullptr;
  if (s->have_forward) {
    const size_t need = 3 * (size_t)(2 * c.n_steps + 1) + 6;
    if (cudaMalloc((void**)&tmp, need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return NBODY_ENOMEM;
    }
    ox = tmp;
    ovh = tmp + 3 * (c.n_steps + 1);
    g6 = ovh + 3 * c.n_steps;
  }
  k_orbit<<<1, 32, 0, s->s>>>(P, c.X0[0], c.X0[1], c.X0[2], c.V0[0], c.V0[1], c.V0[2],
                              c.n_steps, ox, ovh, g6);
  nb::count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_ic<<<blocks_for(n, 256), 256, 0, s->s>>>(s->xhat, s->vhat, g6, c.a_prog,
                                               std::sqrt(c.G * theta[1] / c.a_prog),
                                               theta[1] / (double)n, n, x0, v0, m);
    nb::count_launch();
    e = cudaGetLastError();
  }
  double h6[6];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h6, g6, sizeof(h6), cudaMemcpyDeviceToHost, s->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->s);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return NBODY_ECUDA;
  if (com)
    for (int k = 0; k < 6; ++k) com[k] = h6[k];
  return NBODY_OK;
}

int nbody_stream_initial_states(nbody_stream* s, int64_t count, const double* thetas,
                                double* x0, double* v0, double* m, double* com) {
  if (!s || count < 1 || !thetas || !x0 || !v0 || !m) return NBODY_EINVAL;
  const nbody_stream_cfg& c = s->cfg;
  const int64_t n = s->n;
  std::vector<double> th((size_t)count * 4);
  if (cudaMemcpy(th.data(), thetas, th.size() * sizeof(double), cudaMemcpyDefault) !=
      cudaSuccess)
    return NBODY_ECUDA;
  for (double t : th)
    if (!(t > 0.0) || !std::isfinite(t)) return NBODY_EINVAL;
  double* dth = nullptr;
  double* g6 = nullptr;
  int rc = salloc(&dth, th.size());
  if (!rc) rc = salloc(&g6, (size_t)count * 6);
  cudaError_t e = cudaSuccess;
  if (!rc) {
    e = cudaMemcpyAsync(dth, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice,
                        s->s);
    DevParams P{};
    P.G = c.G;
    P.ext = NBODY_EXT_NFW | NBODY_EXT_MN;
    P.nfw_rs = c.nfw_rs;
    P.mn_a = c.mn_a;
    P.mn_b = c.mn_b;
    if (e == cudaSuccess) {
      k_orbit_batch<<<blocks_for(count, 64), 64, 0, s->s>>>(P, c.X0[0], c.X0[1], c.X0[2],
                                                             c.V0[0], c.V0[1], c.V0[2],
                                                             c.n_steps, dth, count, g6);
      nb::count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_ic_batch<<<blocks_for(n * count, 256), 256, 0, s->s>>>(s->xhat, s->vhat, g6, dth,
                                                               c.a_prog, c.G, n, count, x0,
                                                               v0, m);
      nb::count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && com)
      e = cudaMemcpyAsync(com, g6, (size_t)count * 6 * sizeof(double), cudaMemcpyDefault, s->s);
    if (cudaStreamSynchronize(s->s) != cudaSuccess) e = cudaErrorUnknown;
  }
  sfree(dth);
  sfree(g6);
  if (rc) return rc;
  return e == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}

int nbody_stream_autotune(nbody_stream* s, const double theta[4], int probe_launches) {
  if (!s || !theta || probe_launches < 1) return NBODY_EINVAL;
  double com[6];
  int rc = nbody_stream_initial_state(s, theta, s->x0, s->v0, s->m, com);
  if (rc) return rc;
  const nbody_stream_cfg& c = s->cfg;
  nbody_params p{};
  p.G = c.G;
  p.eps = c.eps;
  p.dt = theta[0] / (double)c.n_steps;
  p.ext_flags = NBODY_EXT_NFW | NBODY_EXT_MN;
  p.center_mode = NBODY_CENTER_FIXED;
  p.nfw_M = theta[2];
  p.nfw_rs = c.nfw_rs;
  p.mn_M = theta[3];
  p.mn_a = c.mn_a;
  p.mn_b = c.mn_b;
  for (int k = 0; k < 3; ++k) p.center[k] = com[k];
  s->have_forward = false;
  if ((rc = nbody_set_params(s->ctx, &p))) return rc;
  if ((rc = nbody_set_state(s->ctx, s->x0, s->v0, s->m))) return rc;
  return nbody_autotune_pair(s->ctx, probe_launches, nullptr, nullptr);
}

int nbody_stream_get_pair_shape(nbody_stream* s, int vjp, int out[4]) {
  if (!s || !out) return NBODY_EINVAL;
  return nbody_get_pair_shape(s->ctx, vjp, out);
}

int nbody_stream_head(nbody_stream* s, const double* x, double* density, double* loss) {
  if (!s || !x || !density) return NBODY_EINVAL;
  const nbody_stream_cfg& c = s->cfg;
  const int64_t n = s->n;
  // scratch of the head: its own weight / angle / histogram buffers would
  // duplicate the pipeline's; reuse them only when no forward is recorded
  double *phi = s->phi, *w = s->w, *rho = s->rho, *rb = s->rbar, *ls = s->loss;
  double* tmp = nullptr;
  if (s->have_forward) {
    const size_t need = (size_t)n * (2 + c.nb1 + c.nb2) + 2 * (size_t)s->nb + 1;
    if (cudaMalloc((void**)&tmp, need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return NBODY_ENOMEM;
    }
    phi = tmp;
    w = phi + 2 * n;
    rho = w + (size_t)n * (c.nb1 + c.nb2);
    rb = rho + s->nb;
    ls = rb + s->nb;
  }
  k_head_weights<<<blocks_for(n, 128), 128, 0, s->s>>>(s->geom, x, n, phi, w);
  nb::count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_hist<<<c.nb1, 256, 0, s->s>>>(w, n, c.nb1, c.nb2, rho);
    nb::count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_loss<<<1, 256, 0, s->s>>>(rho, s->target, (int)s->nb, ls, rb);
    nb::count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(density, rho, (size_t)s->nb * sizeof(double), cudaMemcpyDefault, s->s);
  double L = 0.0;
  if (e == cudaSuccess && loss)
    e = cudaMemcpyAsync(&L, ls, sizeof(double), cudaMemcpyDeviceToHost, s->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->s);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return NBODY_ECUDA;
  if (loss) *loss = L;
  return NBODY_OK;
}

void nbody_stream_destroy(nbody_stream* s) {
  if (!s) return;
  cudaStreamSynchronize(s->s);
  free_stream(s);
  delete s;
}

int nbody_stream_set_target_cloud(nbody_stream* s, int64_t m, const double* tx,
                                  const double* tv, const double* scale_or_null,
                                  int n_sigma, const double* sigma) {
  if (!s || !tx || !tv || !sigma) return NBODY_EINVAL;
  // same size and bandwidths: the evaluator takes the new target in place
  if (s->mmd && nb::mmd_retarget(s->mmd, s->n, m, tx, tv, scale_or_null, n_sigma, sigma) ==
                    NBODY_OK) {
    s->have_forward = false;
    return NBODY_OK;
  }
  nbody_mmd* h = nullptr;
  const int rc = nbody_mmd_create(&h, s->n, 1, m, tx, tv, scale_or_null, n_sigma, sigma, s->s);
  if (rc) return rc;
  if (s->mmd) nbody_mmd_destroy(s->mmd);
  s->mmd = h;
  s->have_forward = false;
  return NBODY_OK;
}

int nbody_stream_set_target(nbody_stream* s, const double* target) {
  if (!s || !target) return NBODY_EINVAL;
  if (s->mmd) nbody_mmd_destroy(s->mmd);
  s->mmd = nullptr;
  s->have_forward = false;
  SCK(cudaMemcpyAsync(s->target, target, (size_t)s->nb * sizeof(double),
                      cudaMemcpyDefault, s->s));
  SCK(cudaStreamSynchronize(s->s));
  return NBODY_OK;
}

int nbody_stream_forward(nbody_stream* s, const double theta[4], double* loss,
                         double* density) {
  if (!s || !theta) return NBODY_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (!(theta[k] > 0.0) || !std::isfinite(theta[k])) return NBODY_EINVAL;
  s->have_forward = false;
  for (int k = 0; k < 4; ++k) s->theta[k] = theta[k];
  const nbody_stream_cfg& c = s->cfg;
  const int64_t n = s->n, ns = c.n_steps;
  // 1. backward orbit of the centre of mass
  const DevParams P = orbit_params(s);
  k_orbit<<<1, 32, 0, s->s>>>(P, c.X0[0], c.X0[1], c.X0[2], c.V0[0], c.V0[1],
                              c.V0[2], ns, s->ox, s->ovh, s->g6);
  nb::count_launch();
  SCK(cudaGetLastError());
  // 2. Plummer sphere at the recovered point
  k_ic<<<blocks_for(n, 256), 256, 0, s->s>>>(
      s->xhat, s->vhat, s->g6, c.a_prog, std::sqrt(c.G * theta[1] / c.a_prog),
      theta[1] / (double)n, n, s->x0, s->v0, s->m);
  nb::count_launch();
  SCK(cudaGetLastError());
  double g6[6];
  SCK(cudaMemcpyAsync(g6, s->g6, sizeof(g6), cudaMemcpyDeviceToHost, s->s));
  SCK(cudaStreamSynchronize(s->s));
  // 3. forward n-body run; the FP32 recentring origin follows the orbit
  nbody_params p{};
  p.G = c.G;
  p.eps = c.eps;
  p.dt = theta[0] / (double)ns;
  p.checkpoint_every = c.checkpoint_every;
  p.ext_flags = NBODY_EXT_NFW | NBODY_EXT_MN;
  p.center_mode = NBODY_CENTER_GUIDE;
  p.tape_mode = NBODY_TAPE_KEEP_LAST;
  p.nfw_M = theta[2];
  p.nfw_rs = c.nfw_rs;
  p.mn_M = theta[3];
  p.mn_a = c.mn_a;
  p.mn_b = c.mn_b;
  for (int k = 0; k < 3; ++k) {
    p.center[k] = g6[k];
    p.center_vel[k] = g6[3 + k];
  }
  int rc = nbody_set_params(s->ctx, &p);
  if (!rc) rc = nbody_set_state(s->ctx, s->x0, s->v0, s->m);
  if (!rc) rc = nbody_integrate(s->ctx, ns, s->xT, s->mmd ? s->vT : nullptr);
  if (rc) return rc;
  if (s->mmd) {
    // 4-5. point-cloud head: MMD^2 of the final phase-space cloud
    double L = 0.0;
    if ((rc = nbody_mmd_eval(s->mmd, s->xT, s->vT, &L, nullptr, nullptr))) return rc;
    if (density) {
      k_head_weights<<<blocks_for(n, 128), 128, 0, s->s>>>(s->geom, s->xT, n, s->phi, s->w);
      nb::count_launch();
      SCK(cudaGetLastError());
      k_hist<<<c.nb1, 256, 0, s->s>>>(s->w, n, c.nb1, c.nb2, s->rho);
      nb::count_launch();
      SCK(cudaGetLastError());
      SCK(cudaMemcpyAsync(density, s->rho, (size_t)s->nb * sizeof(double),
                          cudaMemcpyDefault, s->s));
      SCK(cudaStreamSynchronize(s->s));
    }
    if (loss) *loss = L;
    s->have_forward = true;
    return NBODY_OK;
  }
  // 4-5. head
  k_head_weights<<<blocks_for(n, 128), 128, 0, s->s>>>(s->geom, s->xT, n, s->phi, s->w);
  nb::count_launch();
  SCK(cudaGetLastError());
  k_hist<<<c.nb1, 256, 0, s->s>>>(s->w, n, c.nb1, c.nb2, s->rho);
  nb::count_launch();
  SCK(cudaGetLastError());
  k_loss<<<1, 256, 0, s->s>>>(s->rho, s->target, (int)s->nb, s->loss, s->rbar);
  nb::count_launch();
  SCK(cudaGetLastError());
  if (density)
    SCK(cudaMemcpyAsync(density, s->rho, (size_t)s->nb * sizeof(double),
                        cudaMemcpyDefault, s->s));
  double L = 0.0;
  SCK(cudaMemcpyAsync(&L, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->s));
  SCK(cudaStreamSynchronize(s->s));
  if (!std::isfinite(L)) return NBODY_ENAN;
  if (loss) *loss = L;
  s->have_forward = true;
  return NBODY_OK;
}

int nbody_stream_grad(nbody_stream* s, double theta_bar[4]) {
  if (!s || !theta_bar) return NBODY_EINVAL;
  if (!s->have_forward) return NBODY_ESTATE;
  const nbody_stream_cfg& c = s->cfg;
  const int64_t n = s->n, ns = c.n_steps;
  double tb[4];
  int rc;
  if (s->mmd) {
    double L = 0.0;
    if ((rc = nbody_mmd_eval(s->mmd, s->xT, s->vT, &L, s->xbar, s->vbar))) return rc;
    rc = nbody_vjp(s->ctx, s->xbar, s->vbar, s->x0bar, s->v0bar, nullptr, tb);
  } else {
    k_head_vjp<<<blocks_for(n, 128), 128, 0, s->s>>>(s->geom, s->xT, s->phi, s->w,
                                                     s->rbar, n, s->xbar);
    nb::count_launch();
    SCK(cudaGetLastError());
    rc = nbody_vjp(s->ctx, s->xbar, nullptr, s->x0bar, s->v0bar, nullptr, tb);
  }
  if (rc) return rc;
  SCK(cudaMemsetAsync(s->blk, 0, (size_t)s->nblk * 7 * sizeof(double), s->s));
  k_ic_vjp<<<s->nblk, 256, 0, s->s>>>(s->x0bar, s->v0bar, s->vhat, n, s->blk);
  nb::count_launch();
  SCK(cudaGetLastError());
  SCK(nb::launch_reduce_rows(s->blk, s->nblk, 7, s->red, s->s));
  const DevParams P = orbit_params(s);
  k_orbit_vjp<<<1, 32, 0, s->s>>>(P, s->ox, s->ovh, ns, s->red, s->orb);
  nb::count_launch();
  SCK(cudaGetLastError());
  k_theta_bar<<<1, 32, 0, s->s>>>(tb[0], tb[1], tb[2], tb[3], ns, c.G, c.a_prog,
                                  s->theta[1], s->red, s->orb, s->tbar);
  nb::count_launch();
  SCK(cudaGetLastError());
  SCK(cudaMemcpyAsync(theta_bar, s->tbar, 4 * sizeof(double),
                      cudaMemcpyDeviceToHost, s->s));
  SCK(cudaStreamSynchronize(s->s));
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(theta_bar[k])) return NBODY_ENAN;
  return NBODY_OK;
}

int nbody_stream_batch_create(nbody_stream_batch** out, const nbody_stream_cfg* cfg,
                              int64_t count, const double* xhat, const double* vhat, int64_t m,
                              const double* tx, const double* tv, const double* scale,
                              int n_sigma, const double* sigma, void* cuda_stream) {
  if (!out || !cfg || !xhat || !vhat || !tx || !tv || !scale || !sigma) return NBODY_EINVAL;
  *out = nullptr;
  const nbody_stream_cfg& c = *cfg;
  if (c.n < 1 || c.n_steps < 1 || !(c.eps > 0.0) || !(c.a_prog > 0.0) || !(c.nfw_rs > 0.0) ||
      c.mn_a < 0.0 || c.mn_b < 0.0 || count < 1 || count > 65535 || m < 1)
    return NBODY_EINVAL;
  nbody_stream_batch* s = new (std::nothrow) nbody_stream_batch();
  if (!s) return NBODY_ENOMEM;
  s->cfg = c;
  s->s = (cudaStream_t)cuda_stream;
  s->n = c.n;
  s->count = count;
  const size_t n3 = 3 * (size_t)c.n, all3 = n3 * (size_t)count, ns = (size_t)c.n_steps;
  std::vector<nbody_params> prm((size_t)count);
  for (auto& p : prm) {
    p = nbody_params{};
    p.G = c.G;
    p.eps = c.eps;
    p.dt = 1.0;
    p.checkpoint_every = 1;  // record the trajectories for the reverse sweep
    p.ext_flags = NBODY_EXT_NFW | NBODY_EXT_MN;
    p.center_mode = NBODY_CENTER_GUIDE;
    p.nfw_M = 1.0;
    p.nfw_rs = c.nfw_rs;
    p.mn_M = 1.0;
    p.mn_a = c.mn_a;
    p.mn_b = c.mn_b;
  }
  std::vector<int64_t> offs((size_t)count + 1);
  for (int64_t b = 0; b <= count; ++b) offs[(size_t)b] = b * c.n;
  int rc = nbody_create_batch(&s->ctx, (int)count, offs.data(), prm.data(), cuda_stream);
  // the pipeline needs the masses' gradients only, not the shape parameters'
  if (!rc) nb::batch_set_vjp_shape(nb::context_batch(s->ctx), false);
  double *dtx = nullptr, *dtv = nullptr;
  const size_t tm3 = 3 * (size_t)m * (size_t)count;
  if (!rc) rc = salloc(&s->xhat, n3);
  if (!rc) rc = salloc(&s->vhat, n3);
  if (!rc) rc = salloc(&s->theta, 4 * (size_t)count);
  for (double** p : {&s->x0, &s->v0, &s->xT, &s->vT, &s->xbar, &s->vbar, &s->x0bar, &s->v0bar})
    if (!rc) rc = salloc(p, all3);
  if (!rc) rc = salloc(&s->m, n3 / 3 * (size_t)count);
  if (!rc) rc = salloc(&s->ox, 3 * (ns + 1) * (size_t)count);
  if (!rc) rc = salloc(&s->ovh, 3 * ns * (size_t)count);
  if (!rc) rc = salloc(&s->g6, 6 * (size_t)count);
  if (!rc) rc = salloc(&s->loss, (size_t)count);
  if (!rc) rc = salloc(&s->tb, 8 * (size_t)count);
  if (!rc) rc = salloc(&s->red, 7 * (size_t)count);
  if (!rc) rc = salloc(&s->orb, 3 * (size_t)count);
  if (!rc) rc = salloc(&s->out, 4 * (size_t)count);
  if (!rc) rc = salloc(&s->nmark, 1);
  if (!rc) rc = salloc(&s->parts, 8 * (size_t)count);
  if (!rc) rc = salloc(&dtx, tm3);
  if (!rc) rc = salloc(&dtv, tm3);
  if (!rc && (cudaMemcpyAsync(s->xhat, xhat, n3 * sizeof(double), cudaMemcpyDefault, s->s) ||
              cudaMemcpyAsync(s->vhat, vhat, n3 * sizeof(double), cudaMemcpyDefault, s->s) ||
              cudaMemcpyAsync(dtx, tx, tm3 * sizeof(double), cudaMemcpyDefault, s->s) ||
              cudaMemcpyAsync(dtv, tv, tm3 * sizeof(double), cudaMemcpyDefault, s->s)))
    rc = NBODY_ECUDA;
  if (!rc) rc = nb::mmd_create_multi(&s->mmd, c.n, count, m, dtx, dtv, scale, n_sigma, sigma, s->s);
  cudaStreamSynchronize(s->s);
  sfree(dtx);
  sfree(dtv);
  if (rc) {
    free_stream_batch(s);
    delete s;
    return rc;
  }
  *out = s;
  return NBODY_OK;
}

int nbody_stream_batch_loss_grad(nbody_stream_batch* s, const double* thetas, double* losses,
                                 double* theta_bars) {
  if (!s || !thetas || !losses) return NBODY_EINVAL;
  const nbody_stream_cfg& c = s->cfg;
  const int64_t n = s->n, ns = c.n_steps, count = s->count;
  std::vector<double> th(4 * (size_t)count);
  SCK(cudaMemcpyAsync(th.data(), thetas, th.size() * sizeof(double), cudaMemcpyDefault, s->s));
  SCK(cudaStreamSynchronize(s->s));
  for (double t : th)
    if (!(t > 0.0) || !std::isfinite(t)) return NBODY_EINVAL;
  SCK(cudaMemcpyAsync(s->theta, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice,
                      s->s));
  // 1-2. backward orbits (kept for their adjoint) and Plummer spheres
  DevParams P0{};
  P0.G = c.G;
  P0.ext = NBODY_EXT_NFW | NBODY_EXT_MN;
  P0.nfw_rs = c.nfw_rs;
  P0.mn_a = c.mn_a;
  P0.mn_b = c.mn_b;
  k_orbit_batch_tape<<<blocks_for(count, 64), 64, 0, s->s>>>(
      P0, c.X0[0], c.X0[1], c.X0[2], c.V0[0], c.V0[1], c.V0[2], ns, s->theta, count, s->ox,
      s->ovh, s->g6);
  nb::count_launch();
  SCK(cudaGetLastError());
  k_ic_batch<<<blocks_for(n * count, 256), 256, 0, s->s>>>(s->xhat, s->vhat, s->g6, s->theta,
                                                           c.a_prog, c.G, n, count, s->x0,
                                                           s->v0, s->m);
  nb::count_launch();
  SCK(cudaGetLastError());
  std::vector<double> g6(6 * (size_t)count);
  SCK(cudaMemcpyAsync(g6.data(), s->g6, g6.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      s->s));
  SCK(cudaStreamSynchronize(s->s));
  // 3. the n-body runs, every member with its own step, potential and centre
  std::vector<nbody_params> prm((size_t)count);
  for (int64_t b = 0; b < count; ++b) {
    nbody_params& p = prm[(size_t)b];
    p = nbody_params{};
    p.G = c.G;
    p.eps = c.eps;
    p.dt = th[4 * b] / (double)ns;
    p.checkpoint_every = 1;
    p.ext_flags = NBODY_EXT_NFW | NBODY_EXT_MN;
    p.center_mode = NBODY_CENTER_GUIDE;
    p.nfw_M = th[4 * b + 2];
    p.nfw_rs = c.nfw_rs;
    p.mn_M = th[4 * b + 3];
    p.mn_a = c.mn_a;
    p.mn_b = c.mn_b;
    for (int k = 0; k < 3; ++k) {
      p.center[k] = g6[6 * b + k];
      p.center_vel[k] = g6[6 * b + 3 + k];
    }
  }
  int rc;
  bool nan_seen = false;
  // every call starts from a clean status: a member that fails (its run
  // leaves the finite range) is reported in its own loss and gradient
  nb::Batch* bt = nb::context_batch(s->ctx);
  if ((rc = nb::batch_clear_status(bt))) return rc;
  if ((rc = nbody_set_params(s->ctx, prm.data()))) return rc;
  if ((rc = nbody_set_state(s->ctx, s->x0, s->v0, s->m))) return rc;
  if (!s->tuned) {  // launch shape of the pair kernels, once, on the first state
    if ((rc = nbody_autotune(s->ctx, 2, nullptr, nullptr))) return rc;
    s->tuned = true;
  }
  if ((rc = nbody_integrate(s->ctx, ns, s->xT, s->vT))) return rc;
  // 4. MMD^2 of every member against its target, and its gradient
  if ((rc = nb::mmd_eval_multi(s->mmd, s->xT, s->vT, s->loss, theta_bars ? s->xbar : nullptr,
                               theta_bars ? s->vbar : nullptr)))
    return rc;
  if (theta_bars) {
    // 5. reverse: n-body runs, Plummer shifts, backward orbits
    rc = nbody_vjp_batch(s->ctx, s->xbar, s->vbar, s->x0bar, s->v0bar, s->tb);
    if (rc == NBODY_ENAN) {  // failed members are marked below
      nan_seen = true;
      rc = nb::batch_clear_status(bt);
    }
    if (rc) return rc;
    SCK(cudaMemsetAsync(s->red, 0, 7 * (size_t)count * sizeof(double), s->s));
    k_ic_vjp_batch<<<(unsigned)count, 256, 0, s->s>>>(s->x0bar, s->v0bar, s->vhat, n, count,
                                                      s->red);
    nb::count_launch();
    SCK(cudaGetLastError());
    k_orbit_vjp_batch<<<blocks_for(count, 64), 64, 0, s->s>>>(P0, s->ox, s->ovh, ns, s->theta,
                                                              count, s->red, s->orb);
    nb::count_launch();
    SCK(cudaGetLastError());
    k_theta_bar_batch<<<blocks_for(count, 64), 64, 0, s->s>>>(s->tb, ns, c.G, c.a_prog,
                                                              s->theta, count, s->red, s->orb,
                                                              s->out, s->parts);
    s->have_parts = true;
    nb::count_launch();
    SCK(cudaGetLastError());
  }
  SCK(cudaMemsetAsync(s->nmark, 0, sizeof(unsigned), s->s));
  k_mark_failed_batch<<<blocks_for(count, 64), 64, 0, s->s>>>(
      s->loss, theta_bars ? s->out : nullptr, count, s->nmark);
  nb::count_launch();
  SCK(cudaGetLastError());
  if (theta_bars)
    SCK(cudaMemcpyAsync(theta_bars, s->out, 4 * (size_t)count * sizeof(double),
                        cudaMemcpyDefault, s->s));
  SCK(cudaMemcpyAsync(losses, s->loss, (size_t)count * sizeof(double), cudaMemcpyDefault, s->s));
  unsigned marked = 0;
  SCK(cudaMemcpyAsync(&marked, s->nmark, sizeof(unsigned), cudaMemcpyDeviceToHost, s->s));
  SCK(cudaStreamSynchronize(s->s));
  // the NaN flag came from a value that reached no member's loss or
  // gradient: the failure cannot be attributed, so it is reported
  if (nan_seen && marked == 0) return NBODY_ENAN;
  return NBODY_OK;
}

int nbody_stream_batch_grad_parts(nbody_stream_batch* s, double* parts) {
  if (!s || !parts) return NBODY_EINVAL;
  if (!s->have_parts) return NBODY_ESTATE;
  SCK(cudaMemcpyAsync(parts, s->parts, 8 * (size_t)s->count * sizeof(double),
                      cudaMemcpyDefault, s->s));
  SCK(cudaStreamSynchronize(s->s));
  return NBODY_OK;
}

void nbody_stream_batch_destroy(nbody_stream_batch* s) {
  if (!s) return;
  cudaStreamSynchronize(s->s);
  free_stream_batch(s);
  delete s;
}

}  // extern "C"
