// update.cu -- O(N) kernels of the integrator and its adjoint.
//
//  * external potential of MWPotential2014's halo and disk (paper
//    Sec. 2.2.1), in FP64: NFW  Phi = -G M ln(1 + r/r_s) / r and
//    Miyamoto-Nagai  Phi = -G M / sqrt(R^2 + (a + sqrt(z^2 + b^2))^2),
//    their accelerations and the Jacobian-vector products of the
//    accelerations;
//  * the fused kick-drift-kick update (Velocity-Verlet, Sec. 2.2.1) with
//    first-same-as-last kicks: at point k the closing half kick of step k-1
//    and the opening half kick of step k are one kick of dt (dt/2 at the
//    ends), followed by the drift and the FP32 restaging of the positions
//    for the next pair pass; the same pass writes checkpoints and tape;
//  * the adjoint update (reverse-mode gradients, Sec. 2): at point k
//    xbar += c_k J(x_k)^T vbar with J = J_pair + J_ext, then the adjoint of
//    the drift vbar += dt xbar, plus the parameter-gradient sums;
//  * the guide orbit that carries the FP32 recentring origin;
//  * energy / momentum diagnostics and fixed-order reductions.
// State is FP64 throughout; one thread per particle.
#include <cmath>

#include "block_reduce.cuh"
#include "ext_potential.cuh"
#include "nbody_internal.cuh"
#include "staging.cuh"

namespace nb {

namespace {

__global__ void k_stage(const double* __restrict__ x,
                        const double* __restrict__ m,
                        const double* __restrict__ c, int64_t n, int64_t npad,
                        float4* __restrict__ st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  if (i < n)
    put_stage(st, i, (float)(x[i] - c[0]), (float)(x[npad + i] - c[1]),
              (float)(x[2 * npad + i] - c[2]), (float)m[i]);
  else
    put_stage(st, i, kPadPos, kPadPos, kPadPos, 0.f);
}

// power-of-two scale 2^-e bringing the largest |lambda| (bit pattern) near 1
__device__ __forceinline__ double lam_scale_from(unsigned long long bits) {
  const double mx = __longlong_as_double((long long)bits);
  if (!(mx > 0.0) || !isfinite(mx)) return 1.0;
  return ldexp(1.0, -ilogb(mx));
}

__device__ __forceinline__ void block_absmax(double v, unsigned long long* out) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) mx = fmax(mx, sh[k]);
    if (mx > 0.0 && isfinite(mx))
      atomicMax(out, (unsigned long long)__double_as_longlong(mx));
  }
}

__global__ void __launch_bounds__(256)
    k_lam_absmax(const double* __restrict__ lam, int64_t n, int64_t npad,
                 double* __restrict__ lsc, int slot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n)
    v = fmax(fabs(lam[i]), fmax(fabs(lam[npad + i]), fabs(lam[2 * npad + i])));
  block_absmax(v, reinterpret_cast<unsigned long long*>(lsc + 2) + slot);
}

__global__ void k_stage_vjp(const double* __restrict__ x,
                            const double* __restrict__ m,
                            const double* __restrict__ lam,
                            const double* __restrict__ c, int64_t n,
                            int64_t npad, float4* __restrict__ vst,
                            double* __restrict__ lsc, int slot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double sc =
      lam_scale_from(reinterpret_cast<const unsigned long long*>(lsc + 2)[slot]);
  if (i == 0) lsc[slot] = sc;
  if (i >= npad) return;
  if (i < n)
    put_vstage(vst, i, (float)(x[i] - c[0]), (float)(x[npad + i] - c[1]),
               (float)(x[2 * npad + i] - c[2]), (float)m[i],
               (float)(sc * lam[i]), (float)(sc * lam[npad + i]),
               (float)(sc * lam[2 * npad + i]));
  else
    put_vstage(vst, i, kPadPos, kPadPos, kPadPos, 0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------- update
__global__ void __launch_bounds__(256) k_update(UpdateArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const DevParams& P = *a.P;
  const int64_t np = a.npad;
  double ap[3];
  if (a.part_is_final) {
#pragma unroll
    for (int d = 0; d < 3; ++d) ap[d] = a.part[d * np + i];
  } else {
    double s[3];
    slice_sums<3>(a.part + i, a.S, 3 * np, np, s);
#pragma unroll
    for (int d = 0; d < 3; ++d) ap[d] = P.G * a.mscale * s[d];
  }
  double x[3], v[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    x[d] = a.x[d * np + i];
    v[d] = a.v[d * np + i];
    if (a.acc_out) a.acc_out[d * np + i] = ap[d];
    if (a.cp_x) {
      a.cp_x[d * np + i] = x[d];
      a.cp_v[d * np + i] = v[d];
      a.cp_a[d * np + i] = ap[d];
    }
    if (a.tape_x) {
      a.tape_x[d * np + i] = x[d];
      a.tape_a[d * np + i] = ap[d];
    }
  }
  double ae[3];
  if (a.aext) {
#pragma unroll
    for (int d = 0; d < 3; ++d) ae[d] = a.aext[d * np + i];
  } else {
    ext_accel(P, x[0], x[1], x[2], ae);
  }
  const double kick = a.kick * P.dt;
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) v[d] += kick * (ap[d] + ae[d]);
  if (a.drift) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (a.tape_vh) a.tape_vh[d * np + i] = v[d];
      x[d] += P.dt * v[d];
      a.x[d * np + i] = x[d];
    }
    put_stage_xyz(a.st, i, (float)(x[0] - a.c_next[0]),
                  (float)(x[1] - a.c_next[1]), (float)(x[2] - a.c_next[2]));
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    a.v[d * np + i] = v[d];
    bad |= !isfinite(v[d]) || !isfinite(x[d]);
  }
  if (bad) atomicOr(a.status, kStatusNaN);
}

// ------------------------------------------------------------------ adjoint
// EA: the external field's adjoint terms come from a.ea (computed beside the
// pair VJP); otherwise the kernel computes them.  Two instances, so that the
// one reading a.ea carries none of the field's code (a smaller kernel:
// instruction fetch, not arithmetic, was what stalled it).
template <bool EA>
__global__ void __launch_bounds__(256) k_adjoint(AdjointArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const DevParams& P = *a.P;
  const int64_t np = a.npad;
  double contrib[kAdjCols] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  // scale of the cotangents this point's VJP was computed with, and the one
  // for the cotangents staged now (from the largest |lambda| at this point)
  const double s_here = a.lsc[a.slot];
  // the scale is a power of two, so multiplying by its reciprocal gives the
  // quotient's bits: one FP64 division per thread instead of one per
  // component (divisions are slow at GB300's FP64 rate)
  const double inv_here = 1.0 / s_here;
  const unsigned long long* maxbits =
      reinterpret_cast<const unsigned long long*>(a.lsc + 2);
  const double s_next = a.drift ? lam_scale_from(maxbits[a.slot]) : 1.0;
  double vmax = 0.0;
  if (i < a.n) {
    double lam[3], x[3], ap[3], g[3], gs[3];
    slice_sums<3>(a.gpart + i, a.S, 3 * np, np, gs);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lam[d] = a.vbar[d * np + i];
      x[d] = a.xk[d * np + i];
      ap[d] = a.ak[d * np + i];
      g[d] = -P.G * a.mscale * (gs[d] * inv_here);
    }
    ExtAdj ea;
    if (EA) {  // computed beside this point's pair VJP (k_ext_adjoint)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ea.jl[d] = a.ea[d * np + i];
        ea.sh[d] = a.ea[(6 + d) * np + i];
      }
      ea.ln = a.ea[3 * np + i];
      ea.lm = a.ea[4 * np + i];
      ea.lb = a.ea[5 * np + i];
    } else {
      ext_adjoint<true>(P, x[0], x[1], x[2], lam, ea);
    }
    const double ck = a.ck * P.dt;
    double xb[3];
    double la = 0.0, lp = 0.0;
    const double ln = ea.ln, lm = ea.lm, lb = ea.lb;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      xb[d] = a.xbar[d * np + i] + ck * (g[d] + ea.jl[d]);
      lp += lam[d] * ap[d];
    }
    la = lp + P.nfw_GM * ln + P.mn_GM * lm + P.bulge_GM * lb;
    if (a.mpart) {  // per-particle mass gradient of this kick
      double sm[1];
      slice_sums<1>(a.mpart + i, a.S, np, 0, sm);
      a.mbar[i] += ck * P.G * (sm[0] * inv_here);
    }
    contrib[0] = a.ck * la;          // dL/d dt from the kick(s)
    contrib[1] = ck * lp;            // sum_j m_j dL/dm_j
    contrib[2] = ck * P.G * ln;      // dL/d M_NFW
    contrib[3] = ck * P.G * lm;      // dL/d M_MN
    if (P.ext) {                     // dL/d (r_s, a_MN, b_MN)
      contrib[4] = ck * ea.sh[0];
      contrib[5] = ck * ea.sh[1];
      contrib[6] = ck * ea.sh[2];
      contrib[7] = ck * P.G * lb;    // dL/d M_bulge
    }
    double vb[3] = {lam[0], lam[1], lam[2]};
    if (a.drift) {
      double xv = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        xv += xb[d] * a.vh_prev[d * np + i];
        vb[d] += P.dt * xb[d];
        a.vbar[d * np + i] = vb[d];
        vmax = fmax(vmax, fabs(vb[d]));
      }
      contrib[0] += xv;              // dL/d dt from the drift
      put_vstage(a.vst, i, (float)(a.x_prev[i] - a.c_prev[0]),
                 (float)(a.x_prev[np + i] - a.c_prev[1]),
                 (float)(a.x_prev[2 * np + i] - a.c_prev[2]), (float)a.m[i],
                 (float)(s_next * vb[0]), (float)(s_next * vb[1]),
                 (float)(s_next * vb[2]));
    }
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      a.xbar[d * np + i] = xb[d];
      bad |= !isfinite(xb[d]) || !isfinite(vb[d]);
    }
    if (bad) atomicOr(a.status, kStatusNaN);
  }
  block_accumulate<kAdjCols>(contrib, a.blk);
  if (a.drift) {
    if (i == 0) a.lsc[1 - a.slot] = s_next;
    block_absmax(vmax, reinterpret_cast<unsigned long long*>(a.lsc + 2) + (1 - a.slot));
  }
}

// the external potential's adjoint terms of every particle at one point
// (positions x, cotangents lam): the FP64 part of the adjoint update, run
// on a side stream beside that point's pair VJP; layout [kExtAdjCols][npad]
// = H lam (3), lam . a_NFW, lam . a_MN, lam . a_bulge per unit mass, shape
// terms (3)
__global__ void __launch_bounds__(256)
    k_ext_adjoint(const DevParams* __restrict__ Pp, const double* __restrict__ x,
                  const double* __restrict__ lam, int64_t n, int64_t npad,
                  double* __restrict__ ea) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l[3] = {lam[i], lam[npad + i], lam[2 * npad + i]};
  ExtAdj e;
  ext_adjoint<true>(*Pp, x[i], x[npad + i], x[2 * npad + i], l, e);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ea[d * npad + i] = e.jl[d];
    ea[(6 + d) * npad + i] = e.sh[d];
  }
  ea[3 * npad + i] = e.ln;
  ea[4 * npad + i] = e.lm;
  ea[5 * npad + i] = e.lb;
}

// external acceleration of the state (x [3][npad]) into aext [3][npad]: the
// same ext_accel the update applies when it computes the field itself
__global__ void __launch_bounds__(256)
    k_field(const DevParams* __restrict__ P, const double* __restrict__ x, int64_t n,
            int64_t npad, double* __restrict__ aext) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[3];
  ext_accel(*P, x[i], x[npad + i], x[2 * npad + i], a);
#pragma unroll
  for (int d = 0; d < 3; ++d) aext[d * npad + i] = a[d];
}

// external acceleration at caller points (3 x n SoA in and out)
__global__ void k_ext_accel(DevParams P, const double* __restrict__ x, int64_t n,
                            double* __restrict__ acc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[3];
  ext_accel(P, x[i], x[n + i], x[2 * n + i], a);
#pragma unroll
  for (int d = 0; d < 3; ++d) acc[d * n + i] = a[d];
}

// ------------------------------------------------------------ reductions etc
__global__ void __launch_bounds__(256)
    k_reduce_rows(const double* __restrict__ blk, int nblk, int ncol,
                  double* __restrict__ out) {
  __shared__ double sh[256];
  for (int q = 0; q < ncol; ++q) {
    double s = 0.0;
    for (int r = threadIdx.x; r < nblk; r += 256) s += blk[(int64_t)r * ncol + q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
    __syncthreads();
  }
}

__global__ void k_guide(const DevParams* __restrict__ Pp,
                        const double* __restrict__ g0, int64_t n_steps,
                        double* __restrict__ centers, double* __restrict__ gout) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const DevParams P = *Pp;
  double x[3] = {g0[0], g0[1], g0[2]};
  double v[3] = {g0[3], g0[4], g0[5]};
  ExtUnit e;
  ext_unit(P, x[0], x[1], x[2], e);
  for (int d = 0; d < 3; ++d) centers[d] = x[d];
  for (int64_t s = 0; s < n_steps; ++s) {
    for (int d = 0; d < 3; ++d) {
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
      x[d] += P.dt * v[d];
    }
    ext_unit(P, x[0], x[1], x[2], e);
    for (int d = 0; d < 3; ++d) {
      v[d] += 0.5 * P.dt * (P.nfw_GM * e.n[d] + P.mn_GM * e.d[d] + P.bulge_GM * e.b[d]);
      centers[3 * (s + 1) + d] = x[d];
    }
  }
  for (int d = 0; d < 3; ++d) {
    gout[d] = x[d];
    gout[3 + d] = v[d];
  }
}

__global__ void __launch_bounds__(256)
    k_energy(const DevParams* __restrict__ Pp, const double* __restrict__ x,
             const double* __restrict__ v, const double* __restrict__ m,
             int64_t n, const double* __restrict__ pot, int S, int64_t np,
             double* __restrict__ blk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const DevParams& P = *Pp;
  double val[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (i < n) {
    const double mi = m[i];
    double v2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double vd = v[d * np + i];
      v2 += vd * vd;
      val[3 + d] = mi * vd;
    }
    val[0] = 0.5 * mi * v2;
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += pot[(int64_t)q * np + i];
    // remove the self term m_i / eps that the pair loop includes
    val[1] = -0.5 * P.G * mi * (s - mi / sqrt(P.eps2));
    val[2] = mi * ext_potential(P, x[i], x[np + i], x[2 * np + i]);
  }
  block_accumulate<6>(val, blk);
}

__global__ void k_reduce_partials(const double* __restrict__ part, int S,
                                  int64_t np, int64_t n, double G,
                                  double* __restrict__ acc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += part[((int64_t)q * 3 + d) * np + i];
    acc[d * n + i] = G * s;
  }
}

// out = {min, max} of m[0..n) (one block; order-independent, deterministic)
__global__ void __launch_bounds__(1024)
    k_minmax(const double* __restrict__ m, int64_t n, double* __restrict__ out) {
  __shared__ double smin[32], smax[32];
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    lo = fmin(lo, m[i]);
    hi = fmax(hi, m[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    smin[w] = lo;
    smax[w] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      lo = fmin(lo, smin[k]);
      hi = fmax(hi, smax[k]);
    }
    out[0] = lo;
    out[1] = hi;
  }
}

inline unsigned blocks_for(int64_t n, int t) {
  return (unsigned)((n + t - 1) / t);
}

// threads per block of the per-particle FP64 kernels: 256 when that still
// gives several blocks per SM, fewer for small systems so that the (slow)
// FP64 work spreads over every SM -- one warp below 65 536 particles, where
// the block reductions then need no barrier
inline int particle_threads(int64_t n) { return n >= 262144 ? 256 : n >= 65536 ? 64 : 32; }

}  // namespace

cudaError_t launch_stage(const double* x, const double* m, const double* c,
                         int64_t n, int64_t npad, float4* st, cudaStream_t s) {
  k_stage<<<blocks_for(npad, 256), 256, 0, s>>>(x, m, c, n, npad, st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  const int t = particle_threads(a.n);
  k_update<<<blocks_for(a.n, t), t, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_lam_absmax(const double* lam, int64_t n, int64_t npad,
                              double* lsc, int slot, cudaStream_t s) {
  k_lam_absmax<<<blocks_for(n, 256), 256, 0, s>>>(lam, n, npad, lsc, slot);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_stage_vjp(const double* x, const double* m,
                             const double* lam, const double* c, int64_t n,
                             int64_t npad, float4* vst, double* lsc, int slot,
                             cudaStream_t s) {
  k_stage_vjp<<<blocks_for(npad, 256), 256, 0, s>>>(x, m, lam, c, n, npad, vst,
                                                    lsc, slot);
  count_launch();
  return cudaGetLastError();
}

int adjoint_blocks(int64_t n) { return (int)blocks_for(n, particle_threads(n)); }

cudaError_t launch_ext_adjoint(const DevParams* P, const double* x, const double* lam,
                               int64_t n, int64_t npad, double* ea, cudaStream_t s) {
  k_ext_adjoint<<<blocks_for(n, 64), 64, 0, s>>>(P, x, lam, n, npad, ea);
  count_launch();
  return cudaGetLastError();
}

void set_bulge(DevParams& d, double G, double M, double alpha, double rc) {
  const double s = 0.5 * (3.0 - alpha);
  d.bulge_GM = G * M;
  d.bulge_s = s;
  d.bulge_irc2 = 1.0 / (rc * rc);
  d.bulge_irc = 1.0 / rc;
  d.bulge_igs = 1.0 / std::tgamma(s);
  d.bulge_gsh = std::tgamma(s - 0.5);
}

cudaError_t launch_field(const DevParams* P, const double* x, int64_t n, int64_t npad,
                         double* aext, cudaStream_t s) {
  k_field<<<blocks_for(n, 64), 64, 0, s>>>(P, x, n, npad, aext);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ext_accel(const DevParams& P, const double* x, int64_t n, double* acc,
                             cudaStream_t s) {
  k_ext_accel<<<blocks_for(n, 256), 256, 0, s>>>(P, x, n, acc);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_minmax(const double* m, int64_t n, double* out, cudaStream_t s) {
  k_minmax<<<1, 1024, 0, s>>>(m, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointArgs& a, cudaStream_t s) {
  if (a.ea)
    k_adjoint<true><<<adjoint_blocks(a.n), particle_threads(a.n), 0, s>>>(a);
  else
    k_adjoint<false><<<adjoint_blocks(a.n), particle_threads(a.n), 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_reduce_rows(const double* blk, int nblk, int ncol,
                               double* out, cudaStream_t s) {
  k_reduce_rows<<<1, 256, 0, s>>>(blk, nblk, ncol, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_guide(const DevParams* P, const double* g0, int64_t n_steps,
                         double* centers, double* g_out, cudaStream_t s) {
  k_guide<<<1, 32, 0, s>>>(P, g0, n_steps, centers, g_out);
  count_launch();
  return cudaGetLastError();
}

int energy_blocks(int64_t n) { return (int)blocks_for(n, 256); }

cudaError_t launch_energy(const DevParams* P, const double* x,
                          const double* v, const double* m, int64_t n,
                          const double* pot_part, int S, int64_t npad,
                          double* blk, int nblk, cudaStream_t s) {
  (void)nblk;
  k_energy<<<energy_blocks(n), 256, 0, s>>>(P, x, v, m, n, pot_part, S, npad, blk);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* part, int S, int64_t npad,
                                   int64_t n, double G, double* acc,
                                   cudaStream_t s) {
  k_reduce_partials<<<blocks_for(n, 256), 256, 0, s>>>(part, S, npad, n, G, acc);
  count_launch();
  return cudaGetLastError();
}

}  // namespace nb
