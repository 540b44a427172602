// batch.cu -- many simulations of uneven N, each with its own parameters,
// advanced together: one persistent pair-force launch per step over a work
// list of (simulation, i-tile, j-chunk) items, one batched update launch,
// the whole step loop captured once as a CUDA graph and replayed.  The
// physics per simulation is the same as the single-system path (softened
// pair sum, paper Sec. 1; NFW + MN potential and kick-drift-kick, Sec.
// 2.2.1).
//
// Work list: items are sorted by cost, largest first (LPT), and handed out
// through an atomic counter, so the persistent blocks stay busy to the end
// of the step; every item writes its own FP64 partial slice and the update
// kernel sums the slices in a fixed order, so the result does not depend on
// which block took which item.
//
// Autotuning: the launch shape (threads per block, i-particles per thread,
// j-chunk length) is chosen among kNTune candidates by timing the pair
// kernel on the batch itself (nbody_autotune).
//
// Reverse sweep (nbody_vjp_batch): when every simulation asks for an
// adjoint tape, the forward run keeps its whole trajectory in device memory
// (positions and pair accelerations at every point, half-step velocities of
// every step: 72 B per particle and step), so the reverse sweep recomputes
// nothing.  One persistent launch per point computes the pair VJP of a work
// item's rows over their simulation's whole j-range and applies the adjoint
// update to those rows (the discrete adjoint of the kick-drift-kick step,
// Sec. 2), staging the cotangents of the previous point into the other
// adjoint staging buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "block_reduce.cuh"
#include "ext_potential.cuh"
#include "nbody_internal.cuh"
#include "pair_body.cuh"
#include "staging.cuh"
#include "vjp_body.cuh"

namespace nb {

namespace {

// launch shape candidates: threads, i-particles per thread, j-chunk length
// (particles), j-pairs per shared-memory tile
struct TuneCfg {
  int nt, r, jchunk, tj;
};
// (the last takes every simulation's j-range whole: one chunk each, so the
// step always runs fused)
constexpr TuneCfg kTune[NBODY_NTUNE] = {
    {128, 4, 4096, 512}, {128, 4, 2048, 512}, {128, 4, 8192, 512}, {128, 2, 2048, 512},
    {256, 2, 4096, 512}, {128, 4, 4096, 128}, {128, 8, 8192, 512}, {128, 4, 1 << 30, 512}};

struct SimMeta {
  int64_t npad, poff, part_off;
  int64_t n, off;  // particles and offset in the caller's unpadded layout
  int S, ntiles;
  float eps2f;
  int pad;
  double mscale;  // multiplies the raw sums (the common mass with EQM, else 1)
};

// Pair sums of one work item w = (simulation, i-tile, j-chunk): FP32 within
// a shared-memory tile of kTJ j-pairs, FP64 across tiles, into dax/day/daz.
// EQM: every simulation has equal masses; the sums leave the mass out.
template <int NT, int R, int kTJ, bool EQM>
__device__ __forceinline__ void pair_item(const float4* __restrict__ st, const SimMeta& M,
                                          int4 w, float4* sj, int64_t i0, double (&dax)[R],
                                          double (&day)[R], double (&daz)[R]) {
  const int t = threadIdx.x;
  const int tile_b = (int)(((int64_t)w.z * M.ntiles) / M.S);
  const int tile_e = (int)(((int64_t)(w.z + 1) * M.ntiles) / M.S);
  const float4* sts = st + M.poff;  // one float4 per particle
  float2 nx[R], ny[R], nz[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float xi, yi, zi;
    load_i(sts, i0 + r * NT, xi, yi, zi);
    nx[r] = make_float2(-xi, -xi);
    ny[r] = make_float2(-yi, -yi);
    nz[r] = make_float2(-zi, -zi);
    dax[r] = day[r] = daz[r] = 0.0;
  }
  const float2 e2 = make_float2(M.eps2f, M.eps2f);
  for (int tile = tile_b; tile < tile_e; ++tile) {
    __syncthreads();
    const float4* src = sts + (int64_t)tile * (2 * kTJ);
#pragma unroll
    for (int q = t; q < 2 * kTJ; q += NT) sj[q] = src[q];
    __syncthreads();
    float2 ax[R], ay[R], az[R], ph[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ax[r] = ay[r] = az[r] = ph[r] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int jj = 0; jj < kTJ; ++jj) {
      const float4 A = sj[2 * jj];
      const float4 B = sj[2 * jj + 1];
      const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
      const float2 zj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (EQM)
          body_eqm(xj, yj, zj, nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r]);
        else
          body<false>(xj, yj, zj, mj, nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r], ph[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      dax[r] += (double)ax[r].x + (double)ax[r].y;
      day[r] += (double)ay[r].x + (double)ay[r].y;
      daz[r] += (double)az[r].x + (double)az[r].y;
    }
  }
}

// one pair pass for every simulation: persistent blocks take work items
// (largest first) from an atomic counter; per-chunk partial sums to part
template <int NT, int R, int kTJ, bool EQM>
__global__ void __launch_bounds__(NT)
    k_pair_batch(const float4* __restrict__ st, const SimMeta* __restrict__ meta,
                 const int4* __restrict__ items, int nitems,
                 unsigned* __restrict__ ctr, double* __restrict__ part) {
  __shared__ float4 sj[2 * kTJ];
  __shared__ int s_item;
  const int t = threadIdx.x;
  for (;;) {
    __syncthreads();
    if (t == 0) s_item = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int4 w = items[it];
    const SimMeta M = meta[w.x];
    const int64_t i0 = (int64_t)w.y * (NT * R) + t;  // local index
    double dax[R], day[R], daz[R];
    pair_item<NT, R, kTJ, EQM>(st, M, w, sj, i0, dax, day, daz);
    double* p = part + M.part_off + (int64_t)w.z * 3 * M.npad;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = i0 + r * NT;
      p[i] = dax[r];
      p[M.npad + i] = day[r];
      p[2 * M.npad + i] = daz[r];
    }
  }
}

// KDK update of one particle (global index g of simulation s) from its
// complete pair sums (the arithmetic of the separate update kernel)
// Tape of a recorded forward run at one point k (NULL when not recording):
// positions x_k and pair accelerations a_k at the point, and the velocity
// after its kick (the half-step velocity of the drift that follows).
struct TapePoint {
  double* x;
  double* a;
  double* vh;
};

__device__ __forceinline__ bool update_one(const DevParams& Q, const SimMeta& M, int s,
                                           int64_t g, const double sum[3], double* x,
                                           double* v, int64_t ptot, double kick, int drift,
                                           const double* centers, int64_t cstride,
                                           int64_t k_next, float4* st_next, TapePoint tp) {
  double ap[3];
  for (int d = 0; d < 3; ++d) ap[d] = Q.G * M.mscale * (0.0 + sum[d]);
  double xx[3], vv[3];
  for (int d = 0; d < 3; ++d) {
    xx[d] = x[d * ptot + g];
    vv[d] = v[d * ptot + g];
    if (tp.x) {
      tp.x[d * ptot + g] = xx[d];
      tp.a[d * ptot + g] = ap[d];
    }
  }
  ExtUnit e;
  ext_unit(Q, xx[0], xx[1], xx[2], e);
  bool bad = false;
  for (int d = 0; d < 3; ++d) {
    vv[d] += kick * Q.dt * (ap[d] + Q.nfw_GM * e.n[d] + Q.mn_GM * e.d[d] + Q.bulge_GM * e.b[d]);
    if (drift && tp.vh) tp.vh[d * ptot + g] = vv[d];
    if (drift) xx[d] += Q.dt * vv[d];
    x[d * ptot + g] = xx[d];
    v[d * ptot + g] = vv[d];
    bad |= !isfinite(xx[d]) || !isfinite(vv[d]);
  }
  if (drift) {
    const double* c = centers + (int64_t)s * cstride + 3 * k_next;
    put_stage_xyz(st_next, g, (float)(xx[0] - c[0]), (float)(xx[1] - c[1]),
                  (float)(xx[2] - c[2]));
  }
  return bad;
}

// Fused step for batches whose simulations each take one j-chunk: a work
// item holds the complete pair sums of its i-tile, so the block applies the
// kick (and drift) to those particles itself and stages them into the other
// staging buffer.  FP64 update work of some blocks then overlaps the FP32
// pair loops of others on the same SM (separate pipes).  The work counter
// of the next step is re-armed here (ctr_next), this step's by the last.
template <int NT, int R, int kTJ, bool EQM>
__global__ void __launch_bounds__(NT)
    k_step_batch(const float4* __restrict__ st, float4* __restrict__ st_next,
                 const SimMeta* __restrict__ meta, const int4* __restrict__ items, int nitems,
                 unsigned* __restrict__ ctr, unsigned* __restrict__ ctr_next,
                 const DevParams* __restrict__ P, double* __restrict__ x,
                 double* __restrict__ v, int64_t ptot, double kick, int drift,
                 const double* __restrict__ centers, int64_t cstride, int64_t k_next,
                 int* __restrict__ status, TapePoint tp) {
  __shared__ float4 sj[2 * kTJ];
  __shared__ int s_item;
  const int t = threadIdx.x;
  if (blockIdx.x == 0 && t == 0) *ctr_next = 0u;
  bool bad = false;
  for (;;) {
    __syncthreads();
    if (t == 0) s_item = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int4 w = items[it];
    const SimMeta M = meta[w.x];
    const int64_t i0 = (int64_t)w.y * (NT * R) + t;
    double dax[R], day[R], daz[R];
    pair_item<NT, R, kTJ, EQM>(st, M, w, sj, i0, dax, day, daz);
    const DevParams Q = P[w.x];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = i0 + r * NT;
      if (i < M.n) {
        const double sum[3] = {dax[r], day[r], daz[r]};
        bad |= update_one(Q, M, w.x, M.poff + i, sum, x, v, ptot, kick, drift, centers,
                          cstride, k_next, st_next, tp);
      }
    }
  }
  if (bad) atomicOr(status, kStatusNaN);
}

// one thread per simulation: FP32 recentring origins of every point
__global__ void k_guide_batch(const DevParams* __restrict__ P,
                              const int* __restrict__ mode, double* __restrict__ g,
                              int n_sims, int64_t n_steps, double* __restrict__ centers,
                              int64_t cstride) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sims) return;
  const DevParams Q = P[s];
  double* c = centers + (int64_t)s * cstride;
  double x[3] = {g[6 * s], g[6 * s + 1], g[6 * s + 2]};
  double v[3] = {g[6 * s + 3], g[6 * s + 4], g[6 * s + 5]};
  for (int d = 0; d < 3; ++d) c[d] = x[d];
  if (!mode[s]) {
    for (int64_t k = 1; k <= n_steps; ++k)
      for (int d = 0; d < 3; ++d) c[3 * k + d] = x[d];
    return;
  }
  ExtUnit e;
  ext_unit(Q, x[0], x[1], x[2], e);
  for (int64_t k = 0; k < n_steps; ++k) {
    for (int d = 0; d < 3; ++d) {
      v[d] += 0.5 * Q.dt * (Q.nfw_GM * e.n[d] + Q.mn_GM * e.d[d] + Q.bulge_GM * e.b[d]);
      x[d] += Q.dt * v[d];
    }
    ext_unit(Q, x[0], x[1], x[2], e);
    for (int d = 0; d < 3; ++d) {
      v[d] += 0.5 * Q.dt * (Q.nfw_GM * e.n[d] + Q.mn_GM * e.d[d] + Q.bulge_GM * e.b[d]);
      c[3 * (k + 1) + d] = x[d];
    }
  }
  for (int d = 0; d < 3; ++d) {
    g[6 * s + d] = x[d];
    g[6 * s + 3 + d] = v[d];
  }
}

__global__ void __launch_bounds__(256)
    k_stage_batch(const SimMeta* __restrict__ meta, const int* __restrict__ blk_sim,
                  const double* __restrict__ x, const double* __restrict__ m,
                  int64_t ptot, const double* __restrict__ centers, int64_t cstride,
                  float4* __restrict__ st, float4* __restrict__ st2) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blk_sim[blockIdx.x];
  const SimMeta M = meta[s];
  const int64_t i = g - M.poff;
  float px = kPadPos, py = kPadPos, pz = kPadPos, pm = 0.f;
  if (i < M.n) {
    const double* c = centers + (int64_t)s * cstride;
    px = (float)(x[g] - c[0]);
    py = (float)(x[ptot + g] - c[1]);
    pz = (float)(x[2 * ptot + g] - c[2]);
    pm = (float)m[g];
  }
  put_stage(st, g, px, py, pz, pm);
  if (st2) put_stage(st2, g, px, py, pz, pm);
}

__global__ void __launch_bounds__(256)
    k_update_batch(const DevParams* __restrict__ P, const SimMeta* __restrict__ meta,
                   const int* __restrict__ blk_sim, double* __restrict__ x,
                   double* __restrict__ v, const double* __restrict__ part,
                   int64_t ptot, double kick, int drift,
                   const double* __restrict__ centers, int64_t cstride,
                   int64_t k_next, float4* __restrict__ st, int* __restrict__ status,
                   unsigned* __restrict__ ctr, TapePoint tp) {
  // the pair launch of this step has finished: re-arm its work counter
  if (blockIdx.x == 0 && threadIdx.x == 0) *ctr = 0u;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blk_sim[blockIdx.x];
  const SimMeta M = meta[s];
  const int64_t i = g - M.poff;
  if (i >= M.n) return;
  const DevParams Q = P[s];
  double ap[3], acc[3];
  slice_sums<3>(part + M.part_off + i, M.S, 3 * M.npad, M.npad, acc);
  for (int d = 0; d < 3; ++d) ap[d] = Q.G * M.mscale * acc[d];
  double xx[3], vv[3];
  for (int d = 0; d < 3; ++d) {
    xx[d] = x[d * ptot + g];
    vv[d] = v[d * ptot + g];
    if (tp.x) {
      tp.x[d * ptot + g] = xx[d];
      tp.a[d * ptot + g] = ap[d];
    }
  }
  ExtUnit e;
  ext_unit(Q, xx[0], xx[1], xx[2], e);
  bool bad = false;
  for (int d = 0; d < 3; ++d) {
    vv[d] += kick * Q.dt * (ap[d] + Q.nfw_GM * e.n[d] + Q.mn_GM * e.d[d] + Q.bulge_GM * e.b[d]);
    if (drift && tp.vh) tp.vh[d * ptot + g] = vv[d];
    if (drift) xx[d] += Q.dt * vv[d];
    x[d * ptot + g] = xx[d];
    v[d * ptot + g] = vv[d];
    bad |= !isfinite(xx[d]) || !isfinite(vv[d]);
  }
  if (drift) {
    const double* c = centers + (int64_t)s * cstride + 3 * k_next;
    put_stage_xyz(st, g, (float)(xx[0] - c[0]), (float)(xx[1] - c[1]),
                  (float)(xx[2] - c[2]));
  }
  if (bad) atomicOr(status, kStatusNaN);
}

// ------------------------------------------------------------ reverse sweep
// VJP work items: (simulation, row tile of kVNT * kVR rows), each over its
// simulation's whole j-range (kVTJ j-pairs per shared-memory tile)
constexpr int kVNT = 128, kVR = 2, kVTJ = 256;

// FP32 cotangent scaling, per simulation (the single-system sweep's scheme):
// the cotangents staged for point k are multiplied by an exact power of two
// s = 2^-e chosen from the largest |lambda| of the simulation at the point
// before, so their FP32 copies neither overflow nor underflow while the
// FP64 cotangents grow or shrink.  lsc[(k & 1) * n_sims + s] holds the
// scale of point k's staging, lmax[...] (bit patterns of non-negative
// doubles) the running maxima.
__device__ __forceinline__ double lam_scale(unsigned long long bits) {
  const double mx = __longlong_as_double((long long)bits);
  if (!(mx > 0.0) || !isfinite(mx)) return 1.0;
  return ldexp(1.0, -ilogb(mx));
}

// block maximum of v (>= 0) into *out by an atomic max of its bit pattern
__device__ __forceinline__ void block_max_into(double v, unsigned long long* out) {
  __shared__ double sm[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) mx = fmax(mx, sm[k]);
    if (mx > 0.0 && isfinite(mx)) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
  }
}

// per-simulation max |lam| of the final cotangents into lmax[s]
__global__ void __launch_bounds__(256)
    k_vabsmax_batch(const SimMeta* __restrict__ meta, const int* __restrict__ blk_sim,
                    const double* __restrict__ lam, int64_t ptot,
                    unsigned long long* __restrict__ lmax) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blk_sim[blockIdx.x];
  const SimMeta M = meta[s];
  double v = 0.0;
  if (g - M.poff < M.n)
    v = fmax(fabs(lam[g]), fmax(fabs(lam[ptot + g]), fabs(lam[2 * ptot + g])));
  block_max_into(v, lmax + s);
}

// adjoint staging of point k (positions x, cotangents lam scaled by the
// simulation's power of two from lmax) of every simulation into vst, the
// scale into lsc[s]; the pads (far away, zero mass and cotangent) into vst2
// as well
__global__ void __launch_bounds__(256)
    k_vstage_batch(const SimMeta* __restrict__ meta, const int* __restrict__ blk_sim,
                   const double* __restrict__ x, const double* __restrict__ m,
                   const double* __restrict__ lam, int64_t ptot,
                   const double* __restrict__ centers, int64_t cstride, int64_t k,
                   const unsigned long long* __restrict__ lmax, double* __restrict__ lsc,
                   float4* __restrict__ vst, float4* __restrict__ vst2) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blk_sim[blockIdx.x];
  const SimMeta M = meta[s];
  const int64_t i = g - M.poff;
  const double sc = lam_scale(lmax[s]);
  if (i == 0) lsc[s] = sc;
  if (i < M.n) {
    const double* c = centers + (int64_t)s * cstride + 3 * k;
    put_vstage(vst, g, (float)(x[g] - c[0]), (float)(x[ptot + g] - c[1]),
               (float)(x[2 * ptot + g] - c[2]), (float)m[g], (float)(sc * lam[g]),
               (float)(sc * lam[ptot + g]), (float)(sc * lam[2 * ptot + g]));
  } else {
    put_vstage(vst, g, kPadPos, kPadPos, kPadPos, 0.f, 0.f, 0.f, 0.f);
    put_vstage(vst2, g, kPadPos, kPadPos, kPadPos, 0.f, 0.f, 0.f, 0.f);
  }
}

// One reverse point k for every simulation: persistent blocks take VJP work
// items (sim, row tile); per row the raw VJP sums Q over all j (FP32 within
// a tile, FP64 across tiles, the single-system kernel's inner step), then
// the adjoint of the point's kick(s) with coefficient ck (G Q and the
// external Hessian product, parameter-gradient terms) and, when drift, of
// the drift that led to it, staging (x_{k-1}, new vbar) into vst_next.
// Per-item sums of the parameter-gradient terms accumulate in blk[item][8]
// (fixed order: one block per item per point, points in sequence); SHAPE
// adds the shape-parameter terms (r_s, a_MN, b_MN), otherwise left at 0.
// The work counter of the next point is re-armed here.
template <bool EQM, bool SHAPE>
__global__ void __launch_bounds__(kVNT, 4)
    k_adj_step_batch(const float4* __restrict__ vst, float4* __restrict__ vst_next,
                     const SimMeta* __restrict__ vmeta, const int4* __restrict__ items,
                     int nitems, unsigned* __restrict__ ctr, unsigned* __restrict__ ctr_next,
                     const DevParams* __restrict__ P, double* __restrict__ xbar,
                     double* __restrict__ vbar, const double* __restrict__ m, int64_t ptot,
                     const double* __restrict__ xk, const double* __restrict__ ak, double ck,
                     int drift, const double* __restrict__ vh_prev,
                     const double* __restrict__ x_prev, const double* __restrict__ centers,
                     int64_t cstride, int64_t k_prev, double* __restrict__ blk,
                     const double* __restrict__ lsc_here, double* __restrict__ lsc_next,
                     const unsigned long long* __restrict__ lmax_here,
                     unsigned long long* __restrict__ lmax_next, int* __restrict__ status) {
  constexpr int NT = kVNT, R = kVR;
  __shared__ float4 sj[4 * kVTJ];
  __shared__ double sred[kAdjCols][NT / 32];
  __shared__ int s_item;
  const int t = threadIdx.x;
  if (blockIdx.x == 0 && t == 0) *ctr_next = 0u;
  bool bad = false;
  for (;;) {
    __syncthreads();
    if (t == 0) s_item = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int4 w = items[it];
    const SimMeta M = vmeta[w.x];
    const float4* vs = vst + 2 * M.poff;  // two float4 per particle
    const int64_t k0 = (int64_t)w.y * (NT * R) + t;
    IState st[R];
    double gx[R], gy[R], gz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      st[r] = load_k(vs, k0 + r * NT);
      gx[r] = gy[r] = gz[r] = 0.0;
    }
    const float2 e2 = make_float2(M.eps2f, M.eps2f);
    for (int tile = 0; tile < M.ntiles; ++tile) {
      __syncthreads();
      const float4* src = vs + (int64_t)tile * (4 * kVTJ);
#pragma unroll
      for (int q = t; q < 4 * kVTJ; q += NT) sj[q] = src[q];
      __syncthreads();
      float2 qa[R][3], qb[R][3];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int d = 0; d < 3; ++d) qa[r][d] = qb[r][d] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int jj = 0; jj < kVTJ; ++jj) {
        const float4 A = sj[4 * jj], B = sj[4 * jj + 1];
        const float4 L1 = sj[4 * jj + 2], L2 = sj[4 * jj + 3];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (EQM)
            vjp_body_eqm(A, B, L1, L2, st[r], e2, qa[r], qb[r]);
          else
            vjp_body(A, B, L1, L2, st[r], e2, qa[r][0], qa[r][1], qa[r][2]);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        gx[r] += (double)qa[r][0].x + (double)qa[r][0].y;
        gy[r] += (double)qa[r][1].x + (double)qa[r][1].y;
        gz[r] += (double)qa[r][2].x + (double)qa[r][2].y;
        if (EQM) {
          gx[r] -= 3.0 * ((double)qb[r][0].x + (double)qb[r][0].y);
          gy[r] -= 3.0 * ((double)qb[r][1].x + (double)qb[r][1].y);
          gz[r] -= 3.0 * ((double)qb[r][2].x + (double)qb[r][2].y);
        }
      }
    }
    const DevParams Q = P[w.x];
    // the scale this point's cotangents were staged with, and the one for
    // the staging of the previous point (from this point's largest |lambda|)
    const double s_here = lsc_here[w.x];
    const double inv_here = 1.0 / s_here;  // a power of two: exact
    const double s_next = drift ? lam_scale(lmax_here[w.x]) : 1.0;
    if (drift && w.y == 0 && t == 0) lsc_next[w.x] = s_next;
    double vmax = 0.0;
    double contrib[kAdjCols] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = k0 + r * NT;
      if (i >= M.n) continue;
      const int64_t g = M.poff + i;
      double lam[3], x[3], ap[3], gv[3];
      const double qs[3] = {gx[r], gy[r], gz[r]};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        lam[d] = vbar[d * ptot + g];
        x[d] = xk[d * ptot + g];
        ap[d] = ak[d * ptot + g];
        gv[d] = -Q.G * M.mscale * (qs[d] * inv_here);
      }
      ExtAdj ea;
      ext_adjoint<SHAPE>(Q, x[0], x[1], x[2], lam, ea);
      const double ckdt = ck * Q.dt;
      double xb[3];
      double lp = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        xb[d] = xbar[d * ptot + g] + ckdt * (gv[d] + ea.jl[d]);
        lp += lam[d] * ap[d];
      }
      const double la = lp + Q.nfw_GM * ea.ln + Q.mn_GM * ea.lm + Q.bulge_GM * ea.lb;
      contrib[0] += ck * la;             // dL/d dt from the kick(s)
      contrib[1] += ckdt * lp;           // sum_j m_j dL/dm_j
      contrib[2] += ckdt * Q.G * ea.ln;  // dL/d M_NFW
      contrib[3] += ckdt * Q.G * ea.lm;  // dL/d M_MN
      contrib[7] += ckdt * Q.G * ea.lb;  // dL/d M_bulge
      if (SHAPE) {                       // dL/d (r_s, a_MN, b_MN)
        contrib[4] += ckdt * ea.sh[0];
        contrib[5] += ckdt * ea.sh[1];
        contrib[6] += ckdt * ea.sh[2];
      }
      double vb[3] = {lam[0], lam[1], lam[2]};
      if (drift) {
        double xv = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          xv += xb[d] * vh_prev[d * ptot + g];
          vb[d] += Q.dt * xb[d];
          vbar[d * ptot + g] = vb[d];
          vmax = fmax(vmax, fabs(vb[d]));
        }
        contrib[0] += xv;             // dL/d dt from the drift
        const double* c = centers + (int64_t)w.x * cstride + 3 * k_prev;
        put_vstage(vst_next, g, (float)(x_prev[g] - c[0]), (float)(x_prev[ptot + g] - c[1]),
                   (float)(x_prev[2 * ptot + g] - c[2]), (float)m[g], (float)(s_next * vb[0]),
                   (float)(s_next * vb[1]), (float)(s_next * vb[2]));
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        xbar[d * ptot + g] = xb[d];
        bad |= !isfinite(xb[d]) || !isfinite(vb[d]);
      }
    }
    // the item's parameter-gradient terms: fixed-order block sum
    const int lane = t & 31, wp = t >> 5;
#pragma unroll
    for (int q = 0; q < kAdjCols; ++q) {
      double v = contrib[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sred[q][wp] = v;
    }
    __syncthreads();
    if (t < kAdjCols) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < NT / 32; ++k) v += sred[t][k];
      blk[(int64_t)it * kAdjCols + t] += v;
    }
    if (drift) block_max_into(vmax, lmax_next + w.x);
  }
  if (bad) atomicOr(status, kStatusNaN);
}

// per-simulation parameter gradient: the sum of its items' rows of blk in
// item order (items of one simulation are contiguous), into out[s][8]
__global__ void k_adj_reduce_batch(const double* __restrict__ blk,
                                   const int* __restrict__ first_item, int n_sims,
                                   double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sims) return;
  for (int q = 0; q < kAdjCols; ++q) {
    double v = 0.0;
    for (int it = first_item[s]; it < first_item[s + 1]; ++it) v += blk[(int64_t)it * kAdjCols + q];
    out[(int64_t)s * kAdjCols + q] = v;
  }
}

// caller layout -> padded (3 x ntot -> 3 x ptot), or back when to_caller
__global__ void k_move_batch(const SimMeta* __restrict__ meta, int n_sims,
                             const double* __restrict__ src, double* __restrict__ dst,
                             int64_t ntot, int64_t ptot, int to_caller) {
  for (int s = blockIdx.y; s < n_sims; s += gridDim.y) {
    const SimMeta M = meta[s];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M.n;
         i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (to_caller)
          dst[d * ntot + M.off + i] = src[d * ptot + M.poff + i];
        else
          dst[d * ptot + M.poff + i] = src[d * ntot + M.off + i];
      }
  }
}

// caller layout (3 x ntot SoA, simulation s at columns off .. off+n-1) ->
// padded state (3 x ptot, simulation s at poff); one grid row per simulation
__global__ void k_gather_batch(const SimMeta* __restrict__ meta, int n_sims,
                               const double* __restrict__ x, const double* __restrict__ v,
                               const double* __restrict__ m, int64_t ntot, int64_t ptot,
                               double* __restrict__ X, double* __restrict__ V,
                               double* __restrict__ Mo) {
  for (int s = blockIdx.y; s < n_sims; s += gridDim.y) {
    const SimMeta M = meta[s];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M.n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        X[d * ptot + M.poff + i] = x[d * ntot + M.off + i];
        V[d * ptot + M.poff + i] = v[d * ntot + M.off + i];
      }
      Mo[M.poff + i] = m[M.off + i];
    }
  }
}

// per-simulation minimum and maximum mass (out[2 s], out[2 s + 1])
__global__ void __launch_bounds__(256)
    k_minmax_batch(const SimMeta* __restrict__ meta, int n_sims, const double* __restrict__ m,
                   double* __restrict__ out) {
  __shared__ double smin[8], smax[8];
  for (int s = blockIdx.x; s < n_sims; s += gridDim.x) {
    const SimMeta M = meta[s];
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = threadIdx.x; i < M.n; i += 256) {
      lo = fmin(lo, m[M.poff + i]);
      hi = fmax(hi, m[M.poff + i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
      smin[threadIdx.x >> 5] = lo;
      smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < 8; ++k) {
        lo = fmin(lo, smin[k]);
        hi = fmax(hi, smax[k]);
      }
      out[2 * s] = lo;
      out[2 * s + 1] = hi;
    }
    __syncthreads();
  }
}

#define BCK(call)                              \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return NBODY_ECUDA; \
  } while (0)

}  // namespace

struct Batch {
  int n_sims = 0;
  int sm_count = 0;
  int64_t ntot = 0, ptot = 0;
  cudaStream_t user = nullptr, gs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<int64_t> n, npad, off, poff;
  std::vector<nbody_params> prm;
  DevParams* dp = nullptr;
  int* mode = nullptr;      // guide (1) or fixed (0) origin per simulation
  double* guide = nullptr;  // [n_sims][6]
  double *x = nullptr, *v = nullptr, *m = nullptr;
  float4* st = nullptr;
  float4* st2 = nullptr;    // second staging buffer of the fused step
  double* part = nullptr;
  size_t part_cap = 0;
  SimMeta* meta = nullptr;
  int* blk_sim = nullptr;
  int4* items = nullptr;
  size_t items_cap = 0;
  int nitems = 0;
  unsigned* ctr = nullptr;
  int* status = nullptr;
  double* centers = nullptr;
  int64_t centers_cap = -1;
  int tune = 0;
  int grid_pair = 0;
  int grid_step = 0;
  bool fused = false;          // every simulation takes one j-chunk: fused steps
  bool eqm = false;            // every simulation has equal masses
  std::vector<double> m_eq;    // their common masses
  cudaGraphExec_t exec = nullptr;
  int64_t exec_steps = -1;
  int exec_tune = -1;
  bool exec_record = false;
  int graph_nodes = 0;
  // reverse sweep
  bool record = false;          // every simulation asks for an adjoint tape
  double* tape = nullptr;       // x, a at points 0..n; vh of steps 0..n-1
  int64_t tape_cap = -1;        // steps the tape holds room for
  int64_t tape_steps = -1;      // steps of the recorded run (-1: none)
  SimMeta* vmeta = nullptr;     // VJP plan: whole j-range per item
  int4* vitems = nullptr;
  int nvitems = 0;
  int grid_vjp = 0;
  std::vector<int> first_item;  // first VJP item of every simulation (+ end)
  int* dfirst = nullptr;
  double *xbar = nullptr, *vbar = nullptr;
  float4 *vst = nullptr, *vst2 = nullptr;
  double* vblk = nullptr;       // [nvitems][kAdjCols]
  double* vlsc = nullptr;       // cotangent scales [2][n_sims] (point parity)
  unsigned long long* vlmax = nullptr;  // their running maxima [2][n_sims]
  double* tbar = nullptr;       // [n_sims][kAdjCols]
  double* cot = nullptr;        // caller-layout scratch of host cotangents
  cudaGraphExec_t vexec = nullptr;
  int64_t vexec_steps = -1;
  bool vexec_eqm = false;
  bool vexec_shape = true;
  int vgraph_nodes = 0;
  bool vplan_valid = false;     // vmeta matches the current masses and eps
  bool vjp_shape = true;        // the sweep also forms dL/d(r_s, a_MN, b_MN)
};

namespace {

template <class T>
int balloc(T** p, size_t count) {
  if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return NBODY_ENOMEM;
  }
  return NBODY_OK;
}

template <class T>
void bfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

DevParams dev_params(const nbody_params& p) {
  DevParams d{};
  d.G = p.G;
  d.eps2 = p.eps * p.eps;
  d.dt = p.dt;
  d.ext = p.ext_flags;
  d.nfw_GM = (p.ext_flags & NBODY_EXT_NFW) ? p.G * p.nfw_M : 0.0;
  d.nfw_rs = (p.ext_flags & NBODY_EXT_NFW) ? p.nfw_rs : 1.0;
  d.mn_GM = (p.ext_flags & NBODY_EXT_MN) ? p.G * p.mn_M : 0.0;
  d.mn_a = p.mn_a;
  d.mn_b = p.mn_b;
  d.eps2f = (float)(p.eps * p.eps);
  if (p.ext_flags & NBODY_EXT_BULGE) set_bulge(d, p.G, p.bulge_M, p.bulge_alpha, p.bulge_rc);
  return d;
}

// calls f(kernel, threads) with the pair kernel of candidate k
template <class F>
cudaError_t with_kernel(const Batch* b, int k, F f) {
  const TuneCfg c = kTune[k];
#define NB_K(NT, R, TJ)                                                         \
  if (c.nt == NT && c.r == R && c.tj == TJ)                                     \
    return b->eqm ? f(k_pair_batch<NT, R, TJ, true>, NT) : f(k_pair_batch<NT, R, TJ, false>, NT);
  NB_K(128, 4, 512) NB_K(128, 2, 512) NB_K(256, 2, 512) NB_K(128, 8, 512)
  NB_K(128, 4, 128) NB_K(128, 2, 128)
#undef NB_K
  return cudaErrorInvalidValue;
}

// calls f(kernel, threads) with the fused step kernel of candidate k
template <class F>
cudaError_t with_step_kernel(const Batch* b, int k, F f) {
  const TuneCfg c = kTune[k];
#define NB_K(NT, R, TJ)                                                         \
  if (c.nt == NT && c.r == R && c.tj == TJ)                                     \
    return b->eqm ? f(k_step_batch<NT, R, TJ, true>, NT) : f(k_step_batch<NT, R, TJ, false>, NT);
  NB_K(128, 4, 512) NB_K(128, 2, 512) NB_K(256, 2, 512) NB_K(128, 8, 512)
  NB_K(128, 4, 128) NB_K(128, 2, 128)
#undef NB_K
  return cudaErrorInvalidValue;
}

// metadata, partial-slice layout and LPT work list for tuning candidate k
int build_plan(Batch* b, int k) {
  const TuneCfg c = kTune[k];
  const int per_block = c.nt * c.r;
  std::vector<SimMeta> meta(b->n_sims);
  struct Item {
    int64_t cost;
    int4 w;
  };
  std::vector<Item> list;
  int64_t part_off = 0;
  for (int s = 0; s < b->n_sims; ++s) {
    SimMeta M{};
    M.npad = b->npad[s];
    M.poff = b->poff[s];
    M.n = b->n[s];
    M.off = b->off[s];
    M.ntiles = (int)(M.npad / (2 * c.tj));
    M.mscale = b->eqm ? b->m_eq[s] : 1.0;
    int S = (int)std::max<int64_t>(1, (M.npad + c.jchunk / 2) / c.jchunk);
    S = std::min(S, M.ntiles);
    M.S = S;
    M.part_off = part_off;
    M.eps2f = (float)(b->prm[s].eps * b->prm[s].eps);
    part_off += (int64_t)S * 3 * M.npad;
    meta[s] = M;
    const int64_t itiles = M.npad / per_block;
    for (int64_t it = 0; it < itiles; ++it)
      for (int q = 0; q < S; ++q) {
        const int64_t tb = ((int64_t)q * M.ntiles) / S, te = ((int64_t)(q + 1) * M.ntiles) / S;
        list.push_back({(te - tb) * per_block, make_int4(s, (int)it, q, 0)});
      }
  }
  std::stable_sort(list.begin(), list.end(),
                   [](const Item& a, const Item& o) { return a.cost > o.cost; });
  if (((size_t)part_off > b->part_cap || list.size() > b->items_cap) && b->exec) {
    // a captured run refers to the buffers about to be replaced
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if ((size_t)part_off > b->part_cap) {
    bfree(b->part);
    b->part_cap = 0;
    int rc = balloc(&b->part, (size_t)part_off);
    if (rc) return rc;
    b->part_cap = (size_t)part_off;
  }
  if (list.size() > b->items_cap) {
    bfree(b->items);
    b->items_cap = 0;
    int rc = balloc(&b->items, list.size());
    if (rc) return rc;
    b->items_cap = list.size();
  }
  std::vector<int4> w(list.size());
  for (size_t i = 0; i < list.size(); ++i) w[i] = list[i].w;
  BCK(cudaMemcpy(b->items, w.data(), w.size() * sizeof(int4), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->meta, meta.data(), meta.size() * sizeof(SimMeta),
                 cudaMemcpyHostToDevice));
  b->nitems = (int)list.size();
  int occ = 1;
  const cudaError_t e = with_kernel(b, k, [&](auto kern, int nt) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, 0);
  });
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  b->grid_pair = std::min(b->nitems, occ * b->sm_count);
  bool fused = true;
  for (const SimMeta& M : meta) fused = fused && M.S == 1;
  if (fused != b->fused && b->exec) {  // the captured run bakes the kernels in
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->fused = fused;
  if (fused) {
    int occ2 = 1;
    const cudaError_t e2 = with_step_kernel(b, k, [&](auto kern, int nt) {
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, kern, nt, 0);
    });
    if (e2 != cudaSuccess || occ2 < 1) {
      cudaGetLastError();
      occ2 = 1;
    }
    b->grid_step = std::min(b->nitems, occ2 * b->sm_count);
  }
  b->tune = k;
  return NBODY_OK;
}

cudaError_t launch_pair_batch(Batch* b, cudaStream_t s) {
  const unsigned g = (unsigned)std::max(1, b->grid_pair);
  const cudaError_t e = with_kernel(b, b->tune, [&](auto kern, int nt) {
    kern<<<g, nt, 0, s>>>(b->st, b->meta, b->items, b->nitems, b->ctr, b->part);
    return cudaGetLastError();
  });
  return e;
}

int ensure_centers(Batch* b, int64_t n_steps) {
  if (b->centers && b->centers_cap >= n_steps) return NBODY_OK;
  bfree(b->centers);
  b->centers_cap = -1;
  int rc = balloc(&b->centers, (size_t)b->n_sims * 3 * (n_steps + 1));
  if (rc) return rc;
  b->centers_cap = n_steps;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return NBODY_OK;
}

// tape slots of point k of a recorded run of n_steps (all NULL when the
// batch does not record)
TapePoint tape_point(const Batch* b, int64_t n_steps, int64_t k) {
  TapePoint tp{nullptr, nullptr, nullptr};
  if (!b->record) return tp;
  const size_t slot = 3 * (size_t)b->ptot;
  tp.x = b->tape + (size_t)k * slot;
  tp.a = b->tape + (size_t)(n_steps + 1 + k) * slot;
  tp.vh = k < n_steps ? b->tape + (size_t)(2 * (n_steps + 1) + k) * slot : nullptr;
  return tp;
}

int ensure_tape(Batch* b, int64_t n_steps) {
  if (!b->record || (b->tape && b->tape_cap == n_steps)) return NBODY_OK;
  if (b->exec) {  // a captured run refers to the buffer about to be replaced
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->vexec) {
    cudaGraphExecDestroy(b->vexec);
    b->vexec = nullptr;
  }
  bfree(b->tape);
  b->tape_cap = -1;
  b->tape_steps = -1;
  int rc = balloc(&b->tape, (size_t)(3 * n_steps + 2) * 3 * (size_t)b->ptot);
  if (rc) return rc;
  b->tape_cap = n_steps;
  return NBODY_OK;
}

// the kernels of one n_steps run, in stream order
int record_run(Batch* b, int64_t n_steps, cudaStream_t s, int* nodes) {
  const int64_t cs = 3 * (b->centers_cap + 1);
  const unsigned nblk = (unsigned)(b->ptot / 256);
  int cnt = 0;
  BCK(cudaMemsetAsync(b->ctr, 0, 2 * sizeof(unsigned), s));
  k_guide_batch<<<(b->n_sims + 63) / 64, 64, 0, s>>>(b->dp, b->mode, b->guide, b->n_sims,
                                                     n_steps, b->centers, cs);
  BCK(cudaGetLastError());
  k_stage_batch<<<nblk, 256, 0, s>>>(b->meta, b->blk_sim, b->x, b->m, b->ptot,
                                     b->centers, cs, b->st, b->fused ? b->st2 : nullptr);
  BCK(cudaGetLastError());
  cnt += 2;
  if (b->fused) {
    // one launch per step: pair sums and update of the same rows
    float4* sbuf[2] = {b->st, b->st2};
    const unsigned g = (unsigned)std::max(1, b->grid_step);
    for (int64_t k = 0; k <= n_steps; ++k) {
      const double kick = (k == 0 || k == n_steps) ? 0.5 : 1.0;
      const int cur = (int)(k & 1);
      BCK(with_step_kernel(b, b->tune, [&](auto kern, int nt) {
        kern<<<g, nt, 0, s>>>(sbuf[cur], sbuf[1 - cur], b->meta, b->items, b->nitems,
                              b->ctr + cur, b->ctr + (1 - cur), b->dp, b->x, b->v, b->ptot,
                              kick, k < n_steps ? 1 : 0, b->centers, cs, k + 1, b->status,
                              tape_point(b, n_steps, k));
        return cudaGetLastError();
      }));
      cnt += 1;
    }
    *nodes = cnt;
    return NBODY_OK;
  }
  for (int64_t k = 0; k <= n_steps; ++k) {
    BCK(launch_pair_batch(b, s));
    const double kick = (k == 0 || k == n_steps) ? 0.5 : 1.0;
    k_update_batch<<<nblk, 256, 0, s>>>(b->dp, b->meta, b->blk_sim, b->x, b->v, b->part,
                                        b->ptot, kick, k < n_steps ? 1 : 0, b->centers,
                                        cs, k + 1, b->st, b->status, b->ctr,
                                        tape_point(b, n_steps, k));
    BCK(cudaGetLastError());
    cnt += 2;
  }
  *nodes = cnt;
  return NBODY_OK;
}

int upload(Batch* b) {
  std::vector<DevParams> d(b->n_sims);
  std::vector<int> mode(b->n_sims);
  bool record = true;
  for (int s = 0; s < b->n_sims; ++s) record = record && b->prm[s].checkpoint_every > 0;
  if (record != b->record && b->exec) {  // the captured run bakes the tape in
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->record = record;
  b->vplan_valid = false;  // eps may have changed
  std::vector<double> g(6 * (size_t)b->n_sims);
  for (int s = 0; s < b->n_sims; ++s) {
    d[s] = dev_params(b->prm[s]);
    mode[s] = b->prm[s].center_mode == NBODY_CENTER_GUIDE ? 1 : 0;
    for (int k = 0; k < 3; ++k) {
      g[6 * s + k] = b->prm[s].center[k];
      g[6 * s + 3 + k] = b->prm[s].center_vel[k];
    }
  }
  BCK(cudaMemcpy(b->dp, d.data(), d.size() * sizeof(DevParams), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->mode, mode.data(), mode.size() * sizeof(int), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->guide, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice));
  // eps is part of the work-list metadata
  return build_plan(b, b->tune);
}

}  // namespace

int batch_create(Batch** out, int n_sims, const int64_t* offsets,
                 const nbody_params* p, cudaStream_t user, int sm_count) {
  Batch* b = new (std::nothrow) Batch();
  if (!b) return NBODY_ENOMEM;
  b->n_sims = n_sims;
  b->sm_count = sm_count;
  b->user = user;
  b->prm.assign(p, p + n_sims);
  b->ntot = offsets[n_sims];
  int64_t poff = 0;
  for (int s = 0; s < n_sims; ++s) {
    const int64_t ns = offsets[s + 1] - offsets[s];
    b->n.push_back(ns);
    b->off.push_back(offsets[s]);
    const int64_t np = ((ns + kPad - 1) / kPad) * kPad;
    b->npad.push_back(np);
    b->poff.push_back(poff);
    poff += np;
  }
  b->ptot = poff;
  const size_t pt = (size_t)b->ptot;
  std::vector<int> bs(pt / 256);
  for (int s = 0; s < n_sims; ++s)
    for (int64_t k = b->poff[s] / 256; k < (b->poff[s] + b->npad[s]) / 256; ++k) bs[k] = s;
  int rc;
  if ((rc = balloc(&b->dp, n_sims)) || (rc = balloc(&b->mode, n_sims)) ||
      (rc = balloc(&b->guide, 6 * (size_t)n_sims)) || (rc = balloc(&b->x, 3 * pt)) ||
      (rc = balloc(&b->v, 3 * pt)) || (rc = balloc(&b->m, pt)) ||
      (rc = balloc(&b->st, pt)) || (rc = balloc(&b->st2, pt)) ||
      (rc = balloc(&b->meta, n_sims)) ||
      (rc = balloc(&b->blk_sim, bs.size())) || (rc = balloc(&b->ctr, 4)) ||
      (rc = balloc(&b->status, 1))) {
    batch_destroy(b);
    return rc;
  }
  if (cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking) ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) ||
      cudaMemset(b->x, 0, 3 * pt * sizeof(double)) ||
      cudaMemset(b->v, 0, 3 * pt * sizeof(double)) ||
      cudaMemset(b->m, 0, pt * sizeof(double)) || cudaMemset(b->status, 0, sizeof(int)) ||
      cudaMemcpy(b->blk_sim, bs.data(), bs.size() * sizeof(int), cudaMemcpyHostToDevice)) {
    cudaGetLastError();
    batch_destroy(b);
    return NBODY_ECUDA;
  }
  rc = upload(b);
  if (rc) {
    batch_destroy(b);
    return rc;
  }
  *out = b;
  return NBODY_OK;
}

void batch_destroy(Batch* b) {
  if (!b) return;
  if (b->gs) cudaStreamSynchronize(b->gs);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->gs) cudaStreamDestroy(b->gs);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  bfree(b->dp); bfree(b->mode); bfree(b->guide); bfree(b->x); bfree(b->v);
  bfree(b->m); bfree(b->st); bfree(b->st2); bfree(b->part); bfree(b->meta); bfree(b->blk_sim);
  bfree(b->items); bfree(b->ctr); bfree(b->status); bfree(b->centers);
  if (b->vexec) cudaGraphExecDestroy(b->vexec);
  bfree(b->tape); bfree(b->vmeta); bfree(b->vitems); bfree(b->dfirst); bfree(b->xbar);
  bfree(b->vbar); bfree(b->vst); bfree(b->vst2); bfree(b->vblk); bfree(b->tbar); bfree(b->cot);
  bfree(b->vlsc); bfree(b->vlmax);
  delete b;
}

int batch_set_params(Batch* b, const nbody_params* p) {
  BCK(cudaStreamSynchronize(b->user));
  BCK(cudaStreamSynchronize(b->gs));
  b->prm.assign(p, p + b->n_sims);
  return upload(b);
}

bool on_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int batch_set_state(Batch* b, const double* x, const double* v, const double* m) {
  // host inputs are first copied whole (three copies), then every
  // simulation is gathered into its padded place by one kernel
  double* tmp = nullptr;
  const bool dev = on_device(x) && on_device(v) && on_device(m);
  if (!dev) {
    BCK(cudaMalloc((void**)&tmp, 7 * (size_t)b->ntot * sizeof(double)));
    const size_t n3 = 3 * (size_t)b->ntot;
    if (cudaMemcpyAsync(tmp, x, n3 * sizeof(double), cudaMemcpyDefault, b->user) ||
        cudaMemcpyAsync(tmp + n3, v, n3 * sizeof(double), cudaMemcpyDefault, b->user) ||
        cudaMemcpyAsync(tmp + 2 * n3, m, (size_t)b->ntot * sizeof(double), cudaMemcpyDefault,
                        b->user)) {
      cudaStreamSynchronize(b->user);
      cudaFree(tmp);
      return NBODY_ECUDA;
    }
    x = tmp;
    v = tmp + n3;
    m = tmp + 2 * n3;
  }
  int64_t nmax = 1;
  for (int s = 0; s < b->n_sims; ++s) nmax = std::max(nmax, b->n[s]);
  dim3 grid((unsigned)std::min<int64_t>((nmax + 255) / 256, 64),
            (unsigned)std::min(b->n_sims, 65535));
  k_gather_batch<<<grid, 256, 0, b->user>>>(b->meta, b->n_sims, x, v, m, b->ntot, b->ptot,
                                            b->x, b->v, b->m);
  count_launch();
  cudaError_t eg = cudaGetLastError();
  // equal masses within every simulation select the kernels that leave the
  // mass out of the pair sums
  double* mm = nullptr;
  if (eg == cudaSuccess &&
      cudaMalloc((void**)&mm, 2 * (size_t)b->n_sims * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    eg = cudaErrorMemoryAllocation;
  }
  if (eg == cudaSuccess) {
    k_minmax_batch<<<(unsigned)std::min(b->n_sims, 65535), 256, 0, b->user>>>(
        b->meta, b->n_sims, b->m, mm);
    count_launch();
    eg = cudaGetLastError();
  }
  std::vector<double> hmm(2 * (size_t)b->n_sims);
  cudaError_t em = cudaSuccess;
  if (eg == cudaSuccess)
    em = cudaMemcpyAsync(hmm.data(), mm, hmm.size() * sizeof(double), cudaMemcpyDeviceToHost,
                         b->user);
  const cudaError_t es = cudaStreamSynchronize(b->user);
  if (mm) cudaFree(mm);
  if (tmp) cudaFree(tmp);
  if (eg != cudaSuccess || em != cudaSuccess || es != cudaSuccess) return NBODY_ECUDA;
  bool eqm = true;
  b->m_eq.assign(b->n_sims, 1.0);
  for (int s = 0; s < b->n_sims; ++s) {
    eqm = eqm && hmm[2 * s] == hmm[2 * s + 1] && hmm[2 * s] > 0.0;
    b->m_eq[s] = hmm[2 * s];
  }
  if (eqm != b->eqm && b->exec) {  // the captured run bakes the kernel in
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->eqm = eqm;
  b->vplan_valid = false;
  b->tape_steps = -1;
  const int rc = build_plan(b, b->tune);  // per-simulation mass scales
  if (rc) return rc;
  // restart every guide from its parameters
  std::vector<double> g(6 * (size_t)b->n_sims);
  for (int s = 0; s < b->n_sims; ++s)
    for (int k = 0; k < 3; ++k) {
      g[6 * s + k] = b->prm[s].center[k];
      g[6 * s + 3 + k] = b->prm[s].center_vel[k];
    }
  BCK(cudaMemcpyAsync(b->guide, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice,
                      b->user));
  BCK(cudaStreamSynchronize(b->user));
  return NBODY_OK;
}

// padded state -> caller layout: one kernel per array into device memory,
// or into a scratch copy and one transfer for host memory
int batch_get_state(Batch* b, double* x, double* v) {
  const size_t n3 = 3 * (size_t)b->ntot;
  dim3 grid((unsigned)std::min<int64_t>(64, (b->ptot / b->n_sims + 255) / 256 + 1),
            (unsigned)std::min(b->n_sims, 65535));
  double* out[2] = {x, v};
  const double* src[2] = {b->x, b->v};
  for (int q = 0; q < 2; ++q) {
    if (!out[q]) continue;
    const bool dev = on_device(out[q]);
    if (!dev && !b->cot) {
      int rc = balloc(&b->cot, n3);
      if (rc) return rc;
    }
    double* p = dev ? out[q] : b->cot;
    k_move_batch<<<grid, 256, 0, b->user>>>(b->meta, b->n_sims, src[q], p, b->ntot, b->ptot, 1);
    BCK(cudaGetLastError());
    count_launch();
    if (!dev) {
      BCK(cudaMemcpyAsync(out[q], b->cot, n3 * sizeof(double), cudaMemcpyDefault, b->user));
      BCK(cudaStreamSynchronize(b->user));  // the scratch is reused
    }
  }
  BCK(cudaStreamSynchronize(b->user));
  return NBODY_OK;
}

int batch_integrate(Batch* b, int64_t n_steps) {
  int rc = ensure_centers(b, n_steps);
  if (rc) return rc;
  if ((rc = ensure_tape(b, n_steps))) return rc;
  b->tape_steps = -1;
  if (!b->exec || b->exec_steps != n_steps || b->exec_tune != b->tune ||
      b->exec_record != b->record) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal));
    int nodes = 0;
    rc = record_run(b, n_steps, b->gs, &nodes);
    cudaError_t e = cudaStreamEndCapture(b->gs, &graph);
    if (rc || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : NBODY_ECUDA;
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return NBODY_ECUDA;
    }
    b->exec_steps = n_steps;
    b->exec_tune = b->tune;
    b->exec_record = b->record;
    b->graph_nodes = nodes;
  }
  BCK(cudaEventRecord(b->ev_in, b->user));
  BCK(cudaStreamWaitEvent(b->gs, b->ev_in, 0));
  BCK(cudaGraphLaunch(b->exec, b->gs));
  BCK(cudaEventRecord(b->ev_out, b->gs));
  BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  count_launch(b->graph_nodes);
  if (b->record) b->tape_steps = n_steps;
  return NBODY_OK;
}

namespace {

// calls f(kernel) with the reverse-point kernel for the batch's masses and
// gradient set
template <class F>
cudaError_t with_adj_kernel(const Batch* b, F f) {
  if (b->eqm) return b->vjp_shape ? f(k_adj_step_batch<true, true>) : f(k_adj_step_batch<true, false>);
  return b->vjp_shape ? f(k_adj_step_batch<false, true>) : f(k_adj_step_batch<false, false>);
}

// VJP plan and reverse-sweep buffers (once per batch)
int ensure_vjp_plan(Batch* b) {
  if (b->vmeta && b->vplan_valid) return NBODY_OK;
  const int per_block = kVNT * kVR;
  std::vector<SimMeta> vm(b->n_sims);
  std::vector<int4> items;
  b->first_item.assign(b->n_sims + 1, 0);
  for (int s = 0; s < b->n_sims; ++s) {
    SimMeta M{};
    M.npad = b->npad[s];
    M.poff = b->poff[s];
    M.n = b->n[s];
    M.off = b->off[s];
    M.S = 1;
    M.ntiles = (int)(M.npad / (2 * kVTJ));
    M.eps2f = (float)(b->prm[s].eps * b->prm[s].eps);
    M.mscale = b->eqm ? b->m_eq[s] : 1.0;
    vm[s] = M;
    b->first_item[s] = (int)items.size();
    for (int64_t it = 0; it < M.npad / per_block; ++it) items.push_back(make_int4(s, (int)it, 0, 0));
  }
  b->first_item[b->n_sims] = (int)items.size();
  b->nvitems = (int)items.size();
  const size_t pt = (size_t)b->ptot;
  int rc;
  if (!b->vmeta &&
      ((rc = balloc(&b->vitems, items.size())) ||
       (rc = balloc(&b->dfirst, b->first_item.size())) || (rc = balloc(&b->xbar, 3 * pt)) ||
       (rc = balloc(&b->vbar, 3 * pt)) || (rc = balloc(&b->vst, 2 * pt)) ||
       (rc = balloc(&b->vst2, 2 * pt)) ||
       (rc = balloc(&b->vblk, (size_t)b->nvitems * kAdjCols)) ||
       (rc = balloc(&b->tbar, (size_t)b->n_sims * kAdjCols)) ||
       (rc = balloc(&b->vlsc, 2 * (size_t)b->n_sims)) ||
       (rc = balloc(&b->vlmax, 2 * (size_t)b->n_sims)) ||
       (rc = balloc(&b->vmeta, (size_t)b->n_sims))))
    return rc;
  BCK(cudaMemcpyAsync(b->vmeta, vm.data(), vm.size() * sizeof(SimMeta), cudaMemcpyHostToDevice,
                      b->gs));
  BCK(cudaMemcpyAsync(b->vitems, items.data(), items.size() * sizeof(int4),
                      cudaMemcpyHostToDevice, b->gs));
  BCK(cudaMemcpyAsync(b->dfirst, b->first_item.data(), b->first_item.size() * sizeof(int),
                      cudaMemcpyHostToDevice, b->gs));
  BCK(cudaStreamSynchronize(b->gs));
  int occ = 1;
  const cudaError_t e = with_adj_kernel(b, [&](auto kern) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kVNT, 0);
  });
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  b->grid_vjp = std::min(b->nvitems, occ * b->sm_count);
  b->vplan_valid = true;
  return NBODY_OK;
}

// the kernels of the reverse sweep over a recorded run of n_steps
int record_sweep(Batch* b, int64_t n_steps, cudaStream_t s, int* nodes) {
  const int64_t cs = 3 * (b->centers_cap + 1);
  const unsigned nblk = (unsigned)(b->ptot / 256);
  const int ns_ = b->n_sims;
  BCK(cudaMemsetAsync(b->ctr + 2, 0, 2 * sizeof(unsigned), s));
  BCK(cudaMemsetAsync(b->vblk, 0, (size_t)b->nvitems * kAdjCols * sizeof(double), s));
  BCK(cudaMemsetAsync(b->vlmax, 0, 2 * (size_t)ns_ * sizeof(unsigned long long), s));
  const TapePoint tn = tape_point(b, n_steps, n_steps);
  const int sl_n = (int)(n_steps & 1);
  k_vabsmax_batch<<<nblk, 256, 0, s>>>(b->meta, b->blk_sim, b->vbar, b->ptot,
                                       b->vlmax + (size_t)sl_n * ns_);
  BCK(cudaGetLastError());
  k_vstage_batch<<<nblk, 256, 0, s>>>(b->meta, b->blk_sim, tn.x, b->m, b->vbar, b->ptot,
                                      b->centers, cs, n_steps, b->vlmax + (size_t)sl_n * ns_,
                                      b->vlsc + (size_t)sl_n * ns_, b->vst, b->vst2);
  BCK(cudaGetLastError());
  float4* vbuf[2] = {b->vst, b->vst2};
  const unsigned g = (unsigned)std::max(1, b->grid_vjp);
  int cnt = 2;
  for (int64_t k = n_steps; k >= 0; --k) {
    const int cur = (int)((n_steps - k) & 1);
    const size_t here = (size_t)(k & 1) * ns_, next = (size_t)(1 - (k & 1)) * ns_;
    // the maxima of the cotangents staged now start from zero
    BCK(cudaMemsetAsync(b->vlmax + next, 0, (size_t)ns_ * sizeof(unsigned long long), s));
    const TapePoint tk = tape_point(b, n_steps, k);
    const TapePoint tp = k > 0 ? tape_point(b, n_steps, k - 1) : TapePoint{nullptr, nullptr, nullptr};
    const double ck = (k == n_steps || k == 0) ? 0.5 : 1.0;
    const int drift = k > 0 ? 1 : 0;
    BCK(with_adj_kernel(b, [&](auto kern) {
      kern<<<g, kVNT, 0, s>>>(vbuf[cur], vbuf[1 - cur], b->vmeta, b->vitems, b->nvitems,
                              b->ctr + 2 + cur, b->ctr + 2 + (1 - cur), b->dp, b->xbar, b->vbar,
                              b->m, b->ptot, tk.x, tk.a, ck, drift, tp.vh, tp.x, b->centers, cs,
                              k > 0 ? k - 1 : 0, b->vblk, b->vlsc + here, b->vlsc + next,
                              b->vlmax + here, b->vlmax + next, b->status);
      return cudaGetLastError();
    }));
    ++cnt;
  }
  k_adj_reduce_batch<<<(b->n_sims + 127) / 128, 128, 0, s>>>(b->vblk, b->dfirst, b->n_sims,
                                                             b->tbar);
  BCK(cudaGetLastError());
  *nodes = cnt + 1;
  return NBODY_OK;
}

}  // namespace

void batch_set_vjp_shape(Batch* b, bool on) {
  if (on != b->vjp_shape) b->vplan_valid = false;  // the occupancy differs
  b->vjp_shape = on;
}

int batch_vjp(Batch* b, const double* xbar, const double* vbar, double* x0bar, double* v0bar,
              double* theta_bar) {
  if (!b->record || b->tape_steps < 0) return NBODY_ESTATE;
  const int64_t n_steps = b->tape_steps;
  int rc = ensure_vjp_plan(b);
  if (rc) return rc;
  // the sweep runs on the batch's stream after the caller's work so far
  BCK(cudaEventRecord(b->ev_in, b->user));
  BCK(cudaStreamWaitEvent(b->gs, b->ev_in, 0));
  const size_t n3 = 3 * (size_t)b->ntot;
  // cotangents of the final state into the padded layout (host arrays go
  // through one scratch copy)
  const double* src[2] = {xbar, vbar};
  double* dst[2] = {b->xbar, b->vbar};
  dim3 grid((unsigned)std::min<int64_t>(64, (b->ptot / b->n_sims + 255) / 256 + 1),
            (unsigned)std::min(b->n_sims, 65535));
  for (int q = 0; q < 2; ++q) {
    BCK(cudaMemsetAsync(dst[q], 0, 3 * (size_t)b->ptot * sizeof(double), b->gs));
    if (!src[q]) continue;
    const double* p = src[q];
    if (!on_device(p)) {
      if (!b->cot && (rc = balloc(&b->cot, n3))) return rc;
      BCK(cudaMemcpyAsync(b->cot, p, n3 * sizeof(double), cudaMemcpyDefault, b->gs));
      p = b->cot;
    }
    k_move_batch<<<grid, 256, 0, b->gs>>>(b->meta, b->n_sims, p, dst[q], b->ntot, b->ptot, 0);
    BCK(cudaGetLastError());
    if (p == b->cot) BCK(cudaStreamSynchronize(b->gs));  // the scratch is reused
  }
  count_launch(2);
  if (!b->vexec || b->vexec_steps != n_steps || b->vexec_eqm != b->eqm ||
      b->vexec_shape != b->vjp_shape) {
    if (b->vexec) {
      cudaGraphExecDestroy(b->vexec);
      b->vexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal));
    int nodes = 0;
    rc = record_sweep(b, n_steps, b->gs, &nodes);
    cudaError_t e = cudaStreamEndCapture(b->gs, &graph);
    if (rc || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : NBODY_ECUDA;
    }
    e = cudaGraphInstantiate(&b->vexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->vexec = nullptr;
      return NBODY_ECUDA;
    }
    b->vexec_steps = n_steps;
    b->vexec_eqm = b->eqm;
    b->vexec_shape = b->vjp_shape;
    b->vgraph_nodes = nodes;
  }
  BCK(cudaGraphLaunch(b->vexec, b->gs));
  count_launch(b->vgraph_nodes);
  double* out[2] = {x0bar, v0bar};
  const double* res[2] = {b->xbar, b->vbar};
  for (int q = 0; q < 2; ++q) {
    if (!out[q]) continue;
    double* p = out[q];
    const bool dev = on_device(p);
    if (!dev) {
      if (!b->cot && (rc = balloc(&b->cot, n3))) return rc;
      p = b->cot;
    }
    k_move_batch<<<grid, 256, 0, b->gs>>>(b->meta, b->n_sims, res[q], p, b->ntot, b->ptot, 1);
    BCK(cudaGetLastError());
    count_launch();
    if (!dev) {
      BCK(cudaMemcpyAsync(out[q], b->cot, n3 * sizeof(double), cudaMemcpyDefault, b->gs));
      BCK(cudaStreamSynchronize(b->gs));
    }
  }
  if (theta_bar)
    BCK(cudaMemcpyAsync(theta_bar, b->tbar, (size_t)b->n_sims * kAdjCols * sizeof(double),
                        cudaMemcpyDefault, b->gs));
  BCK(cudaStreamSynchronize(b->gs));
  return batch_status(b);
}

int batch_clear_status(Batch* b) {
  BCK(cudaMemsetAsync(b->status, 0, sizeof(int), b->gs));
  BCK(cudaStreamSynchronize(b->gs));
  return NBODY_OK;
}

int batch_status(Batch* b) {
  int st = 0;
  BCK(cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->gs));
  BCK(cudaStreamSynchronize(b->gs));
  return (st & kStatusNaN) ? NBODY_ENAN : NBODY_OK;
}

int batch_set_tuning(Batch* b, int k) {
  if (k < 0 || k >= NBODY_NTUNE) return NBODY_EINVAL;
  BCK(cudaStreamSynchronize(b->user));
  BCK(cudaStreamSynchronize(b->gs));
  return build_plan(b, k);
}

int batch_autotune(Batch* b, int64_t probe_steps, int* best, double* ms_out) {
  if (probe_steps < 1) probe_steps = 1;
  BCK(cudaStreamSynchronize(b->user));
  BCK(cudaStreamSynchronize(b->gs));
  int rc = ensure_centers(b, 0);
  if (rc) return rc;
  // stage the current positions once (pair forces only: the state is not
  // advanced)
  const int64_t cs = 3 * (b->centers_cap + 1);
  k_guide_batch<<<(b->n_sims + 63) / 64, 64, 0, b->gs>>>(b->dp, b->mode, b->guide, b->n_sims,
                                                         0, b->centers, cs);
  BCK(cudaGetLastError());
  k_stage_batch<<<(unsigned)(b->ptot / 256), 256, 0, b->gs>>>(b->meta, b->blk_sim, b->x, b->m,
                                                              b->ptot, b->centers, cs, b->st, nullptr);
  BCK(cudaGetLastError());
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  double best_ms = 1e300;
  int best_k = b->tune;
  // one probe = a whole step of the candidate (fused, or pair + update) with
  // zero kick and no drift, which leaves positions and velocities as they are
  const unsigned nblk = (unsigned)(b->ptot / 256);
  auto probe = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(b->ctr, 0, 2 * sizeof(unsigned), b->gs);
    if (e != cudaSuccess) return e;
    if (b->fused) {
      const unsigned g = (unsigned)std::max(1, b->grid_step);
      return with_step_kernel(b, b->tune, [&](auto kern, int nt) {
        kern<<<g, nt, 0, b->gs>>>(b->st, b->st2, b->meta, b->items, b->nitems, b->ctr,
                                  b->ctr + 1, b->dp, b->x, b->v, b->ptot, 0.0, 0, b->centers,
                                  cs, 0, b->status, TapePoint{nullptr, nullptr, nullptr});
        return cudaGetLastError();
      });
    }
    e = launch_pair_batch(b, b->gs);
    if (e != cudaSuccess) return e;
    k_update_batch<<<nblk, 256, 0, b->gs>>>(b->dp, b->meta, b->blk_sim, b->x, b->v, b->part,
                                            b->ptot, 0.0, 0, b->centers, cs, 0, b->st,
                                            b->status, b->ctr, TapePoint{nullptr, nullptr, nullptr});
    return cudaGetLastError();
  };
  for (int k = 0; k < NBODY_NTUNE; ++k) {
    rc = build_plan(b, k);
    if (rc) break;
    BCK(probe());  // warm-up
    BCK(cudaEventRecord(e0, b->gs));
    for (int64_t q = 0; q < probe_steps; ++q) BCK(probe());
    BCK(cudaEventRecord(e1, b->gs));
    BCK(cudaEventSynchronize(e1));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, e0, e1));
    const double per = (double)ms / (double)probe_steps;
    if (ms_out) ms_out[k] = per;
    if (per < best_ms) {
      best_ms = per;
      best_k = k;
    }
  }
  count_launch(2 + 2 * NBODY_NTUNE * (int)(probe_steps + 1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = build_plan(b, best_k);
  if (rc) return rc;
  if (best) *best = best_k;
  return NBODY_OK;
}

int batch_tuning(Batch* b) { return b->tune; }

}  // namespace nb
