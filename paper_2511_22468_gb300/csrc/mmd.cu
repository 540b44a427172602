// mmd.cu -- maximum mean discrepancy between phase-space point clouds
// (paper Sec. 2.2.1, Fig. 2 step 4: the simulated and the observed stream
// compared as point clouds; the grid search ranks parameter vectors by it).
//
// A point is q = (x, y, z, vx, vy, vz).  Coordinates are standardised by
// the target cloud's per-dimension mean mu and standard deviation s (or a
// caller's scale) and the kernel is a sum of Gaussians,
//   k(a, b) = sum_l exp(-|u_a - u_b|^2 / (2 sigma_l^2)),  u = (q - mu) / s.
// The biased estimator over the union Z = X u Y with weights w = 1/n on X
// and -1/m on Y is MMD^2 = sum_{a,b in Z} w_a w_b k(a, b), and
//   dMMD^2/du_i = 2 w_i sum_b w_b dk(u_i, u_b)/du_i.
//
// GPU form.  The staged coordinates are u' = u sqrt(c0) with
// c0 = log2(e) / (2 sigma_0^2), sigma_0 the smallest bandwidth, so that
// k = sum_l exp2(-rho_l |u'_a - u'_b|^2) with rho_l = sigma_0^2/sigma_l^2 <= 1:
// one MUFU ex2 per bandwidth and pair.  A row kernel holds R points of X in
// registers and sweeps column tiles of X (weight 1/n) and of Y (weight -1/m)
// through shared memory, accumulating in FP32 within a tile (packed f32x2:
// two columns per instruction) and in FP64 across tiles:
//   S0A_i = sum_{j in X} w_j k_ij, S0B_i = sum_{j in Y} w_j k_ij,
//   S1_i  = sum_j w_j (sum_l rho_l k_l,ij) (u'_j - u'_i).
// Then MMD^2 = Kyy + sum_i (1/n) (S0A_i + 2 S0B_i) (the Y-Y term Kyy once at
// creation) and dMMD^2/du'_i = 4 ln2 (1/n) S1_i.  Column pads sit at 1e18,
// where every kernel value is exactly zero.  Sums are in fixed order, so
// results are bitwise reproducible.  Per pair: 19 FP32-pipe operations and
// one MUFU for one bandwidth, 4 operations and one MUFU more per extra one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "nbody_internal.cuh"
#include "staging.cuh"

namespace nb {
namespace {

constexpr int kMT = 256;          // column pairs per shared-memory tile
constexpr int kMPts = 2 * kMT;    // points per tile (padding unit)
constexpr int kMaxSigma = 4;

struct Standardise {
  double mu[6];
  double f[6];  // sqrt(c0) / s_d
};

static __device__ __forceinline__ float ex2_ftz(float v) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
  return y;
}

// pair p of a staged cloud: 3 float4 = (u0,u0',u1,u1'), (u2,..), (u4,..)
static __device__ __forceinline__ float load_u(const float4* st, int64_t i, int d) {
  const float* f = reinterpret_cast<const float*>(st) + 12 * (i >> 1) + (i & 1);
  return f[2 * d];
}

// Stage sets of n points into pair-interleaved FP32 records, npad per set.
// x, v: 3 x ld SoA; set b's point i is column b * n + i.
__global__ void k_mmd_stage(const double* __restrict__ x, const double* __restrict__ v,
                            int64_t ld, int64_t n, int64_t npad, Standardise S,
                            float4* __restrict__ st) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // pair
  const int64_t b = blockIdx.y;
  if (2 * p >= npad) return;
  float u[2][6];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t i = 2 * p + h;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (i < n) {
        const double q = d < 3 ? x[d * ld + b * n + i] : v[(d - 3) * ld + b * n + i];
        u[h][d] = (float)((q - S.mu[d]) * S.f[d]);
      } else {
        u[h][d] = kPadPos;
      }
    }
  }
  float4* o = st + b * (3 * (npad / 2)) + 3 * p;
  o[0] = make_float4(u[0][0], u[1][0], u[0][1], u[1][1]);
  o[1] = make_float4(u[0][2], u[1][2], u[0][3], u[1][3]);
  o[2] = make_float4(u[0][4], u[1][4], u[0][5], u[1][5]);
}

// Row sums.  Grid: x = row blocks of NT*R points, y = set, z = column chunk.
// Rows of set b: rows + b * rstride; columns: ntA tiles of colA + b * astride
// then ntB tiles of colB + b * bstride.  part: [set][chunk][8][npad_r] FP64 (S0A, S0B, S1).
template <int R, int NS>
__global__ void __launch_bounds__(128)
    k_mmd_rows(const float4* __restrict__ rows, int64_t rstride, int64_t npad_r,
               const float4* __restrict__ colA, int64_t astride, int ntA,
               const float4* __restrict__ colB, int64_t bstride, int ntB, double wA,
               double wB, float4 rho, double* __restrict__ part) {
  constexpr int NT = 128;
  __shared__ float4 sj[3 * kMT];
  const int t = threadIdx.x;
  const int64_t b = blockIdx.y;
  const int S = gridDim.z;
  const int nt = ntA + ntB;
  const int tile_b = (int)(((int64_t)blockIdx.z * nt) / S);
  const int tile_e = (int)(((int64_t)(blockIdx.z + 1) * nt) / S);
  const float4* rs = rows + b * rstride;
  const float4* ca = colA + b * astride;
  const float4* cb = colB + b * bstride;
  const int64_t i0 = (int64_t)blockIdx.x * (NT * R) + t;

  float2 nu[R][6];
  double s0a[R], s0b[R], s1[R][6];
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const float u = load_u(rs, i0 + r * NT, d);
      nu[r][d] = make_float2(-u, -u);
      s1[r][d] = 0.0;
    }
    s0a[r] = s0b[r] = 0.0;
  }
  const float rl[4] = {1.f, rho.y, rho.z, rho.w};

  for (int tile = tile_b; tile < tile_e; ++tile) {
    const bool inA = tile < ntA;
    const float4* src = inA ? ca + (int64_t)tile * (3 * kMT)
                            : cb + (int64_t)(tile - ntA) * (3 * kMT);
    __syncthreads();
    for (int q = t; q < 3 * kMT; q += NT) sj[q] = src[q];
    __syncthreads();

    float2 a0[R], a1[R][6];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      a0[r] = make_float2(0.f, 0.f);
#pragma unroll
      for (int d = 0; d < 6; ++d) a1[r][d] = make_float2(0.f, 0.f);
    }
#pragma unroll 2
    for (int jj = 0; jj < kMT; ++jj) {
      const float4 P0 = sj[3 * jj], P1 = sj[3 * jj + 1], P2 = sj[3 * jj + 2];
      const float2 c[6] = {make_float2(P0.x, P0.y), make_float2(P0.z, P0.w),
                           make_float2(P1.x, P1.y), make_float2(P1.z, P1.w),
                           make_float2(P2.x, P2.y), make_float2(P2.z, P2.w)};
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 dd[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) dd[d] = __fadd2_rn(c[d], nu[r][d]);
        float2 r2 = __fmul2_rn(dd[0], dd[0]);
#pragma unroll
        for (int d = 1; d < 6; ++d) r2 = __ffma2_rn(dd[d], dd[d], r2);
        float2 sk = make_float2(ex2_ftz(-r2.x), ex2_ftz(-r2.y));
        float2 sg = sk;
#pragma unroll
        for (int l = 1; l < NS; ++l) {
          const float2 rr = make_float2(rl[l], rl[l]);
          const float2 e = __fmul2_rn(r2, rr);
          const float2 kl = make_float2(ex2_ftz(-e.x), ex2_ftz(-e.y));
          sk = __fadd2_rn(sk, kl);
          sg = __ffma2_rn(kl, rr, sg);
        }
        a0[r] = __fadd2_rn(a0[r], sk);
#pragma unroll
        for (int d = 0; d < 6; ++d) a1[r][d] = __ffma2_rn(sg, dd[d], a1[r][d]);
      }
    }
    const double w = inA ? wA : wB;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double k0 = (double)(a0[r].x + a0[r].y);
      if (inA)
        s0a[r] = fma(w, k0, s0a[r]);
      else
        s0b[r] = fma(w, k0, s0b[r]);
#pragma unroll
      for (int d = 0; d < 6; ++d) s1[r][d] = fma(w, (double)(a1[r][d].x + a1[r][d].y), s1[r][d]);
    }
  }

  double* p = part + ((int64_t)b * S + blockIdx.z) * 8 * npad_r;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i0 + r * NT;
    p[i] = s0a[r];
    p[npad_r + i] = s0b[r];
#pragma unroll
    for (int d = 0; d < 6; ++d) p[(2 + d) * npad_r + i] = s1[r][d];
  }
}

// Loss-only kernel sums between clouds: block (x, a, c) sums k(u_i, u_j)
// over its rows i of row set a (NT*R rows from x * NT*R; rows >= n_r are
// pads and left out) and every column j of column set (a, c) (nct tiles;
// pad columns add exactly 0), FP32 within a tile, FP64 across tiles, then a
// fixed-order block reduction into out[(c * gridDim.y + a) * gridDim.x + x].
// Rows of set a: rows + a * rstride; columns: cols + a * cas + c * ccs (a
// cloud against itself: cas = rstride, ccs = 0; clouds against other
// clouds: cas = 0, ccs = their stride).  The squared distance is expanded,
// |u_i - u_j|^2 = |u_i'|^2 + |u_j'|^2 - 2 u_i' . u_j' with u' = u - c, c the
// row set's first point, and the column norms formed once per tile in
// shared memory: per two pairs one packed add and six packed FMAs instead
// of twelve operations.  The expansion's rounding error, about |u'|^2 2^-24,
// matters only for near pairs, whose u' are of the size of the clouds'
// extent.  Per two pairs: 8 + 2 (NS - 1) + 1 FP32-pipe instructions and
// 2 NS ex2 (the ex2 unit bounds it).
template <int R, int NS>
__global__ void __launch_bounds__(128)
    k_mmd_sum(const float4* __restrict__ rows, int64_t rstride, int64_t n_r,
              const float4* __restrict__ cols, int64_t cas, int64_t ccs, int nct, float4 rho,
              double* __restrict__ out) {
  constexpr int NT = 128;
  __shared__ float4 sj[3 * kMT];
  __shared__ float2 snb[kMT];  // column norms |u_j|^2 of the tile's pairs
  __shared__ double sw[NT / 32];
  const int t = threadIdx.x;
  const int64_t a = blockIdx.y, c = blockIdx.z;
  const float4* rs = rows + a * rstride;
  const float4* cs = cols + a * cas + c * ccs;
  const int64_t i0 = (int64_t)blockIdx.x * (NT * R) + t;
  // distances are formed relative to the row set's first point, so that
  // the norms stay of the size of the clouds' extent rather than of their
  // offset from the standardisation origin (the expansion's rounding error
  // scales with the norms)
  float cr[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) cr[d] = load_u(rs, 0, d);
  const float4 cq0 = make_float4(cr[0], cr[0], cr[1], cr[1]);
  const float4 cq1 = make_float4(cr[2], cr[2], cr[3], cr[3]);
  const float4 cq2 = make_float4(cr[4], cr[4], cr[5], cr[5]);
  float2 m2u[R][6], na[R];  // -2 (u_i - c) and |u_i - c|^2, both lanes alike
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float n2 = 0.f;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const float u = load_u(rs, i0 + r * NT, d) - cr[d];
      m2u[r][d] = make_float2(-2.f * u, -2.f * u);
      n2 = fmaf(u, u, n2);
    }
    na[r] = make_float2(n2, n2);
  }
  const float rl[4] = {1.f, rho.y, rho.z, rho.w};
  double s0[R];
#pragma unroll
  for (int r = 0; r < R; ++r) s0[r] = 0.0;
  for (int tile = 0; tile < nct; ++tile) {
    const float4* src = cs + (int64_t)tile * (3 * kMT);
    __syncthreads();
    for (int q = t; q < 3 * kMT; q += NT) {
      const int k3 = q % 3;
      const float4 v = src[q], c = k3 == 0 ? cq0 : (k3 == 1 ? cq1 : cq2);
      sj[q] = make_float4(v.x - c.x, v.y - c.y, v.z - c.z, v.w - c.w);
    }
    __syncthreads();
    for (int q = t; q < kMT; q += NT) {
      const float4 P0 = sj[3 * q], P1 = sj[3 * q + 1], P2 = sj[3 * q + 2];
      float2 n2 = make_float2(P0.x * P0.x, P0.y * P0.y);
      n2 = __ffma2_rn(make_float2(P0.z, P0.w), make_float2(P0.z, P0.w), n2);
      n2 = __ffma2_rn(make_float2(P1.x, P1.y), make_float2(P1.x, P1.y), n2);
      n2 = __ffma2_rn(make_float2(P1.z, P1.w), make_float2(P1.z, P1.w), n2);
      n2 = __ffma2_rn(make_float2(P2.x, P2.y), make_float2(P2.x, P2.y), n2);
      n2 = __ffma2_rn(make_float2(P2.z, P2.w), make_float2(P2.z, P2.w), n2);
      snb[q] = n2;
    }
    __syncthreads();
    float2 a0[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a0[r] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int jj = 0; jj < kMT; ++jj) {
      const float4 P0 = sj[3 * jj], P1 = sj[3 * jj + 1], P2 = sj[3 * jj + 2];
      const float2 nb2 = snb[jj];
      const float2 cc[6] = {make_float2(P0.x, P0.y), make_float2(P0.z, P0.w),
                            make_float2(P1.x, P1.y), make_float2(P1.z, P1.w),
                            make_float2(P2.x, P2.y), make_float2(P2.z, P2.w)};
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 r2 = __fadd2_rn(na[r], nb2);
#pragma unroll
        for (int d = 0; d < 6; ++d) r2 = __ffma2_rn(cc[d], m2u[r][d], r2);
        float2 sk = make_float2(ex2_ftz(-r2.x), ex2_ftz(-r2.y));
#pragma unroll
        for (int l = 1; l < NS; ++l) {
          const float2 e = __fmul2_rn(r2, make_float2(rl[l], rl[l]));
          sk = __fadd2_rn(sk, make_float2(ex2_ftz(-e.x), ex2_ftz(-e.y)));
        }
        a0[r] = __fadd2_rn(a0[r], sk);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) s0[r] += (double)(a0[r].x + a0[r].y);
  }
  double acc = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (i0 + r * NT < n_r) acc += s0[r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((t & 31) == 0) sw[t >> 5] = acc;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) tot += sw[w];
    out[(c * gridDim.y + a) * gridDim.x + blockIdx.x] = tot;
  }
}

// per-set sums of k_mmd_sum's block sums: res[q] = w * sum_x bs[q * nrb + x]
__global__ void k_mmd_block_total(const double* __restrict__ bs, int64_t count, int nrb,
                                  double w, double* __restrict__ res) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double s = 0.0;
  for (int x = 0; x < nrb; ++x) s += bs[q * nrb + x];
  res[q] = w * s;
}

// loss[t * sets + b] = kxx[b] + kyy[t] - 2/(n m) sum_x cross[(t sets + b) nrb + x]
__global__ void k_mmd_cross_finish(const double* __restrict__ cross, int64_t sets,
                                   int64_t targets, int nrb, double wxy,
                                   const double* __restrict__ kxx,
                                   const double* __restrict__ kyy, double* __restrict__ loss) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= sets * targets) return;
  const int64_t b = q % sets, t = q / sets;
  double s = 0.0;
  for (int x = 0; x < nrb; ++x) s += cross[q * nrb + x];
  loss[q] = kxx[b] + kyy[t] - wxy * s;
}

// loss_b = base[b * base_stride] + wrow sum_{i<n} sum_chunks (S0A + cB S0B),
// one block per set
__global__ void __launch_bounds__(256)
    k_mmd_finish(const double* __restrict__ part, int S, int64_t npad_r, int64_t n,
                 double wrow, double cB, const double* __restrict__ base, int base_stride,
                 double* __restrict__ loss) {
  __shared__ double sh[256];
  const int64_t b = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) {
    double r = 0.0;
    for (int q = 0; q < S; ++q) {
      const double* p = part + ((int64_t)b * S + q) * 8 * npad_r;
      r += p[i] + cB * p[npad_r + i];
    }
    acc += r;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[b] = (base ? base[b * base_stride] : 0.0) + wrow * sh[0];
}

// dMMD^2/dq of set b = blockIdx.y: gscale_d = 4 ln2 (1/n) f_d; out 3 x ld
// each, set b in columns b n .. b n + n - 1
__global__ void k_mmd_grad(const double* __restrict__ part, int S, int64_t npad_r,
                           int64_t n, int64_t ld, Standardise Sd, double g0,
                           double* __restrict__ xbar, double* __restrict__ vbar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  if (i >= n) return;
  const double* pb = part + b * S * 8 * npad_r;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += pb[((int64_t)q * 8 + 2 + d) * npad_r + i];
    const double g = g0 * Sd.f[d] * s;
    if (d < 3)
      xbar[d * ld + b * n + i] = g;
    else
      vbar[(d - 3) * ld + b * n + i] = g;
  }
}

// mean and standard deviation per dimension of a cloud (3 x m x, 3 x m v),
// one block, two passes, fixed order
__global__ void __launch_bounds__(256)
    k_cloud_stats(const double* __restrict__ x, const double* __restrict__ v, int64_t m,
                  double* __restrict__ out) {
  __shared__ double sh[256];
  for (int d = 0; d < 6; ++d) {
    const double* q = d < 3 ? x + d * m : v + (d - 3) * m;
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += 256) a += q[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    const double mu = sh[0] / (double)m;
    __syncthreads();
    a = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += 256) a += (q[i] - mu) * (q[i] - mu);
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[d] = mu;
      out[6 + d] = sqrt(sh[0] / (double)m);
    }
    __syncthreads();
  }
}

int64_t pad_points(int64_t n) { return ((n + kMPts - 1) / kMPts) * kMPts; }

}  // namespace
}  // namespace nb

struct nbody_mmd {
  cudaStream_t s = nullptr;
  int64_t n = 0, m = 0, max_sets = 0, npad = 0, mpad = 0;
  int ns = 1;
  double sigma[4] = {0, 0, 0, 0};  // the caller's bandwidths, in its order
  float4 rho{1.f, 1.f, 1.f, 1.f};
  double c0 = 0.0;
  nb::Standardise st{};
  int sms = 0;
  float4* xs = nullptr;   // staged clouds [max_sets][3 npad/2]
  float4* ys = nullptr;   // staged target [3 mpad/2]
  double* part = nullptr; // [max(max_sets * S1, Smax)][8][npad] (and target rows)
  int64_t part_cap = 0;   // doubles
  double* kyy = nullptr;  // [1]
  double* loss = nullptr; // [max_sets]
  double* stats = nullptr;  // [12]
  double* gx = nullptr;     // gradient scratch [3][n]
  double* gv = nullptr;
  int64_t tsets = 1;        // targets: 1, or one per set (mmd_create_multi)
};

namespace {

using nb::kMT;

template <class T>
int malloc_dev(T** p, size_t count) {
  if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return NBODY_ENOMEM;
  }
  return NBODY_OK;
}

void free_mmd(nbody_mmd* h) {
  if (h->xs) cudaFree(h->xs);
  if (h->ys) cudaFree(h->ys);
  if (h->part) cudaFree(h->part);
  if (h->kyy) cudaFree(h->kyy);
  if (h->loss) cudaFree(h->loss);
  if (h->stats) cudaFree(h->stats);
  if (h->gx) cudaFree(h->gx);
  if (h->gv) cudaFree(h->gv);
}

#define MCK(call)                              \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return NBODY_ECUDA; \
  } while (0)

template <int NS>
cudaError_t rows_ns(int R, dim3 grid, const float4* rows, int64_t rstride, int64_t npad_r,
                    const float4* colA, int64_t astride, int ntA, const float4* colB,
                    int64_t bstride, int ntB, double wA, double wB, float4 rho, double* part,
                    cudaStream_t s) {
  if (R == 2)
    nb::k_mmd_rows<2, NS><<<grid, 128, 0, s>>>(rows, rstride, npad_r, colA, astride, ntA,
                                               colB, bstride, ntB, wA, wB, rho, part);
  else
    nb::k_mmd_rows<1, NS><<<grid, 128, 0, s>>>(rows, rstride, npad_r, colA, astride, ntA,
                                               colB, bstride, ntB, wA, wB, rho, part);
  nb::count_launch();
  return cudaGetLastError();
}

// Row sums of `sets` sets of npad_r rows against ntA + ntB column tiles
// (column set B of set b at colB + b * bstride).
cudaError_t launch_rows(const nbody_mmd* h, int64_t sets, const float4* rows,
                        int64_t rstride, int64_t npad_r, const float4* colA,
                        int64_t astride, int ntA, const float4* colB, int ntB, double wA,
                        double wB, int S, double* part, int64_t bstride = 0) {
  const int R = npad_r >= 256 ? 2 : 1;
  dim3 grid((unsigned)(npad_r / (128 * R)), (unsigned)sets, (unsigned)S);
  switch (h->ns) {
    case 1: return rows_ns<1>(R, grid, rows, rstride, npad_r, colA, astride, ntA, colB, bstride, ntB, wA, wB, h->rho, part, h->s);
    case 2: return rows_ns<2>(R, grid, rows, rstride, npad_r, colA, astride, ntA, colB, bstride, ntB, wA, wB, h->rho, part, h->s);
    case 3: return rows_ns<3>(R, grid, rows, rstride, npad_r, colA, astride, ntA, colB, bstride, ntB, wA, wB, h->rho, part, h->s);
    default: return rows_ns<4>(R, grid, rows, rstride, npad_r, colA, astride, ntA, colB, bstride, ntB, wA, wB, h->rho, part, h->s);
  }
}

template <int NS>
cudaError_t sum_ns(int R, dim3 grid, const float4* rows, int64_t rstride, int64_t n_r,
                   const float4* cols, int64_t cas, int64_t ccs, int nct, float4 rho,
                   double* out, cudaStream_t s) {
  if (R == 2)
    nb::k_mmd_sum<2, NS><<<grid, 128, 0, s>>>(rows, rstride, n_r, cols, cas, ccs, nct, rho, out);
  else
    nb::k_mmd_sum<1, NS><<<grid, 128, 0, s>>>(rows, rstride, n_r, cols, cas, ccs, nct, rho, out);
  nb::count_launch();
  return cudaGetLastError();
}

int rows_per_thread(int64_t npad_r) { return npad_r >= 256 ? 2 : 1; }

// k_mmd_sum over `csets` column sets for every one of `rsets` row sets of
// npad_r rows (n_r real); block sums to out
cudaError_t launch_sum(const nbody_mmd* h, int64_t rsets, int64_t csets, const float4* rows,
                       int64_t rstride, int64_t npad_r, int64_t n_r, const float4* cols,
                       int64_t cas, int64_t ccs, int nct, double* out) {
  const int R = rows_per_thread(npad_r);
  dim3 grid((unsigned)(npad_r / (128 * R)), (unsigned)rsets, (unsigned)csets);
  switch (h->ns) {
    case 1: return sum_ns<1>(R, grid, rows, rstride, n_r, cols, cas, ccs, nct, h->rho, out, h->s);
    case 2: return sum_ns<2>(R, grid, rows, rstride, n_r, cols, cas, ccs, nct, h->rho, out, h->s);
    case 3: return sum_ns<3>(R, grid, rows, rstride, n_r, cols, cas, ccs, nct, h->rho, out, h->s);
    default: return sum_ns<4>(R, grid, rows, rstride, n_r, cols, cas, ccs, nct, h->rho, out, h->s);
  }
}

// column chunks so that a single set fills the GPU (4 blocks per SM)
int chunks_for(const nbody_mmd* h, int64_t sets, int64_t npad_r, int ntiles) {
  const int R = npad_r >= 256 ? 2 : 1;
  const int64_t blocks = sets * (npad_r / (128 * R));
  int64_t S = (4 * (int64_t)h->sms + blocks - 1) / blocks;
  if (S < 1) S = 1;
  if (S > ntiles) S = ntiles;
  if (S > 64) S = 64;
  return (int)S;
}

int ensure_part(nbody_mmd* h, int64_t doubles) {
  if (doubles <= h->part_cap) return NBODY_OK;
  if (h->part) cudaFree(h->part);
  h->part = nullptr;
  h->part_cap = 0;
  int rc = malloc_dev(&h->part, (size_t)doubles);
  if (!rc) h->part_cap = doubles;
  return rc;
}

int stage(nbody_mmd* h, const double* x, const double* v, int64_t ld, int64_t n,
          int64_t npad, int64_t sets, float4* out) {
  dim3 grid((unsigned)((npad / 2 + 127) / 128), (unsigned)sets);
  nb::k_mmd_stage<<<grid, 128, 0, h->s>>>(x, v, ld, n, npad, h->st, out);
  nb::count_launch();
  MCK(cudaGetLastError());
  return NBODY_OK;
}

// device copy of a 3 x count host-or-device array (the kernels read device
// memory; unified addressing lets a device pointer pass straight through)
int device_view(const double* p, size_t count, double** tmp, const double** out,
                cudaStream_t s) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeDevice) {
    *out = p;
    return NBODY_OK;
  }
  cudaGetLastError();
  int rc = malloc_dev(tmp, count);
  if (rc) return rc;
  MCK(cudaMemcpyAsync(*tmp, p, count * sizeof(double), cudaMemcpyDefault, s));
  *out = *tmp;
  return NBODY_OK;
}

// sigma_0 is the smallest bandwidth (first), the others follow in the
// caller's order; rho_l = sigma_0^2 / sigma_l^2 <= 1
void set_bandwidths(nbody_mmd* h, int n_sigma, const double* sigma, double smin) {
  h->ns = n_sigma;
  for (int l = 0; l < n_sigma; ++l) h->sigma[l] = sigma[l];
  double sg[4];
  int k = 0, idx0 = 0;
  for (int l = 0; l < n_sigma; ++l)
    if (sigma[l] == smin) {
      idx0 = l;
      break;
    }
  sg[k++] = sigma[idx0];
  for (int l = 0; l < n_sigma; ++l)
    if (l != idx0) sg[k++] = sigma[l];
  float r[4] = {1.f, 1.f, 1.f, 1.f};
  for (int l = 1; l < n_sigma; ++l) r[l] = (float)((sg[0] * sg[0]) / (sg[l] * sg[l]));
  h->rho = make_float4(r[0], r[1], r[2], r[3]);
  h->c0 = 1.4426950408889634 / (2.0 * sg[0] * sg[0]);  // log2(e) / (2 sigma_0^2)
}

// The target (h->m points, device arrays): its standardisation (mean and
// standard deviation, or the caller's scale), its staged points and its own
// term Kyy = (1/m^2) sum k(y, y').  No allocation beyond the evaluator's
// own buffers (the row-sum scratch grows once).  Synchronises.
int set_target(nbody_mmd* h, const double* dx, const double* dv, const double* scale_or_null) {
  const int64_t m = h->m;
  nb::k_cloud_stats<<<1, 256, 0, h->s>>>(dx, dv, m, h->stats);
  nb::count_launch();
  MCK(cudaGetLastError());
  double stt[12];
  MCK(cudaMemcpyAsync(stt, h->stats, sizeof(stt), cudaMemcpyDeviceToHost, h->s));
  MCK(cudaStreamSynchronize(h->s));
  const double sc0 = std::sqrt(h->c0);
  nb::Standardise st{};
  for (int d = 0; d < 6; ++d) {
    const double sd = scale_or_null ? scale_or_null[d] : stt[6 + d];
    if (!(sd > 0.0) || !std::isfinite(sd)) return NBODY_EINVAL;
    st.mu[d] = stt[d];
    st.f[d] = sc0 / sd;
  }
  h->st = st;
  int rc = stage(h, dx, dv, m, m, h->mpad, 1, h->ys);
  if (rc) return rc;
  const int nty = (int)(h->mpad / nb::kMPts);
  const int Sy = chunks_for(h, 1, h->mpad, nty);
  if ((rc = ensure_part(h, (int64_t)Sy * 8 * h->mpad))) return rc;
  MCK(launch_rows(h, 1, h->ys, 0, h->mpad, h->ys, 0, nty, nullptr, 0, 1.0 / (double)m, 0.0,
                  Sy, h->part));
  nb::k_mmd_finish<<<1, 256, 0, h->s>>>(h->part, Sy, h->mpad, m, 1.0 / (double)m, 0.0,
                                        nullptr, 0, h->kyy);
  nb::count_launch();
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(h->s));
  return NBODY_OK;
}

}  // namespace

namespace nb {

// A new target for an evaluator of clouds of n points when the target keeps
// its size m and the bandwidths are the same: restaged in place (no
// allocation, so no device-wide synchronisation); NBODY_ESTATE otherwise.
int mmd_retarget(nbody_mmd* h, int64_t n, int64_t m, const double* tx, const double* tv,
                 const double* scale_or_null, int n_sigma, const double* sigma) {
  if (!h || h->n != n || h->m != m || h->ns != n_sigma || !tx || !tv || !sigma)
    return NBODY_ESTATE;
  for (int l = 0; l < n_sigma; ++l)
    if (h->sigma[l] != sigma[l]) return NBODY_ESTATE;
  cudaPointerAttributes ax{}, av{};
  if (cudaPointerGetAttributes(&ax, tx) != cudaSuccess || ax.type != cudaMemoryTypeDevice ||
      cudaPointerGetAttributes(&av, tv) != cudaSuccess || av.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return NBODY_ESTATE;
  }
  if (scale_or_null)
    for (int d = 0; d < 6; ++d)
      if (!(scale_or_null[d] > 0.0) || !std::isfinite(scale_or_null[d])) return NBODY_EINVAL;
  return set_target(h, tx, tv, scale_or_null);
}

int mmd_create_multi(nbody_mmd** out, int64_t n, int64_t sets, int64_t m, const double* ty,
                     const double* tv, const double* scale, int n_sigma, const double* sigma,
                     cudaStream_t s) {
  if (!out || n < 1 || sets < 1 || sets > 65535 || m < 1 || !ty || !tv || !scale || !sigma ||
      n_sigma < 1 || n_sigma > kMaxSigma)
    return NBODY_EINVAL;
  *out = nullptr;
  double smin = sigma[0];
  for (int l = 0; l < n_sigma; ++l) {
    if (!(sigma[l] > 0.0) || !std::isfinite(sigma[l])) return NBODY_EINVAL;
    smin = std::fmin(smin, sigma[l]);
  }
  for (int d = 0; d < 6; ++d)
    if (!(scale[d] > 0.0) || !std::isfinite(scale[d])) return NBODY_EINVAL;
  nbody_mmd* h = new (std::nothrow) nbody_mmd();
  if (!h) return NBODY_ENOMEM;
  h->s = s;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  h->n = n;
  h->m = m;
  h->max_sets = sets;
  h->tsets = sets;
  h->npad = pad_points(n);
  h->mpad = pad_points(m);
  set_bandwidths(h, n_sigma, sigma, smin);
  const int nrt = (int)(h->mpad / (128 * rows_per_thread(h->mpad)));
  int rc = malloc_dev(&h->xs, (size_t)sets * 3 * (h->npad / 2));
  if (!rc) rc = malloc_dev(&h->ys, (size_t)sets * 3 * (h->mpad / 2));
  if (!rc) rc = malloc_dev(&h->kyy, (size_t)sets);
  if (!rc) rc = malloc_dev(&h->loss, (size_t)sets);
  if (!rc) rc = malloc_dev(&h->stats, 12);
  if (!rc) rc = ensure_part(h, sets * nrt);
  auto fail = [&](int code) {
    cudaStreamSynchronize(h->s);
    free_mmd(h);
    delete h;
    return code;
  };
  if (rc) return fail(rc);
  // units: the caller's scale; the origin: the first target's mean
  k_cloud_stats<<<1, 256, 0, s>>>(ty, tv, m, h->stats);
  count_launch();
  double stt[12];
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(stt, h->stats, sizeof(stt), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(NBODY_ECUDA);
  const double sc0 = std::sqrt(h->c0);
  for (int d = 0; d < 6; ++d) {
    h->st.mu[d] = stt[d];
    h->st.f[d] = sc0 / scale[d];
  }
  // every target's own term (1/m^2) sum k(y, y')
  const int64_t ystr = 3 * (h->mpad / 2);
  if ((rc = stage(h, ty, tv, sets * m, m, h->mpad, sets, h->ys))) return fail(rc);
  if (launch_sum(h, sets, 1, h->ys, ystr, h->mpad, m, h->ys, ystr, 0,
                 (int)(h->mpad / kMPts), h->part) != cudaSuccess)
    return fail(NBODY_ECUDA);
  k_mmd_block_total<<<(unsigned)((sets + 255) / 256), 256, 0, s>>>(
      h->part, sets, nrt, 1.0 / ((double)m * (double)m), h->kyy);
  count_launch();
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return fail(NBODY_ECUDA);
  *out = h;
  return NBODY_OK;
}

int mmd_eval_multi(nbody_mmd* h, const double* x, const double* v, double* loss, double* xbar,
                   double* vbar) {
  if (!h || h->tsets != h->max_sets || !x || !v || !loss) return NBODY_EINVAL;
  const int64_t sets = h->tsets, n = h->n;
  const int ntx = (int)(h->npad / kMPts), nty = (int)(h->mpad / kMPts);
  const int S = chunks_for(h, sets, h->npad, ntx + nty);
  int rc = ensure_part(h, sets * S * 8 * h->npad);
  if (!rc) rc = stage(h, x, v, sets * n, n, h->npad, sets, h->xs);
  if (rc) return rc;
  const int64_t xstr = 3 * (h->npad / 2), ystr = 3 * (h->mpad / 2);
  MCK(launch_rows(h, sets, h->xs, xstr, h->npad, h->xs, xstr, ntx, h->ys, nty,
                  1.0 / (double)n, -1.0 / (double)h->m, S, h->part, ystr));
  k_mmd_finish<<<(unsigned)sets, 256, 0, h->s>>>(h->part, S, h->npad, n, 1.0 / (double)n, 2.0,
                                                 h->kyy, 1, loss);
  count_launch();
  MCK(cudaGetLastError());
  if (xbar && vbar) {
    const double g0 = 4.0 * 0.6931471805599453 / (double)n;  // 4 ln2 / n
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)sets);
    k_mmd_grad<<<grid, 256, 0, h->s>>>(h->part, S, h->npad, n, sets * n, h->st, g0, xbar, vbar);
    count_launch();
    MCK(cudaGetLastError());
  }
  return NBODY_OK;
}

}  // namespace nb

extern "C" {

int nbody_mmd_create(nbody_mmd** out, int64_t n, int64_t max_sets, int64_t m,
                     const double* tx, const double* tv, const double* scale_or_null,
                     int n_sigma, const double* sigma, void* cuda_stream) {
  if (!out) return NBODY_EINVAL;
  *out = nullptr;
  if (n < 1 || max_sets < 1 || m < 1 || !tx || !tv || !sigma || n_sigma < 1 ||
      n_sigma > nb::kMaxSigma)
    return NBODY_EINVAL;
  double smin = sigma[0];
  for (int l = 0; l < n_sigma; ++l) {
    if (!(sigma[l] > 0.0) || !std::isfinite(sigma[l])) return NBODY_EINVAL;
    smin = std::fmin(smin, sigma[l]);
  }
  if (scale_or_null)
    for (int d = 0; d < 6; ++d)
      if (!(scale_or_null[d] > 0.0) || !std::isfinite(scale_or_null[d])) return NBODY_EINVAL;
  int dev = 0, maj = 0, min = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev) ||
      cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev)) {
    cudaGetLastError();
    return NBODY_ENODEV;
  }
  if (maj != 10 || min != 3) return NBODY_ENODEV;
  nbody_mmd* h = new (std::nothrow) nbody_mmd();
  if (!h) return NBODY_ENOMEM;
  h->s = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  h->n = n;
  h->m = m;
  h->max_sets = max_sets;
  h->npad = nb::pad_points(n);
  h->mpad = nb::pad_points(m);
  set_bandwidths(h, n_sigma, sigma, smin);
  int rc = NBODY_OK;
  double* tmpx = nullptr;
  double* tmpv = nullptr;
  const double* dx = nullptr;
  const double* dv = nullptr;
  if ((rc = malloc_dev(&h->xs, (size_t)max_sets * 3 * (h->npad / 2))) ||
      (rc = malloc_dev(&h->ys, (size_t)3 * (h->mpad / 2))) ||
      (rc = malloc_dev(&h->kyy, 1)) || (rc = malloc_dev(&h->loss, (size_t)max_sets)) ||
      (rc = malloc_dev(&h->stats, 12)) || (rc = malloc_dev(&h->gx, (size_t)3 * n)) ||
      (rc = malloc_dev(&h->gv, (size_t)3 * n)) ||
      (rc = device_view(tx, (size_t)3 * m, &tmpx, &dx, h->s)) ||
      (rc = device_view(tv, (size_t)3 * m, &tmpv, &dv, h->s))) {
    if (tmpx) cudaFree(tmpx);
    if (tmpv) cudaFree(tmpv);
    free_mmd(h);
    delete h;
    return rc;
  }
  rc = set_target(h, dx, dv, scale_or_null);
  if (rc) cudaStreamSynchronize(h->s);
  if (tmpx) cudaFree(tmpx);
  if (tmpv) cudaFree(tmpv);
  if (rc) {
    free_mmd(h);
    delete h;
    return rc;
  }
  *out = h;
  return NBODY_OK;
}

int nbody_mmd_eval_batch(nbody_mmd* h, int64_t sets, const double* x, const double* v,
                         double* losses) {
  if (!h || !x || !v || !losses || sets < 1 || sets > h->max_sets) return NBODY_EINVAL;
  int rc;
  double* tmpx = nullptr;
  double* tmpv = nullptr;
  const double* dx = nullptr;
  const double* dv = nullptr;
  const size_t cnt = (size_t)3 * sets * h->n;
  if ((rc = device_view(x, cnt, &tmpx, &dx, h->s)) ||
      (rc = device_view(v, cnt, &tmpv, &dv, h->s))) {
    if (tmpx) cudaFree(tmpx);
    return rc;
  }
  const int ntx = (int)(h->npad / nb::kMPts), nty = (int)(h->mpad / nb::kMPts);
  const int S = chunks_for(h, sets, h->npad, ntx + nty);
  rc = ensure_part(h, sets * S * 8 * h->npad);
  if (!rc) rc = stage(h, dx, dv, sets * h->n, h->n, h->npad, sets, h->xs);
  const int64_t xstride = 3 * (h->npad / 2);
  if (!rc && launch_rows(h, sets, h->xs, xstride, h->npad, h->xs, xstride, ntx, h->ys, nty,
                         1.0 / (double)h->n, -1.0 / (double)h->m, S, h->part) != cudaSuccess)
    rc = NBODY_ECUDA;
  if (!rc) {
    nb::k_mmd_finish<<<(unsigned)sets, 256, 0, h->s>>>(h->part, S, h->npad, h->n,
                                                       1.0 / (double)h->n, 2.0, h->kyy, 0,
                                                       h->loss);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  std::vector<double> hl((size_t)sets);
  if (!rc && cudaMemcpyAsync(hl.data(), h->loss, (size_t)sets * sizeof(double),
                             cudaMemcpyDeviceToHost, h->s) != cudaSuccess)
    rc = NBODY_ECUDA;
  if (cudaStreamSynchronize(h->s) != cudaSuccess) rc = NBODY_ECUDA;
  if (tmpx) cudaFree(tmpx);
  if (tmpv) cudaFree(tmpv);
  if (rc) return rc;
  if (cudaMemcpy(losses, hl.data(), (size_t)sets * sizeof(double), cudaMemcpyDefault) !=
      cudaSuccess)
    return NBODY_ECUDA;
  for (double L : hl)
    if (!std::isfinite(L)) return NBODY_ENAN;
  return NBODY_OK;
}

int nbody_mmd_eval(nbody_mmd* h, const double* x, const double* v, double* loss,
                   double* xbar, double* vbar) {
  if (!h || !x || !v || !loss) return NBODY_EINVAL;
  int rc;
  double* tmpx = nullptr;
  double* tmpv = nullptr;
  const double* dx = nullptr;
  const double* dv = nullptr;
  const size_t cnt = (size_t)3 * h->n;
  if ((rc = device_view(x, cnt, &tmpx, &dx, h->s)) ||
      (rc = device_view(v, cnt, &tmpv, &dv, h->s))) {
    if (tmpx) cudaFree(tmpx);
    return rc;
  }
  const int ntx = (int)(h->npad / nb::kMPts), nty = (int)(h->mpad / nb::kMPts);
  const int S = chunks_for(h, 1, h->npad, ntx + nty);
  rc = ensure_part(h, (int64_t)S * 8 * h->npad);
  if (!rc) rc = stage(h, dx, dv, h->n, h->n, h->npad, 1, h->xs);
  if (!rc && launch_rows(h, 1, h->xs, 0, h->npad, h->xs, 0, ntx, h->ys, nty,
                         1.0 / (double)h->n, -1.0 / (double)h->m, S, h->part) != cudaSuccess)
    rc = NBODY_ECUDA;
  if (!rc) {
    nb::k_mmd_finish<<<1, 256, 0, h->s>>>(h->part, S, h->npad, h->n, 1.0 / (double)h->n, 2.0,
                                          h->kyy, 0, h->loss);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  if (!rc && (xbar || vbar)) {
    // gradients into the context's buffers, then out to the caller's
    const double g0 = 4.0 * 0.6931471805599453 / (double)h->n;  // 4 ln2 / n
    nb::k_mmd_grad<<<(unsigned)((h->n + 255) / 256), 256, 0, h->s>>>(
        h->part, S, h->npad, h->n, h->n, h->st, g0, h->gx, h->gv);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
    if (!rc && xbar &&
        cudaMemcpyAsync(xbar, h->gx, cnt * sizeof(double), cudaMemcpyDefault, h->s) != cudaSuccess)
      rc = NBODY_ECUDA;
    if (!rc && vbar &&
        cudaMemcpyAsync(vbar, h->gv, cnt * sizeof(double), cudaMemcpyDefault, h->s) != cudaSuccess)
      rc = NBODY_ECUDA;
  }
  double L = 0.0;
  if (!rc && cudaMemcpyAsync(&L, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->s) !=
                 cudaSuccess)
    rc = NBODY_ECUDA;
  if (cudaStreamSynchronize(h->s) != cudaSuccess) rc = NBODY_ECUDA;
  if (tmpx) cudaFree(tmpx);
  if (tmpv) cudaFree(tmpv);
  if (rc) return rc;
  if (!std::isfinite(L)) return NBODY_ENAN;
  *loss = L;
  return NBODY_OK;
}

int nbody_mmd_eval_cross(nbody_mmd* h, int64_t sets, const double* x, const double* v,
                         int64_t targets, int64_t m2, const double* ty, const double* tv,
                         double* losses) {
  constexpr int64_t kMaxGridYZ = 65535;
  if (!h || !x || !v || !ty || !tv || !losses || sets < 1 || targets < 1 || m2 < 1 ||
      sets > kMaxGridYZ || targets > kMaxGridYZ)
    return NBODY_EINVAL;
  const int64_t n = h->n, npad = h->npad, m2pad = nb::pad_points(m2);
  const int64_t xstr = 3 * (npad / 2), tstr = 3 * (m2pad / 2);
  const int nrx = (int)(npad / (128 * rows_per_thread(npad)));
  const int nrt = (int)(m2pad / (128 * rows_per_thread(m2pad)));
  // targets per cross launch: the block sums of one launch stay below 2^25
  // doubles (256 MB)
  int64_t tc = std::max<int64_t>(1, ((int64_t)1 << 25) / (sets * nrx));
  tc = std::min(std::min(tc, targets), kMaxGridYZ);
  const int64_t nbs = std::max(std::max(sets * nrx, targets * nrt), tc * sets * nrx);
  double *tmpx = nullptr, *tmpv = nullptr, *tmpy = nullptr, *tmpw = nullptr;
  const double *dx = nullptr, *dv = nullptr, *dy = nullptr, *dw = nullptr;
  float4 *xs = nullptr, *ts = nullptr;
  double *bs = nullptr, *kxx = nullptr, *kyy = nullptr, *dl = nullptr;
  int rc = device_view(x, (size_t)(3 * sets * n), &tmpx, &dx, h->s);
  if (!rc) rc = device_view(v, (size_t)(3 * sets * n), &tmpv, &dv, h->s);
  if (!rc) rc = device_view(ty, (size_t)(3 * targets * m2), &tmpy, &dy, h->s);
  if (!rc) rc = device_view(tv, (size_t)(3 * targets * m2), &tmpw, &dw, h->s);
  if (!rc) rc = malloc_dev(&xs, (size_t)(sets * xstr));
  if (!rc) rc = malloc_dev(&ts, (size_t)(targets * tstr));
  if (!rc) rc = malloc_dev(&bs, (size_t)nbs);
  if (!rc) rc = malloc_dev(&kxx, (size_t)sets);
  if (!rc) rc = malloc_dev(&kyy, (size_t)targets);
  if (!rc) rc = malloc_dev(&dl, (size_t)(sets * targets));
  // the clouds and the targets in the evaluator's standardisation, staged once
  if (!rc) rc = stage(h, dx, dv, sets * n, n, npad, sets, xs);
  if (!rc) rc = stage(h, dy, dw, targets * m2, m2, m2pad, targets, ts);
  const unsigned tpb = 256;
  // own terms: (1/n^2) sum k(x, x') per cloud, (1/m^2) sum k(y, y') per target
  if (!rc && launch_sum(h, sets, 1, xs, xstr, npad, n, xs, xstr, 0, (int)(npad / nb::kMPts),
                        bs) != cudaSuccess)
    rc = NBODY_ECUDA;
  if (!rc) {
    nb::k_mmd_block_total<<<(unsigned)((sets + tpb - 1) / tpb), tpb, 0, h->s>>>(
        bs, sets, nrx, 1.0 / ((double)n * (double)n), kxx);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  if (!rc && launch_sum(h, targets, 1, ts, tstr, m2pad, m2, ts, tstr, 0,
                        (int)(m2pad / nb::kMPts), bs) != cudaSuccess)
    rc = NBODY_ECUDA;
  if (!rc) {
    nb::k_mmd_block_total<<<(unsigned)((targets + tpb - 1) / tpb), tpb, 0, h->s>>>(
        bs, targets, nrt, 1.0 / ((double)m2 * (double)m2), kyy);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  // cross terms, tc targets per launch
  for (int64_t t0 = 0; !rc && t0 < targets; t0 += tc) {
    const int64_t cnt = std::min(tc, targets - t0);
    if (launch_sum(h, sets, cnt, xs, xstr, npad, n, ts + t0 * tstr, 0, tstr,
                   (int)(m2pad / nb::kMPts), bs) != cudaSuccess) {
      rc = NBODY_ECUDA;
      break;
    }
    const int64_t q = cnt * sets;
    nb::k_mmd_cross_finish<<<(unsigned)((q + tpb - 1) / tpb), tpb, 0, h->s>>>(
        bs, sets, cnt, nrx, 2.0 / ((double)n * (double)m2), kxx, kyy + t0, dl + t0 * sets);
    nb::count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = NBODY_ECUDA;
  }
  std::vector<double> hl;
  if (!rc) {
    hl.resize((size_t)(sets * targets));
    if (cudaMemcpyAsync(hl.data(), dl, hl.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        h->s) != cudaSuccess)
      rc = NBODY_ECUDA;
  }
  if (cudaStreamSynchronize(h->s) != cudaSuccess && !rc) rc = NBODY_ECUDA;
  for (void* p : {(void*)tmpx, (void*)tmpv, (void*)tmpy, (void*)tmpw, (void*)xs, (void*)ts,
                  (void*)bs, (void*)kxx, (void*)kyy, (void*)dl})
    if (p) cudaFree(p);
  if (rc) return rc;
  if (cudaMemcpy(losses, hl.data(), hl.size() * sizeof(double), cudaMemcpyDefault) !=
      cudaSuccess)
    return NBODY_ECUDA;
  for (double L : hl)
    if (!std::isfinite(L)) return NBODY_ENAN;
  return NBODY_OK;
}

int nbody_mmd_target_stats(nbody_mmd* h, double mu[6], double scale[6]) {
  if (!h) return NBODY_EINVAL;
  const double sc0 = std::sqrt(h->c0);
  for (int d = 0; d < 6; ++d) {
    if (mu) mu[d] = h->st.mu[d];
    if (scale) scale[d] = sc0 / h->st.f[d];
  }
  return NBODY_OK;
}

void nbody_mmd_destroy(nbody_mmd* h) {
  if (!h) return;
  cudaStreamSynchronize(h->s);
  free_mmd(h);
  delete h;
}

}  // extern "C"
