// pair_vjp.cu -- vector-Jacobian product of the softened pair acceleration,
// the second O(N^2) loop (reverse-mode gradients, paper Sec. 2).
//
// With a_i = -G sum_j m_j r_ij s_ij^-3, r_ij = x_i - x_j,
// s^2 = |r|^2 + eps^2, the Jacobian blocks are built from the tidal tensor
// K(r) = s^-3 I - 3 s^-5 r r^T (even in r, symmetric):
//   d a_i / d x_i = -G sum_j m_j K(r_ij),   d a_i / d x_k = G m_k K(r_ik),
// so for cotangents l the product (J^T l)_k is
//   g_k = -G sum_j K(r_kj) (m_j l_k - m_k l_j).
// The kernel returns Q_k = sum_j [s^-3 u - 3 s^-5 d (d.u)],
// u = m_j l_k - m_k l_j, d = x_j - x_k, so that g_k = -G Q_k; the j = k term
// vanishes (u = 0).  Same tiling, packed FP32x2 arithmetic and FP32/FP64
// two-level summation as the forward kernel; 26 FP32 operations and one
// rsqrt per interaction.  With equal masses u = m (l_k - l_j), the mass is
// applied by the consumer, and the s^-3 and s^-5 sums are kept apart
// (Q = A - 3 B): 22 FP32 operations per interaction.
#include "async_copy.cuh"
#include "block_reduce.cuh"
#include "nbody_internal.cuh"
#include "vjp_body.cuh"

namespace nb {

namespace {

// Build-time tunables (defaults: the measured best on GB300).
#ifndef NB_VJP_TJ
#define NB_VJP_TJ 256
#endif
#ifndef NB_VJP_UNROLL
#define NB_VJP_UNROLL 2
#endif
#ifndef NB_VJP_MINB
#define NB_VJP_MINB 1
#endif
// 1: j-tiles staged with cp.async into two shared-memory buffers (the copy
// of the next tile overlaps the current one, one barrier per tile);
// 0: loaded through registers into one buffer, two barriers per tile
#ifndef NB_TILE_ASYNC
#define NB_TILE_ASYNC 0
#endif
constexpr int kTJ = NB_VJP_TJ;  // j-pairs per shared-memory tile (4 float4 each)
constexpr int kUnrollJ = NB_VJP_UNROLL;

constexpr int kTJSmall = 128;   // small tiles: finer j-chunks for small systems

template <int NT, int R, bool EQM, bool MB, int TJ = kTJ>
__global__ void __launch_bounds__(NT, NB_VJP_MINB)
    k_vjp_tile(const float4* __restrict__ vst, int ntiles, float eps2,
               int64_t npad, double* __restrict__ part, double* __restrict__ mpart,
               double* __restrict__ fin, unsigned* __restrict__ ctr) {
  constexpr bool kAsync = NB_TILE_ASYNC != 0;
  __shared__ __align__(16) float4 sbuf[kAsync ? 2 : 1][4 * TJ];
  const int t = threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.x * (NT * R) + t;
  const int S = gridDim.y;
  const int tile_b = (int)(((int64_t)blockIdx.y * ntiles) / S);
  const int tile_e = (int)(((int64_t)(blockIdx.y + 1) * ntiles) / S);

  IState st[R];
  double gx[R], gy[R], gz[R], gm[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    st[r] = load_k(vst, k0 + r * NT);
    gx[r] = gy[r] = gz[r] = gm[r] = 0.0;
  }
  const float2 e2 = make_float2(eps2, eps2);
  if (kAsync && tile_b < tile_e) {
    const float4* src = vst + (int64_t)tile_b * (4 * TJ);
    for (int q = t; q < 4 * TJ; q += NT) cp_async16(&sbuf[0][q], src + q);
    cp_async_commit();
  }
  for (int tile = tile_b; tile < tile_e; ++tile) {
    const float4* sj;
    if (kAsync) {
      cp_async_wait_all();
      __syncthreads();  // this tile visible; the previous one no longer read
      if (tile + 1 < tile_e) {
        const float4* src = vst + (int64_t)(tile + 1) * (4 * TJ);
        float4* dst = sbuf[(tile + 1 - tile_b) & 1];
        for (int q = t; q < 4 * TJ; q += NT) cp_async16(dst + q, src + q);
        cp_async_commit();
      }
      sj = sbuf[(tile - tile_b) & 1];
    } else {
      __syncthreads();
      const float4* src = vst + (int64_t)tile * (4 * TJ);
#pragma unroll
      for (int q = t; q < 4 * TJ; q += NT) sbuf[0][q] = src[q];
      __syncthreads();
      sj = sbuf[0];
    }
    float2 qa[R][3], qb[R][3], qm[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      qm[r] = make_float2(0.f, 0.f);
#pragma unroll
      for (int d = 0; d < 3; ++d) qa[r][d] = qb[r][d] = make_float2(0.f, 0.f);
    }
#pragma unroll (kUnrollJ)
    for (int jj = 0; jj < TJ; ++jj) {
      const float4 A = sj[4 * jj], B = sj[4 * jj + 1];
      const float4 L1 = sj[4 * jj + 2], L2 = sj[4 * jj + 3];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (EQM)
          vjp_body_eqm(A, B, L1, L2, st[r], e2, qa[r], qb[r]);
        else
          vjp_body(A, B, L1, L2, st[r], e2, qa[r][0], qa[r][1], qa[r][2]);
        if (MB) mass_body(A, B, L1, L2, st[r], e2, qm[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (MB) gm[r] += (double)qm[r].x + (double)qm[r].y;
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
  double* p = part + (int64_t)blockIdx.y * 3 * npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t k = k0 + r * NT;
    p[k] = gx[r];
    p[npad + k] = gy[r];
    p[2 * npad + k] = gz[r];
    if (MB) mpart[(int64_t)blockIdx.y * npad + k] = gm[r];
  }
  if (fin) finish_row_tile<NT, R>(part, MB ? mpart : nullptr, S, npad, k0, fin, ctr);
}

template <int R, bool EQM, bool MB>
__global__ void __launch_bounds__(256)
    k_vjp_warp(const float4* __restrict__ vst, int64_t npairs, float eps2,
               int64_t npad, double* __restrict__ part, double* __restrict__ mpart) {
  const int lane = threadIdx.x & 31;
  const int64_t kb = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * R;
  const int S = gridDim.y;
  const int64_t pb = ((int64_t)blockIdx.y * npairs) / S;
  const int64_t pe = ((int64_t)(blockIdx.y + 1) * npairs) / S;
  IState st[R];
  float2 qa[R][3], qb[R][3], qm[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    st[r] = load_k(vst, kb + r);
    qm[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = 0; d < 3; ++d) qa[r][d] = qb[r][d] = make_float2(0.f, 0.f);
  }
  const float2 e2 = make_float2(eps2, eps2);
  for (int64_t p = pb + lane; p < pe; p += 32) {
    const float4 A = vst[4 * p], B = vst[4 * p + 1];
    const float4 L1 = vst[4 * p + 2], L2 = vst[4 * p + 3];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (EQM)
        vjp_body_eqm(A, B, L1, L2, st[r], e2, qa[r], qb[r]);
      else
        vjp_body(A, B, L1, L2, st[r], e2, qa[r][0], qa[r][1], qa[r][2]);
      if (MB) mass_body(A, B, L1, L2, st[r], e2, qm[r]);
    }
  }
  double* out = part + (int64_t)blockIdx.y * 3 * npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double sx = (double)qa[r][0].x + (double)qa[r][0].y;
    double sy = (double)qa[r][1].x + (double)qa[r][1].y;
    double sz = (double)qa[r][2].x + (double)qa[r][2].y;
    if (EQM) {
      sx -= 3.0 * ((double)qb[r][0].x + (double)qb[r][0].y);
      sy -= 3.0 * ((double)qb[r][1].x + (double)qb[r][1].y);
      sz -= 3.0 * ((double)qb[r][2].x + (double)qb[r][2].y);
    }
    double sm = MB ? (double)qm[r].x + (double)qm[r].y : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
      if (MB) sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if (lane == 0) {
      const int64_t k = kb + r;
      out[k] = sx;
      out[npad + k] = sy;
      out[2 * npad + k] = sz;
      if (MB) mpart[(int64_t)blockIdx.y * npad + k] = sm;
    }
  }
}

template <bool EQM, bool MB>
cudaError_t launch_vjp_impl(const PairCfg& c, const float4* vst, int64_t npad,
                            float eps2, double* part, double* mpart, double* fin,
                            unsigned* ctr, cudaStream_t s) {
  if (c.variant == kTile && c.vjp_tile_pairs == kTJSmall) {
    const int ntiles = (int)(npad / (2 * kTJSmall));
    dim3 grid((unsigned)(npad / (c.nt * c.r)), (unsigned)c.S);
    if (c.nt == 128 && c.r == 2)
      k_vjp_tile<128, 2, EQM, MB, kTJSmall><<<grid, 128, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else if (c.nt == 128 && c.r == 1)
      k_vjp_tile<128, 1, EQM, MB, kTJSmall><<<grid, 128, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else if (c.nt == 64 && c.r == 2)
      k_vjp_tile<64, 2, EQM, MB, kTJSmall><<<grid, 64, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else
      return cudaErrorInvalidValue;
  } else if (c.variant == kTile) {
    if (c.vjp_tile_pairs != kTJ) return cudaErrorInvalidValue;
    const int ntiles = (int)(npad / (2 * kTJ));
    dim3 grid((unsigned)(npad / (c.nt * c.r)), (unsigned)c.S);
    if (c.nt == 256 && c.r == 2)
      k_vjp_tile<256, 2, EQM, MB><<<grid, 256, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else if (c.nt == 128 && c.r == 4)
      k_vjp_tile<128, 4, EQM, MB><<<grid, 128, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else if (c.nt == 128 && c.r == 2)
      k_vjp_tile<128, 2, EQM, MB><<<grid, 128, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else if (c.nt == 128 && c.r == 1)
      k_vjp_tile<128, 1, EQM, MB><<<grid, 128, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else if (c.nt == 64 && c.r == 2)
      k_vjp_tile<64, 2, EQM, MB><<<grid, 64, 0, s>>>(vst, ntiles, eps2, npad, part, mpart, fin, ctr);
    else
      return cudaErrorInvalidValue;
  } else {
    dim3 grid((unsigned)(npad / (8 * c.r)), (unsigned)c.S);
    if (c.r == 4)
      k_vjp_warp<4, EQM, MB><<<grid, 256, 0, s>>>(vst, npad / 2, eps2, npad, part, mpart);
    else if (c.r == 2)
      k_vjp_warp<2, EQM, MB><<<grid, 256, 0, s>>>(vst, npad / 2, eps2, npad, part, mpart);
    else
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int vjp_tile_pairs() { return kTJ; }

int vjp_blocks_per_sm(const PairCfg& c) {
  int occ = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define NB_OCC(NT, R)                                                             \
  if (c.nt == NT && c.r == R)                                                     \
    e = c.eqm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                    &occ, k_vjp_tile<NT, R, true, false>, NT, 0)                  \
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                    &occ, k_vjp_tile<NT, R, false, false>, NT, 0);
#define NB_OCC_S(NT, R)                                                           \
  if (c.nt == NT && c.r == R)                                                     \
    e = c.eqm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                    &occ, k_vjp_tile<NT, R, true, false, kTJSmall>, NT, 0)        \
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                    \
                    &occ, k_vjp_tile<NT, R, false, false, kTJSmall>, NT, 0);
  if (c.variant == kTile && c.vjp_tile_pairs == kTJSmall) {
    NB_OCC_S(128, 2) NB_OCC_S(128, 1) NB_OCC_S(64, 2)
  } else if (c.variant == kTile) {
    NB_OCC(256, 2) NB_OCC(128, 4) NB_OCC(128, 2) NB_OCC(128, 1) NB_OCC(64, 2)
  } else {
    e = c.eqm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vjp_warp<4, true, false>, 256, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vjp_warp<4, false, false>, 256, 0);
  }
#undef NB_OCC
#undef NB_OCC_S
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return occ > 0 ? occ : 1;
}

cudaError_t launch_pair_vjp_fin(const PairCfg& c, const float4* vst, int64_t npad,
                                float eps2, double* part, double* mpart, double* fin,
                                unsigned* ctr, cudaStream_t s) {
  if (c.variant != kTile || c.S < 2) fin = nullptr;
  if (mpart) {
    if (c.eqm) return launch_vjp_impl<true, true>(c, vst, npad, eps2, part, mpart, fin, ctr, s);
    return launch_vjp_impl<false, true>(c, vst, npad, eps2, part, mpart, fin, ctr, s);
  }
  if (c.eqm) return launch_vjp_impl<true, false>(c, vst, npad, eps2, part, nullptr, fin, ctr, s);
  return launch_vjp_impl<false, false>(c, vst, npad, eps2, part, nullptr, fin, ctr, s);
}

cudaError_t launch_pair_vjp(const PairCfg& c, const float4* vst, int64_t npad,
                            float eps2, double* part, double* mpart, cudaStream_t s) {
  return launch_pair_vjp_fin(c, vst, npad, eps2, part, mpart, nullptr, nullptr, s);
}

}  // namespace nb
