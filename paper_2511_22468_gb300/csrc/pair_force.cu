// pair_force.cu -- softened direct-sum pair acceleration, the O(N^2) hot
// loop of the method (paper Sec. 1, "N-body codes": exact pairwise forces
// with softening, no tree or multipole):
//
//   a_i = G sum_j m_j (x_j - x_i) (|x_j - x_i|^2 + eps^2)^(-3/2)
//
// FP32 CUDA-core work (not a contraction, so no tensor cores).  The j = i
// term is exactly zero because eps > 0, so the loop has no branch.
//
// Tile variant: each thread keeps R i-particles in registers; a block
// streams j-pairs through shared memory in tiles of kTJ pairs.  Two j's are
// processed together with the packed FP32x2 instructions of sm_100+
// (add/fma/mul .f32x2), which halve the issue slots of the FP32 pipe, so the
// loop is bound by the FP32 pipe itself (12 FP32 operations and one MUFU
// rsqrt per interaction).  Sums are FP32 within a tile and FP64 across
// tiles; each j-chunk (grid.y) writes its own FP64 partial slice, reduced
// later in fixed order, so results are bitwise reproducible.
//
// Warp variant (small N): a warp owns R i-particles and its 32 lanes split
// the j-range; lane sums are combined by a fixed xor-shuffle butterfly.
#include "async_copy.cuh"
#include "block_reduce.cuh"
#include "nbody_internal.cuh"
#include "pair_body.cuh"

namespace nb {

namespace {

// Build-time tunables (the defaults are the measured best on GB300):
// j-pairs per shared-memory tile, unroll of the j-loop, and the minimum
// resident blocks per SM the register allocation must allow.
#ifndef NB_PAIR_TJ
#define NB_PAIR_TJ 512
#endif
#ifndef NB_PAIR_UNROLL
#define NB_PAIR_UNROLL 2
#endif
#ifndef NB_PAIR_MINB
#define NB_PAIR_MINB 1
#endif
// 1: j-tiles staged with cp.async into two shared-memory buffers (the copy
// of the next tile overlaps the current one, one barrier per tile);
// 0: loaded through registers into one buffer, two barriers per tile
#ifndef NB_TILE_ASYNC
#define NB_TILE_ASYNC 0
#endif
constexpr int kTJ = NB_PAIR_TJ;  // j-pairs per shared-memory tile
constexpr int kTJSmall = 128;    // small tiles: more j-chunks for small N
constexpr int kUnrollJ = NB_PAIR_UNROLL;

template <int NT, int R, bool POT, bool EQM, int TJ = kTJ>
__global__ void __launch_bounds__(NT, NB_PAIR_MINB)
    k_pair_tile(const float4* __restrict__ st, int ntiles, float eps2,
                int64_t npad, double* __restrict__ part,
                double* __restrict__ pot, double* __restrict__ fin,
                unsigned* __restrict__ ctr) {
  constexpr bool kAsync = NB_TILE_ASYNC != 0;
  __shared__ __align__(16) float4 sbuf[kAsync ? 2 : 1][2 * TJ];
  const int t = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * (NT * R) + t;
  const int S = gridDim.y;
  const int tile_b = (int)(((int64_t)blockIdx.y * ntiles) / S);
  const int tile_e = (int)(((int64_t)(blockIdx.y + 1) * ntiles) / S);

  float2 nx[R], ny[R], nz[R];
  double dax[R], day[R], daz[R], dph[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float xi, yi, zi;
    load_i(st, i0 + r * NT, xi, yi, zi);
    nx[r] = make_float2(-xi, -xi);
    ny[r] = make_float2(-yi, -yi);
    nz[r] = make_float2(-zi, -zi);
    dax[r] = day[r] = daz[r] = dph[r] = 0.0;
  }
  const float2 e2 = make_float2(eps2, eps2);

  if (kAsync && tile_b < tile_e) {
    const float4* src = st + (int64_t)tile_b * (2 * TJ);
    for (int q = t; q < 2 * TJ; q += NT) cp_async16(&sbuf[0][q], src + q);
    cp_async_commit();
  }
  for (int tile = tile_b; tile < tile_e; ++tile) {
    const float4* sj;
    if (kAsync) {
      cp_async_wait_all();
      __syncthreads();  // this tile visible; the previous one no longer read
      if (tile + 1 < tile_e) {
        const float4* src = st + (int64_t)(tile + 1) * (2 * TJ);
        float4* dst = sbuf[(tile + 1 - tile_b) & 1];
        for (int q = t; q < 2 * TJ; q += NT) cp_async16(dst + q, src + q);
        cp_async_commit();
      }
      sj = sbuf[(tile - tile_b) & 1];
    } else {
      __syncthreads();
      const float4* src = st + (int64_t)tile * (2 * TJ);
#pragma unroll
      for (int q = t; q < 2 * TJ; q += NT) sbuf[0][q] = src[q];
      __syncthreads();
      sj = sbuf[0];
    }

    float2 ax[R], ay[R], az[R], ph[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
      ax[r] = ay[r] = az[r] = ph[r] = make_float2(0.f, 0.f);
#pragma unroll (kUnrollJ)
    for (int jj = 0; jj < TJ; ++jj) {
      const float4 A = sj[2 * jj];
      const float4 B = sj[2 * jj + 1];
      const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
      const float2 zj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (EQM)
          body_eqm(xj, yj, zj, nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r]);
        else
          body<POT>(xj, yj, zj, mj, nx[r], ny[r], nz[r], e2, ax[r], ay[r],
                    az[r], ph[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      dax[r] += (double)ax[r].x + (double)ax[r].y;
      day[r] += (double)ay[r].x + (double)ay[r].y;
      daz[r] += (double)az[r].x + (double)az[r].y;
      if (POT) dph[r] += (double)ph[r].x + (double)ph[r].y;
    }
  }

  double* p = part + (int64_t)blockIdx.y * 3 * npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i0 + r * NT;
    p[i] = dax[r];
    p[npad + i] = day[r];
    p[2 * npad + i] = daz[r];
    if (POT) pot[(int64_t)blockIdx.y * npad + i] = dph[r];
  }
  if (fin) finish_row_tile<NT, R>(part, nullptr, S, npad, i0, fin, ctr);
}

// Warp variant: block of 8 warps; warp w owns i = (blockIdx.x*8 + w)*R + r.
template <int R, bool POT, bool EQM>
__global__ void __launch_bounds__(256)
    k_pair_warp(const float4* __restrict__ st, int64_t npairs, float eps2,
                int64_t npad, double* __restrict__ part,
                double* __restrict__ pot) {
  const int lane = threadIdx.x & 31;
  const int64_t ib = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * R;
  const int S = gridDim.y;
  const int64_t pb = ((int64_t)blockIdx.y * npairs) / S;
  const int64_t pe = ((int64_t)(blockIdx.y + 1) * npairs) / S;

  float2 nx[R], ny[R], nz[R], ax[R], ay[R], az[R], ph[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float xi, yi, zi;
    load_i(st, ib + r, xi, yi, zi);
    nx[r] = make_float2(-xi, -xi);
    ny[r] = make_float2(-yi, -yi);
    nz[r] = make_float2(-zi, -zi);
    ax[r] = ay[r] = az[r] = ph[r] = make_float2(0.f, 0.f);
  }
  const float2 e2 = make_float2(eps2, eps2);
  for (int64_t p = pb + lane; p < pe; p += 32) {
    const float4 A = st[2 * p];
    const float4 B = st[2 * p + 1];
    const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
    const float2 zj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (EQM)
        body_eqm(xj, yj, zj, nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r]);
      else
        body<POT>(xj, yj, zj, mj, nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r],
                  ph[r]);
    }
  }
  double* out = part + (int64_t)blockIdx.y * 3 * npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double sx = (double)ax[r].x + (double)ax[r].y;
    double sy = (double)ay[r].x + (double)ay[r].y;
    double sz = (double)az[r].x + (double)az[r].y;
    double sp = POT ? (double)ph[r].x + (double)ph[r].y : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
      if (POT) sp += __shfl_xor_sync(0xffffffffu, sp, o);
    }
    if (lane == 0) {
      const int64_t i = ib + r;
      out[i] = sx;
      out[npad + i] = sy;
      out[2 * npad + i] = sz;
      if (POT) pot[(int64_t)blockIdx.y * npad + i] = sp;
    }
  }
}

template <bool POT, bool EQM>
cudaError_t launch_impl(const PairCfg& c, const float4* st, int64_t npad,
                        float eps2, double* part, double* pot, double* fin,
                        unsigned* ctr, cudaStream_t s) {
  if (c.variant == kTile && c.vjp_tile_pairs == kTJSmall) {
    const int ntiles = (int)(npad / (2 * kTJSmall));
    dim3 grid((unsigned)(npad / (c.nt * c.r)), (unsigned)c.S);
    if (c.nt == 128 && c.r == 4)
      k_pair_tile<128, 4, POT, EQM, kTJSmall><<<grid, 128, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 128 && c.r == 2)
      k_pair_tile<128, 2, POT, EQM, kTJSmall><<<grid, 128, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 128 && c.r == 1)
      k_pair_tile<128, 1, POT, EQM, kTJSmall><<<grid, 128, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 64 && c.r == 2)
      k_pair_tile<64, 2, POT, EQM, kTJSmall><<<grid, 64, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 64 && c.r == 4)
      k_pair_tile<64, 4, POT, EQM, kTJSmall><<<grid, 64, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else
      return cudaErrorInvalidValue;
  } else if (c.variant == kTile) {
    if (c.vjp_tile_pairs != kTJ) return cudaErrorInvalidValue;
    const int ntiles = (int)(npad / (2 * kTJ));
    const int per_block = c.nt * c.r;
    dim3 grid((unsigned)(npad / per_block), (unsigned)c.S);
    if (c.nt == 128 && c.r == 4)
      k_pair_tile<128, 4, POT, EQM><<<grid, 128, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 128 && c.r == 8)
      k_pair_tile<128, 8, POT, EQM><<<grid, 128, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 256 && c.r == 4)
      k_pair_tile<256, 4, POT, EQM><<<grid, 256, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 256 && c.r == 2)
      k_pair_tile<256, 2, POT, EQM><<<grid, 256, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 128 && c.r == 2)
      k_pair_tile<128, 2, POT, EQM><<<grid, 128, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 128 && c.r == 1)
      k_pair_tile<128, 1, POT, EQM><<<grid, 128, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 64 && c.r == 2)
      k_pair_tile<64, 2, POT, EQM><<<grid, 64, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else if (c.nt == 64 && c.r == 4)
      k_pair_tile<64, 4, POT, EQM><<<grid, 64, 0, s>>>(st, ntiles, eps2, npad, part, pot, fin, ctr);
    else
      return cudaErrorInvalidValue;
  } else {
    dim3 grid((unsigned)(npad / (8 * c.r)), (unsigned)c.S);
    if (c.r == 4)
      k_pair_warp<4, POT, EQM><<<grid, 256, 0, s>>>(st, npad / 2, eps2, npad, part, pot);
    else if (c.r == 8)
      k_pair_warp<8, POT, EQM><<<grid, 256, 0, s>>>(st, npad / 2, eps2, npad, part, pot);
    else
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pair_accel(const PairCfg& cfg, const float4* st,
                              int64_t npad, float eps2, double* part,
                              double* pot, cudaStream_t s) {
  if (pot) return launch_impl<true, false>(cfg, st, npad, eps2, part, pot, nullptr, nullptr, s);
  if (cfg.eqm)
    return launch_impl<false, true>(cfg, st, npad, eps2, part, nullptr, nullptr, nullptr, s);
  return launch_impl<false, false>(cfg, st, npad, eps2, part, nullptr, nullptr, nullptr, s);
}

cudaError_t launch_pair_accel_fin(const PairCfg& cfg, const float4* st, int64_t npad,
                                  float eps2, double* part, double* fin, unsigned* ctr,
                                  cudaStream_t s) {
  if (!fin || cfg.variant != kTile || cfg.S < 2)
    return launch_pair_accel(cfg, st, npad, eps2, part, nullptr, s);
  if (cfg.eqm) return launch_impl<false, true>(cfg, st, npad, eps2, part, nullptr, fin, ctr, s);
  return launch_impl<false, false>(cfg, st, npad, eps2, part, nullptr, fin, ctr, s);
}

int pair_blocks_per_sm(const PairCfg& c) {
  int occ = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define NB_OCC(NT, R)                                                               \
  if (c.nt == NT && c.r == R)                                                       \
    e = c.eqm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                      \
                    &occ, k_pair_tile<NT, R, false, true>, NT, 0)                   \
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                      \
                    &occ, k_pair_tile<NT, R, false, false>, NT, 0);
#define NB_OCC_S(NT, R)                                                             \
  if (c.nt == NT && c.r == R)                                                       \
    e = c.eqm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                      \
                    &occ, k_pair_tile<NT, R, false, true, kTJSmall>, NT, 0)         \
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                      \
                    &occ, k_pair_tile<NT, R, false, false, kTJSmall>, NT, 0);
  if (c.variant == kTile && c.vjp_tile_pairs == kTJSmall) {
    NB_OCC_S(128, 4) NB_OCC_S(128, 2) NB_OCC_S(128, 1) NB_OCC_S(64, 2) NB_OCC_S(64, 4)
  } else if (c.variant == kTile) {
    NB_OCC(128, 4) NB_OCC(128, 8) NB_OCC(256, 4) NB_OCC(256, 2) NB_OCC(128, 2) NB_OCC(128, 1)
    NB_OCC(64, 2) NB_OCC(64, 4)
  } else {
    e = c.eqm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_warp<4, false, true>, 256, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_warp<4, false, false>, 256, 0);
  }
#undef NB_OCC
#undef NB_OCC_S
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return occ > 0 ? occ : 1;
}

bool pair_tile_supported(int nt, int r, int tile_pairs, bool vjp) {
  if (tile_pairs == 128) {  // the small-tile instances
    if (vjp) return (nt == 128 && (r == 2 || r == 1)) || (nt == 64 && r == 2);
    return (nt == 128 && (r == 4 || r == 2 || r == 1)) || (nt == 64 && (r == 2 || r == 4));
  }
  return pair_shape_supported(kTile, nt, r, vjp);
}

bool pair_shape_supported(int variant, int nt, int r, bool vjp) {
  if (variant == kWarp) return vjp ? (nt == 256 && (r == 4 || r == 2)) : (nt == 256 && (r == 4 || r == 8));
  if (vjp) return (nt == 256 && r == 2) || (nt == 128 && (r == 4 || r == 2 || r == 1)) ||
                 (nt == 64 && r == 2);
  return (nt == 128 && (r == 4 || r == 8 || r == 2 || r == 1)) || (nt == 256 && (r == 4 || r == 2)) ||
         (nt == 64 && (r == 2 || r == 4));
}

// j-chunk count S for a given shape: the number of blocks covers the
// resident-block slots of the GPU in whole waves as nearly as possible, with
// a mild preference for fewer chunks (less partial-sum traffic)
int choose_chunks(const PairCfg& c, int64_t npad, int sm_count, int blocks_per_sm) {
  if (c.variant == kTile) {
    const int kTJp = c.vjp_tile_pairs;
    const int64_t itiles = npad / (c.nt * c.r);
    const int64_t ntiles = npad / (2 * kTJp);
    const int64_t slots = (int64_t)sm_count * blocks_per_sm;
    double best = 1e30;
    int bestS = 1;
    for (int S = 1; S <= 32 && S <= ntiles; ++S) {
      const int64_t blocks = itiles * S;
      const int64_t waves = (blocks + slots - 1) / slots;
      const double eff = (double)blocks / (double)(waves * slots);
      const double cost = (1.0 / eff) * (1.0 + 0.002 * S);
      if (cost < best - 1e-12) {
        best = cost;
        bestS = S;
      }
    }
    return bestS;
  }
  const int64_t blocks_x = npad / (8 * c.r);
  const int64_t want = (int64_t)sm_count * 8;  // 8 blocks of 8 warps per SM
  int64_t S = (want + blocks_x - 1) / blocks_x;
  const int64_t max_s = (npad / 2) / 64;  // at least 64 pairs per chunk
  if (S > max_s) S = max_s;
  if (S < 1) S = 1;
  return (int)S;
}

// Launch shape: the tile variant when there are enough i-tiles to keep every
// SM busy, otherwise the warp variant.
PairCfg choose_pair_cfg(int64_t npad, int sm_count, bool vjp, bool eqm) {
  PairCfg c;
  c.eqm = eqm;
  c.vjp_tile_pairs = vjp ? vjp_tile_pairs() : kTJ;
  if (npad >= 65536) {
    c.variant = kTile;
    c.nt = vjp ? (eqm ? 128 : 256) : 128;
    c.r = vjp ? 2 : 4;
  } else {
    c.variant = kWarp;
    c.nt = 256;
    c.r = 4;
  }
  const int occ = vjp ? vjp_blocks_per_sm(c) : pair_blocks_per_sm(c);
  c.S = choose_chunks(c, npad, sm_count, occ);
  return c;
}

}  // namespace nb
