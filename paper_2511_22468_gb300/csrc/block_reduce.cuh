// block_reduce.cuh -- deterministic block-level sums (fixed shuffle tree,
// then warps added in index order), used for the parameter-gradient and
// diagnostic reductions.
#pragma once

#include <cuda_runtime.h>

namespace nb {

// deterministic block sum of NV doubles; thread 0 adds the block total to
// out[blockIdx.x * NV + q]
template <int NV>
static __device__ __forceinline__ void block_accumulate(double (&val)[NV],
                                                 double* out) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      val[q] += __shfl_down_sync(0xffffffffu, val[q], o);
    if (lane == 0) sh[q][w] = val[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int k = 0; k < nw; ++k) s += sh[q][k];
      out[(int64_t)blockIdx.x * NV + q] += s;
    }
  }
}

// sum over q = 0..S-1 of p[q * qstride + d * dstride] for d < NV, in
// ascending q (the order fixes the rounding), with the loads of eight
// slices issued before their adds so that their latencies overlap
template <int NV>
static __device__ __forceinline__ void slice_sums(const double* __restrict__ p, int S,
                                                  int64_t qstride, int64_t dstride,
                                                  double (&out)[NV]) {
#pragma unroll
  for (int d = 0; d < NV; ++d) out[d] = 0.0;
  for (int q0 = 0; q0 < S; q0 += 8) {
    double v[8][NV];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int d = 0; d < NV; ++d)
        v[u][d] = (q0 + u < S) ? p[(int64_t)(q0 + u) * qstride + d * dstride] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int d = 0; d < NV; ++d)
        if (q0 + u < S) out[d] += v[u][d];
  }
}

}  // namespace nb
