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

}  // namespace nb
