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
// (CG: loads through L2 only, for slices other blocks of the running kernel
// have just written)
template <int NV, bool CG = false>
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
      for (int d = 0; d < NV; ++d) {
        const double* a = p + (int64_t)(q0 + u) * qstride + d * dstride;
        v[u][d] = (q0 + u < S) ? (CG ? __ldcg(a) : *a) : 0.0;
      }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int d = 0; d < NV; ++d)
        if (q0 + u < S) out[d] += v[u][d];
  }
}

// Last-block reduction of a pair kernel split into S j-chunks (grid.y):
// of the S blocks of row tile blockIdx.x, the one that finishes last sums
// the tile's S partial slices part[q][3][npad] (and mpart[q][npad] when
// given) in ascending q, the order slice_sums gives a consumer, so the sums
// are bitwise the ones the consumer would form; they go to fin[0..2][npad]
// (and fin[3][npad]).  ctr[blockIdx.x] counts the finished chunks and is
// re-armed to 0 by the last block; no block waits for another.  Every thread
// of the block calls this after storing its partial sums; rows i0 + r * NT.
template <int NT, int R>
static __device__ __forceinline__ void finish_row_tile(const double* part, const double* mpart,
                                                       int S, int64_t npad, int64_t i0,
                                                       double* fin, unsigned* ctr) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr + blockIdx.x, 1u) == (unsigned)(S - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i0 + r * NT;
    double s3[3];
    slice_sums<3, true>(part + i, S, 3 * npad, npad, s3);
    fin[i] = s3[0];
    fin[npad + i] = s3[1];
    fin[2 * npad + i] = s3[2];
    if (mpart) {
      double s1[1];
      slice_sums<1, true>(mpart + i, S, npad, 0, s1);
      fin[3 * npad + i] = s1[0];
    }
  }
  if (threadIdx.x == 0) ctr[blockIdx.x] = 0u;
}

}  // namespace nb
