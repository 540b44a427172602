// staging.cuh -- writers of the FP32 pair-interleaved staging layouts
// (see nbody_internal.cuh): forward (x, y, z, m) and adjoint
// (x, y, z, m, lambda) records of particle i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nb {

static __device__ __forceinline__ void put_stage(float4* st, int64_t i, float x,
                                          float y, float z, float m) {
  float* f = reinterpret_cast<float*>(st) + 8 * (i >> 1) + (i & 1);
  f[0] = x;
  f[2] = y;
  f[4] = z;
  f[6] = m;
}

static __device__ __forceinline__ void put_stage_xyz(float4* st, int64_t i, float x,
                                              float y, float z) {
  float* f = reinterpret_cast<float*>(st) + 8 * (i >> 1) + (i & 1);
  f[0] = x;
  f[2] = y;
  f[4] = z;
}

static __device__ __forceinline__ void put_vstage(float4* vst, int64_t i, float x,
                                           float y, float z, float m, float lx,
                                           float ly, float lz) {
  float* f = reinterpret_cast<float*>(vst) + 16 * (i >> 1) + (i & 1);
  f[0] = x;
  f[2] = y;
  f[4] = z;
  f[6] = m;
  f[8] = lx;
  f[10] = ly;
  f[12] = lz;
  f[14] = 0.f;
}

}  // namespace nb
