// staging.cuh -- writers of the FP32 pair-interleaved staging layouts
// (see nbody_internal.cuh): forward (x, y, z, m) and adjoint
// (x, y, z, m, lambda) records of particle i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nb {

// Staged position of pad particles: far enough that their pull on any real
// particle is below 1e-33 of its acceleration even without the mass factor
// (the equal-mass kernels do not multiply by m_j), yet |d|^2 ~ 3e36 stays
// inside the FP32 range.
constexpr float kPadPos = 1e18f;

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

// adjoint record: the cotangent is stored negated (-l), so that the pair
// VJP forms l_k - l_j with one packed add
static __device__ __forceinline__ void put_vstage(float4* vst, int64_t i, float x,
                                           float y, float z, float m, float lx,
                                           float ly, float lz) {
  float* f = reinterpret_cast<float*>(vst) + 16 * (i >> 1) + (i & 1);
  f[0] = x;
  f[2] = y;
  f[4] = z;
  f[6] = m;
  f[8] = -lx;
  f[10] = -ly;
  f[12] = -lz;
  f[14] = 0.f;
}

}  // namespace nb
