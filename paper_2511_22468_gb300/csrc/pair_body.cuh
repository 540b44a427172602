// pair_body.cuh -- the FP32 inner step of the softened pair sum (paper
// Sec. 1): one pair of j-particles against one i-particle with the packed
// f32x2 instructions of sm_100+, shared by the single-system and the batched
// pair kernels.
#pragma once

#include <cuda_runtime.h>

namespace nb {

static __device__ __forceinline__ float rsqrt_ftz(float v) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
  return y;
}

static __device__ __forceinline__ float2 rsqrt2(float2 v) {
  return make_float2(rsqrt_ftz(v.x), rsqrt_ftz(v.y));
}

// one j-pair against one i: accumulates m_j (x_j - x_i) s^-3 into (ax, ay,
// az) and optionally m_j / s into ph.
template <bool POT>
static __device__ __forceinline__ void body(float2 xj, float2 yj, float2 zj,
                                     float2 mj, float2 nx, float2 ny,
                                     float2 nz, float2 e2, float2& ax,
                                     float2& ay, float2& az, float2& ph) {
  const float2 dx = __fadd2_rn(xj, nx);
  const float2 dy = __fadd2_rn(yj, ny);
  const float2 dz = __fadd2_rn(zj, nz);
  float2 s2 = __ffma2_rn(dx, dx, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dz, dz, s2);
  const float2 inv = rsqrt2(s2);
  const float2 inv2 = __fmul2_rn(inv, inv);
  float2 w = __fmul2_rn(mj, inv);
  if (POT) ph = __fadd2_rn(ph, w);
  w = __fmul2_rn(w, inv2);
  ax = __ffma2_rn(dx, w, ax);
  ay = __ffma2_rn(dy, w, ay);
  az = __ffma2_rn(dz, w, az);
}

// equal masses: accumulates (x_j - x_i) s^-3 (the common mass is applied by
// the consumer) -- one multiply fewer per interaction
static __device__ __forceinline__ void body_eqm(float2 xj, float2 yj, float2 zj,
                                                float2 nx, float2 ny, float2 nz,
                                                float2 e2, float2& ax, float2& ay,
                                                float2& az) {
  const float2 dx = __fadd2_rn(xj, nx);
  const float2 dy = __fadd2_rn(yj, ny);
  const float2 dz = __fadd2_rn(zj, nz);
  float2 s2 = __ffma2_rn(dx, dx, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dz, dz, s2);
  const float2 inv = rsqrt2(s2);
  const float2 w = __fmul2_rn(__fmul2_rn(inv, inv), inv);
  ax = __ffma2_rn(dx, w, ax);
  ay = __ffma2_rn(dy, w, ay);
  az = __ffma2_rn(dz, w, az);
}

static __device__ __forceinline__ void load_i(const float4* __restrict__ st,
                                       int64_t i, float& x, float& y,
                                       float& z) {
  const float4 A = st[2 * (i >> 1)];
  const float4 B = st[2 * (i >> 1) + 1];
  const bool odd = (i & 1) != 0;
  x = odd ? A.y : A.x;
  y = odd ? A.w : A.z;
  z = odd ? B.y : B.x;
}

}  // namespace nb
