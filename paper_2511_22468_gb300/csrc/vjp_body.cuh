// vjp_body.cuh -- the FP32 inner step of the pair VJP (paper Sec. 2): one
// pair of j-records against one k-particle with the packed f32x2
// instructions, shared by the single-system and the batched VJP kernels.
// Records are the adjoint staging layout (position, mass, negated
// cotangent; staging.cuh).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pair_body.cuh"

namespace nb {

struct IState {
  float2 nx, ny, nz;  // (-x_k, -x_k) ...
  float2 lx, ly, lz;  // (l_k, l_k)
  float2 mk;          // (m_k, m_k)
};

// general masses: j-side record A = (x), B = (z, m), L1 = -(lx, ly), L2 = (-lz)
static __device__ __forceinline__ void vjp_body(const float4& A, const float4& B,
                                         const float4& L1, const float4& L2,
                                         const IState& s, float2 e2,
                                         float2& qx, float2& qy, float2& qz) {
  const float2 dx = __fadd2_rn(make_float2(A.x, A.y), s.nx);
  const float2 dy = __fadd2_rn(make_float2(A.z, A.w), s.ny);
  const float2 dz = __fadd2_rn(make_float2(B.x, B.y), s.nz);
  const float2 mj = make_float2(B.z, B.w);
  float2 s2 = __ffma2_rn(dx, dx, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dz, dz, s2);
  const float2 inv = make_float2(rsqrt_ftz(s2.x), rsqrt_ftz(s2.y));
  const float2 inv2 = __fmul2_rn(inv, inv);
  const float2 inv3 = __fmul2_rn(inv2, inv);
  // u = m_j l_k - m_k l_j  (the record holds -l_j)
  const float2 ux = __ffma2_rn(mj, s.lx, __fmul2_rn(make_float2(L1.x, L1.y), s.mk));
  const float2 uy = __ffma2_rn(mj, s.ly, __fmul2_rn(make_float2(L1.z, L1.w), s.mk));
  const float2 uz = __ffma2_rn(mj, s.lz, __fmul2_rn(make_float2(L2.x, L2.y), s.mk));
  float2 du = __fmul2_rn(dx, ux);
  du = __ffma2_rn(dy, uy, du);
  du = __ffma2_rn(dz, uz, du);
  // c = -3 s^-5 (d.u)
  const float2 c = __fmul2_rn(__fmul2_rn(inv3, __fmul2_rn(inv2, make_float2(-3.f, -3.f))), du);
  qx = __ffma2_rn(c, dx, __ffma2_rn(inv3, ux, qx));
  qy = __ffma2_rn(c, dy, __ffma2_rn(inv3, uy, qy));
  qz = __ffma2_rn(c, dz, __ffma2_rn(inv3, uz, qz));
}

// equal masses: u = l_k - l_j; A += s^-3 u, B += s^-5 (d.u) d
static __device__ __forceinline__ void vjp_body_eqm(const float4& A, const float4& B,
                                             const float4& L1, const float4& L2,
                                             const IState& s, float2 e2, float2* a,
                                             float2* b) {
  const float2 dx = __fadd2_rn(make_float2(A.x, A.y), s.nx);
  const float2 dy = __fadd2_rn(make_float2(A.z, A.w), s.ny);
  const float2 dz = __fadd2_rn(make_float2(B.x, B.y), s.nz);
  float2 s2 = __ffma2_rn(dx, dx, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dz, dz, s2);
  const float2 inv = make_float2(rsqrt_ftz(s2.x), rsqrt_ftz(s2.y));
  const float2 inv2 = __fmul2_rn(inv, inv);
  const float2 inv3 = __fmul2_rn(inv2, inv);
  const float2 ux = __fadd2_rn(s.lx, make_float2(L1.x, L1.y));
  const float2 uy = __fadd2_rn(s.ly, make_float2(L1.z, L1.w));
  const float2 uz = __fadd2_rn(s.lz, make_float2(L2.x, L2.y));
  float2 du = __fmul2_rn(dx, ux);
  du = __ffma2_rn(dy, uy, du);
  du = __ffma2_rn(dz, uz, du);
  const float2 c = __fmul2_rn(__fmul2_rn(inv3, inv2), du);
  a[0] = __ffma2_rn(inv3, ux, a[0]);
  a[1] = __ffma2_rn(inv3, uy, a[1]);
  a[2] = __ffma2_rn(inv3, uz, a[2]);
  b[0] = __ffma2_rn(c, dx, b[0]);
  b[1] = __ffma2_rn(c, dy, b[1]);
  b[2] = __ffma2_rn(c, dz, b[2]);
}

static __device__ __forceinline__ IState load_k(const float4* __restrict__ vst,
                                         int64_t k) {
  const int64_t p = k >> 1;
  const bool odd = (k & 1) != 0;
  const float4 A = vst[4 * p], B = vst[4 * p + 1];
  const float4 L1 = vst[4 * p + 2], L2 = vst[4 * p + 3];
  const float x = odd ? A.y : A.x, y = odd ? A.w : A.z, z = odd ? B.y : B.x;
  const float m = odd ? B.w : B.z;
  const float lx = -(odd ? L1.y : L1.x), ly = -(odd ? L1.w : L1.z);
  const float lz = -(odd ? L2.y : L2.x);
  IState s;
  s.nx = make_float2(-x, -x);
  s.ny = make_float2(-y, -y);
  s.nz = make_float2(-z, -z);
  s.lx = make_float2(lx, lx);
  s.ly = make_float2(ly, ly);
  s.lz = make_float2(lz, lz);
  s.mk = make_float2(m, m);
  return s;
}

// mass-gradient sum of one j-pair: M_k += ((-l_j) . d) s^-3 (the record
// holds -l_j), so that dL/dm_k = G sum_kicks c M_k
static __device__ __forceinline__ void mass_body(const float4& A, const float4& B,
                                          const float4& L1, const float4& L2,
                                          const IState& s, float2 e2, float2& mk) {
  const float2 dx = __fadd2_rn(make_float2(A.x, A.y), s.nx);
  const float2 dy = __fadd2_rn(make_float2(A.z, A.w), s.ny);
  const float2 dz = __fadd2_rn(make_float2(B.x, B.y), s.nz);
  float2 s2 = __ffma2_rn(dx, dx, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dz, dz, s2);
  const float2 inv = make_float2(rsqrt_ftz(s2.x), rsqrt_ftz(s2.y));
  const float2 inv3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
  float2 dl = __fmul2_rn(dx, make_float2(L1.x, L1.y));
  dl = __ffma2_rn(dy, make_float2(L1.z, L1.w), dl);
  dl = __ffma2_rn(dz, make_float2(L2.x, L2.y), dl);
  mk = __ffma2_rn(dl, inv3, mk);
}

}  // namespace nb
