// peaks.cu -- throughput probes of the units the method's kernels use:
// FP32 FMA (scalar and packed f32x2), FP64 FMA, and the MUFU reciprocal
// square root and base-2 exponential.  Each thread runs 8 independent dependency chains so that
// latency is hidden and the pipe's issue rate is what is measured.
#include <cuda_runtime.h>

#include "nbody_internal.cuh"

namespace {

constexpr int kChains = 8;

__global__ void k_ffma(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma2(float* out, int iters, float a, float b) {
  float2 x[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2(threadIdx.x * 1e-3f + k, k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rsqrt(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0f + threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float y;
      asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[k]));
      x[k] = y;
    }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ex2(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 0.5f + threadIdx.x * 1e-4f + 0.01f * k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[k]));
      x[k] = y;
    }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int nbody_peaks(double out[6], void* cuda_stream) {
  if (!out) return NBODY_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return NBODY_ENODEV;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int threads = 256, blocks = sms * 8;
  const size_t nt = (size_t)threads * blocks;
  void* buf = nullptr;
  if (cudaMallocAsync(&buf, nt * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return NBODY_ENOMEM;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(buf, s);
    return NBODY_ECUDA;
  }
  auto timed = [&](auto launch, double ops) -> double {
    launch();  // warm-up
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ops / (ms * 1e-3);
  };
  const int it32 = 20000, it64 = 500, itr = 4000;
  out[0] = timed([&] { k_ffma<<<blocks, threads, 0, s>>>((float*)buf, it32, 0.999f, 1e-3f); },
                 2.0 * kChains * it32 * (double)nt) / 1e12;
  out[1] = timed([&] { k_ffma2<<<blocks, threads, 0, s>>>((float*)buf, it32, 0.999f, 1e-3f); },
                 4.0 * kChains * it32 * (double)nt) / 1e12;
  out[2] = timed([&] { k_dfma<<<blocks, threads, 0, s>>>((double*)buf, it64, 0.999, 1e-3); },
                 2.0 * kChains * it64 * (double)nt) / 1e12;
  out[3] = timed([&] { k_rsqrt<<<blocks, threads, 0, s>>>((float*)buf, itr); },
                 (double)kChains * itr * (double)nt) / 1e9;
  out[4] = (double)sms;
  out[5] = timed([&] { k_ex2<<<blocks, threads, 0, s>>>((float*)buf, itr); },
                 (double)kChains * itr * (double)nt) / 1e9;
  nb::count_launch(10);
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || e != cudaSuccess) return NBODY_ECUDA;
  return NBODY_OK;
}
