// pair_accel_noalloc.cu -- nbody_pair_accel without any device allocation.
//
// nbody_pair_accel obtains its scratch (a padded copy of the positions and
// masses, the FP32 staging array and the per-chunk partial sums) with
// cudaMallocAsync on every call.  Some callers cannot allocate device memory
// at the point where they need forces: an application that reserves all of
// its device memory up front under a fixed budget, or a hot loop that must
// not take the allocator's locks or pay its latency.  This entry point runs
// the same kernels with the same launch shapes, but its scratch is one
// file-scope device array of fixed size, created when the library is loaded
// and held by every GPU that loads the library until the process exits.
//
// The array is shared by every call on a device and keeps the previous
// call's contents; the parts that must start at zero (the padding of the
// position and mass copy) are cleared on every call.  Two calls that overlap
// on the GPU (different streams, no ordering between them) race on the
// array and give undefined results.
#include <cuda_runtime.h>

#include <mutex>

#include "nbody_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)4 << 20;  // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device-side address of g_scratch, looked up once per device; in host code
// the name g_scratch is only a host-side stand-in, not a device address
void* g_addr[kMaxDevices] = {};
std::mutex g_mu;

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return NBODY_ENODEV;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NBODY_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NBODY_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int nbody_pair_accel_noalloc(int64_t n, const double* x,
                                        const double* m, double G, double eps,
                                        const double center[3], double* acc,
                                        void* cuda_stream) {
  if (n < 1 || !x || !m || !acc || !center || !(eps > 0.0)) return NBODY_EINVAL;
  if (n > NBODY_NOALLOC_MAX_N) return NBODY_ESIZE;
  int dev = 0, maj = 0, min = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev) ||
      cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev) ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
    cudaGetLastError();
    return NBODY_ENODEV;
  }
  if (maj != 10 || min != 3) return NBODY_ENODEV;
  void* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;

  const int64_t npad = ((n + nb::kPad - 1) / nb::kPad) * nb::kPad;
  const nb::PairCfg cfg = nb::choose_pair_cfg(npad, sms, false, false);
  const size_t bytes_x = align256((size_t)4 * npad * sizeof(double));
  const size_t bytes_c = 256;
  const size_t bytes_st = align256((size_t)npad * sizeof(float4));
  const size_t bytes_part = (size_t)cfg.S * 3 * npad * sizeof(double);
  if (bytes_x + bytes_c + bytes_st + bytes_part > kScratchBytes) return NBODY_ESIZE;

  char* buf = static_cast<char*>(base);
  double* xp = (double*)buf;
  double* mp = xp + 3 * npad;
  double* cen = (double*)(buf + bytes_x);
  float4* st = (float4*)(buf + bytes_x + bytes_c);
  double* part = (double*)(buf + bytes_x + bytes_c + bytes_st);
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // padding of the position / mass copy must be zero: clear it every call
  cudaError_t e = cudaMemsetAsync(xp, 0, (size_t)4 * npad * sizeof(double), s);
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaMemcpyAsync(xp + (size_t)d * npad, x + (size_t)d * n,
                        (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mp, m, (size_t)n * sizeof(double),
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cen, center, 3 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = nb::launch_stage(xp, mp, cen, n, npad, st, s);
  if (e == cudaSuccess)
    e = nb::launch_pair_accel(cfg, st, npad, (float)(eps * eps), part, nullptr, s);
  if (e == cudaSuccess)
    e = nb::launch_reduce_partials(part, cfg.S, npad, n, G, acc, s);
  return e == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}
