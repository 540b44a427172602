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
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "nbody_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)4 << 20;  // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The device address of g_scratch, looked up with the device current (in
// host code the name g_scratch is only a host-side stand-in, not a device
// address).  A module's device address belongs to one context: after
// cudaDeviceReset the device's primary context is re-created and the
// library's module may be loaded at another address, so each cached address
// is keyed by the unique id of the context it was looked up in, and looked
// up again when the current context's id differs.
struct Slot {
  unsigned long long ctx_id;
  void* addr;
};
Slot g_slot[kMaxDevices] = {};
std::mutex g_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_fn_looked_up = false;

// id of the calling thread's current context (unique for the life of the
// process), 0 when there is none or the driver does not report it; the
// driver functions are reached through the runtime, so the library does not
// link against the driver library.  Called with g_mu held.
unsigned long long current_context_id() {
  if (!g_fn_looked_up) {
    g_fn_looked_up = true;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                         &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault,
                                         &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f1 = f2 = nullptr;
    }
    g_ctx_current = (CtxGetCurrentFn)f1;
    g_ctx_id = (CtxGetIdFn)f2;
  }
  if (!g_ctx_current || !g_ctx_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (g_ctx_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return NBODY_ENODEV;
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = current_context_id();
  Slot& sl = g_slot[dev];
  if (!sl.addr || id == 0 || id != sl.ctx_id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NBODY_ECUDA;
    }
    sl.addr = p;
    sl.ctx_id = current_context_id();  // the lookup made the context current
  }
  *out = sl.addr;
  return NBODY_OK;
}

// the recentring origin, passed by value, into the scratch array: the
// caller's host copy is read when the call is made, never later by a copy
// waiting on the stream
__global__ void k_put_center(double* cen, double cx, double cy, double cz) {
  cen[0] = cx;
  cen[1] = cy;
  cen[2] = cz;
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
  if (e == cudaSuccess) {
    k_put_center<<<1, 1, 0, s>>>(cen, center[0], center[1], center[2]);
    nb::count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = nb::launch_stage(xp, mp, cen, n, npad, st, s);
  if (e == cudaSuccess)
    e = nb::launch_pair_accel(cfg, st, npad, (float)(eps * eps), part, nullptr, s);
  if (e == cudaSuccess)
    e = nb::launch_reduce_partials(part, cfg.S, npad, n, G, acc, s);
  return e == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}
