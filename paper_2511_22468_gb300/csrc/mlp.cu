// mlp.cu -- the density surrogate's training and inference kernels
// (paper Sec. 3 outlook: coupling the simulator with a neural network).
//
//   y = W3 GELU(W2 GELU(W1 u + b1) + b2) + b3,  GELU(z) = z Phi(z),
//   loss = mean (y - t)^2, optimiser Adam.
//
// The layers are dense FP32 contractions (batch x 4 x 256, batch x 256 x
// 256, batch x 256 x 1024 and their transposes in the backward pass), run
// on the fifth-generation tensor cores: one GEMM kernel whose 128 x 32
// output tile accumulates in tensor memory (tcgen05.mma, kind::tf32, one
// issuing thread, completion through per-stage mbarriers), with operands
// staged by the block's threads in the K-major core-matrix layout into two
// shared-memory stages, the next slice loaded while the tensor cores work.
// FP32 accuracy is kept by the three-term TF32 split: each operand a = a_hi
// + a_lo (both TF32), a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, the dropped
// a_lo b_lo below FP32 rounding.  Epilogues are fused -- bias + GELU
// (keeping the pre-activation), bias only, and the GELU derivative for the
// backward pass -- beside column sums for the bias gradients, the
// squared-error gradient and the Adam update.  Every sum has a fixed order,
// so training is bitwise reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <new>

#include "nbody_internal.cuh"

namespace nb {
namespace {

enum Epi : int { kEpiNone = 0, kEpiBias = 1, kEpiBiasGelu = 2, kEpiGeluBwd = 3 };

// output tile (M x N), k-slice and pipeline depth of the tensor-core GEMM
constexpr int TM = 128, TN = 32, TK = 32, kStages = 2;
// K-major, no-swizzle operand tiles: a core matrix is 8 rows x 16 bytes
// (4 FP32/TF32 values), core matrices adjacent in k are kLBO bytes apart and
// those adjacent in rows kSBO bytes apart
constexpr uint32_t kLBO = 128, kSBO = (TK / 4) * 128;
// bytes of one stage: A hi, A lo (TM x TK), B hi, B lo (TN x TK)
constexpr uint32_t kATile = TM * TK * 4, kBTile = TN * TK * 4;
constexpr uint32_t kStageBytes = 2 * kATile + 2 * kBTile;
constexpr size_t kGemmSmem = (size_t)kStages * kStageBytes + 1024;  // + alignment slack
// per-thread share of one slice: A values, B values
constexpr int kAPer = TM * TK / 128, kBPer = TN * TK / 128;
// nanoseconds (of the GPU's global timer) before an mbarrier wait is given
// up, and a cap on the polls as well (whichever comes first); the MMAs it
// waits for take microseconds
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint32_t kWaitPolls = 1u << 26;

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// FP32 -> TF32 (round to nearest, ties away), kept in a 32-bit container
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) of a K-major tile of TK columns
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 2) * kLBO + (row & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor (K-major, no swizzle): start address,
// leading (k) and stride (row) byte offsets in 16-byte units, descriptor
// version 1 at bit 46, layout type 0
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) |
         ((uint64_t)(kSBO >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B,
// both K-major, N = TN, M = TM
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for phase `parity` of the mbarrier, at most kWaitNs of wall-clock
// time (each poll returns within the hardware's own short suspend limit);
// false when it expired
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t poll = 0; poll < kWaitPolls; ++poll) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = TA ? A[k lda + m] : A[m lda + k],
// B(k,n) = TB ? B[n ldb + k] : B[k ldb + n]; epilogue per EPI.  Block: 4
// warps, output tile TM x TN at (blockIdx.y TM, blockIdx.x TN).  Per k-slice
// the threads write A (TM x TK) and B^T (TN x TK) as TF32 hi and lo parts
// into one of two shared-memory stages, thread 0 issues the 3 x TK/8 MMAs
// into tensor memory and commits them to that stage's mbarrier; the next
// slice's global values are loaded into registers while those MMAs run, and
// a stage is rewritten only after the MMAs that read it have completed.
// Warp w reads accumulator rows 32 w .. 32 w + 31 (its tensor-memory lanes).
// A wait that expires sets bit 1 of *status and skips the epilogue.
// no_mma != 0 (the failure-detection test only) issues no MMA and no commit,
// so that the waits expire.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128)
    k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
           const float* __restrict__ B, int ldb, const float* __restrict__ bias,
           float* __restrict__ C, int ldc, float* __restrict__ Zout,
           const float* __restrict__ Zin, int* __restrict__ status, int no_mma) {
  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ uint32_t tmem_slot;
  // stages start on a 1024-byte boundary of the shared window
  const uint32_t dsm_a = smem_addr(dsm);
  const uint32_t base_a = (dsm_a + 1023u) & ~1023u;
  unsigned char* base = dsm + (base_a - dsm_a);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  if (warp == 0) {  // TN accumulator columns of tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"((uint32_t)TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int q = 0; q < kStages; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[q])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const int nslices = (K + TK - 1) / TK;

  // this thread's global values of slice sl (zero outside the matrices)
  float ra[kAPer], rb[kBPer];
  auto load_slice = [&](int sl) {
    const int k0 = sl * TK;
#pragma unroll
    for (int q = 0; q < kAPer; ++q) {
      const int e = t + 128 * q;
      const int row = TA ? (e % TM) : (e / TK);
      const int kk = TA ? (e / TM) : (e % TK);
      const int gm = m0 + row, gk = k0 + kk;
      ra[q] = (gm < M && gk < K) ? (TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk])
                                 : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kBPer; ++q) {
      const int e = t + 128 * q;
      const int row = TB ? (e / TK) : (e % TN);
      const int kk = TB ? (e % TK) : (e / TN);
      const int gn = n0 + row, gk = k0 + kk;
      rb[q] = (gn < N && gk < K) ? (TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn])
                                 : 0.f;
    }
  };
  if (nslices > 0) load_slice(0);

  bool ok = true;
  int last = -1;  // last committed slice
  for (int sl = 0; sl < nslices && ok; ++sl) {
    const int st = sl % kStages;
    unsigned char* sa_hi = base + st * kStageBytes;
    unsigned char* sa_lo = sa_hi + kATile;
    unsigned char* sb_hi = sa_lo + kATile;
    unsigned char* sb_lo = sb_hi + kBTile;
    // the stage's previous MMAs (slice sl - kStages) have finished reading it
    if (sl >= kStages) {
      ok = mbar_wait(smem_addr(&bars[st]), (uint32_t)(((sl - kStages) / kStages) & 1));
      if (!ok) break;
    }
#pragma unroll
    for (int q = 0; q < kAPer; ++q) {
      const int e = t + 128 * q;
      const uint32_t o = kmajor_off(TA ? (e % TM) : (e / TK), TA ? (e / TM) : (e % TK));
      const float hi = to_tf32(ra[q]);
      *reinterpret_cast<float*>(sa_hi + o) = hi;
      *reinterpret_cast<float*>(sa_lo + o) = to_tf32(ra[q] - hi);
    }
#pragma unroll
    for (int q = 0; q < kBPer; ++q) {
      const int e = t + 128 * q;
      const uint32_t o = kmajor_off(TB ? (e / TK) : (e % TN), TB ? (e % TK) : (e / TN));
      const float hi = to_tf32(rb[q]);
      *reinterpret_cast<float*>(sb_hi + o) = hi;
      *reinterpret_cast<float*>(sb_lo + o) = to_tf32(rb[q] - hi);
    }
    // the staged tiles become visible to the tensor cores' (async) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0 && !no_mma) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_addr(sa_hi), al = smem_addr(sa_lo);
      const uint32_t bh = smem_addr(sb_hi), bl = smem_addr(sb_lo);
#pragma unroll
      for (int ks = 0; ks < TK / 8; ++ks) {  // K = 8 per MMA: two core matrices
        const uint32_t off = (uint32_t)ks * 2 * kLBO;
        const uint32_t acc = (sl == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bh + off), acc);
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bl + off), 1u);
        mma_tf32(tmem, smem_desc(al + off), smem_desc(bh + off), 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&bars[st]))
          : "memory");
    }
    last = sl;
    if (sl + 1 < nslices) load_slice(sl + 1);  // in flight while the MMAs run
  }
  // the last commit covers every MMA issued before it
  if (ok && last >= 0)
    ok = mbar_wait(smem_addr(&bars[last % kStages]), (uint32_t)((last / kStages) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) atomicOr(status, 2);
  if (ok && nslices > 0) {
    const int m = m0 + 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n >= N) break;
          const int64_t o = (int64_t)m * ldc + n;
          float z = __uint_as_float(r[j]);
          if (EPI == kEpiBias || EPI == kEpiBiasGelu) z += bias[n];
          if (EPI == kEpiBiasGelu) {
            Zout[o] = z;
            C[o] = gelu(z);
          } else if (EPI == kEpiGeluBwd) {
            C[o] = z * gelu_grad(Zin[o]);
          } else {
            C[o] = z;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // after an expired wait, give the MMAs in flight one more bounded wait
  // before the accumulator columns are released
  if (!ok && last >= 0) mbar_wait(smem_addr(&bars[last % kStages]), (uint32_t)((last / kStages) & 1));
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TN)
                 : "memory");
}

// out[n] = sum_r X[r][n] (rows in order)
__global__ void k_colsum(const float* __restrict__ X, int rows, int cols,
                         float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += X[(int64_t)r * cols + n];
  out[n] = s;
}

// dY = 2 (y - t) / count; per-block sums of (y - t)^2 in FP64
__global__ void __launch_bounds__(256)
    k_mse(const float* __restrict__ y, const float* __restrict__ t, int64_t count,
          float* __restrict__ dy, double* __restrict__ blk) {
  __shared__ double sh[256];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double s = 0.0;
  if (i < count) {
    const float d = y[i] - t[i];
    dy[i] = 2.0f * d / (float)count;
    s = (double)d * (double)d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) blk[blockIdx.x] = sh[0];
}

__global__ void k_sum_blocks(const double* __restrict__ blk, int nblk, int64_t count,
                             float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += blk[k];
  loss[0] = (float)(s / (double)count);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, int64_t n,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// t_rep[r][o] = target[o]
__global__ void k_rep_rows(const float* __restrict__ target, int rows, int cols,
                           float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  out[i] = target[i % cols];
}

// Adam on the inputs, each row its own problem: the row's error is the mean
// over its cols outputs, so its gradient is rows times the batch gradient
__global__ void k_adam_inputs(float* __restrict__ u, const float* __restrict__ du,
                              float* __restrict__ m, float* __restrict__ v, int64_t n,
                              float scale, float lr, float c1, float c2, float lo,
                              float hi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = du[i] * scale;
  const float mi = 0.9f * m[i] + 0.1f * g;
  const float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  const float x = u[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  u[i] = fminf(fmaxf(x, lo), hi);
}

// per-row mean squared error
__global__ void k_row_mse(const float* __restrict__ y, const float* __restrict__ t,
                          int rows, int cols, float* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float s = 0.f;
  for (int o = 0; o < cols; ++o) {
    const float d = y[(int64_t)r * cols + o] - t[(int64_t)r * cols + o];
    s += d * d;
  }
  out[r] = s / (float)cols;
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const float* B,
                 int ldb, const float* bias, float* C, int ldc, float* Zout,
                 const float* Zin, int* status, int no_mma, cudaStream_t s) {
  // the two stages take more than the default 48 KB of dynamic shared
  // memory: raise the kernel's limit once per device
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(k_gemm<TA, TB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGemmSmem);
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit, std::memory_order_release);
  }
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  k_gemm<TA, TB, EPI><<<grid, 128, kGemmSmem, s>>>(M, N, K, A, lda, B, ldb, bias, C, ldc, Zout,
                                                   Zin, status, no_mma);
  count_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace nb

struct nbody_mlp {
  int nin = 0, nh = 0, nout = 0, maxb = 0;
  cudaStream_t s = nullptr;
  int64_t np = 0;
  float* w = nullptr;  // flat parameters
  float* g = nullptr;  // gradients
  float* am = nullptr; // Adam moments
  float* av = nullptr;
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *y = nullptr;
  float *dy = nullptr, *dz2 = nullptr, *dz1 = nullptr;
  double* blk = nullptr;
  float* loss = nullptr;
  int* status = nullptr;  // bit 1: a tensor-core GEMM's bounded wait expired
  // failure-detection test only (environment NBODY_MLP_TEST_NO_MMA=1 at
  // creation): the GEMMs issue no MMA, so their bounded waits expire
  int no_mma = 0;
  int64_t step = 0;
  bool have_grad = false;
  // parameter views
  float *W1() { return w; }
  float *b1() { return w + (int64_t)nh * nin; }
  float *W2() { return b1() + nh; }
  float *b2() { return W2() + (int64_t)nh * nh; }
  float *W3() { return b2() + nh; }
  float *b3() { return W3() + (int64_t)nout * nh; }
};

namespace {

#define MCK(call)                              \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return NBODY_ECUDA; \
  } while (0)

template <class T>
int malloc_(T** p, size_t n) {
  if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return NBODY_ENOMEM;
  }
  return NBODY_OK;
}

template <class T>
void free_(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_mlp(nbody_mlp* m) {
  free_(m->w); free_(m->g); free_(m->am); free_(m->av); free_(m->z1);
  free_(m->h1); free_(m->z2); free_(m->h2); free_(m->y); free_(m->dy);
  free_(m->dz2); free_(m->dz1); free_(m->blk); free_(m->loss); free_(m->status);
}

// forward pass, keeping pre-activations; output into y (B x nout)
int mlp_forward(nbody_mlp* m, const float* u, int B, float* y) {
  using namespace nb;
  cudaStream_t s = m->s;
  MCK((gemm<false, true, kEpiBiasGelu>(B, m->nh, m->nin, u, m->nin, m->W1(), m->nin,
                                       m->b1(), m->h1, m->nh, m->z1, nullptr, m->status, m->no_mma, s)));
  MCK((gemm<false, true, kEpiBiasGelu>(B, m->nh, m->nh, m->h1, m->nh, m->W2(), m->nh,
                                       m->b2(), m->h2, m->nh, m->z2, nullptr, m->status, m->no_mma, s)));
  MCK((gemm<false, true, kEpiBias>(B, m->nout, m->nh, m->h2, m->nh, m->W3(), m->nh,
                                   m->b3(), y, m->nout, nullptr, nullptr, m->status, m->no_mma, s)));
  return NBODY_OK;
}

}  // namespace

extern "C" {

int nbody_mlp_create(nbody_mlp** out, int n_in, int n_hidden, int n_out,
                     int max_batch, void* cuda_stream) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1) return NBODY_EINVAL;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return NBODY_ENODEV;
  }
  nbody_mlp* m = new (std::nothrow) nbody_mlp();
  if (!m) return NBODY_ENOMEM;
  m->nin = n_in;
  m->nh = n_hidden;
  m->nout = n_out;
  m->maxb = max_batch;
  m->s = (cudaStream_t)cuda_stream;
  {
    const char* e = std::getenv("NBODY_MLP_TEST_NO_MMA");
    m->no_mma = (e && e[0] == '1' && e[1] == '\0') ? 1 : 0;
  }
  m->np = (int64_t)n_hidden * n_in + n_hidden + (int64_t)n_hidden * n_hidden + n_hidden +
          (int64_t)n_out * n_hidden + n_out;
  const size_t bh = (size_t)max_batch * n_hidden, bo = (size_t)max_batch * n_out;
  const int nblk = (int)(((int64_t)bo + 255) / 256);
  int rc;
  if ((rc = malloc_(&m->w, m->np)) || (rc = malloc_(&m->g, m->np)) ||
      (rc = malloc_(&m->am, m->np)) || (rc = malloc_(&m->av, m->np)) ||
      (rc = malloc_(&m->z1, bh)) || (rc = malloc_(&m->h1, bh)) ||
      (rc = malloc_(&m->z2, bh)) || (rc = malloc_(&m->h2, bh)) ||
      (rc = malloc_(&m->y, bo)) || (rc = malloc_(&m->dy, bo)) ||
      (rc = malloc_(&m->dz2, bh)) || (rc = malloc_(&m->dz1, bh)) ||
      (rc = malloc_(&m->blk, nblk)) || (rc = malloc_(&m->loss, 1)) ||
      (rc = malloc_(&m->status, 1))) {
    free_mlp(m);
    delete m;
    return rc;
  }
  if (cudaMemset(m->w, 0, m->np * sizeof(float)) || cudaMemset(m->status, 0, sizeof(int)) ||
      cudaMemset(m->am, 0, m->np * sizeof(float)) ||
      cudaMemset(m->av, 0, m->np * sizeof(float))) {
    cudaGetLastError();
    free_mlp(m);
    delete m;
    return NBODY_ECUDA;
  }
  *out = m;
  return NBODY_OK;
}

int64_t nbody_mlp_num_params(const nbody_mlp* m) { return m ? m->np : 0; }

int nbody_mlp_set_params(nbody_mlp* m, const float* p) {
  if (!m || !p) return NBODY_EINVAL;
  MCK(cudaMemcpyAsync(m->w, p, m->np * sizeof(float), cudaMemcpyDefault, m->s));
  MCK(cudaMemsetAsync(m->am, 0, m->np * sizeof(float), m->s));
  MCK(cudaMemsetAsync(m->av, 0, m->np * sizeof(float), m->s));
  MCK(cudaStreamSynchronize(m->s));
  m->step = 0;
  m->have_grad = false;
  return NBODY_OK;
}

int nbody_mlp_get_params(nbody_mlp* m, float* p) {
  if (!m || !p) return NBODY_EINVAL;
  MCK(cudaMemcpyAsync(p, m->w, m->np * sizeof(float), cudaMemcpyDefault, m->s));
  MCK(cudaStreamSynchronize(m->s));
  return NBODY_OK;
}

int nbody_mlp_forward(nbody_mlp* m, const float* u, int batch, float* y) {
  if (!m || !u || !y || batch < 1 || batch > m->maxb) return NBODY_EINVAL;
  return mlp_forward(m, u, batch, y);
}

int nbody_mlp_loss_grad(nbody_mlp* m, const float* u, const float* t, int batch,
                        float* loss, float* grads, float* du) {
  using namespace nb;
  if (!m || !u || !t || batch < 1 || batch > m->maxb) return NBODY_EINVAL;
  cudaStream_t s = m->s;
  const int B = batch, nin = m->nin, nh = m->nh, no = m->nout;
  int rc = mlp_forward(m, u, B, m->y);
  if (rc) return rc;
  const int64_t count = (int64_t)B * no;
  const int nblk = (int)((count + 255) / 256);
  k_mse<<<nblk, 256, 0, s>>>(m->y, t, count, m->dy, m->blk);
  count_launch();
  MCK(cudaGetLastError());
  k_sum_blocks<<<1, 32, 0, s>>>(m->blk, nblk, count, m->loss);
  count_launch();
  MCK(cudaGetLastError());
  float* gW1 = m->g;
  float* gb1 = gW1 + (int64_t)nh * nin;
  float* gW2 = gb1 + nh;
  float* gb2 = gW2 + (int64_t)nh * nh;
  float* gW3 = gb2 + nh;
  float* gb3 = gW3 + (int64_t)no * nh;
  // layer 3: dW3 = dY^T H2, db3 = colsum dY, dZ2 = (dY W3) * GELU'(Z2)
  MCK((gemm<true, false, kEpiNone>(no, nh, B, m->dy, no, m->h2, nh, nullptr, gW3, nh,
                                   nullptr, nullptr, m->status, m->no_mma, s)));
  k_colsum<<<(no + 127) / 128, 128, 0, s>>>(m->dy, B, no, gb3);
  count_launch();
  MCK(cudaGetLastError());
  MCK((gemm<false, false, kEpiGeluBwd>(B, nh, no, m->dy, no, m->W3(), nh, nullptr, m->dz2,
                                       nh, nullptr, m->z2, m->status, m->no_mma, s)));
  // layer 2
  MCK((gemm<true, false, kEpiNone>(nh, nh, B, m->dz2, nh, m->h1, nh, nullptr, gW2, nh,
                                   nullptr, nullptr, m->status, m->no_mma, s)));
  k_colsum<<<(nh + 127) / 128, 128, 0, s>>>(m->dz2, B, nh, gb2);
  count_launch();
  MCK(cudaGetLastError());
  MCK((gemm<false, false, kEpiGeluBwd>(B, nh, nh, m->dz2, nh, m->W2(), nh, nullptr, m->dz1,
                                       nh, nullptr, m->z1, m->status, m->no_mma, s)));
  // layer 1
  MCK((gemm<true, false, kEpiNone>(nh, nin, B, m->dz1, nh, u, nin, nullptr, gW1, nin,
                                   nullptr, nullptr, m->status, m->no_mma, s)));
  k_colsum<<<(nh + 127) / 128, 128, 0, s>>>(m->dz1, B, nh, gb1);
  count_launch();
  MCK(cudaGetLastError());
  if (du)
    MCK((gemm<false, false, kEpiNone>(B, nin, nh, m->dz1, nh, m->W1(), nin, nullptr, du, nin,
                                      nullptr, nullptr, m->status, m->no_mma, s)));
  if (grads)
    MCK(cudaMemcpyAsync(grads, m->g, m->np * sizeof(float), cudaMemcpyDeviceToDevice, s));
  m->have_grad = true;
  if (loss) {
    MCK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
  }
  return NBODY_OK;
}

int nbody_mlp_get_status(nbody_mlp* m) {
  if (!m) return NBODY_EINVAL;
  int h = 0;
  MCK(cudaMemcpyAsync(&h, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->s));
  MCK(cudaStreamSynchronize(m->s));
  return (h & 2) ? NBODY_ETIMEOUT : NBODY_OK;
}

int nbody_mlp_adam_step(nbody_mlp* m, float lr, float beta1, float beta2, float eps) {
  if (!m) return NBODY_EINVAL;
  if (!m->have_grad) return NBODY_ESTATE;
  m->step += 1;
  const float c1 = 1.0f - powf(beta1, (float)m->step);
  const float c2 = 1.0f - powf(beta2, (float)m->step);
  nb::k_adam<<<(unsigned)((m->np + 255) / 256), 256, 0, m->s>>>(
      m->w, m->g, m->am, m->av, m->np, lr, beta1, beta2, eps, c1, c2);
  nb::count_launch();
  MCK(cudaGetLastError());
  return NBODY_OK;
}

int nbody_mlp_invert(nbody_mlp* m, const float* target, int starts, float* u,
                     int iters, float lr, float lo, float hi, float* loss) {
  using namespace nb;
  if (!m || !target || !u || starts < 1 || starts > m->maxb || iters < 0 || !(hi >= lo))
    return NBODY_EINVAL;
  cudaStream_t s = m->s;
  const int64_t nu = (int64_t)starts * m->nin;
  float *trep = nullptr, *du = nullptr, *am = nullptr, *av = nullptr;
  const size_t bytes = ((size_t)starts * m->nout + 3 * (size_t)nu) * sizeof(float);
  if (cudaMallocAsync((void**)&trep, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return NBODY_ENOMEM;
  }
  du = trep + (size_t)starts * m->nout;
  am = du + nu;
  av = am + nu;
  int rc = NBODY_OK;
  cudaError_t e = cudaMemsetAsync(am, 0, 2 * nu * sizeof(float), s);
  if (e == cudaSuccess) {
    const int64_t tot = (int64_t)starts * m->nout;
    k_rep_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(target, starts, m->nout, trep);
    count_launch();
    e = cudaGetLastError();
  }
  const bool keep = m->have_grad;
  for (int it = 0; it < iters && e == cudaSuccess && rc == NBODY_OK; ++it) {
    rc = nbody_mlp_loss_grad(m, u, trep, starts, nullptr, nullptr, du);
    if (rc) break;
    const float c1 = 1.0f - powf(0.9f, (float)(it + 1));
    const float c2 = 1.0f - powf(0.999f, (float)(it + 1));
    k_adam_inputs<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(u, du, am, av, nu,
                                                              (float)starts, lr, c1, c2, lo, hi);
    count_launch();
    e = cudaGetLastError();
  }
  (void)keep;
  m->have_grad = false;  // the kept parameter gradient was overwritten
  if (rc == NBODY_OK && e == cudaSuccess && loss) {
    rc = mlp_forward(m, u, starts, m->y);
    if (rc == NBODY_OK) {
      k_row_mse<<<(starts + 127) / 128, 128, 0, s>>>(m->y, trep, starts, m->nout, loss);
      count_launch();
      e = cudaGetLastError();
    }
  }
  cudaFreeAsync(trep, s);
  if (rc) return rc;
  return e == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}

void nbody_mlp_destroy(nbody_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->s);
  free_mlp(m);
  delete m;
}

}  // extern "C"
