// mlp.cu -- the density surrogate's training and inference kernels
// (paper Sec. 3 outlook: coupling the simulator with a neural network).
//
//   y = W3 GELU(W2 GELU(W1 u + b1) + b2) + b3,  GELU(z) = z Phi(z),
//   loss = mean (y - t)^2, optimiser Adam.
//
// The layers are small FP32 contractions (batch x 4 x 256, batch x 256 x
// 256, batch x 256 x 1024): one tiled CUDA-core GEMM kernel (64 x 64 output
// tile, 16-deep k-slices in shared memory, 4 x 4 outputs per thread) with
// fused epilogues -- bias + GELU (keeping the pre-activation), bias only,
// and the GELU derivative for the backward pass -- plus column sums for the
// bias gradients, the squared-error gradient and the Adam update.  Every
// sum has a fixed order, so training is bitwise reproducible.
#include <cuda_runtime.h>

#include <cmath>
#include <new>

#include "nbody_internal.cuh"

namespace nb {
namespace {

enum Epi : int { kEpiNone = 0, kEpiBias = 1, kEpiBiasGelu = 2, kEpiGeluBwd = 3 };

constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = TA ? A[k lda + m] : A[m lda + k],
// B(k,n) = TB ? B[n ldb + k] : B[k ldb + n]; epilogue per EPI.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256)
    k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
           const float* __restrict__ B, int ldb, const float* __restrict__ bias,
           float* __restrict__ C, int ldc, float* __restrict__ Zout,
           const float* __restrict__ Zin) {
  __shared__ float As[BK][BM];
  __shared__ float Bs[BK][BN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;  // 0..1023
      // A tile element (kk, mm)
      const int kk = TA ? (e / BM) : (e % BK);
      const int mm = TA ? (e % BM) : (e / BK);
      const int gm = m0 + mm, gk = k0 + kk;
      float a = 0.f;
      if (gm < M && gk < K) a = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = a;
      // B tile element (kk, nn)
      const int kb = TB ? (e % BK) : (e / BN);
      const int nb_ = TB ? (e / BK) : (e % BN);
      const int gn = n0 + nb_, gk2 = k0 + kb;
      float b = 0.f;
      if (gn < N && gk2 < K) b = TB ? B[(int64_t)gn * ldb + gk2] : B[(int64_t)gk2 * ldb + gn];
      Bs[kb][nb_] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      const int64_t o = (int64_t)m * ldc + n;
      float z = acc[i][j];
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
                 const float* Zin, cudaStream_t s) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  k_gemm<TA, TB, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, C, ldc, Zout, Zin);
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
  free_(m->dz2); free_(m->dz1); free_(m->blk); free_(m->loss);
}

// forward pass, keeping pre-activations; output into y (B x nout)
int mlp_forward(nbody_mlp* m, const float* u, int B, float* y) {
  using namespace nb;
  cudaStream_t s = m->s;
  MCK((gemm<false, true, kEpiBiasGelu>(B, m->nh, m->nin, u, m->nin, m->W1(), m->nin,
                                       m->b1(), m->h1, m->nh, m->z1, nullptr, s)));
  MCK((gemm<false, true, kEpiBiasGelu>(B, m->nh, m->nh, m->h1, m->nh, m->W2(), m->nh,
                                       m->b2(), m->h2, m->nh, m->z2, nullptr, s)));
  MCK((gemm<false, true, kEpiBias>(B, m->nout, m->nh, m->h2, m->nh, m->W3(), m->nh,
                                   m->b3(), y, m->nout, nullptr, nullptr, s)));
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
      (rc = malloc_(&m->blk, nblk)) || (rc = malloc_(&m->loss, 1))) {
    free_mlp(m);
    delete m;
    return rc;
  }
  if (cudaMemset(m->w, 0, m->np * sizeof(float)) ||
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
                                   nullptr, nullptr, s)));
  k_colsum<<<(no + 127) / 128, 128, 0, s>>>(m->dy, B, no, gb3);
  count_launch();
  MCK(cudaGetLastError());
  MCK((gemm<false, false, kEpiGeluBwd>(B, nh, no, m->dy, no, m->W3(), nh, nullptr, m->dz2,
                                       nh, nullptr, m->z2, s)));
  // layer 2
  MCK((gemm<true, false, kEpiNone>(nh, nh, B, m->dz2, nh, m->h1, nh, nullptr, gW2, nh,
                                   nullptr, nullptr, s)));
  k_colsum<<<(nh + 127) / 128, 128, 0, s>>>(m->dz2, B, nh, gb2);
  count_launch();
  MCK(cudaGetLastError());
  MCK((gemm<false, false, kEpiGeluBwd>(B, nh, nh, m->dz2, nh, m->W2(), nh, nullptr, m->dz1,
                                       nh, nullptr, m->z1, s)));
  // layer 1
  MCK((gemm<true, false, kEpiNone>(nh, nin, B, m->dz1, nh, u, nin, nullptr, gW1, nin,
                                   nullptr, nullptr, s)));
  k_colsum<<<(nh + 127) / 128, 128, 0, s>>>(m->dz1, B, nh, gb1);
  count_launch();
  MCK(cudaGetLastError());
  if (du)
    MCK((gemm<false, false, kEpiNone>(B, nin, nh, m->dz1, nh, m->W1(), nin, nullptr, du, nin,
                                      nullptr, nullptr, s)));
  if (grads)
    MCK(cudaMemcpyAsync(grads, m->g, m->np * sizeof(float), cudaMemcpyDeviceToDevice, s));
  m->have_grad = true;
  if (loss) {
    MCK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
  }
  return NBODY_OK;
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
