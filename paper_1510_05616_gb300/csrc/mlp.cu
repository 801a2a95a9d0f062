// mlp.cu -- the warm-start network: BF16-weight / FP32-accumulate forward, backward and Adam.
//
// Network (per vesicle): x_hat = (x - mu_in) / sd_in, h1 = silu(W1 x_hat + b1),
// h2 = silu(W2 h1 + b2), y_hat = W3 h2 + b3, prediction y = mu_out + sd_out y_hat.
// Training minimises (1/B) sum_b (1/2)|y_hat_b - t_hat_b|^2 with t_hat = (t - mu_out)/sd_out.
// FP32 master parameters (flattened W1, b1, W2, b2, W3, b3; W row-major (out, in)) are updated
// by Adam; every GEMM reads the BF16-rounded copy of the weights and accumulates in FP32, in a
// fixed order (results are deterministic).  Activations and gradients are FP32.
#include <cuda_bf16.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "stokes_internal.cuh"
#include "stokes_mlp_internal.cuh"

namespace {

constexpr int kT = 32;  // GEMM tile

// C[M x N] = sum_k A(m, k) B(k, n) (+ bias[n]) (+ beta C); row-major storage,
// A(m, k) = TA ? A[k lda + m] : A[m lda + k],  B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
template <bool TA, bool TB, typename BT>
__global__ void gemm_kernel(int M, int N, int K, const float *A, int lda, const BT *B, int ldb,
                            float *C, int ldc, const float *bias, float beta) {
  __shared__ float As[kT][kT + 1], Bs[kT][kT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 16 x 16 threads, 2 x 2 outputs each
  const int m0 = blockIdx.y * kT, n0 = blockIdx.x * kT;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += kT) {
    for (int e = ty * 16 + tx; e < kT * kT; e += 256) {
      const int r = e / kT, c = e % kT;  // As[r = m][c = k], Bs[r = k][c = n]
      const int gm = m0 + r, gk = k0 + c;
      As[r][c] = (gm < M && gk < K) ? (TA ? A[size_t(gk) * lda + gm] : A[size_t(gm) * lda + gk]) : 0.f;
      const int bk = k0 + r, bn = n0 + c;
      float bv = 0.f;
      if (bk < K && bn < N) {
        if constexpr (sizeof(BT) == 2)
          bv = __bfloat162float(TB ? B[size_t(bn) * ldb + bk] : B[size_t(bk) * ldb + bn]);
        else
          bv = TB ? B[size_t(bn) * ldb + bk] : B[size_t(bk) * ldb + bn];
      }
      Bs[r][c] = bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kT; ++k) {
      const float a0 = As[ty * 2][k], a1 = As[ty * 2 + 1][k];
      const float b0 = Bs[k][tx * 2], b1 = Bs[k][tx * 2 + 1];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gm = m0 + ty * 2 + i, gn = n0 + tx * 2 + j;
      if (gm < M && gn < N) {
        float v = acc[i][j] + (bias ? bias[gn] : 0.f);
        if (beta != 0.f) v += beta * C[size_t(gm) * ldc + gn];
        C[size_t(gm) * ldc + gn] = v;
      }
    }
}

template <bool TA, bool TB, typename BT>
void gemm(int M, int N, int K, const float *A, int lda, const BT *B, int ldb, float *C, int ldc,
          const float *bias, float beta, cudaStream_t s) {
  dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT);
  gemm_kernel<TA, TB, BT><<<grid, dim3(16, 16), 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, beta);
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float sg = 1.f / (1.f + __expf(-z));
  return sg * (1.f + z * (1.f - sg));
}

__global__ void silu_kernel(long n, const float *z, float *h) {
  const long t = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) h[t] = silu_f(z[t]);
}

__global__ void dsilu_mul_kernel(long n, const float *z, float *d) {
  const long t = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) d[t] *= dsilu_f(z[t]);
}

// Gather rows idx[b] of X (ld = cols), standardise with (mu, sd): out[b, c].
__global__ void gather_std_kernel(int B, int cols, const float *X, const int *idx, const float *mu,
                                  const float *sd, float *out) {
  const long t = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= long(B) * cols) return;
  const int b = int(t / cols), c = int(t % cols);
  const long r = idx ? idx[b] : b;
  out[t] = (X[r * cols + c] - mu[c]) / sd[c];
}

__global__ void destd_kernel(long n, int cols, const float *yh, const float *mu, const float *sd,
                             float *y) {
  const long t = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = int(t % cols);
  y[t] = mu[c] + sd[c] * yh[t];
}

// dy = (y_hat - t_hat) / B; per-row squared error into rowloss (fixed order).
__global__ void mse_kernel(int B, int cols, const float *yh, const float *th, float *dy,
                           float *rowloss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float s = 0.f;
  for (int c = 0; c < cols; ++c) {
    const float r = yh[size_t(b) * cols + c] - th[size_t(b) * cols + c];
    dy[size_t(b) * cols + c] = r / B;
    s += r * r;
  }
  rowloss[b] = s;
}

// out[c] = sum_b in[b, c] in fixed order (bias gradients, losses).
__global__ void colsum_kernel(int B, int cols, const float *in, float scale, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += in[size_t(b) * cols + c];
  out[c] = float(s * scale);
}

__global__ void adam_kernel(int n, float *theta, const float *g, float *m, float *v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float mm = b1 * m[t] + (1.f - b1) * g[t];
  const float vv = b2 * v[t] + (1.f - b2) * g[t] * g[t];
  m[t] = mm;
  v[t] = vv;
  theta[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void to_bf16_kernel(int n, const float *in, __nv_bfloat16 *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = __float2bfloat16_rn(in[t]);
}

// Column mean and standard deviation of X (rows x cols), FP64 accumulation; sd floor 1e-6.
__global__ void moments_kernel(int rows, int cols, const float *X, float *mu, float *sd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0, q = 0.0;
  for (int r = 0; r < rows; ++r) {
    const double x = X[size_t(r) * cols + c];
    s += x;
    q += x * x;
  }
  const double m = s / rows;
  mu[c] = float(m);
  sd[c] = float(fmax(sqrt(fmax(q / rows - m * m, 0.0)), 1e-6));
}

inline int nb(long n, int b) { return int((n + b - 1) / b); }

}  // namespace

struct stokes_mlp {
  int device = 0;
  std::string err;
  cudaStream_t s = nullptr;
  int n_in = 0, H = 0, n_out = 0, n_params = 0;
  int off[7] = {0};  // offsets of W1, b1, W2, b2, W3, b3 and the end
  float *d_theta = nullptr, *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
  __nv_bfloat16 *d_wb = nullptr;
  float *d_norm = nullptr;  // mu_in, sd_in, mu_out, sd_out
  int t_adam = 0;
  int cap = 0;
  float *d_x = nullptr, *d_z1 = nullptr, *d_h1 = nullptr, *d_z2 = nullptr, *d_h2 = nullptr,
        *d_y = nullptr, *d_t = nullptr, *d_dy = nullptr, *d_d2 = nullptr, *d_d1 = nullptr,
        *d_row = nullptr, *d_loss = nullptr;
};

namespace {

int mfail(stokes_mlp *m, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (m) m->err = buf;
  return code;
}

#define MK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return mfail(m, e_ == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA, \
                   "%s: %s", #call, cudaGetErrorString(e_));                             \
  } while (0)

template <class T>
void mfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <class T>
cudaError_t malloc_n(T *&p, size_t n) {
  mfree(p);
  return cudaMalloc(reinterpret_cast<void **>(&p), std::max<size_t>(n, 1) * sizeof(T));
}

int ensure_batch(stokes_mlp *m, int B) {
  if (B <= m->cap) return STOKES_OK;
  const int H = m->H;
  MK(malloc_n(m->d_x, size_t(B) * m->n_in));
  MK(malloc_n(m->d_z1, size_t(B) * H));
  MK(malloc_n(m->d_h1, size_t(B) * H));
  MK(malloc_n(m->d_z2, size_t(B) * H));
  MK(malloc_n(m->d_h2, size_t(B) * H));
  MK(malloc_n(m->d_y, size_t(B) * m->n_out));
  MK(malloc_n(m->d_t, size_t(B) * m->n_out));
  MK(malloc_n(m->d_dy, size_t(B) * m->n_out));
  MK(malloc_n(m->d_d2, size_t(B) * H));
  MK(malloc_n(m->d_d1, size_t(B) * H));
  MK(malloc_n(m->d_row, B));
  m->cap = B;
  return STOKES_OK;
}

const __nv_bfloat16 *Wb(const stokes_mlp *m, int l) { return m->d_wb + m->off[2 * l]; }
const float *bias(const stokes_mlp *m, int l) { return m->d_theta + m->off[2 * l + 1]; }

// Forward on the standardised inputs in d_x (B rows): y_hat into d_y.
void forward(stokes_mlp *m, int B) {
  const int H = m->H;
  cudaStream_t s = m->s;
  gemm<false, true>(B, H, m->n_in, m->d_x, m->n_in, Wb(m, 0), m->n_in, m->d_z1, H, bias(m, 0), 0.f, s);
  silu_kernel<<<nb(long(B) * H, 256), 256, 0, s>>>(long(B) * H, m->d_z1, m->d_h1);
  gemm<false, true>(B, H, H, m->d_h1, H, Wb(m, 1), H, m->d_z2, H, bias(m, 1), 0.f, s);
  silu_kernel<<<nb(long(B) * H, 256), 256, 0, s>>>(long(B) * H, m->d_z2, m->d_h2);
  gemm<false, true>(B, m->n_out, H, m->d_h2, H, Wb(m, 2), H, m->d_y, m->n_out, bias(m, 2), 0.f, s);
}

// Loss and gradient (into d_grad) of the standardised targets in d_t.
void backward(stokes_mlp *m, int B) {
  const int H = m->H, no = m->n_out;
  cudaStream_t s = m->s;
  float *g = m->d_grad;
  mse_kernel<<<nb(B, 128), 128, 0, s>>>(B, no, m->d_y, m->d_t, m->d_dy, m->d_row);
  colsum_kernel<<<1, 32, 0, s>>>(B, 1, m->d_row, 0.5f / B, m->d_loss);
  // layer 3: gW3 = dy^T h2, gb3 = sum dy, d2 = (dy W3) * silu'(z2)
  gemm<true, false, float>(no, H, B, m->d_dy, no, m->d_h2, H, g + m->off[4], H, nullptr, 0.f, s);
  colsum_kernel<<<nb(no, 64), 64, 0, s>>>(B, no, m->d_dy, 1.f, g + m->off[5]);
  gemm<false, false>(B, H, no, m->d_dy, no, Wb(m, 2), H, m->d_d2, H, nullptr, 0.f, s);
  dsilu_mul_kernel<<<nb(long(B) * H, 256), 256, 0, s>>>(long(B) * H, m->d_z2, m->d_d2);
  // layer 2
  gemm<true, false, float>(H, H, B, m->d_d2, H, m->d_h1, H, g + m->off[2], H, nullptr, 0.f, s);
  colsum_kernel<<<nb(H, 64), 64, 0, s>>>(B, H, m->d_d2, 1.f, g + m->off[3]);
  gemm<false, false>(B, H, H, m->d_d2, H, Wb(m, 1), H, m->d_d1, H, nullptr, 0.f, s);
  dsilu_mul_kernel<<<nb(long(B) * H, 256), 256, 0, s>>>(long(B) * H, m->d_z1, m->d_d1);
  // layer 1
  gemm<true, false, float>(H, m->n_in, B, m->d_d1, H, m->d_x, m->n_in, g + m->off[0], m->n_in,
                           nullptr, 0.f, s);
  colsum_kernel<<<nb(H, 64), 64, 0, s>>>(B, H, m->d_d1, 1.f, g + m->off[1]);
}

}  // namespace

namespace stokes {

int mlp_infer(stokes_mlp *m, int B, const float *x, float *y, cudaStream_t s) {
  cudaStream_t keep = m->s;
  m->s = s;
  int st = ensure_batch(m, B);
  if (st) {
    m->s = keep;
    return st;
  }
  const float *mu_in = m->d_norm, *sd_in = m->d_norm + m->n_in;
  const float *mu_out = m->d_norm + 2 * m->n_in, *sd_out = mu_out + m->n_out;
  gather_std_kernel<<<nb(long(B) * m->n_in, 256), 256, 0, s>>>(B, m->n_in, x, nullptr, mu_in, sd_in, m->d_x);
  forward(m, B);
  destd_kernel<<<nb(long(B) * m->n_out, 256), 256, 0, s>>>(long(B) * m->n_out, m->n_out, m->d_y,
                                                          mu_out, sd_out, y);
  m->s = keep;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? STOKES_OK : mfail(m, STOKES_ERR_CUDA, "mlp_infer: %s", cudaGetErrorString(e));
}

int mlp_dims(const stokes_mlp *m, int *n_in, int *n_out) {
  *n_in = m->n_in;
  *n_out = m->n_out;
  return STOKES_OK;
}

}  // namespace stokes

extern "C" {

int stokes_mlp_create(int device, int n_in, int n_hidden, int n_out, stokes_mlp **out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1) return STOKES_ERR_ARG;
  *out = nullptr;
  stokes_mlp *m = new stokes_mlp();
  m->device = device;
  m->n_in = n_in;
  m->H = n_hidden;
  m->n_out = n_out;
  const int sizes[6] = {n_hidden * n_in, n_hidden, n_hidden * n_hidden, n_hidden, n_out * n_hidden, n_out};
  m->off[0] = 0;
  for (int k = 0; k < 6; ++k) m->off[k + 1] = m->off[k] + sizes[k];
  m->n_params = m->off[6];
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&m->s, cudaStreamNonBlocking) != cudaSuccess) {
    delete m;
    return STOKES_ERR_CUDA;
  }
  int st = STOKES_OK;
  if (malloc_n(m->d_theta, m->n_params) != cudaSuccess || malloc_n(m->d_grad, m->n_params) != cudaSuccess ||
      malloc_n(m->d_m, m->n_params) != cudaSuccess || malloc_n(m->d_v, m->n_params) != cudaSuccess ||
      malloc_n(m->d_wb, m->n_params) != cudaSuccess ||
      malloc_n(m->d_norm, 2 * (n_in + n_out)) != cudaSuccess || malloc_n(m->d_loss, 1) != cudaSuccess)
    st = STOKES_ERR_OOM;
  if (!st) {
    cudaMemset(m->d_theta, 0, sizeof(float) * m->n_params);
    cudaMemset(m->d_m, 0, sizeof(float) * m->n_params);
    cudaMemset(m->d_v, 0, sizeof(float) * m->n_params);
    cudaMemset(m->d_wb, 0, sizeof(__nv_bfloat16) * m->n_params);
    std::vector<float> norm(2 * (n_in + n_out), 0.f);
    for (int c = 0; c < n_in; ++c) norm[n_in + c] = 1.f;
    for (int c = 0; c < n_out; ++c) norm[2 * n_in + n_out + c] = 1.f;
    cudaMemcpy(m->d_norm, norm.data(), sizeof(float) * norm.size(), cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) st = STOKES_ERR_CUDA;
  }
  if (st) {
    stokes_mlp_destroy(m);
    return st;
  }
  *out = m;
  return STOKES_OK;
}

int stokes_mlp_destroy(stokes_mlp *m) {
  if (!m) return STOKES_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  for (float **p : {&m->d_theta, &m->d_grad, &m->d_m, &m->d_v, &m->d_norm, &m->d_x, &m->d_z1, &m->d_h1,
                    &m->d_z2, &m->d_h2, &m->d_y, &m->d_t, &m->d_dy, &m->d_d2, &m->d_d1, &m->d_row,
                    &m->d_loss})
    mfree(*p);
  mfree(m->d_wb);
  if (m->s) cudaStreamDestroy(m->s);
  delete m;
  return STOKES_OK;
}

int stokes_mlp_last_error(const stokes_mlp *m, char *buf, size_t len) {
  if (!m || !buf || len == 0) return STOKES_ERR_ARG;
  snprintf(buf, len, "%s", m->err.c_str());
  return STOKES_OK;
}

int stokes_mlp_num_params(const stokes_mlp *m) { return m ? m->n_params : 0; }

int stokes_mlp_get_dims(const stokes_mlp *m, int *n_in, int *n_hidden, int *n_out) {
  if (!m || !n_in || !n_hidden || !n_out) return STOKES_ERR_ARG;
  *n_in = m->n_in;
  *n_hidden = m->H;
  *n_out = m->n_out;
  return STOKES_OK;
}

int stokes_mlp_set_params(stokes_mlp *m, const float *theta_host) {
  if (!m || !theta_host) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  MK(cudaMemcpy(m->d_theta, theta_host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
  to_bf16_kernel<<<nb(m->n_params, 256), 256, 0, m->s>>>(m->n_params, m->d_theta, m->d_wb);
  MK(cudaMemsetAsync(m->d_m, 0, sizeof(float) * m->n_params, m->s));
  MK(cudaMemsetAsync(m->d_v, 0, sizeof(float) * m->n_params, m->s));
  m->t_adam = 0;
  MK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_mlp_get_adam(stokes_mlp *m, float *m_host, float *v_host, int *t) {
  if (!m || !m_host || !v_host || !t) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  MK(cudaStreamSynchronize(m->s));
  MK(cudaMemcpy(m_host, m->d_m, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
  MK(cudaMemcpy(v_host, m->d_v, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
  *t = m->t_adam;
  return STOKES_OK;
}

int stokes_mlp_set_adam(stokes_mlp *m, const float *m_host, const float *v_host, int t) {
  if (!m || !m_host || !v_host || t < 0) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  MK(cudaStreamSynchronize(m->s));
  MK(cudaMemcpy(m->d_m, m_host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
  MK(cudaMemcpy(m->d_v, v_host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
  m->t_adam = t;
  return STOKES_OK;
}

int stokes_mlp_get_params(stokes_mlp *m, float *theta_host) {
  if (!m || !theta_host) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  MK(cudaStreamSynchronize(m->s));
  MK(cudaMemcpy(theta_host, m->d_theta, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
  return STOKES_OK;
}

int stokes_mlp_set_normalization(stokes_mlp *m, const float *norm_host) {
  if (!m || !norm_host) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  MK(cudaMemcpy(m->d_norm, norm_host, sizeof(float) * 2 * (m->n_in + m->n_out), cudaMemcpyHostToDevice));
  return STOKES_OK;
}

int stokes_mlp_get_normalization(stokes_mlp *m, float *norm_host) {
  if (!m || !norm_host) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  MK(cudaStreamSynchronize(m->s));
  MK(cudaMemcpy(norm_host, m->d_norm, sizeof(float) * 2 * (m->n_in + m->n_out), cudaMemcpyDeviceToHost));
  return STOKES_OK;
}

int stokes_mlp_fit_normalization(stokes_mlp *m, int rows, const float *X, const float *T) {
  if (!m || rows < 1 || !X || !T) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  float *mu_in = m->d_norm, *sd_in = m->d_norm + m->n_in;
  float *mu_out = m->d_norm + 2 * m->n_in, *sd_out = mu_out + m->n_out;
  moments_kernel<<<nb(m->n_in, 64), 64, 0, m->s>>>(rows, m->n_in, X, mu_in, sd_in);
  moments_kernel<<<nb(m->n_out, 64), 64, 0, m->s>>>(rows, m->n_out, T, mu_out, sd_out);
  MK(cudaGetLastError());
  MK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_mlp_forward(stokes_mlp *m, int batch, const float *X, float *Y) {
  if (!m || batch < 0 || (batch && (!X || !Y))) return STOKES_ERR_ARG;
  if (batch == 0) return STOKES_OK;
  MK(cudaSetDevice(m->device));
  int st = stokes::mlp_infer(m, batch, X, Y, m->s);
  if (st) return st;
  MK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_mlp_loss_grad(stokes_mlp *m, int rows, const float *X, const float *T, const int *idx,
                         int batch, float *grad, float *loss) {
  if (!m || batch < 1 || !X || !T) return STOKES_ERR_ARG;
  MK(cudaSetDevice(m->device));
  int st = ensure_batch(m, batch);
  if (st) return st;
  (void)rows;
  const float *mu_in = m->d_norm, *sd_in = m->d_norm + m->n_in;
  const float *mu_out = m->d_norm + 2 * m->n_in, *sd_out = mu_out + m->n_out;
  gather_std_kernel<<<nb(long(batch) * m->n_in, 256), 256, 0, m->s>>>(batch, m->n_in, X, idx, mu_in, sd_in, m->d_x);
  gather_std_kernel<<<nb(long(batch) * m->n_out, 256), 256, 0, m->s>>>(batch, m->n_out, T, idx, mu_out, sd_out, m->d_t);
  forward(m, batch);
  backward(m, batch);
  MK(cudaGetLastError());
  if (grad) MK(cudaMemcpyAsync(grad, m->d_grad, sizeof(float) * m->n_params, cudaMemcpyDefault, m->s));
  if (loss) MK(cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDefault, m->s));
  MK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_mlp_train_step(stokes_mlp *m, int rows, const float *X, const float *T, const int *idx,
                          int batch, float lr, float *loss) {
  if (!m || batch < 1 || !X || !T || !(lr > 0.f)) return STOKES_ERR_ARG;
  int st = stokes_mlp_loss_grad(m, rows, X, T, idx, batch, nullptr, nullptr);
  if (st) return st;
  m->t_adam += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, float(m->t_adam)), c2 = 1.f - powf(b2, float(m->t_adam));
  adam_kernel<<<nb(m->n_params, 256), 256, 0, m->s>>>(m->n_params, m->d_theta, m->d_grad, m->d_m,
                                                      m->d_v, lr, b1, b2, 1e-8f, c1, c2);
  to_bf16_kernel<<<nb(m->n_params, 256), 256, 0, m->s>>>(m->n_params, m->d_theta, m->d_wb);
  MK(cudaGetLastError());
  if (loss) MK(cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDefault, m->s));
  MK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

}  // extern "C"
