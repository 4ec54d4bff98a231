// Learned warm start for dynamic relaxation: proper orthogonal decomposition
// (POD) of relaxed fields and a small multilayer perceptron (MLP), trained and
// evaluated with the kernels of this file.  (The paper lists learning methods
// only as future work, Sec. 8; nothing here is from the paper.)
//
//   gemm_kernel<ACC>   C = alpha op(A) op(B) + beta C, 64 x 64 tiles, 4 x 4 per
//                      thread, FP32 products; ACC = double adds each 16-wide
//                      K-slab into an FP64 accumulator (POD Gram matrices over
//                      ~1e5-1e6 long columns)
//   bias_act_kernel    Z + b, then tanh (hidden layers) or identity (output)
//   mse_grad_kernel    weighted squared error and dL/dY
//   act_bwd_kernel     dZ = dA (1 - A^2)
//   colsum_kernel      bias gradients (fixed-order column sums)
//   adam_kernel        Adam update with bias correction
//
// The dense products here take milliseconds (batch <= 1024, widths <= 256);
// they are SIMT FP32, not tensor-core kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "dj_internal.h"

namespace dj {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

// C[i, j] = alpha sum_k A(i, k) B(k, j) + beta C[i, j], with A(i, k) = A[i * sar + k * sac]
// and B(k, j) = B[k * sbr + j * sbc]; C row-major with leading dimension ldc.
// subA (optional): A(i, k) - subA[k], which centres snapshots inside the product
template <typename ACC>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                   long long sar, long long sac, const float* __restrict__ B,
                                                   long long sbr, long long sbc, float beta, float* __restrict__ C,
                                                   long long ldc, const float* __restrict__ subA) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  ACC acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int q = threadIdx.x; q < TM * TK; q += 256) {
      const int ii = q / TK, kk = q % TK;
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < M && k < K) ? A[i * sar + k * sac] - (subA ? subA[k] : 0.f) : 0.f;
    }
    for (int q = threadIdx.x; q < TN * TK; q += 256) {
      const int jj = q % TN, kk = q / TN;
      const int j = j0 + jj, k = k0 + kk;
      Bs[kk][jj] = (j < N && k < K) ? B[k * sbr + j * sbc] : 0.f;
    }
    __syncthreads();
    float part[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) part[a][b] = 0.f;
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) part[a][b] = fmaf(av[a], bv[b], part[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += (ACC)part[a][b];
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < M && j < N) {
        float* c = C + i * ldc + j;
        const float v = alpha * (float)acc[a][b];
        *c = beta == 0.f ? v : v + beta * *c;
      }
    }
}

__global__ void bias_act_kernel(float* Z, const float* __restrict__ b, int rows, int cols, int tanh_act) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)rows * cols) return;
  const float v = Z[q] + b[q % cols];
  Z[q] = tanh_act ? tanhf(v) : v;
}

// per row partial of sum_j w_j (Y - T)^2 and dY = 2 w_j (Y - T) / (rows cols)
__global__ void mse_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                const float* __restrict__ w, int rows, int cols, float* dY,
                                double* row_loss) {
  const int r = blockIdx.x;
  __shared__ double s[256];
  double acc = 0.0;
  const float scale = 2.f / ((float)rows * (float)cols);
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    const long long q = (long long)r * cols + j;
    const float d = Y[q] - T[q];
    const float wj = w ? w[j] : 1.f;
    acc += (double)wj * d * d;
    dY[q] = scale * wj * d;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) row_loss[r] = s[0];
}

__global__ void sum_kernel(const double* __restrict__ v, int n, double scale, double* out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) acc += v[q];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0] * scale;
}

__global__ void act_bwd_kernel(float* dZ, const float* __restrict__ A, long long n) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) dZ[q] *= 1.f - A[q] * A[q];
}

__global__ void colsum_kernel(const float* __restrict__ D, int rows, int cols, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float acc = 0.f;
  for (int r = 0; r < rows; ++r) acc += D[(long long)r * cols + j];
  out[j] = acc;
}

__global__ void adam_kernel(float* p, const float* __restrict__ g, float* m, float* v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.f - b1) * gq;
  const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

// row means of a column-major snapshot block: Y[r + c * rows]
// F[s] = [x_0 .. x_{n-1}, x_i x_j for 0 <= i <= j < n] of row s of X (leading dim ld)
__global__ void quad_features_kernel(const float* __restrict__ X, int S, int ld, int n, float* __restrict__ F) {
  const int s = blockIdx.x;
  const int nf = n + n * (n + 1) / 2;
  const float* x = X + (size_t)s * ld;
  float* f = F + (size_t)s * nf;
  for (int q = threadIdx.x; q < nf; q += blockDim.x) {
    if (q < n) {
      f[q] = x[q];
    } else {
      // q - n enumerates (i, j), i <= j, row by row
      int r = q - n, i = 0;
      while (r >= n - i) {
        r -= n - i;
        ++i;
      }
      f[q] = x[i] * x[i + r];
    }
  }
}

__global__ void rowmean_kernel(const float* __restrict__ Y, long long rows, int cols, float* mean) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double acc = 0.0;
  for (int c = 0; c < cols; ++c) acc += Y[r + (long long)c * rows];
  mean[r] = (float)(acc / cols);
}

__global__ void center_kernel(const float* __restrict__ Y, const float* __restrict__ mean, long long rows,
                              int cols, float* Yc) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= rows * (long long)cols) return;
  Yc[q] = Y[q] - mean[q % rows];
}

__global__ void add_mean_kernel(float* X, const float* __restrict__ mean, long long rows, int cols) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= rows * (long long)cols) return;
  X[q] += mean[q % rows];
}

template <typename ACC>
cudaError_t gemm(int M, int N, int K, float alpha, const float* A, long long sar, long long sac, const float* B,
                 long long sbr, long long sbc, float beta, float* C, long long ldc, cudaStream_t s,
                 const float* subA = nullptr) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_kernel<ACC><<<grid, 256, 0, s>>>(M, N, K, alpha, A, sar, sac, B, sbr, sbc, beta, C, ldc, subA);
  return cudaGetLastError();
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Symmetric eigen-decomposition (FP64, host): Householder reduction to
// tridiagonal form T = Q^T A Q, then the QL iteration with implicit Wilkinson
// shifts on T, accumulating the plane rotations into Q.  On return w holds the
// eigenvalues and V (row-major n x n) the eigenvectors as columns.
void symmetric_eigen(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& V) {
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), wv(n);
  for (int k = 0; k + 2 < n; ++k) {
    // Householder vector of column k below the diagonal
    double nx = 0.0;
    for (int i = k + 1; i < n; ++i) nx += a(i, k) * a(i, k);
    nx = std::sqrt(nx);
    if (nx == 0.0) continue;
    const double alpha = a(k + 1, k) > 0 ? -nx : nx;
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int i = k + 1; i < n; ++i) v[i] = a(i, k);
    v[k + 1] -= alpha;
    double nv = 0.0;
    for (int i = k + 1; i < n; ++i) nv += v[i] * v[i];
    nv = std::sqrt(nv);
    if (nv == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= nv;
    // A <- H A H with H = I - 2 v v^T:  p = 2 A v, K = v^T p, w = p - K v, A -= v w^T + w v^T
    for (int i = k; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += a(i, j) * v[j];
      p[i] = 2.0 * s;
    }
    double K = 0.0;
    for (int i = k + 1; i < n; ++i) K += v[i] * p[i];
    for (int i = k; i < n; ++i) wv[i] = p[i] - K * v[i];
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j) a(i, j) -= v[i] * wv[j] + wv[i] * v[j];
    // Q <- Q H
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += V[(size_t)i * n + j] * v[j];
      for (int j = k + 1; j < n; ++j) V[(size_t)i * n + j] -= 2.0 * s * v[j];
    }
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
  // QL with implicit shifts: deflate from the top, e[i] couples d[i] and d[i+1]
  for (int l = 0; l < n; ++l) {
    for (int iter = 0; iter < 60; ++iter) {
      int m = l;
      for (; m + 1 < n; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-15 * dd) break;
      }
      if (m == l) break;
      // Wilkinson shift from the leading 2 x 2 block
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = m - 1;
      for (; i >= l; --i) {
        double f = s * e[i];
        const double b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= pp;
          e[m] = 0.0;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        for (int k = 0; k < n; ++k) {  // rotate eigenvector columns i, i+1
          f = V[(size_t)k * n + i + 1];
          V[(size_t)k * n + i + 1] = s * V[(size_t)k * n + i] + c * f;
          V[(size_t)k * n + i] = c * V[(size_t)k * n + i] - s * f;
        }
      }
      if (r == 0.0 && i >= l) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  w = d;
}

}  // namespace
}  // namespace dj

using namespace dj;

struct dj_mlp {
  std::vector<int> widths;
  int L = 0;
  long long n_params = 0;
  std::vector<long long> w_off, b_off;  // offsets of W_l (out x in, row-major) and b_l
  float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
  std::vector<float*> act;  // activations per layer (batch_cap x width)
  float* d_dA = nullptr;
  float* d_dB = nullptr;
  double* d_rowloss = nullptr;
  double* d_loss = nullptr;
  int batch_cap = 0;
  long long t = 0;  // Adam step
  std::string last_error;
};

namespace {
dj_status mfail(dj_mlp* m, dj_status s, const std::string& msg) {
  if (m) m->last_error = msg;
  return s;
}
#define MCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess)                                                              \
      return mfail(m, _e == cudaErrorMemoryAllocation ? DJ_ERR_OOM : DJ_ERR_CUDA,       \
                   std::string(#call) + ": " + cudaGetErrorString(_e));                 \
  } while (0)

dj_status ensure_batch(dj_mlp* m, int batch) {
  if (batch <= m->batch_cap) return DJ_OK;
  for (float* a : m->act)
    if (a) cudaFree(a);
  if (m->d_dA) cudaFree(m->d_dA);
  if (m->d_dB) cudaFree(m->d_dB);
  if (m->d_rowloss) cudaFree(m->d_rowloss);
  m->act.assign(m->L + 1, nullptr);
  int wmax = 0;
  for (int w : m->widths) wmax = std::max(wmax, w);
  for (int l = 0; l <= m->L; ++l) MCK(cudaMalloc(&m->act[l], (size_t)batch * m->widths[l] * sizeof(float)));
  MCK(cudaMalloc(&m->d_dA, (size_t)batch * wmax * sizeof(float)));
  MCK(cudaMalloc(&m->d_dB, (size_t)batch * wmax * sizeof(float)));
  MCK(cudaMalloc(&m->d_rowloss, (size_t)batch * sizeof(double)));
  m->batch_cap = batch;
  return DJ_OK;
}

// forward pass into m->act (act[0] = input copy)
dj_status mlp_forward(dj_mlp* m, const float* X, int batch, cudaStream_t s) {
  dj_status st = ensure_batch(m, batch);
  if (st) return st;
  MCK(cudaMemcpyAsync(m->act[0], X, (size_t)batch * m->widths[0] * sizeof(float), cudaMemcpyDeviceToDevice, s));
  for (int l = 0; l < m->L; ++l) {
    const int in = m->widths[l], out = m->widths[l + 1];
    const float* W = m->d_p + m->w_off[l];
    // Z = A_l W^T : (batch x in)(in x out), W row-major out x in -> B(k, j) = W[j * in + k]
    MCK(gemm<float>(batch, out, in, 1.f, m->act[l], in, 1, W, 1, in, 0.f, m->act[l + 1], out, s));
    const long long n = (long long)batch * out;
    bias_act_kernel<<<blocks(n, 256), 256, 0, s>>>(m->act[l + 1], m->d_p + m->b_off[l], batch, out,
                                                   l + 1 < m->L ? 1 : 0);
    MCK(cudaGetLastError());
  }
  return DJ_OK;
}
}  // namespace

extern "C" {

dj_status dj_mlp_create(const int* widths, int n_layers, unsigned long long seed, dj_mlp** out) {
  if (!out || !widths || n_layers < 1 || n_layers > 16) return DJ_ERR_INVALID_ARG;
  *out = nullptr;
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] <= 0 || widths[l] > 8192) return DJ_ERR_INVALID_ARG;
  dj_mlp* m = new (std::nothrow) dj_mlp();
  if (!m) return DJ_ERR_OOM;
  m->widths.assign(widths, widths + n_layers + 1);
  m->L = n_layers;
  long long off = 0;
  for (int l = 0; l < n_layers; ++l) {
    m->w_off.push_back(off);
    off += (long long)widths[l] * widths[l + 1];
    m->b_off.push_back(off);
    off += widths[l + 1];
  }
  m->n_params = off;
  // Glorot-uniform weights, zero biases, from a seeded host generator
  std::vector<float> h(off, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < n_layers; ++l) {
    const double lim = std::sqrt(6.0 / (widths[l] + widths[l + 1]));
    std::uniform_real_distribution<double> U(-lim, lim);
    for (long long q = 0; q < (long long)widths[l] * widths[l + 1]; ++q) h[m->w_off[l] + q] = (float)U(rng);
  }
  cudaError_t e = cudaMalloc(&m->d_p, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_g, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_m, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_v, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(m->d_p, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->d_g, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, off * sizeof(float));
  if (e != cudaSuccess) {
    delete m;
    return e == cudaErrorMemoryAllocation ? DJ_ERR_OOM : DJ_ERR_CUDA;
  }
  *out = m;
  return DJ_OK;
}

long long dj_mlp_num_params(const dj_mlp* m) { return m ? m->n_params : 0; }

dj_status dj_mlp_get_params(dj_mlp* m, float* host, long long n) {
  if (!m || !host || n != m->n_params) return DJ_ERR_INVALID_ARG;
  MCK(cudaMemcpy(host, m->d_p, n * sizeof(float), cudaMemcpyDeviceToHost));
  return DJ_OK;
}

dj_status dj_mlp_set_params(dj_mlp* m, const float* host, long long n) {
  if (!m || !host || n != m->n_params) return DJ_ERR_INVALID_ARG;
  MCK(cudaMemcpy(m->d_p, host, n * sizeof(float), cudaMemcpyHostToDevice));
  MCK(cudaMemset(m->d_m, 0, n * sizeof(float)));
  MCK(cudaMemset(m->d_v, 0, n * sizeof(float)));
  m->t = 0;
  return DJ_OK;
}

dj_status dj_mlp_get_grads(dj_mlp* m, float* host, long long n) {
  if (!m || !host || n != m->n_params) return DJ_ERR_INVALID_ARG;
  MCK(cudaMemcpy(host, m->d_g, n * sizeof(float), cudaMemcpyDeviceToHost));
  return DJ_OK;
}

dj_status dj_mlp_forward(dj_mlp* m, const float* d_X, int batch, float* d_Y, void* stream) {
  if (!m || !d_X || !d_Y || batch <= 0) return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  dj_status st = mlp_forward(m, d_X, batch, s);
  if (st) return st;
  MCK(cudaMemcpyAsync(d_Y, m->act[m->L], (size_t)batch * m->widths[m->L] * sizeof(float),
                      cudaMemcpyDeviceToDevice, s));
  return DJ_OK;
}

dj_status dj_mlp_loss_grad(dj_mlp* m, const float* d_X, const float* d_T, const float* d_w, int batch,
                           double* loss_out, void* stream) {
  if (!m || !d_X || !d_T || batch <= 0) return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  dj_status st = mlp_forward(m, d_X, batch, s);
  if (st) return st;
  const int outw = m->widths[m->L];
  mse_grad_kernel<<<batch, 256, 0, s>>>(m->act[m->L], d_T, d_w, batch, outw, m->d_dA, m->d_rowloss);
  MCK(cudaGetLastError());
  sum_kernel<<<1, 256, 0, s>>>(m->d_rowloss, batch, 1.0 / ((double)batch * outw), m->d_loss);
  MCK(cudaGetLastError());
  // backward: dA holds dL/dZ of the current layer (output layer is linear)
  float* dcur = m->d_dA;
  float* dnext = m->d_dB;
  for (int l = m->L - 1; l >= 0; --l) {
    const int in = m->widths[l], out = m->widths[l + 1];
    float* gW = m->d_g + m->w_off[l];
    float* gb = m->d_g + m->b_off[l];
    // dW = dZ^T A_l : (out x batch)(batch x in)
    MCK(gemm<float>(out, in, batch, 1.f, dcur, 1, out, m->act[l], in, 1, 0.f, gW, in, s));
    colsum_kernel<<<blocks(out, 128), 128, 0, s>>>(dcur, batch, out, gb);
    MCK(cudaGetLastError());
    if (l > 0) {
      // dA_l = dZ W : (batch x out)(out x in), then through tanh
      MCK(gemm<float>(batch, in, out, 1.f, dcur, out, 1, m->d_p + m->w_off[l], in, 1, 0.f, dnext, in, s));
      const long long n = (long long)batch * in;
      act_bwd_kernel<<<blocks(n, 256), 256, 0, s>>>(dnext, m->act[l], n);
      MCK(cudaGetLastError());
      std::swap(dcur, dnext);
    }
  }
  if (loss_out) {
    MCK(cudaMemcpyAsync(loss_out, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
  }
  return DJ_OK;
}

dj_status dj_mlp_adam_step(dj_mlp* m, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!m || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  m->t += 1;
  const float c1 = 1.f - (float)std::pow((double)beta1, (double)m->t);
  const float c2 = 1.f - (float)std::pow((double)beta2, (double)m->t);
  adam_kernel<<<blocks(m->n_params, 256), 256, 0, s>>>(m->d_p, m->d_g, m->d_m, m->d_v, m->n_params, lr, beta1,
                                                        beta2, eps, c1, c2);
  MCK(cudaGetLastError());
  return DJ_OK;
}

const char* dj_mlp_last_error(const dj_mlp* m) { return m ? m->last_error.c_str() : "null mlp"; }

void dj_mlp_destroy(dj_mlp* m) {
  if (!m) return;
  for (float* a : m->act)
    if (a) cudaFree(a);
  void* ps[] = {m->d_p, m->d_g, m->d_m, m->d_v, m->d_dA, m->d_dB, m->d_rowloss, m->d_loss};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete m;
}

dj_status dj_pod_fit(const float* d_Y, long long rows, int cols, int r, float* d_mean, float* d_modes,
                     double* sigma_out, void* stream) {
  dj_mlp* m = nullptr;  // for MCK
  if (!d_Y || !d_mean || !d_modes || rows <= 0 || cols <= 0 || r <= 0 || r > cols || cols > 4096)
    return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float *Yc = nullptr, *G = nullptr, *Vr = nullptr;
  MCK(cudaMalloc(&Yc, (size_t)rows * cols * sizeof(float)));
  cudaError_t e = cudaMalloc(&G, (size_t)cols * cols * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&Vr, (size_t)cols * r * sizeof(float));
  auto cleanup = [&]() {
    if (Yc) cudaFree(Yc);
    if (G) cudaFree(G);
    if (Vr) cudaFree(Vr);
  };
  if (e == cudaSuccess) {
    rowmean_kernel<<<blocks(rows, 256), 256, 0, s>>>(d_Y, rows, cols, d_mean);
    center_kernel<<<blocks(rows * (long long)cols, 256), 256, 0, s>>>(d_Y, d_mean, rows, cols, Yc);
    e = cudaGetLastError();
  }
  // Gram G = Yc^T Yc (cols x cols), Yc column-major: Yc(k, j) = Yc[k + j * rows]
  if (e == cudaSuccess) e = gemm<double>(cols, cols, (int)std::min<long long>(rows, 0x7fffffff), 1.f, Yc, rows, 1,
                                         Yc, 1, rows, 0.f, G, cols, s);
  std::vector<float> hG((size_t)cols * cols);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hG.data(), G, hG.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup();
    return DJ_ERR_CUDA;
  }
  std::vector<double> a(hG.begin(), hG.end()), w, V;
  for (int i = 0; i < cols; ++i)
    for (int j = 0; j < i; ++j) a[(size_t)i * cols + j] = a[(size_t)j * cols + i] = 0.5 * (a[(size_t)i * cols + j] + a[(size_t)j * cols + i]);
  symmetric_eigen(a, cols, w, V);
  std::vector<int> order(cols);
  for (int i = 0; i < cols; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
  // modes = Yc V_r diag(lambda^-1/2): V_r scaled on the host (cols x r, row-major)
  std::vector<float> hV((size_t)cols * r, 0.f);
  for (int q = 0; q < r; ++q) {
    const double lam = w[order[q]];
    const double sc = lam > 1e-30 ? 1.0 / std::sqrt(lam) : 0.0;
    if (sigma_out) sigma_out[q] = lam > 0 ? std::sqrt(lam) : 0.0;
    for (int k = 0; k < cols; ++k) hV[(size_t)k * r + q] = (float)(V[(size_t)k * cols + order[q]] * sc);
  }
  e = cudaMemcpyAsync(Vr, hV.data(), hV.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  // d_modes row-major rows x r
  if (e == cudaSuccess) e = gemm<float>((int)rows, r, cols, 1.f, Yc, 1, rows, Vr, r, 1, 0.f, d_modes, r, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  return e == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

dj_status dj_pod_project(const float* d_modes, const float* d_mean, long long rows, int r, const float* d_X,
                         int cols, float* d_Q, void* stream) {
  // Q (cols x r, row-major) = (X - mean)^T modes, X column-major rows x cols; the
  // centring happens inside the product, so no temporary is allocated
  if (!d_modes || !d_X || !d_Q || rows <= 0 || r <= 0 || cols <= 0) return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = gemm<double>(cols, r, (int)rows, 1.f, d_X, rows, 1, d_modes, r, 1, 0.f, d_Q, r, s, d_mean);
  return e == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

dj_status dj_pod_expand(const float* d_modes, const float* d_mean, long long rows, int r, const float* d_Q,
                        int cols, float* d_X, void* stream) {
  // X (column-major rows x cols) = mean + modes Q^T, Q row-major cols x r
  if (!d_modes || !d_Q || !d_X || rows <= 0 || r <= 0 || cols <= 0) return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // X(i, c) = sum_q modes[i * r + q] Q[c * r + q]; stored X[i + c * rows] -> treat as C = X^T (cols x rows)
  cudaError_t e = gemm<float>(cols, (int)rows, r, 1.f, d_Q, r, 1, d_modes, 1, r, 0.f, d_X, rows, s);
  if (e == cudaSuccess && d_mean) {
    add_mean_kernel<<<blocks(rows * (long long)cols, 256), 256, 0, s>>>(d_X, d_mean, rows, cols);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

dj_status dj_linear_fit(const float* d_X, const float* d_Y, int S, int n_in, int n_out, double ridge,
                        float* d_W, void* stream) {
  // W (n_out x n_in) minimises |X W^T - Y|^2 + ridge tr(G) / n_in |W|^2, G = X^T X:
  // the normal equations (G + ridge tr(G) / n_in I) W^T = X^T Y, products on the
  // device (FP64 accumulation over K-slabs), Cholesky solve on the host in FP64
  if (!d_X || !d_Y || !d_W || S <= 0 || n_in <= 0 || n_out <= 0 || n_in > 1024 || !(ridge >= 0.0))
    return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float *G = nullptr, *R = nullptr;
  cudaError_t e = cudaMalloc(&G, (size_t)n_in * n_in * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&R, (size_t)n_in * n_out * sizeof(float));
  // G(i, j) = sum_k X[k n_in + i] X[k n_in + j];  R(i, o) = sum_k X[k n_in + i] Y[k n_out + o]
  if (e == cudaSuccess) e = gemm<double>(n_in, n_in, S, 1.f, d_X, 1, n_in, d_X, n_in, 1, 0.f, G, n_in, s);
  if (e == cudaSuccess) e = gemm<double>(n_in, n_out, S, 1.f, d_X, 1, n_in, d_Y, n_out, 1, 0.f, R, n_out, s);
  std::vector<float> hG((size_t)n_in * n_in), hR((size_t)n_in * n_out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hG.data(), G, hG.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hR.data(), R, hR.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (G) cudaFree(G);
  if (R) cudaFree(R);
  if (e != cudaSuccess) return DJ_ERR_CUDA;
  const int n = n_in;
  std::vector<double> L((size_t)n * n, 0.0);
  double tr = 0.0;
  for (int i = 0; i < n; ++i) tr += hG[(size_t)i * n + i];
  // G is accumulated in FP64 but stored in FP32: if its rounding leaves the
  // regularised normal equations indefinite, the ridge grows tenfold (at most
  // four times) before the fit is refused
  bool ok = false;
  double lam = ridge;
  for (int attempt = 0; attempt < 5 && !ok; ++attempt, lam = lam > 0.0 ? 10.0 * lam : 1e-7) {
    const double shift = lam * tr / n + 1e-300;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= i; ++j)
        L[(size_t)i * n + j] = 0.5 * ((double)hG[(size_t)i * n + j] + hG[(size_t)j * n + i]);
    for (int i = 0; i < n; ++i) L[(size_t)i * n + i] += shift;
    ok = true;
    for (int j = 0; j < n && ok; ++j) {  // Cholesky, lower triangle in place
      double d = L[(size_t)j * n + j];
      for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
      if (!(d > 0.0)) {
        ok = false;
        break;
      }
      d = std::sqrt(d);
      L[(size_t)j * n + j] = d;
      for (int i = j + 1; i < n; ++i) {
        double v = L[(size_t)i * n + j];
        for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
        L[(size_t)i * n + j] = v / d;
      }
    }
  }
  if (!ok) return DJ_ERR_INVALID_ARG;  // normal equations not positive definite
  std::vector<float> hW((size_t)n_out * n);
  std::vector<double> z(n);
  for (int o = 0; o < n_out; ++o) {
    for (int i = 0; i < n; ++i) {  // L z = r
      double v = hR[(size_t)i * n_out + o];
      for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * z[k];
      z[i] = v / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T w = z
      double v = z[i];
      for (int k = i + 1; k < n; ++k) v -= L[(size_t)k * n + i] * z[k];
      z[i] = v / L[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) hW[(size_t)o * n + i] = (float)z[i];
  }
  e = cudaMemcpyAsync(d_W, hW.data(), hW.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

dj_status dj_quad_features(const float* d_X, int S, int ld, int n, float* d_F, void* stream) {
  // row s of d_F (S x (n + n (n + 1) / 2), row-major): the first n entries of row s
  // of d_X (leading dimension ld) and their pairwise products x_i x_j, i <= j
  if (!d_X || !d_F || S <= 0 || n <= 0 || ld < n || n > 256) return DJ_ERR_INVALID_ARG;
  quad_features_kernel<<<S, 128, 0, (cudaStream_t)stream>>>(d_X, S, ld, n, d_F);
  return cudaGetLastError() == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

dj_status dj_linear_apply(const float* d_W, int n_out, int n_in, const float* d_X, int S, float alpha, float beta,
                          float* d_Y, void* stream) {
  // Y (S x n_out) = alpha X W^T + beta Y, X row-major S x n_in, W row-major n_out x n_in
  if (!d_W || !d_X || !d_Y || n_out <= 0 || n_in <= 0 || S <= 0) return DJ_ERR_INVALID_ARG;
  cudaError_t e = gemm<float>(S, n_out, n_in, alpha, d_X, n_in, 1, d_W, 1, n_in, beta, d_Y, n_out,
                              (cudaStream_t)stream);
  return e == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

}  // extern "C"
