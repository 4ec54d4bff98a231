// Learned warm start for dynamic relaxation: proper orthogonal decomposition
// (POD) of relaxed fields and a small multilayer perceptron (MLP), trained and
// evaluated with the kernels of this file.  (The paper lists learning methods
// only as future work, Sec. 8; nothing here is from the paper.)
//
//   gemm_kernel<ACC>   C = alpha op(A) op(B) + beta C, 64 x 64 tiles, 4 x 4 per
//                      thread, FP32 products; ACC = double adds each 16-wide
//                      K-slab into an FP64 accumulator (POD products over
//                      ~1e5-1e6 long columns)
//   bias_act_kernel    Z + b, then tanh (hidden layers) or identity (output)
//   mse_grad_kernel    weighted squared error and dL/dY
//   act_bwd_kernel     dZ = dA (1 - A^2)
//   colsum_kernel      bias gradients (fixed-order column sums)
//   adam_kernel        Adam update with bias correction
//
// The dense products here take milliseconds (batch <= 1024, widths <= 256):
// SIMT FP32 by default; the MLP's BF16 variant runs its products on the
// tensor cores (gemm_tc.cu).
#include <cuda_bf16.h>
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
                                                   long long ldc, const float* __restrict__ subA, int bf16) {
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
      const float v = (i < M && k < K) ? A[i * sar + k * sac] - (subA ? subA[k] : 0.f) : 0.f;
      As[kk][ii] = bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
    }
    for (int q = threadIdx.x; q < TN * TK; q += 256) {
      const int jj = q % TN, kk = q / TN;
      const int j = j0 + jj, k = k0 + kk;
      const float v = (j < N && k < K) ? B[k * sbr + j * sbc] : 0.f;
      Bs[kk][jj] = bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
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
                 const float* subA = nullptr, int bf16 = 0) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_kernel<ACC><<<grid, 256, 0, s>>>(M, N, K, alpha, A, sar, sac, B, sbr, sbc, beta, C, ldc, subA, bf16);
  return cudaGetLastError();
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// the MLP's products: FP32 on CUDA cores (precision 0), BF16 operands on the
// tensor cores (1, gemm_tc.cu), BF16-rounded operands on CUDA cores (2)
cudaError_t mlp_gemm(int precision, int M, int N, int K, const float* A, long long sar, long long sac,
                     const float* B, long long sbr, long long sbc, float* C, long long ldc, cudaStream_t s) {
  if (precision == 1) return gemm_bf16_tc(M, N, K, 1.f, A, sar, sac, B, sbr, sbc, 0.f, C, ldc, s);
  return gemm<float>(M, N, K, 1.f, A, sar, sac, B, sbr, sbc, 0.f, C, ldc, s, nullptr, precision == 2 ? 1 : 0);
}

// Symmetric eigen-decomposition (FP64, host) by the cyclic Jacobi method: sweeps
// over the pairs (p, q), p < q, row by row; each pair is annihilated by the plane
// rotation J = [[c, s], [-s, c]] in the (p, q) plane with t = s / c the root of
// t^2 + 2 theta t - 1 = 0 of smaller magnitude, theta = (a_qq - a_pp) / (2 a_pq)
// (A <- J^T A J, V <- V J).  Sweeps stop when the off-diagonal Frobenius norm is
// below 1e-15 of the whole matrix's (at most 60 sweeps).  Used for small
// matrices only (the POD's Rayleigh-Ritz and orthonormalisation steps, sizes
// of a few hundred).  A (row-major n x n) is overwritten; w gets the
// eigenvalues in descending order, V (row-major n x n) the eigenvectors as
// columns in the same order.
void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& V) {
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  std::vector<double> Vw((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Vw[(size_t)i * n + i] = 1.0;
  double total = 0.0;
  for (size_t q = 0; q < A.size(); ++q) total += A[q] * A[q];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += 2.0 * a(i, j) * a(i, j);
    if (!(off > 1e-30 * total)) break;
    for (int p = 0; p + 1 < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (apq == 0.0) continue;
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(1.0 + theta * theta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q of A J
          const double kp = a(k, p), kq = a(k, q);
          a(k, p) = c * kp - sn * kq;
          a(k, q) = sn * kp + c * kq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q of J^T (A J)
          const double pk = a(p, k), qk = a(q, k);
          a(p, k) = c * pk - sn * qk;
          a(q, k) = sn * pk + c * qk;
        }
        a(p, q) = a(q, p) = 0.0;
        for (int k = 0; k < n; ++k) {
          double* vr = &Vw[(size_t)k * n];
          const double kp = vr[p], kq = vr[q];
          vr[p] = c * kp - sn * kq;
          vr[q] = sn * kp + c * kq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return a(x, x) > a(y, y); });
  w.resize(n);
  V.assign((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    w[c] = a(order[c], order[c]);
    for (int k = 0; k < n; ++k) V[(size_t)k * n + c] = Vw[(size_t)k * n + order[c]];
  }
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
  int bf16 = 0;     // products: 0 FP32, 1 BF16 tensor cores, 2 BF16-rounded operands on CUDA cores
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
    MCK(mlp_gemm(m->bf16, batch, out, in, m->act[l], in, 1, W, 1, in, m->act[l + 1], out, s));
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
    MCK(mlp_gemm(m->bf16, out, in, batch, dcur, 1, out, m->act[l], in, 1, gW, in, s));
    colsum_kernel<<<blocks(out, 128), 128, 0, s>>>(dcur, batch, out, gb);
    MCK(cudaGetLastError());
    if (l > 0) {
      // dA_l = dZ W : (batch x out)(out x in), then through tanh
      MCK(mlp_gemm(m->bf16, batch, in, out, dcur, out, 1, m->d_p + m->w_off[l], in, 1, dnext, in, s));
      const long long n = (long long)batch * in;
      act_bwd_kernel<<<blocks(n, 256), 256, 0, s>>>(dnext, m->act[l], n);
      MCK(cudaGetLastError());
      std::swap(dcur, dnext);
    }
  }
  if (loss_out) {
    MCK(cudaMemcpyAsync(loss_out, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    if (m->bf16 == 1 && gemm_tc_timed_out()) return mfail(m, DJ_ERR_CUDA, "a tensor-core wait timed out");
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

dj_status dj_mlp_set_precision(dj_mlp* m, int precision) {
  if (!m || precision < 0 || precision > 2) return DJ_ERR_INVALID_ARG;
  m->bf16 = precision;
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

}  // extern "C"

namespace {

// standard normal numbers from a counter (splitmix64 of seed + index, two
// uniforms, Box-Muller); the same on every host
double normal_at(unsigned long long seed, unsigned long long i) {
  auto mix = [](unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const double u1 = ((mix(seed + 2 * i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((mix(seed + 2 * i + 1) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// Device scratch of one POD fit, freed on every exit path.
struct PodWork {
  std::vector<float*> bufs;
  float* get(size_t n) {
    float* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(float)) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  }
  ~PodWork() {
    for (float* p : bufs) cudaFree(p);
  }
};

// Orthonormalise the k columns of Z (n x k, row-major, leading dimension ld) in
// place by the eigen-decomposition of its Gram matrix G = Z^T Z = V L V^T:
// Z <- Z V_k L_k^-1/2 over the eigenvalues above 1e-10 of the largest (columns
// that FP32 rounding cannot tell apart from a combination of the others are
// dropped).  k is updated to the number of columns kept.  tmp: n x ld floats.
cudaError_t orthonormalise(float* Z, long long n, int ld, int& k, float* tmp, float* d_small, cudaStream_t s) {
  cudaError_t e = gemm<double>(k, k, (int)std::min<long long>(n, 0x7fffffff), 1.f, Z, 1, ld, Z, ld, 1, 0.f,
                               d_small, k, s);
  std::vector<float> hG((size_t)k * k);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hG.data(), d_small, hG.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  std::vector<double> G((size_t)k * k), w, V;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) G[(size_t)i * k + j] = 0.5 * ((double)hG[(size_t)i * k + j] + hG[(size_t)j * k + i]);
  jacobi_eigen(G, k, w, V);
  int kept = 0;
  while (kept < k && w[kept] > 1e-10 * w[0] && w[kept] > 0.0) ++kept;
  std::vector<float> T((size_t)k * ld, 0.f);  // k x kept, leading dimension ld
  for (int i = 0; i < k; ++i)
    for (int c = 0; c < kept; ++c) T[(size_t)i * ld + c] = (float)(V[(size_t)i * k + c] / std::sqrt(w[c]));
  e = cudaMemcpyAsync(d_small, T.data(), T.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && kept > 0)
    e = gemm<double>((int)n, kept, k, 1.f, Z, ld, 1, d_small, ld, 1, 0.f, tmp, ld, s);
  if (e == cudaSuccess && kept > 0)
    e = cudaMemcpyAsync(Z, tmp, (size_t)n * ld * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // T is host memory of this frame
  k = kept;
  return e;
}

}  // namespace

extern "C" {

// POD by a randomised range finder with subspace iteration and a Rayleigh-Ritz
// step (no Gram matrix of the snapshots is formed):
//   Yc = Y - mean 1^T (rows x cols), Omega (cols x l) seeded normal, l = r + p
//   Z = orth(Yc Omega); q times: W = orth(Yc^T Z), Z = orth(Yc W)
//   B^T = Yc^T Z, B B^T = U S^2 U^T (l x l, Jacobi on the host)
//   modes = Z U_r, sigma = S_r
// With l >= cols the range of Z is that of Yc and the result is the exact
// truncated SVD; otherwise q = 3 power steps (subspace iteration) with
// oversampling p = max(32, r / 2) resolve the leading r modes.
dj_status dj_pod_fit(const float* d_Y, long long rows, int cols, int r, float* d_mean, float* d_modes,
                     double* sigma_out, void* stream) {
  if (!d_Y || !d_mean || !d_modes || rows <= 0 || cols <= 0 || r <= 0 || r > cols || cols > 65536 || r > 1024)
    return DJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int p_over = std::max(32, r / 2);
  const int l = std::min(cols, r + p_over);
  const int q_steps = l >= cols ? 0 : 3;
  const int Kr = (int)std::min<long long>(rows, 0x7fffffff);
  PodWork wk;
  float* Yc = wk.get((size_t)rows * cols);
  float* Z = wk.get((size_t)rows * l);
  float* Zt = wk.get((size_t)rows * l);
  float* W = wk.get((size_t)cols * l);
  float* Wt = wk.get((size_t)cols * l);
  float* sm = wk.get((size_t)l * l);
  if (!Yc || !Z || !Zt || !W || !Wt || !sm) return DJ_ERR_OOM;
  rowmean_kernel<<<blocks(rows, 256), 256, 0, s>>>(d_Y, rows, cols, d_mean);
  center_kernel<<<blocks(rows * (long long)cols, 256), 256, 0, s>>>(d_Y, d_mean, rows, cols, Yc);
  cudaError_t e = cudaGetLastError();
  // Omega: cols x l, row-major (staged through W)
  {
    std::vector<float> om((size_t)cols * l);
    for (size_t i = 0; i < om.size(); ++i) om[i] = (float)normal_at(0x5EEDull + (unsigned long long)cols, i);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W, om.data(), om.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  // Yc(i, c) = Yc[i + c rows]: as A(i, k) with sar = 1, sac = rows; as A^T with sar = rows, sac = 1
  int k = l;
  if (e == cudaSuccess) e = gemm<double>((int)rows, k, cols, 1.f, Yc, 1, rows, W, l, 1, 0.f, Z, l, s);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) e = orthonormalise(Z, rows, l, k, Zt, sm, s);
  for (int it = 0; it < q_steps && e == cudaSuccess && k > 0; ++it) {
    e = gemm<double>(cols, k, Kr, 1.f, Yc, rows, 1, Z, l, 1, 0.f, W, l, s);
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) e = orthonormalise(W, cols, l, k, Wt, sm, s);
    if (e == cudaSuccess && k > 0) e = gemm<double>((int)rows, k, cols, 1.f, Yc, 1, rows, W, l, 1, 0.f, Z, l, s);
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) e = orthonormalise(Z, rows, l, k, Zt, sm, s);
  }
  // Rayleigh-Ritz: B^T = Yc^T Z (cols x k), C = B B^T (k x k)
  std::vector<double> wv, U;
  if (e == cudaSuccess && k > 0) e = gemm<double>(cols, k, Kr, 1.f, Yc, rows, 1, Z, l, 1, 0.f, W, l, s);
  if (e == cudaSuccess && k > 0) e = gemm<double>(k, k, cols, 1.f, W, 1, l, W, l, 1, 0.f, sm, k, s);
  if (e == cudaSuccess && k > 0) {
    std::vector<float> hC((size_t)k * k);
    e = cudaMemcpyAsync(hC.data(), sm, hC.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::vector<double> C((size_t)k * k);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) C[(size_t)i * k + j] = 0.5 * ((double)hC[(size_t)i * k + j] + hC[(size_t)j * k + i]);
    if (e == cudaSuccess) jacobi_eigen(C, k, wv, U);
  }
  if (e != cudaSuccess) return DJ_ERR_CUDA;
  // modes = Z U_r (rows x r, row-major); columns beyond the rank found are zero
  std::vector<float> hU((size_t)std::max(k, 1) * r, 0.f);
  for (int c = 0; c < r; ++c) {
    const double lam = c < k ? wv[c] : 0.0;
    if (sigma_out) sigma_out[c] = lam > 0 ? std::sqrt(lam) : 0.0;
    if (c < k && lam > 0)
      for (int i = 0; i < k; ++i) hU[(size_t)i * r + c] = (float)U[(size_t)i * k + c];
  }
  if (k > 0) {
    e = cudaMemcpyAsync(sm, hU.data(), (size_t)k * r * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = gemm<double>((int)rows, r, k, 1.f, Z, l, 1, sm, r, 1, 0.f, d_modes, r, s);
  } else {
    e = cudaMemsetAsync(d_modes, 0, (size_t)rows * r * sizeof(float), s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

// Host-only symmetric eigen-decomposition (the cyclic Jacobi method the POD uses).
dj_status dj_symmetric_eigen(const double* A, int n, double* w, double* V) {
  if (!A || !w || n <= 0 || n > 4096) return DJ_ERR_INVALID_ARG;
  std::vector<double> a(A, A + (size_t)n * n), wv, Vv;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double m = 0.5 * (a[(size_t)i * n + j] + a[(size_t)j * n + i]);
      if (!std::isfinite(m)) return DJ_ERR_INVALID_ARG;
      a[(size_t)i * n + j] = a[(size_t)j * n + i] = m;
    }
  jacobi_eigen(a, n, wv, Vv);
  std::copy(wv.begin(), wv.end(), w);
  if (V) std::copy(Vv.begin(), Vv.end(), V);
  return DJ_OK;
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
