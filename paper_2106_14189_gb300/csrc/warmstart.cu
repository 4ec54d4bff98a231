// Learned warm start for dynamic relaxation, inside the library (the paper
// lists learning methods only as future work, Sec. 8; nothing here is from
// the paper).  A dj_ws maps the prescribed values of a load case to an initial
// nodal field for the relaxation of Sec. 6:
//
//   c = Phi_in^T (t - mean_in)          leading POD coefficients of the targets,
//                                       scaled to unit spread over the training loads
//   q = W f(c) [+ MLP(c)]               f: the kept coefficients and (second order)
//                                       their pairwise products; W by ridge least
//                                       squares; the MLP learns what W leaves
//   U0 = mean_out + Phi_out q           the relaxed field's leading POD modes
//
// Training data are the method's own relaxed fields (dj_ws_train relaxes every
// load case from rest on the caller's mesh); a seeded share of the loads is
// held out to choose between the first- and second-order polynomial parts and
// to decide whether the MLP is kept.  dj_ws_relax_to_tol checks the predicted
// field before using it (inverted elements, residual against the field with the
// prescribed values alone) and otherwise relaxes from rest, so the answer is
// always a relaxation of the method to the same tolerance.
//
// Everything numerical runs in the library's kernels (POD, features, ridge
// normal equations, MLP forward / backward / Adam in csrc/mlp.cu; the small
// kernels of this file); the host only holds sizes, seeds and the held-out
// losses of at most a few hundred rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "dj_internal.h"

namespace dj {
// dj_api.cu: the mesh's prescribed DOFs (caller order, as dj_mesh_set_bcs got
// them), its ramp length and node count
const std::vector<long long>& mesh_bc_dofs(const dj_mesh* m);
long long mesh_ramp_steps(const dj_mesh* m);
long long mesh_n_nodes(const dj_mesh* m);
}  // namespace dj

using namespace dj;

struct dj_ws {
  dj_ws_params prm{};
  int n_bc = 0, n_in = 0, n_out = 0, n_k = 0, n_feat = 0;
  long long n_dof = 0;
  int quadratic = 0, use_mlp = 0, mlp_in = 0;
  std::vector<long long> bc_dof;
  std::vector<double> sig_in, sig_out;
  float *d_mean_in = nullptr, *d_modes_in = nullptr;    // modes scaled by 1 / spread
  float *d_mean_out = nullptr, *d_modes_out = nullptr;  // modes scaled by spread
  float* d_W = nullptr;                                 // n_out x n_feat
  long long* d_bc = nullptr;
  dj_mlp* mlp = nullptr;
  std::vector<int> widths;
  // prediction scratch
  float *d_t = nullptr, *d_c = nullptr, *d_f = nullptr, *d_q = nullptr, *d_q2 = nullptr;
  float *d_field = nullptr, *d_rest = nullptr;
  dj_ws_info info{};
  std::string last_error;
};

namespace {

dj_status wfail(dj_ws* w, dj_status s, const char* fmt, ...) {
  if (w) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    w->last_error = buf;
  }
  return s;
}

#define WCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t _e = (call);                                                                      \
    if (_e != cudaSuccess)                                                                        \
      return wfail(w, _e == cudaErrorMemoryAllocation ? DJ_ERR_OOM : DJ_ERR_CUDA, "%s: %s", #call, \
                   cudaGetErrorString(_e));                                                       \
  } while (0)
#define WST(call)                                               \
  do {                                                          \
    dj_status _s = (call);                                      \
    if (_s != DJ_OK) return wfail(w, _s, "%s failed", #call);   \
  } while (0)

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// A[i, j] *= s[j] (row-major rows x cols)
__global__ void scale_cols_kernel(float* A, long long rows, int cols, const float* __restrict__ sc) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < rows * cols) A[q] *= sc[q % cols];
}
// out[r, :] = A[idx[r], :]
__global__ void gather_rows_kernel(const float* __restrict__ A, int cols, const int* __restrict__ idx, int n,
                                   float* __restrict__ out) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)n * cols) return;
  const int r = (int)(q / cols), j = (int)(q % cols);
  out[q] = A[(long long)idx[r] * cols + j];
}
// F[s, j] = X[s, j] for j < n (X leading dimension ld)
__global__ void copy_cols_kernel(const float* __restrict__ X, int S, int ld, int n, float* __restrict__ F) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)S * n) return;
  F[q] = X[(q / n) * ld + q % n];
}
// field[dof[i]] = t[i]
__global__ void scatter_kernel(const float* __restrict__ t, const long long* __restrict__ dof, int n,
                               float* __restrict__ field) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) field[dof[i]] = t[i];
}
// Y += X
__global__ void add_kernel(float* Y, const float* __restrict__ X, long long n) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) Y[q] += X[q];
}

struct DevBufs {
  std::vector<void*> p;
  template <class T>
  T* get(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    p.push_back(q);
    return static_cast<T*>(q);
  }
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
};

template <class T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// the polynomial part's inputs for rows of coefficients X (S x n_in)
dj_status features(const dj_ws* w, const float* X, int S, float* F, cudaStream_t s) {
  if (w->quadratic) return dj_quad_features(X, S, w->n_in, w->n_k, F, s);
  copy_cols_kernel<<<nblk((long long)S * w->n_k, 256), 256, 0, s>>>(X, S, w->n_in, w->n_k, F);
  return cudaGetLastError() == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

// held-out loss: sum_j w_j (P_ij - Q_ij)^2 / (n n_out), on host copies (n <= a few hundred)
double weighted_mse(const std::vector<float>& P, const std::vector<float>& Q, const std::vector<float>& wt, int n,
                    int n_out) {
  double acc = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n_out; ++j) {
      const double d = (double)P[(size_t)i * n_out + j] - Q[(size_t)i * n_out + j];
      acc += wt[j] * d * d;
    }
  return acc / ((double)n * n_out);
}

dj_status to_host(std::vector<float>& h, const float* d, size_t n, cudaStream_t s) {
  h.resize(n);
  if (cudaMemcpyAsync(h.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return DJ_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? DJ_OK : DJ_ERR_CUDA;
}

void release(dj_ws* w) {
  void* ps[] = {w->d_mean_in, w->d_modes_in, w->d_mean_out, w->d_modes_out, w->d_W, w->d_bc,
                w->d_t,       w->d_c,        w->d_f,        w->d_q,         w->d_q2, w->d_field, w->d_rest};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (w->mlp) dj_mlp_destroy(w->mlp);
  w->mlp = nullptr;
}

// per-model buffers once the sizes are known
dj_status alloc_model(dj_ws* w) {
  WCK(dalloc(&w->d_mean_in, w->n_bc));
  WCK(dalloc(&w->d_modes_in, (size_t)w->n_bc * w->n_in));
  WCK(dalloc(&w->d_mean_out, w->n_dof));
  WCK(dalloc(&w->d_modes_out, (size_t)w->n_dof * w->n_out));
  WCK(dalloc(&w->d_bc, w->n_bc));
  WCK(cudaMemcpy(w->d_bc, w->bc_dof.data(), w->n_bc * sizeof(long long), cudaMemcpyHostToDevice));
  WCK(dalloc(&w->d_t, w->n_bc));
  WCK(dalloc(&w->d_c, w->n_in));
  WCK(dalloc(&w->d_q, w->n_out));
  WCK(dalloc(&w->d_q2, w->n_out));
  WCK(dalloc(&w->d_field, w->n_dof));
  WCK(dalloc(&w->d_rest, w->n_dof));
  return DJ_OK;
}

dj_status alloc_features(dj_ws* w) {
  WCK(dalloc(&w->d_W, (size_t)w->n_out * w->n_feat));
  WCK(dalloc(&w->d_f, w->n_feat));
  return DJ_OK;
}

int count_features(int n_k, int quadratic) { return n_k + (quadratic ? n_k * (n_k + 1) / 2 : 0); }

// The fit from training loads d_T (S x n_bc) and relaxed fields d_Y (S x n_dof),
// both snapshot-major on the device.
dj_status ws_fit(dj_ws* w, const float* d_T, const float* d_Y, int S, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const dj_ws_params& P = w->prm;
  w->n_in = std::min(P.n_in, S);
  w->n_out = std::min(P.n_out, S);
  dj_status st = alloc_model(w);
  if (st) return st;
  w->sig_in.assign(w->n_in, 0.0);
  w->sig_out.assign(w->n_out, 0.0);
  WST(dj_pod_fit(d_T, w->n_bc, S, w->n_in, w->d_mean_in, w->d_modes_in, w->sig_in.data(), s));
  WST(dj_pod_fit(d_Y, w->n_dof, S, w->n_out, w->d_mean_out, w->d_modes_out, w->sig_out.data(), s));
  // bases scaled to unit coefficient spread over the loads; modes beyond the
  // numerical rank (a load family of low dimension has few input modes) are
  // switched off rather than scaled up to unit-variance noise
  std::vector<float> inv_in(w->n_in, 0.f), sp_out(w->n_out, 0.f), inv_out(w->n_out, 0.f), wt(w->n_out, 0.f);
  w->n_k = 0;
  const double rs = std::sqrt((double)S);
  for (int j = 0; j < w->n_in; ++j)
    if (w->sig_in[j] > 1e-4 * std::max(w->sig_in[0], 1e-300)) {
      inv_in[j] = (float)(rs / w->sig_in[j]);
      w->n_k = j + 1;
    }
  int n_out_kept = 0;
  double var_sum = 0.0;
  for (int j = 0; j < w->n_out; ++j)
    if (w->sig_out[j] > 1e-6 * std::max(w->sig_out[0], 1e-300)) {
      sp_out[j] = (float)(w->sig_out[j] / rs);
      inv_out[j] = (float)(rs / w->sig_out[j]);
      var_sum += w->sig_out[j] * w->sig_out[j];
      ++n_out_kept;
    }
  if (w->n_k == 0 || n_out_kept == 0) return wfail(w, DJ_ERR_INVALID_ARG, "training loads or fields have no spread");
  // loss weights: output variance shares, so the loss tracks the field error
  for (int j = 0; j < w->n_out; ++j)
    if (sp_out[j] > 0) wt[j] = (float)(w->sig_out[j] * w->sig_out[j] * w->n_out / var_sum);
  w->info.n_in_kept = w->n_k;
  w->info.n_out_kept = n_out_kept;
  DevBufs b;
  float* d_sc = b.get<float>(std::max(w->n_in, w->n_out));
  float* d_proj = b.get<float>((size_t)w->n_dof * w->n_out);
  float* d_X = b.get<float>((size_t)S * w->n_in);
  float* d_Q = b.get<float>((size_t)S * w->n_out);
  float* d_wt = b.get<float>(w->n_out);
  if (!d_sc || !d_proj || !d_X || !d_Q || !d_wt) return wfail(w, DJ_ERR_OOM, "warm-start fit scratch");
  // inputs: modes_in / spread; outputs: expansion basis modes * spread,
  // projection basis modes / spread
  WCK(cudaMemcpyAsync(d_sc, inv_in.data(), w->n_in * sizeof(float), cudaMemcpyHostToDevice, s));
  scale_cols_kernel<<<nblk((long long)w->n_bc * w->n_in, 256), 256, 0, s>>>(w->d_modes_in, w->n_bc, w->n_in, d_sc);
  WCK(cudaGetLastError());
  WCK(cudaStreamSynchronize(s));
  WCK(cudaMemcpyAsync(d_proj, w->d_modes_out, (size_t)w->n_dof * w->n_out * sizeof(float), cudaMemcpyDeviceToDevice, s));
  WCK(cudaMemcpyAsync(d_sc, sp_out.data(), w->n_out * sizeof(float), cudaMemcpyHostToDevice, s));
  scale_cols_kernel<<<nblk(w->n_dof * w->n_out, 256), 256, 0, s>>>(w->d_modes_out, w->n_dof, w->n_out, d_sc);
  WCK(cudaGetLastError());
  WCK(cudaStreamSynchronize(s));
  WCK(cudaMemcpyAsync(d_sc, inv_out.data(), w->n_out * sizeof(float), cudaMemcpyHostToDevice, s));
  scale_cols_kernel<<<nblk(w->n_dof * w->n_out, 256), 256, 0, s>>>(d_proj, w->n_dof, w->n_out, d_sc);
  WCK(cudaGetLastError());
  WCK(cudaMemcpyAsync(d_wt, wt.data(), w->n_out * sizeof(float), cudaMemcpyHostToDevice, s));
  WST(dj_pod_project(w->d_modes_in, w->d_mean_in, w->n_bc, w->n_in, d_T, S, d_X, s));
  WST(dj_pod_project(d_proj, w->d_mean_out, w->n_dof, w->n_out, d_Y, S, d_Q, s));
  WCK(cudaStreamSynchronize(s));
  // seeded hold-out split
  const int n_val = (P.holdout > 0.0 && S >= 20) ? std::max(1, (int)std::lround(P.holdout * S)) : 0;
  const int S_tr = S - n_val;
  std::vector<int> perm(S);
  std::iota(perm.begin(), perm.end(), 0);
  std::mt19937_64 rng(P.seed);
  std::shuffle(perm.begin(), perm.end(), rng);
  int* d_idx = b.get<int>(S);
  float* d_Xtr = b.get<float>((size_t)S_tr * w->n_in);
  float* d_Qtr = b.get<float>((size_t)S_tr * w->n_out);
  float* d_Xv = b.get<float>((size_t)std::max(n_val, 1) * w->n_in);
  float* d_Qv = b.get<float>((size_t)std::max(n_val, 1) * w->n_out);
  if (!d_idx || !d_Xtr || !d_Qtr || !d_Xv || !d_Qv) return wfail(w, DJ_ERR_OOM, "warm-start split scratch");
  WCK(cudaMemcpyAsync(d_idx, perm.data(), S * sizeof(int), cudaMemcpyHostToDevice, s));
  const auto gather = [&](const float* A, int cols, const int* idx, int n, float* out) {
    if (n > 0) gather_rows_kernel<<<nblk((long long)n * cols, 256), 256, 0, s>>>(A, cols, idx, n, out);
    return cudaGetLastError();
  };
  WCK(gather(d_X, w->n_in, d_idx, n_val, d_Xv));
  WCK(gather(d_Q, w->n_out, d_idx, n_val, d_Qv));
  WCK(gather(d_X, w->n_in, d_idx + n_val, S_tr, d_Xtr));
  WCK(gather(d_Q, w->n_out, d_idx + n_val, S_tr, d_Qtr));
  WCK(cudaStreamSynchronize(s));
  std::vector<float> hQv, hP;
  if (n_val) {
    st = to_host(hQv, d_Qv, (size_t)n_val * w->n_out, s);
    if (st) return wfail(w, st, "held-out copy");
  }
  // polynomial part by ridge least squares: first order, and second order if
  // it does better on the held-out loads
  const int max_feat = std::max(count_features(w->n_k, 1), w->n_k);
  float* d_Ftr = b.get<float>((size_t)S_tr * max_feat);
  float* d_Fv = b.get<float>((size_t)std::max(n_val, 1) * max_feat);
  float* d_Pv = b.get<float>((size_t)std::max(n_val, 1) * w->n_out);
  float* d_W1 = b.get<float>((size_t)w->n_out * max_feat);
  if (!d_Ftr || !d_Fv || !d_Pv || !d_W1) return wfail(w, DJ_ERR_OOM, "warm-start feature scratch");
  const auto fit_poly = [&](int quadratic, double* loss) -> dj_status {
    w->quadratic = quadratic;
    w->n_feat = count_features(w->n_k, quadratic);
    dj_status q = features(w, d_Xtr, S_tr, d_Ftr, s);
    if (q) return q;
    q = dj_linear_fit(d_Ftr, d_Qtr, S_tr, w->n_feat, w->n_out, quadratic ? 1e-4 : 1e-6, d_W1, s);
    if (q) return q;
    *loss = NAN;
    if (n_val) {
      q = features(w, d_Xv, n_val, d_Fv, s);
      if (q) return q;
      q = dj_linear_apply(d_W1, w->n_out, w->n_feat, d_Fv, n_val, 1.f, 0.f, d_Pv, s);
      if (q) return q;
      q = to_host(hP, d_Pv, (size_t)n_val * w->n_out, s);
      if (q) return q;
      *loss = weighted_mse(hP, hQv, wt, n_val, w->n_out);
    }
    return DJ_OK;
  };
  double l1 = NAN, l2 = NAN;
  st = fit_poly(0, &l1);
  if (st) return wfail(w, st, "first-order fit failed");
  w->info.val_loss_first_order = l1;
  w->info.val_loss_second_order = NAN;
  bool second = false;
  if (P.quadratic && S_tr > 2 * w->n_k && count_features(w->n_k, 1) <= 1024) {
    st = fit_poly(1, &l2);
    if (st) return wfail(w, st, "second-order fit failed");
    w->info.val_loss_second_order = l2;
    second = !(n_val > 0) || (l2 < l1);
    if (!second) {
      st = fit_poly(0, &l1);
      if (st) return wfail(w, st, "first-order refit failed");
    }
  }
  w->quadratic = second ? 1 : 0;
  w->n_feat = count_features(w->n_k, w->quadratic);
  st = alloc_features(w);
  if (st) return st;
  WCK(cudaMemcpyAsync(w->d_W, d_W1, (size_t)w->n_out * w->n_feat * sizeof(float), cudaMemcpyDeviceToDevice, s));
  const double l_poly = second ? l2 : l1;
  w->info.val_loss_polynomial = l_poly;
  w->info.quadratic_used = w->quadratic;
  // remainder the MLP learns: Q - W f(X)
  st = features(w, d_Xtr, S_tr, d_Ftr, s);
  if (st) return wfail(w, st, "features");
  WST(dj_linear_apply(w->d_W, w->n_out, w->n_feat, d_Ftr, S_tr, -1.f, 1.f, d_Qtr, s));
  w->info.val_loss_polynomial_mlp = NAN;
  w->use_mlp = 0;
  w->info.fit_seconds_polynomial = seconds_since(t0);
  if (P.mlp != 0 && S_tr >= 8) {
    // MLP input: the input coefficients, or the polynomial part's features
    w->mlp_in = P.mlp_input == DJ_WS_MLP_ON_FEATURES ? w->n_feat : w->n_in;
    const float* Xm_tr = P.mlp_input == DJ_WS_MLP_ON_FEATURES ? d_Ftr : d_Xtr;
    w->widths.clear();
    w->widths.push_back(w->mlp_in);
    for (int l = 0; l < 4 && P.hidden[l] > 0; ++l) w->widths.push_back(P.hidden[l]);
    w->widths.push_back(w->n_out);
    WST(dj_mlp_create(w->widths.data(), (int)w->widths.size() - 1, P.seed, &w->mlp));
    if (P.mlp_bf16) WST(dj_mlp_set_precision(w->mlp, 1));
    const int bsz = std::min(P.batch, S_tr);
    const int per_epoch = std::max(1, S_tr / bsz);
    const long long n_iter = (long long)P.epochs * per_epoch;
    // minibatch schedule: one permutation of the training rows per epoch
    int* d_sched = b.get<int>((size_t)per_epoch * bsz * std::max(1, P.epochs));
    float* d_xb = b.get<float>((size_t)bsz * w->mlp_in);
    float* d_tb = b.get<float>((size_t)bsz * w->n_out);
    if (!d_sched || !d_xb || !d_tb) return wfail(w, DJ_ERR_OOM, "MLP training scratch");
    {
      std::vector<int> sched((size_t)per_epoch * bsz * P.epochs), order(S_tr);
      std::iota(order.begin(), order.end(), 0);
      for (int ep = 0; ep < P.epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        std::copy(order.begin(), order.begin() + (size_t)per_epoch * bsz, sched.begin() + (size_t)ep * per_epoch * bsz);
      }
      WCK(cudaMemcpyAsync(d_sched, sched.data(), sched.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      WCK(cudaStreamSynchronize(s));
    }
    double last = NAN;
    for (long long it = 0; it < n_iter; ++it) {
      const int* idx = d_sched + it * bsz;
      WCK(gather(Xm_tr, w->mlp_in, idx, bsz, d_xb));
      WCK(gather(d_Qtr, w->n_out, idx, bsz, d_tb));
      const bool want = it == n_iter - 1;
      WST(dj_mlp_loss_grad(w->mlp, d_xb, d_tb, d_wt, bsz, want ? &last : nullptr, s));
      const double frac = n_iter > 1 ? (double)it / (double)(n_iter - 1) : 0.0;
      const double lr = P.lr * std::pow(P.lr_final / P.lr, frac);
      WST(dj_mlp_adam_step(w->mlp, (float)lr, 0.9f, 0.999f, 1e-8f, s));
    }
    w->info.final_train_loss = last;
    w->info.mlp_iterations = n_iter;
    w->use_mlp = 1;
    if (n_val) {
      // held-out: polynomial part alone against polynomial part + MLP
      float* d_Mv = b.get<float>((size_t)n_val * w->n_out);
      if (!d_Mv) return wfail(w, DJ_ERR_OOM, "held-out scratch");
      st = features(w, d_Xv, n_val, d_Fv, s);
      if (st) return wfail(w, st, "features");
      WST(dj_linear_apply(w->d_W, w->n_out, w->n_feat, d_Fv, n_val, 1.f, 0.f, d_Pv, s));
      WST(dj_mlp_forward(w->mlp, P.mlp_input == DJ_WS_MLP_ON_FEATURES ? d_Fv : d_Xv, n_val, d_Mv, s));
      add_kernel<<<nblk((long long)n_val * w->n_out, 256), 256, 0, s>>>(d_Mv, d_Pv, (long long)n_val * w->n_out);
      WCK(cudaGetLastError());
      st = to_host(hP, d_Mv, (size_t)n_val * w->n_out, s);
      if (st) return wfail(w, st, "held-out copy");
      w->info.val_loss_polynomial_mlp = weighted_mse(hP, hQv, wt, n_val, w->n_out);
      if (P.mlp < 0) w->use_mlp = w->info.val_loss_polynomial_mlp < l_poly ? 1 : 0;
    }
  }
  WCK(cudaStreamSynchronize(s));
  w->info.mlp_used = w->use_mlp;
  w->info.n_train = S_tr;
  w->info.n_holdout = n_val;
  w->info.fit_seconds = seconds_since(t0);
  return DJ_OK;
}

dj_status new_ws(const dj_ws_params* prm, dj_ws** out) {
  if (!out) return DJ_ERR_INVALID_ARG;
  *out = nullptr;
  dj_ws_params P;
  if (prm)
    P = *prm;
  else
    dj_ws_params_default(&P);
  if (P.n_in <= 0 || P.n_in > 256 || P.n_out <= 0 || P.n_out > 1024 || P.epochs < 0 || P.batch <= 0 ||
      !(P.lr > 0) || !(P.lr_final > 0) || !(P.holdout >= 0 && P.holdout < 0.9) ||
      (P.mlp_input != DJ_WS_MLP_ON_COEFFS && P.mlp_input != DJ_WS_MLP_ON_FEATURES) ||
      (P.mlp_bf16 != 0 && P.mlp_bf16 != 1) || P.mlp < -1 || P.mlp > 1 || P.bootstrap < 0 ||
      (P.bootstrap > 0 && P.bootstrap < 20))
    return DJ_ERR_INVALID_ARG;
  for (int l = 0; l < 4; ++l)
    if (P.hidden[l] < 0 || P.hidden[l] > 4096) return DJ_ERR_INVALID_ARG;
  dj_ws* w = new (std::nothrow) dj_ws();
  if (!w) return DJ_ERR_OOM;
  w->prm = P;
  *out = w;
  return DJ_OK;
}

// relax the mesh's current state (plain or adaptive damping)
dj_status relax(dj_mesh* m, const dj_ws* w, double tol, long long max_steps, long long* steps, double* r,
                cudaStream_t s) {
  if (w->prm.adaptive) return dj_relax_adaptive(m, tol, max_steps, nullptr, steps, r, nullptr, s);
  return dj_relax_to_tol(m, tol, max_steps, steps, r, s);
}

// U^0 = 0 at step 0 (the relaxation from rest); d_zero: n_dof zero floats
dj_status start_from_rest(dj_mesh* m, const float* d_zero, cudaStream_t s) {
  dj_status st = dj_set_displacements_device(m, d_zero, s);
  if (st) return st;
  return dj_set_step(m, 0);
}

}  // namespace

extern "C" {

void dj_ws_params_default(dj_ws_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_in = 64;
  p->n_out = 128;
  p->hidden[0] = p->hidden[1] = p->hidden[2] = 256;
  p->epochs = 1500;
  p->batch = 128;
  p->lr = 1e-3;
  p->lr_final = 1e-5;
  p->quadratic = 1;
  p->mlp = -1;
  p->mlp_input = DJ_WS_MLP_ON_COEFFS;
  p->mlp_bf16 = 0;
  p->holdout = 0.1;
  p->seed = 0;
  p->adaptive = 1;
  p->bootstrap = 0;
}

dj_status dj_ws_fit(const long long* bc_dof, int n_bc, long long n_nodes, const float* d_targets,
                    const float* d_fields, int n_loads, const dj_ws_params* prm, dj_ws** out, void* stream) {
  if (!out) return DJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (!bc_dof || n_bc <= 0 || n_nodes <= 0 || !d_targets || !d_fields || n_loads < 2) return DJ_ERR_INVALID_ARG;
  for (int i = 0; i < n_bc; ++i)
    if (bc_dof[i] < 0 || bc_dof[i] >= 3 * n_nodes) return DJ_ERR_INVALID_ARG;
  dj_ws* w = nullptr;
  dj_status st = new_ws(prm, &w);
  if (st) return st;
  w->n_bc = n_bc;
  w->n_dof = 3 * n_nodes;
  w->bc_dof.assign(bc_dof, bc_dof + n_bc);
  w->info.n_loads = n_loads;
  w->info.n_kept = n_loads;
  st = ws_fit(w, d_targets, d_fields, n_loads, (cudaStream_t)stream);
  if (st) {
    release(w);
    delete w;
    return st;
  }
  *out = w;
  return DJ_OK;
}

dj_status dj_ws_train(dj_mesh* mesh, const double* targets, int n_loads, double tol, long long max_steps,
                      const dj_ws_params* prm, dj_ws** out, void* stream) {
  if (!out) return DJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !targets || n_loads < 2 || !(tol > 0) || max_steps <= 0) return DJ_ERR_INVALID_ARG;
  dj_info mi{};
  dj_status st = dj_get_info(mesh, &mi);
  if (st) return st;
  const std::vector<long long>& bc = mesh_bc_dofs(mesh);
  const int n_bc = (int)bc.size();
  if (n_bc == 0) return DJ_ERR_INVALID_ARG;
  const long long n_dof = 3 * mi.n_nodes;
  cudaStream_t s = (cudaStream_t)stream;
  dj_ws* w = nullptr;
  st = new_ws(prm, &w);
  if (st) return st;
  w->n_bc = n_bc;
  w->n_dof = n_dof;
  w->bc_dof = bc;
  w->info.n_loads = n_loads;
  const auto t0 = std::chrono::steady_clock::now();
  float *d_Y = nullptr, *d_T = nullptr, *d_zero = nullptr;
  auto cleanup = [&]() {
    if (d_Y) cudaFree(d_Y);
    if (d_T) cudaFree(d_T);
    if (d_zero) cudaFree(d_zero);
  };
  cudaError_t e = dalloc(&d_Y, (size_t)n_loads * n_dof);
  if (e == cudaSuccess) e = dalloc(&d_T, (size_t)n_loads * n_bc);
  if (e == cudaSuccess) e = dalloc(&d_zero, n_dof);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_zero, 0, n_dof * sizeof(float), s);
  if (e != cudaSuccess) {
    cleanup();
    delete w;
    return e == cudaErrorMemoryAllocation ? DJ_ERR_OOM : DJ_ERR_CUDA;
  }
  // training data: every load relaxed by the method to `tol`, from rest or
  // (bootstrap) from a fit to the loads relaxed so far, refitted whenever
  // their number doubles; loads that fail are dropped
  int kept = 0;
  long long steps_sum = 0;
  std::vector<float> tf(n_bc);
  dj_ws* boot = nullptr;  // the current intermediate fit
  int next_fit = w->prm.bootstrap > 0 ? w->prm.bootstrap : INT_MAX;
  for (int i = 0; i < n_loads && st == DJ_OK; ++i) {
    const double* t = targets + (size_t)i * n_bc;
    if (kept >= next_fit && kept < n_loads) {
      if (boot) dj_ws_destroy(boot);
      boot = nullptr;
      st = new_ws(&w->prm, &boot);
      if (st) break;
      boot->n_bc = n_bc;
      boot->n_dof = n_dof;
      boot->bc_dof = bc;
      st = ws_fit(boot, d_T, d_Y, kept, s);
      if (st) {
        w->last_error = boot->last_error;
        break;
      }
      next_fit = 2 * kept;
    }
    long long n = 0;
    double r = 0;
    dj_status rs;
    if (boot) {
      dj_ws_result res{};
      rs = dj_ws_relax_to_tol(mesh, boot, t, DJ_WS_ARM_FITTED, tol, max_steps, &res, stream);
      n = res.steps;
      if (rs == DJ_ERR_INVALID_ARG) {
        st = rs;
        w->last_error = boot->last_error;
        break;
      }
    } else {
      st = dj_mesh_update_bc_targets(mesh, t);
      if (st) break;
      st = start_from_rest(mesh, d_zero, s);
      if (st) break;
      rs = relax(mesh, w, tol, max_steps, &n, &r, s);
    }
    if (rs == DJ_ERR_CUDA || rs == DJ_ERR_OOM) {
      st = rs;
      break;
    }
    if (rs != DJ_OK) continue;
    st = dj_get_displacements_device(mesh, d_Y + (size_t)kept * n_dof, s);
    if (st) break;
    for (int k = 0; k < n_bc; ++k) tf[k] = (float)t[k];
    if (cudaMemcpyAsync(d_T + (size_t)kept * n_bc, tf.data(), n_bc * sizeof(float), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = DJ_ERR_CUDA;
      break;
    }
    steps_sum += n;
    ++kept;
  }
  if (boot) dj_ws_destroy(boot);
  w->info.n_kept = kept;
  w->info.data_seconds = seconds_since(t0);
  w->info.mean_training_steps = kept ? (double)steps_sum / kept : 0.0;
  if (st == DJ_OK && kept < 2) st = DJ_ERR_NOT_CONVERGED;
  if (st == DJ_OK) st = ws_fit(w, d_T, d_Y, kept, s);
  cleanup();
  if (st) {
    release(w);
    delete w;
    return st;
  }
  *out = w;
  return DJ_OK;
}

dj_status dj_ws_predict(dj_ws* w, const double* targets, int parts, float* d_field, void* stream) {
  if (!w) return DJ_ERR_INVALID_ARG;
  if (!targets || !d_field) return wfail(w, DJ_ERR_INVALID_ARG, "null targets or field");
  if (parts == DJ_WS_PARTS_FITTED) parts = DJ_WS_PARTS_POLYNOMIAL | (w->use_mlp ? DJ_WS_PARTS_MLP : 0);
  if (parts < 0 || parts > 3 || ((parts & DJ_WS_PARTS_MLP) && !w->mlp))
    return wfail(w, DJ_ERR_INVALID_ARG, "parts %d not available", parts);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> tf(w->n_bc);
  for (int k = 0; k < w->n_bc; ++k) tf[k] = (float)targets[k];
  WCK(cudaMemcpyAsync(w->d_t, tf.data(), w->n_bc * sizeof(float), cudaMemcpyHostToDevice, s));
  WST(dj_pod_project(w->d_modes_in, w->d_mean_in, w->n_bc, w->n_in, w->d_t, 1, w->d_c, s));
  WCK(cudaMemsetAsync(w->d_q, 0, w->n_out * sizeof(float), s));
  if (parts & DJ_WS_PARTS_POLYNOMIAL) {
    dj_status st = features(w, w->d_c, 1, w->d_f, s);
    if (st) return wfail(w, st, "features");
    WST(dj_linear_apply(w->d_W, w->n_out, w->n_feat, w->d_f, 1, 1.f, 0.f, w->d_q, s));
  }
  if (parts & DJ_WS_PARTS_MLP) {
    const float* xin = w->d_c;
    if (w->prm.mlp_input == DJ_WS_MLP_ON_FEATURES) {
      dj_status st = features(w, w->d_c, 1, w->d_f, s);
      if (st) return wfail(w, st, "features");
      xin = w->d_f;
    }
    WST(dj_mlp_forward(w->mlp, xin, 1, w->d_q2, s));
    add_kernel<<<nblk(w->n_out, 128), 128, 0, s>>>(w->d_q, w->d_q2, w->n_out);
    WCK(cudaGetLastError());
  }
  WST(dj_pod_expand(w->d_modes_out, w->d_mean_out, w->n_dof, w->n_out, w->d_q, 1, d_field, s));
  WCK(cudaStreamSynchronize(s));  // tf is host memory of this frame
  return DJ_OK;
}

dj_status dj_ws_relax_to_tol(dj_mesh* mesh, dj_ws* w, const double* targets, int arm, double tol,
                             long long max_steps, dj_ws_result* res, void* stream) {
  if (!w) return DJ_ERR_INVALID_ARG;
  if (!mesh || !targets || !(tol > 0) || max_steps <= 0 || arm < DJ_WS_ARM_REST || arm > DJ_WS_ARM_FITTED)
    return wfail(w, DJ_ERR_INVALID_ARG, "bad arguments");
  dj_info mi{};
  dj_status st = dj_get_info(mesh, &mi);
  if (st) return wfail(w, st, "dj_get_info");
  if (3 * mi.n_nodes != w->n_dof || (long long)mesh_bc_dofs(mesh).size() != w->n_bc ||
      !std::equal(w->bc_dof.begin(), w->bc_dof.end(), mesh_bc_dofs(mesh).begin()))
    return wfail(w, DJ_ERR_INVALID_ARG, "mesh does not match the warm start (nodes or prescribed DOFs)");
  cudaStream_t s = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  dj_ws_result out{};
  st = dj_mesh_update_bc_targets(mesh, targets);
  if (st) return wfail(w, st, "dj_mesh_update_bc_targets: %s", dj_last_error(mesh));
  WCK(cudaMemsetAsync(w->d_rest, 0, w->n_dof * sizeof(float), s));
  bool warm = false;
  if (arm != DJ_WS_ARM_REST) {
    const int parts = arm == DJ_WS_ARM_POLYNOMIAL ? DJ_WS_PARTS_POLYNOMIAL : DJ_WS_PARTS_FITTED;
    st = dj_ws_predict(w, targets, parts, w->d_field, stream);
    if (st) return st;
    // the prediction is used only if it inverts no element and has a smaller
    // residual than the field that holds the prescribed values alone
    double r_warm = INFINITY, r_bc = INFINITY;
    int inv = 0, inv_bc = 0;
    st = dj_evaluate_field(mesh, w->d_field, &r_warm, &inv, stream);
    if (st) return wfail(w, st, "dj_evaluate_field: %s", dj_last_error(mesh));
    std::vector<float> tf(w->n_bc);
    for (int k = 0; k < w->n_bc; ++k) tf[k] = (float)targets[k];
    WCK(cudaMemcpyAsync(w->d_t, tf.data(), w->n_bc * sizeof(float), cudaMemcpyHostToDevice, s));
    scatter_kernel<<<nblk(w->n_bc, 256), 256, 0, s>>>(w->d_t, w->d_bc, w->n_bc, w->d_rest);
    WCK(cudaGetLastError());
    st = dj_evaluate_field(mesh, w->d_rest, &r_bc, &inv_bc, stream);
    if (st) return wfail(w, st, "dj_evaluate_field: %s", dj_last_error(mesh));
    WCK(cudaMemsetAsync(w->d_rest, 0, w->n_dof * sizeof(float), s));
    out.residual_predicted = r_warm;
    out.residual_prescribed_only = r_bc;
    warm = !inv && r_warm < r_bc;
    out.fallback = warm ? 0 : 1;
  }
  out.predict_seconds = seconds_since(t0);
  long long n = 0;
  double r = 0;
  dj_status rs;
  if (warm) {
    st = dj_set_displacements_device(mesh, w->d_field, stream);
    if (st == DJ_OK) st = dj_set_step(mesh, std::max(0LL, mesh_ramp_steps(mesh)));
    if (st) return wfail(w, st, "warm state: %s", dj_last_error(mesh));
    rs = relax(mesh, w, tol, max_steps, &n, &r, s);
    if (rs != DJ_OK && rs != DJ_ERR_CUDA && rs != DJ_ERR_OOM) {
      // the relaxation from the prediction failed (e.g. an element inverted on
      // the way): the same solve from rest decides
      out.fallback = 1;
      warm = false;
      out.steps_warm_attempt = n;
    }
  }
  if (!warm) {
    st = start_from_rest(mesh, w->d_rest, s);
    if (st) return wfail(w, st, "rest state: %s", dj_last_error(mesh));
    long long n2 = 0;
    rs = relax(mesh, w, tol, max_steps, &n2, &r, s);
    n += n2;
  }
  out.steps = n;
  out.residual = r;
  out.started_warm = warm ? 1 : 0;
  out.seconds = seconds_since(t0);
  if (res) *res = out;
  if (rs != DJ_OK) return wfail(w, rs, "relaxation: %s", dj_last_error(mesh));
  return DJ_OK;
}

namespace {
constexpr char kMagic[8] = {'D', 'J', 'W', 'S', '0', '0', '0', '1'};
struct WsHeader {
  char magic[8];
  int n_bc, n_in, n_out, n_k, n_feat, quadratic, use_mlp, mlp_in, n_widths;
  long long n_dof, n_mlp_params;
  dj_ws_params prm;
  dj_ws_info info;
};
struct Writer {
  char* buf;
  size_t cap, pos = 0;
  bool fits = true;
  void put(const void* p, size_t n) {
    if (buf && pos + n <= cap) std::memcpy(buf + pos, p, n);
    else if (buf) fits = false;
    pos += n;
  }
};
}  // namespace

dj_status dj_ws_save(const dj_ws* wc, void* buf, size_t capacity, size_t* bytes) {
  dj_ws* w = const_cast<dj_ws*>(wc);
  if (!w || !bytes) return DJ_ERR_INVALID_ARG;
  WsHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.n_bc = w->n_bc;
  h.n_in = w->n_in;
  h.n_out = w->n_out;
  h.n_k = w->n_k;
  h.n_feat = w->n_feat;
  h.quadratic = w->quadratic;
  h.use_mlp = w->use_mlp;
  h.mlp_in = w->mlp_in;
  h.n_widths = w->mlp ? (int)w->widths.size() : 0;
  h.n_dof = w->n_dof;
  h.n_mlp_params = w->mlp ? dj_mlp_num_params(w->mlp) : 0;
  h.prm = w->prm;
  h.info = w->info;
  Writer out{static_cast<char*>(buf), capacity};
  out.put(&h, sizeof h);
  out.put(w->bc_dof.data(), w->n_bc * sizeof(long long));
  out.put(w->sig_in.data(), w->n_in * sizeof(double));
  out.put(w->sig_out.data(), w->n_out * sizeof(double));
  const auto dev = [&](const float* d, size_t n) -> dj_status {
    std::vector<float> t(n);
    if (buf && cudaMemcpy(t.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return DJ_ERR_CUDA;
    out.put(t.data(), n * sizeof(float));
    return DJ_OK;
  };
  dj_status st = DJ_OK;
  if (!st) st = dev(w->d_mean_in, w->n_bc);
  if (!st) st = dev(w->d_modes_in, (size_t)w->n_bc * w->n_in);
  if (!st) st = dev(w->d_mean_out, w->n_dof);
  if (!st) st = dev(w->d_modes_out, (size_t)w->n_dof * w->n_out);
  if (!st) st = dev(w->d_W, (size_t)w->n_out * w->n_feat);
  if (st) return wfail(w, st, "copy of the model to the host failed");
  if (w->mlp) {
    out.put(w->widths.data(), w->widths.size() * sizeof(int));
    std::vector<float> prm((size_t)h.n_mlp_params);
    if (buf) WST(dj_mlp_get_params(w->mlp, prm.data(), h.n_mlp_params));
    out.put(prm.data(), prm.size() * sizeof(float));
  }
  *bytes = out.pos;
  if (buf && !out.fits) return wfail(w, DJ_ERR_INVALID_ARG, "capacity %zu < %zu bytes", capacity, out.pos);
  return DJ_OK;
}

dj_status dj_ws_load(const void* buf, size_t bytes, dj_ws** out) {
  if (!out) return DJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (!buf || bytes < sizeof(WsHeader)) return DJ_ERR_INVALID_ARG;
  WsHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.n_bc <= 0 || h.n_in <= 0 || h.n_out <= 0 || h.n_dof <= 0 ||
      h.n_k <= 0 || h.n_k > h.n_in || h.n_feat != count_features(h.n_k, h.quadratic) || h.n_widths < 0 ||
      h.n_widths > 17 || h.n_mlp_params < 0)
    return DJ_ERR_INVALID_ARG;
  const size_t need = sizeof h + h.n_bc * sizeof(long long) + (h.n_in + h.n_out) * sizeof(double) +
                      ((size_t)h.n_bc * (1 + h.n_in) + (size_t)h.n_dof * (1 + h.n_out) + (size_t)h.n_out * h.n_feat) *
                          sizeof(float) +
                      h.n_widths * sizeof(int) + (size_t)h.n_mlp_params * sizeof(float);
  if (bytes != need) return DJ_ERR_INVALID_ARG;
  dj_ws* w = nullptr;
  dj_status st = new_ws(&h.prm, &w);
  if (st) return st;
  w->n_bc = h.n_bc;
  w->n_in = h.n_in;
  w->n_out = h.n_out;
  w->n_k = h.n_k;
  w->n_feat = h.n_feat;
  w->quadratic = h.quadratic;
  w->use_mlp = h.use_mlp;
  w->mlp_in = h.mlp_in;
  w->n_dof = h.n_dof;
  w->info = h.info;
  const char* p = static_cast<const char*>(buf) + sizeof h;
  const auto take = [&](void* dst, size_t n) {
    std::memcpy(dst, p, n);
    p += n;
  };
  w->bc_dof.resize(h.n_bc);
  take(w->bc_dof.data(), h.n_bc * sizeof(long long));
  w->sig_in.resize(h.n_in);
  take(w->sig_in.data(), h.n_in * sizeof(double));
  w->sig_out.resize(h.n_out);
  take(w->sig_out.data(), h.n_out * sizeof(double));
  st = alloc_model(w);
  if (st == DJ_OK) st = alloc_features(w);
  const auto dev = [&](float* d, size_t n) -> dj_status {
    if (cudaMemcpy(d, p, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return DJ_ERR_CUDA;
    p += n * sizeof(float);
    return DJ_OK;
  };
  if (!st) st = dev(w->d_mean_in, w->n_bc);
  if (!st) st = dev(w->d_modes_in, (size_t)w->n_bc * w->n_in);
  if (!st) st = dev(w->d_mean_out, w->n_dof);
  if (!st) st = dev(w->d_modes_out, (size_t)w->n_dof * w->n_out);
  if (!st) st = dev(w->d_W, (size_t)w->n_out * w->n_feat);
  if (!st && h.n_widths > 0) {
    w->widths.resize(h.n_widths);
    take(w->widths.data(), h.n_widths * sizeof(int));
    st = dj_mlp_create(w->widths.data(), h.n_widths - 1, h.prm.seed, &w->mlp);
    if (!st && dj_mlp_num_params(w->mlp) != h.n_mlp_params) st = DJ_ERR_INVALID_ARG;
    if (!st) st = dj_mlp_set_params(w->mlp, reinterpret_cast<const float*>(p), h.n_mlp_params);
    if (!st && h.prm.mlp_bf16) st = dj_mlp_set_precision(w->mlp, 1);
  }
  if (st) {
    release(w);
    delete w;
    return st;
  }
  *out = w;
  return DJ_OK;
}

dj_status dj_ws_get_info(const dj_ws* w, dj_ws_info* info) {
  if (!w || !info) return DJ_ERR_INVALID_ARG;
  *info = w->info;
  info->n_in = w->n_in;
  info->n_out = w->n_out;
  info->n_features = w->n_feat;
  info->n_bc = w->n_bc;
  info->n_dof = w->n_dof;
  info->mlp_params = w->mlp ? dj_mlp_num_params(w->mlp) : 0;
  return DJ_OK;
}

const char* dj_ws_last_error(const dj_ws* w) { return w ? w->last_error.c_str() : "null warm start"; }

void dj_ws_destroy(dj_ws* w) {
  if (!w) return;
  release(w);
  delete w;
}

}  // extern "C"
