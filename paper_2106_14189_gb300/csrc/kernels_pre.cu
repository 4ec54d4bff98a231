// One-time FP64 pre-computation on the GPU (Algorithm 1, pre-computation).
//
// Per element (one thread, FP64): 0J = H_xi X_e (Eq. 3), det 0J, 0V, the
// symmetric I1m = 2 0V 0J^-T 0J^-1 (Eq. 37), I4m / I6m (Eq. 45-46) for fibre
// elements, the Mooney-Rivlin scalar, H8 hourglass constants, the element mass
// rho 0V / n_e and the element's stable step.  Results are rounded once to
// FP32 into the structure-of-arrays table read by the step kernels.
//
// Critical step (Eq. 14, dt <= L_e / c): L_e is taken as the length for which
// Eq. 14 equals 2 / omega_e, with the uniform-strain bound
//   omega_e^2 <= n_e c^2 sum_{i,a} 0B_ia^2  (+ n_e k lmax(Gamma Gamma^T) / (rho 0V), H8)
// c^2 = (kappa + 4/3 mu_eff + 16/9 (eta_a + eta_b)) / rho, lmax by Gershgorin:
// the largest acoustic modulus of the material linearised at rest (a fibre
// family adds 4 eta ((A - I/3) n)^2, largest along the fibre; an upper bound
// for two fibre families).
#include <cuda_runtime.h>
#include <float.h>

#include "dj_internal.h"
#include "dj_io.h"

namespace dj {

namespace {

__device__ constexpr double XI8D[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                          {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
__device__ constexpr double H8D[4][8] = {{1, -1, 1, -1, 1, -1, 1, -1},
                                         {1, 1, -1, -1, -1, -1, 1, 1},
                                         {1, -1, -1, 1, -1, 1, 1, -1},
                                         {-1, 1, -1, 1, 1, -1, 1, -1}};

// table row k of element e: structure of arrays (stride E_pad) or tile-major
__device__ void put(const PreArgs& a, float* t, int k, int e, double v) {
  const int T = a.tile_T;
  if (T > 0)
    t[((size_t)(e / T) * a.n_consts + k) * T + (e % T)] = (float)v;
  else
    t[(size_t)k * a.E_pad + e] = (float)v;
}

// S = 2 V Jinv^T d d^T Jinv  (d unit) -> sym6
__device__ void fibre_tensor(const double Ji[3][3], const double* d, double twoV, double* S) {
  double w[3];
  for (int i = 0; i < 3; ++i) w[i] = Ji[0][i] * d[0] + Ji[1][i] * d[1] + Ji[2][i] * d[2];  // 0J^-T d
  S[0] = twoV * w[0] * w[0];
  S[1] = twoV * w[1] * w[1];
  S[2] = twoV * w[2] * w[2];
  S[3] = twoV * w[0] * w[1];
  S[4] = twoV * w[0] * w[2];
  S[5] = twoV * w[1] * w[2];
}

__global__ void precompute_elements_kernel(PreArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.E) return;
  const int ne = a.ne;
  double Xe[8][3];
  int nid[8];
  for (int b = 0; b < ne; ++b) {
    nid[b] = a.conn[(size_t)e * ne + b];
    for (int j = 0; j < 3; ++j) Xe[b][j] = a.X[(size_t)3 * nid[b] + j];
  }
  if (ne == 4) {
    a.conn4[e] = make_int4(nid[0], nid[1], nid[2], nid[3]);
  } else {
    a.conn4[2 * (size_t)e] = make_int4(nid[0], nid[1], nid[2], nid[3]);
    a.conn4[2 * (size_t)e + 1] = make_int4(nid[4], nid[5], nid[6], nid[7]);
  }
  // H_xi (3 x n_e)
  double Hx[3][8];
  for (int i = 0; i < 3; ++i)
    for (int b = 0; b < 8; ++b) Hx[i][b] = 0.0;
  if (ne == 4) {
    for (int i = 0; i < 3; ++i) {
      Hx[i][0] = -1.0;
      Hx[i][i + 1] = 1.0;
    }
  } else {
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 8; ++b) Hx[i][b] = XI8D[b][i] / 8.0;
  }
  double J0[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int b = 0; b < ne; ++b) s += Hx[i][b] * Xe[b][j];
      J0[i][j] = s;  // Eq. 3
    }
  const double det = J0[0][0] * (J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1]) -
                     J0[0][1] * (J0[1][0] * J0[2][2] - J0[1][2] * J0[2][0]) +
                     J0[0][2] * (J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0]);
  if (!(det > 0.0)) {
    atomicMin(a.bad, e);
    a.dt_elem[e] = DBL_MAX;
    a.elem_mass[e] = 0.0;
    return;
  }
  const double id = 1.0 / det;
  double Ji[3][3];
  Ji[0][0] = (J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1]) * id;
  Ji[0][1] = (J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2]) * id;
  Ji[0][2] = (J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1]) * id;
  Ji[1][0] = (J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2]) * id;
  Ji[1][1] = (J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0]) * id;
  Ji[1][2] = (J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2]) * id;
  Ji[2][0] = (J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0]) * id;
  Ji[2][1] = (J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1]) * id;
  Ji[2][2] = (J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0]) * id;
  const double V0 = ne == 4 ? det / 6.0 : 8.0 * det;
  const double mu = a.mu[e], kappa = a.kappa[e], rho = a.rho[e];
  const int model = a.model[e];
  const double eta_a = (model == DJ_TI || model == DJ_OT) && a.eta_a ? a.eta_a[e] : 0.0;
  const double eta_b = (model == DJ_OT) && a.eta_b ? a.eta_b[e] : 0.0;
  const double c01 = (model == DJ_MR) && a.c01 ? a.c01[e] : 0.0;
  // 0J, P = (mu/2) I1m, kappa 0V, 1/det (common block)
  float* t = a.consts;
  if (a.geometric) {
    // P = mu 0V 0J^-T 0J^-1 = (mu 0V / det^2) adj(0J)^T adj(0J): one scalar
    put(a, t, KG_CP, e, mu * V0 * id * id);
    put(a, t, KG_KV, e, kappa * V0);
  } else {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) put(a, t, K_J0 + 3 * i + j, e, J0[i][j]);
    double K[6];  // 0J^-T 0J^-1
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
      double s = 0.0;
      for (int m = 0; m < 3; ++m) s += Ji[m][ii[k]] * Ji[m][jj[k]];
      K[k] = s;
    }
    for (int k = 0; k < 6; ++k) put(a, t, K_P + k, e, 0.5 * mu * 2.0 * V0 * K[k]);
    put(a, t, K_KV, e, kappa * V0);
    put(a, t, K_R0, e, id);
  }
  if (a.off_fa >= 0) {
    double S[6] = {0, 0, 0, 0, 0, 0};
    if (eta_a > 0.0) {
      double d[3] = {a.adir[3 * (size_t)e], a.adir[3 * (size_t)e + 1], a.adir[3 * (size_t)e + 2]};
      const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int j = 0; j < 3; ++j) d[j] /= n;
      fibre_tensor(Ji, d, 2.0 * V0, S);
    }
    for (int k = 0; k < 6; ++k) put(a, t, a.off_fa + k, e, eta_a * S[k]);
    put(a, t, a.off_fa + 6, e, eta_a > 0.0 ? 1.0 / (2.0 * eta_a * V0) : 0.0);
  }
  if (a.off_fb >= 0) {
    double S[6] = {0, 0, 0, 0, 0, 0};
    if (eta_b > 0.0) {
      double d[3] = {a.bdir[3 * (size_t)e], a.bdir[3 * (size_t)e + 1], a.bdir[3 * (size_t)e + 2]};
      const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int j = 0; j < 3; ++j) d[j] /= n;
      fibre_tensor(Ji, d, 2.0 * V0, S);
    }
    for (int k = 0; k < 6; ++k) put(a, t, a.off_fb + k, e, eta_b * S[k]);
    put(a, t, a.off_fb + 6, e, eta_b > 0.0 ? 1.0 / (2.0 * eta_b * V0) : 0.0);
  }
  if (a.off_mr >= 0) {
    const double c10 = 0.5 * mu;
    put(a, t, a.off_mr, e, c01 / (2.0 * c10 * c10 * V0));
  }
  // 0B = 0J^-1 H_xi and sum of squares
  double B0[3][8];
  double sumB2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int b = 0; b < ne; ++b) {
      B0[i][b] = Ji[i][0] * Hx[0][b] + Ji[i][1] * Hx[1][b] + Ji[i][2] * Hx[2][b];
      sumB2 += B0[i][b] * B0[i][b];
    }
  const double mu_eff = mu + 2.0 * c01;
  const double Mw = kappa + 4.0 / 3.0 * mu_eff + 16.0 / 9.0 * (eta_a + eta_b);
  double w2 = ne * (Mw / rho) * sumB2;
  if (ne == 8) {
    double cq[4][3];
    for (int q = 0; q < 4; ++q)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int b = 0; b < 8; ++b) s += H8D[q][b] * Xe[b][j];
        cq[q][j] = s;
        if (!a.geometric) put(a, t, a.off_hg + 3 * q + j, e, s);
      }
    const double khg = a.hg_coeff * (kappa + 4.0 / 3.0 * mu) * V0 * sumB2 / 8.0;
    put(a, t, a.off_hg + (a.geometric ? 0 : 12), e, khg);
    double gam[4][8];
    for (int q = 0; q < 4; ++q)
      for (int b = 0; b < 8; ++b)
        gam[q][b] = H8D[q][b] - (cq[q][0] * B0[0][b] + cq[q][1] * B0[1][b] + cq[q][2] * B0[2][b]);
    double lmax = 0.0;
    for (int q = 0; q < 4; ++q) {
      double row = 0.0;
      for (int p = 0; p < 4; ++p) {
        double g = 0.0;
        for (int b = 0; b < 8; ++b) g += gam[q][b] * gam[p][b];
        row += fabs(g);
      }
      lmax = row > lmax ? row : lmax;
    }
    w2 += ne * khg * lmax / (rho * V0);
  }
  a.dt_elem[e] = 2.0 / sqrt(w2);
  a.elem_mass[e] = rho * V0 / ne;
}

// lumped mass m_i = sum over the node's slots of rho 0V / n_e (FP64, fixed order),
// then the update coefficient a_i = 2 dt^2 / ((2 + alpha dt) m_i) (Eq. 13)
__global__ void node_mass_kernel(const int* __restrict__ sell, const int* __restrict__ chunk_ptr,
                                 const double* __restrict__ elem_mass, int E_pad, int N, double dt0,
                                 const double* __restrict__ dt_node, double alpha,
                                 const int* __restrict__ bc_index, double* mass_out, float4* U,
                                 float4* V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int chunk = i / SELL_C, lane = i % SELL_C;
  double m = 0.0;
  for (int p = chunk_ptr[chunk] + lane; p < chunk_ptr[chunk + 1]; p += SELL_C) {
    const int s = sell[p];
    if (s >= 0) m += elem_mass[s % E_pad];
  }
  mass_out[i] = m;
  const double dt = dt_node ? dt_node[i] : dt0;
  const double ai = m > 0.0 ? 2.0 * dt * dt / ((2.0 + alpha * dt) * m) : 0.0;
  U[i] = make_float4(0.f, 0.f, 0.f, (float)ai);
  V[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(bc_index[i]));
}

// reads every 16-byte word of a buffer (evicting what the L2 cache held); the
// store never happens for a buffer that was zero-filled, it keeps the loads live
__global__ void read_sweep_kernel(const uint4* __restrict__ p, long long n, unsigned int* sink) {
  unsigned int acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint4 v = __ldcg(p + i);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x9e3779b9u) *sink = acc;
}

__global__ void min_reduce_kernel(const double* __restrict__ v, int n, double* out) {
  __shared__ double sm[256];
  double m = DBL_MAX;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += blockDim.x * gridDim.x)
    m = v[k] < m ? v[k] : m;
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o && sm[threadIdx.x + o] < sm[threadIdx.x]) sm[threadIdx.x] = sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

__global__ void to_caller_order_kernel(const float4* __restrict__ U, const int* __restrict__ perm,
                                       int N, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // caller node id
  if (i >= N) return;
  const float4 u = U[perm[i]];
  out[3 * (size_t)i] = u.x;
  out[3 * (size_t)i + 1] = u.y;
  out[3 * (size_t)i + 2] = u.z;
}

// U (+ compensated low part) in caller order as doubles, the layout of the
// host call's output
// FP64 displacements in caller order.  The block's 3 x 256 values go through
// shared memory so that the stores to `out` (device memory, or a page-locked
// host buffer written over the host link) are contiguous per warp.
constexpr int kOrderThreads = 256;
__global__ void __launch_bounds__(kOrderThreads) to_caller_order_f64_kernel(const float4* __restrict__ U,
                                                                           const float4* __restrict__ Ulo,
                                                                           const int* __restrict__ perm, int N,
                                                                           double* out, const DevState* st,
                                                                           DevState* st_out) {
  // launched behind the node update with a programmatic dependency: U only
  // after that kernel has completed (at once for an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ __align__(16) double sv[3 * kOrderThreads];
  if (st_out && blockIdx.x == 0 && threadIdx.x == 0) *st_out = *st;
  const int i0 = blockIdx.x * kOrderThreads;
  const int i = i0 + threadIdx.x;  // caller node id
  if (i < N) {
    const int v = perm[i];
    const float4 u = U[v];
    double x = u.x, y = u.y, z = u.z;
    if (Ulo) {
      const float4 l = Ulo[v];
      x += l.x;
      y += l.y;
      z += l.z;
    }
    sv[3 * threadIdx.x] = x;
    sv[3 * threadIdx.x + 1] = y;
    sv[3 * threadIdx.x + 2] = z;
  }
  __syncthreads();
  const int n = 3 * min(kOrderThreads, N - i0);
  double* o = out + 3 * (size_t)i0;
  if ((reinterpret_cast<uintptr_t>(o) & 15) == 0) {  // 16-byte stores (pairs of values)
    for (int q = threadIdx.x; q < n / 2; q += kOrderThreads)
      reinterpret_cast<double2*>(o)[q] = reinterpret_cast<const double2*>(sv)[q];
    if ((n & 1) && threadIdx.x == 0) o[n - 1] = sv[n - 1];
  } else {
    for (int q = threadIdx.x; q < n; q += kOrderThreads) o[q] = sv[q];
  }
}

// FP32 displacements (high + low part in the compensated mode, rounded once)
// in caller order, staged through shared memory like the FP64 kernel above.
__global__ void __launch_bounds__(kOrderThreads) to_caller_order_f32_kernel(const float4* __restrict__ U,
                                                                           const float4* __restrict__ Ulo,
                                                                           const int* __restrict__ perm, int N,
                                                                           float* out, const DevState* st,
                                                                           DevState* st_out) {
  // launched behind the node update with a programmatic dependency: U only
  // after that kernel has completed (at once for an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ __align__(16) float sv[3 * kOrderThreads];
  if (st_out && blockIdx.x == 0 && threadIdx.x == 0) *st_out = *st;
  const int i0 = blockIdx.x * kOrderThreads;
  const int i = i0 + threadIdx.x;  // caller node id
  if (i < N) {
    const int v = perm[i];
    float4 u = U[v];
    if (Ulo) {
      const float4 l = Ulo[v];
      u.x += l.x;
      u.y += l.y;
      u.z += l.z;
    }
    sv[3 * threadIdx.x] = u.x;
    sv[3 * threadIdx.x + 1] = u.y;
    sv[3 * threadIdx.x + 2] = u.z;
  }
  __syncthreads();
  const int n = 3 * min(kOrderThreads, N - i0);
  float* o = out + 3 * (size_t)i0;
  if ((reinterpret_cast<uintptr_t>(o) & 15) == 0) {  // 16-byte stores (quads of values)
    for (int q = threadIdx.x; q < n / 4; q += kOrderThreads)
      reinterpret_cast<float4*>(o)[q] = reinterpret_cast<const float4*>(sv)[q];
    for (int q = (n / 4) * 4 + threadIdx.x; q < n; q += kOrderThreads) o[q] = sv[q];
  } else {
    for (int q = threadIdx.x; q < n; q += kOrderThreads) o[q] = sv[q];
  }
}

__global__ void copy_state_kernel(const DevState* st, DevState* st_out) { *st_out = *st; }

__global__ void from_caller_order_kernel(const float* __restrict__ src, const int* __restrict__ perm, int N,
                                         float4* U, float4* V, float4* Ulo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // caller node id
  if (i >= N) return;
  const int v = perm[i];
  const float4 u = U[v];
  U[v] = make_float4(src[3 * (size_t)i], src[3 * (size_t)i + 1], src[3 * (size_t)i + 2], u.w);
  const float4 d = V[v];
  V[v] = make_float4(0.f, 0.f, 0.f, d.w);
  if (Ulo) Ulo[v] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// one step's prescribed targets (Sec. 5.1, Sec. 6) into the per-node table:
// entry k of the caller's FP64 array goes to float index flat[k] of the table
// (4 floats per prescribed node: x, y, z targets and the component mask)
__global__ void bc_targets_kernel(const double* __restrict__ target, const int* __restrict__ flat, int n,
                                  float* __restrict__ table, int* bad_flags) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    const double v = target[k];
    if (isfinite(v))
      table[__ldg(flat + k)] = (float)v;
    else if (bad_flags)  // a non-finite target keeps the previous one
      atomicOr(bad_flags, ERR_BAD_TARGET);
  }
}

}  // namespace

cudaError_t launch_from_caller_order(const float* src, const int* node_new_of_old, int N, float4* U,
                                     float4* V, float4* Ulo, cudaStream_t s) {
  const int t = 256;
  from_caller_order_kernel<<<(N + t - 1) / t, t, 0, s>>>(src, node_new_of_old, N, U, V, Ulo);
  return cudaGetLastError();
}

cudaError_t launch_precompute_elements(const PreArgs& a, cudaStream_t s) {
  const int t = 128;
  precompute_elements_kernel<<<(a.E + t - 1) / t, t, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_node_mass(const int* sell, const int* chunk_ptr, const double* elem_mass,
                             int E_pad, int N, double dt, const double* dt_node, double alpha,
                             const int* bc_index, double* mass_out, float4* U, float4* V,
                             cudaStream_t s) {
  const int t = 256;
  node_mass_kernel<<<(N + t - 1) / t, t, 0, s>>>(sell, chunk_ptr, elem_mass, E_pad, N, dt, dt_node,
                                                 alpha, bc_index, mass_out, U, V);
  return cudaGetLastError();
}

// out must hold 256 doubles; the host takes the min of those
cudaError_t launch_l2_flush(void* buf, size_t bytes, cudaStream_t s) {
  // write the first half, then read the second: the cache ends up holding clean
  // lines of a buffer no kernel of the step touches
  const size_t half = bytes / 2 / 16 * 16;
  cudaError_t e = cudaMemsetAsync(buf, 0, half, s);
  if (e != cudaSuccess) return e;
  char* r = static_cast<char*>(buf) + half;
  read_sweep_kernel<<<1216, 256, 0, s>>>(reinterpret_cast<const uint4*>(r), (long long)(half / 16),
                                        reinterpret_cast<unsigned int*>(buf));
  return cudaGetLastError();
}

cudaError_t launch_min_reduce(const double* v, int n, double* out, cudaStream_t s) {
  min_reduce_kernel<<<256, 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_to_caller_order(const float4* U, const int* node_new_of_old, int N, float* out,
                                   cudaStream_t s) {
  const int t = 256;
  to_caller_order_kernel<<<(N + t - 1) / t, t, 0, s>>>(U, node_new_of_old, N, out);
  return cudaGetLastError();
}

cudaError_t launch_to_caller_order_f64(const float4* U, const float4* Ulo, const int* node_new_of_old, int N,
                                       double* out, cudaStream_t s, const DevState* st, DevState* st_out) {
  const int t = kOrderThreads;
  return launch_pdl(to_caller_order_f64_kernel, dim3((N + t - 1) / t), dim3(t), 0, s, U, Ulo, node_new_of_old, N,
                    out, st, st_out);
}

cudaError_t launch_copy_state(const DevState* st, DevState* st_out, cudaStream_t s) {
  copy_state_kernel<<<1, 1, 0, s>>>(st, st_out);
  return cudaGetLastError();
}

cudaError_t launch_to_caller_order_f32(const float4* U, const float4* Ulo, const int* node_new_of_old, int N,
                                       float* out, cudaStream_t s, const DevState* st, DevState* st_out) {
  const int t = kOrderThreads;
  return launch_pdl(to_caller_order_f32_kernel, dim3((N + t - 1) / t), dim3(t), 0, s, U, Ulo, node_new_of_old, N,
                    out, st, st_out);
}

cudaError_t launch_bc_targets(const double* target, const int* flat, int n, float4* table, cudaStream_t s,
                              int* bad_flags) {
  if (n <= 0) return cudaSuccess;
  bc_targets_kernel<<<(n + 255) / 256, 256, 0, s>>>(target, flat, n, reinterpret_cast<float*>(table), bad_flags);
  return cudaGetLastError();
}

}  // namespace dj
