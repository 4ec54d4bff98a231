// Allocation-free residual norms.
//
// Some callers cannot allocate device memory at the point where they need the
// relaxation residual: code running inside another framework's memory pool,
// real-time loops that must not call into the allocator, or plugins that only
// receive buffers from a host application.  dj_residual_norms_static computes
// the same two FP64 sums as the residual reduction of dj_relax_to_tol (sum of
// squared nodal forces over free and over prescribed DOFs) from buffers the
// caller already owns; its block partial sums live in a fixed, file-scope
// device array instead of memory allocated per call or per mesh.
//
// Scratch: kMaxBlocks double2 = 1 MiB in the library's device image, held on
// every GPU that loads the library until the process exits.  One block of 256
// threads reduces 256 nodes, so n_nodes is limited to kMaxBlocks * 256.
#include <cuda_runtime.h>

#include <mutex>

#include "dj_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

// partial sums (free, prescribed) of every block of the last call
static __device__ __align__(256) double2 g_resid_scratch[kMaxBlocks];

// host-side device address of g_resid_scratch, looked up once per device
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__global__ void __launch_bounds__(kThreads) norms_partial_kernel(const float* __restrict__ F,
                                                                 const unsigned char* __restrict__ pres,
                                                                 long long n_nodes, double2* scratch) {
  const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (i < n_nodes) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double f = F[3 * i + q];
      if (pres[3 * i + q]) den += f * f;
      else num += f * f;
    }
  }
  __shared__ double sn[kThreads], sd[kThreads];
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sn[threadIdx.x] += sn[threadIdx.x + o];
      sd[threadIdx.x] += sd[threadIdx.x + o];
    }
    __syncthreads();
  }
  // every block of this call overwrites its own slot: nothing needs clearing
  if (threadIdx.x == 0) scratch[blockIdx.x] = make_double2(sn[0], sd[0]);
}

__global__ void __launch_bounds__(kThreads) norms_final_kernel(const double2* __restrict__ scratch, int n_blocks,
                                                               double* out) {
  __shared__ double sn[kThreads], sd[kThreads];
  double num = 0.0, den = 0.0;
  for (int b = threadIdx.x; b < n_blocks; b += kThreads) {
    num += scratch[b].x;
    den += scratch[b].y;
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sn[threadIdx.x] += sn[threadIdx.x + o];
      sd[threadIdx.x] += sd[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sn[0];
    out[1] = sd[0];
  }
}

}  // namespace

extern "C" dj_status dj_residual_norms_static(const float* d_F, const unsigned char* d_prescribed,
                                              long long n_nodes, double* d_out, void* stream) {
  if (!d_F || !d_prescribed || !d_out || n_nodes <= 0) return DJ_ERR_INVALID_ARG;
  if (n_nodes > (long long)kMaxBlocks * kThreads) return DJ_ERR_UNSUPPORTED;  // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DJ_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_resid_scratch) != cudaSuccess || !p) return DJ_ERR_CUDA;
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  const int n_blocks = (int)((n_nodes + kThreads - 1) / kThreads);
  cudaStream_t s = (cudaStream_t)stream;
  norms_partial_kernel<<<n_blocks, kThreads, 0, s>>>(d_F, d_prescribed, n_nodes, (double2*)scratch);
  if (cudaGetLastError() != cudaSuccess) return DJ_ERR_CUDA;
  norms_final_kernel<<<1, kThreads, 0, s>>>((const double2*)scratch, n_blocks, d_out);
  if (cudaGetLastError() != cudaSuccess) return DJ_ERR_CUDA;
  return DJ_OK;
}
