// BF16 products on the fifth-generation tensor cores (tcgen05) for the BF16
// variant of the warm-start MLP (the paper has no counterpart; it names
// learning methods only as future work, Sec. 8).
//
//   C = alpha op(A) op(B) + beta C,  A(i, k) = A[i sar + k sac], B(k, j) = B[k sbr + j sbc]
//
// with FP32 operands in global memory (any strides, so the MLP's transposed
// products need no copies), rounded to bfloat16 while they are staged in
// shared memory, and FP32 accumulation in tensor memory.  One CTA of four
// warps computes a 128 x 64 tile of C: per 64-wide slab of K the threads
// stage A (128 x 64) and B (64 x 64) in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices, K-adjacent core matrices 128 bytes
// apart, row groups 1024 bytes apart), one thread issues four
// tcgen05.mma.kind::f16 (M = 128, N = 64, K = 16) and commits them to an
// mbarrier; after the last slab every warp reads its 32 rows of the
// accumulator with tcgen05.ld and applies alpha / beta.  Waits are bounded:
// a wait that gives up sets a device flag (read by gemm_tc_timed_out), the
// CTA skips its epilogue and still frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dj_internal.h"

namespace dj {
namespace {

constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr long long kWaitPolls = 1LL << 22;

__device__ int g_tc_timeout;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (row
// group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// element (row r, k) of a staged tile: core matrix (r / 8, k / 8), 8 values per row
__device__ __forceinline__ int staged(int r, int k) {
  return ((r >> 3) * (kBK / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__global__ void __launch_bounds__(128) gemm_bf16_tc_kernel(int M, int N, int K, float alpha,
                                                            const float* __restrict__ A, long long sar,
                                                            long long sac, const float* __restrict__ B,
                                                            long long sbr, long long sbc, float beta,
                                                            float* __restrict__ C, long long ldc) {
  __shared__ __align__(1024) __nv_bfloat16 sA[kBM * kBK];
  __shared__ __align__(1024) __nv_bfloat16 sB[kBN * kBK];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // instruction descriptor: D FP32, A and B BF16, both K-major, N / 8, M / 16
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                             ((uint32_t)(kBM >> 4) << 24);
  constexpr uint32_t lbo = 128, sbo = (kBK / 8) * 128;
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K; k0 += kBK) {
    for (int q = tid; q < kBM * kBK; q += 128) {
      const int r = q / kBK, k = q % kBK, gi = m0 + r, gk = k0 + k;
      sA[staged(r, k)] = __float2bfloat16_rn((gi < M && gk < K) ? A[gi * sar + gk * sac] : 0.f);
    }
    for (int q = tid; q < kBN * kBK; q += 128) {
      const int r = q / kBK, k = q % kBK, gj = n0 + r, gk = k0 + k;
      sB[staged(r, k)] = __float2bfloat16_rn((gj < N && gk < K) ? B[gk * sbr + gj * sbc] : 0.f);
    }
    // the staged operands are read by the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t da = smem_desc(saddr(sA) + kk * 256, lbo, sbo);
        const uint64_t db = smem_desc(saddr(sB) + kk * 256, lbo, sbo);
        const uint32_t accumulate = (k0 > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&bar))
                   : "memory");
    }
    uint32_t done = 0;
    for (long long it = 0; it < kWaitPolls && !done; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(saddr(&bar)), "r"(phase)
          : "memory");
      if (!done && it > 64) __nanosleep(32);
    }
    if (__syncthreads_or(!done)) {
      ok = false;
      if (tid == 0) atomicExch(&g_tc_timeout, 1);
      break;
    }
    phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;  // accumulator lane = row of the tile
#pragma unroll
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < N) {
            float* c = C + row * ldc + col;
            const float x = alpha * __uint_as_float(v[j]);
            *c = beta == 0.f ? x : x + beta * *c;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN));
}

}  // namespace

cudaError_t gemm_bf16_tc(int M, int N, int K, float alpha, const float* A, long long sar, long long sac,
                         const float* B, long long sbr, long long sbc, float beta, float* C, long long ldc,
                         cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
  gemm_bf16_tc_kernel<<<grid, 128, 0, s>>>(M, N, K, alpha, A, sar, sac, B, sbr, sbc, beta, C, ldc);
  return cudaGetLastError();
}

bool gemm_tc_timed_out() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int)) != cudaSuccess) return true;
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int));
  }
  return v != 0;
}

}  // namespace dj
