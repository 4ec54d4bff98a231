// Average nodal pressure for linear tetrahedra (Sec. 7 names it as the remedy
// for volumetric locking): the two passes that run before the element-force
// kernel of a step.
//
//   anp_volume_kernel     one block per tile: each element's volume change
//                         dV_e = (det tJ - det 0J) / 6, a quarter to each of its
//                         nodes, summed per tile node in the tile reduction's
//                         fixed order into one partial per (tile, node).
//                         det tJ - det 0J comes from the exact expansion
//                           det(A + B) - det A = tr(adj(A) B) + tr(A adj(B)) + det B
//                         (A = 0J from the tile-local coordinates, B = H_xi u),
//                         so it does not cancel against det 0J.
//   anp_pressure_kernel   one thread per node: p_i = kappa_i / V0_i * sum of the
//                         node's partials (node-major, ascending tile), i.e.
//                         kappa_i (J_i - 1) with J_i = V_i / V0_i.
//
// The element-force kernel then averages p over the element's nodes and uses
// it in place of kappa (J - 1) (ElemConsts::pv).
#include <cuda_runtime.h>

#include "dj_elem.cuh"
#include "dj_internal.h"

namespace dj {
namespace {

using namespace elem;

constexpr int kAnpMaxThreads = 256;

// sum per tile node of the scalar records sv (record a T + e at byte offset
// li[p] of the float4 record layout, hence index li[p] / 16), in the list
// order, G lanes per node combined by an xor butterfly (as reduce_tile)
template <int G>
__device__ __forceinline__ void reduce_tile_scalar_g(const float* sv, const unsigned short* li,
                                                     const unsigned short* lp, int n_t, int tid, int T,
                                                     float* out, const int* pdst) {
  const int sub = tid % G, per_pass = T / G;
  for (int q0 = 0; q0 < n_t; q0 += per_pass) {
    const int q = q0 + tid / G;
    float v = 0.f;
    if (q < n_t) {
      const int p1 = lp[q + 1];
      for (int p = lp[q] + sub; p < p1; p += G) v += sv[li[p] >> 4];
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (q < n_t && sub == 0) out[__ldg(pdst + q)] = v;
  }
}

template <bool CMP>
__global__ void __launch_bounds__(kAnpMaxThreads) anp_volume_kernel(TileArgs t, const float4* __restrict__ U,
                                                                    const float4* __restrict__ Ulo, int E,
                                                                    float* __restrict__ vparts) {
  extern __shared__ float4 sm[];
  const int tile = blockIdx.x, tid = threadIdx.x, T = t.T, cap = t.cap;
  float4* su = sm;
  float4* sl = sm + cap;
  float4* sx = sm + (CMP ? 2 : 1) * cap;
  float* sv = reinterpret_cast<float*>(sx + cap);  // 4 T records
  // the tile's slot lists, staged with the nodes (16-byte loads)
  unsigned short* sidx = reinterpret_cast<unsigned short*>(sv + 4 * T);  // 4 T local slot ids
  unsigned short* sptr = sidx + 4 * T;                                   // cap + 8 list offsets
  {
    const uint4* gi = reinterpret_cast<const uint4*>(t.lidx + (size_t)tile * T * 4);
    const uint4* gp = reinterpret_cast<const uint4*>(t.lptr + (size_t)tile * (cap + 8));
    uint4* di = reinterpret_cast<uint4*>(sidx);
    uint4* dp = reinterpret_cast<uint4*>(sptr);
    const int ni = T / 2, np = (cap + 8) / 8;  // 4 T and cap + 8 uint16 values
    for (int q = tid; q < ni + np; q += T) {
      if (q < ni) di[q] = __ldg(gi + q);
      else dp[q - ni] = __ldg(gp + (q - ni));
    }
  }
  const int n_t = __ldg(t.tile_ptr + tile + 1) - __ldg(t.tile_ptr + tile);
  for (int q = tid; q < n_t; q += T) {
    const int gid = __ldg(t.tnodes + (size_t)tile * cap + q);
    sx[q] = __ldg(t.xloc + (size_t)tile * cap + q);
    su[q] = __ldg(U + gid);
    if (CMP) sl[q] = __ldg(Ulo + gid);
  }
  __syncthreads();
  const int e = tile * T + tid;
  float v = 0.f;
  if (e < E) {
    const ushort4 c = __ldg(reinterpret_cast<const ushort4*>(t.lconn) + e);
    const unsigned lc[4] = {c.x, c.y, c.z, c.w};
    const float4 x0 = at16(sx, lc[0]);
    M3 A, B;
    float4 h[4], l[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      h[b] = at16(su, lc[b]);
      l[b] = CMP ? at16(sl, lc[b]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float d[4][3];
    node_deltas<4, CMP>(h, l, d);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float4 xr = at16(sx, lc[r + 1]);
      A.m[r][0] = xr.x - x0.x;
      A.m[r][1] = xr.y - x0.y;
      A.m[r][2] = xr.z - x0.z;
      B.m[r][0] = d[r + 1][0];
      B.m[r][1] = d[r + 1][1];
      B.m[r][2] = d[r + 1][2];
    }
    const M3 aA = adj3(A), aB = adj3(B);
    float dD = det3(B);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) dD = fmaf(aA.m[i][j], B.m[j][i], fmaf(A.m[i][j], aB.m[j][i], dD));
    v = dD * (1.f / 24.f);  // a quarter of (det tJ - det 0J) / 6
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) sv[b * T + tid] = v;
  __syncthreads();
  const unsigned short* li = sidx;
  const unsigned short* lp = sptr;
  const int* pd = t.pdst + (size_t)tile * cap;
  if (8 * n_t <= T) reduce_tile_scalar_g<8>(sv, li, lp, n_t, tid, T, vparts, pd);
  else if (4 * n_t <= T) reduce_tile_scalar_g<4>(sv, li, lp, n_t, tid, T, vparts, pd);
  else if (2 * n_t <= T) reduce_tile_scalar_g<2>(sv, li, lp, n_t, tid, T, vparts, pd);
  else reduce_tile_scalar_g<1>(sv, li, lp, n_t, tid, T, vparts, pd);
}

__global__ void anp_pressure_kernel(const int* __restrict__ node_ptr, const float* __restrict__ vparts,
                                    const float* __restrict__ c1, float* __restrict__ pres, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // the node's run in ascending tile order; the first kBatch loads are issued
  // together, then added in that order
  constexpr int kBatch = 4;
  const int p0 = __ldg(node_ptr + i), p1 = __ldg(node_ptr + i + 1);
  const float c = __ldg(c1 + i);
  float v[kBatch];
#pragma unroll
  for (int k = 0; k < kBatch; ++k)
    if (p0 + k < p1) v[k] = __ldg(vparts + p0 + k);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kBatch; ++k)
    if (p0 + k < p1) s += v[k];
  for (int p = p0 + kBatch; p < p1; ++p) s += __ldg(vparts + p);
  pres[i] = c * s;
}

}  // namespace

size_t anp_volume_smem(int cmp, const TileArgs& t) {
  return (size_t)((cmp ? 3 : 2) * t.cap) * sizeof(float4) + (size_t)4 * t.T * sizeof(float) +
         (size_t)(4 * t.T + t.cap + 8) * sizeof(unsigned short);
}

cudaError_t launch_anp(int cmp, const TileArgs& t, const int* node_ptr, const float4* U, const float4* Ulo, int E,
                       int N, float* vparts, const float* c1, float* pres, cudaStream_t s) {
  if (t.T > kAnpMaxThreads) return cudaErrorInvalidValue;
  const size_t smem = anp_volume_smem(cmp, t);
  if (smem > 48 * 1024) {  // tiles with many distinct nodes: opt in to more shared memory
    cudaError_t e = cmp ? cudaFuncSetAttribute(anp_volume_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem)
                        : cudaFuncSetAttribute(anp_volume_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (cmp)
    anp_volume_kernel<true><<<t.n_tiles, t.T, smem, s>>>(t, U, Ulo, E, vparts);
  else
    anp_volume_kernel<false><<<t.n_tiles, t.T, smem, s>>>(t, U, Ulo, E, vparts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  anp_pressure_kernel<<<(N + 255) / 256, 256, 0, s>>>(node_ptr, vparts, c1, pres, N);
  return cudaGetLastError();
}

}  // namespace dj
