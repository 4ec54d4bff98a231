// Persistent element-force kernel with bulk asynchronous copies (TMA) for sm_103a.
//
// Each block walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The
// per-tile segments (tile-major element table, tile-local coordinates, local
// connectivity, local slot index, node list, partial destinations, node
// offsets; see TileArgs) are
// copied with cp.async.bulk into one of two shared-memory stages, two tiles
// ahead; an mbarrier per stage counts the arriving bytes.  A tile's stage
// carries the node list of the block's next tile, so the nodal values of the
// next tile are gathered with cp.async while the current tile's element forces
// are computed and reduced.  Every wait is bounded: on timeout the kernel
// records ERR_TIMEOUT, lets the copies in flight land (bounded) and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dj_elem.cuh"
#include "dj_internal.h"

namespace dj {
namespace {

using namespace elem;

constexpr long long kWaitLimit = 1LL << 22;  // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for the completion of phase `parity`; true if it completed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <int NE>
struct StageLayout {
  uint32_t xloc, tab, lconn, lidx, tnodes, pdst, lptr, bytes;  // byte offsets inside a stage
  __device__ __host__ StageLayout(const TileArgs& t) {
    xloc = 0;  // tile-local reference coordinates (geometric table)
    tab = xloc + (uint32_t)t.cap * 16;
    lconn = tab + (uint32_t)t.n_consts * t.T * 4;
    lidx = lconn + (uint32_t)t.T * NE * 2;
    tnodes = lidx + (uint32_t)t.T * NE * 2;
    pdst = tnodes + (uint32_t)t.cap * 4;
    lptr = pdst + (uint32_t)t.cap * 4;
    bytes = lptr + (uint32_t)(t.cap + 8) * 2;
  }
};

// issue the bulk copies of tile `tile` into `stage` (one thread)
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// the stage of `tile` carries the node list of `tnext` (the block's next tile)
template <int NE>
__device__ __forceinline__ void issue_tile(const ForceArgs& a, const TileArgs& t, const StageLayout<NE>& L,
                                           char* stage, uint64_t* bar, int tile, int tnext) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bar, L.bytes);
  bulk_copy(stage + L.xloc, t.xloc + (size_t)tile * t.cap, L.tab - L.xloc, bar);
  bulk_copy(stage + L.tab, a.consts + (size_t)tile * t.n_consts * t.T, L.lconn - L.tab, bar);
  bulk_copy(stage + L.lconn, t.lconn + (size_t)tile * t.T * NE, L.lidx - L.lconn, bar);
  bulk_copy(stage + L.lidx, t.lidx + (size_t)tile * t.T * NE, L.tnodes - L.lidx, bar);
  bulk_copy(stage + L.tnodes, t.tnodes + (size_t)(tnext < t.n_tiles ? tnext : tile) * t.cap, L.pdst - L.tnodes, bar);
  bulk_copy(stage + L.pdst, t.pdst + (size_t)tile * t.cap, L.lptr - L.pdst, bar);
  bulk_copy(stage + L.lptr, t.lptr + (size_t)tile * (t.cap + 8), L.bytes - L.lptr, bar);
}

// cp.async of one 16-byte record global -> shared (completion per thread)
__device__ __forceinline__ void async_copy16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void async_copy4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// stage the tile's nodal U (and low parts, and nodal pressures) into su / sl /
// sp with cp.async
template <bool CMP, bool ANP>
__device__ __forceinline__ void gather_nodes(const ForceArgs& a, const int* tnodes, int n_t, float4* su,
                                             float4* sl, float* sp, int tid, int T) {
  for (int q = tid; q < n_t; q += T) {
    const int gid = tnodes[q];
    async_copy16(su + q, a.U + gid);
    if (CMP) async_copy16(sl + q, a.Ulo + gid);
    if (ANP) async_copy4(sp + q, a.pres + gid);
  }
}

// Software pipeline per block, tiles blockIdx.x + k gridDim.x:
//   bulk copies of a tile's segments are issued two tiles ahead (stages 0/1),
//   the nodal gather of tile k+1 (cp.async, from the node list that came with
//   tile k's stage) is in flight while tile k's element forces are computed
//   and reduced, and a tile costs two block barriers.
template <int NE, bool FA, bool FB, bool MR, bool CMP, bool ANP>
__global__ void __launch_bounds__(256) force_tma_kernel(ForceArgs a, TileArgs t) {
  extern __shared__ __align__(128) char smem[];
  const StageLayout<NE> L(t);
  const int T = t.T, tid = threadIdx.x, cap = t.cap;
  const uint32_t stage_bytes = (L.bytes + 127) & ~127u;
  float4* sbase = reinterpret_cast<float4*>(smem + 2 * stage_bytes);
  float4* su2 = sbase;                              // [2][cap] staged U, by tile parity
  float4* sl2 = sbase + 2 * cap;                    // [2][cap] staged low parts (compensated)
  float4* sf4 = sbase + (CMP ? 4 : 2) * cap;        // NE T force records (slot a T + e)
  float* sp2 = reinterpret_cast<float*>(sf4 + NE * T);  // [2][cap] nodal pressures (ANP)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sp2 + (ANP ? 2 * cap : 0));
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int first = blockIdx.x, stride = gridDim.x;
  const bool second = first + stride < t.n_tiles;
  if (tid == 0 && first < t.n_tiles) {  // constant tables: before the wait
    // the first tile's own node list goes to the (still unused) record area
    mbar_expect_tx(&bars[0], (uint32_t)cap * 4);
    bulk_copy(sf4, t.tnodes + (size_t)first * cap, (uint32_t)cap * 4, &bars[0]);
    issue_tile<NE>(a, t, L, smem, &bars[0], first, first + stride);
    if (second) issue_tile<NE>(a, t, L, smem + stage_bytes, &bars[1], first + stride, first + 2 * stride);
  }
  const double tgt = targets_load(a);
  pdl_wait();  // U of the previous update; the partials are read by it
  pdl_launch_dependents();
  advance_clock(a);
  if (first >= t.n_tiles) {
    targets_store(a, tgt);
    return;
  }
  // prologue: the first tile's nodes
  {
    const bool ok = mbar_wait(&bars[0], 0u);
    if (__syncthreads_or(!ok)) {
      // both stages' copies may still be in flight: bounded waits for them
      if (tid == 0) {
        atomicOr(&a.st->err_flags, ERR_TIMEOUT);
        mbar_wait(&bars[0], 0u);
        if (second) mbar_wait(&bars[1], 0u);
      }
      return;
    }
    const int* tn = reinterpret_cast<const int*>(sf4);
    const int n0 = __ldg(t.tile_ptr + first + 1) - __ldg(t.tile_ptr + first);
    gather_nodes<CMP, ANP>(a, tn, n0, su2, sl2, sp2, tid, T);
    targets_store(a, tgt);  // the host read has landed by now
    async_wait_all();
    __syncthreads();
  }
  // node counts of the current and the next tile, carried from tile to tile;
  // the one after next is loaded a tile ahead of its use
  int n_cur = __ldg(t.tile_ptr + first + 1) - __ldg(t.tile_ptr + first);
  int n_nxt = second ? __ldg(t.tile_ptr + first + stride + 1) - __ldg(t.tile_ptr + first + stride) : 0;
  int i = 0;
  for (int tile = first; tile < t.n_tiles; tile += stride, ++i) {
    const int s = i & 1;
    const char* st = smem + s * stage_bytes;
    const float4* sx = reinterpret_cast<const float4*>(st + L.xloc);
    const float* tab = reinterpret_cast<const float*>(st + L.tab);
    const unsigned short* lconn = reinterpret_cast<const unsigned short*>(st + L.lconn);
    const unsigned short* lidx = reinterpret_cast<const unsigned short*>(st + L.lidx);
    const unsigned short* lptr = reinterpret_cast<const unsigned short*>(st + L.lptr);
    const int* pdst = reinterpret_cast<const int*>(st + L.pdst);
    const float4* su = su2 + s * cap;
    const float4* sl = sl2 + s * cap;
    const float* sp = sp2 + s * cap;
    const int n_t = n_cur;
    const int next = tile + stride;
    const bool has_next = next < t.n_tiles;
    const int after = next + stride;
    const int n_after = after < t.n_tiles ? __ldg(t.tile_ptr + after + 1) - __ldg(t.tile_ptr + after) : 0;
    // 0. the next tile's nodes: its list came with this tile's stage
    if (has_next) {
      const int* tn = reinterpret_cast<const int*>(st + L.tnodes);
      gather_nodes<CMP, ANP>(a, tn, n_nxt, su2 + (s ^ 1) * cap, sl2 + (s ^ 1) * cap, sp2 + (s ^ 1) * cap, tid, T);
    }
    // 1. element forces of this tile into shared memory
    const int e = tile * T + tid;
    if (e < a.E) {
      const auto ld = [&](int r) { return tab[r * T + tid]; };
      ElemConsts<FA, FB, MR, ANP> k;
      int lc[NE];  // the element's local connectivity: one 8- or 16-byte load
      if constexpr (NE == 4) {
        const ushort4 v = reinterpret_cast<const ushort4*>(lconn)[tid];
        lc[0] = v.x; lc[1] = v.y; lc[2] = v.z; lc[3] = v.w;
      } else {
        const uint4 v = reinterpret_cast<const uint4*>(lconn)[tid];
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          lc[2 * b] = (int)(w[b] & 0xffffu);
          lc[2 * b + 1] = (int)(w[b] >> 16);
        }
      }
      k.load_geometric(ld, a);
      if constexpr (ANP) {  // mean nodal pressure times 0V / det 0J = 1 / 6
        float ps = sp[lc[0] >> 4];
#pragma unroll
        for (int b = 1; b < NE; ++b) ps += sp[lc[b] >> 4];
        k.pv = ps * (1.f / 24.f);
      }
      bool inv;
      if constexpr (NE == 8) {
        HgConsts hg;
        hg.load_k(ld, a.off_hg);
        const auto ldn = [&](int b, float4& h, float4& l) {
          h = at16(su, lc[b]);
          l = CMP ? at16(sl, lc[b]) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        const auto ldx = [&](int b) { return at16(sx, lc[b]); };
        const auto out = [&](int b, float4 f) { sf4[b * T + tid] = f; };
        hex8_forces_stream<FA, FB, MR, CMP, true>(ldn, ldx, k, hg, out, inv);
      } else {
        const float4 x0 = at16(sx, lc[0]);
        float xd[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float4 xr = at16(sx, lc[r + 1]);
          xd[r][0] = xr.x - x0.x;
          xd[r][1] = xr.y - x0.y;
          xd[r][2] = xr.z - x0.z;
        }
        k.geometry(xd);
        float4 h[NE], l[NE];
#pragma unroll
        for (int b = 0; b < NE; ++b) {
          h[b] = at16(su, lc[b]);
          l[b] = CMP ? at16(sl, lc[b]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float d[NE][3];
        node_deltas<NE, CMP>(h, l, d);
        float f[NE][3];
        ElemExtra<NE> x;
        elem_forces<NE, FA, FB, MR, CMP>(d, k, x, f, inv);
#pragma unroll
        for (int b = 0; b < NE; ++b) sf4[b * T + tid] = make_float4(f[b][0], f[b][1], f[b][2], 0.f);
      }
      flag_inverted(a.st, e, inv);
    }
    // 2. the next tile's segments must have landed; barrier: records complete
    const bool ok = has_next ? mbar_wait(&bars[s ^ 1], (uint32_t)(((i + 1) >> 1) & 1)) : true;
    if (__syncthreads_or(!ok)) {
      // the next tile's gather and the copy that timed out are in flight:
      // let both land (bounded) before the block's shared memory is released
      async_wait_all();
      if (tid == 0) {
        atomicOr(&a.st->err_flags, ERR_TIMEOUT);
        mbar_wait(&bars[s ^ 1], (uint32_t)(((i + 1) >> 1) & 1));
      }
      return;
    }
    reduce_tile(sf4, lidx, lptr, n_t, tid, T, [&](int q, float4 f) { t.partials[pdst[q]] = f; });
    async_wait_all();
    // 4. barrier: stage s and the records are free, the next tile's nodes staged
    __syncthreads();
    if (tid == 0 && next + stride < t.n_tiles)
      issue_tile<NE>(a, t, L, smem + s * stage_bytes, &bars[s], next + stride, next + 2 * stride);
    n_cur = n_nxt;
    n_nxt = n_after;
  }
}

template <int NE, bool CMP, bool ANP>
size_t smem_bytes_t(const TileArgs& t) {
  const StageLayout<NE> L(t);
  const size_t stage = (L.bytes + 127) & ~size_t(127);
  return 2 * stage + (size_t)(CMP ? 4 : 2) * t.cap * sizeof(float4) + (size_t)NE * t.T * sizeof(float4) +
         (ANP ? 2 * (size_t)t.cap * sizeof(float) : 0) + 16;
}

template <int NE, bool FA, bool FB, bool MR, bool CMP, bool ANP>
cudaError_t launch_t(const ForceArgs& a, const TileArgs& t, int grid, cudaStream_t s) {
  const size_t smem = smem_bytes_t<NE, CMP, ANP>(t);
  return launch_pdl(force_tma_kernel<NE, FA, FB, MR, CMP, ANP>, dim3(grid), dim3(t.T), smem, s, a, t);
}

template <int NE, bool FA, bool FB, bool MR, bool CMP, bool ANP>
int occupancy_t(const TileArgs& t) {
  const size_t smem = smem_bytes_t<NE, CMP, ANP>(t);
  // allow the largest dynamic shared memory once, outside any stream capture
  if (cudaFuncSetAttribute(force_tma_kernel<NE, FA, FB, MR, CMP, ANP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, force_tma_kernel<NE, FA, FB, MR, CMP, ANP>, t.T, smem) !=
      cudaSuccess)
    return 0;
  return n;
}

template <int NE, bool CMP, bool ANP>
cudaError_t launch_v(int variant, const ForceArgs& a, const TileArgs& t, int grid, cudaStream_t s) {
  switch (variant) {
    case VAR_NH: return launch_t<NE, false, false, false, CMP, ANP>(a, t, grid, s);
    case VAR_TI: return launch_t<NE, true, false, false, CMP, ANP>(a, t, grid, s);
    case VAR_OT: return launch_t<NE, true, true, false, CMP, ANP>(a, t, grid, s);
    case VAR_MR: return launch_t<NE, false, false, true, CMP, ANP>(a, t, grid, s);
    default: return launch_t<NE, true, true, true, CMP, ANP>(a, t, grid, s);
  }
}

template <int NE, bool CMP, bool ANP>
int occupancy_v(int variant, const TileArgs& t) {
  switch (variant) {
    case VAR_NH: return occupancy_t<NE, false, false, false, CMP, ANP>(t);
    case VAR_TI: return occupancy_t<NE, true, false, false, CMP, ANP>(t);
    case VAR_OT: return occupancy_t<NE, true, true, false, CMP, ANP>(t);
    case VAR_MR: return occupancy_t<NE, false, false, true, CMP, ANP>(t);
    default: return occupancy_t<NE, true, true, true, CMP, ANP>(t);
  }
}

}  // namespace

// anp (average nodal pressure) is built for T4 only; H8 ignores it
size_t tma_smem_bytes(int elem_type, int cmp, int anp, const TileArgs& t) {
  if (elem_type == DJ_TET4) {
    if (anp) return cmp ? smem_bytes_t<4, true, true>(t) : smem_bytes_t<4, false, true>(t);
    return cmp ? smem_bytes_t<4, true, false>(t) : smem_bytes_t<4, false, false>(t);
  }
  return cmp ? smem_bytes_t<8, true, false>(t) : smem_bytes_t<8, false, false>(t);
}

int tma_blocks_per_sm(int elem_type, int variant, int cmp, int anp, const TileArgs& t) {
  if (elem_type == DJ_TET4) {
    if (anp) return cmp ? occupancy_v<4, true, true>(variant, t) : occupancy_v<4, false, true>(variant, t);
    return cmp ? occupancy_v<4, true, false>(variant, t) : occupancy_v<4, false, false>(variant, t);
  }
  return cmp ? occupancy_v<8, true, false>(variant, t) : occupancy_v<8, false, false>(variant, t);
}

cudaError_t launch_force_tma(int elem_type, int variant, int cmp, int anp, const ForceArgs& a, const TileArgs& t,
                             int grid, cudaStream_t s) {
  if (elem_type == DJ_TET4) {
    if (anp)
      return cmp ? launch_v<4, true, true>(variant, a, t, grid, s) : launch_v<4, false, true>(variant, a, t, grid, s);
    return cmp ? launch_v<4, true, false>(variant, a, t, grid, s) : launch_v<4, false, false>(variant, a, t, grid, s);
  }
  return cmp ? launch_v<8, true, false>(variant, a, t, grid, s) : launch_v<8, false, false>(variant, a, t, grid, s);
}

}  // namespace dj
