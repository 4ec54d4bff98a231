// DJ-TLED time-step kernels for sm_103a.
//
//  force_kernel<ELEM, FA, FB, MR>   one thread per element: Algorithm 1 runtime
//      steps 1-4 (tJ, J, g_hat, invariants, Table 3 force), written to the
//      element-force slots (slot = a * E_pad + e, so each store instruction of a
//      warp is one contiguous 512-byte run).
//  node_kernel<MODE, CMP, SELL>     one thread per node: deterministic gather of
//      the node's slots (sliced ELL, fixed order) or tile partials (node-major
//      runs, ascending tile), central-difference update
//      with mass-proportional damping (Eq. 13) and prescribed displacements;
//      optional FP64 residual partial sums for dynamic relaxation.
//
// FP32 arithmetic throughout the step.  The force is evaluated in this
// algebraically equivalent form of Table 3 (P = dPsi/dI1 I1m, adj = det(tJ) tJ^-1):
//
//   F = [ J^-2/3 tJ^T (P + psi_a Q_a + psi_b Q_b + MR term)
//         + ( -J^-2/3 (P:g + psi_a Q_a:g + psi_b Q_b:g) / 3 - MR vol term ) adj / det tJ
//         + kappa 0V (J - 1) r0 adj ] H_xi
//
// using  I1 = g_hat^T m1 = g:P / (mu 0V)  (m1 from I1m, Eq. 22/37),
//        I4 = g:Q_a / (2 eta_a 0V), psi_a = I4bar - 1, and
//        J tJ^-1 / det tJ ... = r0 adj  (Eq. 12).
#include <cuda_runtime.h>

#include "dj_elem.cuh"
#include "dj_internal.h"

namespace dj {

namespace {

using namespace elem;

// Element-slot assembly: one thread per element, forces to slot a * E_pad + e.
template <int NE, bool FA, bool FB, bool MR, bool CMP>
__global__ void __launch_bounds__(NE == 4 ? 256 : 128) force_slots_kernel(ForceArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = e < a.E;
  const int E_pad = a.E_pad;
  const float* __restrict__ c = a.consts;
  const auto ld = [&](int r) { return __ldcs(c + (size_t)r * E_pad + e); };
  ElemConsts<FA, FB, MR> k;
  int nid[NE];
  if (valid) {  // the table and the connectivity do not depend on the previous kernel
    k.load(ld, a);
    const int4 n0 = __ldcs(a.conn + (NE / 4) * (size_t)e);
    nid[0] = n0.x; nid[1] = n0.y; nid[2] = n0.z; nid[3] = n0.w;
    if constexpr (NE == 8) {
      const int4 n1 = __ldcs(a.conn + 2 * (size_t)e + 1);
      nid[4] = n1.x; nid[5] = n1.y; nid[6] = n1.z; nid[7] = n1.w;
    }
  }
  const double tgt = targets_load(a);
  pdl_wait();  // U of the previous update; the slots are read by it
  // the next update kernel may start now: what it reads before its own wait
  // (U, V) is final once the previous update has completed
  pdl_launch_dependents();
  advance_clock(a);
  targets_store(a, tgt);
  if (!valid) return;
  bool inv;
  if constexpr (NE == 8) {
    HgConsts hg;
    hg.load(ld, a.off_hg);
    const auto ldn = [&](int b, float4& h, float4& l) {
      h = __ldg(a.U + nid[b]);
      l = CMP ? __ldg(a.Ulo + nid[b]) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    const auto ldx = [&](int) { return make_float4(0.f, 0.f, 0.f, 0.f); };
    const auto out = [&](int b, float4 f) { a.slots[(size_t)b * E_pad + e] = f; };
    hex8_forces_stream<FA, FB, MR, CMP, false>(ldn, ldx, k, hg, out, inv);
  } else {
    float4 h[NE], l[NE];
#pragma unroll
    for (int b = 0; b < NE; ++b) {
      h[b] = __ldg(a.U + nid[b]);
      l[b] = CMP ? __ldg(a.Ulo + nid[b]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float d[NE][3];
    node_deltas<NE, CMP>(h, l, d);
    float f[NE][3];
    ElemExtra<NE> x;
    elem_forces<NE, FA, FB, MR, CMP>(d, k, x, f, inv);
#pragma unroll
    for (int b = 0; b < NE; ++b) a.slots[(size_t)b * E_pad + e] = make_float4(f[b][0], f[b][1], f[b][2], 0.f);
  }
  flag_inverted(a.st, e, inv);
}

// Tiled assembly: block = tile of T elements.  The tile's unique nodes are
// staged in shared memory, element forces go to shared memory (slot a * T + e),
// and each unique node sums its slots in the fixed order of the local index.
// T4 neo-Hookean / transversely isotropic FP32 variants are held to 40
// registers (3 blocks of 512 or 6 of 256 per SM): the kernel is latency-bound
// and the extra resident warps outweigh a few spilled words.
template <int NE, bool FA, bool FB, bool MR, bool CMP>
constexpr int tiles_min_blocks() { return (NE == 4 && !CMP && !FB && !MR) ? 3 : 1; }

// Shared memory of one tile (float4 units): staged U, (low parts), coordinates,
// the NE T records, then the uint16 slot ids and list offsets.
__host__ __device__ inline int tile_smem_f4(int NE, bool CMP, int T, int cap) {
  const int nstage = 2 + (CMP ? 1 : 0);
  return nstage * cap + NE * T + (2 * (NE * T + cap + 8) + 15) / 16;
}

// WARP: T = 32 and one warp per tile (a block holds blockDim / 32 tiles, each
// with its own shared-memory region); the tile's phases are separated by warp
// barriers instead of block barriers, so warps never wait for one another.
template <int NE, bool FA, bool FB, bool MR, bool CMP, bool WARP>
__global__ void __launch_bounds__(NE == 4 ? 512 : 256, (tiles_min_blocks<NE, FA, FB, MR, CMP>()))
    force_tiles_kernel(ForceArgs a, TileArgs t) {
  extern __shared__ float4 smem_all[];
  const int T = t.T;
  const int tile = WARP ? blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32 : blockIdx.x;
  const int tid = WARP ? threadIdx.x % 32 : threadIdx.x;
  if (WARP && tile >= t.n_tiles) {
    if (a.n_tgt) {  // this thread's share of the targets' copy
      const double tgt = targets_load(a);
      pdl_wait();
      targets_store(a, tgt);
    }
    return;
  }
  float4* smem4 = WARP ? smem_all + (threadIdx.x / 32) * tile_smem_f4(NE, CMP, T, t.cap) : smem_all;
  const auto tile_sync = [] {
    if (WARP) __syncwarp();
    else __syncthreads();
  };
  const int S = NE * T;  // slots per tile
  constexpr int NSTAGE = 2 + (CMP ? 1 : 0);  // U, (low parts), reference coordinates
  float4* su = smem4;                            // staged U (high part)
  float4* sl = smem4 + t.cap;                    // staged low part (compensated)
  float4* sx = smem4 + (NSTAGE - 1) * t.cap;     // staged tile-local reference coordinates
  float4* sf4 = smem4 + NSTAGE * t.cap;          // S force records (slot a T + e)
  // the tile's reduction lists, staged with the inputs so that their latency
  // overlaps the node gather instead of following the element math
  unsigned short* sidx = reinterpret_cast<unsigned short*>(sf4 + S);  // S local slot ids
  unsigned short* sptr = sidx + S;                                     // cap + 8 list offsets
  {
    const uint4* gi = reinterpret_cast<const uint4*>(t.lidx + (size_t)tile * S);
    const uint4* gp = reinterpret_cast<const uint4*>(t.lptr + (size_t)tile * (t.cap + 8));
    uint4* di = reinterpret_cast<uint4*>(sidx);
    uint4* dp = reinterpret_cast<uint4*>(sptr);
    const int ni = S / 8, np = (t.cap + 8) / 8;
    for (int q = tid; q < ni + np; q += T) {
      if (q < ni) di[q] = __ldcs(gi + q);
      else dp[q - ni] = __ldcs(gp + (q - ni));
    }
  }
  const int base = __ldg(t.tile_ptr + tile);
  const int n_t = __ldg(t.tile_ptr + tile + 1) - base;
  const int e = tile * T + tid;
  const bool valid = e < a.E;
  const float* __restrict__ c = a.consts;
  ElemConsts<FA, FB, MR> k;
  HgConsts hg;
  unsigned short lc[NE];
  if (valid) {
    // tile-major table: row r of element (tile, tid) at ((tile n_consts) + r) T + tid
    const float* ct = c + (size_t)tile * t.n_consts * T + tid;
    const auto ld = [&](int r) { return __ldcs(ct + (size_t)r * T); };
    k.load_geometric(ld, a);
    if constexpr (NE == 8) hg.load_k(ld, a.off_hg);
    if constexpr (NE == 4) {
      const ushort4 v = __ldcs(reinterpret_cast<const ushort4*>(t.lconn) + e);
      lc[0] = v.x; lc[1] = v.y; lc[2] = v.z; lc[3] = v.w;
    } else {
      const ushort4 v0 = __ldcs(reinterpret_cast<const ushort4*>(t.lconn) + 2 * (size_t)e);
      const ushort4 v1 = __ldcs(reinterpret_cast<const ushort4*>(t.lconn) + 2 * (size_t)e + 1);
      lc[0] = v0.x; lc[1] = v0.y; lc[2] = v0.z; lc[3] = v0.w;
      lc[4] = v1.x; lc[5] = v1.y; lc[6] = v1.z; lc[7] = v1.w;
    }
  }
  const double tgt = targets_load(a);
  pdl_wait();  // U of the previous update; the partials are read by it
  pdl_launch_dependents();  // see force_slots_kernel
  if (!WARP || threadIdx.x < 32) advance_clock(a);
  targets_store(a, tgt);
  for (int q = tid; q < n_t; q += T) {
    const int gid = __ldg(t.tnodes + (size_t)tile * t.cap + q);
    sx[q] = __ldcs(t.xloc + (size_t)tile * t.cap + q);
    su[q] = __ldg(a.U + gid);
    if (CMP) sl[q] = __ldg(a.Ulo + gid);
  }
  tile_sync();
  if (valid) {
    bool inv;
    if constexpr (NE == 8) {
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
      for (int i = 0; i < 3; ++i) {
        const float4 xi = at16(sx, lc[i + 1]);
        xd[i][0] = xi.x - x0.x;
        xd[i][1] = xi.y - x0.y;
        xd[i][2] = xi.z - x0.z;
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
  tile_sync();
  const unsigned short* lp = sptr;
  const unsigned short* li = sidx;
  const int* pd = t.pdst + (size_t)tile * t.cap;
  reduce_tile(sf4, li, lp, n_t, tid, T, [&](int q, float4 f) { t.partials[__ldcs(pd + q)] = f; });
}

// SELL: the slot assembly's sliced-ELL lists (a.node_ptr null), else the
// tiled assembly's node-major partials (compiled apart: the batched slot
// gather takes registers the partials' path does not need)
template <int MODE, bool CMP, bool SELL>
__global__ void __launch_bounds__(NODE_THREADS) node_kernel(NodeArgs a) {
  constexpr bool ADR = MODE == NODE_ADR || MODE == NODE_ADR_RQ;
  constexpr bool TGT = MODE == NODE_UPDATE_TGT;
  constexpr bool UPD = MODE == NODE_UPDATE || MODE == NODE_UPDATE_RESID || TGT || ADR;
  constexpr bool RESID = MODE == NODE_UPDATE_RESID || MODE == NODE_RESID_ONLY || MODE == NODE_ADR_RQ;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = i / SELL_C, lane = i % SELL_C;
  double num2 = 0.0, den2 = 0.0;
  double rq_df = 0.0, rq_m = 0.0, rq_d2 = 0.0, rq_max = 0.0;  // NODE_ADR_RQ sums
  // node state and offsets first: the force kernel before this one does not
  // write them (and launched this kernel only after the previous update had
  // completed), so they are loaded while it finishes
  float4 V = make_float4(0.f, 0.f, 0.f, 0.f), U = V, L = V;
  int beg = 0, end = 0;
  if (i < a.N) {
    V = a.V[i];
    if (UPD) U = a.U[i];
    if (CMP && UPD) L = a.Ulo[i];
    if (!SELL) {
      beg = __ldg(a.node_ptr + i);
      end = __ldg(a.node_ptr + i + 1);
    } else {  // the node's chunk of the sliced-ELL slot lists
      beg = __ldg(a.chunk_ptr + chunk);
      end = __ldg(a.chunk_ptr + chunk + 1);
    }
  }
  pdl_wait();  // the forces of this step; U and V are read by the previous force kernel
  // the next force kernel may start as these blocks retire: before its own wait
  // it reads only the mesh's constant tables (launching it earlier, while this
  // kernel's blocks are still arriving, lets it take their resources)
  pdl_launch_dependents();
  if (i < a.N) {
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (!SELL) {
      // node-major partials: one contiguous run per node, ascending tile.
      // The first kBatch loads are issued together (most nodes have no
      // more), the rest two at a time; all are added in the run's order
      constexpr int kBatch = 4;
      float4 f0[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (beg + k < end) f0[k] = __ldcs(a.slots + beg + k);
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (beg + k < end) {
          fx += f0[k].x;
          fy += f0[k].y;
          fz += f0[k].z;
        }
      for (int p = beg + kBatch; p < end; p += 2) {
        const float4 f = __ldcs(a.slots + p);
        const float4 g = p + 1 < end ? __ldcs(a.slots + p + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        fx += f.x;
        fy += f.y;
        fz += f.z;
        if (p + 1 < end) {
          fx += g.x;
          fy += g.y;
          fz += g.z;
        }
      }
    } else {
      // sliced ELL: the node's slot ids, kB at a time, then their slots,
      // loads issued together and added in the list's order (-1: padding)
      constexpr int kB = 4;
      for (int p0 = beg + lane; p0 < end; p0 += kB * SELL_C) {
        int sid[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) sid[k] = p0 + k * SELL_C < end ? __ldcs(a.sell + p0 + k * SELL_C) : -1;
        float4 f[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k)
          if (sid[k] >= 0) f[k] = __ldcs(a.slots + sid[k]);
#pragma unroll
        for (int k = 0; k < kB; ++k)
          if (sid[k] >= 0) {
            fx += f[k].x;
            fy += f[k].y;
            fz += f[k].z;
          }
      }
    }
    if (a.R) {
      const float4 r = __ldg(a.R + i);
      fx -= r.x;
      fy -= r.y;
      fz -= r.z;
    }
    // now f = F_int - R
    const int bc = __float_as_int(V.w);
    if (MODE == NODE_FORCE_ONLY || MODE == NODE_RESID_ONLY) {
      if (!isfinite(fx + fy + fz)) flag_nonfinite(a.st, i);
    }
    if (MODE == NODE_FORCE_ONLY) {
      a.fout[i] = make_float4(fx, fy, fz, 0.f);
    } else if (MODE == NODE_RESID_ONLY) {
      int mask = 0;
      if (bc >= 0) mask = __float_as_int(__ldg(a.bct + bc).w);
      const double f3[3] = {fx, fy, fz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (mask & (1 << q)) den2 += f3[q] * f3[q];
        else num2 += f3[q] * f3[q];
      }
    } else {
      // velocity form of the central difference: D^{n+1} = a (R - F) + (b - 1) D^n;
      // adaptive steps take b - 1 and the scale of a_i from the relaxation state
      const float ai = ADR ? U.w * a.adr->ai_scale : U.w;
      const float bm1 = ADR ? a.adr->bm1 : (a.bm1_node ? __ldg(a.bm1_node + i) : a.bm1);
      float dd[3] = {fmaf(-ai, fx, bm1 * V.x), fmaf(-ai, fy, bm1 * V.y), fmaf(-ai, fz, bm1 * V.z)};
      const float uh[3] = {U.x, U.y, U.z};
      float nh[3], nl[3] = {0.f, 0.f, 0.f}, ul[3] = {0.f, 0.f, 0.f};
      if (CMP) {
        ul[0] = L.x;
        ul[1] = L.y;
        ul[2] = L.z;
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (CMP) {
          // (hi, lo) + D with an error-free sum of the high parts
          const float s = uh[q] + dd[q];
          const float bb = s - uh[q];
          const float err = (uh[q] - (s - bb)) + (dd[q] - bb);
          const float lo = ul[q] + err;
          nh[q] = s + lo;
          nl[q] = lo - (nh[q] - s);
        } else {
          nh[q] = uh[q] + dd[q];
        }
      }
      int mask = 0;
      if (bc >= 0) {
        float tv[3];
        if (TGT) {
          // this step's targets (the device copy of the caller's array); the
          // node's table row takes them for later steps.  A non-finite entry
          // is not applied: the row's previous target stays and the step
          // records ERR_BAD_TARGET.
          const int4 en = __ldg(a.bc_entry + bc);
          mask = en.w;
          const int ek[3] = {en.x, en.y, en.z};
          double v[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) v[q] = ek[q] >= 0 ? a.tgt[ek[q]] : 0.0;  // loads issued together
          float4 row = a.bct[bc];
          float* rv[3] = {&row.x, &row.y, &row.z};
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            if (ek[q] >= 0) {
              if (isfinite(v[q])) *rv[q] = (float)v[q];
              else atomicOr(&a.st->err_flags, ERR_BAD_TARGET);
            }
            tv[q] = *rv[q];
          }
          const_cast<float4*>(a.bct)[bc] = row;
        } else {
          const float4 t = __ldg(a.bct + bc);
          mask = __float_as_int(t.w);
          tv[0] = t.x;
          tv[1] = t.y;
          tv[2] = t.z;
        }
        const float rs = a.st->ramp_s;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (mask & (1 << q)) {
            nh[q] = tv[q] * rs;
            nl[q] = 0.f;
            dd[q] = (nh[q] - uh[q]) - ul[q];
          }
      }
      // a non-finite element force reaches U^{n+1} of its nodes (NaN and Inf
      // propagate through the update), or the reaction of prescribed ones
      if (!isfinite(nh[0] + nh[1] + nh[2] + fx + fy + fz)) flag_nonfinite(a.st, i);
      a.U[i] = make_float4(nh[0], nh[1], nh[2], U.w);  // w keeps the precomputed a_i
      if (CMP) a.Ulo[i] = make_float4(nl[0], nl[1], nl[2], 0.f);
      a.V[i] = make_float4(dd[0], dd[1], dd[2], V.w);
      if (MODE == NODE_UPDATE_RESID || MODE == NODE_ADR_RQ) {
        const double f3[3] = {fx, fy, fz};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (mask & (1 << q)) den2 += f3[q] * f3[q];
          else num2 += f3[q] * f3[q];
        }
      }
      if (MODE == NODE_ADR_RQ) {
        // D = U^n - U^{n-k} and F(U^n) - F(U^{n-k}) against the previous
        // check's snapshot, over the free DOFs; the lumped mass enters as
        // 1 / a_i(alpha_0) (times kappa0 dt^2, applied once at the end).  Then
        // this check's U^n and F - R become the snapshot.
        const float4 fp = a.fout[i];
        const double4 us = a.usnap[i];
        const double un[3] = {(double)uh[0] + ul[0], (double)uh[1] + ul[1], (double)uh[2] + ul[2]};
        const double df[3] = {(double)fx - fp.x, (double)fy - fp.y, (double)fz - fp.z};
        const double d[3] = {un[0] - us.x, un[1] - us.y, un[2] - us.z};
        const double inv_a = U.w > 0.f ? 1.0 / (double)U.w : 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (!(mask & (1 << q))) {
            rq_df += d[q] * df[q];
            rq_m += d[q] * d[q] * inv_a;
            rq_d2 += d[q] * d[q];
            rq_max = fmax(rq_max, fabs(d[q]));
          }
        a.usnap[i] = make_double4(un[0], un[1], un[2], 0.0);
        a.fout[i] = make_float4(fx, fy, fz, 0.f);
      }
    }
  }
  if (RESID && a.node_resid) {
    if (i < a.N) a.node_resid[i] = make_double2(num2, den2);
    return;
  }
  if (RESID) {
    __shared__ double sn[NODE_THREADS / 32], sd[NODE_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num2 += __shfl_down_sync(0xffffffffu, num2, o);
      den2 += __shfl_down_sync(0xffffffffu, den2, o);
    }
    const int w = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0) {
      sn[w] = num2;
      sd[w] = den2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tn = 0.0, td = 0.0;
      for (int q = 0; q < NODE_THREADS / 32; ++q) {
        tn += sn[q];
        td += sd[q];
      }
      a.partials[blockIdx.x] = make_double2(tn, td);
    }
  }
  if (MODE == NODE_ADR_RQ) {
    __shared__ double sr[4][NODE_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rq_df += __shfl_down_sync(0xffffffffu, rq_df, o);
      rq_m += __shfl_down_sync(0xffffffffu, rq_m, o);
      rq_d2 += __shfl_down_sync(0xffffffffu, rq_d2, o);
      rq_max = fmax(rq_max, __shfl_down_sync(0xffffffffu, rq_max, o));
    }
    const int w = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0) {
      sr[0][w] = rq_df;
      sr[1][w] = rq_m;
      sr[2][w] = rq_d2;
      sr[3][w] = rq_max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
      for (int q = 0; q < NODE_THREADS / 32; ++q) {
        t0 += sr[0][q];
        t1 += sr[1][q];
        t2 += sr[2][q];
        t3 = fmax(t3, sr[3][q]);
      }
      double* o = a.rq_partials + 4 * (size_t)blockIdx.x;
      o[0] = t0;
      o[1] = t1;
      o[2] = t2;
      o[3] = t3;
    }
  }
}

// Adaptive dynamic relaxation, after the check step: fixed-order sums of the
// per-block Rayleigh-quotient terms, then (one thread) the damping update and
// the convergence-rate estimate described at AdrState.
__global__ void adr_finalize_kernel(const double* __restrict__ p, int n, const DevState* st, AdrState* adr) {
  __shared__ double s[4][256];
  double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    t0 += p[4 * q];
    t1 += p[4 * q + 1];
    t2 += p[4 * q + 2];
    t3 = fmax(t3, p[4 * q + 3]);
  }
  s[0][threadIdx.x] = t0;
  s[1][threadIdx.x] = t1;
  s[2][threadIdx.x] = t2;
  s[3][threadIdx.x] = t3;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s[0][threadIdx.x] += s[0][threadIdx.x + o];
      s[1][threadIdx.x] += s[1][threadIdx.x + o];
      s[2][threadIdx.x] += s[2][threadIdx.x + o];
      s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double dfd = s[0][0], dmd_a = s[1][0], d2 = s[2][0], dmax = s[3][0];
  // the force of this step was evaluated at U^n, n = step - 1; the interval
  // counts once the previous check's state is past the ramp
  const long long n_eval = st->step - 1;
  const bool past = adr->has_prev && (adr->ramp_steps <= 0 || adr->snap_step >= adr->ramp_steps);
  const double mdd = adr->kappa0 * adr->dt * adr->dt * dmd_a;  // D . M D
  if (past && mdd > 0.0 && dfd > 0.0) {
    const double lam = dfd / mdd;
    const double al = fmin(fmax(2.0 * sqrt(lam), adr->alpha_min), adr->alpha_max);
    const double adt = al * adr->dt;
    adr->lambda = lam;
    adr->alpha = al;
    adr->bm1 = (float)((2.0 - adt) / (2.0 + adt));
    adr->ai_scale = (float)(2.0 / (2.0 + adt) / adr->kappa0);
    adr->n_est += 1;
  }
  const double dn = sqrt(d2);
  adr->du_max = dmax;
  if (past && adr->du_norm > 0.0 && dn > 0.0) {
    const double r = dn / adr->du_norm;  // contraction over one interval
    adr->rho = pow(r, 1.0 / (double)adr->k);
    adr->err_est = r < 1.0 ? r / (1.0 - r) * dmax : INFINITY;
  } else {
    adr->rho = 0.0;
    adr->err_est = INFINITY;
  }
  adr->du_norm = past ? dn : 0.0;
  adr->snap_step = n_eval;
  adr->has_prev = 1;
}

__global__ void resid_finalize_kernel(const double2* __restrict__ p, int n, DevState* st) {
  __shared__ double sn[256], sd[256];
  double tn = 0.0, td = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    tn += p[q].x;
    td += p[q].y;
  }
  sn[threadIdx.x] = tn;
  sd[threadIdx.x] = td;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sn[threadIdx.x] += sn[threadIdx.x + o];
      sd[threadIdx.x] += sd[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->resid_num2 = sn[0];
    st->resid_den2 = sd[0];
  }
}

// one block per group: fixed-order sum of the per-node residual terms of the
// group's contiguous node range
__global__ void group_resid_kernel(const double2* __restrict__ nr, const int* __restrict__ gptr,
                                   double2* out) {
  __shared__ double sn[256], sd[256];
  const int g = blockIdx.x;
  double tn = 0.0, td = 0.0;
  for (int q = gptr[g] + threadIdx.x; q < gptr[g + 1]; q += blockDim.x) {
    tn += nr[q].x;
    td += nr[q].y;
  }
  sn[threadIdx.x] = tn;
  sd[threadIdx.x] = td;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sn[threadIdx.x] += sn[threadIdx.x + o];
      sd[threadIdx.x] += sd[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[g] = make_double2(sn[0], sd[0]);
}

template <int NE, bool FA, bool FB, bool MR, bool CMP>
cudaError_t launch_force_t(const ForceArgs& a, int threads, cudaStream_t s) {
  const int grid = (a.E + threads - 1) / threads;
  cudaError_t e = launch_pdl(force_slots_kernel<NE, FA, FB, MR, CMP>, dim3(grid), dim3(threads), 0, s, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NE, bool FA, bool FB, bool MR, bool CMP>
cudaError_t launch_tiles_t(const ForceArgs& a, const TileArgs& t, int n_tiles, cudaStream_t s) {
  const size_t per_tile = (size_t)tile_smem_f4(NE, CMP, t.T, t.cap) * sizeof(float4);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(force_tiles_kernel<NE, FA, FB, MR, CMP, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    cudaFuncSetAttribute(force_tiles_kernel<NE, FA, FB, MR, CMP, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr_set = true;
  }
  if (t.T == 32) {
    constexpr int W = 8;  // tiles (warps) per block
    return launch_pdl(force_tiles_kernel<NE, FA, FB, MR, CMP, true>, dim3((n_tiles + W - 1) / W), dim3(32 * W),
                      W * per_tile, s, a, t);
  }
  return launch_pdl(force_tiles_kernel<NE, FA, FB, MR, CMP, false>, dim3(n_tiles), dim3(t.T), per_tile, s, a, t);
}

template <int NE, bool CMP>
cudaError_t launch_force_e(int variant, const ForceArgs& a, int threads, cudaStream_t s) {
  switch (variant) {
    case VAR_NH: return launch_force_t<NE, false, false, false, CMP>(a, threads, s);
    case VAR_TI: return launch_force_t<NE, true, false, false, CMP>(a, threads, s);
    case VAR_OT: return launch_force_t<NE, true, true, false, CMP>(a, threads, s);
    case VAR_MR: return launch_force_t<NE, false, false, true, CMP>(a, threads, s);
    default: return launch_force_t<NE, true, true, true, CMP>(a, threads, s);
  }
}

template <int NE, bool CMP>
cudaError_t launch_tiles_e(int variant, const ForceArgs& a, const TileArgs& t, int n_tiles,
                           cudaStream_t s) {
  switch (variant) {
    case VAR_NH: return launch_tiles_t<NE, false, false, false, CMP>(a, t, n_tiles, s);
    case VAR_TI: return launch_tiles_t<NE, true, false, false, CMP>(a, t, n_tiles, s);
    case VAR_OT: return launch_tiles_t<NE, true, true, false, CMP>(a, t, n_tiles, s);
    case VAR_MR: return launch_tiles_t<NE, false, false, true, CMP>(a, t, n_tiles, s);
    default: return launch_tiles_t<NE, true, true, true, CMP>(a, t, n_tiles, s);
  }
}

}  // namespace

cudaError_t launch_force(int elem_type, int variant, int cmp, const ForceArgs& a, int threads,
                         cudaStream_t s) {
  if (elem_type == DJ_TET4)
    return cmp ? launch_force_e<4, true>(variant, a, threads, s) : launch_force_e<4, false>(variant, a, threads, s);
  return cmp ? launch_force_e<8, true>(variant, a, threads, s) : launch_force_e<8, false>(variant, a, threads, s);
}

cudaError_t launch_force_tiled(int elem_type, int variant, int cmp, const ForceArgs& a,
                               const TileArgs& t, int n_tiles, cudaStream_t s) {
  if (elem_type == DJ_TET4)
    return cmp ? launch_tiles_e<4, true>(variant, a, t, n_tiles, s)
               : launch_tiles_e<4, false>(variant, a, t, n_tiles, s);
  return cmp ? launch_tiles_e<8, true>(variant, a, t, n_tiles, s)
             : launch_tiles_e<8, false>(variant, a, t, n_tiles, s);
}

template <int MODE>
cudaError_t launch_node_m(int cmp, const NodeArgs& a, cudaStream_t s) {
  const int grid = (a.N + NODE_THREADS - 1) / NODE_THREADS;
  const bool sell = a.node_ptr == nullptr;
  cudaError_t e =
      cmp ? (sell ? launch_pdl(node_kernel<MODE, true, true>, dim3(grid), dim3(NODE_THREADS), 0, s, a)
                  : launch_pdl(node_kernel<MODE, true, false>, dim3(grid), dim3(NODE_THREADS), 0, s, a))
          : (sell ? launch_pdl(node_kernel<MODE, false, true>, dim3(grid), dim3(NODE_THREADS), 0, s, a)
                  : launch_pdl(node_kernel<MODE, false, false>, dim3(grid), dim3(NODE_THREADS), 0, s, a));
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_node(int mode, int cmp, const NodeArgs& a, cudaStream_t s) {
  if (mode == NODE_UPDATE) return launch_node_m<NODE_UPDATE>(cmp, a, s);
  if (mode == NODE_UPDATE_TGT) return launch_node_m<NODE_UPDATE_TGT>(cmp, a, s);
  if (mode == NODE_ADR) return launch_node_m<NODE_ADR>(cmp, a, s);
  if (mode == NODE_ADR_RQ) return launch_node_m<NODE_ADR_RQ>(cmp, a, s);
  if (mode == NODE_UPDATE_RESID) return launch_node_m<NODE_UPDATE_RESID>(cmp, a, s);
  if (mode == NODE_RESID_ONLY) return launch_node_m<NODE_RESID_ONLY>(cmp, a, s);
  return launch_node_m<NODE_FORCE_ONLY>(cmp, a, s);
}

cudaError_t launch_group_resid(const double2* node_resid, const int* group_node_ptr, int n_groups,
                               double2* out, cudaStream_t s) {
  group_resid_kernel<<<n_groups, 256, 0, s>>>(node_resid, group_node_ptr, out);
  return cudaGetLastError();
}

cudaError_t launch_resid_finalize(const double2* partials, int n, DevState* st, cudaStream_t s) {
  resid_finalize_kernel<<<1, 256, 0, s>>>(partials, n, st);
  return cudaGetLastError();
}

cudaError_t launch_adr_finalize(const double* rq_partials, int n, const DevState* st, AdrState* adr,
                                cudaStream_t s) {
  adr_finalize_kernel<<<1, 256, 0, s>>>(rq_partials, n, st, adr);
  return cudaGetLastError();
}

}  // namespace dj
