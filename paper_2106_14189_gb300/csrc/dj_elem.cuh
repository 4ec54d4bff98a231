// Device-side element math shared by the step kernels (included by .cu files).
#pragma once

#include <cuda_runtime.h>

#include "dj_internal.h"

namespace dj {
namespace elem {

// x / 3 as a product (an IEEE division by a variable-free constant is not
// contracted without fast-math; the product differs by at most an ulp)
constexpr float kThird = 1.f / 3.f;


__device__ __forceinline__ float ldg_stream(const float* p) { return __ldcs(p); }

struct M3 {
  float m[3][3];
};

__device__ __forceinline__ float det3(const M3& a) {
  return a.m[0][0] * (a.m[1][1] * a.m[2][2] - a.m[1][2] * a.m[2][1]) -
         a.m[0][1] * (a.m[1][0] * a.m[2][2] - a.m[1][2] * a.m[2][0]) +
         a.m[0][2] * (a.m[1][0] * a.m[2][1] - a.m[1][1] * a.m[2][0]);
}

// adjugate: adj(a) = det(a) a^-1
__device__ __forceinline__ M3 adj3(const M3& a) {
  M3 r;
  r.m[0][0] = a.m[1][1] * a.m[2][2] - a.m[1][2] * a.m[2][1];
  r.m[0][1] = a.m[0][2] * a.m[2][1] - a.m[0][1] * a.m[2][2];
  r.m[0][2] = a.m[0][1] * a.m[1][2] - a.m[0][2] * a.m[1][1];
  r.m[1][0] = a.m[1][2] * a.m[2][0] - a.m[1][0] * a.m[2][2];
  r.m[1][1] = a.m[0][0] * a.m[2][2] - a.m[0][2] * a.m[2][0];
  r.m[1][2] = a.m[0][2] * a.m[1][0] - a.m[0][0] * a.m[1][2];
  r.m[2][0] = a.m[1][0] * a.m[2][1] - a.m[1][1] * a.m[2][0];
  r.m[2][1] = a.m[0][1] * a.m[2][0] - a.m[0][0] * a.m[2][1];
  r.m[2][2] = a.m[0][0] * a.m[1][1] - a.m[0][1] * a.m[1][0];
  return r;
}

// symmetric 3x3 stored as s[6] = {00, 11, 22, 01, 02, 12}
__device__ __forceinline__ float sym_at(const float* s, int i, int j) {
  if (i == j) return s[i];
  int k = i + j;  // (0,1)->1, (0,2)->2, (1,2)->3
  return s[2 + k];
}

__device__ __forceinline__ void load_sym(const float* c, int off, int E_pad, int e, float* s) {
#pragma unroll
  for (int k = 0; k < 6; ++k) s[k] = ldg_stream(c + (size_t)(off + k) * E_pad + e);
}

// g : S  (Frobenius product of symmetric g with symmetric S)
__device__ __forceinline__ float frob_sym(const float* g, const float* s) {
  return g[0] * s[0] + g[1] * s[1] + g[2] * s[2] + 2.f * (g[3] * s[3] + g[4] * s[4] + g[5] * s[5]);
}

// acc += w * tJ^T S  (S symmetric)
__device__ __forceinline__ void add_tJT_sym(M3& acc, const M3& tJ, const float* s, float w) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float v = tJ.m[0][i] * sym_at(s, 0, j) + tJ.m[1][i] * sym_at(s, 1, j) +
                tJ.m[2][i] * sym_at(s, 2, j);
      acc.m[i][j] = fmaf(w, v, acc.m[i][j]);
    }
}

// Per-element constants of the table, loaded once into registers.  ANP: the
// volumetric factor kappa 0V (J - 1) / det 0J is replaced by pv = pbar / 6, the
// element's mean nodal pressure times 0V / det 0J (T4, average nodal pressure).
template <bool FA, bool FB, bool MR, bool ANP = false>
struct ElemConsts {
  float J0[3][3];
  float P[6];
  float kV, r0;
  float pv;
  float Qa[FA ? 6 : 1], sa;
  float Qb[FB ? 6 : 1], sb;
  float gm;

  // ld(k) returns row k of the element's table entry
  template <class Ld>
  __device__ __forceinline__ void load(Ld ld, const ForceArgs& a) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) J0[i][j] = ld(K_J0 + 3 * i + j);
#pragma unroll
    for (int q = 0; q < 6; ++q) P[q] = ld(K_P + q);
    kV = ld(K_KV);
    r0 = ld(K_R0);
    if (FA) {
#pragma unroll
      for (int q = 0; q < 6; ++q) Qa[q] = ld(a.off_fa + q);
      sa = ld(a.off_fa + 6);
    }
    if (FB) {
#pragma unroll
      for (int q = 0; q < 6; ++q) Qb[q] = ld(a.off_fb + q);
      sb = ld(a.off_fb + 6);
    }
    if (MR) gm = ld(a.off_mr);
  }

  // geometric T4 table (KG_*): the stored scalars first, then geometry()
  float cP;
  template <class Ld>
  __device__ __forceinline__ void load_geometric(Ld ld, const ForceArgs& a) {
    cP = ld(KG_CP);
    kV = ld(KG_KV);
    if (FA) {
#pragma unroll
      for (int q = 0; q < 6; ++q) Qa[q] = ld(a.off_fa + q);
      sa = ld(a.off_fa + 6);
    }
    if (FB) {
#pragma unroll
      for (int q = 0; q < 6; ++q) Qb[q] = ld(a.off_fb + q);
      sb = ld(a.off_fb + 6);
    }
    if (MR) gm = ld(a.off_mr);
  }

  // xd[i] = X_{i+1} - X_0 (tile-local reference coordinates) is 0J (Eq. 3);
  // det 0J, r0 and P = c_P adj(0J)^T adj(0J) (Eq. 37) follow
  __device__ __forceinline__ void geometry(const float (&xd)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) J0[i][j] = xd[i][j];
    float ad[3][3];  // adj(0J): 0J adj(0J) = det I
    ad[0][0] = J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1];
    ad[0][1] = J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2];
    ad[0][2] = J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1];
    ad[1][0] = J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2];
    ad[1][1] = J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0];
    ad[1][2] = J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2];
    ad[2][0] = J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0];
    ad[2][1] = J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1];
    ad[2][2] = J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0];
    const float det = J0[0][0] * ad[0][0] + J0[0][1] * ad[1][0] + J0[0][2] * ad[2][0];
    r0 = __fdividef(1.f, det);  // fast reciprocal, ~1 ulp: J carries FP32 rounding anyway
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int q = 0; q < 6; ++q)
      P[q] = cP * (ad[0][ii[q]] * ad[0][jj[q]] + ad[1][ii[q]] * ad[1][jj[q]] + ad[2][ii[q]] * ad[2][jj[q]]);
  }
};

// Hourglass constants of a brick: c_{alpha j} = h_alpha . X_j and k.
struct HgConsts {
  float cc[4][3];
  float k;
  template <class Ld>
  __device__ __forceinline__ void load(Ld ld, int off) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < 3; ++j) cc[q][j] = ld(off + 3 * q + j);
    k = ld(off + 12);
  }
  // geometric table: only k is stored; c is formed from reference coordinates
  template <class Ld>
  __device__ __forceinline__ void load_k(Ld ld, int off) {
    k = ld(off);
  }
};

// F = J^-2/3 tJ^T (P + psi_a Q_a + psi_b Q_b + MR) + coefficient * adj(tJ)   (Table 3)
template <bool FA, bool FB, bool MR, bool ANP>
__device__ __forceinline__ M3 dj_force_matrix(const M3& tJ, const ElemConsts<FA, FB, MR, ANP>& k,
                                              bool& bad) {
  const M3 A = adj3(tJ);  // det(tJ) tJ^-1
  const float D = tJ.m[0][0] * A.m[0][0] + tJ.m[0][1] * A.m[1][0] + tJ.m[0][2] * A.m[2][0];
  const float J = D * k.r0;  // Eq. 12
  bad = !(D > 0.f);
  const float Jm23 = __powf(J, -2.f * kThird);  // J^-2/3 (fast exp2/log2 intrinsics, ~1e-7 relative)
  // T = tJ^T P, and P : g = tr(tJ^T P tJ) = T : tJ^T  (g = tJ tJ^T, Eq. 17)
  M3 T;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      T.m[i][j] = tJ.m[0][i] * sym_at(k.P, 0, j) + tJ.m[1][i] * sym_at(k.P, 1, j) +
                  tJ.m[2][i] * sym_at(k.P, 2, j);
  float gP = 0.f;  // = mu 0V I1
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) gP = fmaf(T.m[i][j], tJ.m[j][i], gP);
  float vol_over_D = -gP * kThird;  // multiplies Jm23 adj / D
  float g[6];
  if (FA || FB || MR) {
    g[0] = tJ.m[0][0] * tJ.m[0][0] + tJ.m[0][1] * tJ.m[0][1] + tJ.m[0][2] * tJ.m[0][2];
    g[1] = tJ.m[1][0] * tJ.m[1][0] + tJ.m[1][1] * tJ.m[1][1] + tJ.m[1][2] * tJ.m[1][2];
    g[2] = tJ.m[2][0] * tJ.m[2][0] + tJ.m[2][1] * tJ.m[2][1] + tJ.m[2][2] * tJ.m[2][2];
    g[3] = tJ.m[0][0] * tJ.m[1][0] + tJ.m[0][1] * tJ.m[1][1] + tJ.m[0][2] * tJ.m[1][2];
    g[4] = tJ.m[0][0] * tJ.m[2][0] + tJ.m[0][1] * tJ.m[2][1] + tJ.m[0][2] * tJ.m[2][2];
    g[5] = tJ.m[1][0] * tJ.m[2][0] + tJ.m[1][1] * tJ.m[2][1] + tJ.m[1][2] * tJ.m[2][2];
  }
  if (FA) {
    const float gQ = frob_sym(g, k.Qa);
    const float psi = Jm23 * gQ * k.sa - 1.f;  // I4bar - 1 (Eq. 31, Table 1)
    add_tJT_sym(T, tJ, k.Qa, psi);
    vol_over_D -= psi * gQ * kThird;
  }
  if (FB) {
    const float gQ = frob_sym(g, k.Qb);
    const float psi = Jm23 * gQ * k.sb - 1.f;  // I6bar - 1 (Eq. 32)
    add_tJT_sym(T, tJ, k.Qb, psi);
    vol_over_D -= psi * gQ * kThird;
  }
  float mr_vol = 0.f;
  if (MR) {
    // C01 g_hat^T I2m = gm (g:P P - P g P), gm = C01 / (2 C10^2 0V)   (Eq. 39-42)
    float Pg[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Pg[i][j] = sym_at(k.P, i, 0) * sym_at(g, 0, j) + sym_at(k.P, i, 1) * sym_at(g, 1, j) +
                   sym_at(k.P, i, 2) * sym_at(g, 2, j);
    float S2[6];
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int i = ii[q], j = jj[q];
      const float PgP = Pg[i][0] * sym_at(k.P, 0, j) + Pg[i][1] * sym_at(k.P, 1, j) +
                        Pg[i][2] * sym_at(k.P, 2, j);
      S2[q] = k.gm * (gP * sym_at(k.P, i, j) - PgP);
    }
    float trPgPg = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) trPgPg += Pg[i][j] * Pg[j][i];
    add_tJT_sym(T, tJ, S2, Jm23);                               // extra J^-2/3 of Eq. 39
    mr_vol = -Jm23 * Jm23 * k.gm * (gP * gP - trPgPg) * kThird;  // -2/3 2 C01 I2bar 0V
  }
  const float invD = __fdividef(1.f, D);
  const float ca = (Jm23 * vol_over_D + mr_vol) * invD + (ANP ? k.pv : k.kV * (J - 1.f) * k.r0);
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F.m[i][j] = fmaf(Jm23, T.m[i][j], ca * A.m[i][j]);
  return F;
}

__device__ __forceinline__ void flag_nonfinite(DevState* st, int node) {
  atomicOr(&st->err_flags, ERR_NONFINITE);
  atomicMin(&st->bad_node, node);
}

// det tJ <= 0 (or not a number) in element e.  Non-finite values are detected
// per node in the update kernel, where U^{n+1} is formed.
__device__ __forceinline__ void flag_inverted(DevState* st, int e, bool inverted) {
  if (inverted) {
    atomicOr(&st->err_flags, ERR_INVERTED);
    atomicMin(&st->bad_elem, e);
  }
}

// griddepcontrol (programmatic dependent launch, see launch_pdl)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Writes the step state that the update kernel of the previous step reads:
// only after pdl_wait.
__device__ __forceinline__ void advance_clock(const ForceArgs& a) {
  if (a.advance && blockIdx.x == 0 && threadIdx.x == 0) {
    const long long n1 = a.st->step + 1;
    double s = 1.0;
    if (a.ramp_steps > 0) {
      double tau = (double)n1 / (double)a.ramp_steps;
      tau = tau > 1.0 ? 1.0 : tau;
      s = a.ramp_kind == DJ_RAMP_LINEAR ? tau : tau * tau * tau * (10.0 - 15.0 * tau + 6.0 * tau * tau);
    }
    a.st->ramp_s = (float)s;
    a.st->step = n1;
  }
}

// The step's prescribed targets from the caller's page-locked array (read
// coalesced over the host link, one value per thread, before the wait) into
// the device copy the update kernel reads (stored after the wait, once the
// previous update has completed).  A grid with fewer threads than targets
// copies the rest in a loop.
__device__ __forceinline__ double targets_load(const ForceArgs& a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  return g < a.n_tgt ? a.tgt_src[g] : 0.0;
}
__device__ __forceinline__ void targets_store(const ForceArgs& a, double v) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n_tgt) return;
  a.tgt_dst[g] = v;
  const int n = gridDim.x * blockDim.x;
  for (int q = g + n; q < a.n_tgt; q += n) a.tgt_dst[q] = a.tgt_src[q];
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
  return isfinite(x) && isfinite(y) && isfinite(z);
}

// natural coordinates of the brick nodes (bottom face CCW, then top face)
__device__ constexpr float XI8[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                        {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
// hourglass base vectors h1 = xi eta, h2 = eta zeta, h3 = zeta xi, h4 = xi eta zeta
__device__ constexpr float H8[4][8] = {{1, -1, 1, -1, 1, -1, 1, -1},
                                       {1, 1, -1, -1, -1, -1, 1, 1},
                                       {1, -1, -1, 1, -1, 1, 1, -1},
                                       {-1, 1, -1, 1, 1, -1, 1, -1}};

template <int NE>
struct ElemExtra;
template <>
struct ElemExtra<4> {
  template <class Ld>
  __device__ __forceinline__ void load(Ld, int) {}
};
template <>
struct ElemExtra<8> : HgConsts {};

// adj(A + B) - adj(A), expanded so that no O(1) terms cancel
__device__ __forceinline__ M3 adj_delta(const M3& A, const M3& B) {
#define DJ_ADJD(p0, p1, q0, q1, r0, r1, s0, s1)                                                  \
  (A.m[p0][p1] * B.m[q0][q1] + B.m[p0][p1] * A.m[q0][q1] + B.m[p0][p1] * B.m[q0][q1] -           \
   (A.m[r0][r1] * B.m[s0][s1] + B.m[r0][r1] * A.m[s0][s1] + B.m[r0][r1] * B.m[s0][s1]))
  M3 r;
  r.m[0][0] = DJ_ADJD(1, 1, 2, 2, 1, 2, 2, 1);
  r.m[0][1] = DJ_ADJD(0, 2, 2, 1, 0, 1, 2, 2);
  r.m[0][2] = DJ_ADJD(0, 1, 1, 2, 0, 2, 1, 1);
  r.m[1][0] = DJ_ADJD(1, 2, 2, 0, 1, 0, 2, 2);
  r.m[1][1] = DJ_ADJD(0, 0, 2, 2, 0, 2, 2, 0);
  r.m[1][2] = DJ_ADJD(0, 2, 1, 0, 0, 0, 1, 2);
  r.m[2][0] = DJ_ADJD(1, 0, 2, 1, 1, 1, 2, 0);
  r.m[2][1] = DJ_ADJD(0, 1, 2, 0, 0, 0, 2, 1);
  r.m[2][2] = DJ_ADJD(0, 0, 1, 1, 0, 1, 1, 0);
#undef DJ_ADJD
  return r;
}

// Compensated form of the same force: with A = 0J and B = tJ - 0J (Eq. 11),
//   J - 1        = (tr(adj(A) B) + tr(A adj(B)) + det B) / det A          (Eq. 12)
//   g:P - 3 mu0V = P : (A B^T + B A^T + B B^T),  mu 0V = P : A A^T / 3
//   tJ^T P - (g:P)/3 tJ^-1
//                = mu0V (J-1) adj(A) / D + B^T P - mu0V (adj(tJ) - adj(A)) / D
//                  - (g:P - 3 mu0V) / 3 adj(tJ) / D
//   I4bar - 1    = (J^-2/3 - 1) + J^-2/3 (P_a : (A B^T + B A^T + B B^T)) s_a
// Every term is of the order of the increment, so FP32 keeps its relative
// accuracy at small strain instead of losing it to cancellation.
template <bool FA, bool FB, bool MR, bool ANP>
__device__ __forceinline__ M3 dj_force_matrix_cmp(const M3& A, const M3& B, const ElemConsts<FA, FB, MR, ANP>& k,
                                                  bool& bad) {
  M3 tJ;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) tJ.m[i][j] = A.m[i][j] + B.m[i][j];
  const M3 adjA = adj3(A);
  const M3 adjB = adj3(B);
  float dD = det3(B);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) dD += adjA.m[i][j] * B.m[j][i] + A.m[i][j] * adjB.m[j][i];
  const float jm1 = dD * k.r0;  // J - 1
  const float J = 1.f + jm1;
  bad = !(J > 0.f);
  const float D = __fdividef(1.f, k.r0) + dD;
  const float invD = __fdividef(1.f, D);
  const float lJ = log1pf(jm1);
  const float Jm23 = __expf(-2.f * kThird * lJ);  // a factor near 1: the fast exponential suffices
  const float Jm23m1 = expm1f(-2.f * kThird * lJ);
  // g0 = A A^T and dg = A B^T + B A^T + B B^T (symmetric, {00,11,22,01,02,12})
  const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
  float g0[6], dg[6], g[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int i = ii[q], j = jj[q];
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      s0 += A.m[i][m] * A.m[j][m];
      s1 += A.m[i][m] * B.m[j][m] + B.m[i][m] * A.m[j][m] + B.m[i][m] * B.m[j][m];
    }
    g0[q] = s0;
    dg[q] = s1;
    g[q] = s0 + s1;
  }
  const float mV = frob_sym(g0, k.P) * kThird;  // mu 0V
  const float dgP = frob_sym(dg, k.P);       // g:P - 3 mu 0V
  const M3 adjD = adj_delta(A, B);
  M3 adjT;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) adjT.m[i][j] = adjA.m[i][j] + adjD.m[i][j];
  M3 T;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) T.m[i][j] = 0.f;
  add_tJT_sym(T, B, k.P, 1.f);  // B^T P
  float cT = -dgP * kThird * invD;  // coefficient of adj(tJ) inside the J^-2/3 bracket
  if (FA) {
    const float d4 = frob_sym(dg, k.Qa);
    const float psi = Jm23m1 + Jm23 * d4 * k.sa;  // I4bar - 1
    add_tJT_sym(T, tJ, k.Qa, psi);
    cT -= psi * frob_sym(g, k.Qa) * kThird * invD;
  }
  if (FB) {
    const float d6 = frob_sym(dg, k.Qb);
    const float psi = Jm23m1 + Jm23 * d6 * k.sb;  // I6bar - 1
    add_tJT_sym(T, tJ, k.Qb, psi);
    cT -= psi * frob_sym(g, k.Qb) * kThird * invD;
  }
  float mr_vol = 0.f;
  if (MR) {
    const float gP = 3.f * mV + dgP;
    float Pg[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Pg[i][j] = sym_at(k.P, i, 0) * sym_at(g, 0, j) + sym_at(k.P, i, 1) * sym_at(g, 1, j) +
                   sym_at(k.P, i, 2) * sym_at(g, 2, j);
    float S2[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int i = ii[q], j = jj[q];
      const float PgP = Pg[i][0] * sym_at(k.P, 0, j) + Pg[i][1] * sym_at(k.P, 1, j) +
                        Pg[i][2] * sym_at(k.P, 2, j);
      S2[q] = k.gm * (gP * sym_at(k.P, i, j) - PgP);
    }
    float trPgPg = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) trPgPg += Pg[i][j] * Pg[j][i];
    add_tJT_sym(T, tJ, S2, Jm23);
    mr_vol = -Jm23 * Jm23 * k.gm * (gP * gP - trPgPg) * kThird;
  }
  const float cA = mV * jm1 * invD, cD = -mV * invD;
  const float cadj = mr_vol * invD + (ANP ? k.pv : k.kV * jm1 * k.r0);  // volumetric: kappa 0V (J-1) r0 adj(tJ)
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float br = T.m[i][j] + cA * adjA.m[i][j] + cD * adjD.m[i][j] + cT * adjT.m[i][j];
      F.m[i][j] = fmaf(Jm23, br, cadj * adjT.m[i][j]);
    }
  return F;
}

template <bool FA, bool FB, bool MR, bool CMP, bool ANP>
__device__ __forceinline__ M3 force_matrix(const M3& A, const M3& B, const ElemConsts<FA, FB, MR, ANP>& k,
                                           bool& bad) {
  if constexpr (CMP) {
    return dj_force_matrix_cmp<FA, FB, MR>(A, B, k, bad);
  } else {
    M3 tJ;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) tJ.m[i][j] = A.m[i][j] + B.m[i][j];
    return dj_force_matrix<FA, FB, MR>(tJ, k, bad);
  }
}

// u_b - u_0 of one component; compensated mode: from the (hi, lo) pairs with an
// error-free difference of the high parts
template <bool CMP>
__device__ __forceinline__ float node_diff(float hb, float h0, float lb, float l0) {
  if constexpr (!CMP) {
    return hb - h0;
  } else {
    const float s = hb - h0;
    const float bb = s - hb;
    const float err = (hb - (s - bb)) + (-h0 - bb);
    return s + (err + (lb - l0));
  }
}

// Nodal forces of one T4 element from d_b = u_b - u_0 (b = 1..3):
// tJ = 0J + H_xi u has rows d_1, d_2, d_3 (Eq. 11); F H_xi gives node b = 1..3
// column b-1 and node 0 minus their sum (Sec. 7).
template <bool FA, bool FB, bool MR, bool CMP, bool ANP>
__device__ __forceinline__ void tet4_forces(const float (&d)[4][3], const ElemConsts<FA, FB, MR, ANP>& k,
                                            const ElemExtra<4>&, float (&f)[4][3], bool& inv) {
  M3 A, B;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A.m[i][j] = k.J0[i][j];
      B.m[i][j] = d[i + 1][j];
    }
  const M3 F = force_matrix<FA, FB, MR, CMP>(A, B, k, inv);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    f[1][j] = F.m[j][0];
    f[2][j] = F.m[j][1];
    f[3][j] = F.m[j][2];
    f[0][j] = -(F.m[j][0] + F.m[j][1] + F.m[j][2]);
  }
}

// Nodal forces of one 1-point H8 element with hourglass control, from
// d_b = u_b - u_0 (H_xi and the hourglass vectors annihilate constants, so
// sums over d_b equal sums over u_b).
template <bool FA, bool FB, bool MR, bool CMP>
__device__ __forceinline__ void hex8_forces(const float (&d)[8][3], const ElemConsts<FA, FB, MR>& k,
                                            const ElemExtra<8>& hg, float (&f)[8][3], bool& inv) {
  // s_i = (H_xi u)_i = sum_b xi_{b,i} d_b / 8
  float s[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int b = 1; b < 8; ++b) acc += XI8[b][i] * d[b][j];
      s[i][j] = 0.125f * acc;
    }
  M3 A, B;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A.m[i][j] = k.J0[i][j];
      B.m[i][j] = s[i][j];  // Eq. 11
    }
  const M3 F = force_matrix<FA, FB, MR, CMP>(A, B, k, inv);
  // hourglass: q_alpha = gamma_alpha . u, gamma_alpha = h_alpha - sum_j c_aj 0B_j,
  // 0B = 0J^-1 H_xi with 0J^-1 = adj(0J) / det 0J
  const M3 J0a = adj3(A);
  float eq[4][3];  // e_{alpha,i} = sum_j c_{alpha j} (0J^-1)_{j i}
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      eq[q][i] = k.r0 * (hg.cc[q][0] * J0a.m[0][i] + hg.cc[q][1] * J0a.m[1][i] + hg.cc[q][2] * J0a.m[2][i]);
  float H[4][3];  // k q_alpha
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float hu = 0.f;
#pragma unroll
      for (int b = 1; b < 8; ++b) hu += H8[q][b] * d[b][j];
      H[q][j] = hg.k * (hu - (eq[q][0] * s[0][j] + eq[q][1] * s[1][j] + eq[q][2] * s[2][j]));
    }
  // G_i = F[:, i] / 8 - (1/8) sum_alpha e_{alpha,i} H_alpha;  f_b = sum_i xi_{b,i} G_i + sum_alpha h_{alpha,b} H_alpha
  float G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      G[i][j] = 0.125f * (F.m[j][i] - (eq[0][i] * H[0][j] + eq[1][i] * H[1][j] + eq[2][i] * H[2][j] +
                                       eq[3][i] * H[3][j]));
#pragma unroll
  for (int b = 0; b < 8; ++b)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      f[b][j] = XI8[b][0] * G[0][j] + XI8[b][1] * G[1][j] + XI8[b][2] * G[2][j] + H8[0][b] * H[0][j] +
                H8[1][b] * H[1][j] + H8[2][b] * H[2][j] + H8[3][b] * H[3][j];
}

// The same H8 forces, consuming the element's nodes one at a time and emitting
// each node's force as soon as it is known, so that neither the 24 nodal
// differences nor the 24 forces are live at once (register pressure sets the
// occupancy of the H8 kernels):
//   ld(b, hi, lo)  nodal displacement of local node b (low part: compensated)
//   ldx(b)         reference coordinates (GEO: 0J = H_xi X, Eq. 3, and the
//                  hourglass c_{alpha j} = h_alpha . X_j are formed from them)
//   out(b, f)      force on local node b
// Summation orders equal those of hex8_forces.
template <bool FA, bool FB, bool MR, bool CMP, bool GEO, class Ld, class LdX, class Out>
__device__ __forceinline__ void hex8_forces_stream(Ld ld, LdX ldx, ElemConsts<FA, FB, MR>& k, HgConsts& hg,
                                                   Out out, bool& inv) {
  float s[3][3], hu[4][3], jx[3][3], cx[4][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i][j] = jx[i][j] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) hu[q][j] = cx[q][j] = 0.f;
  }
  float4 h0, l0;
  ld(0, h0, l0);
  float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (GEO) x0 = ldx(0);
#pragma unroll
  for (int b = 1; b < 8; ++b) {
    float4 hb, lb;
    ld(b, hb, lb);
    const float db[3] = {node_diff<CMP>(hb.x, h0.x, lb.x, l0.x), node_diff<CMP>(hb.y, h0.y, lb.y, l0.y),
                         node_diff<CMP>(hb.z, h0.z, lb.z, l0.z)};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
      for (int i = 0; i < 3; ++i) s[i][j] += XI8[b][i] * db[j];
#pragma unroll
      for (int q = 0; q < 4; ++q) hu[q][j] += H8[q][b] * db[j];
    }
    if (GEO) {
      const float4 xb = ldx(b);
      const float dx[3] = {xb.x - x0.x, xb.y - x0.y, xb.z - x0.z};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int i = 0; i < 3; ++i) jx[i][j] += XI8[b][i] * dx[j];
#pragma unroll
        for (int q = 0; q < 4; ++q) cx[q][j] += H8[q][b] * dx[j];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s[i][j] *= 0.125f;
  if (GEO) {
    float xd[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) xd[i][j] = 0.125f * jx[i][j];
    k.geometry(xd);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < 3; ++j) hg.cc[q][j] = cx[q][j];
  }
  M3 A, B;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A.m[i][j] = k.J0[i][j];
      B.m[i][j] = s[i][j];  // Eq. 11
    }
  const M3 F = force_matrix<FA, FB, MR, CMP>(A, B, k, inv);
  const M3 J0a = adj3(A);
  float eq[4][3];  // e_{alpha,i} = sum_j c_{alpha j} (0J^-1)_{j i}
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      eq[q][i] = k.r0 * (hg.cc[q][0] * J0a.m[0][i] + hg.cc[q][1] * J0a.m[1][i] + hg.cc[q][2] * J0a.m[2][i]);
  float H[4][3];  // k q_alpha
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      H[q][j] = hg.k * (hu[q][j] - (eq[q][0] * s[0][j] + eq[q][1] * s[1][j] + eq[q][2] * s[2][j]));
  float G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      G[i][j] = 0.125f * (F.m[j][i] - (eq[0][i] * H[0][j] + eq[1][i] * H[1][j] + eq[2][i] * H[2][j] +
                                       eq[3][i] * H[3][j]));
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    float fb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      fb[j] = XI8[b][0] * G[0][j] + XI8[b][1] * G[1][j] + XI8[b][2] * G[2][j] + H8[0][b] * H[0][j] +
              H8[1][b] * H[1][j] + H8[2][b] * H[2][j] + H8[3][b] * H[3][j];
    out(b, make_float4(fb[0], fb[1], fb[2], 0.f));
  }
}

template <int NE, bool FA, bool FB, bool MR, bool CMP, bool ANP>
__device__ __forceinline__ void elem_forces(const float (&d)[NE][3], const ElemConsts<FA, FB, MR, ANP>& k,
                                            const ElemExtra<NE>& x, float (&f)[NE][3], bool& inv) {
  if constexpr (NE == 4)
    tet4_forces<FA, FB, MR, CMP>(d, k, x, f, inv);
  else
    hex8_forces<FA, FB, MR, CMP>(d, k, x, f, inv);
}

// element at byte offset `off` of a shared float4 array (local node and slot
// indices are stored as byte offsets, which spares an index scaling per access)
__device__ __forceinline__ float4 at16(const float4* base, unsigned off) {
  return *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + off);
}

// Per-tile reduction of the force records into one partial per local node
// (li: byte offsets of the records), spread over the whole block: G
// consecutive lanes share a node (G = 8 or 4 when G n_t <= T, else 2, in
// passes of T / G nodes: a tile of more than T / 2 nodes takes two passes, the
// second over its lightest nodes, rather than one lane per node), lane r adds
// the node's records r, r + G, r + 2G, ... in order, and the G lane sums are
// combined by an xor butterfly (fixed order).  All lanes of a warp take part
// in every butterfly.
// store(q, f) receives node q's partial.  The choice of G depends only on n_t
// and T, so every kernel that uses this gives bit-identical partials.
template <int G, class Store>
__device__ __forceinline__ void reduce_tile_g(const float4* sf4, const unsigned short* li,
                                              const unsigned short* lp, int n_t, int tid, int T, Store store) {
  const int sub = tid % G, per_pass = T / G;
  for (int q0 = 0; q0 < n_t; q0 += per_pass) {
    const int q = q0 + tid / G;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (q < n_t) {
      const int p1 = lp[q + 1];
      for (int p = lp[q] + sub; p < p1; p += G) {
        const float4 v = at16(sf4, li[p]);
        fx += v.x;
        fy += v.y;
        fz += v.z;
      }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
      fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (q < n_t && sub == 0) store(q, make_float4(fx, fy, fz, 0.f));
  }
}

template <class Store>
__device__ __forceinline__ void reduce_tile(const float4* sf4, const unsigned short* li, const unsigned short* lp,
                                            int n_t, int tid, int T, Store store) {
  if (8 * n_t <= T) reduce_tile_g<8>(sf4, li, lp, n_t, tid, T, store);
  else if (4 * n_t <= T) reduce_tile_g<4>(sf4, li, lp, n_t, tid, T, store);
  else reduce_tile_g<2>(sf4, li, lp, n_t, tid, T, store);
}

// d_b = u_b - u_0 from the nodal records (hi, lo)
template <int NE, bool CMP>
__device__ __forceinline__ void node_deltas(const float4 (&h)[NE], const float4 (&l)[NE], float (&d)[NE][3]) {
  d[0][0] = d[0][1] = d[0][2] = 0.f;
#pragma unroll
  for (int b = 1; b < NE; ++b) {
    d[b][0] = node_diff<CMP>(h[b].x, h[0].x, l[b].x, l[0].x);
    d[b][1] = node_diff<CMP>(h[b].y, h[0].y, l[b].y, l[0].y);
    d[b][2] = node_diff<CMP>(h[b].z, h[0].z, l[b].z, l[0].z);
  }
}


}  // namespace elem
}  // namespace dj
