// DJ-TLED time-step kernels for sm_103a.
//
//  force_kernel<ELEM, FA, FB, MR>   one thread per element: Algorithm 1 runtime
//      steps 1-4 (tJ, J, g_hat, invariants, Table 3 force), written to the
//      element-force slots (slot = a * E_pad + e, so each store instruction of a
//      warp is one contiguous 512-byte run).
//  node_kernel<MODE>                one thread per node: deterministic gather of
//      the node's slots (sliced ELL, fixed order), central-difference update
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

#include "dj_internal.h"

namespace dj {

namespace {

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

// Per-element constants of the table, loaded once into registers.
template <bool FA, bool FB, bool MR>
struct ElemConsts {
  float J0[3][3];
  float P[6];
  float kV, r0;
  float Qa[FA ? 6 : 1], sa;
  float Qb[FB ? 6 : 1], sb;
  float gm;

  __device__ __forceinline__ void load(const float* __restrict__ c, int E_pad, int e,
                                       const ForceArgs& a) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) J0[i][j] = ldg_stream(c + (size_t)(K_J0 + 3 * i + j) * E_pad + e);
    load_sym(c, K_P, E_pad, e, P);
    kV = ldg_stream(c + (size_t)K_KV * E_pad + e);
    r0 = ldg_stream(c + (size_t)K_R0 * E_pad + e);
    if (FA) {
      load_sym(c, a.off_fa, E_pad, e, Qa);
      sa = ldg_stream(c + (size_t)(a.off_fa + 6) * E_pad + e);
    }
    if (FB) {
      load_sym(c, a.off_fb, E_pad, e, Qb);
      sb = ldg_stream(c + (size_t)(a.off_fb + 6) * E_pad + e);
    }
    if (MR) gm = ldg_stream(c + (size_t)a.off_mr * E_pad + e);
  }
};

// Hourglass constants of a brick: c_{alpha j} = h_alpha . X_j and k.
struct HgConsts {
  float cc[4][3];
  float k;
  __device__ __forceinline__ void load(const float* __restrict__ c, int E_pad, int e, int off) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < 3; ++j) cc[q][j] = ldg_stream(c + (size_t)(off + 3 * q + j) * E_pad + e);
    k = ldg_stream(c + (size_t)(off + 12) * E_pad + e);
  }
};

// F = J^-2/3 tJ^T (P + psi_a Q_a + psi_b Q_b + MR) + coefficient * adj(tJ)   (Table 3)
template <bool FA, bool FB, bool MR>
__device__ __forceinline__ M3 dj_force_matrix(const M3& tJ, const ElemConsts<FA, FB, MR>& k,
                                              bool& bad) {
  const float D = det3(tJ);
  const float J = D * k.r0;  // Eq. 12
  bad = !(D > 0.f);
  const float rc = rcbrtf(J);
  const float Jm23 = rc * rc;  // J^-2/3
  // g = tJ tJ^T (Eq. 17), symmetric
  float g[6];
  g[0] = tJ.m[0][0] * tJ.m[0][0] + tJ.m[0][1] * tJ.m[0][1] + tJ.m[0][2] * tJ.m[0][2];
  g[1] = tJ.m[1][0] * tJ.m[1][0] + tJ.m[1][1] * tJ.m[1][1] + tJ.m[1][2] * tJ.m[1][2];
  g[2] = tJ.m[2][0] * tJ.m[2][0] + tJ.m[2][1] * tJ.m[2][1] + tJ.m[2][2] * tJ.m[2][2];
  g[3] = tJ.m[0][0] * tJ.m[1][0] + tJ.m[0][1] * tJ.m[1][1] + tJ.m[0][2] * tJ.m[1][2];
  g[4] = tJ.m[0][0] * tJ.m[2][0] + tJ.m[0][1] * tJ.m[2][1] + tJ.m[0][2] * tJ.m[2][2];
  g[5] = tJ.m[1][0] * tJ.m[2][0] + tJ.m[1][1] * tJ.m[2][1] + tJ.m[1][2] * tJ.m[2][2];

  const float gP = frob_sym(g, k.P);  // = mu 0V I1
  M3 T;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) T.m[i][j] = 0.f;
  float vol_over_D = -gP / 3.f;  // multiplies Jm23 adj / D
  if (FA) {
    const float gQ = frob_sym(g, k.Qa);
    const float psi = Jm23 * gQ * k.sa - 1.f;  // I4bar - 1 (Eq. 31, Table 1)
    add_tJT_sym(T, tJ, k.Qa, psi);
    vol_over_D -= psi * gQ / 3.f;
  }
  if (FB) {
    const float gQ = frob_sym(g, k.Qb);
    const float psi = Jm23 * gQ * k.sb - 1.f;  // I6bar - 1 (Eq. 32)
    add_tJT_sym(T, tJ, k.Qb, psi);
    vol_over_D -= psi * gQ / 3.f;
  }
  add_tJT_sym(T, tJ, k.P, 1.f);
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
    mr_vol = -Jm23 * Jm23 * k.gm * (gP * gP - trPgPg) / 3.f;  // -2/3 2 C01 I2bar 0V
  }
  const M3 A = adj3(tJ);
  const float invD = 1.f / D;
  const float ca = (Jm23 * vol_over_D + mr_vol) * invD + k.kV * (J - 1.f) * k.r0;
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F.m[i][j] = fmaf(Jm23, T.m[i][j], ca * A.m[i][j]);
  return F;
}

__device__ __forceinline__ void flag_error(DevState* st, int e, bool inverted, bool nonfinite) {
  int f = (inverted ? ERR_INVERTED : 0) | (nonfinite ? ERR_NONFINITE : 0);
  if (f) {
    atomicOr(&st->err_flags, f);
    atomicMin(&st->bad_elem, e);
  }
}

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
  __device__ __forceinline__ void load(const float*, int, int, int) {}
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
template <bool FA, bool FB, bool MR>
__device__ __forceinline__ M3 dj_force_matrix_cmp(const M3& A, const M3& B, const ElemConsts<FA, FB, MR>& k,
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
  const float D = 1.f / k.r0 + dD;
  const float invD = 1.f / D;
  const float lJ = log1pf(jm1);
  const float Jm23 = expf(-2.f / 3.f * lJ);
  const float Jm23m1 = expm1f(-2.f / 3.f * lJ);
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
  const float mV = frob_sym(g0, k.P) / 3.f;  // mu 0V
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
  float cT = -dgP / 3.f * invD;  // coefficient of adj(tJ) inside the J^-2/3 bracket
  if (FA) {
    const float d4 = frob_sym(dg, k.Qa);
    const float psi = Jm23m1 + Jm23 * d4 * k.sa;  // I4bar - 1
    add_tJT_sym(T, tJ, k.Qa, psi);
    cT -= psi * frob_sym(g, k.Qa) / 3.f * invD;
  }
  if (FB) {
    const float d6 = frob_sym(dg, k.Qb);
    const float psi = Jm23m1 + Jm23 * d6 * k.sb;  // I6bar - 1
    add_tJT_sym(T, tJ, k.Qb, psi);
    cT -= psi * frob_sym(g, k.Qb) / 3.f * invD;
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
    mr_vol = -Jm23 * Jm23 * k.gm * (gP * gP - trPgPg) / 3.f;
  }
  const float cA = mV * jm1 * invD, cD = -mV * invD;
  const float cadj = mr_vol * invD + k.kV * jm1 * k.r0;  // volumetric: kappa 0V (J-1) r0 adj(tJ)
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

template <bool FA, bool FB, bool MR, bool CMP>
__device__ __forceinline__ M3 force_matrix(const M3& A, const M3& B, const ElemConsts<FA, FB, MR>& k,
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
template <bool FA, bool FB, bool MR, bool CMP>
__device__ __forceinline__ void tet4_forces(const float (&d)[4][3], const ElemConsts<FA, FB, MR>& k,
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

template <int NE, bool FA, bool FB, bool MR, bool CMP>
__device__ __forceinline__ void elem_forces(const float (&d)[NE][3], const ElemConsts<FA, FB, MR>& k,
                                            const ElemExtra<NE>& x, float (&f)[NE][3], bool& inv) {
  if constexpr (NE == 4)
    tet4_forces<FA, FB, MR, CMP>(d, k, x, f, inv);
  else
    hex8_forces<FA, FB, MR, CMP>(d, k, x, f, inv);
}

template <int NE>
__device__ __forceinline__ bool all_finite(const float (&f)[NE][3]) {
  bool ok = true;
#pragma unroll
  for (int b = 0; b < NE; ++b) ok &= finite3(f[b][0], f[b][1], f[b][2]);
  return ok;
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

// Element-slot assembly: one thread per element, forces to slot a * E_pad + e.
template <int NE, bool FA, bool FB, bool MR, bool CMP>
__global__ void __launch_bounds__(NE == 4 ? 256 : 128) force_slots_kernel(ForceArgs a) {
  advance_clock(a);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.E) return;
  const int E_pad = a.E_pad;
  const float* __restrict__ c = a.consts;
  ElemConsts<FA, FB, MR> k;
  k.load(c, E_pad, e, a);
  ElemExtra<NE> x;
  if constexpr (NE == 8) x.load(c, E_pad, e, a.off_hg);
  int nid[NE];
  {
    const int4 n0 = __ldcs(a.conn + (NE / 4) * (size_t)e);
    nid[0] = n0.x; nid[1] = n0.y; nid[2] = n0.z; nid[3] = n0.w;
    if constexpr (NE == 8) {
      const int4 n1 = __ldcs(a.conn + 2 * (size_t)e + 1);
      nid[4] = n1.x; nid[5] = n1.y; nid[6] = n1.z; nid[7] = n1.w;
    }
  }
  float4 h[NE], l[NE];
#pragma unroll
  for (int b = 0; b < NE; ++b) {
    h[b] = __ldg(a.U + nid[b]);
    l[b] = CMP ? __ldg(a.Ulo + nid[b]) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float d[NE][3];
  node_deltas<NE, CMP>(h, l, d);
  float f[NE][3];
  bool inv;
  elem_forces<NE, FA, FB, MR, CMP>(d, k, x, f, inv);
  flag_error(a.st, e, inv, !inv && !all_finite<NE>(f));
#pragma unroll
  for (int b = 0; b < NE; ++b) a.slots[(size_t)b * E_pad + e] = make_float4(f[b][0], f[b][1], f[b][2], 0.f);
}

// Tiled assembly: block = tile of T elements.  The tile's unique nodes are
// staged in shared memory, element forces go to shared memory (slot a * T + e),
// and each unique node sums its slots in the fixed order of the local index.
template <int NE, bool FA, bool FB, bool MR, bool CMP>
__global__ void __launch_bounds__(NE == 4 ? 512 : 256) force_tiles_kernel(ForceArgs a, TileArgs t) {
  extern __shared__ float4 smem4[];
  advance_clock(a);
  const int tile = blockIdx.x, tid = threadIdx.x, T = t.T;
  float4* su = smem4;                                          // staged U (high part)
  float4* sl = smem4 + t.smem_nodes;                           // staged low part (compensated)
  float* sf = reinterpret_cast<float*>(smem4 + (CMP ? 2 : 1) * t.smem_nodes);  // 3 x (NE T) forces
  const int base = __ldg(t.tile_ptr + tile);
  const int n_t = __ldg(t.tile_ptr + tile + 1) - base;
  const int e = tile * T + tid;
  const bool valid = e < a.E;
  const float* __restrict__ c = a.consts;
  ElemConsts<FA, FB, MR> k;
  ElemExtra<NE> x;
  unsigned short lc[NE];
  if (valid) {
    k.load(c, a.E_pad, e, a);
    if constexpr (NE == 8) x.load(c, a.E_pad, e, a.off_hg);
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
  for (int q = tid; q < n_t; q += T) {
    const int gid = __ldg(t.tile_nodes + base + q);
    su[q] = __ldg(a.U + gid);
    if (CMP) sl[q] = __ldg(a.Ulo + gid);
  }
  __syncthreads();
  if (valid) {
    float4 h[NE], l[NE];
#pragma unroll
    for (int b = 0; b < NE; ++b) {
      h[b] = su[lc[b]];
      l[b] = CMP ? sl[lc[b]] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float d[NE][3];
    node_deltas<NE, CMP>(h, l, d);
    float f[NE][3];
    bool inv;
    elem_forces<NE, FA, FB, MR, CMP>(d, k, x, f, inv);
    flag_error(a.st, e, inv, !inv && !all_finite<NE>(f));
    const int S = NE * T;
#pragma unroll
    for (int b = 0; b < NE; ++b) {
      sf[b * T + tid] = f[b][0];
      sf[S + b * T + tid] = f[b][1];
      sf[2 * S + b * T + tid] = f[b][2];
    }
  }
  __syncthreads();
  const int S = NE * T;
  const unsigned short* lp = t.lptr + base + tile;
  const unsigned short* li = t.lidx + (size_t)tile * S;
  for (int q = tid; q < n_t; q += T) {
    const int p0 = lp[q], p1 = lp[q + 1];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int p = p0; p < p1; ++p) {
      const int l = li[p];
      fx += sf[l];
      fy += sf[S + l];
      fz += sf[2 * S + l];
    }
    t.partials[base + q] = make_float4(fx, fy, fz, 0.f);
  }
}

template <int MODE, bool CMP>
__global__ void __launch_bounds__(NODE_THREADS) node_kernel(NodeArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = i / SELL_C, lane = i % SELL_C;
  double num2 = 0.0, den2 = 0.0;
  if (i < a.N) {
    const int beg = __ldg(a.chunk_ptr + chunk), end = __ldg(a.chunk_ptr + chunk + 1);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int p = beg + lane; p < end; p += SELL_C) {
      const int sid = __ldcs(a.sell + p);
      if (sid >= 0) {
        const float4 f = __ldcs(a.slots + sid);
        fx += f.x;
        fy += f.y;
        fz += f.z;
      }
    }
    if (a.R) {
      const float4 r = __ldg(a.R + i);
      fx -= r.x;
      fy -= r.y;
      fz -= r.z;
    }
    // now f = F_int - R
    const float4 V = a.V[i];
    const int bc = __float_as_int(V.w);
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
      const float4 U = a.U[i];
      const float ai = U.w;
      // velocity form of the central difference: D^{n+1} = a (R - F) + (b - 1) D^n
      const float bm1 = a.bm1_node ? __ldg(a.bm1_node + i) : a.bm1;
      float dd[3] = {fmaf(-ai, fx, bm1 * V.x), fmaf(-ai, fy, bm1 * V.y), fmaf(-ai, fz, bm1 * V.z)};
      const float uh[3] = {U.x, U.y, U.z};
      float nh[3], nl[3] = {0.f, 0.f, 0.f}, ul[3] = {0.f, 0.f, 0.f};
      if (CMP) {
        const float4 L = a.Ulo[i];
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
        const float4 t = __ldg(a.bct + bc);
        mask = __float_as_int(t.w);
        const float rs = a.st->ramp_s;
        const float tv[3] = {t.x, t.y, t.z};
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (mask & (1 << q)) {
            nh[q] = tv[q] * rs;
            nl[q] = 0.f;
            dd[q] = (nh[q] - uh[q]) - ul[q];
          }
      }
      a.U[i] = make_float4(nh[0], nh[1], nh[2], ai);
      if (CMP) a.Ulo[i] = make_float4(nl[0], nl[1], nl[2], 0.f);
      a.V[i] = make_float4(dd[0], dd[1], dd[2], V.w);
      if (MODE == NODE_UPDATE_RESID) {
        const double f3[3] = {fx, fy, fz};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (mask & (1 << q)) den2 += f3[q] * f3[q];
          else num2 += f3[q] * f3[q];
        }
      }
    }
  }
  constexpr bool RESID = MODE == NODE_UPDATE_RESID || MODE == NODE_RESID_ONLY;
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
  force_slots_kernel<NE, FA, FB, MR, CMP><<<grid, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int NE, bool FA, bool FB, bool MR, bool CMP>
cudaError_t launch_tiles_t(const ForceArgs& a, const TileArgs& t, int n_tiles, cudaStream_t s) {
  const size_t smem = (size_t)(CMP ? 2 : 1) * t.smem_nodes * sizeof(float4) +
                      (size_t)3 * NE * t.T * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(force_tiles_kernel<NE, FA, FB, MR, CMP>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr_set = true;
  }
  force_tiles_kernel<NE, FA, FB, MR, CMP><<<n_tiles, t.T, smem, s>>>(a, t);
  return cudaGetLastError();
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
  if (cmp)
    node_kernel<MODE, true><<<grid, NODE_THREADS, 0, s>>>(a);
  else
    node_kernel<MODE, false><<<grid, NODE_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_node(int mode, int cmp, const NodeArgs& a, cudaStream_t s) {
  if (mode == NODE_UPDATE) return launch_node_m<NODE_UPDATE>(cmp, a, s);
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

}  // namespace dj
