// Internal declarations of the DJ-TLED library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dj_tled.h"

namespace dj {

// ---------------------------------------------------------------------------
// per-element FP32 table (structure of arrays, stride E_pad), built by the FP64
// pre-computation.  Common part (19 floats):
//   0..8   0J row-major, 0J[i][j] = d x_j / d xi_i               (Eq. 3)
//   9..14  P = (mu / 2) I1m = mu 0V 0J^-T 0J^-1, as P00 P11 P22 P01 P02 P12
//          (Eq. 37 scaled by dPsi/dI1 of NH / TI / OT; C10 I1m for MR)
//   15     kappa 0V                                               (Table 3)
//   16     r0 = 1 / det 0J                                        (Eq. 12)
// optional blocks (offset -1 when absent):
//   fibre a: Q_a = eta_a I4m (6 floats, Eq. 45), s_a = 1 / (2 eta_a 0V)
//   fibre b: Q_b = eta_b I6m (6 floats, Eq. 46), s_b = 1 / (2 eta_b 0V)
//   MR:      c01 / c10 ratio, 1 / (2 0V)            (Eq. 39-42 rewritten)
//   H8 hourglass: c_{alpha j} = h_alpha . X_{:,j} (12 floats, alpha-major), k
// ---------------------------------------------------------------------------
enum { K_J0 = 0, K_P = 9, K_KV = 15, K_R0 = 16, K_COMMON = 17 };
// Geometric table (tiled assembly): the common part is only
//   0      c_P = mu 0V / det(0J)^2, so that P = c_P adj(0J)^T adj(0J)  (Eq. 37)
//   1      kappa 0V
// and 0J, det 0J and P are rebuilt per step from tile-local reference
// coordinates (TileArgs::xloc); the optional blocks follow as above, except
// that the H8 hourglass block holds k alone (c_{alpha j} = h_alpha . X_j is
// rebuilt from the coordinates too).
enum { KG_CP = 0, KG_KV = 1, KG_COMMON = 2 };

// Device-resident stepping state, one per mesh.
struct DevState {
  long long step;     // n of the current displacement U^n
  float ramp_s;       // s(tau) for the step being computed (U^{n+1})
  int err_flags;      // bit 0: det tJ <= 0, bit 1: non-finite value, bit 2: wait timeout, bit 3: bad target
  int bad_elem;       // smallest internal element id with det tJ <= 0
  int bad_node;       // smallest internal node id with a non-finite force or displacement
  double resid_num2;  // sum of squared residual over free DOFs
  double resid_den2;  // sum of squared reaction over prescribed DOFs
};

// ERR_BAD_TARGET: a non-finite prescribed target was handed to dj_step_host
// and not applied (reported and cleared by that call)
enum { ERR_INVERTED = 1, ERR_NONFINITE = 2, ERR_TIMEOUT = 4, ERR_BAD_TARGET = 8 };

struct ForceArgs {
  const int4* conn;      // tet: E_pad int4; hex: 2 E_pad int4 (nodes 0-3, 4-7)
  const float* consts;   // n_consts * E_pad
  const float4* U;       // U^n (xyz), w = node update coefficient
  const float4* Ulo;     // compensated mode: low part of U^n (U = U + Ulo), else unused
  float4* slots;         // element-force slots, slot = a * E_pad + e
  int E, E_pad;
  int off_fa, off_fb, off_mr, off_hg;
  DevState* st;
  int advance;           // 1: this launch is a time step (bump step, ramp)
  long long ramp_steps;
  int ramp_kind;
  const float* pres;     // average nodal pressure: p_i of every node (else unused)
  // the step's prescribed targets (host-driven steps): the caller's FP64
  // array through its device mapping, copied by the launch into tgt_dst (the
  // device copy the update kernel reads); n_tgt = 0: nothing to copy
  const double* tgt_src;
  double* tgt_dst;
  int n_tgt;
};

// Adaptive dynamic relaxation (one per mesh, device memory).  The damping in
// use is alpha; the update kernels of the adaptive steps take b - 1 and the
// scale of the precomputed a_i (a_i(alpha) / a_i(alpha_0)) from here.  At every
// check (every k steps) the change over the interval, D = U^n - U^{n-k}, and
// that of the force give the Rayleigh quotient
//   lambda = D . (F(U^n) - F(U^{n-k})) / (D . M D)    (free DOFs)
// of M^-1 K along D, alpha becomes 2 sqrt(lambda) (critical damping of that
// mode, clamped), and the ratio r of ||D|| at successive checks gives the
// per-step rate rho = r^(1/k) and err_est = r / (1 - r) max|D|, the estimated
// distance to equilibrium.
struct AdrState {
  // inputs, written by the host before each relaxation
  double dt;          // time step
  double kappa0;      // 2 / (2 + alpha_0 dt): M = kappa0 dt^2 / a_i(alpha_0)
  double alpha_min, alpha_max;
  long long ramp_steps;
  int k;              // steps between checks
  // damping in use
  float bm1;          // (2 - alpha dt) / (2 + alpha dt)
  float ai_scale;     // (2 + alpha_0 dt) / (2 + alpha dt)
  double alpha;
  // estimates of the last check
  double lambda;      // Rayleigh quotient [1/s^2] (0: none yet)
  double rho;         // per-step convergence rate (0: none)
  double err_est;     // rho / (1 - rho) max|D| (inf: none)
  double du_norm;     // ||D||_2 over free DOFs at the previous check past the ramp (0: none)
  double du_max;      // max |D| over free DOFs
  long long n_est;    // damping updates made
  long long snap_step;  // step index of the snapshot (U, F - R) of the previous check
  int has_prev;         // 0 until the first check has stored a snapshot
};

struct NodeArgs {
  const int* sell;        // sliced-ELL slot ids, chunks of 32 nodes, column-major
  const int* chunk_ptr;   // n_chunks + 1 offsets into sell
  const int* node_ptr;    // tiled assembly: N + 1 offsets of each node's partials in `slots`
                          // (node-major, ascending tile); nullptr: sliced-ELL gather
  const float4* slots;
  float4* U;              // in/out: U^n -> U^{n+1}; w = a_i
  float4* Ulo;            // compensated mode: low part of U
  float4* V;              // in/out: U^n - U^{n-1} -> U^{n+1} - U^n; w = bc index bits
  const float4* bct;      // per prescribed node: target xyz, w = component mask bits
  const float4* R;        // external loads or nullptr
  float4* fout;           // force-only mode output
  double2* partials;      // residual partial sums per block
  double2* node_resid;    // grouped meshes: per-node residual sums (else nullptr)
  const float* bm1_node;  // grouped meshes with damping: per-node b - 1 (else nullptr)
  DevState* st;           // ramp value (read), error flags (written)
  const AdrState* adr;    // adaptive modes: damping in use (else nullptr)
  // NODE_UPDATE_TGT only: prescribed targets read from the caller's FP64 array
  // (a device copy, or page-locked host memory through its device mapping;
  // entry bc_entry[b].{x,y,z} of prescribed-node row b, -1 if that component
  // is free; .w the component mask) instead of the per-node table; a
  // non-finite entry keeps the table's value.  nullptr: the table
  const double* tgt;
  const int4* bc_entry;
  double* rq_partials;    // NODE_ADR_RQ: 4 sums per block (D.dF, D^2 / a_i, D^2, max |D|)
  double4* usnap;         // NODE_ADR_RQ: U of the previous check (FP64, hi + lo); F - R of it in fout
  int N;
  float bm1;              // b - 1 = (2 - alpha dt) / (2 + alpha dt)
};

// Tiled assembly: a tile is the T consecutive (Morton-ordered) elements of one
// block.  Its unique nodes are staged in shared memory, the element forces are
// summed per unique node inside the tile in a fixed order, and one partial force
// per (tile, node) is written; the node kernel gathers those partials.
// Per-tile data is stored in fixed-size segments (multiples of 16 bytes) so a
// tile can be staged with bulk asynchronous copies:
//   element table   n_consts x T floats, tile-major: row r of element (t, i) at
//                   (t n_consts + r) T + i
//   lconn           T x n_e local node indices (element-major)
//   lidx            T x n_e local slots a T + e_local, grouped by node
//   tnodes          cap internal node ids (n_t used)
//   lptr            cap + 8 offsets into lidx (n_t + 1 used)
struct TileArgs {
  const int* tile_ptr;          // n_tiles + 1: first partial of each tile
  const int* tnodes;            // n_tiles x cap
  const unsigned short* lconn;  // n_tiles x T x n_e
  const unsigned short* lptr;   // n_tiles x (cap + 8)
  const unsigned short* lidx;   // n_tiles x T x n_e
  float4* partials;             // per (tile, node) force
  const float4* xloc;           // n_tiles x cap reference coordinates minus the tile's first node
  const int* pdst;              // n_tiles x cap: node-major position of each (tile, node) partial
  int T;
  int cap;                      // node capacity of a tile segment (multiple of 8, >= max n_t)
  int n_consts;
  int n_tiles;
};

enum { NODE_UPDATE = 0, NODE_UPDATE_RESID = 1, NODE_FORCE_ONLY = 2, NODE_RESID_ONLY = 3,
       // adaptive dynamic relaxation: the update with the damping of AdrState;
       // at a check also the Rayleigh-quotient and interval sums against the
       // previous check's snapshot (U, F - R), which it then replaces
       NODE_ADR = 4, NODE_ADR_RQ = 5,
       // the update with this step's prescribed targets read from the
       // caller's FP64 array (NodeArgs::tgt, required) and stored into the
       // prescribed-node rows of the table
       NODE_UPDATE_TGT = 6 };

// Programmatic dependent launch: the kernels of a step may start while the
// kernel before them in the stream finishes; each of them reads or writes what
// the previous one produces or consumes only after griddepcontrol.wait, which
// returns once that kernel has completed and its writes are visible (and at
// once when there is no programmatic dependency).  Used for launches made
// directly on a stream; kernels captured into a CUDA graph keep ordinary
// edges unless tl_graph_pdl is set (graph replays of back-to-back steps of a
// large mesh were measured faster with ordinary edges).
// Set by the host around a graph capture when the mesh's schedule keeps the
// programmatic edges inside graphs (dj_params.graph_pdl).
inline thread_local bool tl_graph_pdl = false;

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (cs == cudaStreamCaptureStatusNone || tl_graph_pdl) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
enum { ASSEMBLY_SLOTS = 0, ASSEMBLY_TILES = 1, ASSEMBLY_TILES_TMA = 2 };

constexpr int NODE_THREADS = 256;
constexpr int SELL_C = 32;

// kernels_step.cu
// cmp = 1: compensated precision (double-float U, increment-based forces)
cudaError_t launch_force(int elem_type, int variant, int cmp, const ForceArgs& a, int threads,
                         cudaStream_t s);
cudaError_t launch_force_tiled(int elem_type, int variant, int cmp, const ForceArgs& a,
                               const TileArgs& t, int n_tiles, cudaStream_t s);
// kernels_tma.cu: persistent, double-buffered tiles staged with bulk async copies
// anp: average nodal pressure (T4 only; reads ForceArgs::pres)
cudaError_t launch_force_tma(int elem_type, int variant, int cmp, int anp, const ForceArgs& a,
                             const TileArgs& t, int grid, cudaStream_t s);
size_t tma_smem_bytes(int elem_type, int cmp, int anp, const TileArgs& t);
int tma_blocks_per_sm(int elem_type, int variant, int cmp, int anp, const TileArgs& t);
cudaError_t launch_node(int mode, int cmp, const NodeArgs& a, cudaStream_t s);
cudaError_t launch_resid_finalize(const double2* partials, int n, DevState* st, cudaStream_t s);
// average nodal pressure (T4, tiles): volume pass and nodal pressures
size_t anp_volume_smem(int cmp, const TileArgs& t);
cudaError_t launch_anp(int cmp, const TileArgs& t, const int* node_ptr, const float4* U, const float4* Ulo, int E,
                       int N, float* vparts, const float* c1, float* pres, cudaStream_t s);
cudaError_t launch_adr_finalize(const double* rq_partials, int n, const DevState* st, AdrState* adr,
                                cudaStream_t s);
// per-group residual sums over contiguous node ranges (one block per group)
cudaError_t launch_group_resid(const double2* node_resid, const int* group_node_ptr, int n_groups,
                               double2* out, cudaStream_t s);

// gemm_tc.cu: C = alpha op(A) op(B) + beta C (strided FP32 operands, rounded
// to BF16 in shared memory; FP32 accumulation in tensor memory, tcgen05)
cudaError_t gemm_bf16_tc(int M, int N, int K, float alpha, const float* A, long long sar, long long sac,
                         const float* B, long long sbr, long long sbc, float beta, float* C, long long ldc,
                         cudaStream_t s);
// true (and the flag cleared) if a bounded wait of that kernel gave up
bool gemm_tc_timed_out();

// force kernel variants
enum { VAR_NH = 0, VAR_TI = 1, VAR_OT = 2, VAR_MR = 3, VAR_ALL = 4 };

// kernels_pre.cu
struct PreArgs {
  const double* X;          // internal order, N * 3
  const int* conn;          // internal order, E * ne
  const unsigned char* model;
  const double* mu;
  const double* kappa;
  const double* rho;
  const double* eta_a;
  const double* eta_b;
  const double* c01;
  const double* adir;       // E * 3
  const double* bdir;
  float* consts;
  int4* conn4;
  double* elem_mass;        // rho 0V / n_e
  double* dt_elem;
  int* bad;                 // first inverted element (atomicMin), init E
  int E, E_pad, ne;
  int off_fa, off_fb, off_mr, off_hg;
  double hg_coeff;
  int tile_T;    // > 0: tile-major table with tiles of tile_T elements
  int n_consts;
  int geometric; // 1: geometric table (KG_*, tiled assembly), else the full table (K_*)
};
cudaError_t launch_precompute_elements(const PreArgs& a, cudaStream_t s);
// dt_node: per-node time step (grouped meshes) or nullptr to use dt
cudaError_t launch_node_mass(const int* sell, const int* chunk_ptr, const double* elem_mass,
                             int E_pad, int N, double dt, const double* dt_node, double alpha,
                             const int* bc_index, double* mass_out, float4* U, float4* V,
                             cudaStream_t s);
cudaError_t launch_min_reduce(const double* v, int n, double* out, cudaStream_t s);
// evict the L2 cache: write the first half of buf, read the second (bytes >= 2 x L2)
cudaError_t launch_l2_flush(void* buf, size_t bytes, cudaStream_t s);
// st_out (optional): block 0 also copies the device state *st there (e.g. a
// mapped page-locked host copy), so one synchronisation returns both
cudaError_t launch_to_caller_order_f64(const float4* U, const float4* Ulo, const int* node_new_of_old, int N,
                                       double* out, cudaStream_t s, const DevState* st = nullptr,
                                       DevState* st_out = nullptr);
cudaError_t launch_copy_state(const DevState* st, DevState* st_out, cudaStream_t s);
cudaError_t launch_to_caller_order(const float4* U, const int* node_new_of_old, int N, float* out,
                                   cudaStream_t s);
// FP32 caller-order output (U + low part when Ulo is given), stores contiguous per warp
cudaError_t launch_to_caller_order_f32(const float4* U, const float4* Ulo, const int* node_new_of_old, int N,
                                       float* out, cudaStream_t s, const DevState* st = nullptr,
                                       DevState* st_out = nullptr);
// U (internal) = caller-order field (N x 3 floats); w of U and of V kept,
// U^n - U^{n-1} = 0, low part = 0
cudaError_t launch_from_caller_order(const float* src, const int* node_new_of_old, int N, float4* U,
                                     float4* V, float4* Ulo, cudaStream_t s);

}  // namespace dj
