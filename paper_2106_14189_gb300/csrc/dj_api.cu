// Host implementation of the C ABI declared in include/dj_tled.h.
//
// Data layout in device memory (E_pad = E rounded up to 128, internal order):
//   conn      int4[E_pad] (T4) or int4[2 E_pad] (H8)                16 / 32 B per element
//   consts    float[n_consts * E_pad], structure of arrays (dj_internal.h)
//   slots     float4[n_e * E_pad], element force of local node a at a * E_pad + e
//   sell      int[...] node -> slot ids, sliced ELL with chunks of 32 nodes
//   U, V      float4[N]: U^n (w = update coefficient a_i) and U^n - U^{n-1}
//             (w = index into the prescribed-node table, -1 if free)
//   bct       float4[n_bc_nodes]: target displacement, w = component mask
//   state     DevState (step counter, ramp value, error flags, residual sums)
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dj_internal.h"
#include "dj_io.h"

using namespace dj;

struct dj_mesh {
  int elem_type = 0, ne = 0;
  long long N = 0, E = 0;
  std::vector<double> X;
  std::vector<int> conn;
  bool materials_set = false;
  std::vector<unsigned char> model;
  std::vector<double> mu, kappa, rho, eta_a, eta_b, c01, adir, bdir;
  std::vector<long long> bc_dof;
  std::vector<double> bc_target;
  std::vector<double> R;
  std::vector<int> elem_group;  // independent bodies (caller element order), empty = one body
  int n_groups = 0;
  dj_params params{};
  // renumbering
  std::vector<int> node_new_of_old, node_old_of_new, elem_old_of_new;
  // device data
  bool precomputed = false;
  int device = -1;
  int E_pad = 0, n_consts = 0, off_fa = -1, off_fb = -1, off_mr = -1, off_hg = -1;
  int variant = VAR_NH, model_flags = 0;
  int4* d_conn = nullptr;
  float* d_consts = nullptr;
  float4* d_slots = nullptr;
  int* d_sell = nullptr;
  int* d_chunk_ptr = nullptr;
  float4* d_U = nullptr;
  float4* d_V = nullptr;
  float4* d_bct = nullptr;
  int* d_bc_flat = nullptr;  // bc_flat_of_entry on the device (target updates)
  float4* d_R = nullptr;
  float4* d_fout = nullptr;
  float4* d_Ulo = nullptr;  // compensated mode: low part of U
  int cmp = 0;
  float4* d_save = nullptr;  // dj_evaluate_field: saved U, V, low part (3 N), allocated on first use
  double* d_out64 = nullptr;  // dj_get_displacements: caller-order FP64 output (3 N), allocated on first use
  // groups: per-group time step, damping factor and residual
  std::vector<double> group_dt, group_dt_crit, group_r;
  std::vector<int> group_node_ptr;  // internal node range of each group
  float* d_bm1 = nullptr;
  double2* d_node_resid = nullptr;
  double2* d_group_resid = nullptr;
  int* d_group_node_ptr = nullptr;
  double2* h_group_resid = nullptr;  // pinned
  int* d_perm = nullptr;  // node_new_of_old on device
  DevState* d_state = nullptr;
  double2* d_partials = nullptr;
  DevState* h_state = nullptr;  // pinned
  int n_node_blocks = 0;
  int n_bc_nodes = 0;
  std::vector<int> bc_node_of_entry;  // per bc entry: prescribed-node row
  std::vector<int> bc_comp_of_entry;
  std::vector<int> bc_flat_of_entry;  // per bc entry: float index 4 row + comp in the node table
  std::vector<float4> h_bct;
  float4* h_bct_pinned = nullptr;  // pinned staging of h_bct for target updates
  std::vector<float> h_ai;
  std::vector<int> h_bcidx;
  double dt = 0, dt_crit = 0, total_mass = 0;
  float bm1 = 1.f;
  int threads_force = 256;
  long long device_bytes = 0;
  long long sell_entries = 0;
  // tiled assembly
  int assembly = ASSEMBLY_TILES, T = 0, n_tiles = 0, cap = 0, tma_grid = 0;
  long long n_parts = 0;
  int* d_tile_ptr = nullptr;
  int* d_tile_nodes = nullptr;
  unsigned short* d_lconn = nullptr;
  unsigned short* d_lptr = nullptr;
  unsigned short* d_lidx = nullptr;
  float4* d_xloc = nullptr;  // geometric table: tile-local reference coordinates
  int* d_pdst = nullptr;     // tiles: node-major position of each (tile, node) partial
  int* d_node_ptr = nullptr; // tiles: N + 1 offsets of each node's partials
  int geometric = 0;
  float4* d_parts = nullptr;
  cudaStream_t cap_stream = nullptr;
  int4* d_bc_entry = nullptr;    // per prescribed-node row: target entries of x, y, z (-1: free), mask
  double* d_tgt_stage = nullptr; // device copy of the caller's targets (dj_step_host; allocated on first use)
  bool targets_on_device = false;  // bc_target lags d_tgt_stage (dj_step_host)
  DevState* h_state_map = nullptr;  // device address of the page-locked state copy
  cudaGraphExec_t run_exec = nullptr;
  int run_chunk = 0;
  cudaGraphExec_t relax_exec = nullptr;
  int relax_k = 0;
  // adaptive dynamic relaxation (allocated on first use)
  // average nodal pressure (T4, bulk-copy tiles)
  int anp = 0;
  float* d_vparts = nullptr;  // per (tile, node): a quarter of the element volume changes
  float* d_c1 = nullptr;      // per node: kappa_i / V0_i
  float* d_pres = nullptr;    // per node: p_i
  AdrState* d_adr = nullptr;
  AdrState* h_adr = nullptr;  // pinned
  double* d_rq = nullptr;     // 4 sums per node block
  double4* d_usnap = nullptr; // U of the previous check (FP64)
  cudaGraphExec_t adr_exec = nullptr;
  int adr_k = 0;
  std::string last_error;
};

namespace {

inline float bits_to_float(int v) {
  float f;
  std::memcpy(&f, &v, 4);
  return f;
}
inline int float_to_bits(float f) {
  int v;
  std::memcpy(&v, &f, 4);
  return v;
}

dj_status fail(dj_mesh* m, dj_status s, const char* fmt, ...) {
  if (m) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    m->last_error = buf;
  }
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return fail(m, _e == cudaErrorMemoryAllocation ? DJ_ERR_OOM : DJ_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(_e), __FILE__, __LINE__);                          \
  } while (0)

// a named range around a library call for profilers (NVTX; no cost without a tool)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

template <class T>
cudaError_t dalloc(dj_mesh* m, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
  if (e == cudaSuccess) m->device_bytes += (long long)(count * sizeof(T));
  return e;
}

void release_device(dj_mesh* m) {
  if (m->run_exec) cudaGraphExecDestroy(m->run_exec);
  if (m->relax_exec) cudaGraphExecDestroy(m->relax_exec);
  if (m->adr_exec) cudaGraphExecDestroy(m->adr_exec);
  m->run_exec = m->relax_exec = m->adr_exec = nullptr;
  m->run_chunk = m->relax_k = m->adr_k = 0;
  if (m->h_adr) cudaFreeHost(m->h_adr);
  m->h_adr = nullptr;
  void* ptrs[] = {m->d_adr, m->d_rq, m->d_usnap, m->d_vparts, m->d_c1, m->d_pres,
                  m->d_conn,     m->d_consts,     m->d_slots, m->d_sell, m->d_chunk_ptr, m->d_U,
                  m->d_V,        m->d_bct,        m->d_R,     m->d_fout, m->d_perm,      m->d_state,
                  m->d_partials, m->d_tile_ptr,   m->d_tile_nodes, m->d_lconn, m->d_lptr, m->d_lidx, m->d_xloc, m->d_pdst, m->d_node_ptr, m->d_save, m->d_out64,
                  m->d_parts,    m->d_Ulo,        m->d_bm1,   m->d_node_resid, m->d_group_resid,
                  m->d_group_node_ptr, m->d_bc_flat};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  m->d_adr = nullptr;
  m->d_rq = nullptr;
  m->d_usnap = nullptr;
  m->d_vparts = m->d_c1 = m->d_pres = nullptr;
  m->d_tile_ptr = m->d_tile_nodes = nullptr;
  m->d_lconn = m->d_lptr = m->d_lidx = nullptr;
  m->d_xloc = nullptr;
  m->d_pdst = m->d_node_ptr = nullptr;
  m->d_parts = nullptr;
  m->d_Ulo = nullptr;
  m->d_save = nullptr;
  m->d_out64 = nullptr;
  m->d_bm1 = nullptr;
  m->d_node_resid = m->d_group_resid = nullptr;
  m->d_group_node_ptr = nullptr;
  m->d_bc_flat = nullptr;
  if (m->h_group_resid) cudaFreeHost(m->h_group_resid);
  m->h_group_resid = nullptr;
  if (m->h_state) cudaFreeHost(m->h_state);
  if (m->h_bct_pinned) cudaFreeHost(m->h_bct_pinned);
  m->h_bct_pinned = nullptr;
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  if (m->d_bc_entry) cudaFree(m->d_bc_entry);
  if (m->d_tgt_stage) cudaFree(m->d_tgt_stage);
  m->d_bc_entry = nullptr;
  m->d_tgt_stage = nullptr;
  m->h_state_map = nullptr;
  m->d_conn = nullptr;
  m->d_consts = nullptr;
  m->d_slots = nullptr;
  m->d_sell = nullptr;
  m->d_chunk_ptr = nullptr;
  m->d_U = m->d_V = m->d_bct = m->d_R = m->d_fout = nullptr;
  m->d_perm = nullptr;
  m->d_state = nullptr;
  m->d_partials = nullptr;
  m->h_state = nullptr;
  m->cap_stream = nullptr;
  m->device_bytes = 0;
  m->precomputed = false;
}

// Morton key of a point in the unit cube, 21 bits per axis
uint64_t spread21(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

std::vector<int> morton_order(const std::vector<double>& P, long long n) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (long long i = 0; i < n; ++i)
    for (int j = 0; j < 3; ++j) {
      lo[j] = std::min(lo[j], P[3 * i + j]);
      hi[j] = std::max(hi[j], P[3 * i + j]);
    }
  double ext = 0;
  for (int j = 0; j < 3; ++j) ext = std::max(ext, hi[j] - lo[j]);
  if (!(ext > 0)) ext = 1;
  std::vector<uint64_t> key(n);
  for (long long i = 0; i < n; ++i) {
    uint64_t k = 0;
    for (int j = 0; j < 3; ++j) {
      double t = (P[3 * i + j] - lo[j]) / ext;
      uint64_t q = (uint64_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
      k |= spread21(q) << j;
    }
    key[i] = k;
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
  return order;
}

int count_bits(int v) {
  int c = 0;
  while (v) {
    c += v & 1;
    v >>= 1;
  }
  return c;
}

dj_status read_state(dj_mesh* m, cudaStream_t s) {
  CK(cudaMemcpyAsync(m->h_state, m->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return DJ_OK;
}

dj_status check_flags(dj_mesh* m) {
  const DevState& st = *m->h_state;
  if (st.err_flags & ~ERR_BAD_TARGET) {
    const int be = st.bad_elem;
    const int caller = (be >= 0 && be < (int)m->E) ? m->elem_old_of_new[be] : -1;
    if (st.err_flags & ERR_INVERTED)
      return fail(m, DJ_ERR_INVERTED_ELEMENT, "element %d inverted (det tJ <= 0) by step %lld",
                  caller, st.step);
    if (st.err_flags & ERR_NONFINITE) {
      const int bn = st.bad_node;
      const int node = (bn >= 0 && bn < (int)m->N) ? m->node_old_of_new[bn] : -1;
      return fail(m, DJ_ERR_NONFINITE, "non-finite force or displacement at node %d by step %lld", node,
                  st.step);
    }
    return fail(m, DJ_ERR_CUDA, "a bounded device wait timed out by step %lld", st.step);
  }
  return DJ_OK;
}

// A new displacement field starts a new trajectory: its error record starts
// empty (err_flags = 0, bad_elem above every element id).
cudaError_t clear_error_flags(dj_mesh* m, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&m->d_state->err_flags, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&m->d_state->bad_elem, 0x7f, 2 * sizeof(int), s);  // and bad_node
  return e;
}

// byte extent of a tile's force records (n_e T float4), the largest slot byte offset + 16
long long T_slots_bytes(const dj_mesh* m) { return (long long)m->ne * m->T * 16; }

// Sliced ELL (chunks of SELL_C rows, column-major, -1 padding) of CSR lists.
void build_sell(const std::vector<int>& ptr, const std::vector<int>& idx, long long N,
                std::vector<int>& chunk_ptr, std::vector<int>& sell) {
  const long long n_chunks = (N + SELL_C - 1) / SELL_C;
  chunk_ptr.assign(n_chunks + 1, 0);
  for (long long c = 0; c < n_chunks; ++c) {
    int w = 0;
    for (long long i = c * SELL_C; i < std::min(N, (c + 1) * SELL_C); ++i) w = std::max(w, ptr[i + 1] - ptr[i]);
    chunk_ptr[c + 1] = chunk_ptr[c] + w * SELL_C;
  }
  sell.assign(chunk_ptr[n_chunks], -1);
  for (long long i = 0; i < N; ++i) {
    const long long c = i / SELL_C, lane = i % SELL_C;
    for (int j = 0; j < ptr[i + 1] - ptr[i]; ++j) sell[chunk_ptr[c] + j * SELL_C + lane] = idx[ptr[i] + j];
  }
}

// Shared-memory positions of a tile's nodes.  The element phase reads the
// staged U and reference coordinates of each element's nodes with 16-byte
// loads; eight consecutive lanes (elements) share a wavefront when the
// distinct positions they touch fall in distinct groups of four banks
// (position mod 8), and each extra node in a group costs one more.  The
// groups are given greedily: nodes in descending record count, each to the
// group, among those with room left, that adds the fewest such conflicts
// over the eight-element blocks that read it; within a group the nodes keep
// descending record count.  `lnode` holds the local node (index into the
// tile's sorted node list) of record (e, b), e < n_el; the result maps that
// index to a position in [0, n_t).  Only the layout changes: every node's
// sum keeps its order of additions.
std::vector<int> bank_positions(int n_t, const std::vector<int>& lnode, int n_el, int ne,
                                const std::vector<int>& deg) {
  constexpr int G = 8, W = 8;  // bank groups of a 16-byte load; lanes of one wavefront
  const int n_sets = (n_el + W - 1) / W * ne;
  // the distinct nodes of each (eight-element block, local node b) set, and
  // the sets of each node
  std::vector<std::array<int, W>> setn(n_sets);
  std::vector<int> setsz(n_sets, 0), ptr(n_t + 1, 0);
  for (int qd = 0; qd * W < n_el; ++qd)
    for (int b = 0; b < ne; ++b) {
      const int si = qd * ne + b;
      for (int j = 0; j < W && qd * W + j < n_el; ++j) {
        const int k = lnode[(size_t)(qd * W + j) * ne + b];
        if (std::find(setn[si].begin(), setn[si].begin() + setsz[si], k) == setn[si].begin() + setsz[si]) {
          setn[si][setsz[si]++] = k;
          ptr[k + 1]++;
        }
      }
    }
  for (int k = 0; k < n_t; ++k) ptr[k + 1] += ptr[k];
  std::vector<int> memb(ptr[n_t]), fill(ptr.begin(), ptr.end() - 1);
  for (int si = 0; si < n_sets; ++si)
    for (int q = 0; q < setsz[si]; ++q) memb[fill[setn[si][q]]++] = si;
  std::vector<std::array<int, G>> cnt(n_sets);
  for (auto& c : cnt) c.fill(0);
  std::vector<int> mx(n_sets, 0), room(G, 0), grp(n_t, 0), order(n_t);
  for (int p = 0; p < n_t; ++p) room[p % G]++;
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return deg[x] > deg[y]; });
  for (int k : order) {
    int best = -1, best_add = INT_MAX;
    for (int g = 0; g < G; ++g) {
      if (!room[g]) continue;
      int add = 0;
      for (int q = ptr[k]; q < ptr[k + 1]; ++q) add += cnt[memb[q]][g] + 1 > mx[memb[q]] ? 1 : 0;
      if (add < best_add) best_add = add, best = g;
    }
    grp[k] = best;
    room[best]--;
    for (int q = ptr[k]; q < ptr[k + 1]; ++q) mx[memb[q]] = std::max(mx[memb[q]], ++cnt[memb[q]][best]);
  }
  // positions g, g + 8, ... of each group, in descending record count
  std::vector<int> pos(n_t), next(G);
  for (int g = 0; g < G; ++g) next[g] = g;
  for (int k : order) {
    pos[k] = next[grp[k]];
    next[grp[k]] += G;
  }
  return pos;
}

ForceArgs force_args(dj_mesh* m, int advance) {
  ForceArgs a;
  a.conn = m->d_conn;
  a.consts = m->d_consts;
  a.U = m->d_U;
  a.Ulo = m->d_Ulo;
  a.slots = m->d_slots;
  a.E = (int)m->E;
  a.E_pad = m->E_pad;
  a.off_fa = m->off_fa;
  a.off_fb = m->off_fb;
  a.off_mr = m->off_mr;
  a.off_hg = m->off_hg;
  a.st = m->d_state;
  a.advance = advance;
  a.ramp_steps = m->params.ramp_steps;
  a.ramp_kind = m->params.ramp_kind;
  a.pres = m->d_pres;
  a.tgt_src = nullptr;
  a.tgt_dst = nullptr;
  a.n_tgt = 0;
  return a;
}

TileArgs tile_args(dj_mesh* m) {
  TileArgs t;
  t.tile_ptr = m->d_tile_ptr;
  t.tnodes = m->d_tile_nodes;
  t.lconn = m->d_lconn;
  t.lptr = m->d_lptr;
  t.lidx = m->d_lidx;
  t.xloc = m->d_xloc;
  t.pdst = m->d_pdst;
  t.partials = m->d_parts;
  t.T = m->T;
  t.cap = m->cap;
  t.n_consts = m->n_consts;
  t.n_tiles = m->n_tiles;
  return t;
}

// tgt_src: the step's targets in the caller's page-locked array (device
// address of its mapping), copied by the force kernel into d_tgt_stage
cudaError_t launch_force_any(dj_mesh* m, int advance, cudaStream_t s, const double* tgt_src = nullptr) {
  if (m->anp) {  // nodal pressures of U^n first
    cudaError_t e = launch_anp(m->cmp, tile_args(m), m->d_node_ptr, m->d_U, m->d_Ulo, (int)m->E, (int)m->N,
                               m->d_vparts, m->d_c1, m->d_pres, s);
    if (e != cudaSuccess) return e;
  }
  ForceArgs a = force_args(m, advance);
  if (tgt_src) {
    a.tgt_src = tgt_src;
    a.tgt_dst = m->d_tgt_stage;
    a.n_tgt = (int)m->bc_dof.size();
  }
  if (m->assembly == ASSEMBLY_TILES_TMA)
    return launch_force_tma(m->elem_type, m->variant, m->cmp, m->anp, a, tile_args(m), m->tma_grid, s);
  if (m->assembly == ASSEMBLY_TILES)
    return launch_force_tiled(m->elem_type, m->variant, m->cmp, a, tile_args(m), m->n_tiles, s);
  return launch_force(m->elem_type, m->variant, m->cmp, a, m->threads_force, s);
}

NodeArgs node_args(dj_mesh* m) {
  NodeArgs a;
  a.sell = m->d_sell;
  a.chunk_ptr = m->d_chunk_ptr;
  a.node_ptr = m->assembly != ASSEMBLY_SLOTS ? m->d_node_ptr : nullptr;
  a.slots = m->assembly != ASSEMBLY_SLOTS ? m->d_parts : m->d_slots;
  a.U = m->d_U;
  a.Ulo = m->d_Ulo;
  a.V = m->d_V;
  a.bct = m->d_bct;
  a.R = m->d_R;
  a.fout = m->d_fout;
  a.partials = m->d_partials;
  a.node_resid = m->n_groups > 0 ? m->d_node_resid : nullptr;
  a.bm1_node = m->d_bm1;
  a.st = m->d_state;
  a.tgt = nullptr;
  a.bc_entry = m->d_bc_entry;
  a.adr = m->d_adr;
  a.rq_partials = m->d_rq;
  a.usnap = m->d_usnap;
  a.N = (int)m->N;
  a.bm1 = m->bm1;
  return a;
}

cudaError_t launch_step(dj_mesh* m, cudaStream_t s, int mode) {
  cudaError_t e = launch_force_any(m, 1, s);
  if (e != cudaSuccess) return e;
  e = launch_node(mode, m->cmp, node_args(m), s);
  if (e != cudaSuccess) return e;
  if (mode == NODE_UPDATE_RESID || mode == NODE_ADR_RQ) {
    if (m->n_groups > 0)
      e = launch_group_resid(m->d_node_resid, m->d_group_node_ptr, m->n_groups, m->d_group_resid, s);
    else
      e = launch_resid_finalize(m->d_partials, m->n_node_blocks, m->d_state, s);
  }
  if (e == cudaSuccess && mode == NODE_ADR_RQ)
    e = launch_adr_finalize(m->d_rq, m->n_node_blocks, m->d_state, m->d_adr, s);
  return e;
}

dj_status need_ready(dj_mesh* m) {
  if (!m) return DJ_ERR_INVALID_ARG;
  if (!m->precomputed) return fail(m, DJ_ERR_NOT_PRECOMPUTED, "call dj_precompute first");
  CK(cudaSetDevice(m->device));
  (void)cudaGetLastError();  // drop a non-sticky error left by an earlier failed call
  return DJ_OK;
}

// Capture `body` on the mesh's capture stream into an executable graph.
template <class F>
dj_status capture(dj_mesh* m, cudaGraphExec_t* out, F body) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
  tl_graph_pdl = m->params.graph_pdl != 0;
  cudaError_t be = body(m->cap_stream);
  tl_graph_pdl = false;
  cudaError_t ee = cudaStreamEndCapture(m->cap_stream, &g);
  if (be != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(m, DJ_ERR_CUDA, "graph capture: %s", cudaGetErrorString(be));
  }
  CK(ee);
  cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(ie);
  return DJ_OK;
}

}  // namespace

namespace {
// After dj_step_host the host copy of the targets lags the device copy: bring
// it up to date (non-finite entries, which were not applied, keep their value).
dj_status sync_host_targets(dj_mesh* m) {
  if (!m->targets_on_device || !m->d_tgt_stage) {
    m->targets_on_device = false;
    return DJ_OK;
  }
  const size_t nb = m->bc_dof.size();
  std::vector<double> t(nb);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(t.data(), m->d_tgt_stage, nb * sizeof(double), cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < nb; ++k)
    if (std::isfinite(t[k])) m->bc_target[k] = t[k];
  m->targets_on_device = false;
  return DJ_OK;
}
}  // namespace

namespace dj {
// accessors for the warm-start layer (warmstart.cu)
const std::vector<long long>& mesh_bc_dofs(const dj_mesh* m) { return m->bc_dof; }
long long mesh_ramp_steps(const dj_mesh* m) { return m->params.ramp_steps; }
long long mesh_n_nodes(const dj_mesh* m) { return m->N; }
}  // namespace dj

extern "C" {

void dj_params_default(dj_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dt = 0.0;
  p->dt_scale = 0.9;
  p->alpha = 0.0;
  p->hg_coeff = 0.1;
  p->ramp_steps = 0;
  p->ramp_kind = DJ_RAMP_SMOOTH;
  p->relax_check_every = 100;
  p->renumber = 1;
  p->assembly = ASSEMBLY_TILES;
  p->tile_size = 0;
  p->precision = 0;
  p->anp = 0;
  p->graph_pdl = 0;
}

const char* dj_status_string(dj_status s) {
  switch (s) {
    case DJ_OK: return "ok";
    case DJ_ERR_INVALID_ARG: return "invalid argument";
    case DJ_ERR_BAD_MESH: return "bad mesh";
    case DJ_ERR_INVERTED_ELEMENT: return "inverted element";
    case DJ_ERR_NOT_PRECOMPUTED: return "not precomputed";
    case DJ_ERR_NONFINITE: return "non-finite value";
    case DJ_ERR_NOT_CONVERGED: return "not converged";
    case DJ_ERR_CUDA: return "CUDA error";
    case DJ_ERR_OOM: return "out of memory";
    case DJ_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* dj_last_error(const dj_mesh* m) { return m ? m->last_error.c_str() : "null mesh"; }

dj_status dj_mesh_create(int elem_type, const double* X, long long n_nodes, const int* conn,
                         long long n_elems, dj_mesh** out) {
  if (!out) return DJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (elem_type != DJ_TET4 && elem_type != DJ_HEX8) return DJ_ERR_INVALID_ARG;
  if (n_nodes <= 0 || n_elems <= 0) return DJ_ERR_BAD_MESH;
  if (!X || !conn) return DJ_ERR_INVALID_ARG;
  if (n_nodes >= INT_MAX / 2 || (long long)elem_type * (n_elems + 128) >= INT_MAX)
    return DJ_ERR_UNSUPPORTED;
  for (long long i = 0; i < 3 * n_nodes; ++i)
    if (!std::isfinite(X[i])) return DJ_ERR_INVALID_ARG;
  for (long long i = 0; i < elem_type * n_elems; ++i)
    if (conn[i] < 0 || conn[i] >= n_nodes) return DJ_ERR_BAD_MESH;
  dj_mesh* m = new (std::nothrow) dj_mesh();
  if (!m) return DJ_ERR_OOM;
  m->elem_type = elem_type;
  m->ne = elem_type;
  m->N = n_nodes;
  m->E = n_elems;
  m->X.assign(X, X + 3 * n_nodes);
  m->conn.assign(conn, conn + elem_type * n_elems);
  dj_params_default(&m->params);
  *out = m;
  return DJ_OK;
}

dj_status dj_mesh_set_materials(dj_mesh* m, const unsigned char* model, const double* mu,
                                const double* kappa, const double* rho, const double* eta_a,
                                const double* eta_b, const double* c01, const double* a_dir,
                                const double* b_dir) {
  if (!m) return DJ_ERR_INVALID_ARG;
  if (!model || !mu || !kappa || !rho)
    return fail(m, DJ_ERR_INVALID_ARG, "model, mu, kappa and rho are required");
  const long long E = m->E;
  for (long long e = 0; e < E; ++e) {
    if (model[e] > DJ_MR) return fail(m, DJ_ERR_INVALID_ARG, "element %lld: unknown model", e);
    if (!(mu[e] > 0) || !(kappa[e] > 0) || !(rho[e] > 0) || !std::isfinite(mu[e]) ||
        !std::isfinite(kappa[e]) || !std::isfinite(rho[e]))
      return fail(m, DJ_ERR_INVALID_ARG, "element %lld: mu, kappa, rho must be finite and > 0", e);
    const double ea = eta_a ? eta_a[e] : 0.0, eb = eta_b ? eta_b[e] : 0.0, c = c01 ? c01[e] : 0.0;
    if (!(ea >= 0) || !(eb >= 0) || !(c >= 0) || !std::isfinite(ea + eb + c))
      return fail(m, DJ_ERR_INVALID_ARG, "element %lld: eta and c01 must be finite and >= 0", e);
    if ((model[e] == DJ_TI || model[e] == DJ_OT) && ea > 0) {
      const double* d = a_dir ? a_dir + 3 * e : nullptr;
      if (d && !(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] > 0))
        return fail(m, DJ_ERR_INVALID_ARG, "element %lld: zero fibre direction a", e);
    }
    if (model[e] == DJ_OT && eb > 0) {
      const double* d = b_dir ? b_dir + 3 * e : nullptr;
      if (d && !(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] > 0))
        return fail(m, DJ_ERR_INVALID_ARG, "element %lld: zero fibre direction b", e);
    }
  }
  m->model.assign(model, model + E);
  m->mu.assign(mu, mu + E);
  m->kappa.assign(kappa, kappa + E);
  m->rho.assign(rho, rho + E);
  m->eta_a.assign(E, 0.0);
  m->eta_b.assign(E, 0.0);
  m->c01.assign(E, 0.0);
  if (eta_a) m->eta_a.assign(eta_a, eta_a + E);
  if (eta_b) m->eta_b.assign(eta_b, eta_b + E);
  if (c01) m->c01.assign(c01, c01 + E);
  m->adir.resize(3 * E);
  m->bdir.resize(3 * E);
  for (long long e = 0; e < E; ++e) {
    for (int j = 0; j < 3; ++j) {
      m->adir[3 * e + j] = a_dir ? a_dir[3 * e + j] : (j == 0 ? 1.0 : 0.0);
      m->bdir[3 * e + j] = b_dir ? b_dir[3 * e + j] : (j == 1 ? 1.0 : 0.0);
    }
  }
  m->materials_set = true;
  m->precomputed = false;
  return DJ_OK;
}

dj_status dj_mesh_set_bcs(dj_mesh* m, const long long* dof, const double* target, long long n) {
  if (!m) return DJ_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!dof || !target))) return fail(m, DJ_ERR_INVALID_ARG, "bad bc arrays");
  std::vector<char> seen(3 * m->N, 0);
  for (long long k = 0; k < n; ++k) {
    if (dof[k] < 0 || dof[k] >= 3 * m->N)
      return fail(m, DJ_ERR_INVALID_ARG, "bc entry %lld: dof %lld out of range", k, dof[k]);
    if (seen[dof[k]]) return fail(m, DJ_ERR_INVALID_ARG, "bc entry %lld: duplicate dof %lld", k, dof[k]);
    if (!std::isfinite(target[k])) return fail(m, DJ_ERR_INVALID_ARG, "bc entry %lld: non-finite", k);
    seen[dof[k]] = 1;
  }
  m->bc_dof.assign(dof, dof + n);
  m->bc_target.assign(target, target + n);
  m->targets_on_device = false;
  m->precomputed = false;
  return DJ_OK;
}

dj_status dj_mesh_set_groups(dj_mesh* m, const int* elem_group, int n_groups) {
  if (!m) return DJ_ERR_INVALID_ARG;
  if (!elem_group || n_groups <= 0) {
    m->elem_group.clear();
    m->n_groups = 0;
    m->precomputed = false;
    return DJ_OK;
  }
  std::vector<int> node_group(m->N, -1);
  for (long long e = 0; e < m->E; ++e) {
    const int g = elem_group[e];
    if (g < 0 || g >= n_groups) return fail(m, DJ_ERR_INVALID_ARG, "element %lld: group %d out of range", e, g);
    for (int b = 0; b < m->ne; ++b) {
      int& ng = node_group[m->conn[e * m->ne + b]];
      if (ng >= 0 && ng != g)
        return fail(m, DJ_ERR_INVALID_ARG, "node %d is shared by groups %d and %d", m->conn[e * m->ne + b], ng, g);
      ng = g;
    }
  }
  m->elem_group.assign(elem_group, elem_group + m->E);
  m->n_groups = n_groups;
  m->precomputed = false;
  return DJ_OK;
}

dj_status dj_mesh_set_loads(dj_mesh* m, const double* R) {
  if (!m) return DJ_ERR_INVALID_ARG;
  if (!R) {
    m->R.clear();
  } else {
    for (long long i = 0; i < 3 * m->N; ++i)
      if (!std::isfinite(R[i]) || std::fabs(R[i]) > 3.0e38)
        return fail(m, DJ_ERR_INVALID_ARG, "load not finite in single precision");
    m->R.assign(R, R + 3 * m->N);
  }
  m->precomputed = false;
  return DJ_OK;
}

dj_status dj_precompute(dj_mesh* m, const dj_params* p, double* dt_out) {
  const Range range("dj_precompute");
  if (!m) return DJ_ERR_INVALID_ARG;
  if (!m->materials_set) return fail(m, DJ_ERR_INVALID_ARG, "call dj_mesh_set_materials first");
  if (m->precomputed) {
    dj_status ts = sync_host_targets(m);
    if (ts) return ts;
  }
  dj_params prm;
  if (p)
    prm = *p;
  else
    dj_params_default(&prm);
  if (!(prm.dt_scale > 0) || !(prm.alpha >= 0) || !(prm.hg_coeff >= 0) || prm.relax_check_every <= 0 ||
      (prm.ramp_kind != DJ_RAMP_LINEAR && prm.ramp_kind != DJ_RAMP_SMOOTH) || !std::isfinite(prm.dt) ||
      (prm.assembly != ASSEMBLY_SLOTS && prm.assembly != ASSEMBLY_TILES && prm.assembly != ASSEMBLY_TILES_TMA) ||
      (prm.precision != 0 && prm.precision != 1) || (prm.anp != 0 && prm.anp != 1) ||
      (prm.graph_pdl != 0 && prm.graph_pdl != 1) || prm.max_blocks < 0)
    return fail(m, DJ_ERR_INVALID_ARG, "invalid dj_params");
  if (prm.anp && (m->ne != 4 || prm.assembly != ASSEMBLY_TILES_TMA))
    return fail(m, DJ_ERR_INVALID_ARG, "average nodal pressure needs T4 elements and assembly 2");
  {
    const int tmax = prm.assembly == ASSEMBLY_TILES_TMA ? 256 : (m->ne == 4 ? 512 : 256);
    if (prm.tile_size < 0 || prm.tile_size % 32 != 0 || prm.tile_size > tmax)
      return fail(m, DJ_ERR_INVALID_ARG, "tile_size must be a multiple of 32 and <= %d", tmax);
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  (void)cudaGetLastError();
  release_device(m);
  m->device = dev;
  m->params = prm;
  const long long N = m->N, E = m->E;
  const int ne = m->ne;
  // ---- renumbering (caller -> internal) --------------------------------
  m->node_old_of_new.resize(N);
  m->elem_old_of_new.resize(E);
  std::vector<int> node_group_c;  // caller order
  if (m->n_groups > 0) {
    node_group_c.assign(N, 0);
    for (long long e = 0; e < E; ++e)
      for (int b = 0; b < ne; ++b) node_group_c[m->conn[e * ne + b]] = m->elem_group[e];
  }
  if (prm.renumber) {
    m->node_old_of_new = morton_order(m->X, N);
  } else {
    std::iota(m->node_old_of_new.begin(), m->node_old_of_new.end(), 0);
  }
  if (m->n_groups > 0)  // group-major: every group is a contiguous range of nodes and elements
    std::stable_sort(m->node_old_of_new.begin(), m->node_old_of_new.end(),
                     [&](int a, int b) { return node_group_c[a] < node_group_c[b]; });
  m->node_new_of_old.assign(N, 0);
  for (long long i = 0; i < N; ++i) m->node_new_of_old[m->node_old_of_new[i]] = (int)i;
  if (prm.renumber) {
    std::vector<double> cen(3 * E, 0.0);
    for (long long e = 0; e < E; ++e)
      for (int b = 0; b < ne; ++b)
        for (int j = 0; j < 3; ++j) cen[3 * e + j] += m->X[3 * (size_t)m->conn[e * ne + b] + j] / ne;
    m->elem_old_of_new = morton_order(cen, E);
  } else {
    std::iota(m->elem_old_of_new.begin(), m->elem_old_of_new.end(), 0);
  }
  if (m->n_groups > 0) {
    std::stable_sort(m->elem_old_of_new.begin(), m->elem_old_of_new.end(),
                     [&](int a, int b) { return m->elem_group[a] < m->elem_group[b]; });
    m->group_node_ptr.assign(m->n_groups + 1, 0);
    for (long long i = 0; i < N; ++i) m->group_node_ptr[node_group_c[i] + 1]++;
    for (int g = 0; g < m->n_groups; ++g) m->group_node_ptr[g + 1] += m->group_node_ptr[g];
  }
  std::vector<double> Xn(3 * N);
  for (long long i = 0; i < N; ++i)
    for (int j = 0; j < 3; ++j) Xn[3 * i + j] = m->X[3 * (size_t)m->node_old_of_new[i] + j];
  std::vector<int> cn((size_t)E * ne);
  for (long long e = 0; e < E; ++e)
    for (int b = 0; b < ne; ++b)
      cn[e * ne + b] = m->node_new_of_old[m->conn[(size_t)m->elem_old_of_new[e] * ne + b]];
  // ---- table layout ---------------------------------------------------------
  m->E_pad = (int)((E + 127) / 128 * 128);
  const int E_pad = m->E_pad;
  m->model_flags = 0;
  for (long long e = 0; e < E; ++e) m->model_flags |= 1 << m->model[e];
  bool fa = false, fb = false, mr = (m->model_flags >> DJ_MR) & 1;
  for (long long e = 0; e < E; ++e) {
    if ((m->model[e] == DJ_TI || m->model[e] == DJ_OT) && m->eta_a[e] > 0) fa = true;
    if (m->model[e] == DJ_OT && m->eta_b[e] > 0) fb = true;
  }
  // kernel variant, then the table blocks it reads (unused fibre blocks hold zeros)
  if (fb) fa = true;
  if (mr && fa) {
    m->variant = VAR_ALL;
    fb = true;
  } else if (mr) {
    m->variant = VAR_MR;
  } else if (fb) {
    m->variant = VAR_OT;
  } else if (fa) {
    m->variant = VAR_TI;
  } else {
    m->variant = VAR_NH;
  }
  // tiled meshes rebuild 0J, det 0J, P (and the H8 hourglass c) from staged
  // reference coordinates
  m->geometric = prm.assembly != ASSEMBLY_SLOTS;
  int nc = m->geometric ? KG_COMMON : K_COMMON;
  m->off_fa = m->off_fb = m->off_mr = m->off_hg = -1;
  if (fa) { m->off_fa = nc; nc += 7; }
  if (fb) { m->off_fb = nc; nc += 7; }
  if (mr) { m->off_mr = nc; nc += 1; }
  if (ne == 8) { m->off_hg = nc; nc += m->geometric ? 1 : 13; }
  m->n_consts = nc;
  m->threads_force = ne == 4 ? 256 : 128;
  // ---- gather index: node -> slots (ascending element, local node) ---------
  std::vector<int> cnt(N + 1, 0);
  for (size_t k = 0; k < cn.size(); ++k) cnt[cn[k] + 1]++;
  for (long long i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> csr(cn.size()), fillp(cnt.begin(), cnt.end() - 1);
  for (long long e = 0; e < E; ++e)
    for (int b = 0; b < ne; ++b) csr[fillp[cn[e * ne + b]]++] = b * E_pad + (int)e;
  std::vector<int> chunk_ptr, sell;
  build_sell(cnt, csr, N, chunk_ptr, sell);  // node -> element slots (lumped mass, slot assembly)
  m->assembly = prm.assembly;
  std::vector<int> tile_ptr, tile_nodes, tnodes_pad;
  std::vector<float4> xloc_pad;
  std::vector<int> node_ptr, pdst_pad;
  std::vector<unsigned short> lconn, lptr, lidx;
  if (m->assembly != ASSEMBLY_SLOTS) {
    const int T = prm.tile_size > 0 ? prm.tile_size : (ne == 4 ? 256 : 128);
    m->T = T;
    m->n_tiles = (int)((E + T - 1) / T);
    tile_ptr.assign(m->n_tiles + 1, 0);
    lconn.assign((size_t)m->n_tiles * T * ne, 0);
    lidx.assign((size_t)m->n_tiles * T * ne, 0);
    std::vector<std::vector<int>> tile_loc(m->n_tiles);
    std::vector<std::vector<unsigned short>> tile_lptr(m->n_tiles);
    std::vector<int> tile_x0(m->n_tiles);  // smallest node id of the tile: origin of xloc
    int smax = 0;
    std::vector<int> loc;
    for (int t = 0; t < m->n_tiles; ++t) {
      const long long e0 = (long long)t * T, e1 = std::min(E, e0 + T);
      loc.assign(cn.begin() + e0 * ne, cn.begin() + e1 * ne);
      std::sort(loc.begin(), loc.end());
      loc.erase(std::unique(loc.begin(), loc.end()), loc.end());
      const int n_t = (int)loc.size();
      smax = std::max(smax, n_t);
      tile_ptr[t + 1] = tile_ptr[t] + n_t;
      tile_x0[t] = loc[0];
      // local node positions: chosen against the shared-memory bank conflicts
      // of the element phase's node loads (bank_positions)
      std::vector<int> deg(n_t, 0), lnode((size_t)(e1 - e0) * ne), ord(n_t);
      for (long long e = e0; e < e1; ++e)
        for (int b = 0; b < ne; ++b) {
          const int k = (int)(std::lower_bound(loc.begin(), loc.end(), cn[e * ne + b]) - loc.begin());
          lnode[(size_t)(e - e0) * ne + b] = k;
          deg[k]++;
        }
      const std::vector<int> pos = bank_positions(n_t, lnode, (int)(e1 - e0), ne, deg);
      for (int k = 0; k < n_t; ++k) ord[pos[k]] = k;
      // local connectivity and the per-node slot lists (ascending element, then local node)
      std::vector<int> kcnt(n_t + 1, 0);
      for (long long e = e0; e < e1; ++e)
        for (int b = 0; b < ne; ++b) {
          const int k = pos[std::lower_bound(loc.begin(), loc.end(), cn[e * ne + b]) - loc.begin()];
          lconn[e * ne + b] = (unsigned short)k;
          kcnt[k + 1]++;
        }
      std::vector<int> reordered(n_t);
      for (int k = 0; k < n_t; ++k) reordered[k] = loc[ord[k]];
      loc.swap(reordered);
      tile_nodes.insert(tile_nodes.end(), loc.begin(), loc.end());
      for (int k = 0; k < n_t; ++k) kcnt[k + 1] += kcnt[k];
      for (int k = 0; k <= n_t; ++k) tile_lptr[t].push_back((unsigned short)kcnt[k]);
      std::vector<int> fillk(kcnt.begin(), kcnt.end() - 1);
      for (long long e = e0; e < e1; ++e)
        for (int b = 0; b < ne; ++b) {
          const int k = lconn[e * ne + b];
          lidx[(size_t)t * T * ne + fillk[k]++] = (unsigned short)(b * T + (int)(e - e0));
        }
      tile_loc[t] = loc;
    }
    m->cap = (smax + 7) / 8 * 8;
    m->n_parts = tile_ptr[m->n_tiles];
    // fixed-size per-tile segments
    tnodes_pad.assign((size_t)m->n_tiles * m->cap, 0);
    lptr.assign((size_t)m->n_tiles * (m->cap + 8), 0);
    for (int t = 0; t < m->n_tiles; ++t) {
      std::copy(tile_loc[t].begin(), tile_loc[t].end(), tnodes_pad.begin() + (size_t)t * m->cap);
      std::copy(tile_lptr[t].begin(), tile_lptr[t].end(), lptr.begin() + (size_t)t * (m->cap + 8));
    }
    if (m->geometric) {
      // reference coordinates relative to the tile's node of smallest id, formed
      // in FP64 and rounded once, so that FP32 differences keep the element's scale
      xloc_pad.assign((size_t)m->n_tiles * m->cap, make_float4(0.f, 0.f, 0.f, 0.f));
      for (int t = 0; t < m->n_tiles; ++t) {
        const double* x0 = &Xn[3 * (size_t)tile_x0[t]];
        for (size_t q = 0; q < tile_loc[t].size(); ++q) {
          const double* x = &Xn[3 * (size_t)tile_loc[t][q]];
          xloc_pad[(size_t)t * m->cap + q] =
              make_float4((float)(x[0] - x0[0]), (float)(x[1] - x0[1]), (float)(x[2] - x0[2]), 0.f);
        }
      }
    }
    // node-major order of the partials: node i owns [node_ptr[i], node_ptr[i+1]),
    // ascending tile; every (tile, local node) gets its destination there
    node_ptr.assign(N + 1, 0);
    for (int v : tile_nodes) node_ptr[v + 1]++;
    for (long long i = 0; i < N; ++i) node_ptr[i + 1] += node_ptr[i];
    std::vector<int> fillp(node_ptr.begin(), node_ptr.end() - 1);
    pdst_pad.assign((size_t)m->n_tiles * m->cap, 0);
    for (int t = 0; t < m->n_tiles; ++t)
      for (int q = 0; q < tile_ptr[t + 1] - tile_ptr[t]; ++q)
        pdst_pad[(size_t)t * m->cap + q] = fillp[tile_nodes[tile_ptr[t] + q]]++;
    // every index the kernels follow, checked once on the host: a table that
    // would send a kernel out of bounds is refused before anything runs
    std::vector<char> seen(m->T * ne);
    for (int t = 0; t < m->n_tiles; ++t) {
      const int n_t = tile_ptr[t + 1] - tile_ptr[t];
      const long long e0 = (long long)t * m->T, e1 = std::min(E, e0 + m->T);
      const int R = (int)((e1 - e0) * ne);
      const unsigned short* lp = &lptr[(size_t)t * (m->cap + 8)];
      bool ok = n_t >= 1 && n_t <= m->cap && lp[0] == 0 && lp[n_t] == R;
      for (int q = 0; ok && q < n_t; ++q) {
        ok = lp[q] <= lp[q + 1] && tnodes_pad[(size_t)t * m->cap + q] >= 0 &&
             tnodes_pad[(size_t)t * m->cap + q] < N && pdst_pad[(size_t)t * m->cap + q] >= 0 &&
             pdst_pad[(size_t)t * m->cap + q] < m->n_parts;
      }
      std::fill(seen.begin(), seen.end(), 0);
      for (long long e = e0; ok && e < e1; ++e)
        for (int b = 0; ok && b < ne; ++b) ok = lconn[e * ne + b] < n_t;
      // node k's list holds each of its records (slot b T + e_local) once
      const unsigned short* li = &lidx[(size_t)t * m->T * ne];
      for (int k = 0; ok && k < n_t; ++k)
        for (int p = lp[k]; ok && p < lp[k + 1]; ++p) {
          const int slot = li[p], b = slot / m->T, el = slot % m->T;
          ok = b < ne && e0 + el < e1 && !seen[slot] && lconn[(e0 + el) * ne + b] == k;
          if (ok) seen[slot] = 1;
        }
      if (!ok) {
        return fail(m, DJ_ERR_BAD_MESH, "internal error: tile %d tables out of range", t);
      }
    }
    for (long long i = 0; i < N; ++i)
      if (node_ptr[i] > node_ptr[i + 1]) return fail(m, DJ_ERR_BAD_MESH, "internal error: node offsets");
    if (node_ptr[N] != m->n_parts) return fail(m, DJ_ERR_BAD_MESH, "internal error: partial count");
  }
  m->sell_entries = (long long)sell.size();
  // ---- prescribed nodes ----------------------------------------------------
  std::vector<int> bcidx(N, -1);
  m->h_bct.clear();
  m->bc_node_of_entry.assign(m->bc_dof.size(), 0);
  m->bc_comp_of_entry.assign(m->bc_dof.size(), 0);
  m->bc_flat_of_entry.assign(m->bc_dof.size(), 0);
  for (size_t k = 0; k < m->bc_dof.size(); ++k) {
    const int node = m->node_new_of_old[m->bc_dof[k] / 3];
    const int comp = (int)(m->bc_dof[k] % 3);
    if (bcidx[node] < 0) {
      bcidx[node] = (int)m->h_bct.size();
      m->h_bct.push_back(make_float4(0.f, 0.f, 0.f, bits_to_float(0)));
    }
    float4& t = m->h_bct[bcidx[node]];
    int mask = float_to_bits(t.w) | (1 << comp);
    if (comp == 0) t.x = (float)m->bc_target[k];
    if (comp == 1) t.y = (float)m->bc_target[k];
    if (comp == 2) t.z = (float)m->bc_target[k];
    t.w = bits_to_float(mask);
    m->bc_node_of_entry[k] = bcidx[node];
    m->bc_comp_of_entry[k] = comp;
    m->bc_flat_of_entry[k] = 4 * bcidx[node] + comp;
  }
  m->n_bc_nodes = (int)m->h_bct.size();
  m->h_bcidx = bcidx;
  // ---- device buffers --------------------------------------------------------
  const size_t conn4_count = (size_t)E_pad * (ne / 4);
  CK(dalloc(m, &m->d_conn, conn4_count));
  CK(cudaMemset(m->d_conn, 0, conn4_count * sizeof(int4)));
  const size_t table_floats = m->assembly != ASSEMBLY_SLOTS ? (size_t)m->n_tiles * nc * m->T : (size_t)nc * E_pad;
  CK(dalloc(m, &m->d_consts, table_floats));
  CK(cudaMemset(m->d_consts, 0, table_floats * sizeof(float)));
  int* d_mass_sell = nullptr;  // node -> element slots, for the lumped mass (tiled mode)
  int* d_mass_chunk = nullptr;
  if (m->assembly == ASSEMBLY_SLOTS) {
    CK(dalloc(m, &m->d_slots, (size_t)ne * E_pad));
    CK(cudaMemset(m->d_slots, 0, (size_t)ne * E_pad * sizeof(float4)));
    CK(dalloc(m, &m->d_sell, sell.size() + 1));
    CK(cudaMemcpy(m->d_sell, sell.data(), sell.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(dalloc(m, &m->d_chunk_ptr, chunk_ptr.size()));
    CK(cudaMemcpy(m->d_chunk_ptr, chunk_ptr.data(), chunk_ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    d_mass_sell = m->d_sell;
    d_mass_chunk = m->d_chunk_ptr;
  } else {
    CK(dalloc(m, &m->d_tile_ptr, tile_ptr.size()));
    CK(cudaMemcpy(m->d_tile_ptr, tile_ptr.data(), tile_ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(dalloc(m, &m->d_tile_nodes, tnodes_pad.size()));
    CK(cudaMemcpy(m->d_tile_nodes, tnodes_pad.data(), tnodes_pad.size() * sizeof(int), cudaMemcpyHostToDevice));
    // the kernels index shared float4 arrays with these: stored as byte offsets
    // (x 16), which keeps them in 16 bits for up to 4095 tile nodes / slots
    if ((long long)m->cap * 16 > 65535 || (long long)T_slots_bytes(m) > 65535)
      return fail(m, DJ_ERR_INVALID_ARG, "tile too large (tile_size %d, %d nodes)", m->T, m->cap);
    for (auto& v : lconn) v = (unsigned short)(v * 16);
    for (auto& v : lidx) v = (unsigned short)(v * 16);
    CK(dalloc(m, &m->d_lconn, lconn.size()));
    CK(cudaMemcpy(m->d_lconn, lconn.data(), lconn.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
    CK(dalloc(m, &m->d_lptr, lptr.size()));
    CK(cudaMemcpy(m->d_lptr, lptr.data(), lptr.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
    CK(dalloc(m, &m->d_lidx, lidx.size()));
    CK(cudaMemcpy(m->d_lidx, lidx.data(), lidx.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
    if (m->geometric) {
      CK(dalloc(m, &m->d_xloc, xloc_pad.size()));
      CK(cudaMemcpy(m->d_xloc, xloc_pad.data(), xloc_pad.size() * sizeof(float4), cudaMemcpyHostToDevice));
    }
    CK(dalloc(m, &m->d_parts, (size_t)m->n_parts));
    CK(cudaMemset(m->d_parts, 0, (size_t)m->n_parts * sizeof(float4)));
    CK(dalloc(m, &m->d_pdst, pdst_pad.size()));
    CK(cudaMemcpy(m->d_pdst, pdst_pad.data(), pdst_pad.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(dalloc(m, &m->d_node_ptr, node_ptr.size()));
    CK(cudaMemcpy(m->d_node_ptr, node_ptr.data(), node_ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    m->sell_entries = (long long)node_ptr.size();
    m->anp = prm.anp;
    if (m->anp) {
      // kappa_i / V0_i: V0_i = sum of 0V_e / 4 over the node's elements (FP64),
      // kappa_i their 0V-weighted bulk modulus
      std::vector<double> v0n(N, 0.0), kv0n(N, 0.0);
      for (long long e = 0; e < E; ++e) {
        const int* c = &cn[e * 4];
        double d[3][3];
        for (int r = 0; r < 3; ++r)
          for (int j = 0; j < 3; ++j) d[r][j] = Xn[3 * (size_t)c[r + 1] + j] - Xn[3 * (size_t)c[0] + j];
        const double det = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                           d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                           d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
        const double q = det / 6.0 / 4.0, kq = m->kappa[m->elem_old_of_new[e]] * q;
        for (int b = 0; b < 4; ++b) {
          v0n[c[b]] += q;
          kv0n[c[b]] += kq;
        }
      }
      std::vector<float> c1(N, 0.f);
      for (long long i = 0; i < N; ++i)
        if (v0n[i] > 0) c1[i] = (float)(kv0n[i] / v0n[i] / v0n[i]);
      CK(dalloc(m, &m->d_c1, N));
      CK(cudaMemcpy(m->d_c1, c1.data(), N * sizeof(float), cudaMemcpyHostToDevice));
      CK(dalloc(m, &m->d_pres, N));
      CK(cudaMemset(m->d_pres, 0, N * sizeof(float)));
      CK(dalloc(m, &m->d_vparts, (size_t)m->n_parts));
      CK(cudaMemset(m->d_vparts, 0, (size_t)m->n_parts * sizeof(float)));
    }
    CK(cudaMalloc(&d_mass_sell, (sell.size() + 1) * sizeof(int)));
    CK(cudaMemcpy(d_mass_sell, sell.data(), sell.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&d_mass_chunk, chunk_ptr.size() * sizeof(int)));
    CK(cudaMemcpy(d_mass_chunk, chunk_ptr.data(), chunk_ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  CK(dalloc(m, &m->d_U, N));
  CK(dalloc(m, &m->d_V, N));
  m->cmp = prm.precision;
  if (m->cmp) {
    CK(dalloc(m, &m->d_Ulo, N));
    CK(cudaMemset(m->d_Ulo, 0, N * sizeof(float4)));
  }
  CK(dalloc(m, &m->d_fout, N));
  CK(dalloc(m, &m->d_bct, std::max(1, m->n_bc_nodes)));
  if (m->n_bc_nodes) {
    CK(cudaMemcpy(m->d_bct, m->h_bct.data(), m->h_bct.size() * sizeof(float4), cudaMemcpyHostToDevice));
    const size_t nb = m->bc_flat_of_entry.size();
    CK(dalloc(m, &m->d_bc_flat, nb));
    CK(cudaMemcpy(m->d_bc_flat, m->bc_flat_of_entry.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
    // per prescribed-node row, the target entries of its components (read by
    // the node update when dj_step_host hands it the targets directly)
    std::vector<int4> ent(m->n_bc_nodes, make_int4(-1, -1, -1, 0));
    for (size_t k = 0; k < nb; ++k) {
      int4& e = ent[m->bc_node_of_entry[k]];
      const int c = m->bc_comp_of_entry[k];
      (c == 0 ? e.x : (c == 1 ? e.y : e.z)) = (int)k;
      e.w |= 1 << c;
    }
    CK(dalloc(m, &m->d_bc_entry, ent.size()));
    CK(cudaMemcpy(m->d_bc_entry, ent.data(), ent.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  CK(dalloc(m, &m->d_perm, N));
  CK(cudaMemcpy(m->d_perm, m->node_new_of_old.data(), N * sizeof(int), cudaMemcpyHostToDevice));
  if (!m->R.empty()) {
    std::vector<float4> Rn(N);
    for (long long i = 0; i < N; ++i) {
      const size_t o = 3 * (size_t)m->node_old_of_new[i];
      Rn[i] = make_float4((float)m->R[o], (float)m->R[o + 1], (float)m->R[o + 2], 0.f);
    }
    CK(dalloc(m, &m->d_R, N));
    CK(cudaMemcpy(m->d_R, Rn.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  }
  if (m->assembly == ASSEMBLY_TILES_TMA) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int per_sm = tma_blocks_per_sm(m->elem_type, m->variant, m->cmp, m->anp, tile_args(m));
    if (per_sm <= 0) return fail(m, DJ_ERR_UNSUPPORTED, "tile too large for shared memory (tile_size %d)", m->T);
    m->tma_grid = std::min(m->n_tiles, per_sm * sms);
    if (prm.max_blocks > 0) m->tma_grid = std::min(m->tma_grid, prm.max_blocks);
  }
  m->n_node_blocks = (int)((N + NODE_THREADS - 1) / NODE_THREADS);
  CK(dalloc(m, &m->d_partials, m->n_node_blocks));
  CK(dalloc(m, &m->d_state, 1));
  CK(cudaMallocHost((void**)&m->h_state, sizeof(DevState)));
  CK(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
  // ---- FP64 pre-computation on the device ------------------------------------
  {
    std::vector<unsigned char> mo(E);
    std::vector<double> mu(E), ka(E), rh(E), ea(E), eb(E), c1(E), ad(3 * E), bd(3 * E);
    for (long long e = 0; e < E; ++e) {
      const int o = m->elem_old_of_new[e];
      mo[e] = m->model[o];
      mu[e] = m->mu[o];
      ka[e] = m->kappa[o];
      rh[e] = m->rho[o];
      ea[e] = m->eta_a[o];
      eb[e] = m->eta_b[o];
      c1[e] = m->c01[o];
      for (int j = 0; j < 3; ++j) {
        ad[3 * e + j] = m->adir[3 * (size_t)o + j];
        bd[3 * e + j] = m->bdir[3 * (size_t)o + j];
      }
    }
    double *dX = nullptr, *dmu = nullptr, *dka = nullptr, *drh = nullptr, *dea = nullptr, *deb = nullptr,
           *dc1 = nullptr, *dad = nullptr, *dbd = nullptr, *dem = nullptr, *ddt = nullptr, *dmass = nullptr,
           *dred = nullptr;
    unsigned char* dmo = nullptr;
    int *dcn = nullptr, *dbad = nullptr, *dbc = nullptr;
    auto cleanup = [&]() {
      void* ps[] = {dX, dmu, dka, drh, dea, deb, dc1, dad, dbd, dem, ddt, dmass, dred, dmo, dcn, dbad, dbc};
      for (void* q : ps)
        if (q) cudaFree(q);
      if (m->assembly != ASSEMBLY_SLOTS) {
        if (d_mass_sell) cudaFree(d_mass_sell);
        if (d_mass_chunk) cudaFree(d_mass_chunk);
        d_mass_sell = d_mass_chunk = nullptr;
      }
    };
#define CKP(call)                                                                   \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess) {                                                        \
      cleanup();                                                                    \
      release_device(m);                                                            \
      return fail(m, _e == cudaErrorMemoryAllocation ? DJ_ERR_OOM : DJ_ERR_CUDA,    \
                  "precompute: %s: %s", #call, cudaGetErrorString(_e));             \
    }                                                                               \
  } while (0)
    CKP(cudaMalloc(&dX, 3 * N * sizeof(double)));
    CKP(cudaMalloc(&dcn, (size_t)E * ne * sizeof(int)));
    CKP(cudaMalloc(&dmo, E));
    CKP(cudaMalloc(&dmu, E * sizeof(double)));
    CKP(cudaMalloc(&dka, E * sizeof(double)));
    CKP(cudaMalloc(&drh, E * sizeof(double)));
    CKP(cudaMalloc(&dea, E * sizeof(double)));
    CKP(cudaMalloc(&deb, E * sizeof(double)));
    CKP(cudaMalloc(&dc1, E * sizeof(double)));
    CKP(cudaMalloc(&dad, 3 * E * sizeof(double)));
    CKP(cudaMalloc(&dbd, 3 * E * sizeof(double)));
    CKP(cudaMalloc(&dem, E * sizeof(double)));
    CKP(cudaMalloc(&ddt, E * sizeof(double)));
    CKP(cudaMalloc(&dmass, N * sizeof(double)));
    CKP(cudaMalloc(&dred, 256 * sizeof(double)));
    CKP(cudaMalloc(&dbad, sizeof(int)));
    CKP(cudaMalloc(&dbc, N * sizeof(int)));
    CKP(cudaMemcpy(dX, Xn.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dcn, cn.data(), (size_t)E * ne * sizeof(int), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dmo, mo.data(), E, cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dmu, mu.data(), E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dka, ka.data(), E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(drh, rh.data(), E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dea, ea.data(), E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(deb, eb.data(), E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dc1, c1.data(), E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dad, ad.data(), 3 * E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dbd, bd.data(), 3 * E * sizeof(double), cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(dbc, bcidx.data(), N * sizeof(int), cudaMemcpyHostToDevice));
    const int big = INT_MAX;
    CKP(cudaMemcpy(dbad, &big, sizeof(int), cudaMemcpyHostToDevice));
    PreArgs pa;
    pa.X = dX;
    pa.conn = dcn;
    pa.model = dmo;
    pa.mu = dmu;
    pa.kappa = dka;
    pa.rho = drh;
    pa.eta_a = dea;
    pa.eta_b = deb;
    pa.c01 = dc1;
    pa.adir = dad;
    pa.bdir = dbd;
    pa.consts = m->d_consts;
    pa.conn4 = m->d_conn;
    pa.elem_mass = dem;
    pa.dt_elem = ddt;
    pa.bad = dbad;
    pa.E = (int)E;
    pa.E_pad = E_pad;
    pa.ne = ne;
    pa.off_fa = m->off_fa;
    pa.off_fb = m->off_fb;
    pa.off_mr = m->off_mr;
    pa.off_hg = m->off_hg;
    pa.hg_coeff = prm.hg_coeff;
    pa.tile_T = m->assembly != ASSEMBLY_SLOTS ? m->T : 0;
    pa.n_consts = nc;
    pa.geometric = m->geometric;
    CKP(launch_precompute_elements(pa, 0));
    int bad = 0;
    CKP(cudaMemcpy(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad != INT_MAX) {
      const int caller = m->elem_old_of_new[bad];
      cleanup();
      release_device(m);
      return fail(m, DJ_ERR_INVERTED_ELEMENT, "element %d has det 0J <= 0", caller);
    }
    CKP(launch_min_reduce(ddt, (int)E, dred, 0));
    std::vector<double> red(256);
    CKP(cudaMemcpy(red.data(), dred, 256 * sizeof(double), cudaMemcpyDeviceToHost));
    m->dt_crit = *std::min_element(red.begin(), red.end());
    const int G = std::max(1, m->n_groups);
    m->group_dt_crit.assign(G, m->dt_crit);
    if (m->n_groups > 0) {
      std::vector<double> dte(E);
      CKP(cudaMemcpy(dte.data(), ddt, E * sizeof(double), cudaMemcpyDeviceToHost));
      m->group_dt_crit.assign(G, 1e300);
      for (long long e = 0; e < E; ++e) {
        const int g = m->elem_group[m->elem_old_of_new[e]];
        m->group_dt_crit[g] = std::min(m->group_dt_crit[g], dte[e]);
      }
    }
    m->group_dt.assign(G, 0.0);
    for (int g = 0; g < G; ++g) {
      if (prm.dt > 0) {
        if (prm.dt > m->group_dt_crit[g] * (1.0 + 1e-12)) {
          const double dc = m->group_dt_crit[g];
          cleanup();
          release_device(m);
          return fail(m, DJ_ERR_INVALID_ARG, "dt %.6g exceeds the critical step %.6g", prm.dt, dc);
        }
        m->group_dt[g] = prm.dt;
      } else {
        if (prm.dt_scale > 1.0) {
          cleanup();
          release_device(m);
          return fail(m, DJ_ERR_INVALID_ARG, "dt_scale above 1 exceeds the critical step");
        }
        m->group_dt[g] = prm.dt_scale * m->group_dt_crit[g];
      }
    }
    m->dt = *std::min_element(m->group_dt.begin(), m->group_dt.end());
    const double adt = prm.alpha * m->dt;
    m->bm1 = (float)((2.0 - adt) / (2.0 + adt));
    double* ddtn = nullptr;
    if (m->n_groups > 0) {
      std::vector<double> dtn(N);
      std::vector<float> bm1n(N);
      for (int g = 0; g < m->n_groups; ++g)
        for (int i = m->group_node_ptr[g]; i < m->group_node_ptr[g + 1]; ++i) {
          dtn[i] = m->group_dt[g];
          const double a = prm.alpha * m->group_dt[g];
          bm1n[i] = (float)((2.0 - a) / (2.0 + a));
        }
      CKP(cudaMalloc(&ddtn, N * sizeof(double)));
      CKP(cudaMemcpy(ddtn, dtn.data(), N * sizeof(double), cudaMemcpyHostToDevice));
      if (prm.alpha > 0) {
        CKP(cudaMalloc(&m->d_bm1, N * sizeof(float)));
        CKP(cudaMemcpy(m->d_bm1, bm1n.data(), N * sizeof(float), cudaMemcpyHostToDevice));
      }
      CKP(cudaMalloc(&m->d_node_resid, N * sizeof(double2)));
      CKP(cudaMalloc(&m->d_group_resid, m->n_groups * sizeof(double2)));
      CKP(cudaMalloc(&m->d_group_node_ptr, (m->n_groups + 1) * sizeof(int)));
      CKP(cudaMemcpy(m->d_group_node_ptr, m->group_node_ptr.data(), (m->n_groups + 1) * sizeof(int),
                     cudaMemcpyHostToDevice));
      CKP(cudaMallocHost((void**)&m->h_group_resid, m->n_groups * sizeof(double2)));
    }
    cudaError_t me = launch_node_mass(d_mass_sell, d_mass_chunk, dem, E_pad, (int)N, m->dt, ddtn, prm.alpha,
                                      dbc, dmass, m->d_U, m->d_V, 0);
    if (me == cudaSuccess) me = cudaDeviceSynchronize();
    if (ddtn) cudaFree(ddtn);
    CKP(me);
    std::vector<double> mass(N);
    CKP(cudaMemcpy(mass.data(), dmass, N * sizeof(double), cudaMemcpyDeviceToHost));
    m->total_mass = 0;
    for (double v : mass) m->total_mass += v;
    std::vector<float4> U0(N);
    CKP(cudaMemcpy(U0.data(), m->d_U, N * sizeof(float4), cudaMemcpyDeviceToHost));
    m->h_ai.resize(N);
    for (long long i = 0; i < N; ++i) m->h_ai[i] = U0[i].w;
    cleanup();
#undef CKP
  }
  DevState st0{};
  st0.step = 0;
  st0.ramp_s = 0.f;
  st0.err_flags = 0;
  st0.bad_elem = INT_MAX;
  st0.bad_node = INT_MAX;
  CK(cudaMemcpy(m->d_state, &st0, sizeof(DevState), cudaMemcpyHostToDevice));
  CK(cudaDeviceSynchronize());
  m->precomputed = true;
  if (dt_out) *dt_out = m->dt;
  return DJ_OK;
}

dj_status dj_mesh_update_bc_targets(dj_mesh* m, const double* target) {
  if (!m || !target) return DJ_ERR_INVALID_ARG;
  const size_t nb = m->bc_dof.size();
  bool finite = true;
  for (size_t k = 0; k < nb; ++k) finite &= std::isfinite(target[k]);
  if (!finite) return fail(m, DJ_ERR_INVALID_ARG, "non-finite target");
  std::memcpy(m->bc_target.data(), target, nb * sizeof(double));
  m->targets_on_device = false;
  if (!m->precomputed) return DJ_OK;
  CK(cudaSetDevice(m->device));
  if (m->n_bc_nodes) {
    // a page-locked caller array (8-byte aligned) is read by the scatter kernel
    // through its device mapping: one launch, no host pass over the table
    cudaPointerAttributes attr;
    const double* mapped = nullptr;
    if (reinterpret_cast<uintptr_t>(target) % alignof(double) == 0 &&
        cudaPointerGetAttributes(&attr, target) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
        attr.devicePointer)
      mapped = static_cast<const double*>(attr.devicePointer);
    else
      (void)cudaGetLastError();
    if (mapped) {
      CK(launch_bc_targets(mapped, m->d_bc_flat, (int)nb, m->d_bct, 0));
      CK(cudaStreamSynchronize(0));  // the caller may reuse the array on return
      return DJ_OK;
    }
    // otherwise the per-node table (targets, w = component mask) lives in
    // pinned memory once the first update has staged it; each update rewrites
    // the targets in place and copies the table once (every target entry is
    // rewritten, so the staged copy never goes stale)
    const size_t bytes = (size_t)m->n_bc_nodes * sizeof(float4);
    if (!m->h_bct_pinned) {
      CK(cudaMallocHost((void**)&m->h_bct_pinned, bytes));
      std::memcpy(m->h_bct_pinned, m->h_bct.data(), bytes);
    }
    float* pin = reinterpret_cast<float*>(m->h_bct_pinned);
    const int* flat = m->bc_flat_of_entry.data();
    for (size_t k = 0; k < nb; ++k) pin[flat[k]] = (float)target[k];
    CK(cudaMemcpy(m->d_bct, m->h_bct_pinned, bytes, cudaMemcpyHostToDevice));
  }
  return DJ_OK;
}

namespace {
// device address of a page-locked host array (8-byte aligned), else nullptr
void* mapped_host(const void* p) {
  cudaPointerAttributes attr;
  if (reinterpret_cast<uintptr_t>(p) % alignof(double) == 0 && cudaPointerGetAttributes(&attr, p) == cudaSuccess &&
      attr.type == cudaMemoryTypeHost && attr.devicePointer)
    return attr.devicePointer;
  (void)cudaGetLastError();
  return nullptr;
}
}  // namespace

dj_status dj_step_host(dj_mesh* m, const double* target, void* U_out, int out_f64, void* stream) {
  const Range range("dj_step_host");
  dj_status s = need_ready(m);
  if (s) return s;
  if (out_f64 != 0 && out_f64 != 1) return fail(m, DJ_ERR_INVALID_ARG, "out_f64 must be 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nb = m->bc_dof.size();
  // the device state reaches the host through the mapping of its page-locked
  // copy, written by the last kernel of the call (no separate copy)
  if (!m->h_state_map) CK(cudaHostGetDevicePointer((void**)&m->h_state_map, m->h_state, 0));
  DevState* st_map = m->h_state_map;
  const bool with_targets = target && nb;
  if (with_targets) {
    // The force kernel copies this step's targets from a page-locked caller
    // array (through its device mapping, coalesced, beside its own work) into
    // the device copy d_tgt_stage; other host memory is copied there before
    // the step.  The update kernel reads the device copy and stores the
    // targets into its prescribed-node rows of the table, so no scatter
    // kernel and no wait on another stream sit between the two step kernels
    // (the update keeps its programmatic launch).  Non-finite entries are not
    // applied (the previous target stays) and are reported after the step.
    // The host's own copy of the targets is refreshed from the device copy
    // when it is next needed (sync_host_targets).
    if (!m->d_tgt_stage) CK(cudaMalloc(&m->d_tgt_stage, nb * sizeof(double)));
    const double* mapped = static_cast<const double*>(mapped_host(target));
    if (!mapped) CK(cudaMemcpyAsync(m->d_tgt_stage, target, nb * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(launch_force_any(m, 1, st, mapped));
    NodeArgs na = node_args(m);
    na.tgt = m->d_tgt_stage;
    CK(launch_node(NODE_UPDATE_TGT, m->cmp, na, st));
    m->targets_on_device = true;
  } else {
    CK(launch_step(m, st, NODE_UPDATE));
  }
  if (U_out) {
    const long long N = m->N;
    void* direct = mapped_host(U_out);
    const float4* lo = m->cmp ? m->d_Ulo : nullptr;
    if (out_f64) {
      if (!direct && !m->d_out64) CK(cudaMalloc(&m->d_out64, 3 * N * sizeof(double)));
      double* dst = direct ? static_cast<double*>(direct) : m->d_out64;
      CK(launch_to_caller_order_f64(m->d_U, lo, m->d_perm, (int)N, dst, st, m->d_state, st_map));
      if (!direct) CK(cudaMemcpyAsync(U_out, m->d_out64, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else {
      if (!direct && !m->d_out64) CK(cudaMalloc(&m->d_out64, 3 * N * sizeof(double)));
      float* dst = direct ? static_cast<float*>(direct) : reinterpret_cast<float*>(m->d_out64);
      CK(launch_to_caller_order_f32(m->d_U, lo, m->d_perm, (int)N, dst, st, m->d_state, st_map));
      if (!direct) CK(cudaMemcpyAsync(U_out, m->d_out64, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
  } else {
    CK(launch_copy_state(m->d_state, st_map, st));
  }
  CK(cudaStreamSynchronize(st));  // the only synchronisation of the call
  if (m->h_state->err_flags & ERR_BAD_TARGET) {
    // not applied: clear the record so that later calls do not report it again
    const int keep = m->h_state->err_flags & ~ERR_BAD_TARGET;
    CK(cudaMemcpy(&m->d_state->err_flags, &keep, sizeof(int), cudaMemcpyHostToDevice));
    m->h_state->err_flags = keep;
    s = check_flags(m);
    if (s) return s;
    return fail(m, DJ_ERR_INVALID_ARG, "non-finite target (not applied; the step kept its previous value)");
  }
  return check_flags(m);
}

dj_status dj_step(dj_mesh* m, void* stream) {
  const Range range("dj_step");
  dj_status s = need_ready(m);
  if (s) return s;
  CK(launch_step(m, (cudaStream_t)stream, NODE_UPDATE));
  return DJ_OK;
}

dj_status dj_run_n(dj_mesh* m, long long n, void* stream) {
  const Range range("dj_run_n");
  dj_status s = need_ready(m);
  if (s) return s;
  if (n < 0) return fail(m, DJ_ERR_INVALID_ARG, "n < 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = 32;
  if (n >= chunk && !m->run_exec) {
    s = capture(m, &m->run_exec, [&](cudaStream_t cs) {
      for (int k = 0; k < chunk; ++k) {
        cudaError_t e = launch_step(m, cs, NODE_UPDATE);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    });
    if (s) return s;
    m->run_chunk = chunk;
  }
  long long left = n;
  while (m->run_exec && left >= m->run_chunk) {
    CK(cudaGraphLaunch(m->run_exec, st));
    left -= m->run_chunk;
  }
  for (; left > 0; --left) CK(launch_step(m, st, NODE_UPDATE));
  return DJ_OK;
}

dj_status dj_run_n_profiled(dj_mesh* m, long long n, void* stream, double* ms_force, double* ms_update) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (n < 0) return fail(m, DJ_ERR_INVALID_ARG, "n < 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (ms_force) *ms_force = 0;
  if (ms_update) *ms_update = 0;
  if (n == 0) return DJ_OK;
  // 1. n time steps (state advances as with dj_run_n)
  s = dj_run_n(m, n, stream);
  if (s) return s;
  // 2. device time of the element-force kernel alone: a graph of up to 64
  //    back-to-back launches that do not advance the clock, replayed; and of the
  //    update kernel alone on a saved copy of the state, which is restored after
  const long long chunk = std::min(64LL, n);
  cudaGraphExec_t gf = nullptr, gu = nullptr;
  s = capture(m, &gf, [&](cudaStream_t cs) {
    for (long long j = 0; j < chunk; ++j) {
      cudaError_t e = launch_force_any(m, 0, cs);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  });
  if (s) return s;
  s = capture(m, &gu, [&](cudaStream_t cs) {
    for (long long j = 0; j < chunk; ++j) {
      cudaError_t e = launch_node(NODE_UPDATE, m->cmp, node_args(m), cs);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  });
  if (s) {
    cudaGraphExecDestroy(gf);
    return s;
  }
  float4 *sU = nullptr, *sV = nullptr, *sL = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  cudaError_t err = cudaMalloc(&sU, m->N * sizeof(float4));
  if (err == cudaSuccess) err = cudaMalloc(&sV, m->N * sizeof(float4));
  if (err == cudaSuccess) err = cudaMemcpyAsync(sU, m->d_U, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(sV, m->d_V, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (err == cudaSuccess && m->cmp) err = cudaMalloc(&sL, m->N * sizeof(float4));
  if (err == cudaSuccess && m->cmp)
    err = cudaMemcpyAsync(sL, m->d_Ulo, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) err = cudaEventCreate(&e2);
  const long long reps = std::max(1LL, n / chunk);
  if (err == cudaSuccess) err = cudaEventRecord(e0, st);
  for (long long r = 0; r < reps && err == cudaSuccess; ++r) err = cudaGraphLaunch(gf, st);
  if (err == cudaSuccess) err = cudaEventRecord(e1, st);
  for (long long r = 0; r < reps && err == cudaSuccess; ++r) err = cudaGraphLaunch(gu, st);
  if (err == cudaSuccess) err = cudaEventRecord(e2, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  float tf = 0, tu = 0;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&tf, e0, e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&tu, e1, e2);
  // restore the state and the element forces of the current step
  if (sU) cudaMemcpyAsync(m->d_U, sU, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (sV) cudaMemcpyAsync(m->d_V, sV, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (sL) cudaMemcpyAsync(m->d_Ulo, sL, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  cudaStreamSynchronize(st);
  cudaGraphExecDestroy(gf);
  cudaGraphExecDestroy(gu);
  if (sU) cudaFree(sU);
  if (sV) cudaFree(sV);
  if (sL) cudaFree(sL);
  for (cudaEvent_t e : {e0, e1, e2})
    if (e) cudaEventDestroy(e);
  if (err != cudaSuccess) return fail(m, DJ_ERR_CUDA, "profiled run: %s", cudaGetErrorString(err));
  // per-step totals scaled to the n steps that were run
  const double per = 1.0 / (double)(reps * chunk) * (double)n;
  if (ms_force) *ms_force = tf * per;
  if (ms_update) *ms_update = tu * per;
  return DJ_OK;
}

dj_status dj_profile_kernels(dj_mesh* m, int launches, void* d_flush, size_t flush_bytes, void* stream,
                             double* ms_force, double* ms_update) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (launches <= 0 || (d_flush && flush_bytes < 32)) return fail(m, DJ_ERR_INVALID_ARG, "bad launches or flush size");
  cudaStream_t st = (cudaStream_t)stream;
  float4 *sU = nullptr, *sV = nullptr, *sL = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&sU, m->N * sizeof(float4));
  if (err == cudaSuccess) err = cudaMalloc(&sV, m->N * sizeof(float4));
  if (err == cudaSuccess && m->cmp) err = cudaMalloc(&sL, m->N * sizeof(float4));
  if (err == cudaSuccess) err = cudaMemcpyAsync(sU, m->d_U, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(sV, m->d_V, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (err == cudaSuccess && m->cmp)
    err = cudaMemcpyAsync(sL, m->d_Ulo, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  double tf = 0.0, tu = 0.0;
  for (int pass = 0; pass < 2 && err == cudaSuccess; ++pass) {
    for (int i = 0; i < launches && err == cudaSuccess; ++i) {
      if (d_flush) err = launch_l2_flush(d_flush, flush_bytes, st);
      if (err == cudaSuccess) err = cudaEventRecord(e0, st);
      if (err == cudaSuccess)
        err = pass == 0 ? launch_force_any(m, 0, st) : launch_node(NODE_UPDATE, m->cmp, node_args(m), st);
      if (err == cudaSuccess) err = cudaEventRecord(e1, st);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      (pass == 0 ? tf : tu) += ms;
    }
  }
  // restore the state (the update launches advanced U and V without new forces)
  if (sU) cudaMemcpyAsync(m->d_U, sU, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (sV) cudaMemcpyAsync(m->d_V, sV, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  if (sL) cudaMemcpyAsync(m->d_Ulo, sL, m->N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (err == cudaSuccess) err = e2;
  for (void* p : {(void*)sU, (void*)sV, (void*)sL})
    if (p) cudaFree(p);
  for (cudaEvent_t e : {e0, e1})
    if (e) cudaEventDestroy(e);
  if (err != cudaSuccess) return fail(m, DJ_ERR_CUDA, "kernel profile: %s", cudaGetErrorString(err));
  if (ms_force) *ms_force = tf / launches;
  if (ms_update) *ms_update = tu / launches;
  return DJ_OK;
}

dj_status dj_sync(dj_mesh* m, void* stream) {
  dj_status s = need_ready(m);
  if (s) return s;
  s = read_state(m, (cudaStream_t)stream);
  if (s) return s;
  return check_flags(m);
}

dj_status dj_relax_to_tol(dj_mesh* m, double tol, long long max_steps, long long* steps_out,
                          double* residual_out, void* stream) {
  const Range range("dj_relax_to_tol");
  dj_status s = need_ready(m);
  if (s) return s;
  if (!(tol >= 0) || max_steps < 0) return fail(m, DJ_ERR_INVALID_ARG, "bad tol or max_steps");
  cudaStream_t st = (cudaStream_t)stream;
  const int k = m->params.relax_check_every;
  if (!m->relax_exec || m->relax_k != k) {
    if (m->relax_exec) cudaGraphExecDestroy(m->relax_exec);
    m->relax_exec = nullptr;
    s = capture(m, &m->relax_exec, [&](cudaStream_t cs) {
      for (int j = 0; j < k - 1; ++j) {
        cudaError_t e = launch_step(m, cs, NODE_UPDATE);
        if (e != cudaSuccess) return e;
      }
      cudaError_t e = launch_step(m, cs, NODE_UPDATE_RESID);
      if (e != cudaSuccess) return e;
      if (m->n_groups > 0) {
        e = cudaMemcpyAsync(m->h_group_resid, m->d_group_resid, m->n_groups * sizeof(double2),
                            cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return e;
      }
      return cudaMemcpyAsync(m->h_state, m->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, cs);
    });
    if (s) return s;
    m->relax_k = k;
  }
  long long done = 0;
  double r = INFINITY;
  while (done + k <= max_steps) {
    CK(cudaGraphLaunch(m->relax_exec, st));
    CK(cudaStreamSynchronize(st));
    done += k;
    s = check_flags(m);
    if (s) {
      if (steps_out) *steps_out = done;
      return s;
    }
    if (m->n_groups > 0) {
      m->group_r.assign(m->n_groups, 0.0);
      r = 0;
      for (int g = 0; g < m->n_groups; ++g) {
        const double num = std::sqrt(m->h_group_resid[g].x), den = std::sqrt(m->h_group_resid[g].y);
        m->group_r[g] = den > 0 ? num / den : num;
        r = std::max(r, m->group_r[g]);
      }
    } else {
      const double num = std::sqrt(m->h_state->resid_num2), den = std::sqrt(m->h_state->resid_den2);
      r = den > 0 ? num / den : num;
    }
    // the checked state is the one before the last step; it counts only once its
    // prescribed values are at their targets
    const long long checked = m->h_state->step - 1;
    if (r <= tol && (m->params.ramp_steps <= 0 || checked >= m->params.ramp_steps)) {
      if (steps_out) *steps_out = done;
      if (residual_out) *residual_out = r;
      return DJ_OK;
    }
  }
  // remaining steps that do not complete a check interval
  for (; done < max_steps; ++done) CK(launch_step(m, st, NODE_UPDATE));
  s = read_state(m, st);
  if (s) return s;
  s = check_flags(m);
  if (steps_out) *steps_out = done;
  if (residual_out) *residual_out = r;
  if (s) return s;
  return fail(m, DJ_ERR_NOT_CONVERGED, "residual %.3e above tol %.3e after %lld steps", r, tol, done);
}

dj_status dj_relax_adaptive(dj_mesh* m, double tol, long long max_steps, const dj_adr_params* opts,
                            long long* steps_out, double* residual_out, dj_adr_report* report, void* stream) {
  const Range range("dj_relax_adaptive");
  dj_status s = need_ready(m);
  if (s) return s;
  if (!(tol >= 0) || max_steps < 0) return fail(m, DJ_ERR_INVALID_ARG, "bad tol or max_steps");
  if (m->n_groups > 0) return fail(m, DJ_ERR_INVALID_ARG, "adaptive relaxation of a mesh with groups");
  const int k = m->params.relax_check_every;
  dj_adr_params o{0.0, 0.0, 0.0};
  if (opts) o = *opts;
  const double dt = m->dt;
  if (!(o.alpha_min >= 0) || !(o.alpha_max == o.alpha_max) || !(o.disp_tol == o.disp_tol))
    return fail(m, DJ_ERR_INVALID_ARG, "bad adaptive relaxation options");
  const double amax = o.alpha_max > 0 ? o.alpha_max : 2.0 / dt;
  if (o.alpha_min > amax) return fail(m, DJ_ERR_INVALID_ARG, "alpha_min above alpha_max");
  cudaStream_t st = (cudaStream_t)stream;
  if (!m->d_adr) {
    CK(dalloc(m, &m->d_adr, 1));
    CK(dalloc(m, &m->d_rq, 4 * (size_t)m->n_node_blocks));
    CK(dalloc(m, &m->d_usnap, (size_t)m->N));
    CK(cudaMemset(m->d_usnap, 0, (size_t)m->N * sizeof(double4)));
    CK(cudaMallocHost((void**)&m->h_adr, sizeof(AdrState)));
  }
  // the damping starts from the mesh's alpha
  const double a0 = m->params.alpha, adt0 = a0 * dt;
  AdrState init{};
  init.dt = dt;
  init.kappa0 = 2.0 / (2.0 + adt0);
  init.alpha_min = o.alpha_min;
  init.alpha_max = amax;
  init.ramp_steps = m->params.ramp_steps;
  init.k = k;
  init.bm1 = m->bm1;
  init.ai_scale = 1.f;
  init.alpha = a0;
  init.err_est = INFINITY;
  CK(cudaStreamSynchronize(st));  // h_adr is not in use by an earlier copy
  *m->h_adr = init;
  CK(cudaMemcpyAsync(m->d_adr, m->h_adr, sizeof(AdrState), cudaMemcpyHostToDevice, st));
  if (!m->adr_exec || m->adr_k != k) {
    if (m->adr_exec) cudaGraphExecDestroy(m->adr_exec);
    m->adr_exec = nullptr;
    s = capture(m, &m->adr_exec, [&](cudaStream_t cs) {
      for (int j = 0; j < k - 1; ++j) {
        cudaError_t e = launch_step(m, cs, NODE_ADR);
        if (e != cudaSuccess) return e;
      }
      cudaError_t e = launch_step(m, cs, NODE_ADR_RQ);
      if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_adr, m->d_adr, sizeof(AdrState), cudaMemcpyDeviceToHost, cs);
      if (e != cudaSuccess) return e;
      return cudaMemcpyAsync(m->h_state, m->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, cs);
    });
    if (s) return s;
    m->adr_k = k;
  }
  const auto fill = [&](const AdrState& a) {
    if (!report) return;
    report->alpha = a.alpha;
    report->lambda = a.lambda;
    report->rho = a.rho;
    report->err_est = a.err_est;
    report->n_estimates = a.n_est;
  };
  long long done = 0;
  double r = INFINITY;
  while (done + k <= max_steps) {
    CK(cudaGraphLaunch(m->adr_exec, st));
    CK(cudaStreamSynchronize(st));
    done += k;
    fill(*m->h_adr);
    s = check_flags(m);
    if (s) {
      if (steps_out) *steps_out = done;
      return s;
    }
    const double num = std::sqrt(m->h_state->resid_num2), den = std::sqrt(m->h_state->resid_den2);
    r = den > 0 ? num / den : num;
    const long long checked = m->h_state->step - 1;
    if (r <= tol && (m->params.ramp_steps <= 0 || checked >= m->params.ramp_steps) &&
        (o.disp_tol <= 0 || m->h_adr->err_est <= o.disp_tol)) {
      if (steps_out) *steps_out = done;
      if (residual_out) *residual_out = r;
      return DJ_OK;
    }
  }
  for (; done < max_steps; ++done) CK(launch_step(m, st, NODE_ADR));
  s = read_state(m, st);
  if (s) return s;
  s = check_flags(m);
  if (steps_out) *steps_out = done;
  if (residual_out) *residual_out = r;
  if (s) return s;
  return fail(m, DJ_ERR_NOT_CONVERGED, "residual %.3e above tol %.3e after %lld adaptive steps", r, tol, done);
}

dj_status dj_set_displacements(dj_mesh* m, const double* U0) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (!U0) return fail(m, DJ_ERR_INVALID_ARG, "null U0");
  const long long N = m->N;
  std::vector<float4> U(N), V(N), L(N);
  for (long long i = 0; i < N; ++i) {
    const size_t o = 3 * (size_t)m->node_old_of_new[i];
    if (!std::isfinite(U0[o]) || !std::isfinite(U0[o + 1]) || !std::isfinite(U0[o + 2]))
      return fail(m, DJ_ERR_INVALID_ARG, "non-finite displacement");
    U[i] = make_float4((float)U0[o], (float)U0[o + 1], (float)U0[o + 2], m->h_ai[i]);
    V[i] = make_float4(0.f, 0.f, 0.f, bits_to_float(m->h_bcidx[i]));
    L[i] = make_float4((float)(U0[o] - U[i].x), (float)(U0[o + 1] - U[i].y), (float)(U0[o + 2] - U[i].z), 0.f);
  }
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(m->d_U, U.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  if (m->cmp) CK(cudaMemcpy(m->d_Ulo, L.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m->d_V, V.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  CK(clear_error_flags(m, 0));
  CK(cudaDeviceSynchronize());
  return DJ_OK;
}

dj_status dj_get_displacements(dj_mesh* m, double* U_out) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (!U_out) return fail(m, DJ_ERR_INVALID_ARG, "null U_out");
  CK(cudaDeviceSynchronize());
  const long long N = m->N;
  // caller order and FP64 on the device.  A page-locked caller buffer
  // (8-byte aligned) is written by the kernel itself through its device
  // mapping; otherwise the values go through a device buffer and one copy.
  double* direct = nullptr;
  cudaPointerAttributes attr;
  if (reinterpret_cast<uintptr_t>(U_out) % alignof(double) == 0 &&
      cudaPointerGetAttributes(&attr, U_out) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
      attr.devicePointer)
    direct = static_cast<double*>(attr.devicePointer);
  else
    (void)cudaGetLastError();
  if (!direct && !m->d_out64) CK(cudaMalloc(&m->d_out64, 3 * N * sizeof(double)));
  CK(launch_to_caller_order_f64(m->d_U, m->cmp ? m->d_Ulo : nullptr, m->d_perm, (int)N,
                                direct ? direct : m->d_out64, 0));
  if (!direct)
    CK(cudaMemcpyAsync(U_out, m->d_out64, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, 0));
  s = read_state(m, 0);  // one synchronisation for the field and the state
  if (s) return s;
  return check_flags(m);
}

dj_status dj_get_displacements_device(dj_mesh* m, float* d_U_out, void* stream) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (!d_U_out) return fail(m, DJ_ERR_INVALID_ARG, "null output");
  CK(launch_to_caller_order(m->d_U, m->d_perm, (int)m->N, d_U_out, (cudaStream_t)stream));
  return DJ_OK;
}

dj_status dj_set_step(dj_mesh* m, long long step) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (step < 0) return fail(m, DJ_ERR_INVALID_ARG, "step < 0");
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&m->d_state->step, &step, sizeof(long long), cudaMemcpyHostToDevice));
  return DJ_OK;
}

dj_status dj_set_displacements_device(dj_mesh* m, const float* d_U0, void* stream) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (!d_U0) return fail(m, DJ_ERR_INVALID_ARG, "null field");
  CK(launch_from_caller_order(d_U0, m->d_perm, (int)m->N, m->d_U, m->d_V, m->d_Ulo, (cudaStream_t)stream));
  CK(clear_error_flags(m, (cudaStream_t)stream));
  return DJ_OK;
}

dj_status dj_evaluate_field(dj_mesh* m, const float* d_U, double* residual_out, int* inverted_out, void* stream) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (!d_U) return fail(m, DJ_ERR_INVALID_ARG, "null field");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = m->N, nb = N * sizeof(float4);
  if (!m->d_save) CK(dalloc(m, &m->d_save, 3 * N));
  float4 *sU = m->d_save, *sV = m->d_save + N, *sL = m->d_save + 2 * N;
  // save the stepping state; clear the error flags for the evaluation
  CK(cudaMemcpyAsync(sU, m->d_U, nb, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(sV, m->d_V, nb, cudaMemcpyDeviceToDevice, st));
  if (m->cmp) CK(cudaMemcpyAsync(sL, m->d_Ulo, nb, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(m->h_state, m->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const DevState before = *m->h_state;
  DevState clean = before;
  clean.err_flags = 0;
  clean.bad_elem = INT_MAX;
  clean.bad_node = INT_MAX;
  *m->h_state = clean;
  CK(cudaMemcpyAsync(m->d_state, m->h_state, sizeof(DevState), cudaMemcpyHostToDevice, st));
  cudaError_t e = launch_from_caller_order(d_U, m->d_perm, (int)m->N, m->d_U, m->d_V, m->d_Ulo, st);
  if (e == cudaSuccess) e = launch_force_any(m, 0, st);
  if (e == cudaSuccess) e = launch_node(NODE_RESID_ONLY, m->cmp, node_args(m), st);
  if (e == cudaSuccess) {
    if (m->n_groups > 0) {
      e = launch_group_resid(m->d_node_resid, m->d_group_node_ptr, m->n_groups, m->d_group_resid, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->h_group_resid, m->d_group_resid, m->n_groups * sizeof(double2),
                            cudaMemcpyDeviceToHost, st);
    } else {
      e = launch_resid_finalize(m->d_partials, m->n_node_blocks, m->d_state, st);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // h_state is not yet reused
  DevState after{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_state, m->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) after = *m->h_state;
  // restore the stepping state and its error flags
  *m->h_state = before;
  cudaMemcpyAsync(m->d_U, sU, nb, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(m->d_V, sV, nb, cudaMemcpyDeviceToDevice, st);
  if (m->cmp) cudaMemcpyAsync(m->d_Ulo, sL, nb, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(m->d_state, m->h_state, sizeof(DevState), cudaMemcpyHostToDevice, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return fail(m, DJ_ERR_CUDA, "evaluate field: %s", cudaGetErrorString(e));
  double r = 0;
  if (m->n_groups > 0) {
    for (int g = 0; g < m->n_groups; ++g) {
      const double num = std::sqrt(m->h_group_resid[g].x), den = std::sqrt(m->h_group_resid[g].y);
      r = std::max(r, den > 0 ? num / den : num);
    }
  } else {
    const double num = std::sqrt(after.resid_num2), den = std::sqrt(after.resid_den2);
    r = den > 0 ? num / den : num;
  }
  const int bad = after.err_flags != 0;
  if (residual_out) *residual_out = bad ? INFINITY : r;
  if (inverted_out) *inverted_out = bad;
  return DJ_OK;
}

dj_status dj_internal_forces(dj_mesh* m, const double* U, double* F_out) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (!U || !F_out) return fail(m, DJ_ERR_INVALID_ARG, "null array");
  const long long N = m->N;
  CK(cudaDeviceSynchronize());
  std::vector<float4> save(N), saveL(N), Un(N), Ln(N), F(N);
  CK(cudaMemcpy(save.data(), m->d_U, N * sizeof(float4), cudaMemcpyDeviceToHost));
  if (m->cmp) CK(cudaMemcpy(saveL.data(), m->d_Ulo, N * sizeof(float4), cudaMemcpyDeviceToHost));
  for (long long i = 0; i < N; ++i) {
    const size_t o = 3 * (size_t)m->node_old_of_new[i];
    Un[i] = make_float4((float)U[o], (float)U[o + 1], (float)U[o + 2], save[i].w);
    Ln[i] = make_float4((float)(U[o] - Un[i].x), (float)(U[o + 1] - Un[i].y), (float)(U[o + 2] - Un[i].z), 0.f);
  }
  CK(cudaMemcpy(m->d_U, Un.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  if (m->cmp) CK(cudaMemcpy(m->d_Ulo, Ln.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  CK(launch_force_any(m, 0, 0));
  NodeArgs na = node_args(m);
  na.R = nullptr;
  CK(launch_node(NODE_FORCE_ONLY, m->cmp, na, 0));
  CK(cudaMemcpy(F.data(), m->d_fout, N * sizeof(float4), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(m->d_U, save.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  if (m->cmp) CK(cudaMemcpy(m->d_Ulo, saveL.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  for (long long i = 0; i < N; ++i) {
    const size_t o = 3 * (size_t)m->node_old_of_new[i];
    F_out[o] = F[i].x;
    F_out[o + 1] = F[i].y;
    F_out[o + 2] = F[i].z;
  }
  s = read_state(m, 0);
  if (s) return s;
  return check_flags(m);
}

namespace {
struct StateHeader {
  unsigned long long magic;
  long long N;
  long long step;
  long long pad;
};
const unsigned long long kStateMagic = 0x444a544c45440001ULL;
}  // namespace

dj_status dj_state_size(const dj_mesh* m, size_t* bytes) {
  if (!m || !bytes) return DJ_ERR_INVALID_ARG;
  *bytes = sizeof(StateHeader) + (m->cmp ? 3 : 2) * (size_t)m->N * sizeof(float4);
  return DJ_OK;
}

dj_status dj_get_state(dj_mesh* m, void* buf, size_t bytes) {
  dj_status s = need_ready(m);
  if (s) return s;
  size_t need = 0;
  dj_state_size(m, &need);
  if (!buf || bytes < need) return fail(m, DJ_ERR_INVALID_ARG, "state buffer too small");
  CK(cudaDeviceSynchronize());
  s = read_state(m, 0);
  if (s) return s;
  StateHeader h{kStateMagic, m->N, m->h_state->step, 0};
  char* p = (char*)buf;
  std::memcpy(p, &h, sizeof(h));
  CK(cudaMemcpy(p + sizeof(h), m->d_U, m->N * sizeof(float4), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(p + sizeof(h) + m->N * sizeof(float4), m->d_V, m->N * sizeof(float4), cudaMemcpyDeviceToHost));
  if (m->cmp)
    CK(cudaMemcpy(p + sizeof(h) + 2 * m->N * sizeof(float4), m->d_Ulo, m->N * sizeof(float4),
                  cudaMemcpyDeviceToHost));
  return DJ_OK;
}

dj_status dj_set_state(dj_mesh* m, const void* buf, size_t bytes) {
  dj_status s = need_ready(m);
  if (s) return s;
  size_t need = 0;
  dj_state_size(m, &need);
  if (!buf || bytes < need) return fail(m, DJ_ERR_INVALID_ARG, "state buffer too small");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.N != m->N) return fail(m, DJ_ERR_INVALID_ARG, "state from another mesh");
  const char* p = (const char*)buf;
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(m->d_U, p + sizeof(h), m->N * sizeof(float4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m->d_V, p + sizeof(h) + m->N * sizeof(float4), m->N * sizeof(float4), cudaMemcpyHostToDevice));
  if (m->cmp)
    CK(cudaMemcpy(m->d_Ulo, p + sizeof(h) + 2 * m->N * sizeof(float4), m->N * sizeof(float4),
                  cudaMemcpyHostToDevice));
  DevState st{};
  st.step = h.step;
  st.bad_elem = INT_MAX;
  st.bad_node = INT_MAX;
  CK(cudaMemcpy(m->d_state, &st, sizeof(st), cudaMemcpyHostToDevice));
  return DJ_OK;
}

dj_status dj_get_info(const dj_mesh* mc, dj_info* info) {
  dj_mesh* m = const_cast<dj_mesh*>(mc);
  if (!m || !info) return DJ_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->n_nodes = m->N;
  info->n_elems = m->E;
  info->n_bc_dofs = (long long)m->bc_dof.size();
  info->elem_type = m->elem_type;
  if (!m->precomputed) return DJ_OK;
  CK(cudaSetDevice(m->device));
  CK(cudaDeviceSynchronize());
  dj_status s = read_state(m, 0);
  if (s) return s;
  info->step = m->h_state->step;
  info->model_flags = m->model_flags;
  info->dt = m->dt;
  info->dt_crit = m->dt_crit;
  info->total_mass = m->total_mass;
  info->device_bytes = m->device_bytes;
  if (m->assembly != ASSEMBLY_SLOTS) {
    info->elem_table_bytes_per_elem = (long long)m->n_consts * 4 + 2 * m->ne;
    info->slot_bytes_per_elem = 16 * m->n_parts / std::max(1LL, m->E);
  } else {
    info->elem_table_bytes_per_elem = (long long)m->n_consts * 4 + 4 * m->ne;
    info->slot_bytes_per_elem = 16LL * m->ne;
  }
  info->gather_index_bytes = m->sell_entries * 4;
  info->node_bytes_per_node = 64;
  info->n_parts = m->n_parts;
  info->assembly = m->assembly;
  info->tile_size = m->T;
  info->n_consts = m->n_consts;
  info->precision = m->cmp;
  info->grid = m->assembly == ASSEMBLY_TILES_TMA ? m->tma_grid : 0;
  info->n_tiles = m->assembly != ASSEMBLY_SLOTS ? m->n_tiles : 0;
  return DJ_OK;
}

dj_status dj_autotune(dj_mesh* m, int steps, void* stream, dj_params* chosen, double* ms_per_step) {
  return dj_autotune_cold(m, steps, nullptr, 0, stream, chosen, ms_per_step);
}

dj_status dj_autotune_cold(dj_mesh* m, int steps, void* d_flush, size_t flush_bytes, void* stream,
                           dj_params* chosen, double* ms_per_step) {
  dj_status s = need_ready(m);
  if (s) return s;
  if (steps <= 0) return fail(m, DJ_ERR_INVALID_ARG, "steps <= 0");
  if (d_flush && flush_bytes < 32) return fail(m, DJ_ERR_INVALID_ARG, "flush buffer too small");
  cudaStream_t st = (cudaStream_t)stream;
  size_t bytes = 0;
  dj_state_size(m, &bytes);
  std::vector<char> blob(bytes);
  s = dj_get_state(m, blob.data(), bytes);
  if (s) return s;
  const dj_params base = m->params;
  struct Cand {
    int assembly, tile;
  };
  std::vector<Cand> cands = {{ASSEMBLY_SLOTS, 0}};
  const int tiles4[] = {32, 64, 128, 256, 512}, tiles8[] = {32, 64, 128, 256};  // 32: one warp per tile
  if (m->ne == 4)
    for (int T : tiles4) cands.push_back({ASSEMBLY_TILES, T});
  else
    for (int T : tiles8) cands.push_back({ASSEMBLY_TILES, T});
  for (int T : {64, 128, 256}) cands.push_back({ASSEMBLY_TILES_TMA, T});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = INFINITY;
  dj_params best_p = base;
  // time one schedule from the saved state: ms over `steps` steps, or +inf
  const auto time_schedule = [&](const dj_params& p) -> double {
    if (dj_precompute(m, &p, nullptr) != DJ_OK) return INFINITY;  // e.g. a tile too large for shared memory
    if (dj_set_state(m, blob.data(), bytes) != DJ_OK) return INFINITY;
    if (dj_run_n(m, 8, stream) != DJ_OK) return INFINITY;  // graph capture and warm-up
    float ms = 0;
    if (!d_flush) {
      if (cudaEventRecord(e0, st) != cudaSuccess) return INFINITY;
      if (dj_run_n(m, steps, stream) != DJ_OK) return INFINITY;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return INFINITY;
      cudaEventElapsedTime(&ms, e0, e1);
    } else {
      // every step alone after an L2 eviction
      for (int k = 0; k < steps; ++k) {
        float mk = 0;
        if (launch_l2_flush(d_flush, flush_bytes, st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess ||
            launch_step(m, st, NODE_UPDATE) != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&mk, e0, e1) != cudaSuccess)
          return INFINITY;
        ms += mk;
      }
    }
    if (read_state(m, st) != DJ_OK || check_flags(m) != DJ_OK) return INFINITY;
    return ms;
  };
  for (const Cand& c : cands) {
    dj_params p = base;
    p.assembly = c.assembly;
    p.tile_size = c.tile;
    const double ms = time_schedule(p);
    if (ms < best) {
      best = ms;
      best_p = p;
    }
  }
  // graph replays: the best schedule with the other kind of edges between steps
  if (!d_flush && std::isfinite(best)) {
    dj_params p = best_p;
    p.graph_pdl = !best_p.graph_pdl;
    const double ms = time_schedule(p);
    if (ms < best) {
      best = ms;
      best_p = p;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s = dj_precompute(m, &best_p, nullptr);
  if (s) return s;
  s = dj_set_state(m, blob.data(), bytes);
  if (s) return s;
  if (!std::isfinite(best)) return fail(m, DJ_ERR_CUDA, "no schedule could be timed");
  if (chosen) *chosen = best_p;
  if (ms_per_step) *ms_per_step = best / steps;
  return DJ_OK;
}

dj_status dj_get_group_info(const dj_mesh* mc, int* n_groups, double* dt, double* dt_crit,
                            double* residual) {
  dj_mesh* m = const_cast<dj_mesh*>(mc);
  if (!m) return DJ_ERR_INVALID_ARG;
  const int G = std::max(1, m->n_groups);
  if (n_groups) *n_groups = G;
  if (!m->precomputed) return (dt || dt_crit || residual) ? fail(m, DJ_ERR_NOT_PRECOMPUTED, "not precomputed") : DJ_OK;
  for (int g = 0; g < G; ++g) {
    if (dt) dt[g] = m->group_dt[g];
    if (dt_crit) dt_crit[g] = m->group_dt_crit[g];
    if (residual) residual[g] = g < (int)m->group_r.size() ? m->group_r[g] : NAN;
  }
  return DJ_OK;
}

void dj_mesh_destroy(dj_mesh* m) {
  if (!m) return;
  if (m->device >= 0) cudaSetDevice(m->device);
  release_device(m);
  delete m;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: instances of one element type are merged into one internal mesh
// with one group per instance; the (at most two) internal meshes advance as
// two independent chains of kernels captured in one CUDA graph.
// ---------------------------------------------------------------------------
struct dj_batch {
  int n = 0;
  dj_mesh* part[2] = {nullptr, nullptr};  // 0: T4 instances, 1: H8 instances
  std::vector<int> inst_part, inst_group;
  std::vector<long long> inst_node_off, inst_nodes, inst_elems;
  cudaStream_t cap = nullptr, side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraphExec_t run_exec = nullptr, relax_exec = nullptr;
  int run_chunk = 0, relax_k = 0;
  bool precomputed = false;
  std::string last_error;
};

namespace {
dj_status bfail(dj_batch* b, dj_status s, const char* msg) {
  if (b) b->last_error = msg;
  return s;
}
void batch_release_graphs(dj_batch* b) {
  if (b->run_exec) cudaGraphExecDestroy(b->run_exec);
  if (b->relax_exec) cudaGraphExecDestroy(b->relax_exec);
  b->run_exec = b->relax_exec = nullptr;
  b->run_chunk = b->relax_k = 0;
}

// Capture two independent chains: part 0 on the capture stream, part 1 on a
// forked side stream joined at the end.
template <class F>
dj_status batch_capture(dj_batch* b, cudaGraphExec_t* out, F body) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(b, DJ_ERR_CUDA, cudaGetErrorString(e));
  cudaError_t be = cudaEventRecord(b->fork, b->cap);
  if (be == cudaSuccess) be = cudaStreamWaitEvent(b->side, b->fork, 0);
  if (be == cudaSuccess && b->part[0]) be = body(b->part[0], b->cap);
  if (be == cudaSuccess && b->part[1]) be = body(b->part[1], b->side);
  if (be == cudaSuccess) be = cudaEventRecord(b->join, b->side);
  if (be == cudaSuccess) be = cudaStreamWaitEvent(b->cap, b->join, 0);
  cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
  if (be != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, DJ_ERR_CUDA, cudaGetErrorString(be != cudaSuccess ? be : ee));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, DJ_ERR_CUDA, cudaGetErrorString(e));
  return DJ_OK;
}
}  // namespace

extern "C" {

dj_status dj_batch_create(dj_mesh* const* inst, int n, dj_batch** out) {
  if (!out) return DJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (!inst || n <= 0) return DJ_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!inst[i] || !inst[i]->materials_set) return DJ_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const dj_status ts = sync_host_targets(inst[i]);
    if (ts) return ts;
  }
  dj_batch* b = new (std::nothrow) dj_batch();
  if (!b) return DJ_ERR_OOM;
  b->n = n;
  b->inst_part.resize(n);
  b->inst_group.resize(n);
  b->inst_node_off.resize(n);
  b->inst_nodes.resize(n);
  b->inst_elems.resize(n);
  for (int pt = 0; pt < 2; ++pt) {
    const int et = pt == 0 ? DJ_TET4 : DJ_HEX8;
    std::vector<double> X, mu, ka, rh, ea, eb, c1, ad, bd, tg, R;
    std::vector<int> conn, grp;
    std::vector<unsigned char> mo;
    std::vector<long long> dof;
    long long noff = 0;
    int ng = 0;
    bool any_R = false;
    for (int i = 0; i < n; ++i) {
      const dj_mesh* m = inst[i];
      if (m->elem_type != et) continue;
      b->inst_part[i] = pt;
      b->inst_group[i] = ng;
      b->inst_node_off[i] = noff;
      b->inst_nodes[i] = m->N;
      b->inst_elems[i] = m->E;
      X.insert(X.end(), m->X.begin(), m->X.end());
      for (int v : m->conn) conn.push_back((int)(v + noff));
      grp.insert(grp.end(), m->E, ng);
      mo.insert(mo.end(), m->model.begin(), m->model.end());
      mu.insert(mu.end(), m->mu.begin(), m->mu.end());
      ka.insert(ka.end(), m->kappa.begin(), m->kappa.end());
      rh.insert(rh.end(), m->rho.begin(), m->rho.end());
      ea.insert(ea.end(), m->eta_a.begin(), m->eta_a.end());
      eb.insert(eb.end(), m->eta_b.begin(), m->eta_b.end());
      c1.insert(c1.end(), m->c01.begin(), m->c01.end());
      ad.insert(ad.end(), m->adir.begin(), m->adir.end());
      bd.insert(bd.end(), m->bdir.begin(), m->bdir.end());
      for (size_t k = 0; k < m->bc_dof.size(); ++k) {
        dof.push_back(m->bc_dof[k] + 3 * noff);
        tg.push_back(m->bc_target[k]);
      }
      if (!m->R.empty()) any_R = true;
      noff += m->N;
      ++ng;
    }
    if (ng == 0) continue;
    if (any_R) {
      R.assign(3 * noff, 0.0);
      for (int i = 0; i < n; ++i)
        if (b->inst_part[i] == pt && inst[i]->elem_type == et && !inst[i]->R.empty())
          std::copy(inst[i]->R.begin(), inst[i]->R.end(), R.begin() + 3 * b->inst_node_off[i]);
    }
    dj_mesh* pm = nullptr;
    dj_status st = dj_mesh_create(et, X.data(), noff, conn.data(), (long long)grp.size(), &pm);
    if (st == DJ_OK)
      st = dj_mesh_set_materials(pm, mo.data(), mu.data(), ka.data(), rh.data(), ea.data(), eb.data(),
                                 c1.data(), ad.data(), bd.data());
    if (st == DJ_OK) st = dj_mesh_set_bcs(pm, dof.data(), tg.data(), (long long)dof.size());
    if (st == DJ_OK && any_R) st = dj_mesh_set_loads(pm, R.data());
    if (st == DJ_OK) st = dj_mesh_set_groups(pm, grp.data(), ng);
    if (st != DJ_OK) {
      if (pm) dj_mesh_destroy(pm);
      for (int q = 0; q < 2; ++q)
        if (b->part[q]) dj_mesh_destroy(b->part[q]);
      delete b;
      return st;
    }
    b->part[pt] = pm;
  }
  *out = b;
  return DJ_OK;
}

dj_status dj_batch_precompute(dj_batch* b, const dj_params* params) {
  if (!b) return DJ_ERR_INVALID_ARG;
  batch_release_graphs(b);
  for (int pt = 0; pt < 2; ++pt)
    if (b->part[pt]) {
      dj_status s = dj_precompute(b->part[pt], params, nullptr);
      if (s) return bfail(b, s, b->part[pt]->last_error.c_str());
    }
  if (!b->cap) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e != cudaSuccess) return bfail(b, DJ_ERR_CUDA, cudaGetErrorString(e));
  }
  b->precomputed = true;
  return DJ_OK;
}

dj_status dj_batch_run_n(dj_batch* b, long long n, void* stream) {
  const Range range("dj_batch_run_n");
  if (!b || n < 0) return DJ_ERR_INVALID_ARG;
  if (!b->precomputed) return bfail(b, DJ_ERR_NOT_PRECOMPUTED, "call dj_batch_precompute first");
  (void)cudaGetLastError();
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = 16;
  if (n >= chunk && !b->run_exec) {
    dj_status s = batch_capture(b, &b->run_exec, [&](dj_mesh* m, cudaStream_t cs) {
      for (int k = 0; k < chunk; ++k) {
        cudaError_t e = launch_step(m, cs, NODE_UPDATE);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    });
    if (s) return s;
    b->run_chunk = chunk;
  }
  long long left = n;
  while (b->run_exec && left >= b->run_chunk) {
    cudaError_t e = cudaGraphLaunch(b->run_exec, st);
    if (e != cudaSuccess) return bfail(b, DJ_ERR_CUDA, cudaGetErrorString(e));
    left -= b->run_chunk;
  }
  for (; left > 0; --left)
    for (int pt = 0; pt < 2; ++pt)
      if (b->part[pt]) {
        cudaError_t e = launch_step(b->part[pt], st, NODE_UPDATE);
        if (e != cudaSuccess) return bfail(b, DJ_ERR_CUDA, cudaGetErrorString(e));
      }
  return DJ_OK;
}

dj_status dj_batch_sync(dj_batch* b, void* stream) {
  if (!b) return DJ_ERR_INVALID_ARG;
  for (int pt = 0; pt < 2; ++pt)
    if (b->part[pt]) {
      dj_status s = dj_sync(b->part[pt], stream);
      if (s) return bfail(b, s, b->part[pt]->last_error.c_str());
    }
  return DJ_OK;
}

dj_status dj_batch_relax_to_tol(dj_batch* b, double tol, long long max_steps, long long* steps_out,
                                double* residual_out, void* stream) {
  const Range range("dj_batch_relax_to_tol");
  if (!b || !(tol >= 0) || max_steps < 0) return DJ_ERR_INVALID_ARG;
  if (!b->precomputed) return bfail(b, DJ_ERR_NOT_PRECOMPUTED, "call dj_batch_precompute first");
  (void)cudaGetLastError();
  cudaStream_t st = (cudaStream_t)stream;
  dj_mesh* any = b->part[0] ? b->part[0] : b->part[1];
  const int k = any->params.relax_check_every;
  if (!b->relax_exec || b->relax_k != k) {
    if (b->relax_exec) cudaGraphExecDestroy(b->relax_exec);
    b->relax_exec = nullptr;
    dj_status s = batch_capture(b, &b->relax_exec, [&](dj_mesh* m, cudaStream_t cs) {
      for (int j = 0; j < k - 1; ++j) {
        cudaError_t e = launch_step(m, cs, NODE_UPDATE);
        if (e != cudaSuccess) return e;
      }
      cudaError_t e = launch_step(m, cs, NODE_UPDATE_RESID);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->h_group_resid, m->d_group_resid, m->n_groups * sizeof(double2),
                            cudaMemcpyDeviceToHost, cs);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->h_state, m->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, cs);
      return e;
    });
    if (s) return s;
    b->relax_k = k;
  }
  long long done = 0;
  double r = INFINITY;
  while (done + k <= max_steps) {
    cudaError_t e = cudaGraphLaunch(b->relax_exec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bfail(b, DJ_ERR_CUDA, cudaGetErrorString(e));
    done += k;
    r = 0;
    for (int pt = 0; pt < 2; ++pt) {
      dj_mesh* m = b->part[pt];
      if (!m) continue;
      dj_status s = check_flags(m);
      if (s) {
        if (steps_out) *steps_out = done;
        return bfail(b, s, m->last_error.c_str());
      }
      m->group_r.assign(m->n_groups, 0.0);
      for (int g = 0; g < m->n_groups; ++g) {
        const double num = std::sqrt(m->h_group_resid[g].x), den = std::sqrt(m->h_group_resid[g].y);
        m->group_r[g] = den > 0 ? num / den : num;
        r = std::max(r, m->group_r[g]);
      }
    }
    const long long checked = any->h_state->step - 1;
    if (r <= tol && (any->params.ramp_steps <= 0 || checked >= any->params.ramp_steps)) {
      if (steps_out) *steps_out = done;
      if (residual_out) *residual_out = r;
      return DJ_OK;
    }
  }
  if (steps_out) *steps_out = done;
  if (residual_out) *residual_out = r;
  return bfail(b, DJ_ERR_NOT_CONVERGED, "batch residual above tol");
}

dj_status dj_batch_instance_info(dj_batch* b, int i, long long* n_nodes, long long* n_elems, double* dt,
                                 double* residual) {
  if (!b || i < 0 || i >= b->n) return DJ_ERR_INVALID_ARG;
  dj_mesh* m = b->part[b->inst_part[i]];
  const int g = b->inst_group[i];
  if (n_nodes) *n_nodes = b->inst_nodes[i];
  if (n_elems) *n_elems = b->inst_elems[i];
  if (dt) *dt = m->precomputed ? m->group_dt[g] : NAN;
  if (residual) *residual = g < (int)m->group_r.size() ? m->group_r[g] : NAN;
  return DJ_OK;
}

dj_status dj_batch_get_displacements(dj_batch* b, int i, double* U_out) {
  if (!b || i < 0 || i >= b->n || !U_out) return DJ_ERR_INVALID_ARG;
  if (!b->precomputed) return bfail(b, DJ_ERR_NOT_PRECOMPUTED, "call dj_batch_precompute first");
  dj_mesh* m = b->part[b->inst_part[i]];
  if (cudaDeviceSynchronize() != cudaSuccess) return bfail(b, DJ_ERR_CUDA, "sync failed");
  const long long off = b->inst_node_off[i], nn = b->inst_nodes[i];
  int lo = m->node_new_of_old[off], hi = lo;
  for (long long q = 0; q < nn; ++q) {
    lo = std::min(lo, m->node_new_of_old[off + q]);
    hi = std::max(hi, m->node_new_of_old[off + q]);
  }
  const long long cnt = hi - lo + 1;  // groups are contiguous internal ranges
  std::vector<float4> U(cnt), L(cnt, make_float4(0.f, 0.f, 0.f, 0.f));
  if (cudaMemcpy(U.data(), m->d_U + lo, cnt * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, DJ_ERR_CUDA, "copy failed");
  if (m->cmp && cudaMemcpy(L.data(), m->d_Ulo + lo, cnt * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, DJ_ERR_CUDA, "copy failed");
  for (long long q = 0; q < nn; ++q) {
    const int v = m->node_new_of_old[off + q] - lo;
    U_out[3 * q] = (double)U[v].x + (double)L[v].x;
    U_out[3 * q + 1] = (double)U[v].y + (double)L[v].y;
    U_out[3 * q + 2] = (double)U[v].z + (double)L[v].z;
  }
  return DJ_OK;
}

dj_status dj_batch_set_step(dj_batch* b, long long step) {
  if (!b) return DJ_ERR_INVALID_ARG;
  for (int pt = 0; pt < 2; ++pt)
    if (b->part[pt]) {
      dj_status s = dj_set_step(b->part[pt], step);
      if (s) return bfail(b, s, b->part[pt]->last_error.c_str());
    }
  return DJ_OK;
}

dj_status dj_batch_get_displacements_device(dj_batch* b, int i, float* d_out, void* stream) {
  if (!b || i < 0 || i >= b->n || !d_out) return DJ_ERR_INVALID_ARG;
  if (!b->precomputed) return bfail(b, DJ_ERR_NOT_PRECOMPUTED, "call dj_batch_precompute first");
  dj_mesh* m = b->part[b->inst_part[i]];
  const cudaError_t e = launch_to_caller_order(m->d_U, m->d_perm + b->inst_node_off[i], (int)b->inst_nodes[i],
                                               d_out, (cudaStream_t)stream);
  return e == cudaSuccess ? DJ_OK : bfail(b, DJ_ERR_CUDA, cudaGetErrorString(e));
}

dj_status dj_batch_set_displacements(dj_batch* b, int i, const double* U0) {
  if (!b || i < 0 || i >= b->n || !U0) return DJ_ERR_INVALID_ARG;
  if (!b->precomputed) return bfail(b, DJ_ERR_NOT_PRECOMPUTED, "call dj_batch_precompute first");
  dj_mesh* m = b->part[b->inst_part[i]];
  if (cudaDeviceSynchronize() != cudaSuccess) return bfail(b, DJ_ERR_CUDA, "sync failed");
  const long long off = b->inst_node_off[i], nn = b->inst_nodes[i];
  int lo = m->node_new_of_old[off], hi = lo;
  for (long long q = 0; q < nn; ++q) {
    lo = std::min(lo, m->node_new_of_old[off + q]);
    hi = std::max(hi, m->node_new_of_old[off + q]);
  }
  const long long cnt = hi - lo + 1;  // the instance's contiguous internal range
  std::vector<float4> U(cnt), L(cnt), V(cnt);
  for (long long q = 0; q < nn; ++q) {
    const int v = m->node_new_of_old[off + q];
    const int r = v - lo;
    U[r] = make_float4((float)U0[3 * q], (float)U0[3 * q + 1], (float)U0[3 * q + 2], m->h_ai[v]);
    L[r] = make_float4((float)(U0[3 * q] - U[r].x), (float)(U0[3 * q + 1] - U[r].y),
                       (float)(U0[3 * q + 2] - U[r].z), 0.f);
    V[r] = make_float4(0.f, 0.f, 0.f, bits_to_float(m->h_bcidx[v]));
  }
  if (cudaMemcpy(m->d_U + lo, U.data(), cnt * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_V + lo, V.data(), cnt * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
      (m->cmp && cudaMemcpy(m->d_Ulo + lo, L.data(), cnt * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess))
    return bfail(b, DJ_ERR_CUDA, "copy failed");
  return DJ_OK;
}

dj_status dj_batch_get_info(const dj_batch* b, int* n_instances, long long* n_nodes, long long* n_elems,
                            long long* n_tet_elems, long long* n_hex_elems) {
  if (!b) return DJ_ERR_INVALID_ARG;
  long long nn = 0, ne = 0, nt = 0, nh = 0;
  for (int i = 0; i < b->n; ++i) {
    nn += b->inst_nodes[i];
    ne += b->inst_elems[i];
    (b->inst_part[i] == 0 ? nt : nh) += b->inst_elems[i];
  }
  if (n_instances) *n_instances = b->n;
  if (n_nodes) *n_nodes = nn;
  if (n_elems) *n_elems = ne;
  if (n_tet_elems) *n_tet_elems = nt;
  if (n_hex_elems) *n_hex_elems = nh;
  return DJ_OK;
}

dj_status dj_batch_autotune(dj_batch* b, int steps, void* stream) {
  if (!b) return DJ_ERR_INVALID_ARG;
  if (!b->precomputed) return bfail(b, DJ_ERR_NOT_PRECOMPUTED, "call dj_batch_precompute first");
  batch_release_graphs(b);
  for (int pt = 0; pt < 2; ++pt)
    if (b->part[pt]) {
      dj_status s = dj_autotune(b->part[pt], steps, stream, nullptr, nullptr);
      if (s) return bfail(b, s, b->part[pt]->last_error.c_str());
    }
  return DJ_OK;
}

const char* dj_batch_last_error(const dj_batch* b) { return b ? b->last_error.c_str() : "null batch"; }

void dj_batch_destroy(dj_batch* b) {
  if (!b) return;
  batch_release_graphs(b);
  for (int pt = 0; pt < 2; ++pt)
    if (b->part[pt]) dj_mesh_destroy(b->part[pt]);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
}

}  // extern "C"
