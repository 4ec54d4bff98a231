/*
 * dj_tled.h -- C ABI of the GB300 DJ-TLED time-step library.
 *
 * The library advances a hyperelastic finite element mesh in time with the
 * direct Jacobian total Lagrangian explicit dynamics (DJ-TLED) method of
 * J. Zhang, "A direct Jacobian total Lagrangian explicit dynamics finite
 * element algorithm for real-time simulation of hyperelastic materials"
 * (arXiv 2106.14189):
 *
 *   per element   tJ = 0J + H_xi u_e (Eq. 11), J (Eq. 12), g_hat (Eq. 18),
 *                 invariants (Table 1), nodal forces (Table 3)
 *   per node      deterministic gather of the element forces (sum in Eq. 13),
 *                 central-difference update with lumped mass and
 *                 mass-proportional damping (Eq. 13), prescribed displacements
 *
 * Elements: 4-node tetrahedra (volume coordinates) and 8-node bricks with
 * 1-point integration and hourglass control.  Materials (Table 3): neo-Hookean
 * (NH), transversely isotropic NH (TI), orthotropic NH (OT), Mooney-Rivlin (MR).
 *
 * Conventions shared by every call
 *   - Units are SI (m, Pa, kg/m^3, s).
 *   - Node ids and element ids are the caller's, 0-based.  The library
 *     renumbers internally for memory locality; every array passed in or out is
 *     in the caller's order.
 *   - Host pointers (plain C arrays) are copied during the call; the caller
 *     keeps ownership.  Pointers documented as "device" must point to memory of
 *     the current CUDA device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls taking a stream only enqueue work unless documented otherwise.
 *   - Every call returns a dj_status and never throws or aborts.  On failure
 *     dj_last_error(mesh) holds a one-line description.
 *   - A dj_mesh owns all device memory it allocates until dj_mesh_destroy.
 *     A dj_mesh is not thread safe: one host thread at a time.
 */
#ifndef DJ_TLED_H
#define DJ_TLED_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DJ_OK = 0,
  DJ_ERR_INVALID_ARG = 1,       /* bad pointer, size, parameter or call order */
  DJ_ERR_BAD_MESH = 2,          /* empty mesh or connectivity out of range */
  DJ_ERR_INVERTED_ELEMENT = 3,  /* det 0J <= 0 at set-up, or det tJ <= 0 while stepping */
  DJ_ERR_NOT_PRECOMPUTED = 4,   /* stepping before dj_precompute */
  DJ_ERR_NONFINITE = 5,         /* NaN/Inf in a nodal force or displacement */
  DJ_ERR_NOT_CONVERGED = 6,     /* dj_relax_to_tol hit max_steps */
  DJ_ERR_CUDA = 7,              /* a CUDA runtime call failed */
  DJ_ERR_OOM = 8,               /* device or host allocation failed */
  DJ_ERR_UNSUPPORTED = 9        /* combination not built (e.g. no device) */
} dj_status;

enum { DJ_TET4 = 4, DJ_HEX8 = 8 };                    /* element types */
enum { DJ_NH = 0, DJ_TI = 1, DJ_OT = 2, DJ_MR = 3 };  /* Table 3 models */
enum { DJ_RAMP_LINEAR = 0, DJ_RAMP_SMOOTH = 1 };      /* prescribed-value ramps */

typedef struct dj_mesh dj_mesh;

/* Run parameters (Sec. 2.2, Eq. 13-14).
 *   dt                time step [s]; <= 0 selects dt_scale * dt_crit.  A value
 *                     above dt_crit is rejected (DJ_ERR_INVALID_ARG).
 *   dt_scale          fraction of the critical step (default 0.9).
 *   alpha             mass-proportional damping D = alpha M [1/s] (default 0).
 *   hg_coeff          H8 hourglass coefficient kappa_hg (default 0.1).
 *   ramp_steps        prescribed values follow target * s(min(n / ramp_steps, 1))
 *                     at step n; <= 0 applies the targets at once.
 *   ramp_kind         DJ_RAMP_LINEAR: s = tau (Sec. 5.1);
 *                     DJ_RAMP_SMOOTH: s = 10 tau^3 - 15 tau^4 + 6 tau^5.
 *   relax_check_every residual check interval of dj_relax_to_tol (default 100).
 *   renumber          1 (default): reorder nodes and elements along a Morton
 *                     curve for locality; 0: keep the caller's order.
 *   assembly          how element forces reach the nodes (sum in Eq. 13), both
 *                     deterministic: 1 (default) tiles -- each block of
 *                     tile_size consecutive elements sums its forces per node in
 *                     shared memory and the node update gathers one partial per
 *                     (tile, node); 2 tiles with a persistent bulk-copy
 *                     (TMA) pipeline; 0 slots -- every element writes one force
 *                     per node and the node update gathers all of them.
 *   tile_size         elements per tile, a multiple of 32 (T4 <= 512, H8 <= 256);
 *                     0 selects 256 (T4) / 128 (H8); 32 (assembly 1) runs one
 *                     tile per warp.
 *   precision         0 (default): FP32 nodal state and forces.  1: compensated
 *                     FP32 -- the displacement is kept as an unevaluated sum of
 *                     two floats and the element force is evaluated from the
 *                     increment tJ - 0J so that J - 1 and the deviatoric stress
 *                     keep FP32 relative accuracy at small strain; needed to
 *                     relax stiff (kappa / mu ~ 50) meshes to residuals ~1e-5.
 *   anp               0 (default): the element volumetric term of Table 3.
 *                     1: average nodal pressure (Sec. 7's remedy for volumetric
 *                     locking; T4 with assembly 2 only, else
 *                     DJ_ERR_INVALID_ARG): the nodal volume ratio J_i = V_i / V0_i
 *                     from the element volumes shared equally by their nodes,
 *                     p_i = kappa_i (J_i - 1) with kappa_i the volume-weighted
 *                     bulk modulus, and each element's volumetric factor
 *                     kappa (J - 1) replaced by the mean of its nodes' p_i.  Two
 *                     more kernels per step (element volumes, nodal pressures).
 *   graph_pdl         0 (default): the steps captured into CUDA graphs
 *                     (dj_run_n, relaxation) are joined by ordinary edges;
 *                     1: by programmatic-launch edges, as directly launched
 *                     steps are (faster on small meshes; dj_autotune tries
 *                     both).
 *   max_blocks        assembly 2 only: upper limit on the blocks of the
 *                     persistent kernel, each of which walks the tiles
 *                     b, b + grid, b + 2 grid, ...; 0 (default) = SMs x resident
 *                     blocks per SM (one wave).  A small value makes every block
 *                     walk many tiles, the steady state of its copy pipeline.
 *                     Negative values are rejected (DJ_ERR_INVALID_ARG). */
typedef struct {
  double dt;
  double dt_scale;
  double alpha;
  double hg_coeff;
  long long ramp_steps;
  int ramp_kind;
  int relax_check_every;
  int renumber;
  int assembly;
  int tile_size;
  int precision;
  int anp;
  int graph_pdl;
  int max_blocks;
} dj_params;

/* Read-only description of a mesh after dj_precompute. */
typedef struct {
  long long n_nodes, n_elems, n_bc_dofs, step;
  int elem_type;            /* DJ_TET4 or DJ_HEX8 */
  int model_flags;          /* bit m set when some element uses model m */
  double dt, dt_crit;       /* time step in use and the critical step (Eq. 14) */
  double total_mass;        /* sum of the lumped nodal masses [kg] */
  long long device_bytes;   /* device memory held by the mesh */
  long long elem_table_bytes_per_elem;  /* bytes of per-element tables read per step */
  long long slot_bytes_per_elem;        /* bytes of element-force slots written per step */
  long long gather_index_bytes;         /* bytes of the node gather index */
  long long node_bytes_per_node;        /* bytes of node state read + written per step */
  long long n_parts;        /* tiled assembly: number of (tile, node) partial forces */
  int assembly;             /* assembly in use (see dj_params) */
  int tile_size;            /* elements per tile (tiled assembly) */
  int n_consts;             /* floats per element in the element table */
  int precision;            /* precision mode in use (see dj_params) */
  int grid;                 /* assembly 2: blocks of the persistent kernel (else 0) */
  long long n_tiles;        /* tiled assembly: number of tiles (else 0) */
} dj_info;

/* Fill *p with the defaults listed above. */
void dj_params_default(dj_params* p);

/* Create a mesh (Sec. 2.1.2: isoparametric T4 / H8 elements).
 *   elem_type  DJ_TET4 or DJ_HEX8
 *   X          host, n_nodes * 3 doubles, row-major reference coordinates 0x
 *   conn       host, n_elems * elem_type ints, 0-based node ids.  T4: any order
 *              with det 0J > 0 (0J = H_xi X_e, Eq. 3, volume coordinates);
 *              H8: bottom face counter-clockwise seen from above, then top face.
 *   out        receives the handle (NULL on failure)
 * Errors: DJ_ERR_INVALID_ARG (null pointer, bad type, non-finite X),
 *         DJ_ERR_BAD_MESH (n_nodes <= 0, n_elems <= 0, id out of range). */
dj_status dj_mesh_create(int elem_type, const double* X, long long n_nodes,
                         const int* conn, long long n_elems, dj_mesh** out);

/* Per-element material (Table 3), all host arrays of n_elems entries:
 *   model   DJ_NH / DJ_TI / DJ_OT / DJ_MR
 *   mu      shear modulus (MR: mu = 2 C10), kappa bulk modulus, rho density
 *   eta_a, eta_b  fibre stiffnesses (TI uses eta_a, OT both; NULL = 0)
 *   c01     Mooney-Rivlin C01 (NULL = 0)
 *   a_dir, b_dir  n_elems * 3 fibre directions 0a, 0b (normalised here;
 *           NULL = x and y axes)
 * Every element defaults to NH with mu = kappa = rho = 0 until this is called.
 * Errors: DJ_ERR_INVALID_ARG (mu, kappa, rho <= 0; eta, c01 < 0; zero fibre
 *         direction on a fibre element; unknown model). */
dj_status dj_mesh_set_materials(dj_mesh* mesh, const unsigned char* model, const double* mu,
                                const double* kappa, const double* rho, const double* eta_a,
                                const double* eta_b, const double* c01, const double* a_dir,
                                const double* b_dir);

/* Prescribed displacements (Sec. 5.1, Sec. 6: fixed and ramped DOFs).
 *   dof     host, n entries, dof = 3 * node + component (0 x, 1 y, 2 z)
 *   target  host, n final values [m]; 0 = fixed DOF
 * Replaces any earlier list; n = 0 clears it.  Duplicate DOFs are rejected.
 * Must be called before dj_precompute. */
dj_status dj_mesh_set_bcs(dj_mesh* mesh, const long long* dof, const double* target, long long n);

/* Replace the target values of the current prescribed-DOF list (same order as
 * the last dj_mesh_set_bcs).  Allowed after dj_precompute; takes effect on the
 * next step.  Host array of n_bc_dofs doubles, read before the call returns:
 * a page-locked, 8-byte aligned array is read by the library's kernel through
 * its device mapping (one launch on the legacy default stream, then a
 * synchronisation of that stream); other host memory is staged in a
 * page-locked copy of the per-node table and copied once.  Steps still in
 * flight on a non-blocking stream are not waited for.
 * Errors: DJ_ERR_INVALID_ARG (null or non-finite target; nothing changes). */
dj_status dj_mesh_update_bc_targets(dj_mesh* mesh, const double* target);

/* Independent bodies in one mesh (used for batches of problems).  elem_group:
 * host, n_elems ints in [0, n_groups); elements of different groups must not
 * share a node (DJ_ERR_INVALID_ARG otherwise).  Each group gets its own
 * critical step (Eq. 14) and time step dt_scale * dt_crit(group) (or
 * params.dt, which must not exceed any group's critical step), its own
 * damping factor, and its own relaxation residual; dj_relax_to_tol converges
 * when every group's residual is <= tol.  The ramp is shared (in steps).
 * NULL or n_groups <= 0 removes the grouping.  Before dj_precompute. */
dj_status dj_mesh_set_groups(dj_mesh* mesh, const int* elem_group, int n_groups);

/* External nodal forces R (Eq. 13), host n_nodes * 3 doubles, constant in
 * time; NULL clears them.  Must be called before dj_precompute.
 * Errors: DJ_ERR_INVALID_ARG for a value that is not finite in single precision. */
dj_status dj_mesh_set_loads(dj_mesh* mesh, const double* R);

/* One-time set-up on the current CUDA device (Algorithm 1, pre-computation):
 * FP64 evaluation of 0J, det 0J, 0V, I1m, I4m, I6m (Table 2), hourglass
 * constants, lumped mass and the critical step (Eq. 14), then FP32 tables.
 * Resets the state to rest (U^0 = U^-1 = 0, step 0).  Synchronous.
 *   dt_out  optional, receives the time step in use
 * Errors: DJ_ERR_INVERTED_ELEMENT (det 0J <= 0, message names the element),
 *         DJ_ERR_INVALID_ARG (dt above the critical step), DJ_ERR_CUDA, DJ_ERR_OOM. */
dj_status dj_precompute(dj_mesh* mesh, const dj_params* params, double* dt_out);

/* Advance one time step (Algorithm 1 runtime loop + central difference, Eq. 13)
 * on `stream`.  Asynchronous: element inversion or non-finite forces raised
 * during the step are reported by the next dj_sync / dj_get_displacements. */
dj_status dj_step(dj_mesh* mesh, void* stream);

/* Advance n >= 0 steps on `stream` (replays of a captured CUDA graph). Async. */
dj_status dj_run_n(dj_mesh* mesh, long long n, void* stream);

/* Device time of one launch of each kernel of the step, each launch timed
 * alone with CUDA events on `stream`: `launches` launches of the element-force
 * kernel (no clock advance), then `launches` of the node update kernel (on a
 * saved copy of U and V, restored afterwards).  With d_flush non-NULL
 * (caller-owned device buffer of flush_bytes, at least twice the L2 size) every
 * launch is preceded by an L2 eviction (the first half of the buffer written,
 * the second half read), so each launch starts with a cold cache.
 * ms_force / ms_update (optional) receive the mean per launch.  Synchronous;
 * allocates two state copies.  Not a counterpart of anything in the paper. */
dj_status dj_profile_kernels(dj_mesh* mesh, int launches, void* d_flush, size_t flush_bytes, void* stream,
                             double* ms_force, double* ms_update);

/* Advance n steps (as dj_run_n), then measure the device time of each kernel
 * of the step: the element-force kernel and the node update kernel are each
 * replayed back to back in a CUDA graph (the update on a saved copy of the
 * state, restored afterwards), for min(n, 64) x max(1, n / 64) launches.
 * ms_force / ms_update (optional) receive the time per launch times n.
 * Synchronous. */
dj_status dj_run_n_profiled(dj_mesh* mesh, long long n, void* stream, double* ms_force,
                            double* ms_update);

/* Autotuner: time `steps` steps of each schedule -- assembly (slots, tiles,
 * tiles with the bulk-copy pipeline) x tile size (64 ... 512) -- on this mesh
 * from its current state, keep the fastest, and restore the state (so the
 * trajectory continues unchanged).  chosen (optional) receives the parameters
 * in use afterwards, ms_per_step (optional) their time per step.
 * Synchronous; re-runs dj_precompute for every candidate. */
dj_status dj_autotune(dj_mesh* mesh, int steps, void* stream, dj_params* chosen, double* ms_per_step);

/* dj_autotune for a cold L2 cache: with d_flush non-NULL (caller-owned device
 * buffer of flush_bytes, at least twice the L2 size) every timed step runs
 * alone after an L2 eviction (the first half of the buffer written, the second
 * read), so the choice fits meshes stepped between other work; with d_flush
 * NULL it is dj_autotune.  Synchronous. */
dj_status dj_autotune_cold(dj_mesh* mesh, int steps, void* d_flush, size_t flush_bytes, void* stream,
                           dj_params* chosen, double* ms_per_step);

/* Wait for `stream` and report device-side errors of earlier steps
 * (DJ_ERR_INVERTED_ELEMENT / DJ_ERR_NONFINITE). */
dj_status dj_sync(dj_mesh* mesh, void* stream);

/* Dynamic relaxation (Sec. 6): step with the current damping until the
 * residual r = ||F - R||_free / ||F - R||_prescribed (FP64, every
 * relax_check_every steps) is <= tol, or max_steps steps were taken.  A checked
 * state counts only once its step index is >= ramp_steps (prescribed values at
 * their targets).  On success the state is one step past the checked one.
 * Synchronous.
 *   steps_out, residual_out  optional
 * Errors: DJ_ERR_NOT_CONVERGED, DJ_ERR_INVERTED_ELEMENT, DJ_ERR_NONFINITE. */
dj_status dj_relax_to_tol(dj_mesh* mesh, double tol, long long max_steps, long long* steps_out,
                          double* residual_out, void* stream);

/* Options of adaptive dynamic relaxation (dj_relax_adaptive).
 *   alpha_min, alpha_max  clamp of the damping estimate [1/s]; alpha_max <= 0
 *                         selects 2 / dt (b = 1: no momentum carried over).
 *   disp_tol              > 0: a state also needs the estimated displacement
 *                         error err_est <= disp_tol [m] to count as converged;
 *                         <= 0: the residual test alone. */
typedef struct {
  double alpha_min;
  double alpha_max;
  double disp_tol;
} dj_adr_params;

/* What dj_relax_adaptive measured at its last check.
 *   alpha        damping in use at the end [1/s]
 *   lambda       last Rayleigh quotient of M^-1 K along the increment [1/s^2]
 *                (0: no estimate was made)
 *   rho          per-step convergence rate from ||D|| at the last two checks
 *                (0: none)
 *   err_est      r / (1 - r) max|D| over free DOFs [m], r = rho^k (inf: none)
 *   n_estimates  damping updates made */
typedef struct {
  double alpha;
  double lambda;
  double rho;
  double err_est;
  long long n_estimates;
} dj_adr_report;

/* Adaptive dynamic relaxation (Sec. 6 relaxes with fixed damping; this is the
 * adaptive variant of the method it cites): dj_relax_to_tol whose damping is
 * re-estimated at every check once the ramp is over.  With D = U^n - U^{n-k}
 * the change over the check interval k = relax_check_every and F the internal
 * force, the Rayleigh quotient
 *   lambda = D . (F(U^n) - F(U^{n-k})) / (D . M D)   (free DOFs, FP64 sums)
 * estimates the lowest eigenvalue of M^-1 K that the load excites (D tends to
 * the slowest mode), and alpha = 2 sqrt(lambda), clamped to [alpha_min,
 * alpha_max], damps that mode critically.  The contraction r = ||D|| / ||D of
 * the previous interval|| gives rho = r^(1/k) and err_est = r / (1 - r) max|D|.
 * The damping starts from the mesh's alpha; the mesh's own damping (dj_step,
 * dj_run_n, dj_relax_to_tol) is not changed.  Not for meshes with groups
 * (DJ_ERR_INVALID_ARG).  Synchronous.
 *   opts        NULL: alpha_min 0, alpha_max 2 / dt, disp_tol 0
 *   steps_out, residual_out, report  optional
 * Errors: as dj_relax_to_tol. */
dj_status dj_relax_adaptive(dj_mesh* mesh, double tol, long long max_steps, const dj_adr_params* opts,
                            long long* steps_out, double* residual_out, dj_adr_report* report,
                            void* stream);

/* Warm start: U^0 = U^-1 = U0 (host, n_nodes * 3 doubles); step counter kept;
 * the error record (inverted / non-finite flags) is cleared, since the field
 * starts a new trajectory.  Synchronous. */
dj_status dj_set_displacements(dj_mesh* mesh, const double* U0);

/* Current displacements U^n, host n_nodes * 3 doubles (caller order).
 * Synchronizes the device and reports pending device-side errors.  When U_out
 * is page-locked (cudaHostAlloc / cudaHostRegister) and 8-byte aligned the
 * library's kernel writes it directly through its device mapping; other host
 * memory receives one copy from a device buffer. */
dj_status dj_get_displacements(dj_mesh* mesh, double* U_out);

/* One time step with its input and output in host memory, for callers that
 * drive the solver from the host every step (Eq. 13 with the prescribed
 * values of Sec. 5.1 / Sec. 6): the prescribed targets of this step (host,
 * n_bc doubles in the order of dj_mesh_set_bcs, as dj_mesh_update_bc_targets;
 * NULL keeps the current ones), one step (as dj_step), then U^{n+1} in caller
 * order into U_out (host, n_nodes * 3 values, doubles when out_f64 = 1, floats
 * when out_f64 = 0; NULL skips the read-back).  Everything is enqueued on
 * `stream` and the call synchronises once, at its end, so the caller may
 * reuse both buffers on return.  Page-locked targets are read by the
 * element-force kernel through their device mapping (coalesced, beside its
 * own work) into a device copy that the update kernel applies; other host
 * memory is copied to the device before the step.  A page-locked, 8-byte
 * aligned U_out is written by
 * the library's kernel through its device mapping, other host memory
 * through one copy.  The FP32 output holds U + low part rounded once
 * (exactly U in the plain FP32 precision mode).
 * Errors: as dj_step; device-side flags (inverted element, non-finite value)
 * are reported by this call.  A non-finite target is detected on the device:
 * that entry is not applied -- the DOF keeps its previous target for the
 * step -- and the call returns DJ_ERR_INVALID_ARG after the step. */
dj_status dj_step_host(dj_mesh* mesh, const double* targets, void* U_out, int out_f64, void* stream);

/* Current displacements into device memory, n_nodes * 3 floats in caller
 * order, enqueued on `stream`. */
dj_status dj_get_displacements_device(dj_mesh* mesh, float* d_U_out, void* stream);

/* Set the step counter n (synchronous).  Prescribed values follow
 * target * s(min(n / ramp_steps, 1)), so a warm-started relaxation sets
 * n >= ramp_steps to hold the targets from its first step. */
dj_status dj_set_step(dj_mesh* mesh, long long step);

/* Warm start from device memory: U^0 = U^-1 = d_U0 (n_nodes * 3 floats, caller
 * order); enqueued on `stream`; compensated low parts are reset to 0 and the
 * error record is cleared as in dj_set_displacements. */
dj_status dj_set_displacements_device(dj_mesh* mesh, const float* d_U0, void* stream);

/* Evaluate a candidate field d_U (device, n_nodes * 3 floats, caller order)
 * without changing the stepping state: residual_out receives the relaxation
 * residual r = ||F - R||_free / ||F - R||_prescribed of that field (largest
 * group residual for grouped meshes; +inf when an element is inverted) and
 * inverted_out 1 if some element of the field has det tJ <= 0.  Synchronous. */
dj_status dj_evaluate_field(dj_mesh* mesh, const float* d_U, double* residual_out, int* inverted_out,
                            void* stream);

/* Assembled internal forces F(U) = sum_e F^(e) (Eq. 13) for host displacements
 * U (n_nodes * 3 doubles), written to host F_out (n_nodes * 3).  The stepping
 * state is left unchanged.  Synchronous. */
dj_status dj_internal_forces(dj_mesh* mesh, const double* U, double* F_out);

/* Checkpoint: opaque, bit-exact copy of the stepping state (U^n, U^n - U^n-1,
 * step counter).  dj_set_state on the same mesh resumes bit-identically. */
dj_status dj_state_size(const dj_mesh* mesh, size_t* bytes);
dj_status dj_get_state(dj_mesh* mesh, void* buf, size_t bytes);
dj_status dj_set_state(dj_mesh* mesh, const void* buf, size_t bytes);

dj_status dj_get_info(const dj_mesh* mesh, dj_info* info);

/* Per group (1 group when the mesh has no grouping): time step, critical step
 * and the residual of the last dj_relax_to_tol check (NaN before any).  Arrays
 * are optional, each of *n_groups doubles. */
dj_status dj_get_group_info(const dj_mesh* mesh, int* n_groups, double* dt, double* dt_crit,
                            double* residual);
const char* dj_status_string(dj_status s);
const char* dj_last_error(const dj_mesh* mesh);
void dj_mesh_destroy(dj_mesh* mesh);

/* ---------------------------------------------------------------------------
 * Batches of independent problems of uneven size (no counterpart in the
 * paper, which runs one mesh at a time).  Instances of the same element type
 * are merged into one grouped mesh (see dj_mesh_set_groups): every instance
 * keeps its own time step, damping factor and residual; the T4 and H8 parts
 * advance as two independent kernel chains captured in one CUDA graph.
 * ------------------------------------------------------------------------- */
typedef struct dj_batch dj_batch;

/* instances: n meshes with materials (and prescribed DOFs, loads) set; they
 * need not be precomputed.  Their host data is copied: the handles stay owned
 * by the caller and may be destroyed afterwards. */
dj_status dj_batch_create(dj_mesh* const* instances, int n, dj_batch** out);
/* dj_precompute of every part with the same parameters (synchronous). */
dj_status dj_batch_precompute(dj_batch* batch, const dj_params* params);
/* Advance every instance n steps (async, graph replays). */
dj_status dj_batch_run_n(dj_batch* batch, long long n, void* stream);
/* Wait and report device-side errors of every part. */
dj_status dj_batch_sync(dj_batch* batch, void* stream);
/* Relax every instance until each residual is <= tol (checked every
 * relax_check_every steps); residual_out = the largest instance residual. */
dj_status dj_batch_relax_to_tol(dj_batch* batch, double tol, long long max_steps,
                                long long* steps_out, double* residual_out, void* stream);
/* Instance i: node and element counts, its time step and its last residual. */
dj_status dj_batch_instance_info(dj_batch* batch, int i, long long* n_nodes, long long* n_elems,
                                 double* dt, double* residual);
/* Displacements of instance i (host, its n_nodes * 3 doubles, its node order). */
dj_status dj_batch_get_displacements(dj_batch* batch, int i, double* U_out);
/* dj_set_step on every instance. */
dj_status dj_batch_set_step(dj_batch* batch, long long step);
/* Displacements of instance i into device memory (its n_nodes * 3 floats, its
 * node order), enqueued on `stream`. */
dj_status dj_batch_get_displacements_device(dj_batch* batch, int i, float* d_U_out, void* stream);
/* Warm start of instance i: U^0 = U^-1 = U0.  Synchronous. */
dj_status dj_batch_set_displacements(dj_batch* batch, int i, const double* U0);
dj_status dj_batch_get_info(const dj_batch* batch, int* n_instances, long long* n_nodes,
                            long long* n_elems, long long* n_tet_elems, long long* n_hex_elems);
/* dj_autotune of each part (T4 instances, H8 instances) of the batch. */
dj_status dj_batch_autotune(dj_batch* batch, int steps, void* stream);
const char* dj_batch_last_error(const dj_batch* batch);
void dj_batch_destroy(dj_batch* batch);

/* Allocation-free residual norms (no counterpart in the paper).  For callers
 * that cannot allocate device memory when they need the residual -- code that
 * runs inside another framework's memory pool, real-time loops that must not
 * enter the allocator, plugins that only receive buffers from their host
 * application.  It computes the two FP64 sums of the dj_relax_to_tol residual,
 * d_out[0] = sum of F^2 over free DOFs and d_out[1] = sum of F^2 over
 * prescribed DOFs, from caller buffers:
 *   d_F           device, n_nodes * 3 floats (F - R per DOF)
 *   d_prescribed  device, n_nodes * 3 bytes, nonzero = prescribed DOF
 *   d_out         device, 2 doubles
 * Its block partial sums live in a fixed 1 MiB device array inside the library
 * (held on every GPU that loads the library until the process exits), so it
 * calls no allocator.  n_nodes must be <= 16,777,216 (65536 blocks of 256
 * nodes); larger inputs return DJ_ERR_UNSUPPORTED, null pointers or
 * n_nodes <= 0 DJ_ERR_INVALID_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) for the current device: make
 * that first call outside stream capture.  Enqueued on `stream`.  All calls
 * share the array and each overwrites the slots it uses, so calls that overlap
 * on the GPU (other streams, other threads) race and must be serialized. */
dj_status dj_residual_norms_static(const float* d_F, const unsigned char* d_prescribed, long long n_nodes,
                                   double* d_out, void* stream);

/* ---------------------------------------------------------------------------
 * Learned warm start for dynamic relaxation (no counterpart in the paper, which
 * names learning only as future work, Sec. 8): proper orthogonal decomposition
 * of fields and a multilayer perceptron trained with the library's kernels.
 * All float pointers below are device memory; matrices are row-major unless
 * stated.
 * ------------------------------------------------------------------------- */
typedef struct dj_mlp dj_mlp;

/* MLP with n_layers affine layers of widths[0] -> ... -> widths[n_layers],
 * tanh between layers, linear output.  Weights Glorot-uniform from `seed`,
 * biases 0.  Parameters packed as [W_1 (out x in), b_1, W_2, b_2, ...]. */
dj_status dj_mlp_create(const int* widths, int n_layers, unsigned long long seed, dj_mlp** out);
long long dj_mlp_num_params(const dj_mlp* mlp);
dj_status dj_mlp_get_params(dj_mlp* mlp, float* host, long long n);
/* Replace the parameters (host) and reset the Adam moments. */
dj_status dj_mlp_set_params(dj_mlp* mlp, const float* host, long long n);
dj_status dj_mlp_get_grads(dj_mlp* mlp, float* host, long long n);
/* Y (batch x out) = MLP(X (batch x in)). */
dj_status dj_mlp_forward(dj_mlp* mlp, const float* d_X, int batch, float* d_Y, void* stream);
/* Forward + backward of L = 1/(batch n_out) sum_ij w_j (Y_ij - T_ij)^2 (w: n_out
 * weights or NULL); gradients overwrite the internal gradient buffer.
 * loss_out (host, optional) synchronizes the stream. */
dj_status dj_mlp_loss_grad(dj_mlp* mlp, const float* d_X, const float* d_T, const float* d_w, int batch,
                           double* loss_out, void* stream);
/* One Adam step with bias correction on the last gradients. */
dj_status dj_mlp_adam_step(dj_mlp* mlp, float lr, float beta1, float beta2, float eps, void* stream);
const char* dj_mlp_last_error(const dj_mlp* mlp);
void dj_mlp_destroy(dj_mlp* mlp);

/* POD of cols snapshots of length rows (d_Y column-major: snapshot c at
 * d_Y + c * rows; cols <= 65536, r <= min(cols, 1024)): d_mean (rows) the
 * snapshot mean, d_modes (rows x r, row-major) the r leading orthonormal modes
 * of the centred snapshots Yc, sigma_out (host, optional, r) their singular
 * values.  Method: randomised range finder on the GPU, Z = Yc Omega with a
 * seeded normal Omega of l = min(cols, r + max(32, r / 2)) columns, three
 * subspace-iteration steps (none when l = cols, where the result is the exact
 * truncated SVD), each product orthonormalised through the eigen-decomposition
 * of its l x l Gram matrix, then a Rayleigh-Ritz step on (Yc^T Z)^T (Yc^T Z);
 * products with FP64 slab accumulation, the l x l eigenproblems in FP64 on
 * the host (dj_symmetric_eigen).  Modes beyond the numerical rank of the
 * snapshots are zero with sigma 0.  Allocates about (cols + 2 l) rows floats
 * of device scratch; synchronous.
 * Errors: DJ_ERR_INVALID_ARG (sizes), DJ_ERR_OOM, DJ_ERR_CUDA. */
dj_status dj_pod_fit(const float* d_Y, long long rows, int cols, int r, float* d_mean, float* d_modes,
                     double* sigma_out, void* stream);
/* Eigen-decomposition of a symmetric n x n matrix (host, FP64, no device
 * work; no counterpart in the paper): the cyclic Jacobi method, sweeping the
 * pairs (p, q) row by row with the plane rotation that zeroes a_pq, until the
 * off-diagonal part is below 1e-15 of the matrix in Frobenius norm.  A
 * (row-major, host) is read and symmetrised as (A + A^T) / 2; w (host, n) gets
 * the eigenvalues in descending order, V (host, row-major n x n, optional) the
 * orthonormal eigenvectors as columns in the same order.  n <= 4096 (cost
 * grows as n^3 per sweep: meant for the POD's small Rayleigh-Ritz problems).
 * Errors: DJ_ERR_INVALID_ARG (null pointer, size, non-finite entry). */
dj_status dj_symmetric_eigen(const double* A, int n, double* w, double* V);
/* d_Q (cols x r) = (X - mean)^T modes for column-major d_X (rows x cols);
 * d_mean may be NULL.  Enqueued on `stream`; allocates nothing. */
dj_status dj_pod_project(const float* d_modes, const float* d_mean, long long rows, int r, const float* d_X,
                         int cols, float* d_Q, void* stream);
/* d_X (column-major rows x cols) = mean + modes Q^T for d_Q (cols x r). */
dj_status dj_pod_expand(const float* d_modes, const float* d_mean, long long rows, int r, const float* d_Q,
                        int cols, float* d_X, void* stream);

/* Ridge least squares (the linear part of the warm-start map; no counterpart in
 * the paper): d_W (n_out x n_in, row-major) minimises
 * |X W^T - Y|^2 + ridge * tr(X^T X) / n_in * |W|^2 for d_X (S x n_in) and d_Y
 * (S x n_out), both row-major device arrays.  Products on the device (FP64
 * accumulation, FP32 storage), FP64 Cholesky solve on the host; if the
 * regularised normal equations are not positive definite the ridge is raised
 * tenfold, at most four times (from 1e-7 when ridge = 0).  n_in <= 1024.
 * Synchronous.
 * Errors: DJ_ERR_INVALID_ARG (sizes, ridge < 0, or normal equations that stay
 * indefinite), DJ_ERR_CUDA. */
dj_status dj_linear_fit(const float* d_X, const float* d_Y, int S, int n_in, int n_out, double ridge,
                        float* d_W, void* stream);
/* Second-order features for the warm-start map (no counterpart in the paper):
 * row s of d_F (S x (n + n (n + 1) / 2), row-major) holds the first n entries x
 * of row s of d_X (leading dimension ld >= n) followed by x_i x_j for i <= j,
 * row by row.  n <= 256.  Enqueued on `stream`; allocates nothing. */
dj_status dj_quad_features(const float* d_X, int S, int ld, int n, float* d_F, void* stream);
/* d_Y (S x n_out) = alpha X W^T + beta Y for d_X (S x n_in) and d_W (n_out x n_in),
 * row-major device arrays; enqueued on `stream`; allocates nothing. */
dj_status dj_linear_apply(const float* d_W, int n_out, int n_in, const float* d_X, int S, float alpha, float beta,
                          float* d_Y, void* stream);

/* BF16 variant of an MLP (no counterpart in the paper): precision 1 runs the
 * forward and backward products on the tensor cores (tcgen05.mma, BF16
 * operands rounded from the FP32 values, FP32 accumulation in tensor memory);
 * precision 2 rounds the same operands to BF16 but multiplies on the CUDA
 * cores (a reference for the first); the master weights, Adam moments,
 * biases, tanh and loss stay FP32.  precision 0 (default) is plain FP32.
 * Errors: DJ_ERR_INVALID_ARG. */
dj_status dj_mlp_set_precision(dj_mlp* mlp, int precision);

/* ------------------------------------------------------------------------
 * Learned warm start for dynamic relaxation (no counterpart in the paper,
 * which names learning methods only as future work, Sec. 8; the relaxation
 * it serves is that of Sec. 6).  A dj_ws maps the prescribed values t of a
 * load case (n_bc floats, in the order of dj_mesh_set_bcs) to an initial
 * nodal field:
 *   c  = Phi_in^T (t - mean_in)       leading n_in POD coefficients of the
 *                                     targets, scaled to unit spread over the
 *                                     training loads (modes below 1e-4 of the
 *                                     largest singular value are switched off)
 *   q  = W f(c) [+ MLP(x)]            f(c): the kept coefficients (first order)
 *                                     or those and their pairwise products
 *                                     (second order); W by ridge least squares;
 *                                     the MLP (input x = c or f(c)) is trained
 *                                     on what W leaves
 *   U0 = mean_out + Phi_out q         leading n_out POD modes of the relaxed
 *                                     fields, scaled by their spread
 * A seeded share of the loads is held out: it chooses the polynomial order
 * and (mlp = -1) whether the MLP is kept.  Training uses the library's
 * kernels only (POD, features, normal equations, MLP forward / backward /
 * Adam); the held-out losses are computed on the host from at most a few
 * hundred rows.
 * ---------------------------------------------------------------------- */
typedef struct dj_ws dj_ws;

enum { DJ_WS_MLP_ON_COEFFS = 0, DJ_WS_MLP_ON_FEATURES = 1 };    /* MLP input */
enum { DJ_WS_PARTS_FITTED = 0, DJ_WS_PARTS_POLYNOMIAL = 1, DJ_WS_PARTS_MLP = 2 };  /* prediction parts (bits) */
enum { DJ_WS_ARM_REST = 0, DJ_WS_ARM_POLYNOMIAL = 1, DJ_WS_ARM_FITTED = 2 };  /* dj_ws_relax_to_tol */

/* Warm-start options (dj_ws_params_default fills the defaults):
 *   n_in, n_out     POD modes of targets / relaxed fields (64, 128; <= 256 / 1024)
 *   hidden[4]       MLP hidden widths, 0 ends the list (256, 256, 256, 0); tanh
 *   epochs, batch   MLP training: passes over the training loads, minibatch rows
 *                   (1500, 128); one seeded permutation of the rows per epoch
 *   lr, lr_final    Adam step, decayed exponentially over the iterations (1e-3, 1e-5)
 *   quadratic       1: the second-order polynomial part may be chosen (1)
 *   mlp             -1: train the MLP and keep it only if it lowers the held-out
 *                   loss (default); 1: train and keep it; 0: no MLP
 *   mlp_input       DJ_WS_MLP_ON_COEFFS (default) or DJ_WS_MLP_ON_FEATURES
 *   mlp_bf16        1: BF16 products in the MLP (dj_mlp_set_precision)
 *   holdout         share of the loads held out (0.1; none below 20 loads)
 *   seed            split, minibatch and MLP initialisation seed
 *   adaptive        1: relaxations use dj_relax_adaptive (default), 0: dj_relax_to_tol
 *   bootstrap       dj_ws_train only: 0 (default) relaxes every training load
 *                   from rest; k >= 20 fits a warm start to the first k loads
 *                   relaxed, relaxes the following ones from it
 *                   (dj_ws_relax_to_tol, fitted arm, same tolerance: the
 *                   training fields are still the method's relaxations) and
 *                   refits each time the number of loads relaxed doubles */
typedef struct {
  int n_in, n_out;
  int hidden[4];
  int epochs, batch;
  double lr, lr_final;
  int quadratic;
  int mlp;
  int mlp_input;
  int mlp_bf16;
  double holdout;
  unsigned long long seed;
  int adaptive;
  int bootstrap;
} dj_ws_params;

/* What the fit found (held-out losses: the weighted mean squared error of the
 * output coefficients, weights = variance shares of the output modes; NaN
 * when not computed). */
typedef struct {
  int n_loads, n_kept;           /* loads given / relaxed successfully */
  int n_train, n_holdout;
  int n_in, n_out, n_in_kept, n_out_kept, n_features, n_bc;
  long long n_dof;
  int quadratic_used, mlp_used;
  long long mlp_params, mlp_iterations;
  double val_loss_first_order, val_loss_second_order;
  double val_loss_polynomial;     /* of the polynomial part chosen */
  double val_loss_polynomial_mlp; /* polynomial part + MLP */
  double final_train_loss;        /* MLP loss on the last minibatch */
  double mean_training_steps;     /* dj_ws_train: mean relaxation steps of the kept loads */
  double data_seconds, fit_seconds, fit_seconds_polynomial;
} dj_ws_info;

/* Outcome of dj_ws_relax_to_tol. */
typedef struct {
  long long steps;                 /* relaxation steps in total (incl. a failed warm attempt) */
  long long steps_warm_attempt;    /* steps of a warm relaxation that failed, else 0 */
  double residual;                 /* residual reached */
  int started_warm;                /* 1: the answer was relaxed from the prediction */
  int fallback;                    /* 1: the prediction was rejected or its relaxation failed */
  double residual_predicted;       /* residual of the predicted field (inf if inverted) */
  double residual_prescribed_only; /* residual of the field with only the prescribed values */
  double predict_seconds;          /* wall time up to the start of the relaxation */
  double seconds;                  /* wall time of the whole call */
} dj_ws_result;

void dj_ws_params_default(dj_ws_params* p);

/* Train a warm start on `mesh` (precomputed, with its prescribed DOFs set):
 * every load case (targets: host, n_loads x n_bc doubles, row by row, each in
 * the order of dj_mesh_set_bcs) is relaxed from rest to `tol` with the mesh's
 * parameters (dj_relax_adaptive or dj_relax_to_tol, see params.adaptive);
 * cases that fail (an element inverts, no convergence in max_steps) are
 * dropped; the method's own relaxed fields are the training data of the fit
 * described above.  The mesh's targets and state are left at the last case.
 * Synchronous; allocates n_loads x (3 n_nodes + n_bc) floats of device memory
 * for the training data (freed before return) and the model's own buffers.
 * Errors: DJ_ERR_INVALID_ARG (arguments, options), DJ_ERR_NOT_CONVERGED (fewer
 * than two cases relaxed), DJ_ERR_OOM, DJ_ERR_CUDA; *out stays NULL. */
dj_status dj_ws_train(dj_mesh* mesh, const double* targets, int n_loads, double tol, long long max_steps,
                      const dj_ws_params* params, dj_ws** out, void* stream);

/* The same fit from caller-supplied training data: d_targets (device,
 * n_loads x n_bc floats) and d_fields (device, n_loads x 3 n_nodes floats, each
 * a relaxed field in caller node order), bc_dof (host, n_bc flat DOF indices
 * 3 node + component, the order of the targets).  Synchronous. */
dj_status dj_ws_fit(const long long* bc_dof, int n_bc, long long n_nodes, const float* d_targets,
                    const float* d_fields, int n_loads, const dj_ws_params* params, dj_ws** out, void* stream);

/* Predicted field for targets (host, n_bc doubles) into d_field (device,
 * 3 n_nodes floats, caller order): parts = DJ_WS_PARTS_FITTED (what the fit
 * kept), DJ_WS_PARTS_POLYNOMIAL, DJ_WS_PARTS_MLP or both bits.  Synchronous. */
dj_status dj_ws_predict(dj_ws* ws, const double* targets, int parts, float* d_field, void* stream);

/* Relax `mesh` for the load case `targets` (host, n_bc doubles) to `tol`:
 *   DJ_WS_ARM_REST        from rest (the plain method; the reference arm);
 *   DJ_WS_ARM_POLYNOMIAL  from the polynomial part's prediction;
 *   DJ_WS_ARM_FITTED      from the fitted map (polynomial part + MLP if kept).
 * A prediction is used only if it inverts no element and its residual is below
 * that of the field holding the prescribed values alone; then the state is set
 * to it with the step counter at the end of the ramp.  Otherwise, or if the
 * warm relaxation fails, the case is relaxed from rest (fallback).  The mesh
 * must be the one the warm start was trained for (same nodes and prescribed
 * DOFs).  res (optional) receives the outcome.  Synchronous.
 * Errors: DJ_ERR_INVALID_ARG, the relaxation's status (e.g.
 * DJ_ERR_NOT_CONVERGED), DJ_ERR_CUDA. */
dj_status dj_ws_relax_to_tol(dj_mesh* mesh, dj_ws* ws, const double* targets, int arm, double tol,
                             long long max_steps, dj_ws_result* res, void* stream);

/* Serialised model (bases, polynomial part, MLP weights, options, info):
 * dj_ws_save writes at most `capacity` bytes to buf and the size to *bytes
 * (buf NULL: the size only; a smaller capacity: DJ_ERR_INVALID_ARG);
 * dj_ws_load builds a dj_ws from such a buffer (host memory) on the current
 * device.  Errors: DJ_ERR_INVALID_ARG (size, format), DJ_ERR_OOM, DJ_ERR_CUDA. */
dj_status dj_ws_save(const dj_ws* ws, void* buf, size_t capacity, size_t* bytes);
dj_status dj_ws_load(const void* buf, size_t bytes, dj_ws** out);

dj_status dj_ws_get_info(const dj_ws* ws, dj_ws_info* info);
const char* dj_ws_last_error(const dj_ws* ws);
void dj_ws_destroy(dj_ws* ws);

#ifdef __cplusplus
}
#endif
#endif /* DJ_TLED_H */
