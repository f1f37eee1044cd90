/*
 * vfe.h -- C ABI of the GB300 voxel finite-element elastic wave solver.
 *
 * The library advances the explicit structured-mesh elastic wave equation of
 * Ichimura et al., arXiv 2404.13683: the element-by-element internal force
 * f = K u over a voxel mesh (Section 2, Eq. DGE:ORG) followed by the
 * central-difference update with a diagonal mass matrix (Eq. eqtimehistory,
 * and its rearranged update form in Section 3).
 *
 * Two element kinds are supported: the conventional lumped-mass trilinear
 * voxel element VFEM and the orthogonal voxel element OVFEM (Eqs. OVFEMstiff,
 * OVFEMmass, OVFEMbasis1, OVFEMbasis2).  Two arithmetic paths are supported:
 *   VFE_PATH_FP64  plain FP64 on CUDA cores (both element kinds);
 *   VFE_PATH_TC    OVFEM only: K u formed as exact integer-split tensor-core
 *                  products in the spirit of Eq. GE:TC and Eqs.
 *                  int8comp1-int8comp2 (see vfe_options.stages).
 *
 * Conventions shared by every call:
 *   - grid: nx*ny*nz cubic elements of side h; nodes (i,j,k), 0<=i<=nx etc.;
 *     node id = i + (nx+1)*(j + (ny+1)*k); element id = i + nx*(j + ny*k);
 *     z is up and k = 0 is the bottom plane;
 *   - nodal vectors are FP64 arrays [n_nodes][3] (component fastest);
 *   - material_table rows are {Vp, Vs, rho} (m/s, m/s, kg/m^3); an element id
 *     of -1 marks a void cell (no stiffness, no mass);
 *   - every call returns VFE_OK (0) or a negative VFE_E* code; the message of
 *     the last failure on the calling thread is vfe_last_error();
 *   - the library copies every input array; the caller owns every output
 *     buffer; pointers are host pointers unless stated otherwise;
 *   - calls on one mesh must not run concurrently from several threads.
 */
#ifndef VFE_H
#define VFE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VFE_OK 0
#define VFE_EINVAL (-1)   /* bad argument (message says which) */
#define VFE_ENOMEM (-2)   /* host or device allocation failed */
#define VFE_ECUDA (-3)    /* a CUDA call failed (message has the CUDA error) */
#define VFE_ETIMEOUT (-4) /* a device-side bounded wait gave up; results invalid */
#define VFE_ESTATE (-5)   /* call not valid in the current state */

enum vfe_element_kind { VFE_OVFEM = 0, VFE_VFEM = 1 };
enum vfe_path { VFE_PATH_FP64 = 0, VFE_PATH_TC = 1 };

typedef struct vfe_options {
  int element_kind; /* VFE_OVFEM (default) or VFE_VFEM */
  int path;         /* VFE_PATH_TC (default) or VFE_PATH_FP64 */
  int stages;       /* TC path: number of 11-bit integer digit stages, 1..5
                       (default 5 = 55-bit split, >= the FP64 mantissa) */
  int fix_bottom;   /* 1 (default): every node of plane k = 0 is fixed;
                       2: the four corner nodes of plane k = 0 (Section 3);
                       0: no node is fixed (massless nodes always are) */
  double dt;        /* time step; <= 0 selects cfl_fraction * critical step;
                       above the critical step 2/sqrt(lambda_max(M_e^-1 K_e)) of
                       the materials present: VFE_EINVAL (the scheme diverges) */
  double cfl_fraction; /* default 0.5 */
  int device;       /* CUDA device ordinal (default 0) */
  void *stream;     /* cudaStream_t to run on; NULL = a stream the mesh owns */
  int stencil;      /* TC path: 1 (default) forms K u on node planes whose
                       surrounding elements share one material as one node
                       stencil per material part (the element products of
                       Eq. GE:TC summed at the node, same integer split); 0
                       uses the element-by-element kernel everywhere; 2 gives
                       the stencil every node plane but those holding the
                       source or a receiver, each node taking the most
                       frequent material among its eight elements, and a
                       correction launch after it exchanges the material of
                       the node's other elements (another material, void, or
                       outside the mesh); 1 does the same on meshes of 8 Mi
                       elements or more.  They agree to the FP64-equivalent
                       bound of the split. */
  int ctas;         /* TC path: CTAs per kernel launch, i.e. how many pieces the
                       (node column x plane range) work bricks are cut into;
                       0 (default) = one per SM, the most the kernels take */
} vfe_options;

typedef struct vfe_mesh vfe_mesh;

/* Fill *opt with the defaults listed above. */
void vfe_default_options(vfe_options *opt);

/* Create a mesh.  material_ids: nx*ny*nz int32 (element order above, -1 =
 * void); material_table: n_materials rows of {Vp, Vs, rho} with rho > 0,
 * Vs >= 0 and Vp^2 > 4/3 Vs^2.  opt may be NULL for defaults.  Moduli follow
 * Section 2: G = rho Vs^2, kappa = rho (Vp^2 - 4/3 Vs^2).  The critical step
 * is 2/sqrt(max eigenvalue of M_e^-1 K_e) over the materials present.
 * On success *out owns device memory until vfe_destroy. */
int vfe_create_mesh(int nx, int ny, int nz, double h,
                    const int32_t *material_ids, const double *material_table,
                    int n_materials, const vfe_options *opt, vfe_mesh **out);

/* Release everything the mesh owns.  NULL is accepted. */
int vfe_destroy(vfe_mesh *mesh);

/* Point force at node (i,j,k): F(t) = amp * ricker(t; f0, t0) * dir with the
 * Ricker wavelet (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), applied
 * as F^n at t = n dt (Section 3 uses an impulse force in z), evaluated on
 * the device each step.  t0 <= 0 selects t0 = 1/f0.  Forces at a fixed or
 * massless node are ignored.  dir is not normalised.  Waits for the mesh's
 * queued work.  VFE_EINVAL: node outside the grid, f0 <= 0, or a non-finite
 * f0, t0, amp or dir component. */
int vfe_set_source(vfe_mesh *mesh, int i, int j, int k, const double dir[3],
                   double f0_hz, double t0_s, double amp);

/* Receivers at nodes ijk[n][3] (int32 i, j, k per receiver; n = 0 removes
 * them): the observation points of Section 3, whose displacement histories
 * the paper compares (Table 1 lists its source and observation points).
 * Resets the trace buffer: later vfe_step calls append u^{n+1} at
 * every receiver for every step.  Waits for the mesh's queued work.
 * VFE_EINVAL: n < 0, ijk NULL with n > 0, or a node outside the grid. */
int vfe_set_receivers(vfe_mesh *mesh, int n, const int32_t *ijk);

/* f = K u for the whole mesh (fixed DOFs included), u and f FP64 [nodes][3]
 * host arrays: the element-by-element internal force of Eq. DGE:ORG, with
 * K_e of Eq. OVFEMstiff (OVFEM) or of the trilinear element (VFEM).  On the
 * tensor-core path K_e u_e is formed as in Eq. GE:TC from the integer split
 * of Eqs. intscaling and int8comp1-int8comp2, recombined exactly (an integer
 * split of 55 bits, at least the FP64 mantissa, with the default stages).
 * Uses the mesh's path; does not touch the time-stepping state.
 * Synchronous.  VFE_EINVAL: a NULL argument or a non-finite value in u. */
int vfe_internal_force(vfe_mesh *mesh, const double *u, double *f);

/* Advance n >= 0 central-difference steps (Eq. eqtimehistory):
 * u^{n+1} = 2u^n - u^{n-1} + dt^2 M^-1 (F^n - K u^n) on free DOFs.
 * Asynchronous on the mesh's stream (launched as captured CUDA graphs of 32
 * and of 2 steps, so a long run pays the launch cost once per 32 steps);
 * device errors surface at the next synchronising call.  VFE_EINVAL: n < 0;
 * VFE_ENOMEM: growing the device trace buffer; VFE_ECUDA: a launch failed. */
int vfe_step(vfe_mesh *mesh, int n);

/* Advance n >= 0 steps like vfe_step, with the point force at the source
 * node given by the caller instead of the wavelet: step k of these n uses
 * F = force[k][0..2] (newtons, FP64 host array [n][3]) in the update of
 * Eq. eqtimehistory, as the experiment of Section 3 drives its model through
 * a prescribed force at one node.  Needs a prior vfe_set_source (its node is
 * used; its wavelet parameters are not); a force at a fixed or massless node
 * is ignored.  Later vfe_step calls use the wavelet again.  The rows are
 * copied to the device on the mesh's stream: a pageable array is read before
 * the call returns, a page-locked one must stay unchanged until the next
 * synchronising call.  Asynchronous like vfe_step.  Errors: VFE_EINVAL (NULL
 * force, n < 0, a non-finite value), VFE_ESTATE (no source set), VFE_ENOMEM
 * (growing the device copy of the rows), VFE_ECUDA. */
int vfe_step_forced(vfe_mesh *mesh, int n, const double *force);

/* Rayleigh damping C = alpha M + beta K (Section 3 computes attenuation with
 * Rayleigh damping; it gives no time discretisation, and this library uses
 * the one that keeps the step explicit with the diagonal mass):
 *   (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1} - dt^2 M^-1 (K w^n - F^n),
 *   a = alpha dt / 2,  w^n = u^n + (beta / dt) (u^n - u^{n-1}),
 * i.e. the mass term with the central velocity and the stiffness term with
 * the backward velocity.  alpha = beta = 0 (the default) is the undamped
 * step.  Needs alpha, beta >= 0, alpha dt / 2 < 1 and, for stability,
 * (dt / dt_crit)^2 (1 + 2 beta / dt) <= 1 (VFE_EINVAL otherwise).  Takes
 * effect from the next step (the current state is kept).  Not combined with
 * vfe_misfit_gradient (VFE_ESTATE).  Synchronous. */
int vfe_set_damping(vfe_mesh *mesh, double alpha, double beta);

/* The Rayleigh coefficients that give damping ratio h at the frequencies f1
 * and f2 (Hz, 0 < f1 <= f2): alpha = 2 h w1 w2 / (w1 + w2),
 * beta = 2 h / (w1 + w2), w = 2 pi f; between f1 and f2 the ratio
 * alpha / (2 w) + beta w / 2 stays below h.  Host only (no GPU needed). */
int vfe_rayleigh_coefficients(double h, double f1_hz, double f2_hz, double *alpha,
                              double *beta);

/* Block until queued work is done; reports device-side timeouts. */
int vfe_synchronize(vfe_mesh *mesh);

/* Copy the traces recorded since vfe_set_receivers: out[s][r][3] FP64 for
 * s < *n_steps_out (out may be NULL to query the count only): the time
 * histories of displacement at the observation points that Section 3
 * compares between the methods (its Err is computed from them).  Row s is
 * u^{s+1} after step s.  Synchronous. */
int vfe_get_traces(vfe_mesh *mesh, double *out, int64_t *n_steps_out);

/* Copy trace rows [first, first+count) (same layout as vfe_get_traces) after
 * the work queued so far has finished.  Lets a caller read each step's
 * receiver values as they are produced.  Synchronous. */
int vfe_get_trace_rows(vfe_mesh *mesh, int64_t first, int64_t count, double *out);

/* The same copy queued on the mesh's stream behind the steps queued so far,
 * without waiting: for streaming the receiver rows to the host while the GPU
 * keeps stepping.  out (host, [count][n_rec][3] FP64) should be page-locked,
 * so that the copy is asynchronous; it holds the rows once a synchronising
 * call (vfe_synchronize, vfe_get_traces, vfe_get_trace_rows) has returned,
 * which also reports device errors.  Rows must already be queued (first +
 * count <= steps recorded, VFE_EINVAL otherwise); VFE_ECUDA if the copy cannot
 * be queued. */
int vfe_get_trace_rows_async(vfe_mesh *mesh, int64_t first, int64_t count, double *out);

/* Time step in use, number of nodes, and steps taken since creation. */
int vfe_get_dt(vfe_mesh *mesh, double *dt);
int vfe_get_sizes(vfe_mesh *mesh, int64_t *n_nodes, int64_t *n_elements);
int vfe_get_step_count(vfe_mesh *mesh, int64_t *steps);

/* Kernel launches one step enqueues on the mesh's stream: on the TC path the
 * one-thread prologue, the element kernel (when any column-plane needs it),
 * the node-stencil kernel (when enabled) and, when some node of its runs
 * has elements of another material than its own, void or outside the mesh
 * (meshes of 8 Mi elements or more, or stencil option 2), the correction
 * of those nodes; on the FP64 path the prologue and the step kernel.  VFE_EINVAL:
 * a NULL argument. */
int vfe_get_launches_per_step(vfe_mesh *mesh, int *launches);

/* Read / replace the state (u^n, u^{n-1}) as FP64 [nodes][3] host arrays.
 * Values at fixed or massless nodes are forced to zero by vfe_set_state.
 * Both wait for the mesh's queued work.  VFE_EINVAL: a NULL argument, or
 * (vfe_set_state) a non-finite value. */
int vfe_get_state(vfe_mesh *mesh, double *u, double *u_prev);
int vfe_set_state(vfe_mesh *mesh, const double *u, const double *u_prev);

/* Thread-local message of the last failing call ("" if none). */
const char *vfe_last_error(void);

/* Exact integer partial products of the TC path for a list of elements:
 * out[q][48] int64 = (K^kappa q_e, K^G' q_e) for element ids[q], where
 * q_e are the 24 integer inputs the kernel digitised from u at the given
 * shift (q = floor(U / 2^shift) of the fixed-point state); both halves are
 * stored in local DOF order 3a+c.  Diagnostic: lets tests check the tensor
 * core arithmetic bit for bit.  TC path only; synchronous. */
int vfe_debug_tc_partials(vfe_mesh *mesh, const double *u, int n,
                          const int64_t *ids, int64_t *out, int *shift_out,
                          int *frac_bits_out);

/* Node-plane exchange for a z-slab decomposition over several GPUs (the
 * paper's closing remark that the method extends to multiple GPUs, Section
 * 4).  A mesh that is one slab of a larger model holds, besides its own node
 * planes, the plane just below and just above them; after every step the
 * caller copies its own boundary planes of u^n to the neighbouring slabs and
 * writes the planes it receives into its halo planes, so that the next step
 * forms K u (Eq. DGE:ORG) on its own planes from the full neighbourhood.
 * Both calls are queued on the mesh's stream (no wait) and move FP64 values:
 * vfe_pack_plane writes u^n of node plane k (0 <= k <= nz, local to the mesh)
 * to dev_out, a device array [(ny+1)(nx+1)][3] of vfe_plane_values doubles;
 * vfe_unpack_plane writes such an array into u^n of plane k.  On the
 * tensor-core path the value is rounded to the mesh's fixed-point unit (the
 * same rounding the update applies) and enters the bounds from which the
 * next step picks its digit quantum.  u^{n-1} is not touched.  VFE_ESTATE
 * with Rayleigh damping (its state w would need the exchange too). */
int vfe_plane_values(vfe_mesh *mesh, int64_t *n_values);
int vfe_pack_plane(vfe_mesh *mesh, int k, double *dev_out);
int vfe_unpack_plane(vfe_mesh *mesh, int k, const double *dev_in);

/* One fixed-point scale for all slabs (tensor-core path).  Each step picks
 * the power-of-two unit of the state from a bound of |u| and of the source
 * increment (the digit quantum of Eq. intscaling and the update's unit);
 * slabs that exchange planes must pick the same unit every step.  So after
 * the exchange the caller takes the maximum of the slabs' bound words (an
 * all-reduce MAX of one uint64 per slab): vfe_get_scale_bound copies the
 * word the next step reads into dev_word (device, 8 bytes), and
 * vfe_set_scale_bound writes the reduced word back (both queued on the
 * mesh's stream; no-ops on the FP64 path, which has no scale).  A slab
 * without the source learns the source from vfe_set_source_bound (the
 * wavelet of vfe_set_source and dt^2/m at the source node, which the slab
 * holding it reports through vfe_get_source_scale): it then sizes the unit
 * for the source's increment as the source's slab does, without applying
 * any force.  VFE_ESTATE if the mesh holds a source itself. */
int vfe_get_scale_bound(vfe_mesh *mesh, unsigned long long *dev_word);
int vfe_set_scale_bound(vfe_mesh *mesh, const unsigned long long *dev_word);
int vfe_get_source_scale(vfe_mesh *mesh, double *dt2_over_m);
int vfe_set_source_bound(vfe_mesh *mesh, const double dir[3], double f0_hz, double t0_s,
                         double amp, double dt2_over_m);

/* Exact integer partial sums of the node-stencil kernel: for u (FP64
 * [nodes][3], host) digitised as the kernel does (q = floor(U / 2^shift) of
 * the fixed-point state U = round(u 2^frac_bits)), out[node][9] int64 holds
 * P = S^k q, the stencil part S^G q of Q, and q' (the node's own q as its
 * kept digits give it) for every node the node-stencil kernel owns, where
 * covered[node] = 1; 0 elsewhere.  S^k and S^G are the node sums of the
 * integer matrices of Eq. GE:TC (K^kappa and the paper's Kbar^G) over the
 * node's eight elements.  Diagnostic: lets tests check the tensor-core
 * arithmetic of that kernel bit for bit.  TC path only; synchronous. */
int vfe_debug_stencil_partials(vfe_mesh *mesh, const double *u, int64_t *out,
                               int8_t *covered, int *shift_out, int *frac_bits_out);

/* Test hook for the error paths: ORs bits (1 wait timeout, 2 fixed-point
 * shift out of range, 4 tensor-memory allocation failure, 8 forced step past
 * the supplied rows) into the mesh's device status word, as the kernels do
 * when such a failure happens, so that tests can check that every call which
 * reads the word reports it, without making a GPU fault or wait.  The word
 * is sticky: the mesh keeps reporting the error until it is destroyed.
 * Waits for the mesh's queued work.  The paper has no counterpart. */
int vfe_debug_inject_status(vfe_mesh *mesh, int bits);

/* Adjoint-state gradient (the paper's internal-structure estimation use,
 * Section 1).  For a run of nsteps from rest with the mesh's source and the
 * receiver misfit J = 1/2 sum_{n<N} sum_r |u^{n+1}(r) - data[n][r]|^2
 * (data: [nsteps][n_rec][3]), writes dJ/dG_e for every element (grad_G[ne],
 * shear modulus G_e at fixed bulk modulus kappa_e; 0 for void cells) and J.
 * The discrete adjoint of Eq. eqtimehistory is the same leapfrog run backward
 * with the residual injected at the receivers; the forward states are
 * recomputed from checkpoints taken every checkpoint_every steps (memory:
 * checkpoint_every + 1 FP64 states plus two states per checkpoint), and
 * dJ/dG_e = dt^2 sum_n mu^n_e . (dK_e/dG) u^n_e.  Uses the mesh's path for
 * every step.  The mesh is left at rest (step 0, traces cleared).
 * Synchronous. */
int vfe_misfit_gradient(vfe_mesh *mesh, int nsteps, const double *data, int checkpoint_every,
                        double *grad_G, double *misfit);

/* Per-element shear moduli (the parameters of the internal-structure
 * estimation use, Section 1): element e gets shear modulus G[e] (Pa, host
 * array of nx*ny*nz; entries of void cells are ignored) at the bulk modulus
 * and density of its material, so that K_e = kappa K_e(1, 0) + G_e K_e(0, 1)
 * in the element's closed form (Eq. OVFEMstiff; the trilinear element
 * likewise).  G = NULL returns to the materials' moduli.  Takes effect from
 * the next step; the time step is kept: VFE_EINVAL if it exceeds the
 * stability limit with the largest G of some material, or for a negative or
 * non-finite G.  Meshes with per-element moduli use the element-by-element
 * kernel on every plane.  vfe_misfit_gradient then differentiates with
 * respect to these moduli.  Synchronous. */
int vfe_set_shear_moduli(vfe_mesh *mesh, const double *G);

/* Batches: many meshes advanced together (the paper's many-case use, Section 1).
 * vfe_create_batch takes n distinct meshes on the tensor-core path, on one
 * device; it keeps pointers to them (they must outlive the batch).  Meshes
 * may differ in their digit stage count.  vfe_batch_step(b, n) advances every
 * mesh n steps: per step one prologue launch, one fused element-kernel launch
 * per stage count over those meshes' non-uniform node columns (all of a
 * mesh's columns when its stencil option is off), and for each mesh with
 * the node-stencil kernel one stencil launch over its stencil runs (and
 * their correction launch) on a share of the SMs in proportion to its size, on side streams that run side
 * by side; replayed as captured CUDA graphs of 32 and of 2 steps; each mesh
 * keeps its own source, receivers, traces, state and time step.  Work queued
 * on a mesh's own stream before the call runs first; calls on a mesh after it
 * wait for the batch.  Changing a mesh's source or receivers between batch
 * steps is allowed (the batch rebuilds its tables).  vfe_batch_synchronize
 * waits and reports device-side errors of every mesh. */
typedef struct vfe_batch vfe_batch;
int vfe_create_batch(int n, vfe_mesh *const *meshes, vfe_batch **out);
int vfe_batch_step(vfe_batch *batch, int n);
int vfe_batch_synchronize(vfe_batch *batch);
int vfe_destroy_batch(vfe_batch *batch);

/* K u of the tensor-core path for callers that cannot allocate device memory:
 * u and f are FP64 [nodes][3] host arrays as in vfe_internal_force, and the
 * result agrees with it to the same FP64-level tolerance.  The paper has no
 * counterpart to this entry point.
 *
 * Who needs it: code running inside a framework that owns the whole device
 * memory pool, real-time loops where cudaMalloc's implicit synchronisation is
 * not acceptable, and deployments that budget every byte at start-up.  The
 * call performs no cudaMalloc, cudaFree or other allocating routine; all its
 * temporaries live in one statically declared device array of
 * VFE_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU loading the library holds
 * until the process exits.  A mesh whose temporaries exceed the array (about
 * 48 bytes per padded node, so up to roughly 1.3 M nodes) is rejected with
 * VFE_EINVAL and a message giving both sizes.
 *
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress) and caches it, so make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents (each call clears what must start at zero); calls whose GPU
 * work overlaps -- from several threads or streams -- race on it.  TC path
 * only (VFE_ESTATE otherwise).  Synchronous on the mesh's stream. */
#define VFE_NOALLOC_SCRATCH_BYTES (64u << 20)
int vfe_internal_force_noalloc(vfe_mesh *mesh, const double *u, double *f);

#ifdef __cplusplus
}
#endif
#endif
