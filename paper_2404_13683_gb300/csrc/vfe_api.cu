// vfe_api.cu -- C ABI and host logic of the GB300 voxel FE wave solver.
//
// Host responsibilities: argument validation, element matrices (closed form
// of Section 2's element stiffness), node masses, the CFL step, the
// fixed-point scales of the tensor-core path, TMA tensor maps, work
// decomposition, receivers, the Ricker source parameters, and stepping through
// captured CUDA graphs.  Every step of the hot path runs in the kernels of
// vfe_tc.cu / vfe_fp64.cu; there is no CPU fallback.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vfe_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(VFE_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));              \
  } while (0)

// ---- element matrices -------------------------------------------------------
// Both voxel elements have the closed form
//   S_kl(a,b) = 1/16 s^a_k s^b_l prod_{m not in {k,l}} (1 + alpha s^a_m s^b_m)
//   K_(a,i),(b,j) = ds [lambda S_ij + G S_ji + G delta_ij sum_k S_kk]
// with alpha = 3/4 for OVFEM (Heaviside phi, the seven psi stress bases) and
// alpha = 1/3 for VFEM (trilinear phi, exact 2x2x2 Gauss).
int sgn(int a, int k) { return ((a >> k) & 1) ? 1 : -1; }

void element_matrix(int kind, double ds, double lambda, double G, double *K) {
  const double alpha = kind == VFE_OVFEM ? 0.75 : 1.0 / 3.0;
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      double S[3][3];
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          double v = sgn(a, k) * sgn(b, l) / 16.0;
          for (int m = 0; m < 3; ++m)
            if (m != k && m != l) v *= 1.0 + alpha * sgn(a, m) * sgn(b, m);
          S[k][l] = v;
        }
      const double tr = S[0][0] + S[1][1] + S[2][2];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          K[(3 * a + i) * 24 + 3 * b + j] =
              ds * (lambda * S[i][j] + G * S[j][i] + (i == j ? G * tr : 0.0));
    }
}

// Largest eigenvalue of a symmetric PSD 24x24 matrix: power iteration with a
// Rayleigh quotient (the element matrices are tiny, so 20000 sweeps are cheap).
double max_eigenvalue(const double *K) {
  double v[24], w[24];
  for (int i = 0; i < 24; ++i) v[i] = 1.0 + 0.01 * i * ((i % 3) - 1);
  double lam = 0.0;
  for (int it = 0; it < 20000; ++it) {
    double nrm = 0.0;
    for (int i = 0; i < 24; ++i) {
      double acc = 0.0;
      for (int j = 0; j < 24; ++j) acc += K[i * 24 + j] * v[j];
      w[i] = acc;
      nrm += acc * acc;
    }
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return 0.0;
    double num = 0.0, den = 0.0;
    for (int i = 0; i < 24; ++i) {
      num += v[i] * w[i];
      den += v[i] * v[i];
    }
    lam = num / den;
    for (int i = 0; i < 24; ++i) v[i] = w[i] / nrm;
  }
  return lam;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    // the entry point as of CUDA 12.0, where cuTensorMapEncodeTiled first appeared
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}


}  // namespace

struct vfe_mesh {
  int nx = 0, ny = 0, nz = 0;
  double h = 0.0;
  vfe_options opt;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 1;
  int64_t nn = 0, ne = 0;
  int n_mat = 0;
  std::vector<double> kappa, G, rho;
  std::vector<int32_t> mat;
  std::vector<double> mass;
  std::vector<char> fixed;
  double dt = 0.0;
  double dt_crit = 0.0;  // 2 / sqrt(max eigenvalue of M_e^-1 K_e) over the materials
  double alpha = 0.0, beta = 0.0;  // Rayleigh damping C = alpha M + beta K
  bool damped = false;
  double *d_w[2] = {nullptr, nullptr};  // FP64 path: w^n, w^{n+1} (damped only)
  int64_t *d_W[2] = {nullptr, nullptr};  // TC path: the same in the state's fixed point
  CUtensorMap tmap_w[2];                 // TMA maps over d_W (damped TC path)
  int64_t steps = 0;  // host mirror of the device step counter

  int32_t *d_mat = nullptr;
  int *d_status = nullptr;
  double *d_traces = nullptr;
  int64_t trace_cap = 0, trace_rows = 0;
  int n_rec = 0;
  std::vector<int64_t> rec_nodes;
  std::vector<int32_t> rec_ijk;

  // per-element shear moduli (vfe_set_shear_moduli)
  bool elem_g = false;
  std::vector<double> elem_G;
  int64_t *d_elemB = nullptr;             // TC: round(G_e ds/384 2^e_ref)
  double *d_elemG = nullptr, *d_kappa = nullptr, *d_Kkg = nullptr;  // FP64 path
  bool has_src = false;
  bool src_bound_only = false;  // the source lies in another slab: it only
                                // enters the choice of the fixed-point scale
  bool src_set = false;  // vfe_set_source was called
  int64_t src_node = -1;
  double src_dir[3] = {0, 0, 0}, f0 = 0, t0 = 0, amp = 0;
  int cur = 0;  // which state buffer holds u^n

  // FP64 path
  double *d_u[2] = {nullptr, nullptr};
  double *d_dt2m = nullptr;
  double *d_K = nullptr;
  int64_t *d_recnodes = nullptr;
  void *d_f64params = nullptr;
  int64_t *d_f64persist = nullptr;

  // TC path
  int nxp = 0, nyp = 0;
  int64_t plane = 0, comp = 0;
  int64_t *d_U[2] = {nullptr, nullptr};
  int64_t *d_C = nullptr;
  uint16_t *d_Bop = nullptr;
  TcMaterial *d_mats = nullptr;
  TcRecv *d_recv = nullptr;
  int32_t *d_recv_off = nullptr;
  unsigned long long *d_or = nullptr;
  TcStepParams *d_tcparams = nullptr;
  int64_t *d_tcpersist = nullptr;
  CUtensorMap tmap[2];
  int tiles_x = 0, tiles_y = 0, n_ctas = 0;
  std::vector<int4> segs;         // element kernel: (tile x, tile y, z0, z1)
  std::vector<int32_t> seg_off;   // CTA -> first segment
  int4 *d_segs = nullptr;
  int32_t *d_seg_off = nullptr;
  // every column-plane on the element kernel (its exact-partials mode)
  int4 *d_all_segs = nullptr;
  int32_t *d_all_off = nullptr;
  int all_ctas = 0;
  // node-stencil kernel on the stencil runs (stencil_on): its segments, its
  // CTA ranges, its B image and its tensor maps (box 20x18x1x3)
  bool stencil_on = false;
  // the runs before their split over the CTAs (a batch splits them again):
  // element-kernel runs and stencil runs
  std::vector<int4> el_runs, st_runs;
  std::vector<int4> st_segs;
  std::vector<int32_t> st_off;
  int st_ctas = 0;
  // per-node material and corrections (meshes of ST_FIX_MIN_ELEMENTS or
  // more, or stencil option 2): every column-plane but the source and
  // receiver planes goes to the stencil kernel, with the reference material
  // of each node of its runs and the correction entries of stencil_fix
  bool fix_on = false;
  uint8_t *d_node_mat = nullptr;
  int4 *d_fix = nullptr;
  int n_fix = 0;
  int4 *d_st_segs = nullptr;
  int32_t *d_st_off = nullptr;
  uint16_t *d_Bst = nullptr;
  CUtensorMap st_tmap[2];
  int e_ref = 0, eC = 0;
  double src_scale = 0.0;  // dt^2 / m at the source node

  cudaGraphExec_t graph[2] = {nullptr, nullptr};       // two steps from state parity p
  bool graph_valid[2] = {false, false};
  cudaGraphExec_t graph_long[2] = {nullptr, nullptr};  // kLongSteps steps
  bool graph_long_valid[2] = {false, false};
  int64_t gen = 0;  // bumped whenever kernel arguments change (batches rebuild)
  double *d_inj = nullptr;  // injection array [rows][n_rec][3] (adjoint source)
  double *d_force = nullptr;  // explicit force rows of vfe_step_forced [k][3], then one
                              // int64 -1 (copied to the "first step" slot to end a series)
  int64_t force_cap = 0;      // rows d_force holds
  std::vector<double> table;  // the caller's {Vp, Vs, rho} rows
};

static void invalidate_graphs(vfe_mesh *m) {
  m->gen++;
  for (int i = 0; i < 2; ++i) {
    if (m->graph[i]) cudaGraphExecDestroy(m->graph[i]);
    m->graph[i] = nullptr;
    m->graph_valid[i] = false;
    if (m->graph_long[i]) cudaGraphExecDestroy(m->graph_long[i]);
    m->graph_long[i] = nullptr;
    m->graph_long_valid[i] = false;
  }
}

// steps per long graph: runs of many steps replay one graph of this many
// steps (the launch cost of small meshes is paid once per graph, not per step)
constexpr int kLongSteps = 32;

static int64_t node_id(const vfe_mesh *m, int i, int j, int k) {
  return (int64_t)i + (int64_t)(m->nx + 1) * ((int64_t)j + (int64_t)(m->ny + 1) * k);
}

// padded SoA index of node (i,j,k) in the TC nodal arrays (component 0)
static int64_t tc_index(const vfe_mesh *m, int64_t n) {
  const int64_t i = n % (m->nx + 1), j = (n / (m->nx + 1)) % (m->ny + 1),
                k = n / ((int64_t)(m->nx + 1) * (m->ny + 1));
  return k * m->plane + j * m->nxp + i;
}

static TcDevice tc_device(const vfe_mesh *m, int cur) {
  TcDevice d;
  memset(&d, 0, sizeof(d));
  d.nx = m->nx; d.ny = m->ny; d.nz = m->nz; d.nxp = m->nxp;
  d.n_ctas = m->n_ctas;
  d.segs = m->d_segs; d.seg_off = m->d_seg_off;
  d.n_mat = m->n_mat; d.stages = m->opt.stages; d.n_rec = m->n_rec;
  d.plane = m->plane; d.comp = m->comp;
  d.mat = m->d_mat; d.C = m->d_C;
  d.U_prev = m->d_U[1 - cur]; d.U_next = m->d_U[1 - cur];
  d.Bop = m->d_Bop; d.mats = m->d_mats; d.recv = m->d_recv; d.recv_off = m->d_recv_off;
  d.src_node = m->has_src ? tc_index(m, m->src_node) : -1;
  d.traces = m->d_traces; d.or_slots = m->d_or; d.status = m->d_status;
  d.tiles_x = m->tiles_x; d.tiles_y = m->tiles_y;
  d.elem_B = m->elem_g ? m->d_elemB : nullptr;
  d.params = m->d_tcparams;
  d.inj = m->d_inj;
  d.damped = m->damped ? 1 : 0;
  if (m->damped) {
    const double a = 0.5 * m->alpha * m->dt, g = 1.0 / (1.0 + a);
    d.U_cur = m->d_U[cur];
    d.W_next = m->d_W[1 - cur];
    d.dG = llrint(std::ldexp(g, 62));
    d.dH = llrint(std::ldexp((1.0 - a) * g, 62));
    d.dB = llrint(std::ldexp(m->beta / m->dt, 62));
  }
  return d;
}

// the same arguments for the node-stencil kernel over the stencil runs
static TcDevice tc_stencil_device(const vfe_mesh *m, int cur) {
  TcDevice d = tc_device(m, cur);
  d.segs = m->d_st_segs;
  d.seg_off = m->d_st_off;
  d.n_ctas = m->stencil_on ? m->st_ctas : 0;
  d.Bst = m->d_Bst;
  d.U_cur = m->d_U[cur];  // u^n: the corrections read it
  d.node_mat = m->d_node_mat;
  d.fix = m->d_fix;
  d.n_fix = m->stencil_on ? m->n_fix : 0;
  d.recv = nullptr;
  d.recv_off = nullptr;
  d.n_rec = 0;
  d.src_node = -1;
  return d;
}

static F64Device f64_device(const vfe_mesh *m, int cur) {
  F64Device d;
  memset(&d, 0, sizeof(d));
  d.nx = m->nx; d.ny = m->ny; d.nz = m->nz; d.n_mat = m->n_mat; d.n_rec = m->n_rec;
  d.nn = m->nn; d.mat = m->d_mat; d.K = m->d_K;
  d.u = m->d_u[cur]; d.u_prev = m->d_u[1 - cur]; d.u_next = m->d_u[1 - cur];
  d.dt2_m = m->d_dt2m; d.recv_nodes = m->d_recnodes; d.traces = m->d_traces;
  d.src_node = m->has_src ? m->src_node : -1;
  d.inj = m->d_inj;
  d.damped = m->damped ? 1 : 0;
  d.elem_G = m->elem_g ? m->d_elemG : nullptr;
  d.kappa = m->d_kappa;
  d.Kkg = m->d_Kkg;
  d.w = m->d_w[cur];
  d.w_next = m->d_w[1 - cur];
  d.da = 0.5 * m->alpha * m->dt;
  d.db = m->beta / m->dt;
  return d;
}

// one time step on the stream (prologue + kernel) starting from state cur
static int enqueue_step(vfe_mesh *m, int cur) {
  const int trace_on = m->n_rec > 0 ? 1 : 0;
  TcSource src;
  src.dt = m->dt;
  src.f0 = m->f0;
  src.t0 = m->t0;
  for (int c = 0; c < 3; ++c) src.dir[c] = m->src_dir[c];
  src.force = m->d_force;
  src.force_rows = m->force_cap;
  if (m->opt.path == VFE_PATH_TC) {
    // with damping the step's increments carry the factor 1 / (1 + alpha dt / 2)
    const double g = m->damped ? 1.0 / (1.0 + 0.5 * m->alpha * m->dt) : 1.0;
    src.amp_scale = m->amp * m->src_scale * g;
    src.force_scale = m->src_scale * g;
    CUDA_TRY(tc_launch_prologue_ex(m->stream, m->d_tcparams, m->d_tcpersist, src, m->d_or,
                                   m->tiles_x * m->tiles_y,
                                   (m->has_src || m->src_bound_only) ? 1 : 0, trace_on,
                                   m->d_status, m->d_inj, 3 * m->n_rec));
    TcDevice d = tc_device(m, cur);
    if (d.n_ctas > 0)
      CUDA_TRY(tc_launch_step(m->stream, d, m->damped ? &m->tmap_w[cur] : &m->tmap[cur],
                              TC_MODE_STEP));
    if (m->stencil_on) {
      TcDevice ds = tc_stencil_device(m, cur);
      CUDA_TRY(stencil_launch(m->stream, ds, &m->st_tmap[cur], TC_MODE_STEP));
      CUDA_TRY(stencil_fix(m->stream, ds, TC_MODE_STEP));
    }
  } else {
    src.amp_scale = m->amp;
    src.force_scale = 1.0;
    CUDA_TRY(f64_launch_prologue(m->stream, m->d_f64params, m->d_f64persist, src,
                                 m->has_src ? 1 : 0, trace_on, m->d_status));
    F64Device d = f64_device(m, cur);
    CUDA_TRY(f64_launch_step(m->stream, d, m->d_f64params, 0));
  }
  return VFE_OK;
}

// a captured graph of `len` (even) steps from state parity cur
static int capture_steps(vfe_mesh *m, int cur, int len, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
  int rc = VFE_OK;
  for (int k = 0; k < len && rc == VFE_OK; ++k) rc = enqueue_step(m, cur ^ (k & 1));
  cudaError_t e = cudaStreamEndCapture(m->stream, &g);
  if (rc != VFE_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(VFE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return fail(VFE_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return VFE_OK;
}

static int ensure_graph(vfe_mesh *m, int cur) {
  if (m->graph_valid[cur]) return VFE_OK;
  const int rc = capture_steps(m, cur, 2, &m->graph[cur]);
  if (rc == VFE_OK) m->graph_valid[cur] = true;
  return rc;
}

static int ensure_long_graph(vfe_mesh *m, int cur) {
  if (m->graph_long_valid[cur]) return VFE_OK;
  const int rc = capture_steps(m, cur, kLongSteps, &m->graph_long[cur]);
  if (rc == VFE_OK) m->graph_long_valid[cur] = true;
  return rc;
}

static int check_status(vfe_mesh *m) {
  int st = 0;
  CUDA_TRY(cudaMemcpy(&st, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & 1) return fail(VFE_ETIMEOUT, "a device-side wait timed out (status %d)", st);
  if (st & 2) return fail(VFE_ETIMEOUT, "fixed-point shift out of range (status %d)", st);
  if (st & 4) return fail(VFE_ECUDA, "tensor-memory allocation failed (status %d)", st);
  if (st & 8) return fail(VFE_ESTATE, "a forced step ran past the supplied force rows (status %d)", st);
  return VFE_OK;
}

// ---- C ABI ------------------------------------------------------------------

extern "C" {

const char *vfe_last_error(void) { return g_last_error.c_str(); }

void vfe_default_options(vfe_options *o) {
  if (!o) return;
  o->element_kind = VFE_OVFEM;
  o->path = VFE_PATH_TC;
  o->stages = TC_MAX_STAGES;
  o->fix_bottom = 1;
  o->dt = 0.0;
  o->cfl_fraction = 0.5;
  o->device = 0;
  o->stream = nullptr;
  o->stencil = 1;
  o->ctas = 0;
}

int vfe_destroy(vfe_mesh *m) {
  if (!m) return VFE_OK;
  cudaSetDevice(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  invalidate_graphs(m);
  void *ptrs[] = {m->d_mat, m->d_status, m->d_traces, m->d_u[0], m->d_u[1],
                  m->d_dt2m, m->d_K, m->d_recnodes, m->d_f64params, m->d_f64persist,
                  m->d_U[0], m->d_U[1], m->d_C, m->d_Bop, m->d_mats, m->d_recv,
                  m->d_recv_off, m->d_or, m->d_tcparams, m->d_tcpersist, m->d_segs,
                  m->d_seg_off, m->d_inj, m->d_force, m->d_w[0], m->d_w[1],
                  m->d_W[0], m->d_W[1], m->d_all_segs, m->d_all_off, m->d_st_segs,
                  m->d_st_off, m->d_Bst, m->d_elemB, m->d_elemG, m->d_kappa,
                  m->d_Kkg, m->d_fix, m->d_node_mat};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
  return VFE_OK;
}

static int build_tc(vfe_mesh *m);
static int build_f64(vfe_mesh *m);
static int rebuild_receivers(vfe_mesh *m);
static int rebuild_work(vfe_mesh *m);

int vfe_create_mesh(int nx, int ny, int nz, double h, const int32_t *material_ids,
                    const double *material_table, int n_materials, const vfe_options *opt_in,
                    vfe_mesh **out) {
  if (!out) return fail(VFE_EINVAL, "out is NULL");
  *out = nullptr;
  vfe_options opt;
  vfe_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (nx < 1 || ny < 1 || nz < 1) return fail(VFE_EINVAL, "grid must be at least 1x1x1");
  if ((int64_t)nx * ny * nz > ((int64_t)1 << 31))
    return fail(VFE_EINVAL, "grid too large (more than 2^31 elements)");
  if (!(h > 0.0) || !std::isfinite(h)) return fail(VFE_EINVAL, "h must be positive");
  if (!material_ids || !material_table) return fail(VFE_EINVAL, "NULL material array");
  if (n_materials < 1) return fail(VFE_EINVAL, "n_materials must be >= 1");
  if (opt.element_kind != VFE_OVFEM && opt.element_kind != VFE_VFEM)
    return fail(VFE_EINVAL, "unknown element kind %d", opt.element_kind);
  if (opt.path != VFE_PATH_FP64 && opt.path != VFE_PATH_TC)
    return fail(VFE_EINVAL, "unknown path %d", opt.path);
  if (opt.path == VFE_PATH_TC && opt.element_kind != VFE_OVFEM)
    return fail(VFE_EINVAL, "the tensor-core path implements the orthogonal element only");
  if (opt.path == VFE_PATH_TC && (opt.stages < 1 || opt.stages > TC_MAX_STAGES))
    return fail(VFE_EINVAL, "stages must be in [1, %d]", TC_MAX_STAGES);
  if (opt.path == VFE_PATH_TC && n_materials > TC_MAX_MAT)
    return fail(VFE_EINVAL, "at most %d materials on the tensor-core path", TC_MAX_MAT);
  if (opt.path == VFE_PATH_FP64 && n_materials > F64_MAX_MAT)
    return fail(VFE_EINVAL, "at most %d materials on the FP64 path", F64_MAX_MAT);
  if (!(opt.cfl_fraction > 0.0) || opt.cfl_fraction > 1.0)
    return fail(VFE_EINVAL, "cfl_fraction must be in (0, 1]");
  if (opt.fix_bottom < 0 || opt.fix_bottom > 2)
    return fail(VFE_EINVAL, "fix_bottom must be 0, 1 or 2");
  if (opt.stencil < 0 || opt.stencil > 2) return fail(VFE_EINVAL, "stencil must be 0, 1 or 2");
  if (opt.ctas < 0) return fail(VFE_EINVAL, "ctas must be >= 0");

  vfe_mesh *m = new vfe_mesh();
  m->nx = nx; m->ny = ny; m->nz = nz; m->h = h; m->opt = opt; m->device = opt.device;
  m->nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  m->ne = (int64_t)nx * ny * nz;
  m->n_mat = n_materials;
  m->kappa.resize(n_materials); m->G.resize(n_materials); m->rho.resize(n_materials);
  for (int i = 0; i < n_materials; ++i) {
    const double vp = material_table[3 * i], vs = material_table[3 * i + 1],
                 rho = material_table[3 * i + 2];
    if (!(rho > 0.0) || !(vs >= 0.0) || !(vp * vp > 4.0 / 3.0 * vs * vs) || !std::isfinite(vp) ||
        !std::isfinite(rho)) {
      delete m;
      return fail(VFE_EINVAL, "material %d: need rho > 0, Vs >= 0, Vp^2 > 4/3 Vs^2", i);
    }
    m->G[i] = rho * vs * vs;
    m->kappa[i] = rho * (vp * vp - 4.0 / 3.0 * vs * vs);
    m->rho[i] = rho;
  }
  m->mat.assign(material_ids, material_ids + m->ne);
  m->table.assign(material_table, material_table + 3 * (size_t)n_materials);
  std::vector<char> used(n_materials, 0);
  for (int64_t e = 0; e < m->ne; ++e) {
    const int32_t v = m->mat[e];
    if (v < -1 || v >= n_materials) {
      delete m;
      return fail(VFE_EINVAL, "material id %d at element %lld out of range", v, (long long)e);
    }
    if (v >= 0) used[v] = 1;
  }
  // node masses rho ds^3 / 8 per element corner (exact for OVFEM, lumped VFEM)
  m->mass.assign(m->nn, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int32_t v = m->mat[i + (int64_t)nx * (j + (int64_t)ny * k)];
        if (v < 0) continue;
        const double me = m->rho[v] * h * h * h / 8.0;
        for (int a = 0; a < 8; ++a)
          m->mass[node_id(m, i + (a & 1), j + ((a >> 1) & 1), k + (a >> 2))] += me;
      }
  m->fixed.assign(m->nn, 0);
  for (int64_t n = 0; n < m->nn; ++n) {
    const int64_t i = n % (nx + 1), j = (n / (nx + 1)) % (ny + 1);
    const int64_t k = n / ((int64_t)(nx + 1) * (ny + 1));
    const bool corner = (i == 0 || i == nx) && (j == 0 || j == ny);
    m->fixed[n] = (char)((k == 0 && (opt.fix_bottom == 1 || (opt.fix_bottom == 2 && corner))) ||
                         m->mass[n] == 0.0);
  }
  // critical step over the materials present
  double dtc = -1.0;
  for (int i = 0; i < n_materials; ++i) {
    if (!used[i]) continue;
    double K[576];
    element_matrix(opt.element_kind, h, m->kappa[i] - 2.0 * m->G[i] / 3.0, m->G[i], K);
    const double lmax = max_eigenvalue(K) / (m->rho[i] * h * h * h / 8.0);
    const double c = 2.0 / std::sqrt(lmax);
    if (dtc < 0.0 || c < dtc) dtc = c;
  }
  if (dtc <= 0.0) {
    delete m;
    return fail(VFE_EINVAL, "the mesh has no solid element");
  }
  if (opt.dt > dtc) {  // the central-difference scheme would diverge
    delete m;
    return fail(VFE_EINVAL, "dt %g exceeds the stability limit %g of the materials present",
                opt.dt, dtc);
  }
  m->dt = opt.dt > 0.0 ? opt.dt : opt.cfl_fraction * dtc;
  m->dt_crit = dtc;

  cudaError_t e = cudaSetDevice(m->device);
  if (e != cudaSuccess) {
    delete m;
    return fail(VFE_ECUDA, "cudaSetDevice(%d): %s", opt.device, cudaGetErrorString(e));
  }
  int rc = VFE_OK;
  do {
    if (opt.stream) {
      m->stream = reinterpret_cast<cudaStream_t>(opt.stream);
    } else {
      e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) { rc = fail(VFE_ECUDA, "stream: %s", cudaGetErrorString(e)); break; }
      m->own_stream = true;
    }
    cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device);
    if ((e = cudaMalloc(&m->d_mat, sizeof(int32_t) * m->ne)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_status, sizeof(int))) != cudaSuccess) {
      rc = fail(VFE_ENOMEM, "device allocation: %s", cudaGetErrorString(e));
      break;
    }
    if ((e = cudaMemcpy(m->d_mat, m->mat.data(), sizeof(int32_t) * m->ne,
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(m->d_status, 0, sizeof(int))) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "device upload: %s", cudaGetErrorString(e));
      break;
    }
    rc = opt.path == VFE_PATH_TC ? build_tc(m) : build_f64(m);
    if (rc == VFE_OK) rc = rebuild_receivers(m);
  } while (0);
  if (rc != VFE_OK) {
    std::string msg = g_last_error;
    vfe_destroy(m);
    g_last_error = msg;
    return rc;
  }
  *out = m;
  return VFE_OK;
}

}  // extern "C"

// ---- path-specific construction ---------------------------------------------

static int build_f64(vfe_mesh *m) {
  CUDA_TRY(f64_prepare());
  std::vector<double> K((size_t)m->n_mat * 576);
  for (int i = 0; i < m->n_mat; ++i)
    element_matrix(m->opt.element_kind, m->h, m->kappa[i] - 2.0 * m->G[i] / 3.0, m->G[i],
                   &K[(size_t)i * 576]);
  std::vector<double> dt2m(m->nn, 0.0);
  for (int64_t n = 0; n < m->nn; ++n)
    if (!m->fixed[n]) dt2m[n] = m->dt * m->dt / m->mass[n];
  CUDA_TRY(cudaMalloc(&m->d_K, sizeof(double) * K.size()));
  CUDA_TRY(cudaMalloc(&m->d_dt2m, sizeof(double) * m->nn));
  CUDA_TRY(cudaMalloc(&m->d_u[0], sizeof(double) * 3 * m->nn));
  CUDA_TRY(cudaMalloc(&m->d_u[1], sizeof(double) * 3 * m->nn));
  CUDA_TRY(cudaMalloc(&m->d_f64params, f64_params_bytes()));
  CUDA_TRY(cudaMalloc(&m->d_f64persist, sizeof(int64_t) * 6));
  CUDA_TRY(cudaMemcpy(m->d_K, K.data(), sizeof(double) * K.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->d_dt2m, dt2m.data(), sizeof(double) * m->nn, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(m->d_u[0], 0, sizeof(double) * 3 * m->nn));
  CUDA_TRY(cudaMemset(m->d_u[1], 0, sizeof(double) * 3 * m->nn));
  const int64_t f64persist[6] = {0, 0, -1, 0, -1, 0};
  CUDA_TRY(cudaMemcpy(m->d_f64persist, f64persist, sizeof(f64persist), cudaMemcpyHostToDevice));
  return VFE_OK;
}

// per-node update multiplier round(g dt^2/m 2^eC) in the padded SoA layout,
// g = 1 / (1 + alpha dt / 2) with damping (1 without); 0 at fixed nodes
static std::vector<int64_t> tc_update_multipliers(const vfe_mesh *m) {
  const double g = m->damped ? 1.0 / (1.0 + 0.5 * m->alpha * m->dt) : 1.0;
  std::vector<int64_t> C(m->plane * (m->nz + 1), 0);
  for (int64_t n = 0; n < m->nn; ++n)
    if (!m->fixed[n]) C[tc_index(m, n)] = llrint(std::ldexp(g * m->dt * m->dt / m->mass[n], m->eC));
  return C;
}

// TMA map over a padded SoA int64 nodal array: (x, y, z, component), box
// 18x17x1x3 (element kernel) or 20x18x1x3 (node-stencil kernel)
static int encode_state_tmap(const vfe_mesh *m, EncodeTiledFn enc, void *base, CUtensorMap *map,
                             bool stencil_box = false) {
  cuuint64_t dims[4] = {(cuuint64_t)m->nxp, (cuuint64_t)m->nyp, (cuuint64_t)(m->nz + 1), 3};
  cuuint64_t strides[3] = {(cuuint64_t)m->nxp * 8, (cuuint64_t)m->plane * 8,
                           (cuuint64_t)m->comp * 8};
  cuuint32_t box[4] = {stencil_box ? (cuuint32_t)ST_BOXX : (cuuint32_t)TC_BOXX,
                       stencil_box ? (cuuint32_t)ST_BOXY : (cuuint32_t)TC_NODES, 1, 3};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(VFE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return VFE_OK;
}

// Runs (column x, column y, z0, z1) in order cut into at most `sms` CTA
// ranges of equal cost, a segment costing its planes plus `seg_cost` (the
// fixed work of starting one: its first planes' copies and digits); a run is
// cut where a range is full, and every piece is a segment.
static void split_runs(const std::vector<int4> &runs, const std::vector<int32_t> *run_mat,
                       int sms, double seg_cost, std::vector<int4> &segs,
                       std::vector<int32_t> *seg_mat, std::vector<int32_t> &off,
                       int min_piece = 1) {
  double total = 0.0;
  int64_t planes = 0;
  for (const int4 &r : runs) {
    total += (r.w - r.z) + seg_cost;
    planes += r.w - r.z;
  }
  // at least twice a segment's cost per range, so that a range's target
  // exceeds what its first segment may take beyond it
  const int64_t G = planes > 0 ? std::min<int64_t>(
                                     std::min<int64_t>(sms, planes),
                                     std::max<int64_t>(1, (int64_t)(total / (2.0 * (seg_cost + 1.0)))))
                               : 0;
  // a range boundary usually cuts a run, which adds a segment
  if (G > 1) total += (double)(G - 1) * seg_cost;
  segs.clear();
  if (seg_mat) seg_mat->clear();
  off.assign(G + 1, 0);
  int64_t b = 0;      // CTA being filled
  double have = 0.0;  // cost given to CTAs 0..b
  for (size_t ri = 0; ri < runs.size(); ++ri) {
    const int4 r = runs[ri];
    int64_t z = r.z;
    while (z < r.w) {
      int64_t take = r.w - z;
      if (b + 1 < G) {
        const double room = total * (double)(b + 1) / (double)G - have - seg_cost;
        if (room < 1.0 && (int64_t)segs.size() > off[b]) {  // CTA b is full
          ++b;
          off[b] = (int32_t)segs.size();
          continue;
        }
        take = std::max<int64_t>(1, std::min<int64_t>(take, (int64_t)std::llround(room)));
        // no piece, and no remainder, below min_piece planes (the runs
        // themselves are at least that long)
        const int64_t left = r.w - z;
        take = std::min<int64_t>(std::max<int64_t>(take, min_piece), left);
        if (left - take > 0 && left - take < min_piece)
          take = left - min_piece >= min_piece ? left - min_piece : left;
      }
      segs.push_back(make_int4(r.x, r.y, (int)z, (int)(z + take)));
      if (seg_mat) seg_mat->push_back((*run_mat)[ri]);
      have += (double)take + seg_cost;
      z += take;
    }
  }
  for (int64_t k = b + 1; k <= G; ++k) off[k] = (int32_t)segs.size();
}

template <typename T>
static int upload_vec(T **dptr, const std::vector<T> &v) {
  if (*dptr) cudaFree(*dptr);
  *dptr = nullptr;
  CUDA_TRY(cudaMalloc(dptr, sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (!v.empty())
    CUDA_TRY(cudaMemcpy(*dptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return VFE_OK;
}

// Work decomposition of the TC path.  A column-plane (15x15 node column, one
// node plane) is void when every element around the column's nodes on both
// sides of the plane is void or outside the mesh (massless nodes stay at
// rest: no work).  With per-node corrections (fix_on) every other
// column-plane goes to the node-stencil kernel, but for the planes holding
// the source or a receiver (element kernel); without them only the uniform
// ones do (every element around the column's nodes of material m, the column
// inside the mesh, not the end planes) and mixed planes go to the element
// kernel.  A stencil run of one plane goes to the element kernel.  With the
// node-stencil kernel off (option, or Rayleigh damping) every column-plane
// goes to the element kernel, as does the exact-partials list.
static int build_segments(vfe_mesh *m) {
  const int nx = m->nx, ny = m->ny, nz = m->nz, TX = m->tiles_x, TY = m->tiles_y;
  const int planes = nz + 1;
  m->stencil_on = m->opt.path == VFE_PATH_TC && m->opt.stencil != 0 && !m->damped && !m->elem_g;
  m->fix_on = m->stencil_on &&
               (m->opt.stencil == 2 || (int64_t)nx * ny * nz >= ST_FIX_MIN_ELEMENTS);
  std::vector<int4> all_runs, el_runs, st_runs;
  // the stencil runs' nodes: reference material, correction entries
  std::vector<uint8_t> node_mat(m->stencil_on ? (size_t)m->comp : 0, (uint8_t)ST_NO_MAT);
  std::vector<int4> fix;
  auto elem_mat = [&](int ex, int ey, int ez) -> int {  // material; -1 void or outside
    if (ex < 0 || ey < 0 || ez < 0 || ex >= nx || ey >= ny || ez >= nz) return -1;
    const int v = m->mat[(size_t)ex + (size_t)nx * (ey + (size_t)ny * ez)];
    return v < 0 ? -1 : v;
  };
  std::vector<char> forced((size_t)TX * TY * planes, 0);
  auto force = [&](int64_t n) {
    const int i = (int)(n % (nx + 1)), j = (int)((n / (nx + 1)) % (ny + 1));
    const int k = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
    forced[((size_t)(j / TC_OWN) * TX + i / TC_OWN) * planes + k] = 1;
  };
  if (m->has_src) force(m->src_node);
  for (int r = 0; r < m->n_rec; ++r) force(m->rec_nodes[r]);
  std::vector<int> layer(nz);
  for (int ty = 0; ty < TY; ++ty)
    for (int tx = 0; tx < TX; ++tx) {
      all_runs.push_back(make_int4(tx, ty, 0, planes));
      if (!m->stencil_on) continue;
      // elements around the owned nodes: x in [15 tx - 1, 15 tx + 15), y likewise
      const int ex0 = TC_OWN * tx - 1, ex1 = TC_OWN * tx + TC_OWN;
      const int ey0 = TC_OWN * ty - 1, ey1 = TC_OWN * ty + TC_OWN;
      const int cx0 = std::max(ex0, 0), cx1 = std::min(ex1, nx);
      const int cy0 = std::max(ey0, 0), cy1 = std::min(ey1, ny);
      for (int ez = 0; ez < nz; ++ez) {  // per element layer: material, -1 void, -2 mixed
        int v = m->mat[(size_t)cx0 + (size_t)nx * (cy0 + (size_t)ny * ez)];
        for (int ey = cy0; ey < cy1 && v != -2; ++ey) {
          const int32_t *row = &m->mat[(size_t)nx * (ey + (size_t)ny * ez)];
          for (int ex = cx0; ex < cx1; ++ex)
            if (row[ex] != v) { v = -2; break; }
        }
        // without corrections a column at the x or y faces is not uniform
        if (!m->fix_on && !(ex0 >= 0 && ex1 <= nx && ey0 >= 0 && ey1 <= ny) && v >= 0) v = -2;
        layer[ez] = v;
      }
      int run_cls = -3, run_z0 = 0;
      // a stencil run of one plane goes to the element kernel (the stencil
      // kernel's segments own two planes or more); element runs that touch
      // are merged
      auto flush = [&](int z1) {
        if (run_cls >= 0 && z1 - run_z0 >= 2) {
          st_runs.push_back(make_int4(tx, ty, run_z0, z1));
        } else if (run_cls != -1 && run_cls != -3) {
          if (!el_runs.empty() && el_runs.back().x == tx && el_runs.back().y == ty &&
              el_runs.back().w == run_z0)
            el_runs.back().w = z1;
          else
            el_runs.push_back(make_int4(tx, ty, run_z0, z1));
        }
      };
      const size_t st_first = st_runs.size();
      for (int L = 0; L < planes; ++L) {
        const int a = L > 0 ? layer[L - 1] : -1, b = L < nz ? layer[L] : -1;
        int cls;
        if (m->fix_on) {
          cls = a == -1 && b == -1 ? -1 : 0;  // 0: stencil, per-node material
        } else {
          cls = a == b ? a : -2;
          if (cls >= 0 && (L == 0 || L == nz)) cls = -2;
        }
        if (forced[((size_t)ty * TX + tx) * planes + L]) cls = -2;
        if (cls != run_cls) {
          flush(L);
          run_cls = cls;
          run_z0 = L;
        }
      }
      flush(planes);
      // the nodes of this column's stencil runs: the reference material is
      // the most frequent material among the node's eight elements (the
      // first in octant order on a tie); each other value among them (a
      // material, or absent: void or outside) is one correction entry
      for (size_t q = st_first; q < st_runs.size(); ++q) {
        const int4 r = st_runs[q];
        const int i0 = TC_OWN * tx, i1 = std::min(TC_OWN * tx + TC_OWN - 1, nx);
        const int j0 = TC_OWN * ty, j1 = std::min(TC_OWN * ty + TC_OWN - 1, ny);
        for (int k = r.z; k < r.w; ++k) {
          // both element layers uniform: the column's inner nodes need nothing
          const bool flat = k >= 1 && k < nz && layer[k - 1] >= 0 && layer[k - 1] == layer[k];
          for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
              const size_t n = (size_t)k * m->plane + (size_t)j * m->nxp + i;
              if (flat && i > 0 && i < nx && j > 0 && j < ny) {
                node_mat[n] = (uint8_t)layer[k];
                continue;
              }
              int v[8];
              for (int o = 0; o < 8; ++o)
                v[o] = elem_mat(i - (o & 1), j - ((o >> 1) & 1), k - (o >> 2));
              int ref = -1, best = 0;
              for (int o = 0; o < 8; ++o) {
                if (v[o] < 0) continue;
                int c = 0;
                for (int p = 0; p < 8; ++p) c += v[p] == v[o];
                if (c > best) {
                  best = c;
                  ref = v[o];
                }
              }
              if (ref < 0) continue;  // no solid element: zero material, no entry
              node_mat[n] = (uint8_t)ref;
              int done = 0, cont = 0;
              for (int o = 0; o < 8; ++o) {
                if ((done >> o) & 1) continue;
                int mask = 0;
                for (int p = 0; p < 8; ++p) mask |= (v[p] == v[o]) << p;
                done |= mask;
                if (v[o] == ref) continue;
                const int f = v[o] < 0 ? ST_NO_MAT : v[o];
                fix.push_back(make_int4(i, j, k, mask | (f << 8) | (ref << 16) | cont));
                cont = ST_FIX_CONT;
              }
            }
        }
      }
    }
  // CTAs per launch: one per SM unless the options ask for fewer
  const int ctas = m->opt.ctas > 0 ? std::min(m->opt.ctas, m->sms) : m->sms;
  std::vector<int32_t> all_off;
  std::vector<int4> all_segs;
  split_runs(all_runs, nullptr, ctas, 0.0, all_segs, nullptr, all_off);
  m->all_ctas = (int)all_off.size() - 1;
  int rc;
  if ((rc = upload_vec(&m->d_all_segs, all_segs)) != VFE_OK) return rc;
  if ((rc = upload_vec(&m->d_all_off, all_off)) != VFE_OK) return rc;
  if (m->stencil_on) {
    split_runs(el_runs, nullptr, ctas, 2.0, m->segs, nullptr, m->seg_off);
    split_runs(st_runs, nullptr, ctas, 0.0, m->st_segs, nullptr, m->st_off, 2);
    m->el_runs = el_runs;
    m->st_runs = st_runs;
    if (fix.size() > (size_t)INT32_MAX) return fail(VFE_EINVAL, "too many correction entries");
    for (const int4 &e : fix)
      if (e.x < 0 || e.x > nx || e.y < 0 || e.y > ny || e.z < 0 || e.z > nz ||
          ((e.w >> 8) & 255) > ST_NO_MAT || ((e.w >> 16) & 255) >= m->n_mat)
        return fail(VFE_EINVAL, "internal: correction entry out of range");
    m->n_fix = (int)fix.size();
    if ((rc = upload_vec(&m->d_fix, fix)) != VFE_OK) return rc;
    if ((rc = upload_vec(&m->d_node_mat, node_mat)) != VFE_OK) return rc;
  } else {
    m->segs = all_segs;
    m->seg_off = all_off;
    m->el_runs.clear();
    m->st_runs.clear();
    m->st_segs.clear();
    m->st_off.assign(1, 0);
    m->n_fix = 0;
  }
  m->n_ctas = (int)m->seg_off.size() - 1;
  m->st_ctas = (int)m->st_off.size() - 1;
  // the kernels index global memory from these tables: check them here
  auto bad_segs = [&](const std::vector<int4> &segs, const std::vector<int32_t> &off,
                      int min_planes) {
    if (off.empty() || off.front() != 0 || off.back() != (int32_t)segs.size()) return true;
    for (size_t b = 1; b < off.size(); ++b)
      if (off[b] < off[b - 1]) return true;
    for (const int4 &q : segs)
      if (q.x < 0 || q.x >= TX || q.y < 0 || q.y >= TY || q.z < 0 || q.w > planes ||
          q.w - q.z < min_planes)
        return true;
    return false;
  };
  if (bad_segs(m->segs, m->seg_off, 1) || (m->stencil_on && bad_segs(m->st_segs, m->st_off, 2)))
    return fail(VFE_EINVAL, "internal: inconsistent segment tables");
  if ((rc = upload_vec(&m->d_segs, m->segs)) != VFE_OK) return rc;
  if ((rc = upload_vec(&m->d_seg_off, m->seg_off)) != VFE_OK) return rc;
  if ((rc = upload_vec(&m->d_st_segs, m->st_segs)) != VFE_OK) return rc;
  if ((rc = upload_vec(&m->d_st_off, m->st_off)) != VFE_OK) return rc;
  invalidate_graphs(m);
  return VFE_OK;
}

static int build_tc(vfe_mesh *m) {
  const int nx = m->nx, ny = m->ny, nz = m->nz;
  CUDA_TRY(tc_prepare());
  // integer matrices K^kappa = 256/ds K_e(kappa=1,G=0), K^G' = 384/ds K_e(kappa=0,G=1)
  double Kk[576], Kg[576];
  element_matrix(VFE_OVFEM, 1.0, 1.0, 0.0, Kk);
  element_matrix(VFE_OVFEM, 1.0, -2.0 / 3.0, 1.0, Kg);
  int64_t Ik[576], Ig[576];
  int64_t l1max = 0;
  for (int r = 0; r < 24; ++r) {
    int64_t l1 = 0;
    for (int c = 0; c < 24; ++c) {
      Ik[r * 24 + c] = llround(256.0 * Kk[r * 24 + c]);
      Ig[r * 24 + c] = llround(384.0 * Kg[r * 24 + c]);
      if (std::fabs(256.0 * Kk[r * 24 + c] - Ik[r * 24 + c]) > 1e-9 ||
          std::fabs(384.0 * Kg[r * 24 + c] - Ig[r * 24 + c]) > 1e-9)
        return fail(VFE_EINVAL, "internal: integer element matrix is not integral");
      l1 += std::llabs(Ik[r * 24 + c]) + std::llabs(Ig[r * 24 + c]);
    }
    l1max = std::max(l1max, l1);
  }
  // node sums of up to 8 elements of (|P| A + |Q| B)/2^64 < 8 * l1 * 2^52 * 2^60 / 2^64
  if (l1max >= 2048) return fail(VFE_EINVAL, "internal: element row norm too large");
  // B operand image: core matrices (kg, ng) of 8 N-rows x 8 K-values (fp16)
  std::vector<uint16_t> bop(TC_N * 32);
  for (int kg = 0; kg < 4; ++kg)
    for (int ng = 0; ng < 6; ++ng)
      for (int r = 0; r < 8; ++r)
        for (int l = 0; l < 8; ++l) {
          const int n = 8 * ng + r;
          const int go = n / 12, rem = n % 12, dxo = rem / 6, part = (rem % 6) / 3, co = rem % 3;
          const int ao = dxo + 2 * (go & 1) + 4 * (go >> 1);
          float v;
          if (l >= 6) {
            v = TC_MAGIC_B;
          } else {
            const int dx = l / 3, c = l % 3, dy = kg & 1, dz = kg >> 1;
            const int col = 3 * (dx + 2 * dy + 4 * dz) + c, row = 3 * ao + co;
            v = (float)(part == 0 ? Ik[row * 24 + col] : Ig[row * 24 + col]);
          }
          bop[((kg * 6 + ng) * 8 + r) * 8 + l] = __half_as_ushort(__float2half(v));
        }
  // per-material multipliers in one mesh-wide unit: A = kappa ds/256 2^e_ref,
  // B = G ds/384 2^e_ref, the largest in [2^60, 2^61).  With |q| < 2^51 an
  // element term (|P| A + |Q| B)/2^63 stays below 1258 2^49 and a node sum
  // of eight below 2^63.
  std::vector<TcMaterial> mats(m->n_mat);
  double mxall = 0.0;
  for (int i = 0; i < m->n_mat; ++i)
    mxall = std::max(mxall, std::max(m->kappa[i] * m->h / 256.0, m->G[i] * m->h / 384.0));
  const int e_ref = 60 - std::ilogb(mxall);
  for (int i = 0; i < m->n_mat; ++i) {
    mats[i].A = llrint(std::ldexp(m->kappa[i] * m->h / 256.0, e_ref));
    mats[i].B = llrint(std::ldexp(m->G[i] * m->h / 384.0, e_ref));
    mats[i].shift = 0;
    mats[i].pad = 0;
  }
  m->e_ref = e_ref;
  // per-node multiplier C = round(dt^2/m 2^eC), max in [2^61, 2^62)
  double cmax = 0.0;
  for (int64_t n = 0; n < m->nn; ++n)
    if (!m->fixed[n]) cmax = std::max(cmax, m->dt * m->dt / m->mass[n]);
  m->eC = 61 - std::ilogb(cmax);
  // padded nodal layout (x pitch >= TMA box, y rows >= box)
  m->nxp = ((std::max(nx + 1, std::max(TC_BOXX, ST_BOXX)) + 3) / 4) * 4;
  m->nyp = std::max(ny + 1, std::max(TC_NODES, ST_BOXY));
  m->plane = (int64_t)m->nxp * m->nyp;
  m->comp = m->plane * (nz + 1);
  std::vector<int64_t> C = tc_update_multipliers(m);
  m->tiles_x = (nx + 1 + TC_OWN - 1) / TC_OWN;
  m->tiles_y = (ny + 1 + TC_OWN - 1) / TC_OWN;
  // node-stencil B images (vfe_stencil.cu): per (variant v, dy) 16 K rows
  // (x-shift d of the pair's first node - 1, component; rows 12..15 zero) x
  // 80 N columns: five 16-column blocks, the contributions of an input plane
  // p to the outputs p + o, o = -1, 0, 1, -1, 0 (column 8 node of the pair +
  // 2 component + part; 6, 7, 14, 15 zero), K-major core matrices (N groups
  // at 128 B, K groups at 1280 B).  Variant 1 zeroes the o = -1 blocks, variant 2 the
  // o = -1 and o = 0 blocks.  Parts: S^k of K^kappa and S^G of
  // Kbar^G = K^G' - 128 I, each summed over the eight elements around a node.
  std::vector<uint16_t> bst(9 * 1280, 0);
  {
    int64_t Sk[27][9] = {}, Sg[27][9] = {};
    for (int e = 0; e < 8; ++e) {
      const int o[3] = {-(e & 1), -((e >> 1) & 1), -((e >> 2) & 1)};
      const int a = -o[0] - 2 * o[1] - 4 * o[2];  // the node's corner in element e
      for (int b = 0; b < 8; ++b) {
        const int off = (o[0] + (b & 1) + 1) + 3 * (o[1] + ((b >> 1) & 1) + 1) +
                        9 * (o[2] + ((b >> 2) & 1) + 1);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            Sk[off][3 * i + j] += Ik[(3 * a + i) * 24 + 3 * b + j];
            Sg[off][3 * i + j] += Ig[(3 * a + i) * 24 + 3 * b + j] - (a == b && i == j ? 128 : 0);
          }
      }
    }
    int64_t l1k = 0, l1g = 0;
    for (int i = 0; i < 3; ++i) {
      int64_t rk = 0, rg = 0;
      for (int off = 0; off < 27; ++off)
        for (int j = 0; j < 3; ++j) {
          rk += std::llabs(Sk[off][3 * i + j]);
          rg += std::llabs(Sg[off][3 * i + j]);
          if (std::llabs(Sk[off][3 * i + j]) > 2048 || std::llabs(Sg[off][3 * i + j]) > 2048)
            return fail(VFE_EINVAL, "internal: stencil entry not exact in fp16");
        }
      l1k = std::max(l1k, rk);
      l1g = std::max(l1g, rg);
    }
    // fp32-exact partial sums inside the magic-bias window: row L1 x 1024 < 2^22
    if (std::max(l1k, l1g) * 1024 >= (1 << 22))
      return fail(VFE_EINVAL, "internal: stencil row norm too large");
    for (int v = 0; v < 3; ++v)
      for (int dy = -1; dy <= 1; ++dy)
        for (int nn = 0; nn < 80; ++nn)
          for (int k = 0; k < 12; ++k) {
            const int blk = nn / 16, n = nn % 16;
            const int o = blk % 3 - 1;  // output plane p + o
            if ((v >= 1 && o == -1) || (v == 2 && o == 0) || n % 8 >= 6) continue;
            const int j = n / 8, co = (n % 8) / 2, part = n % 2;  // column 8 j + 2 co + part
            const int d = k / 3, c = k % 3, ox = (d - 1) - j;
            if (ox < -1 || ox > 1) continue;
            // input node = output node + (ox, dy, -o)
            const int off = (ox + 1) + 3 * (dy + 1) + 9 * (-o + 1);
            const float val = (float)(part == 0 ? Sk[off][3 * co + c] : Sg[off][3 * co + c]);
            const int byte = (v * 3 + dy + 1) * 2560 + (nn / 8) * 128 + (k / 8) * 1280 +
                             (nn % 8) * 16 + (k % 8) * 2;
            bst[byte / 2] = __half_as_ushort(__float2half(val));
          }
  }
  // correction table, after the B images (ST_MASK_IDX_OFF): for every octant
  // mask M of the eight elements around a node (bit o: element origin
  // (i - (o & 1), j - (o >> 1 & 1), k - (o >> 2))), the neighbour offsets the
  // mask's elements reach, each with the 3x3 blocks of K^kappa and of Kbar^G
  // (the node's rows, the neighbour's columns) summed over those elements,
  // which stencil_fix applies.  Index: per mask, first row and row count;
  // row: [0] offset (dx+1) + 3 (dy+1) + 9 (dz+1), [1..9] the K^kappa block
  // (row: output component), [10..18] the Kbar^G block, [19] zero.
  {
    const size_t idx_base = bst.size();
    bst.resize(idx_base + 256 * 2, 0);
    const size_t row_base = bst.size();
    int rows = 0;
    for (int mask = 0; mask < 256; ++mask) {
      int64_t Gk[27][9] = {}, Gg[27][9] = {};
      bool used[27] = {};
      for (int e = 0; e < 8; ++e) {
        if (!(mask >> e & 1)) continue;
        const int o[3] = {-(e & 1), -((e >> 1) & 1), -((e >> 2) & 1)};  // element origin
        const int a = -o[0] - 2 * o[1] - 4 * o[2];                       // the node's corner
        for (int bn = 0; bn < 8; ++bn) {
          const int off = (o[0] + (bn & 1) + 1) + 3 * (o[1] + ((bn >> 1) & 1) + 1) +
                          9 * (o[2] + ((bn >> 2) & 1) + 1);
          used[off] = true;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              Gk[off][3 * i + j] += Ik[(3 * a + i) * 24 + 3 * bn + j];
              Gg[off][3 * i + j] += Ig[(3 * a + i) * 24 + 3 * bn + j] - (a == bn && i == j ? 128 : 0);
            }
        }
      }
      // |P_M|, |Q_M| < row L1 x 2^51 must stay below 2^63
      for (int i = 0; i < 3; ++i) {
        int64_t rk = 0, rg = 0;
        for (int off = 0; off < 27; ++off)
          for (int j = 0; j < 3; ++j) {
            rk += std::llabs(Gk[off][3 * i + j]);
            rg += std::llabs(Gg[off][3 * i + j]);
          }
        if (std::max(rk, rg) >= 4096) return fail(VFE_EINVAL, "internal: correction row norm");
      }
      const int first = rows;
      for (int off = 0; off < 27; ++off) {
        if (!used[off]) continue;
        if (rows >= ST_MASK_ROWS) return fail(VFE_EINVAL, "internal: correction table size");
        bst.resize(row_base + (size_t)(rows + 1) * 20, 0);
        int16_t *ent = reinterpret_cast<int16_t *>(&bst[row_base + (size_t)rows * 20]);
        ent[0] = (int16_t)off;
        for (int q = 0; q < 9; ++q) {
          ent[1 + q] = (int16_t)Gk[off][q];
          ent[10 + q] = (int16_t)Gg[off][q];
        }
        ++rows;
      }
      int16_t *ix = reinterpret_cast<int16_t *>(&bst[idx_base + 2 * (size_t)mask]);
      ix[0] = (int16_t)first;
      ix[1] = (int16_t)(rows - first);
    }
    if (rows != ST_MASK_ROWS) return fail(VFE_EINVAL, "internal: correction table size");
  }
  if (sizeof(uint16_t) * bst.size() != ST_BST_BYTES)
    return fail(VFE_EINVAL, "internal: stencil operand buffer size");
  const size_t ubytes = sizeof(int64_t) * 3 * m->comp;
  CUDA_TRY(cudaMalloc(&m->d_U[0], ubytes));
  CUDA_TRY(cudaMalloc(&m->d_U[1], ubytes));
  CUDA_TRY(cudaMalloc(&m->d_C, sizeof(int64_t) * C.size()));
  CUDA_TRY(cudaMalloc(&m->d_Bop, sizeof(uint16_t) * bop.size()));
  // TC_MAX_MAT + 1 entries, zero beyond n_mat (ST_NO_MAT: no solid element)
  CUDA_TRY(cudaMalloc(&m->d_mats, sizeof(TcMaterial) * (TC_MAX_MAT + 1)));
  CUDA_TRY(cudaMemset(m->d_mats, 0, sizeof(TcMaterial) * (TC_MAX_MAT + 1)));
  const size_t or_words = 3 * (1 + (size_t)m->tiles_x * m->tiles_y);
  CUDA_TRY(cudaMalloc(&m->d_or, sizeof(unsigned long long) * or_words));
  CUDA_TRY(cudaMalloc(&m->d_tcparams, sizeof(TcStepParams)));
  CUDA_TRY(cudaMalloc(&m->d_tcpersist, sizeof(int64_t) * 8));
  CUDA_TRY(cudaMalloc(&m->d_Bst, sizeof(uint16_t) * bst.size()));
  CUDA_TRY(cudaMemcpy(m->d_Bst, bst.data(), sizeof(uint16_t) * bst.size(),
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(m->d_U[0], 0, ubytes));
  CUDA_TRY(cudaMemset(m->d_U[1], 0, ubytes));
  CUDA_TRY(cudaMemcpy(m->d_C, C.data(), sizeof(int64_t) * C.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->d_Bop, bop.data(), sizeof(uint16_t) * bop.size(),
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->d_mats, mats.data(), sizeof(TcMaterial) * mats.size(),
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(m->d_or, 0, sizeof(unsigned long long) * or_words));
  int64_t persist[8] = {0, 0, 0, 0, (int64_t)(m->eC + m->e_ref), 0, -1, -1};
  CUDA_TRY(cudaMemcpy(m->d_tcpersist, persist, sizeof(persist), cudaMemcpyHostToDevice));
  // TMA maps over the two state buffers: (x, y, z, component), int64, box 18x17x1x3
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(VFE_ECUDA, "cuTensorMapEncodeTiled is not available");
  for (int b = 0; b < 2; ++b) {
    int rc = encode_state_tmap(m, enc, m->d_U[b], &m->tmap[b]);
    if (rc == VFE_OK) rc = encode_state_tmap(m, enc, m->d_U[b], &m->st_tmap[b], true);
    if (rc != VFE_OK) return rc;
  }
  CUDA_TRY(stencil_prepare());
  return build_segments(m);
}

// the receivers of each element-kernel segment (the TC path) or the receiver
// node list (FP64 path); the recorded trace rows are kept
static int receiver_tables(vfe_mesh *m) {
  if (m->opt.path == VFE_PATH_TC) {
    const int items = (int)m->segs.size();
    std::vector<std::vector<TcRecv>> per(items);
    for (int r = 0; r < m->n_rec; ++r) {
      const int i = m->rec_ijk[3 * r], j = m->rec_ijk[3 * r + 1], k = m->rec_ijk[3 * r + 2];
      const int tx = i / TC_OWN, ty = j / TC_OWN;
      TcRecv v;
      v.ei = (int16_t)(i - TC_OWN * tx);
      v.ej = (int16_t)(j - TC_OWN * ty);
      v.k = k;
      v.r = r;
      v.pad = 0;
      for (int sg = 0; sg < items; ++sg) {
        const int4 q = m->segs[sg];
        if (q.x == tx && q.y == ty && k >= q.z && k < q.w) {
          per[sg].push_back(v);
          break;
        }
      }
    }
    std::vector<TcRecv> flat;
    std::vector<int32_t> off(items + 1, 0);
    for (int it = 0; it < items; ++it) {
      if ((int)per[it].size() > TC_MAX_REC_CTA)
        return fail(VFE_EINVAL, "more than %d receivers in one %dx%d node column segment",
                    TC_MAX_REC_CTA, TC_OWN, TC_OWN);
      off[it] = (int32_t)flat.size();
      flat.insert(flat.end(), per[it].begin(), per[it].end());
    }
    off[items] = (int32_t)flat.size();
    if (m->d_recv) cudaFree(m->d_recv);
    if (m->d_recv_off) cudaFree(m->d_recv_off);
    m->d_recv = nullptr;
    m->d_recv_off = nullptr;
    CUDA_TRY(cudaMalloc(&m->d_recv, sizeof(TcRecv) * std::max<size_t>(flat.size(), 1)));
    CUDA_TRY(cudaMalloc(&m->d_recv_off, sizeof(int32_t) * off.size()));
    if (!flat.empty())
      CUDA_TRY(cudaMemcpy(m->d_recv, flat.data(), sizeof(TcRecv) * flat.size(),
                          cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(m->d_recv_off, off.data(), sizeof(int32_t) * off.size(),
                        cudaMemcpyHostToDevice));
  } else {
    if (m->d_recnodes) cudaFree(m->d_recnodes);
    m->d_recnodes = nullptr;
    CUDA_TRY(cudaMalloc(&m->d_recnodes, sizeof(int64_t) * std::max(m->n_rec, 1)));
    if (m->n_rec)
      CUDA_TRY(cudaMemcpy(m->d_recnodes, m->rec_nodes.data(), sizeof(int64_t) * m->n_rec,
                          cudaMemcpyHostToDevice));
  }
  invalidate_graphs(m);
  return VFE_OK;
}

// segments (TC path: they depend on the source and receiver nodes, and on
// damping) and receiver tables after a change of either
static int rebuild_work(vfe_mesh *m) {
  if (m->opt.path == VFE_PATH_TC) {
    const int rc = build_segments(m);
    if (rc != VFE_OK) return rc;
  }
  return receiver_tables(m);
}

// new receivers: the trace rows restart
static int rebuild_receivers(vfe_mesh *m) {
  m->trace_rows = 0;
  if (m->opt.path == VFE_PATH_TC) {
    int64_t persist2 = 0;
    CUDA_TRY(cudaMemcpy(m->d_tcpersist + 2, &persist2, sizeof(int64_t), cudaMemcpyHostToDevice));
  } else {
    int64_t z = 0;
    CUDA_TRY(cudaMemcpy(m->d_f64persist + 1, &z, sizeof(int64_t), cudaMemcpyHostToDevice));
  }
  return rebuild_work(m);
}

extern "C" {

int vfe_set_source(vfe_mesh *m, int i, int j, int k, const double dir[3], double f0_hz,
                   double t0_s, double amp) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  if (!dir) return fail(VFE_EINVAL, "dir is NULL");
  if (i < 0 || j < 0 || k < 0 || i > m->nx || j > m->ny || k > m->nz)
    return fail(VFE_EINVAL, "source node (%d,%d,%d) outside the grid", i, j, k);
  if (!(f0_hz > 0.0) || !std::isfinite(f0_hz) || !std::isfinite(amp) || !std::isfinite(t0_s))
    return fail(VFE_EINVAL, "need f0 > 0 and finite t0, amp");
  if (!std::isfinite(dir[0]) || !std::isfinite(dir[1]) || !std::isfinite(dir[2]))
    return fail(VFE_EINVAL, "dir has non-finite components");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  const int64_t n = node_id(m, i, j, k);
  m->has_src = !m->fixed[n];
  m->src_set = true;
  m->src_node = n;
  for (int c = 0; c < 3; ++c) m->src_dir[c] = dir[c];
  m->f0 = f0_hz;
  m->t0 = t0_s > 0.0 ? t0_s : 1.0 / f0_hz;
  m->amp = amp;
  m->src_scale = m->has_src ? m->dt * m->dt / m->mass[n] : 0.0;
  invalidate_graphs(m);
  return rebuild_work(m);
}

int vfe_set_receivers(vfe_mesh *m, int n, const int32_t *ijk) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  if (n < 0 || (n > 0 && !ijk)) return fail(VFE_EINVAL, "bad receiver list");
  for (int r = 0; r < n; ++r) {
    const int i = ijk[3 * r], j = ijk[3 * r + 1], k = ijk[3 * r + 2];
    if (i < 0 || j < 0 || k < 0 || i > m->nx || j > m->ny || k > m->nz)
      return fail(VFE_EINVAL, "receiver %d at (%d,%d,%d) outside the grid", r, i, j, k);
  }
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->n_rec = n;
  m->rec_ijk.assign(ijk, ijk + 3 * (size_t)n);
  m->rec_nodes.resize(n);
  for (int r = 0; r < n; ++r)
    m->rec_nodes[r] = node_id(m, ijk[3 * r], ijk[3 * r + 1], ijk[3 * r + 2]);
  if (m->d_traces) cudaFree(m->d_traces);
  m->d_traces = nullptr;
  m->trace_cap = 0;
  return rebuild_receivers(m);
}

static int ensure_trace_capacity(vfe_mesh *m, int64_t rows) {
  if (m->n_rec == 0 || rows <= m->trace_cap) return VFE_OK;
  int64_t cap = std::max<int64_t>(rows, std::max<int64_t>(2 * m->trace_cap, 1024));
  double *p = nullptr;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (cudaMalloc(&p, sizeof(double) * 3 * m->n_rec * cap) != cudaSuccess)
    return fail(VFE_ENOMEM, "trace buffer of %lld rows", (long long)cap);
  if (m->d_traces && m->trace_rows > 0)
    CUDA_TRY(cudaMemcpy(p, m->d_traces, sizeof(double) * 3 * m->n_rec * m->trace_rows,
                        cudaMemcpyDeviceToDevice));
  if (m->d_traces) cudaFree(m->d_traces);
  m->d_traces = p;
  m->trace_cap = cap;
  invalidate_graphs(m);
  return VFE_OK;
}

// queue n steps on the mesh's stream (n >= 1, device already current)
static int run_steps(vfe_mesh *m, int n) {
  int rc = ensure_trace_capacity(m, m->trace_rows + n);
  if (rc != VFE_OK) return rc;
  // pairs of steps replay a captured two-step graph; the source term, scales
  // and trace rows live in device memory, so the graph is reusable
  int64_t left = n;
  while (left >= kLongSteps) {
    rc = ensure_long_graph(m, m->cur);
    if (rc != VFE_OK) return rc;
    CUDA_TRY(cudaGraphLaunch(m->graph_long[m->cur], m->stream));
    left -= kLongSteps;
  }
  while (left >= 2) {
    rc = ensure_graph(m, m->cur);
    if (rc != VFE_OK) return rc;
    CUDA_TRY(cudaGraphLaunch(m->graph[m->cur], m->stream));
    left -= 2;
  }
  if (left == 1) {
    rc = enqueue_step(m, m->cur);
    if (rc != VFE_OK) return rc;
    m->cur = 1 - m->cur;
  }
  m->steps += n;
  if (m->n_rec) m->trace_rows += n;
  return VFE_OK;
}

int vfe_step(vfe_mesh *m, int n) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  if (n < 0) return fail(VFE_EINVAL, "n must be >= 0");
  if (n == 0) return VFE_OK;
  cudaSetDevice(m->device);
  return run_steps(m, n);
}

int vfe_step_forced(vfe_mesh *m, int n, const double *force) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  if (n < 0) return fail(VFE_EINVAL, "n must be >= 0");
  if (n == 0) return VFE_OK;
  if (!force) return fail(VFE_EINVAL, "force is NULL");
  if (!m->src_set) return fail(VFE_ESTATE, "no source node: call vfe_set_source first");
  for (int64_t k = 0; k < 3 * (int64_t)n; ++k)
    if (!std::isfinite(force[k])) return fail(VFE_EINVAL, "force[%lld] is not finite", (long long)k);
  cudaSetDevice(m->device);
  if (n > m->force_cap) {  // the prologues capture the buffer's address: new graphs
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    const int64_t cap = std::max<int64_t>(n, std::max<int64_t>(2 * m->force_cap, 64));
    double *p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * (3 * cap + 1)) != cudaSuccess)
      return fail(VFE_ENOMEM, "force buffer of %lld rows", (long long)cap);
    const int64_t off = -1;
    if (cudaMemcpy(p + 3 * cap, &off, sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(p);
      return fail(VFE_ECUDA, "force buffer initialisation failed");
    }
    if (m->d_force) cudaFree(m->d_force);
    m->d_force = p;
    m->force_cap = cap;
    invalidate_graphs(m);
  }
  // the rows, then first step := the device's own step counter, the steps,
  // and the series ended again, all in stream order and without host staging
  CUDA_TRY(cudaMemcpyAsync(m->d_force, force, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                           m->stream));
  const bool tc = m->opt.path == VFE_PATH_TC;
  int64_t *pers = tc ? m->d_tcpersist : m->d_f64persist;
  const int slot_first = tc ? 7 : 4, slot_step = tc ? 1 : 0;
  CUDA_TRY(cudaMemcpyAsync(pers + slot_first, pers + slot_step, sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, m->stream));
  const int rc = run_steps(m, n);
  CUDA_TRY(cudaMemcpyAsync(pers + slot_first, m->d_force + 3 * m->force_cap, sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, m->stream));
  return rc;
}

int vfe_synchronize(vfe_mesh *m) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return check_status(m);
}

int vfe_get_traces(vfe_mesh *m, double *out, int64_t *n_steps_out) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  int rc = vfe_synchronize(m);
  if (rc != VFE_OK) return rc;
  if (n_steps_out) *n_steps_out = m->trace_rows;
  if (out && m->n_rec && m->trace_rows)
    CUDA_TRY(cudaMemcpy(out, m->d_traces, sizeof(double) * 3 * m->n_rec * m->trace_rows,
                        cudaMemcpyDeviceToHost));
  return VFE_OK;
}

// queue the copy of trace rows [first, first + count) on the mesh's stream
static int enqueue_trace_rows(vfe_mesh *m, int64_t first, int64_t count, double *out) {
  if (first < 0 || count < 0 || (count > 0 && !out)) return fail(VFE_EINVAL, "bad row range");
  cudaSetDevice(m->device);
  if (first + count > m->trace_rows)
    return fail(VFE_EINVAL, "rows [%lld, %lld) beyond the %lld recorded", (long long)first,
                (long long)(first + count), (long long)m->trace_rows);
  if (count == 0 || m->n_rec == 0) return VFE_OK;
  CUDA_TRY(cudaMemcpyAsync(out, m->d_traces + first * 3 * m->n_rec,
                           sizeof(double) * 3 * m->n_rec * count, cudaMemcpyDeviceToHost,
                           m->stream));
  return VFE_OK;
}

int vfe_get_trace_rows(vfe_mesh *m, int64_t first, int64_t count, double *out) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  const int rc = enqueue_trace_rows(m, first, count, out);
  if (rc != VFE_OK || count == 0 || m->n_rec == 0) return rc;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return check_status(m);
}

int vfe_get_trace_rows_async(vfe_mesh *m, int64_t first, int64_t count, double *out) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  return enqueue_trace_rows(m, first, count, out);
}

int vfe_get_dt(vfe_mesh *m, double *dt) {
  if (!m || !dt) return fail(VFE_EINVAL, "NULL argument");
  *dt = m->dt;
  return VFE_OK;
}

int vfe_get_sizes(vfe_mesh *m, int64_t *n_nodes, int64_t *n_elements) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  if (n_nodes) *n_nodes = m->nn;
  if (n_elements) *n_elements = m->ne;
  return VFE_OK;
}

int vfe_get_step_count(vfe_mesh *m, int64_t *steps) {
  if (!m || !steps) return fail(VFE_EINVAL, "NULL argument");
  *steps = m->steps;
  return VFE_OK;
}

int vfe_get_launches_per_step(vfe_mesh *m, int *launches) {
  if (!m || !launches) return fail(VFE_EINVAL, "NULL argument");
  if (m->opt.path == VFE_PATH_TC)
    *launches = 1 + (tc_device(m, 0).n_ctas > 0 ? 1 : 0) + (m->stencil_on ? 1 : 0) +
                (m->stencil_on && m->n_fix > 0 ? 1 : 0);
  else
    *launches = 2;
  return VFE_OK;
}

}  // extern "C"

// ---- state conversion (FP64 <-> fixed point for the TC path) -----------------

// F such that max|u| 2^F lies in [2^57, 2^58); 0 for an all-zero field
static int pick_frac_bits(const double *a, const double *b, int64_t n) {
  double mx = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    mx = std::max(mx, std::fabs(a[i]));
    if (b) mx = std::max(mx, std::fabs(b[i]));
  }
  if (mx == 0.0) return 0;
  return (TC_UNITS_BITS - 1) - std::ilogb(mx);
}

static void to_fixed(const vfe_mesh *m, const double *u, int F, std::vector<int64_t> &U,
                     bool zero_fixed, unsigned long long *orv) {
  U.assign(3 * m->comp, 0);
  unsigned long long acc = 0;
  for (int64_t n = 0; n < m->nn; ++n) {
    if (zero_fixed && m->fixed[n]) continue;
    const int64_t t = tc_index(m, n);
    for (int c = 0; c < 3; ++c) {
      const int64_t v = llrint(std::ldexp(u[3 * n + c], F));
      U[c * m->comp + t] = v;
      acc |= (unsigned long long)(v < 0 ? -v : v);
    }
  }
  if (orv) *orv = acc;
}

static int bitlen(unsigned long long v) { return v ? 64 - __builtin_clzll(v) : 0; }

extern "C" {

int vfe_set_state(vfe_mesh *m, const double *u, const double *u_prev) {
  if (!m || !u || !u_prev) return fail(VFE_EINVAL, "NULL argument");
  for (int64_t i = 0; i < 3 * m->nn; ++i)
    if (!std::isfinite(u[i]) || !std::isfinite(u_prev[i]))
      return fail(VFE_EINVAL, "state has non-finite values");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (m->opt.path == VFE_PATH_TC) {
    const int F = pick_frac_bits(u, u_prev, 3 * m->nn);
    std::vector<int64_t> U0, U1;
    unsigned long long o0 = 0, o1 = 0;
    to_fixed(m, u, F, U0, true, &o0);
    to_fixed(m, u_prev, F, U1, true, &o1);
    CUDA_TRY(cudaMemcpy(m->d_U[m->cur], U0.data(), sizeof(int64_t) * U0.size(),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(m->d_U[1 - m->cur], U1.data(), sizeof(int64_t) * U1.size(),
                        cudaMemcpyHostToDevice));
    // the next step reads slot (step + 2) % 3: the global bound of |u^n|,
    // |u^{n-1}| and one bound per 15x15 node column (its digit quantum)
    // with damping the digitised vector is w^n = u^n + (beta / dt)(u^n - u^{n-1})
    std::vector<int64_t> W0;
    unsigned long long ow = 0;
    if (m->damped) {
      const double bb = m->beta / m->dt;
      std::vector<double> w(3 * m->nn);
      for (size_t i = 0; i < w.size(); ++i) w[i] = u[i] + bb * (u[i] - u_prev[i]);
      to_fixed(m, w.data(), F, W0, true, &ow);
      CUDA_TRY(cudaMemcpy(m->d_W[m->cur], W0.data(), sizeof(int64_t) * W0.size(),
                          cudaMemcpyHostToDevice));
    }
    const int ncols = m->tiles_x * m->tiles_y;
    std::vector<unsigned long long> slots(3 * (size_t)(1 + ncols), 0);
    unsigned long long *sl = slots.data() + (size_t)((m->steps + 2) % 3) * (1 + ncols);
    sl[0] = o0 | o1 | ow;
    for (int64_t n = 0; n < m->nn; ++n) {
      const int64_t i = n % (m->nx + 1), j = (n / (m->nx + 1)) % (m->ny + 1);
      const int64_t t = tc_index(m, n);
      unsigned long long o = 0;
      for (int c = 0; c < 3; ++c) {
        const int64_t a = U0[c * m->comp + t], b = U1[c * m->comp + t];
        o |= (unsigned long long)(a < 0 ? -a : a) | (unsigned long long)(b < 0 ? -b : b);
        if (m->damped) {
          const int64_t w = W0[c * m->comp + t];
          o |= (unsigned long long)(w < 0 ? -w : w);
        }
      }
      sl[1 + (j / TC_OWN) * m->tiles_x + (i / TC_OWN)] |= o;
    }
    CUDA_TRY(cudaMemcpy(m->d_or, slots.data(), sizeof(unsigned long long) * slots.size(),
                        cudaMemcpyHostToDevice));
    int64_t F64 = F, zero = 0;
    CUDA_TRY(cudaMemcpy(m->d_tcpersist, &F64, sizeof(int64_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(m->d_tcpersist + 5, &zero, sizeof(int64_t), cudaMemcpyHostToDevice));
  } else {
    std::vector<double> a(u, u + 3 * m->nn), b(u_prev, u_prev + 3 * m->nn);
    for (int64_t n = 0; n < m->nn; ++n)
      if (m->fixed[n])
        for (int c = 0; c < 3; ++c) a[3 * n + c] = b[3 * n + c] = 0.0;
    CUDA_TRY(cudaMemcpy(m->d_u[m->cur], a.data(), sizeof(double) * a.size(),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(m->d_u[1 - m->cur], b.data(), sizeof(double) * b.size(),
                        cudaMemcpyHostToDevice));
    if (m->damped) {  // w^n = u^n + (beta / dt) (u^n - u^{n-1})
      const double bb = m->beta / m->dt;
      std::vector<double> w(a.size());
      for (size_t i = 0; i < w.size(); ++i) w[i] = a[i] + bb * (a[i] - b[i]);
      CUDA_TRY(cudaMemcpy(m->d_w[m->cur], w.data(), sizeof(double) * w.size(),
                          cudaMemcpyHostToDevice));
    }
  }
  return VFE_OK;
}

int vfe_rayleigh_coefficients(double h, double f1_hz, double f2_hz, double *alpha,
                              double *beta) {
  if (!alpha || !beta) return fail(VFE_EINVAL, "NULL output");
  if (!(h >= 0.0) || !std::isfinite(h) || !(f1_hz > 0.0) || !(f2_hz >= f1_hz) ||
      !std::isfinite(f2_hz))
    return fail(VFE_EINVAL, "need h >= 0 and 0 < f1 <= f2");
  const double w1 = 2.0 * M_PI * f1_hz, w2 = 2.0 * M_PI * f2_hz;
  *alpha = 2.0 * h * w1 * w2 / (w1 + w2);
  *beta = 2.0 * h / (w1 + w2);
  return VFE_OK;
}

int vfe_set_damping(vfe_mesh *m, double alpha, double beta) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  if (!(alpha >= 0.0) || !(beta >= 0.0) || !std::isfinite(alpha) || !std::isfinite(beta))
    return fail(VFE_EINVAL, "need finite alpha >= 0 and beta >= 0");
  const double a = 0.5 * alpha * m->dt, b = beta / m->dt, r = m->dt / m->dt_crit;
  if (a >= 1.0) return fail(VFE_EINVAL, "alpha dt / 2 = %g must be below 1", a);
  if (r * r * (1.0 + 2.0 * b) > 1.0)
    return fail(VFE_EINVAL,
                "unstable: (dt / dt_crit)^2 (1 + 2 beta / dt) = %g exceeds 1 (dt %g, dt_crit %g)",
                r * r * (1.0 + 2.0 * b), m->dt, m->dt_crit);
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  // rebuild w from the current state with the new coefficients
  std::vector<double> u(3 * m->nn), up(3 * m->nn);
  int rc = vfe_get_state(m, u.data(), up.data());
  if (rc != VFE_OK) return rc;
  const bool damped = alpha > 0.0 || beta > 0.0;
  // each buffer is allocated on its own, so a failed call leaves no half-built
  // pair behind (the next call allocates whatever is still missing)
  if (damped && m->opt.path == VFE_PATH_FP64)
    for (int i = 0; i < 2; ++i)
      if (!m->d_w[i] && cudaMalloc(&m->d_w[i], sizeof(double) * 3 * m->nn) != cudaSuccess) {
        m->d_w[i] = nullptr;
        return fail(VFE_ENOMEM, "damping state");
      }
  if (damped && m->opt.path == VFE_PATH_TC)
    for (int i = 0; i < 2; ++i) {
      if (m->d_W[i]) continue;
      EncodeTiledFn enc = encode_fn();
      if (!enc) return fail(VFE_ECUDA, "cuTensorMapEncodeTiled is not available");
      int64_t *p = nullptr;
      if (cudaMalloc(&p, sizeof(int64_t) * 3 * m->comp) != cudaSuccess)
        return fail(VFE_ENOMEM, "damping state");
      if (cudaMemset(p, 0, sizeof(int64_t) * 3 * m->comp) != cudaSuccess ||
          (rc = encode_state_tmap(m, enc, p, &m->tmap_w[i])) != VFE_OK) {
        cudaFree(p);
        return rc != VFE_OK ? rc : fail(VFE_ECUDA, "damping state");
      }
      m->d_W[i] = p;
    }
  m->alpha = alpha;
  m->beta = beta;
  m->damped = damped;
  if (m->opt.path == VFE_PATH_TC) {  // the update multipliers carry 1 / (1 + alpha dt / 2)
    const std::vector<int64_t> C = tc_update_multipliers(m);
    CUDA_TRY(cudaMemcpy(m->d_C, C.data(), sizeof(int64_t) * C.size(), cudaMemcpyHostToDevice));
    if ((rc = rebuild_work(m)) != VFE_OK) return rc;  // damped steps: element kernel only
  }
  invalidate_graphs(m);
  return vfe_set_state(m, u.data(), up.data());
}

int vfe_get_state(vfe_mesh *m, double *u, double *u_prev) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  int rc = vfe_synchronize(m);
  if (rc != VFE_OK) return rc;
  if (m->opt.path == VFE_PATH_TC) {
    int64_t pers[8];
    CUDA_TRY(cudaMemcpy(pers, m->d_tcpersist, sizeof(pers), cudaMemcpyDeviceToHost));
    std::vector<int64_t> U(3 * m->comp);
    for (int which = 0; which < 2; ++which) {
      double *dst = which == 0 ? u : u_prev;
      if (!dst) continue;
      // u^n is stored with F = pers[0], u^{n-1} with F + (shift of the last step)
      const int64_t F = which == 0 ? pers[0] : pers[0] + pers[5];
      CUDA_TRY(cudaMemcpy(U.data(), m->d_U[which == 0 ? m->cur : 1 - m->cur],
                          sizeof(int64_t) * U.size(), cudaMemcpyDeviceToHost));
      for (int64_t n = 0; n < m->nn; ++n) {
        const int64_t t = tc_index(m, n);
        for (int c = 0; c < 3; ++c) dst[3 * n + c] = std::ldexp((double)U[c * m->comp + t], -(int)F);
      }
    }
  } else {
    if (u)
      CUDA_TRY(cudaMemcpy(u, m->d_u[m->cur], sizeof(double) * 3 * m->nn, cudaMemcpyDeviceToHost));
    if (u_prev)
      CUDA_TRY(cudaMemcpy(u_prev, m->d_u[1 - m->cur], sizeof(double) * 3 * m->nn,
                          cudaMemcpyDeviceToHost));
  }
  return VFE_OK;
}

// K u through the kernels (mode 1: S output, mode 2: exact partials)
static int tc_apply(vfe_mesh *m, const double *u, int mode, std::vector<int64_t> &out, int *shq_out,
                    int *F_out) {
  const int F = pick_frac_bits(u, nullptr, 3 * m->nn);
  std::vector<int64_t> U;
  unsigned long long orv = 0;
  to_fixed(m, u, F, U, false, &orv);
  const int shq = std::max(0, bitlen(orv) - TC_QBITS);
  int64_t *dU = nullptr, *dout = nullptr;
  TcStepParams *dp = nullptr;
  const size_t ubytes = sizeof(int64_t) * U.size();
  const size_t obytes = mode == TC_MODE_KU ? ubytes : sizeof(int64_t) * 48 * m->ne;
  int rc = VFE_OK;
  cudaError_t e;
  do {
    if ((e = cudaMalloc(&dU, ubytes)) != cudaSuccess || (e = cudaMalloc(&dout, obytes)) != cudaSuccess ||
        (e = cudaMalloc(&dp, sizeof(TcStepParams))) != cudaSuccess) {
      rc = fail(VFE_ENOMEM, "scratch allocation: %s", cudaGetErrorString(e));
      break;
    }
    TcStepParams p;
    memset(&p, 0, sizeof(p));
    p.trace_row = -1;
    p.shq = shq;
    p.F = F;
    if ((e = cudaMemcpy(dU, U.data(), ubytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(dout, 0, obytes)) != cudaSuccess ||
        (e = cudaMemcpy(dp, &p, sizeof(p), cudaMemcpyHostToDevice)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "upload: %s", cudaGetErrorString(e));
      break;
    }
    // tensor maps over the scratch copy of u (element and node-stencil boxes)
    CUtensorMap tm, tms;
    if ((rc = encode_state_tmap(m, encode_fn(), dU, &tm)) != VFE_OK ||
        (rc = encode_state_tmap(m, encode_fn(), dU, &tms, true)) != VFE_OK)
      break;
    TcDevice d = tc_device(m, m->cur);
    d.params = dp;
    d.src_node = -1;
    d.n_rec = 0;
    d.S_out = mode == TC_MODE_KU ? dout : nullptr;
    d.partials_out = mode == TC_MODE_PARTIALS ? dout : nullptr;
    if (mode == TC_MODE_PARTIALS) {  // every element, on the element kernel
      d.segs = m->d_all_segs;
      d.seg_off = m->d_all_off;
      d.n_ctas = m->all_ctas;
    }
    if (d.n_ctas > 0 && (e = tc_launch_step(m->stream, d, &tm, mode)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "K u kernel: %s", cudaGetErrorString(e));
      break;
    }
    if (mode == TC_MODE_KU && m->stencil_on) {  // the stencil runs
      TcDevice ds = tc_stencil_device(m, m->cur);
      ds.params = dp;
      ds.S_out = dout;
      ds.U_cur = dU;
      if ((e = stencil_launch(m->stream, ds, &tms, TC_MODE_KU)) != cudaSuccess ||
          (e = stencil_fix(m->stream, ds, TC_MODE_KU)) != cudaSuccess) {
        rc = fail(VFE_ECUDA, "node-stencil K u kernel: %s", cudaGetErrorString(e));
        break;
      }
    }
    if ((e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "K u kernel: %s", cudaGetErrorString(e));
      break;
    }
    rc = check_status(m);
    if (rc != VFE_OK) break;
    out.resize(obytes / sizeof(int64_t));
    if ((e = cudaMemcpy(out.data(), dout, obytes, cudaMemcpyDeviceToHost)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "download: %s", cudaGetErrorString(e));
      break;
    }
  } while (0);
  if (dU) cudaFree(dU);
  if (dout) cudaFree(dout);
  if (dp) cudaFree(dp);
  *shq_out = shq;
  *F_out = F;
  return rc;
}

int vfe_internal_force(vfe_mesh *m, const double *u, double *f) {
  if (!m || !u || !f) return fail(VFE_EINVAL, "NULL argument");
  for (int64_t i = 0; i < 3 * m->nn; ++i)
    if (!std::isfinite(u[i])) return fail(VFE_EINVAL, "u has non-finite values");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (m->opt.path == VFE_PATH_TC) {
    std::vector<int64_t> S;
    int shq = 0, F = 0;
    int rc = tc_apply(m, u, TC_MODE_KU, S, &shq, &F);
    if (rc != VFE_OK) return rc;
    const int ex = 63 - m->e_ref + shq - F;
    for (int64_t n = 0; n < m->nn; ++n) {
      const int64_t t = tc_index(m, n);
      for (int c = 0; c < 3; ++c) f[3 * n + c] = std::ldexp((double)S[c * m->comp + t], ex);
    }
    return VFE_OK;
  }
  double *du = nullptr, *df = nullptr;
  int rc = VFE_OK;
  cudaError_t e;
  do {
    if ((e = cudaMalloc(&du, sizeof(double) * 3 * m->nn)) != cudaSuccess ||
        (e = cudaMalloc(&df, sizeof(double) * 3 * m->nn)) != cudaSuccess) {
      rc = fail(VFE_ENOMEM, "scratch allocation: %s", cudaGetErrorString(e));
      break;
    }
    if ((e = cudaMemcpy(du, u, sizeof(double) * 3 * m->nn, cudaMemcpyHostToDevice)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "upload: %s", cudaGetErrorString(e));
      break;
    }
    F64Device d = f64_device(m, m->cur);
    d.u = du;
    d.f_out = df;
    if ((e = f64_launch_step(m->stream, d, m->d_f64params, 1)) != cudaSuccess ||
        (e = cudaStreamSynchronize(m->stream)) != cudaSuccess ||
        (e = cudaMemcpy(f, df, sizeof(double) * 3 * m->nn, cudaMemcpyDeviceToHost)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "K u kernel: %s", cudaGetErrorString(e));
      break;
    }
  } while (0);
  if (du) cudaFree(du);
  if (df) cudaFree(df);
  if (rc == VFE_OK) rc = check_status(m);  // a failure flagged by earlier work
  return rc;
}

}  // extern "C"

void vfe_set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

int vfe_mesh_view(vfe_mesh *m, VfeMeshView *v) {
  if (!m || !v) return VFE_EINVAL;
  v->nx = m->nx; v->ny = m->ny; v->nz = m->nz; v->nxp = m->nxp; v->nyp = m->nyp;
  v->nn = m->nn; v->plane = m->plane; v->comp = m->comp;
  v->e_ref = m->e_ref;
  v->device = m->device;
  v->tc = m->opt.path == VFE_PATH_TC ? 1 : 0;
  v->stream = m->stream;
  v->dev = tc_device(m, m->cur);
  v->stencil_on = m->stencil_on ? 1 : 0;
  v->st = tc_stencil_device(m, m->cur);
  return VFE_OK;
}

CUresult vfe_encode_state_map(CUtensorMap *map, void *base, const VfeMeshView &v,
                              bool stencil_box) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return CUDA_ERROR_NOT_SUPPORTED;
  cuuint64_t dims[4] = {(cuuint64_t)v.nxp, (cuuint64_t)v.nyp, (cuuint64_t)(v.nz + 1), 3};
  cuuint64_t strides[3] = {(cuuint64_t)v.nxp * 8, (cuuint64_t)v.plane * 8, (cuuint64_t)v.comp * 8};
  cuuint32_t box[4] = {stencil_box ? (cuuint32_t)ST_BOXX : (cuuint32_t)TC_BOXX,
                       stencil_box ? (cuuint32_t)ST_BOXY : (cuuint32_t)TC_NODES, 1, 3};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, base, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

extern "C" {

// the TC path's material unit e_ref and multipliers for the largest of the
// bulk and shear terms (per material, and per element when elem_g)
static int tc_encode_moduli(vfe_mesh *m) {
  double mx = 0.0;
  for (int i = 0; i < m->n_mat; ++i)
    mx = std::max(mx, std::max(m->kappa[i] * m->h / 256.0, m->G[i] * m->h / 384.0));
  if (m->elem_g)
    for (int64_t e = 0; e < m->ne; ++e)
      if (m->mat[e] >= 0) mx = std::max(mx, m->elem_G[e] * m->h / 384.0);
  const int e_ref = 60 - std::ilogb(mx);
  std::vector<TcMaterial> mats(m->n_mat);
  for (int i = 0; i < m->n_mat; ++i) {
    mats[i].A = llrint(std::ldexp(m->kappa[i] * m->h / 256.0, e_ref));
    mats[i].B = llrint(std::ldexp(m->G[i] * m->h / 384.0, e_ref));
    mats[i].shift = 0;
    mats[i].pad = 0;
  }
  CUDA_TRY(cudaMemcpy(m->d_mats, mats.data(), sizeof(TcMaterial) * mats.size(),
                      cudaMemcpyHostToDevice));
  if (m->elem_g) {
    std::vector<int64_t> B(m->ne, 0);
    for (int64_t e = 0; e < m->ne; ++e)
      if (m->mat[e] >= 0) B[e] = llrint(std::ldexp(m->elem_G[e] * m->h / 384.0, e_ref));
    if (!m->d_elemB) CUDA_TRY(cudaMalloc(&m->d_elemB, sizeof(int64_t) * m->ne));
    CUDA_TRY(cudaMemcpy(m->d_elemB, B.data(), sizeof(int64_t) * m->ne, cudaMemcpyHostToDevice));
  }
  m->e_ref = e_ref;
  const int64_t pe = m->eC + m->e_ref;  // the exponent the step prologue reads
  CUDA_TRY(cudaMemcpy(m->d_tcpersist + 4, &pe, sizeof(int64_t), cudaMemcpyHostToDevice));
  return VFE_OK;
}

int vfe_set_shear_moduli(vfe_mesh *m, const double *G) {
  if (!m) return fail(VFE_EINVAL, "mesh is NULL");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (G) {
    for (int64_t e = 0; e < m->ne; ++e)
      if (m->mat[e] >= 0 && !(G[e] >= 0.0 && std::isfinite(G[e])))
        return fail(VFE_EINVAL, "G[%lld] must be finite and >= 0", (long long)e);
    // stability with the largest shear modulus of each material (lambda_max of
    // M_e^-1 K_e grows with G at fixed kappa)
    std::vector<double> gmax(m->n_mat, -1.0);
    for (int64_t e = 0; e < m->ne; ++e)
      if (m->mat[e] >= 0) gmax[m->mat[e]] = std::max(gmax[m->mat[e]], G[e]);
    double dtc = -1.0;
    for (int i = 0; i < m->n_mat; ++i) {
      if (gmax[i] < 0.0) continue;
      double K[576];
      element_matrix(m->opt.element_kind, m->h, m->kappa[i] - 2.0 * gmax[i] / 3.0, gmax[i], K);
      const double lmax = max_eigenvalue(K) / (m->rho[i] * m->h * m->h * m->h / 8.0);
      const double c = lmax > 0.0 ? 2.0 / std::sqrt(lmax) : 1e300;
      if (dtc < 0.0 || c < dtc) dtc = c;
    }
    if (dtc > 0.0 && m->dt > dtc)
      return fail(VFE_EINVAL, "dt %g exceeds the stability limit %g with these moduli", m->dt, dtc);
    m->elem_G.assign(G, G + m->ne);
    m->elem_g = true;
    if (dtc > 0.0) m->dt_crit = dtc;
  } else {
    m->elem_g = false;
    m->elem_G.clear();
  }
  if (m->opt.path == VFE_PATH_TC) {
    const int rc = tc_encode_moduli(m);
    if (rc != VFE_OK) return rc;
  } else if (m->elem_g) {
    std::vector<double> Kkg(2 * 576), gE(m->elem_G);
    element_matrix(m->opt.element_kind, m->h, 1.0, 0.0, Kkg.data());
    element_matrix(m->opt.element_kind, m->h, -2.0 / 3.0, 1.0, Kkg.data() + 576);
    for (int64_t e = 0; e < m->ne; ++e)
      if (m->mat[e] < 0) gE[e] = 0.0;
    if (!m->d_elemG) CUDA_TRY(cudaMalloc(&m->d_elemG, sizeof(double) * m->ne));
    if (!m->d_kappa) CUDA_TRY(cudaMalloc(&m->d_kappa, sizeof(double) * m->n_mat));
    if (!m->d_Kkg) CUDA_TRY(cudaMalloc(&m->d_Kkg, sizeof(double) * 2 * 576));
    CUDA_TRY(cudaMemcpy(m->d_elemG, gE.data(), sizeof(double) * m->ne, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(m->d_kappa, m->kappa.data(), sizeof(double) * m->n_mat,
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(m->d_Kkg, Kkg.data(), sizeof(double) * 2 * 576, cudaMemcpyHostToDevice));
  }
  invalidate_graphs(m);
  return rebuild_work(m);  // per-element moduli: the element kernel everywhere
}

int vfe_get_source_scale(vfe_mesh *m, double *dt2_over_m) {
  if (!m || !dt2_over_m) return fail(VFE_EINVAL, "NULL argument");
  *dt2_over_m = m->has_src ? m->src_scale : 0.0;
  return VFE_OK;
}

int vfe_set_source_bound(vfe_mesh *m, const double dir[3], double f0_hz, double t0_s, double amp,
                         double dt2_over_m) {
  if (!m || !dir) return fail(VFE_EINVAL, "NULL argument");
  if (m->has_src) return fail(VFE_ESTATE, "the mesh holds the source itself");
  if (!(f0_hz > 0.0) || !std::isfinite(f0_hz) || !std::isfinite(amp) || !std::isfinite(t0_s) ||
      !(dt2_over_m >= 0.0) || !std::isfinite(dt2_over_m))
    return fail(VFE_EINVAL, "need f0 > 0, dt2_over_m >= 0 and finite t0, amp");
  if (!std::isfinite(dir[0]) || !std::isfinite(dir[1]) || !std::isfinite(dir[2]))
    return fail(VFE_EINVAL, "dir has non-finite components");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->src_bound_only = m->opt.path == VFE_PATH_TC;  // the FP64 path has no scale
  for (int c = 0; c < 3; ++c) m->src_dir[c] = dir[c];
  m->f0 = f0_hz;
  m->t0 = t0_s > 0.0 ? t0_s : 1.0 / f0_hz;
  m->amp = amp;
  m->src_scale = dt2_over_m;
  invalidate_graphs(m);
  return VFE_OK;
}

static unsigned long long *next_bound_word(vfe_mesh *m) {
  return m->d_or + (size_t)((m->steps + 2) % 3) * (1 + m->tiles_x * m->tiles_y);
}

int vfe_get_scale_bound(vfe_mesh *m, unsigned long long *dev_word) {
  if (!m || !dev_word) return fail(VFE_EINVAL, "NULL argument");
  cudaSetDevice(m->device);
  if (m->opt.path == VFE_PATH_TC)
    CUDA_TRY(cudaMemcpyAsync(dev_word, next_bound_word(m), sizeof(unsigned long long),
                             cudaMemcpyDeviceToDevice, m->stream));
  else
    CUDA_TRY(cudaMemsetAsync(dev_word, 0, sizeof(unsigned long long), m->stream));
  return VFE_OK;
}

int vfe_set_scale_bound(vfe_mesh *m, const unsigned long long *dev_word) {
  if (!m || !dev_word) return fail(VFE_EINVAL, "NULL argument");
  cudaSetDevice(m->device);
  if (m->opt.path == VFE_PATH_TC)
    CUDA_TRY(cudaMemcpyAsync(next_bound_word(m), dev_word, sizeof(unsigned long long),
                             cudaMemcpyDeviceToDevice, m->stream));
  return VFE_OK;
}

int vfe_plane_values(vfe_mesh *m, int64_t *n_values) {
  if (!m || !n_values) return fail(VFE_EINVAL, "NULL argument");
  *n_values = 3 * (int64_t)(m->nx + 1) * (m->ny + 1);
  return VFE_OK;
}

int vfe_pack_plane(vfe_mesh *m, int k, double *dev_out) {
  if (!m || !dev_out) return fail(VFE_EINVAL, "NULL argument");
  if (k < 0 || k > m->nz) return fail(VFE_EINVAL, "node plane %d outside [0, %d]", k, m->nz);
  if (m->damped) return fail(VFE_ESTATE, "plane exchange is not combined with damping");
  cudaSetDevice(m->device);
  const int64_t np = (int64_t)(m->nx + 1) * (m->ny + 1);
  if (m->opt.path == VFE_PATH_TC) {
    CUDA_TRY(slab_pack_tc(m->stream, m->d_U[m->cur], m->nx, m->ny, m->nxp, m->plane, m->comp, k,
                          m->d_tcpersist, dev_out));
  } else {
    CUDA_TRY(cudaMemcpyAsync(dev_out, m->d_u[m->cur] + 3 * np * k, sizeof(double) * 3 * np,
                             cudaMemcpyDeviceToDevice, m->stream));
  }
  return VFE_OK;
}

int vfe_unpack_plane(vfe_mesh *m, int k, const double *dev_in) {
  if (!m || !dev_in) return fail(VFE_EINVAL, "NULL argument");
  if (k < 0 || k > m->nz) return fail(VFE_EINVAL, "node plane %d outside [0, %d]", k, m->nz);
  if (m->damped) return fail(VFE_ESTATE, "plane exchange is not combined with damping");
  cudaSetDevice(m->device);
  const int64_t np = (int64_t)(m->nx + 1) * (m->ny + 1);
  if (m->opt.path == VFE_PATH_TC) {
    // the bound records the next step reads
    unsigned long long *slot = next_bound_word(m);
    CUDA_TRY(slab_unpack_tc(m->stream, m->d_U[m->cur], m->nx, m->ny, m->nxp, m->plane, m->comp, k,
                            m->d_tcpersist, dev_in, slot, m->tiles_x));
  } else {
    CUDA_TRY(cudaMemcpyAsync(m->d_u[m->cur] + 3 * np * k, dev_in, sizeof(double) * 3 * np,
                             cudaMemcpyDeviceToDevice, m->stream));
  }
  return VFE_OK;
}

int vfe_debug_stencil_partials(vfe_mesh *m, const double *u, int64_t *out, int8_t *covered,
                               int *shift_out, int *frac_bits_out) {
  if (!m || !u || !out || !covered) return fail(VFE_EINVAL, "NULL argument");
  if (m->opt.path != VFE_PATH_TC) return fail(VFE_ESTATE, "mesh is not on the tensor-core path");
  for (int64_t i = 0; i < 3 * m->nn; ++i)
    if (!std::isfinite(u[i])) return fail(VFE_EINVAL, "u has non-finite values");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  const int F = pick_frac_bits(u, nullptr, 3 * m->nn);
  std::vector<int64_t> U;
  unsigned long long orv = 0;
  to_fixed(m, u, F, U, false, &orv);
  const int shq = std::max(0, bitlen(orv) - TC_QBITS);
  std::vector<char> cov(m->nn, 0);
  if (m->stencil_on)
    for (const int4 &q : m->st_segs)
      for (int k = q.z; k < q.w; ++k)
        for (int j = TC_OWN * q.y; j < std::min(TC_OWN * q.y + TC_OWN, m->ny + 1); ++j)
          for (int i = TC_OWN * q.x; i < std::min(TC_OWN * q.x + TC_OWN, m->nx + 1); ++i)
            cov[node_id(m, i, j, k)] = 1;
  int64_t *dU = nullptr, *dout = nullptr;
  TcStepParams *dp = nullptr;
  const size_t ubytes = sizeof(int64_t) * U.size(), obytes = 3 * ubytes;
  int rc = VFE_OK;
  cudaError_t e;
  do {
    if ((e = cudaMalloc(&dU, ubytes)) != cudaSuccess || (e = cudaMalloc(&dout, obytes)) != cudaSuccess ||
        (e = cudaMalloc(&dp, sizeof(TcStepParams))) != cudaSuccess) {
      rc = fail(VFE_ENOMEM, "scratch allocation: %s", cudaGetErrorString(e));
      break;
    }
    TcStepParams p;
    memset(&p, 0, sizeof(p));
    p.trace_row = -1;
    p.shq = shq;
    p.F = F;
    if ((e = cudaMemcpy(dU, U.data(), ubytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(dout, 0, obytes)) != cudaSuccess ||
        (e = cudaMemcpy(dp, &p, sizeof(p), cudaMemcpyHostToDevice)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "upload: %s", cudaGetErrorString(e));
      break;
    }
    CUtensorMap tms;
    if ((rc = encode_state_tmap(m, encode_fn(), dU, &tms, true)) != VFE_OK) break;
    TcDevice ds = tc_stencil_device(m, m->cur);
    ds.params = dp;
    ds.partials_out = dout;
    if ((e = stencil_launch(m->stream, ds, &tms, TC_MODE_PARTIALS)) != cudaSuccess ||
        (e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "node-stencil partials: %s", cudaGetErrorString(e));
      break;
    }
    if ((rc = check_status(m)) != VFE_OK) break;
    std::vector<int64_t> P(obytes / sizeof(int64_t));
    if ((e = cudaMemcpy(P.data(), dout, obytes, cudaMemcpyDeviceToHost)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "download: %s", cudaGetErrorString(e));
      break;
    }
    for (int64_t n = 0; n < m->nn; ++n) {
      const int64_t t = tc_index(m, n);
      covered[n] = cov[n];
      for (int c = 0; c < 9; ++c) out[9 * n + c] = cov[n] ? P[c * m->comp + t] : 0;
    }
  } while (0);
  if (dU) cudaFree(dU);
  if (dout) cudaFree(dout);
  if (dp) cudaFree(dp);
  if (shift_out) *shift_out = shq;
  if (frac_bits_out) *frac_bits_out = F;
  return rc;
}

int vfe_debug_inject_status(vfe_mesh *m, int bits) {
  if (!m) return fail(VFE_EINVAL, "NULL mesh");
  if (bits & ~15) return fail(VFE_EINVAL, "status bits outside 1, 2, 4, 8");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  int st = 0;
  CUDA_TRY(cudaMemcpy(&st, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  st |= bits;
  CUDA_TRY(cudaMemcpy(m->d_status, &st, sizeof(int), cudaMemcpyHostToDevice));
  return VFE_OK;
}

int vfe_debug_tc_partials(vfe_mesh *m, const double *u, int n, const int64_t *ids, int64_t *out,
                          int *shift_out, int *frac_bits_out) {
  if (!m || !u || (n > 0 && (!ids || !out))) return fail(VFE_EINVAL, "NULL argument");
  if (m->opt.path != VFE_PATH_TC) return fail(VFE_ESTATE, "mesh is not on the tensor-core path");
  for (int q = 0; q < n; ++q)
    if (ids[q] < 0 || ids[q] >= m->ne) return fail(VFE_EINVAL, "element id %lld out of range",
                                                   (long long)ids[q]);
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  std::vector<int64_t> all;
  int shq = 0, F = 0;
  int rc = tc_apply(m, u, TC_MODE_PARTIALS, all, &shq, &F);
  if (rc != VFE_OK) return rc;
  for (int q = 0; q < n; ++q) memcpy(out + 48 * q, all.data() + 48 * ids[q], 48 * sizeof(int64_t));
  if (shift_out) *shift_out = shq;
  if (frac_bits_out) *frac_bits_out = F;
  return VFE_OK;
}

}  // extern "C"

// ---- batches: many meshes advanced by one launch per step -------------------

struct vfe_batch {
  std::vector<vfe_mesh *> meshes;
  std::vector<int64_t> gens;
  std::vector<int> base_cur;
  int device = 0, stages = 0, sms = 1;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int64_t steps = 0;  // steps taken since the arrays were built
  std::vector<int4> segs;
  std::vector<int32_t> seg_mesh, seg_off;
  // meshes grouped by digit stage count, one launch per group: its stage
  // count, its CTAs, and where its CTA offsets start in seg_off
  struct Group {
    int stages, n_ctas, off_base;
  };
  std::vector<Group> groups;
  int4 *d_segs = nullptr;
  int32_t *d_seg_mesh = nullptr, *d_seg_off = nullptr, *d_recv_off = nullptr;
  TcRecv *d_recv = nullptr;
  TcDevice *d_devs[2] = {nullptr, nullptr};
  CUtensorMap *d_maps[2] = {nullptr, nullptr};
  TcPrologueArgs *d_pro = nullptr;
  // meshes with the node-stencil kernel: their stencil runs go to one stencil
  // launch per mesh, split over a share of the SMs in proportion to the
  // mesh's planes, on side streams that run side by side with the batched
  // element kernel (the two touch disjoint nodes of each mesh)
  struct StencilPart {
    int mesh, n_ctas;
    int4 *d_segs;
    int32_t *d_off;
  };
  std::vector<StencilPart> st_parts;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_done;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};       // two steps from parity p
  cudaGraphExec_t graph_long[2] = {nullptr, nullptr};  // kLongSteps steps
};

static void batch_free_arrays(vfe_batch *b) {
  void *ptrs[] = {b->d_segs, b->d_seg_mesh, b->d_seg_off, b->d_recv_off, b->d_recv,
                  b->d_devs[0], b->d_devs[1], b->d_maps[0], b->d_maps[1], b->d_pro};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (vfe_batch::StencilPart &q : b->st_parts) {
    if (q.d_segs) cudaFree(q.d_segs);
    if (q.d_off) cudaFree(q.d_off);
  }
  b->st_parts.clear();
  b->d_segs = nullptr; b->d_seg_mesh = nullptr; b->d_seg_off = nullptr; b->d_recv_off = nullptr;
  b->d_recv = nullptr; b->d_devs[0] = b->d_devs[1] = nullptr; b->d_maps[0] = b->d_maps[1] = nullptr;
  b->d_pro = nullptr;
  for (int i = 0; i < 2; ++i) {
    if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
    b->graph[i] = nullptr;
    if (b->graph_long[i]) cudaGraphExecDestroy(b->graph_long[i]);
    b->graph_long[i] = nullptr;
  }
}

// (Re)build the partition, receivers and per-mesh argument arrays.
static int batch_build(vfe_batch *b) {
  batch_free_arrays(b);
  const int nm = (int)b->meshes.size();
  b->segs.clear();
  b->seg_mesh.clear();
  b->seg_off.clear();
  b->groups.clear();
  // per stage count (ascending), the element-kernel runs of its meshes (all
  // of a mesh's column-planes when it has no stencil kernel), split over the
  // SMs in the element kernel's cost model
  for (int st = 1; st <= TC_MAX_STAGES; ++st) {
    std::vector<int4> runs;
    std::vector<int32_t> run_mesh;
    for (int i = 0; i < nm; ++i) {
      const vfe_mesh *m = b->meshes[i];
      if (m->opt.stages != st) continue;
      if (m->stencil_on) {
        runs.insert(runs.end(), m->el_runs.begin(), m->el_runs.end());
        run_mesh.insert(run_mesh.end(), m->el_runs.size(), i);
      } else {
        for (int ty = 0; ty < m->tiles_y; ++ty)
          for (int tx = 0; tx < m->tiles_x; ++tx) {
            runs.push_back(make_int4(tx, ty, 0, m->nz + 1));
            run_mesh.push_back(i);
          }
      }
    }
    if (runs.empty()) continue;
    std::vector<int4> gsegs;
    std::vector<int32_t> gmesh, goff;
    split_runs(runs, &run_mesh, b->sms, 2.0, gsegs, &gmesh, goff);
    vfe_batch::Group grp;
    grp.stages = st;
    grp.n_ctas = (int)goff.size() - 1;
    grp.off_base = (int)b->seg_off.size();
    const int32_t base = (int32_t)b->segs.size();
    for (int32_t o : goff) b->seg_off.push_back(base + o);
    b->segs.insert(b->segs.end(), gsegs.begin(), gsegs.end());
    b->seg_mesh.insert(b->seg_mesh.end(), gmesh.begin(), gmesh.end());
    b->groups.push_back(grp);
  }
  // the stencil parts: each mesh's stencil runs over its share of the SMs
  {
    int64_t all = 0;
    for (int i = 0; i < nm; ++i)
      for (const int4 &r : b->meshes[i]->st_runs) all += r.w - r.z;
    for (int i = 0; i < nm && all > 0; ++i) {
      vfe_mesh *m = b->meshes[i];
      if (!m->stencil_on || m->st_runs.empty()) continue;
      int64_t planes = 0;
      for (const int4 &r : m->st_runs) planes += r.w - r.z;
      const int ctas = (int)std::max<int64_t>(
          1, std::min<int64_t>(b->sms, (planes * b->sms + all / 2) / all));
      std::vector<int4> psegs;
      std::vector<int32_t> poff;
      split_runs(m->st_runs, nullptr, ctas, 0.0, psegs, nullptr, poff, 2);
      vfe_batch::StencilPart q;
      q.mesh = i;
      q.n_ctas = (int)poff.size() - 1;
      q.d_segs = nullptr;
      q.d_off = nullptr;
      b->st_parts.push_back(q);
      vfe_batch::StencilPart &qq = b->st_parts.back();
      int rc;
      if ((rc = upload_vec(&qq.d_segs, psegs)) != VFE_OK) return rc;
      if ((rc = upload_vec(&qq.d_off, poff)) != VFE_OK) return rc;
    }
  }
  // receivers per batch segment (indices into each mesh's own trace rows)
  const int ns = (int)b->segs.size();
  std::vector<std::vector<TcRecv>> per(ns);
  for (int sg = 0; sg < ns; ++sg) {
    const vfe_mesh *m = b->meshes[b->seg_mesh[sg]];
    const int4 q = b->segs[sg];
    for (int r = 0; r < m->n_rec; ++r) {
      const int i = m->rec_ijk[3 * r], j = m->rec_ijk[3 * r + 1], k = m->rec_ijk[3 * r + 2];
      if (i / TC_OWN == q.x && j / TC_OWN == q.y && k >= q.z && k < q.w) {
        TcRecv v;
        v.ei = (int16_t)(i - TC_OWN * q.x);
        v.ej = (int16_t)(j - TC_OWN * q.y);
        v.k = k;
        v.r = r;
        v.pad = 0;
        per[sg].push_back(v);
      }
    }
    if ((int)per[sg].size() > TC_MAX_REC_CTA)
      return fail(VFE_EINVAL, "more than %d receivers in one node column segment", TC_MAX_REC_CTA);
  }
  std::vector<TcRecv> flat;
  std::vector<int32_t> roff(ns + 1, 0);
  for (int sg = 0; sg < ns; ++sg) {
    roff[sg] = (int32_t)flat.size();
    flat.insert(flat.end(), per[sg].begin(), per[sg].end());
  }
  roff[ns] = (int32_t)flat.size();
  // kernel arguments of each mesh for both buffer parities, and prologue args
  std::vector<TcDevice> devs[2];
  std::vector<CUtensorMap> maps[2];
  std::vector<TcPrologueArgs> pro(nm);
  b->gens.resize(nm);
  b->base_cur.resize(nm);
  for (int i = 0; i < nm; ++i) {
    vfe_mesh *m = b->meshes[i];
    b->gens[i] = m->gen;
    b->base_cur[i] = m->cur;
    for (int p = 0; p < 2; ++p) {
      const int cur = m->cur ^ p;
      devs[p].push_back(tc_device(m, cur));
      maps[p].push_back(m->tmap[cur]);
    }
    TcPrologueArgs &A = pro[i];
    memset(&A, 0, sizeof(A));
    A.params = m->d_tcparams;
    A.persist = m->d_tcpersist;
    A.or_slots = m->d_or;
    A.status = m->d_status;
    A.amp_scale = m->amp * m->src_scale;
    A.dt = m->dt;
    A.f0 = m->f0;
    A.t0 = m->t0;
    for (int c = 0; c < 3; ++c) A.dir[c] = m->src_dir[c];
    A.ncols = m->tiles_x * m->tiles_y;
    A.have_src = m->has_src ? 1 : 0;
    A.trace_on = m->n_rec > 0 ? 1 : 0;
    A.n_inj = 3 * m->n_rec;
    A.inj = m->d_inj;
  }
  CUDA_TRY(cudaMalloc(&b->d_segs, sizeof(int4) * ns));
  CUDA_TRY(cudaMalloc(&b->d_seg_mesh, sizeof(int32_t) * ns));
  CUDA_TRY(cudaMalloc(&b->d_seg_off, sizeof(int32_t) * b->seg_off.size()));
  CUDA_TRY(cudaMalloc(&b->d_recv, sizeof(TcRecv) * std::max<size_t>(flat.size(), 1)));
  CUDA_TRY(cudaMalloc(&b->d_recv_off, sizeof(int32_t) * roff.size()));
  CUDA_TRY(cudaMalloc(&b->d_pro, sizeof(TcPrologueArgs) * nm));
  CUDA_TRY(cudaMemcpy(b->d_segs, b->segs.data(), sizeof(int4) * ns, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_seg_mesh, b->seg_mesh.data(), sizeof(int32_t) * ns,
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_seg_off, b->seg_off.data(), sizeof(int32_t) * b->seg_off.size(),
                      cudaMemcpyHostToDevice));
  if (!flat.empty())
    CUDA_TRY(cudaMemcpy(b->d_recv, flat.data(), sizeof(TcRecv) * flat.size(),
                        cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_recv_off, roff.data(), sizeof(int32_t) * roff.size(),
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_pro, pro.data(), sizeof(TcPrologueArgs) * nm, cudaMemcpyHostToDevice));
  for (int p = 0; p < 2; ++p) {
    CUDA_TRY(cudaMalloc(&b->d_devs[p], sizeof(TcDevice) * nm));
    CUDA_TRY(cudaMalloc(&b->d_maps[p], sizeof(CUtensorMap) * nm));  // cudaMalloc: 256-B aligned
    CUDA_TRY(cudaMemcpy(b->d_devs[p], devs[p].data(), sizeof(TcDevice) * nm,
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b->d_maps[p], maps[p].data(), sizeof(CUtensorMap) * nm,
                        cudaMemcpyHostToDevice));
  }
  b->steps = 0;
  return VFE_OK;
}

static TcBatch batch_args(const vfe_batch *b, int parity, const vfe_batch::Group &g) {
  TcBatch a;
  a.devs = b->d_devs[parity];
  a.maps = b->d_maps[parity];
  a.segs = b->d_segs;
  a.seg_mesh = b->d_seg_mesh;
  a.seg_off = b->d_seg_off + g.off_base;
  a.recv = b->d_recv;
  a.recv_off = b->d_recv_off;
  a.n_ctas = g.n_ctas;
  return a;
}

// one step of every mesh: the prologues, then one fused launch per group of
// meshes with the same digit stage count
static int batch_enqueue(vfe_batch *b, int parity) {
  CUDA_TRY(tc_launch_batch_prologue(b->stream, b->d_pro, (int)b->meshes.size()));
  const int ns = (int)b->side.size();
  if (!b->st_parts.empty()) {
    CUDA_TRY(cudaEventRecord(b->fork, b->stream));
    for (int k = 0; k < ns; ++k) CUDA_TRY(cudaStreamWaitEvent(b->side[k], b->fork, 0));
    for (size_t k = 0; k < b->st_parts.size(); ++k) {
      const vfe_batch::StencilPart &q = b->st_parts[k];
      vfe_mesh *m = b->meshes[q.mesh];
      const int cur = b->base_cur[q.mesh] ^ parity;
      TcDevice d = tc_stencil_device(m, cur);
      d.segs = q.d_segs;
      d.seg_off = q.d_off;
      d.n_ctas = q.n_ctas;
      CUDA_TRY(stencil_launch_ex(b->side[k % ns], d, &m->st_tmap[cur], TC_MODE_STEP, false));
      CUDA_TRY(stencil_fix(b->side[k % ns], d, TC_MODE_STEP));
    }
  }
  for (const vfe_batch::Group &g : b->groups)
    if (g.n_ctas > 0) CUDA_TRY(tc_launch_batch_step(b->stream, batch_args(b, parity, g), g.stages));
  if (!b->st_parts.empty())
    for (int k = 0; k < ns; ++k) {
      CUDA_TRY(cudaEventRecord(b->side_done[k], b->side[k]));
      CUDA_TRY(cudaStreamWaitEvent(b->stream, b->side_done[k], 0));
    }
  return VFE_OK;
}

extern "C" {

int vfe_create_batch(int n, vfe_mesh *const *meshes, vfe_batch **out) {
  if (!out) return fail(VFE_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !meshes) return fail(VFE_EINVAL, "need at least one mesh");
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) return fail(VFE_EINVAL, "mesh %d is NULL", i);
    if (meshes[i]->opt.path != VFE_PATH_TC)
      return fail(VFE_EINVAL, "mesh %d is not on the tensor-core path", i);
    if (meshes[i]->device != meshes[0]->device)
      return fail(VFE_EINVAL, "mesh %d is on another device", i);
    if (meshes[i]->damped)
      return fail(VFE_EINVAL, "mesh %d is damped: batches step undamped meshes only", i);
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) return fail(VFE_EINVAL, "mesh %d appears twice", i);
  }
  vfe_batch *b = new vfe_batch();
  b->meshes.assign(meshes, meshes + n);
  b->device = meshes[0]->device;
  b->stages = meshes[0]->opt.stages;
  b->sms = meshes[0]->sms;
  int rc = VFE_OK;
  cudaSetDevice(b->device);
  bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  const int nside = std::min(n, 128);  // one side stream per mesh: the stencil launches run side by side
  for (int k = 0; k < nside && ok; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->side.push_back(s);
    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->side_done.push_back(e);
  }
  if (!ok) {
    rc = fail(VFE_ECUDA, "batch stream/event creation failed");
  } else {
    for (vfe_mesh *m : b->meshes)
      if (cudaStreamSynchronize(m->stream) != cudaSuccess) rc = fail(VFE_ECUDA, "mesh stream");
    if (rc == VFE_OK) rc = batch_build(b);
  }
  if (rc != VFE_OK) {
    std::string msg = g_last_error;
    vfe_destroy_batch(b);
    g_last_error = msg;
    return rc;
  }
  *out = b;
  return VFE_OK;
}

int vfe_destroy_batch(vfe_batch *b) {
  if (!b) return VFE_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (cudaStream_t s : b->side) cudaStreamSynchronize(s);
  batch_free_arrays(b);
  if (b->done) cudaEventDestroy(b->done);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->side_done) cudaEventDestroy(e);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return VFE_OK;
}

int vfe_batch_step(vfe_batch *b, int n) {
  if (!b) return fail(VFE_EINVAL, "batch is NULL");
  if (n < 0) return fail(VFE_EINVAL, "n must be >= 0");
  if (n == 0) return VFE_OK;
  cudaSetDevice(b->device);
  // earlier work queued on the meshes' own streams comes first
  for (vfe_mesh *m : b->meshes) {
    CUDA_TRY(cudaEventRecord(b->done, m->stream));
    CUDA_TRY(cudaStreamWaitEvent(b->stream, b->done, 0));
  }
  bool rebuild = false;
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    vfe_mesh *m = b->meshes[i];
    int rc = ensure_trace_capacity(m, m->trace_rows + n);
    if (rc != VFE_OK) return rc;
    if (m->gen != b->gens[i] || m->cur != (b->base_cur[i] ^ (int)(b->steps & 1))) rebuild = true;
  }
  if (rebuild) {
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    int rc = batch_build(b);
    if (rc != VFE_OK) return rc;
  }
  // runs of steps replay captured graphs of kLongSteps, then of 2 steps
  auto capture = [&](int parity, int len, cudaGraphExec_t *out) -> int {
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = VFE_OK;
    for (int k = 0; k < len && rc == VFE_OK; ++k) rc = batch_enqueue(b, parity ^ (k & 1));
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != VFE_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(VFE_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(VFE_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    return VFE_OK;
  };
  int64_t left = n;
  while (left >= kLongSteps) {
    const int parity = (int)(b->steps & 1);
    if (!b->graph_long[parity]) {
      const int rc = capture(parity, kLongSteps, &b->graph_long[parity]);
      if (rc != VFE_OK) return rc;
    }
    CUDA_TRY(cudaGraphLaunch(b->graph_long[parity], b->stream));
    b->steps += kLongSteps;
    left -= kLongSteps;
  }
  while (left >= 2) {
    const int parity = (int)(b->steps & 1);
    if (!b->graph[parity]) {
      const int rc = capture(parity, 2, &b->graph[parity]);
      if (rc != VFE_OK) return rc;
    }
    CUDA_TRY(cudaGraphLaunch(b->graph[parity], b->stream));
    b->steps += 2;
    left -= 2;
  }
  if (left == 1) {
    int rc = batch_enqueue(b, (int)(b->steps & 1));
    if (rc != VFE_OK) return rc;
    b->steps += 1;
  }
  for (vfe_mesh *m : b->meshes) {
    if (n & 1) m->cur = 1 - m->cur;
    m->steps += n;
    if (m->n_rec) m->trace_rows += n;
  }
  // later work on the meshes' own streams (traces, state) waits for the batch
  CUDA_TRY(cudaEventRecord(b->done, b->stream));
  for (vfe_mesh *m : b->meshes) CUDA_TRY(cudaStreamWaitEvent(m->stream, b->done, 0));
  return VFE_OK;
}

int vfe_batch_synchronize(vfe_batch *b) {
  if (!b) return fail(VFE_EINVAL, "batch is NULL");
  cudaSetDevice(b->device);
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (vfe_mesh *m : b->meshes) {
    int rc = check_status(m);
    if (rc != VFE_OK) return rc;
  }
  return VFE_OK;
}

}  // extern "C"

// ---- adjoint-state gradient of the receiver misfit ----------------------------

namespace {

struct Snapshot {  // a mesh's time-stepping state at one step
  void *a = nullptr, *b = nullptr;  // u^n, u^{n-1} buffers
  int64_t persist[8] = {0};
  std::vector<unsigned long long> slots;
  int cur = 0;
  int64_t steps = 0, trace_rows = 0;
};

size_t state_bytes(const vfe_mesh *m) {
  return m->opt.path == VFE_PATH_TC ? sizeof(int64_t) * 3 * m->comp : sizeof(double) * 3 * m->nn;
}

void *state_buf(vfe_mesh *m, int which) {
  return m->opt.path == VFE_PATH_TC ? (void *)m->d_U[which] : (void *)m->d_u[which];
}

int64_t *persist_ptr(vfe_mesh *m) {
  return m->opt.path == VFE_PATH_TC ? m->d_tcpersist : m->d_f64persist;
}

int persist_len(const vfe_mesh *m) { return m->opt.path == VFE_PATH_TC ? 8 : 6; }

size_t slot_words(const vfe_mesh *m) { return 3 * (1 + (size_t)m->tiles_x * m->tiles_y); }

int snap_save(vfe_mesh *m, Snapshot &s) {
  const size_t sb = state_bytes(m);
  if (!s.a) {
    if (cudaMalloc(&s.a, sb) != cudaSuccess || cudaMalloc(&s.b, sb) != cudaSuccess)
      return fail(VFE_ENOMEM, "checkpoint of %zu bytes", 2 * sb);
  }
  CUDA_TRY(cudaMemcpyAsync(s.a, state_buf(m, m->cur), sb, cudaMemcpyDeviceToDevice, m->stream));
  CUDA_TRY(cudaMemcpyAsync(s.b, state_buf(m, 1 - m->cur), sb, cudaMemcpyDeviceToDevice, m->stream));
  CUDA_TRY(cudaMemcpyAsync(s.persist, persist_ptr(m), sizeof(int64_t) * persist_len(m),
                           cudaMemcpyDeviceToHost, m->stream));
  if (m->opt.path == VFE_PATH_TC) {
    s.slots.resize(slot_words(m));
    CUDA_TRY(cudaMemcpyAsync(s.slots.data(), m->d_or, sizeof(unsigned long long) * s.slots.size(),
                             cudaMemcpyDeviceToHost, m->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  s.cur = m->cur;
  s.steps = m->steps;
  s.trace_rows = m->trace_rows;
  return VFE_OK;
}

int snap_restore(vfe_mesh *m, const Snapshot &s) {
  const size_t sb = state_bytes(m);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->cur = s.cur;
  CUDA_TRY(cudaMemcpyAsync(state_buf(m, m->cur), s.a, sb, cudaMemcpyDeviceToDevice, m->stream));
  CUDA_TRY(cudaMemcpyAsync(state_buf(m, 1 - m->cur), s.b, sb, cudaMemcpyDeviceToDevice, m->stream));
  CUDA_TRY(cudaMemcpyAsync(persist_ptr(m), s.persist, sizeof(int64_t) * persist_len(m),
                           cudaMemcpyHostToDevice, m->stream));
  if (m->opt.path == VFE_PATH_TC)
    CUDA_TRY(cudaMemcpyAsync(m->d_or, s.slots.data(), sizeof(unsigned long long) * s.slots.size(),
                             cudaMemcpyHostToDevice, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->steps = s.steps;
  m->trace_rows = s.trace_rows;
  return VFE_OK;
}

void snap_free(Snapshot &s) {
  if (s.a) cudaFree(s.a);
  if (s.b) cudaFree(s.b);
  s.a = s.b = nullptr;
}

// back to rest at step 0 with empty traces; the injection stays off
int rewind_mesh(vfe_mesh *m) {
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  const size_t sb = state_bytes(m);
  CUDA_TRY(cudaMemset(state_buf(m, 0), 0, sb));
  CUDA_TRY(cudaMemset(state_buf(m, 1), 0, sb));
  if (m->opt.path == VFE_PATH_TC) {
    const int64_t p[8] = {0, 0, 0, 0, (int64_t)(m->eC + m->e_ref), 0, -1, -1};
    CUDA_TRY(cudaMemcpy(m->d_tcpersist, p, sizeof(p), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(m->d_or, 0, sizeof(unsigned long long) * slot_words(m)));
  } else {
    const int64_t p[6] = {0, 0, -1, 0, -1, 0};
    CUDA_TRY(cudaMemcpy(m->d_f64persist, p, sizeof(p), cudaMemcpyHostToDevice));
  }
  m->cur = 0;
  m->steps = 0;
  m->trace_rows = 0;
  return VFE_OK;
}

// per-step increments at the receivers from the mesh's current step on
int set_injection(vfe_mesh *m, const double *host, int64_t rows) {
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (m->d_inj) cudaFree(m->d_inj);
  m->d_inj = nullptr;
  const size_t bytes = sizeof(double) * 3 * (size_t)m->n_rec * rows;
  if (cudaMalloc(&m->d_inj, bytes) != cudaSuccess) return fail(VFE_ENOMEM, "injection array");
  CUDA_TRY(cudaMemcpy(m->d_inj, host, bytes, cudaMemcpyHostToDevice));
  const int64_t base = m->steps;
  CUDA_TRY(cudaMemcpy(persist_ptr(m) + (m->opt.path == VFE_PATH_TC ? 6 : 2), &base,
                      sizeof(int64_t), cudaMemcpyHostToDevice));
  invalidate_graphs(m);
  return VFE_OK;
}

// u^n of the mesh as FP64 [nn][3] on the device
int state_to_f64(vfe_mesh *m, double *dst) {
  if (m->opt.path == VFE_PATH_TC) {
    CUDA_TRY(tc_state_to_f64(m->stream, m->d_U[m->cur], m->d_tcpersist, 0, m->nx, m->ny, m->nn,
                             m->nxp, m->plane, m->comp, dst));
  } else {
    CUDA_TRY(cudaMemcpyAsync(dst, m->d_u[m->cur], sizeof(double) * 3 * m->nn,
                             cudaMemcpyDeviceToDevice, m->stream));
  }
  return VFE_OK;
}

}  // namespace

extern "C" {

int vfe_misfit_gradient(vfe_mesh *m, int nsteps, const double *data, int checkpoint_every,
                        double *grad_G, double *misfit_out) {
  if (!m || !data || !grad_G) return fail(VFE_EINVAL, "NULL argument");
  if (nsteps < 1 || checkpoint_every < 1) return fail(VFE_EINVAL, "need nsteps, checkpoint >= 1");
  if (m->n_rec < 1) return fail(VFE_ESTATE, "the misfit needs receivers");
  if (m->damped) return fail(VFE_ESTATE, "the misfit gradient supports undamped meshes only");
  cudaSetDevice(m->device);
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  const int N = nsteps, C = checkpoint_every, nr = m->n_rec;
  const int nb = (N + C - 1) / C;
  vfe_mesh *adj = nullptr;
  std::vector<Snapshot> snaps(nb);
  double *d_block = nullptr, *d_mu = nullptr, *d_grad = nullptr;
  // tensor-core path: the recomputed forward states stay in fixed point, with
  // the exponent of each step
  void *d_ublock = nullptr;
  int64_t *d_uexp = nullptr;
  const bool tc = m->opt.path == VFE_PATH_TC;
  int rc = VFE_OK;
  do {
    // the adjoint runs on a twin mesh: same geometry, materials, dt and path,
    // no source, the forward receivers as injection points
    vfe_options o = m->opt;
    o.dt = m->dt;
    o.stream = m->stream;
    if ((rc = vfe_create_mesh(m->nx, m->ny, m->nz, m->h, m->mat.data(), m->table.data(),
                              m->n_mat, &o, &adj)) != VFE_OK)
      break;
    if ((rc = vfe_set_receivers(adj, nr, m->rec_ijk.data())) != VFE_OK) break;
    if (m->elem_g && (rc = vfe_set_shear_moduli(adj, m->elem_G.data())) != VFE_OK) break;
    // forward from rest with checkpoints every C steps
    if ((rc = rewind_mesh(m)) != VFE_OK) break;
    if ((rc = ensure_trace_capacity(m, N)) != VFE_OK) break;
    for (int b = 0; b < nb && rc == VFE_OK; ++b) {
      if ((rc = snap_save(m, snaps[b])) != VFE_OK) break;
      rc = vfe_step(m, std::min(C, N - b * C));
    }
    if (rc != VFE_OK) break;
    std::vector<double> tr((size_t)N * nr * 3);
    int64_t rows = 0;
    if ((rc = vfe_get_traces(m, tr.data(), &rows)) != VFE_OK) break;
    // misfit and the adjoint source -M^-1 dJ/du^m, m = N - k for adjoint step k
    double J = 0.0;
    std::vector<double> inj((size_t)N * nr * 3, 0.0);
    for (int n = 0; n < N; ++n)
      for (int r = 0; r < nr; ++r) {
        const int64_t node = m->rec_nodes[r];
        for (int c = 0; c < 3; ++c) {
          const size_t q = ((size_t)n * nr + r) * 3 + c;
          const double res = tr[q] - data[q];
          J += 0.5 * res * res;
          const int k = N - 1 - n;  // residual of u^{n+1} drives mu^n: adjoint step k
          if (!m->fixed[node]) inj[((size_t)k * nr + r) * 3 + c] = -res / m->mass[node];
        }
      }
    if (misfit_out) *misfit_out = J;
    if ((rc = rewind_mesh(adj)) != VFE_OK) break;
    if ((rc = set_injection(adj, inj.data(), N)) != VFE_OK) break;
    // dK_e/dG at fixed kappa comes from the element's closed form (alpha)
    const double alpha = m->opt.element_kind == VFE_OVFEM ? 0.75 : 1.0 / 3.0;
    const size_t fb = sizeof(double) * 3 * m->nn;
    const size_t sb = state_bytes(m);
    cudaError_t e;
    if (tc && (adj->nxp != m->nxp || adj->plane != m->plane || adj->comp != m->comp)) {
      rc = fail(VFE_EINVAL, "internal: adjoint twin has another state layout");
      break;
    }
    if ((tc ? ((e = cudaMalloc(&d_ublock, sb * (C + 1))) != cudaSuccess ||
               (e = cudaMalloc((void **)&d_uexp, sizeof(int64_t) * (C + 1))) != cudaSuccess)
            : ((e = cudaMalloc(&d_block, fb * (C + 1))) != cudaSuccess ||
               (e = cudaMalloc(&d_mu, fb)) != cudaSuccess)) ||
        (e = cudaMalloc(&d_grad, sizeof(double) * m->ne)) != cudaSuccess) {
      rc = fail(VFE_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(e));
      break;
    }
    // u^n of the forward run into block slot j (fixed point and its exponent
    // on the tensor-core path, FP64 otherwise)
    auto keep_state = [&](int j) -> int {
      if (!tc) return state_to_f64(m, d_block + (size_t)j * 3 * m->nn);
      CUDA_TRY(cudaMemcpyAsync((char *)d_ublock + sb * j, m->d_U[m->cur], sb,
                               cudaMemcpyDeviceToDevice, m->stream));
      CUDA_TRY(cudaMemcpyAsync(d_uexp + j, m->d_tcpersist, sizeof(int64_t),
                               cudaMemcpyDeviceToDevice, m->stream));
      return VFE_OK;
    };
    if ((e = cudaMemset(d_grad, 0, sizeof(double) * m->ne)) != cudaSuccess) {
      rc = fail(VFE_ECUDA, "gradient buffer: %s", cudaGetErrorString(e));
      break;
    }
    // backward over the blocks: recompute u^{s0..s0+len}, then adjoint steps
    for (int b = nb - 1; b >= 0 && rc == VFE_OK; --b) {
      const int s0 = b * C, len = std::min(C, N - s0);
      if ((rc = snap_restore(m, snaps[b])) != VFE_OK) break;
      if ((rc = keep_state(0)) != VFE_OK) break;
      for (int j = 1; j <= len && rc == VFE_OK; ++j) {
        if ((rc = vfe_step(m, 1)) != VFE_OK) break;
        rc = keep_state(j);
      }
      for (int mi = s0 + len; mi >= s0 + 1 && rc == VFE_OK; --mi) {
        if ((rc = vfe_step(adj, 1)) != VFE_OK) break;  // mu^{mi-1}
        const int j = mi - 1 - s0;
        cudaError_t ge;
        if (tc) {
          // straight from the two fixed-point states (same stream)
          ge = grad_g_tc_accumulate(m->stream, m->nx, m->ny, m->nz, m->d_mat, m->h,
                                    (const int64_t *)((char *)d_ublock + sb * j), d_uexp + j,
                                    adj->d_U[adj->cur], adj->d_tcpersist, m->nxp, m->plane,
                                    m->comp, m->dt * m->dt, d_grad);
        } else {
          if ((rc = state_to_f64(adj, d_mu)) != VFE_OK) break;
          ge = grad_g_accumulate(m->stream, m->nx, m->ny, m->nz, m->d_mat, alpha, m->h,
                                 d_block + (size_t)j * 3 * m->nn, d_mu, m->dt * m->dt, d_grad);
        }
        if (ge != cudaSuccess) rc = fail(VFE_ECUDA, "gradient kernel: %s", cudaGetErrorString(ge));
      }
    }
    if (rc != VFE_OK) break;
    if ((rc = vfe_synchronize(adj)) != VFE_OK) break;
    if ((e = cudaMemcpy(grad_G, d_grad, sizeof(double) * m->ne, cudaMemcpyDeviceToHost)) !=
        cudaSuccess) {
      rc = fail(VFE_ECUDA, "gradient read-back: %s", cudaGetErrorString(e));
      break;
    }
    rc = rewind_mesh(m);
  } while (0);
  std::string msg = g_last_error;
  for (auto &s : snaps) snap_free(s);
  if (d_block) cudaFree(d_block);
  if (d_mu) cudaFree(d_mu);
  if (d_ublock) cudaFree(d_ublock);
  if (d_uexp) cudaFree(d_uexp);
  if (d_grad) cudaFree(d_grad);
  if (adj) vfe_destroy(adj);
  g_last_error = msg;
  return rc;
}

}  // extern "C"
