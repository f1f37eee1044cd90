// vfe_internal.h -- structures shared by the host code and the kernels of the
// GB300 voxel FE wave solver.  Not part of the public ABI (see include/vfe.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vfe.h"

// ----------------------------------------------------------------------------
// TC path geometry.  A CTA owns a column of TC_OWN x TC_OWN nodes in x-y and a
// chunk of node planes in z, and computes the (TC_OWN+1)^2 = 256 elements per
// layer that touch its nodes (one element of halo on the low x and y sides).
// The 256 elements form two MMA tiles of M = 128 rows.
// ----------------------------------------------------------------------------
#define TC_EX 16                 // elements per layer tile in x and in y
#define TC_OWN (TC_EX - 1)       // owned nodes per tile in x and in y
#define TC_NODES (TC_EX + 1)     // node rows/columns touched by the tile
#define TC_BOXX 18               // TMA box width in x (int64; 144 B)
#define TC_MAX_STAGES 5          // 11-bit digit stages (5 x 11 = 55 bits)
#define TC_DIGIT_BITS 11
#define TC_QBITS 51              // |q| < 2^51 after the per-step shift
#define TC_N 48                  // MMA N: 24 K^kappa rows + 24 K^G' rows
#define TC_THREADS 512          // two threads per element: corner groups dz = 0 / 1
#define TC_MAX_MAT 64            // materials per mesh on the TC path
#define TC_MAX_REC_CTA 64        // receivers handled per CTA work item
#define ST_BOXX 20               // stencil kernel: TMA box width in x (int64; 160 B)
#define ST_BOXY 18               // stencil kernel: node rows per box
// the node-stencil kernel's operand buffer: 9 B images of 2560 bytes, then
// the correction table: per octant mask (256 x int16 pairs: first row, rows)
// and ST_MASK_ROWS rows of 20 int16 (neighbour offset, 3x3 K^kappa block,
// 3x3 Kbar^G block, zero) summed over the mask's elements
#define ST_MASK_ROWS 5023
#define ST_MASK_IDX_OFF (9 * 2560)
#define ST_MASK_ROW_OFF (ST_MASK_IDX_OFF + 256 * 2 * 2)
#define ST_BST_BYTES (ST_MASK_ROW_OFF + ST_MASK_ROWS * 20 * 2)
// meshes of at least this many elements give every column-plane but the
// source and receiver planes to the stencil kernel, with per-node material
// and a correction launch for the nodes whose eight elements are not all of
// that material (material and void interfaces, the mesh faces); smaller
// meshes give it the uniform runs alone
#define ST_FIX_MIN_ELEMENTS (8LL << 20)
// per-node reference material of the stencil kernel: a material index, or
// ST_NO_MAT (no solid element; the material table's zero entry)
#define ST_NO_MAT TC_MAX_MAT
// correction entry (i, j, k, code): code bits 0-7 the octant mask of the
// elements to correct (bit o: element origin (i - (o & 1), j - (o >> 1 & 1),
// k - (o >> 2))), 8-15 their material (ST_NO_MAT: absent), 16-23 the
// node's reference material, bit 24 set when the entry continues the
// previous entry's node
#define ST_FIX_CONT (1 << 24)
#define TC_UNITS_BITS 59         // target bit length of max |U| after rescale
                                 // (a step's growth keeps |U| below 2^62)

// fp32 magic bias: 8 padding K-rows carry A = 128, B = 12288 so that every
// accumulator starts from 1.5 * 2^23; its bit pattern is then 0x4B400000 + d
// for the exact integer d (|d| < 2^22).
#define TC_MAGIC_A 128.0f
#define TC_MAGIC_B 12288.0f
#define TC_MAGIC_BITS 0x4B400000

struct TcStepParams {     // written by the per-step prologue kernel
  int64_t step;           // global step index n (source time n*dt)
  int64_t trace_row;      // row of the trace buffer for this step (-1: none)
  int64_t inj_row;        // row of the injection array for this step (-1: none)
  int64_t dU_src[3];      // source increment in the new fixed-point units
  int rs;                 // rescale: U_new units = old units * 2^rs
  int shq;                // digit shift: q = U_raw >> shq
  int R;                  // right shift of S*C (128-bit) giving dU
  int F;                  // fraction bits after this step (u = U * 2^-F)
  int or_slot;            // slot this step ORs |U_new| into
  int rs_prev;            // shift of the previous step: u^{n-1} is stored in
                          // units 2^-(F_old + rs_prev)
  int eCref;              // eC + e_ref (exponent bookkeeping for R)
  int pad;
};

struct TcMaterial {       // per-material integer multipliers, mesh-wide unit
  int64_t A;              // round(kappa ds/256 * 2^e_ref) < 2^61
  int64_t B;              // round(G ds/384 * 2^e_ref)
  int shift;              // unused (0)
  int pad;
};

struct TcRecv {           // receiver handled by a CTA work item
  int16_t ei, ej;         // owning thread's element coordinates in the tile
  int32_t k;              // node plane
  int32_t r;              // receiver index
  int32_t pad;
};

struct TcDevice {         // everything the TC kernels read (by value)
  int nx, ny, nz, nxp;    // nxp: padded x pitch of nodal arrays (multiple of 4)
  int n_ctas;             // one CTA per SM; CTA b owns segments seg_off[b..b+1)
  int n_mat, stages, n_rec;
  int64_t plane;          // nxp*(ny+1): nodal plane stride
  int64_t comp;           // plane*(nz+1): component stride
  const int32_t *mat;     // element material ids (x fastest)
  const int64_t *C;       // per-node update multiplier round(dt^2/m 2^eC)
  const int64_t *U_prev;  // u^{n-1} (also receives u^{n+1})
  int64_t *U_next;        // same buffer as U_prev
  const uint16_t *Bop;    // B operand image (fp16 bits), 48x32, core-matrix order
  const TcMaterial *mats;
  const int4 *segs;       // (tile x, tile y, first owned plane, end plane)
  const int32_t *seg_off; // CTA -> first segment, size n_ctas+1
  const TcRecv *recv;     // receivers, grouped per segment
  const int32_t *recv_off;// segment -> first receiver, size n_segs+1
  int64_t src_node;       // -1: none
  double *traces;         // [rows][n_rec][3]
  unsigned long long *or_slots;  // 3 slots x (1 + tiles_x*tiles_y): OR(|U|), global
                                 // then per 15x15 node column
  int tiles_x, tiles_y;
  int *status;            // device error flags (bit 0: wait timeout)
  const TcStepParams *params;
  const double *inj;      // [rows][n_rec][3] displacement increments at the receivers
  int64_t *S_out;         // K u mode: per-node S (int64 x 3, SoA like U)
  int64_t *partials_out;  // partials mode: per element 48 int64 (element order)
  // Rayleigh damping (damped != 0; the TMA map then covers W = w^n instead of
  // u^n, see F64Device): u^n of the updated node comes from U_cur, and with
  // g = 1 / (1 + a) folded into C and the source,
  //   u^{n+1} = 2 g u^n - (1 - a) g u^{n-1} - C S,  w^{n+1} = u^{n+1} + b (u^{n+1} - u^n),
  // using the fixed-point constants dG = round(g 2^62),
  // dH = round((1 - a) g 2^62), dB = round(b 2^62)
  const int64_t *U_cur;
  int64_t *W_next;
  int64_t dG, dH, dB;
  int damped;
  // node-stencil kernel (vfe_stencil.cu): its own segments and operand
  // buffer (B images, then the correction table), the reference material of
  // every node of its runs (mats[] has TC_MAX_MAT + 1 entries, zero beyond
  // n_mat); U_cur above holds u^n for the corrections
  const uint16_t *Bst;
  const uint8_t *node_mat;
  // the correction entries of the stencil runs' nodes (stencil_fix, after
  // the kernel)
  const int4 *fix;
  int n_fix;
  // per-element shear modulus (vfe_set_shear_moduli): the element kernel's
  // G multiplier round(G_e ds/384 2^e_ref) per element, or nullptr
  const int64_t *elem_B;
};

// Several meshes advanced by one launch: each segment belongs to one mesh,
// whose kernel arguments and tensor map live in global memory.
struct TcBatch {
  const TcDevice *devs;       // per mesh; nullptr for a single-mesh launch
  const CUtensorMap *maps;    // per mesh (64-byte aligned)
  const int4 *segs;           // (tile x, tile y, z0, z1) of every segment
  const int32_t *seg_mesh;    // mesh of each segment
  const int32_t *seg_off;     // CTA -> first segment, size n_ctas+1
  const TcRecv *recv;         // receivers grouped per batch segment
  const int32_t *recv_off;    // segment -> first receiver
  int n_ctas;
};

struct TcPrologueArgs {       // one mesh's inputs to the per-step prologue
  TcStepParams *params;
  int64_t *persist;
  unsigned long long *or_slots;
  int *status;
  double amp_scale, dt, f0, t0;
  double dir[3];
  int ncols, have_src, trace_on, n_inj;  // n_inj: values per injection row (3 n_rec)
  const double *inj;                     // injection array (see TcDevice::inj)
  const double *force;                   // explicit force rows [k][3] (see TcSource)
  double force_scale;
  int64_t force_rows;
};

// FP64 path ------------------------------------------------------------------
#define F64_MAX_MAT 24    // element matrices kept in shared memory

struct F64Device {
  int nx, ny, nz, n_mat, n_rec;
  int64_t nn;
  const int32_t *mat;
  const double *K;        // n_mat * 576 element matrices
  const double *u;        // u^n [nn][3]
  const double *u_prev;   // u^{n-1}
  double *u_next;         // u^{n+1}
  const double *dt2_m;    // dt^2 / m per node, 0 for fixed / massless nodes
  const int64_t *recv_nodes;
  double *traces;
  int64_t src_node;
  double *f_out;          // K u mode output
  const double *inj;      // [rows][n_rec][3] displacement increments at the receivers
  // Rayleigh damping (damped != 0): K acts on w^n = u^n + b (u^n - u^{n-1});
  // (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1} + dt^2/m (F - K w^n)
  // per-element shear modulus (elem_G != nullptr): K_e = kappa_m Kk + G_e Kg
  // with Kk = K_e(kappa = 1, G = 0), Kg = K_e(kappa = 0, G = 1) of the element kind
  const double *elem_G;   // per element
  const double *kappa;    // per material
  const double *Kkg;      // Kk then Kg (2 x 576)
  const double *w;        // w^n [nn][3]
  double *w_next;         // w^{n+1}
  double da, db;          // a = alpha dt / 2, b = beta / dt
  int damped;
};

// Ricker point source (Section 3 applies an impulse force in z):
// F(t) = amp_scale * (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2) * dir,
// evaluated by the per-step prologue at t = n dt.  amp_scale is amp on the
// FP64 path and amp * dt^2 / m(source node) on the TC path.  While an explicit
// force series is active (persist slot "first step" >= 0), step n takes
// F^n = force[n - first][0..2] instead (force holds force_rows rows), scaled by
// force_scale (1 on the FP64 path, dt^2 / m(source node) on the TC path).
struct TcSource {
  double amp_scale, dt, f0, t0;
  double dir[3];
  const double *force;
  double force_scale;
  int64_t force_rows;
};

__device__ __forceinline__ double ricker_wavelet(double t, double f0, double t0) {
  const double a = 9.869604401089358 * f0 * f0 * (t - t0) * (t - t0);  // pi^2 f0^2 (t-t0)^2
  return (1.0 - 2.0 * a) * exp(-a);
}

// read-only view of a mesh for code outside vfe_api.cu ------------------------
struct VfeMeshView {
  int nx, ny, nz, nxp, nyp;
  int64_t nn, plane, comp;
  int e_ref;
  int device;
  int tc;                 // 1 on the tensor-core path
  cudaStream_t stream;
  TcDevice dev;           // kernel arguments with the mesh's own pointers
  int stencil_on;         // the node-stencil kernel takes the stencil runs
  TcDevice st;            // its arguments (segments, materials, B image)
};
int vfe_mesh_view(vfe_mesh *mesh, VfeMeshView *view);
void vfe_set_last_error(const char *msg);  // message returned by vfe_last_error()
// tensor map of a padded SoA int64 nodal array laid out like the state
CUresult vfe_encode_state_map(CUtensorMap *map, void *base, const VfeMeshView &v,
                              bool stencil_box = false);

// launch helpers implemented in the .cu files ---------------------------------
enum { TC_MODE_STEP = 0, TC_MODE_KU = 1, TC_MODE_PARTIALS = 2 };
int tc_smem_bytes();
cudaError_t tc_prepare();
cudaError_t f64_prepare();
cudaError_t tc_launch_prologue_ex(cudaStream_t s, TcStepParams *params, int64_t *persist,
                                  const TcSource &src, unsigned long long *or_slots, int ncols,
                                  int have_src, int trace_on, int *status, const double *inj,
                                  int n_inj);
cudaError_t tc_launch_step(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap, int mode);
cudaError_t tc_launch_batch_prologue(cudaStream_t s, const TcPrologueArgs *args, int n_meshes);
cudaError_t tc_launch_batch_step(cudaStream_t s, const TcBatch &b, int stages);
// node-plane exchange of the z-slab decomposition (vfe_slab.cu)
cudaError_t slab_pack_tc(cudaStream_t s, const int64_t *U, int nx, int ny, int nxp, int64_t plane,
                         int64_t comp, int k, const int64_t *persist, double *out);
cudaError_t slab_unpack_tc(cudaStream_t s, int64_t *U, int nx, int ny, int nxp, int64_t plane,
                           int64_t comp, int k, const int64_t *persist, const double *in,
                           unsigned long long *slot, int tiles_x);
cudaError_t stencil_prepare();
// the node-stencil kernel over d.segs / d.seg_off (d.n_ctas CTAs;
// nothing is launched for 0); tmap: box ST_BOXX x ST_BOXY x 1 x 3
cudaError_t stencil_launch(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap, int mode);
cudaError_t stencil_launch_ex(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap, int mode,
                              bool pdl);
// after a stencil launch (modes STEP and KU): at the listed nodes, replace
// the contributions of the elements that are not of the node's reference
// material (another material, void, outside the mesh) that the node stencil
// includes (u^n from d.U_cur)
cudaError_t stencil_fix(cudaStream_t s, const TcDevice &d, int mode);

cudaError_t tc_state_to_f64(cudaStream_t s, const int64_t *U, const int64_t *persist,
                            int extra_shift, int nx, int ny, int64_t nn, int nxp, int64_t plane,
                            int64_t comp, double *out);
// alpha: 3/4 for the orthogonal element, 1/3 for the trilinear one; ds: edge length
cudaError_t grad_g_accumulate(cudaStream_t s, int nx, int ny, int nz, const int32_t *mat,
                              double alpha, double ds, const double *u, const double *mu,
                              double scale, double *grad);
// the same on the tensor-core path from the fixed-point states (forward U with
// its exponent *Fu, adjoint Mu with *Fm; padded SoA layout)
cudaError_t grad_g_tc_accumulate(cudaStream_t s, int nx, int ny, int nz, const int32_t *mat,
                                 double ds, const int64_t *Uf, const int64_t *Fu,
                                 const int64_t *Mu, const int64_t *Fm, int nxp, int64_t plane,
                                 int64_t comp, double scale, double *grad);

size_t f64_params_bytes();
cudaError_t f64_launch_prologue(cudaStream_t s, void *params, int64_t *persist,
                                const TcSource &src, int have_src, int trace_on, int *status);
cudaError_t f64_launch_step(cudaStream_t s, const F64Device &d, const void *params, int mode);
