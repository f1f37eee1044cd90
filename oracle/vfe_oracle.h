/*
 * vfe_oracle.h -- plain FP64 CPU oracle for the voxel finite-element wave step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this code; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no source with the CUDA path.
 *
 * Everything here is written from Ichimura et al., "Low-ordered Orthogonal
 * Voxel Finite Element with INT8 Tensor Cores for GPU-based Explicit Elastic
 * Wave Propagation Analysis" (arXiv 2404.13683), Section 2:
 *   - governing equation and FE semi-discretisation (Eqs. GE:ORG, DGE:ORG),
 *   - the conventional voxel element VFEM (trilinear basis, lumped mass),
 *   - the orthogonal voxel element OVFEM (Hellinger-Reissner functional
 *     Eq. HRfunctional, element stiffness Eq. OVFEMstiff, mass Eq. OVFEMmass,
 *     bases Eqs. OVFEMbasis1/OVFEMbasis2),
 *   - the integer reformulation TCOVFEM (K^INT8, Eq. GE:TC) and its scaled
 *     hierarchical integer expansion (Eqs. intscaling, intcomp1-3,
 *     int8comp1-2),
 *   - the central-difference time integration (Eq. eqtimehistory).
 *
 * Conventions (readings of the paper where it is silent; each is listed in
 * the design notes):
 *   local node a = dx + 2*dy + 4*dz (dx,dy,dz in {0,1}); sign s_k = 2*d_k - 1;
 *   global node (i,j,k), 0<=i<=nx, id = i + (nx+1)*(j + (ny+1)*k);
 *   element (i,j,k), id = i + nx*(j + ny*k); DOF index = 3*node + component;
 *   material table rows are {Vp, Vs, rho}; id -1 marks a void cell;
 *   G = rho*Vs^2, kappa = rho*(Vp^2 - 4/3*Vs^2), lambda = kappa - 2G/3.
 * All functions return 0 on success and a negative value on bad input.
 */
#ifndef VFE_ORACLE_H
#define VFE_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_OVFEM = 0, ORACLE_VFEM = 1 };

/* Element stiffness K_e (24x24 row-major, DOF order 3*a + c) of a cube of
 * side ds with bulk modulus kappa and shear modulus G.
 * OVFEM: Eq. OVFEMstiff with Heaviside phi (Eq. OVFEMbasis1) and the seven
 * stress bases psi (Eq. OVFEMbasis2); VFEM: trilinear basis, 2x2x2 Gauss. */
int oracle_element_stiffness(int kind, double ds, double kappa, double G,
                             double *Ke);

/* Diagonal element mass per node (both elements): rho*ds^3/8.
 * OVFEM: exact (Eq. OVFEMmass with Heaviside phi); VFEM: lumped. */
double oracle_element_node_mass(int kind, double ds, double rho);

/* The constant 24x48 integer matrix K^INT8 = (K^kappa, Kbar^G) of the
 * TCOVFEM section, built from its definitions with Dbar^kappa, Dbar^G and the
 * equivalent strain-displacement matrix Bbar at element size ds.  Written as
 * doubles (the values are integral up to rounding; see the tests). */
int oracle_kint8(double ds, double *Kint8 /* 24*48 row-major */);

/* Eq. GE:TC evaluated in FP64 for one element: f = kappa*ds/256*(K^INT8*ubar
 * + 256/3*G/kappa*u), ubar = (u, 2/3*G/kappa*u). */
int oracle_ku_element_tc_fp64(double ds, double kappa, double G,
                              const double *ue, double *fe);

/* Eq. GE:TC with the paper's scaled hierarchical integer expansion: per
 * element scale s_e = max|ubar| (Eq. intscaling), one FP64->INT64 truncation
 * with a = 2^(7M) (Eqs. intcomp1-2 with N=1), M INT8 digit vectors with
 * b = 2^7 (Eq. int8comp1), integer products summed with weights b^(j-1)
 * (Eq. int8comp2), and the FP64 assembly of Eq. GE:TC.  M in [1, 8]. */
int oracle_ku_element_tc_int(double ds, double kappa, double G, int M,
                             const double *ue, double *fe);

/* Mesh-level helpers. mat: nx*ny*nz ids (x fastest, -1 = void);
 * table: n_mat rows of {Vp, Vs, rho}. */
int oracle_node_mass(int kind, int nx, int ny, int nz, double ds,
                     const int32_t *mat, const double *table, int n_mat,
                     double *mass /* (nx+1)(ny+1)(nz+1) */);

/* Element-by-element f = K u over the whole mesh (FP64, definition of
 * K_e; the INT path flag selects Eq. GE:TC with the M-stage integer
 * expansion instead: tc_stages = 0 means plain FP64 K_e). */
int oracle_ku(int kind, int nx, int ny, int nz, double ds,
              const int32_t *mat, const double *table, int n_mat,
              int tc_stages, const double *u, double *f);

/* Threads for oracle_ku's element loop and the runs' update loops (built
 * with OpenMP; 1 thread otherwise).  With n > 1 the elements are visited in
 * eight colours of (i, j, k) parity, so that no two elements summed at the
 * same time share a node; each element's K_e u_e is the same arithmetic as
 * with one thread, and only the order of the at most eight additions into a
 * node differs.  Returns the count in effect (default 1). */
int oracle_set_threads(int n);
int oracle_get_threads(void);

/* Same as oracle_ku but only for the listed nodes: f_sel[3*q+c] is the
 * force at node sel[q].  Used to check sampled outputs of large meshes. */
int oracle_ku_nodes(int kind, int nx, int ny, int nz, double ds,
                    const int32_t *mat, const double *table, int n_mat,
                    const double *u, int n_sel, const int64_t *sel,
                    double *f_sel);

/* Largest eigenvalue of M_e^{-1} K_e (Jacobi rotations on the symmetric
 * 24x24 K_e scaled by the diagonal mass). */
double oracle_element_max_eig(int kind, double ds, double kappa, double G,
                              double rho);

/* dt = cfl_fraction * min over materials present of 2/sqrt(lambda_max). */
double oracle_dt(int kind, int nx, int ny, int nz, double ds,
                 const int32_t *mat, const double *table, int n_mat,
                 double cfl_fraction);

/* Ricker wavelet (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2). */
double oracle_ricker(double t, double f0, double t0);

/* Central-difference run (Eq. eqtimehistory; update form of Section 3 with
 * the force sign F - Ku):  u^0 = u^-1 = 0 unless u0/um1 are given;
 *   u^{n+1} = 2u^n - u^{n-1} + dt^2 M^{-1} (F^n - K u^n) on free DOFs,
 * F^n = amp*ricker(n*dt)*dir at the source node (src_node < 0: no source).
 * Fixed DOFs: every node of the plane k = 0 when fix_bottom, and every node
 * with zero mass.  traces[(n*n_rec + r)*3 + c] = u^{n+1} at receiver r.
 * u_out/um1_out (optional) receive u^{nsteps} and u^{nsteps-1}. */
/* fix_bottom (here and below): 0 none, 1 the bottom plane k = 0, 2 the four
 * corner nodes of the bottom plane (Section 3). */
int oracle_run(int kind, int nx, int ny, int nz, double ds,
               const int32_t *mat, const double *table, int n_mat,
               int fix_bottom, double dt, int nsteps,
               int64_t src_node, const double *src_dir, double f0,
               double t0, double amp,
               int n_rec, const int64_t *rec_nodes,
               const double *u0, const double *um1,
               double *traces, double *u_out, double *um1_out);

/* oracle_run with Rayleigh damping C = alpha M + beta K (Section 3 uses
 * Rayleigh damping without giving its time discretisation; the reading used
 * here): the mass term with the central velocity (u^{n+1} - u^{n-1}) / (2 dt),
 * the stiffness term with the backward velocity (u^n - u^{n-1}) / dt, so the
 * step stays explicit:
 *   (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1} - dt^2 M^-1 (K w^n - F^n),
 *   a = alpha dt / 2,  w^n = u^n + (beta / dt) (u^n - u^{n-1}).
 * alpha = beta = 0 gives oracle_run exactly. */
int oracle_run_damped(int kind, int nx, int ny, int nz, double ds,
                      const int32_t *mat, const double *table, int n_mat,
                      int fix_bottom, double dt, int nsteps,
                      int64_t src_node, const double *src_dir, double f0,
                      double t0, double amp, double alpha, double beta,
                      int n_rec, const int64_t *rec_nodes,
                      const double *u0, const double *um1,
                      double *traces, double *u_out, double *um1_out);

/* Adjoint-state gradient of the receiver misfit
 *   J = 1/2 sum_{n<N} sum_r |u^{n+1}(r) - data[n][r]|^2
 * for the run of oracle_run (from rest), with respect to each element's shear
 * modulus G_e at fixed kappa_e: with multipliers mu^n of the step equations,
 *   mu^{m-1} = 2 mu^m - mu^{m+1} - dt^2 M^-1 K mu^m - M^-1 dJ/du^m,
 *   mu^N = mu^{N+1} = 0, fixed DOFs zero, and
 *   dJ/dG_e = dt^2 sum_{n=0}^{N-1} mu^n_e . (dK_e/dG) u^n_e.
 * Stores every forward state (small meshes only).  grad: nx*ny*nz. */
int oracle_misfit_gradient(int kind, int nx, int ny, int nz, double ds,
                           const int32_t *mat, const double *table, int n_mat,
                           int fix_bottom, double dt, int nsteps,
                           int64_t src_node, const double *src_dir, double f0,
                           double t0, double amp, int n_rec,
                           const int64_t *rec_nodes, const double *data,
                           double *grad, double *misfit);

#ifdef __cplusplus
}
#endif
#endif
