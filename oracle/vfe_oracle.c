/*
 * vfe_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Slow, obvious loops that follow the definitions of arXiv 2404.13683,
 * Section 2, one step at a time.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library; the product never
 * does, and this file shares no code with the CUDA path.
 *
 * Parity pins live in tests/test_oracle_*.py: closed forms of both element
 * matrices derived by hand, rigid-body null space, symmetry/PSD/rank,
 * integrality of K^INT8, exact rational evaluation of Eq. GE:TC, assembled
 * dense K vs element-by-element K u, energy conservation and the discrete
 * dispersion relation.
 */
#include "vfe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NDOF 24

/* ---------- small dense helpers ---------------------------------------- */

/* sign of local node a along axis k: s = 2*d - 1 with a = dx + 2dy + 4dz. */
static int node_sign(int a, int k) { return ((a >> k) & 1) ? 1 : -1; }

/* Isotropic Voigt elasticity (engineering shear), order 11,22,33,12,23,13,
 * with lambda = kappa - 2G/3.  C is linear in (kappa, G), so C(1,0) and
 * C(0,1) are its derivatives with respect to kappa and G. */
static void voigt_c(double kappa, double G, double C[6][6]) {
  double lam = kappa - 2.0 * G / 3.0;
  memset(C, 0, sizeof(double) * 36);
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) C[p][q] = lam + (p == q ? 2.0 * G : 0.0);
  for (int p = 3; p < 6; ++p) C[p][p] = G;
}

/* Voigt component index of the pair (k,l), k<=l. */
static int voigt_index(int k, int l) {
  if (k == l) return k;
  if (k > l) { int t = k; k = l; l = t; }
  if (k == 0 && l == 1) return 3;
  if (k == 1 && l == 2) return 4;
  return 5; /* (0,2) */
}

/* Gauss-Jordan inverse of an n x n matrix (n <= 8), partial pivoting. */
static int invert(int n, const double *A, double *Ainv) {
  double M[8][16];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      M[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
    if (M[p][c] == 0.0) return -1;
    if (p != c)
      for (int j = 0; j < 2 * n; ++j) { double t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
    double d = M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double fct = M[r][c];
      if (fct != 0.0)
        for (int j = 0; j < 2 * n; ++j) M[r][j] -= fct * M[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i][j + n];
  return 0;
}

/* ---------- OVFEM ingredients (Eqs. OVFEMbasis1, OVFEMbasis2) ---------- */

/* psi^beta, beta = 0..6: 1, r1, r2, r3, r1 r2, r2 r3, r1 r3 (Eq. OVFEMbasis2,
 * axes numbered 0,1,2 here).  Returns the value at local point r. */
static double psi(int beta, const double r[3]) {
  switch (beta) {
    case 0: return 1.0;
    case 1: return r[0];
    case 2: return r[1];
    case 3: return r[2];
    case 4: return r[0] * r[1];
    case 5: return r[1] * r[2];
    default: return r[0] * r[2];
  }
}

/* Two-point Gauss-Legendre on [lo, hi]: exact for cubics in each variable,
 * and every integrand below has degree <= 2 per variable. */
static void gauss2(double lo, double hi, double x[2], double w[2]) {
  double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo), g = 1.0 / sqrt(3.0);
  x[0] = c - h * g; x[1] = c + h * g; w[0] = h; w[1] = h;
}

/* Gmat[beta][a][k] = (psi^beta d(phi^a)/dx_k)_e with the Heaviside basis
 * phi^a = H(s1 r1) H(s2 r2) H(s3 r3) (Eq. OVFEMbasis1).  As a global basis
 * function phi^a is the indicator of the dual cell of its node, so it does
 * not jump across element faces and its distributional gradient lives on the
 * element mid-planes only:  d phi^a/dr_k = s_k delta(r_k) prod_{j!=k} H(s_j r_j).
 * With x = ds/2 r: dV = (ds/2)^3 dr and d/dx = (2/ds) d/dr, so
 *   (psi d phi/dx_k)_e = (ds/2)^2 s_k * int_{quadrant} psi|_{r_k=0} dr_j dr_l.
 * The quadrant integral is evaluated with Gauss quadrature. */
static void ovfem_gmat(double ds, double Gm[7][8][3]) {
  for (int beta = 0; beta < 7; ++beta)
    for (int a = 0; a < 8; ++a)
      for (int k = 0; k < 3; ++k) {
        int j = (k + 1) % 3, l = (k + 2) % 3;
        double lo_j = node_sign(a, j) > 0 ? 0.0 : -1.0, hi_j = lo_j + 1.0;
        double lo_l = node_sign(a, l) > 0 ? 0.0 : -1.0, hi_l = lo_l + 1.0;
        double xj[2], wj[2], xl[2], wl[2];
        gauss2(lo_j, hi_j, xj, wj);
        gauss2(lo_l, hi_l, xl, wl);
        double acc = 0.0;
        for (int p = 0; p < 2; ++p)
          for (int q = 0; q < 2; ++q) {
            double r[3];
            r[k] = 0.0; r[j] = xj[p]; r[l] = xl[q];
            acc += wj[p] * wl[q] * psi(beta, r);
          }
        Gm[beta][a][k] = 0.25 * ds * ds * node_sign(a, k) * acc;
      }
}

/* Gram matrix (psi^beta psi^beta')_e over the cube, by Gauss quadrature. */
static void ovfem_gram(double ds, double Gr[7][7]) {
  double x[2], w[2];
  gauss2(-1.0, 1.0, x, w);
  double vol = ds * ds * ds / 8.0;
  for (int b1 = 0; b1 < 7; ++b1)
    for (int b2 = 0; b2 < 7; ++b2) {
      double acc = 0.0;
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q)
          for (int s = 0; s < 2; ++s) {
            double r[3] = {x[p], x[q], x[s]};
            acc += w[p] * w[q] * w[s] * psi(b1, r) * psi(b2, r);
          }
      Gr[b1][b2] = vol * acc;
    }
}

/* Strain-displacement block B_beta (6 x 24, engineering shear) built from
 * (psi^beta grad phi^a)_e: eps_kk <- G[a][k] u_ak,
 * gamma_kl <- G[a][k] u_al + G[a][l] u_ak. */
static void ovfem_bmat(double Gm[7][8][3], int beta, double B[6][NDOF]) {
  memset(B, 0, sizeof(double) * 6 * NDOF);
  for (int a = 0; a < 8; ++a)
    for (int k = 0; k < 3; ++k)
      for (int l = k; l < 3; ++l) {
        int v = voigt_index(k, l);
        if (k == l) {
          B[v][3 * a + k] += Gm[beta][a][k];
        } else {
          B[v][3 * a + l] += Gm[beta][a][k];
          B[v][3 * a + k] += Gm[beta][a][l];
        }
      }
}

/* K = sum_{beta,beta'} B_beta^T (Gram^-1)_{beta beta'} Cmat B_beta' -- the
 * stationary point of Eq. HRfunctional in the stress coefficients, which is
 * Eq. OVFEMstiff with c acting on each stress coefficient sigma^beta. */
static int ovfem_assemble(double ds, double C[6][6], double *Ke) {
  double Gm[7][8][3], Gr[7][7], Gi[49];
  double B[7][6][NDOF];
  ovfem_gmat(ds, Gm);
  ovfem_gram(ds, Gr);
  if (invert(7, &Gr[0][0], Gi)) return -1;
  for (int beta = 0; beta < 7; ++beta) ovfem_bmat(Gm, beta, B[beta]);
  memset(Ke, 0, sizeof(double) * NDOF * NDOF);
  for (int b1 = 0; b1 < 7; ++b1)
    for (int b2 = 0; b2 < 7; ++b2) {
      double g = Gi[b1 * 7 + b2];
      if (g == 0.0) continue;
      double CB[6][NDOF];
      for (int p = 0; p < 6; ++p)
        for (int n = 0; n < NDOF; ++n) {
          double acc = 0.0;
          for (int q = 0; q < 6; ++q) acc += C[p][q] * B[b2][q][n];
          CB[p][n] = acc;
        }
      for (int m = 0; m < NDOF; ++m)
        for (int n = 0; n < NDOF; ++n) {
          double acc = 0.0;
          for (int p = 0; p < 6; ++p) acc += B[b1][p][m] * CB[p][n];
          Ke[m * NDOF + n] += g * acc;
        }
    }
  return 0;
}

/* ---------- VFEM (trilinear, 2x2x2 Gauss) ------------------------------- */

static int vfem_assemble(double ds, double C[6][6], double *Ke) {
  double g = 1.0 / sqrt(3.0), pts[2] = {-g, g};
  double jac = ds * ds * ds / 8.0; /* dV = (ds/2)^3 dr, weights 1 */
  memset(Ke, 0, sizeof(double) * NDOF * NDOF);
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q)
      for (int s = 0; s < 2; ++s) {
        double r[3] = {pts[p], pts[q], pts[s]};
        double dN[8][3];
        for (int a = 0; a < 8; ++a)
          for (int k = 0; k < 3; ++k) {
            /* N_a = 1/8 prod (1 + s_m r_m) (basis of the VFEM paragraph with
             * the sign read as 1/8 prod(1 + rbar_i r_i)) */
            double v = 0.125 * node_sign(a, k) * (2.0 / ds);
            for (int m = 0; m < 3; ++m)
              if (m != k) v *= 1.0 + node_sign(a, m) * r[m];
            dN[a][k] = v;
          }
        double B[6][NDOF];
        memset(B, 0, sizeof(B));
        for (int a = 0; a < 8; ++a)
          for (int k = 0; k < 3; ++k)
            for (int l = k; l < 3; ++l) {
              int v = voigt_index(k, l);
              if (k == l) {
                B[v][3 * a + k] += dN[a][k];
              } else {
                B[v][3 * a + l] += dN[a][k];
                B[v][3 * a + k] += dN[a][l];
              }
            }
        for (int m = 0; m < NDOF; ++m)
          for (int n = 0; n < NDOF; ++n) {
            double acc = 0.0;
            for (int x = 0; x < 6; ++x)
              for (int y = 0; y < 6; ++y) acc += B[x][m] * C[x][y] * B[y][n];
            Ke[m * NDOF + n] += jac * acc;
          }
      }
  return 0;
}

int oracle_element_stiffness(int kind, double ds, double kappa, double G,
                             double *Ke) {
  if (!Ke || !(ds > 0.0)) return -1;
  double C[6][6];
  voigt_c(kappa, G, C);
  if (kind == ORACLE_OVFEM) return ovfem_assemble(ds, C, Ke);
  if (kind == ORACLE_VFEM) return vfem_assemble(ds, C, Ke);
  return -1;
}

/* (phi^a phi^b)_e: Heaviside phi are indicators of disjoint octants, so the
 * OVFEM mass is exactly diagonal with rho*ds^3/8 (Eq. OVFEMmass); for VFEM
 * this is the lumped value rho/8 (1)_e. */
double oracle_element_node_mass(int kind, double ds, double rho) {
  (void)kind;
  return rho * ds * ds * ds / 8.0;
}

/* ---------- TCOVFEM (K^INT8 and Eq. GE:TC) ------------------------------ */

/* Dbar^kappa = 3 d[(psi psi)^-1 c]/d kappa ds^3, Dbar^G likewise; Bbar is the
 * stacked B_beta divided by ds^4 (the reading under which the paper's
 * K^kappa = 256/3 Bbar^t Dbar^kappa Bbar ds^4 equals 256/ds K_e at kappa=1,
 * G=0).  Kbar^G = 128 Bbar^t Dbar^G Bbar ds^4 - 128 I. */
int oracle_kint8(double ds, double *Kint8) {
  if (!Kint8 || !(ds > 0.0)) return -1;
  double Gm[7][8][3], Gr[7][7], Gi[49];
  double B[7][6][NDOF];
  ovfem_gmat(ds, Gm);
  ovfem_gram(ds, Gr);
  if (invert(7, &Gr[0][0], Gi)) return -1;
  for (int beta = 0; beta < 7; ++beta) ovfem_bmat(Gm, beta, B[beta]);
  /* dC/dkappa and dC/dG from the Voigt matrix by exact linearity. */
  double C10[6][6], C01[6][6];
  voigt_c(1.0, 0.0, C10);
  voigt_c(0.0, 1.0, C01);
  double ds3 = ds * ds * ds, ds4 = ds3 * ds;
  double Kk[NDOF][NDOF], Kg[NDOF][NDOF];
  memset(Kk, 0, sizeof(Kk));
  memset(Kg, 0, sizeof(Kg));
  for (int b1 = 0; b1 < 7; ++b1)
    for (int b2 = 0; b2 < 7; ++b2) {
      double g = Gi[b1 * 7 + b2];
      if (g == 0.0) continue;
      for (int m = 0; m < NDOF; ++m)
        for (int n = 0; n < NDOF; ++n) {
          double ak = 0.0, ag = 0.0;
          for (int p = 0; p < 6; ++p)
            for (int q = 0; q < 6; ++q) {
              /* Bbar = B/ds^4 on both sides; D = 3 ds^3 g dC */
              double bb = (B[b1][p][m] / ds4) * (B[b2][q][n] / ds4);
              ak += bb * 3.0 * ds3 * g * C10[p][q];
              ag += bb * 3.0 * ds3 * g * C01[p][q];
            }
          Kk[m][n] += ak;
          Kg[m][n] += ag;
        }
    }
  for (int m = 0; m < NDOF; ++m)
    for (int n = 0; n < NDOF; ++n) {
      Kint8[m * 48 + n] = 256.0 / 3.0 * Kk[m][n] * ds4;
      Kint8[m * 48 + 24 + n] = 128.0 * Kg[m][n] * ds4 - (m == n ? 128.0 : 0.0);
    }
  return 0;
}

int oracle_ku_element_tc_fp64(double ds, double kappa, double G,
                              const double *ue, double *fe) {
  double K[24 * 48];
  if (oracle_kint8(ds, K)) return -1;
  double ubar[48];
  for (int i = 0; i < 24; ++i) {
    ubar[i] = ue[i];
    ubar[24 + i] = 2.0 / 3.0 * G / kappa * ue[i];
  }
  for (int m = 0; m < 24; ++m) {
    double acc = 0.0;
    for (int n = 0; n < 48; ++n) acc += K[m * 48 + n] * ubar[n];
    fe[m] = kappa * ds / 256.0 * (acc + 256.0 / 3.0 * G / kappa * ue[m]);
  }
  return 0;
}

/* K^INT8 as exact integers (the definition yields integral values; the
 * nearest integer removes the FP64 rounding of the construction). */
static int kint8_integers(int32_t Ki[24][48]) {
  double K[24 * 48];
  if (oracle_kint8(1.0, K)) return -1;
  for (int m = 0; m < 24; ++m)
    for (int n = 0; n < 48; ++n) Ki[m][n] = (int32_t)llround(K[m * 48 + n]);
  return 0;
}

int oracle_ku_element_tc_int(double ds, double kappa, double G, int M,
                             const double *ue, double *fe) {
  if (M < 1 || M > 8 || !ue || !fe) return -1;
  int32_t Ki[24][48];
  if (kint8_integers(Ki)) return -1;
  /* ubar_e = (u_e, 2/3 G/kappa u_e) (text after Eq. GE:TC) */
  double ubar[48];
  for (int i = 0; i < 24; ++i) {
    ubar[i] = ue[i];
    ubar[24 + i] = 2.0 / 3.0 * G / kappa * ue[i];
  }
  /* s_e = max_i |ubar_i| (Eq. intscaling) */
  double se = 0.0;
  for (int i = 0; i < 48; ++i) se = fmax(se, fabs(ubar[i]));
  __int128 r[24];
  memset(r, 0, sizeof(r));
  if (se > 0.0) {
    /* one FP64 -> INT64 truncation with a = 2^(7M) (Eqs. intcomp1-2, N=1) */
    int64_t lim = ((int64_t)1 << (7 * M)) - 1;
    int64_t q[48];
    for (int i = 0; i < 48; ++i) {
      double us = ubar[i] / se;
      double t = trunc(ldexp(us, 7 * M));
      int64_t v = (int64_t)t;
      if (v > lim) v = lim; /* |us| = 1 would need 7M+1 bits */
      if (v < -lim) v = -lim;
      q[i] = v;
    }
    /* M INT8 digit vectors, b = 2^7 (Eq. int8comp1): sign-magnitude digits,
     * d_j = sgn(q) ((|q| >> 7(j-1)) & 127) in [-127, 127]. */
    for (int j = 1; j <= M; ++j) {
      int32_t d[48];
      for (int i = 0; i < 48; ++i) {
        int64_t mag = q[i] < 0 ? -q[i] : q[i];
        int32_t dig = (int32_t)((mag >> (7 * (j - 1))) & 127);
        d[i] = q[i] < 0 ? -dig : dig;
      }
      /* K^INT8 d_j in integers, weighted by b^(j-1) (Eq. int8comp2) */
      for (int m = 0; m < 24; ++m) {
        int64_t acc = 0;
        for (int n = 0; n < 48; ++n) acc += (int64_t)Ki[m][n] * d[n];
        r[m] += (__int128)acc << (7 * (j - 1));
      }
    }
  }
  /* K^INT8 ubar_e = s_e r / a (Eq. intcomp3), then Eq. GE:TC in FP64 */
  for (int m = 0; m < 24; ++m) {
    double kub = se * ldexp((double)r[m], -7 * M);
    fe[m] = kappa * ds / 256.0 * (kub + 256.0 / 3.0 * G / kappa * ue[m]);
  }
  return 0;
}

/* ---------- mesh-level operations --------------------------------------- */

static int material_moduli(const double *row, double *kappa, double *G,
                           double *rho) {
  double vp = row[0], vs = row[1], rh = row[2];
  if (!(rh > 0.0) || !(vs >= 0.0) || !(vp * vp > 4.0 / 3.0 * vs * vs)) return -1;
  *G = rh * vs * vs;
  *kappa = rh * (vp * vp - 4.0 / 3.0 * vs * vs);
  *rho = rh;
  return 0;
}

static int64_t node_id(int nx, int ny, int i, int j, int k) {
  return (int64_t)i + (int64_t)(nx + 1) * ((int64_t)j + (int64_t)(ny + 1) * k);
}

/* Per-material element matrices, n_mat * 576 doubles. */
static double *material_matrices(int kind, double ds, const double *table,
                                 int n_mat, double *kap, double *gg,
                                 double *rho) {
  double *Km = (double *)malloc(sizeof(double) * 576 * (n_mat > 0 ? n_mat : 1));
  if (!Km) return NULL;
  for (int m = 0; m < n_mat; ++m) {
    double k, g, r;
    if (material_moduli(table + 3 * m, &k, &g, &r) ||
        oracle_element_stiffness(kind, ds, k, g, Km + 576 * m)) {
      free(Km);
      return NULL;
    }
    if (kap) kap[m] = k;
    if (gg) gg[m] = g;
    if (rho) rho[m] = r;
  }
  return Km;
}

static int check_mesh(int nx, int ny, int nz, const int32_t *mat, int n_mat) {
  if (nx < 1 || ny < 1 || nz < 1 || !mat || n_mat < 1) return -1;
  int64_t ne = (int64_t)nx * ny * nz;
  for (int64_t e = 0; e < ne; ++e)
    if (mat[e] < -1 || mat[e] >= n_mat) return -1;
  return 0;
}

int oracle_node_mass(int kind, int nx, int ny, int nz, double ds,
                     const int32_t *mat, const double *table, int n_mat,
                     double *mass) {
  if (check_mesh(nx, ny, nz, mat, n_mat) || !mass) return -1;
  int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int64_t n = 0; n < nn; ++n) mass[n] = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int32_t m = mat[i + (int64_t)nx * (j + (int64_t)ny * k)];
        if (m < 0) continue;
        double kap, g, rho;
        if (material_moduli(table + 3 * m, &kap, &g, &rho)) return -1;
        double me = oracle_element_node_mass(kind, ds, rho);
        for (int a = 0; a < 8; ++a)
          mass[node_id(nx, ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))] += me;
      }
  return 0;
}

/* K_e u_e of element (i,j,k) with material m (FP64 K_e, or Eq. GE:TC with
 * the M-stage integer expansion when tc_stages > 0), and its 8 node ids. */
static int element_ku(int nx, int ny, int i, int j, int k, int m, double ds,
                      const double *Km, const double *kap, const double *gg,
                      int tc_stages, const double *u, int64_t nodes[8],
                      double fe[24]) {
  double ue[24];
  for (int a = 0; a < 8; ++a) {
    nodes[a] = node_id(nx, ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    for (int c = 0; c < 3; ++c) ue[3 * a + c] = u[3 * nodes[a] + c];
  }
  if (tc_stages > 0)
    return oracle_ku_element_tc_int(ds, kap[m], gg[m], tc_stages, ue, fe);
  const double *K = Km + 576 * m;
  for (int r = 0; r < 24; ++r) {
    double acc = 0.0;
    for (int s = 0; s < 24; ++s) acc += K[r * 24 + s] * ue[s];
    fe[r] = acc;
  }
  return 0;
}

/* Threads used by the element loop of oracle_ku and the update loops of the
 * runs (1 = the plain sequential loops). */
static int g_threads = 1;

int oracle_set_threads(int n) {
#ifdef _OPENMP
  g_threads = n < 1 ? 1 : n;
#else
  g_threads = 1;
  (void)n;
#endif
  return g_threads;
}

int oracle_get_threads(void) { return g_threads; }

int oracle_ku(int kind, int nx, int ny, int nz, double ds,
              const int32_t *mat, const double *table, int n_mat,
              int tc_stages, const double *u, double *f) {
  if (check_mesh(nx, ny, nz, mat, n_mat) || !u || !f) return -1;
  if (tc_stages < 0 || tc_stages > 8) return -1;
  if (tc_stages > 0 && kind != ORACLE_OVFEM) return -1;
  double *kap = (double *)malloc(sizeof(double) * n_mat);
  double *gg = (double *)malloc(sizeof(double) * n_mat);
  double *Km = material_matrices(kind, ds, table, n_mat, kap, gg, NULL);
  if (!Km || !kap || !gg) { free(Km); free(kap); free(gg); return -1; }
  int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int64_t d = 0; d < 3 * nn; ++d) f[d] = 0.0;
  int bad = 0;
  if (g_threads <= 1) {
    /* f = sum_e P_e^T K_e P_e u in element order */
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          int32_t m = mat[i + (int64_t)nx * (j + (int64_t)ny * k)];
          if (m < 0) continue;
          int64_t nodes[8];
          double fe[24];
          if (element_ku(nx, ny, i, j, k, m, ds, Km, kap, gg, tc_stages, u, nodes, fe)) {
            bad = 1;
            continue;
          }
          for (int a = 0; a < 8; ++a)
            for (int c = 0; c < 3; ++c) f[3 * nodes[a] + c] += fe[3 * a + c];
        }
  } else {
    /* The same sum over elements in eight colours (i, j, k parities): two
     * elements of one colour share no node, so each colour's elements are
     * added in parallel without races.  Only the order in which a node's
     * (at most eight) contributions are added differs from the loop above. */
    for (int color = 0; color < 8; ++color) {
      const int ci = color & 1, cj = (color >> 1) & 1, ck = color >> 2;
      const int mz = (nz - ck + 1) / 2, my = (ny - cj + 1) / 2;
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(g_threads) reduction(|| : bad)
#endif
      for (int kk = 0; kk < mz; ++kk)
        for (int jj = 0; jj < my; ++jj) {
          const int k = ck + 2 * kk, j = cj + 2 * jj;
          for (int i = ci; i < nx; i += 2) {
            int32_t m = mat[i + (int64_t)nx * (j + (int64_t)ny * k)];
            if (m < 0) continue;
            int64_t nodes[8];
            double fe[24];
            if (element_ku(nx, ny, i, j, k, m, ds, Km, kap, gg, tc_stages, u, nodes, fe)) {
              bad = 1;
              continue;
            }
            for (int a = 0; a < 8; ++a)
              for (int c = 0; c < 3; ++c) f[3 * nodes[a] + c] += fe[3 * a + c];
          }
        }
    }
  }
  free(Km); free(kap); free(gg);
  return bad ? -1 : 0;
}

int oracle_ku_nodes(int kind, int nx, int ny, int nz, double ds,
                    const int32_t *mat, const double *table, int n_mat,
                    const double *u, int n_sel, const int64_t *sel,
                    double *f_sel) {
  if (nx < 1 || ny < 1 || nz < 1 || !mat || n_mat < 1 || !u || !sel || !f_sel || n_sel < 0)
    return -1;
  double *Km = material_matrices(kind, ds, table, n_mat, NULL, NULL, NULL);
  if (!Km) return -1;
  int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int q = 0; q < n_sel; ++q) {
    int64_t n = sel[q];
    if (n < 0 || n >= nn) { free(Km); return -1; }
    int ni = (int)(n % (nx + 1));
    int nj = (int)((n / (nx + 1)) % (ny + 1));
    int nk = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
    double acc[3] = {0.0, 0.0, 0.0};
    /* the (up to) eight elements that contain node n; a is n's local index */
    for (int a = 0; a < 8; ++a) {
      int ei = ni - (a & 1), ej = nj - ((a >> 1) & 1), ek = nk - ((a >> 2) & 1);
      if (ei < 0 || ej < 0 || ek < 0 || ei >= nx || ej >= ny || ek >= nz) continue;
      int32_t m = mat[ei + (int64_t)nx * (ej + (int64_t)ny * ek)];
      if (m < -1 || m >= n_mat) { free(Km); return -1; }
      if (m < 0) continue;
      const double *K = Km + 576 * m;
      for (int b = 0; b < 8; ++b) {
        int64_t nb = node_id(nx, ny, ei + (b & 1), ej + ((b >> 1) & 1), ek + ((b >> 2) & 1));
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) acc[c] += K[(3 * a + c) * 24 + 3 * b + d] * u[3 * nb + d];
      }
    }
    for (int c = 0; c < 3; ++c) f_sel[3 * q + c] = acc[c];
  }
  free(Km);
  return 0;
}

/* Cyclic Jacobi eigenvalue iteration on a symmetric n x n matrix (in place);
 * the diagonal holds the eigenvalues at exit. */
static void jacobi_eigen(int n, double *A) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (fabs(apq) < 1e-300) continue;
        double app = A[p * n + p], aqq = A[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
      }
  }
}

double oracle_element_max_eig(int kind, double ds, double kappa, double G,
                              double rho) {
  double K[576];
  if (oracle_element_stiffness(kind, ds, kappa, G, K)) return -1.0;
  double m = oracle_element_node_mass(kind, ds, rho);
  for (int i = 0; i < 576; ++i) K[i] /= m;
  jacobi_eigen(24, K);
  double lmax = 0.0;
  for (int i = 0; i < 24; ++i) lmax = fmax(lmax, K[i * 24 + i]);
  return lmax;
}

double oracle_dt(int kind, int nx, int ny, int nz, double ds,
                 const int32_t *mat, const double *table, int n_mat,
                 double cfl_fraction) {
  if (check_mesh(nx, ny, nz, mat, n_mat)) return -1.0;
  int64_t ne = (int64_t)nx * ny * nz;
  char *used = (char *)calloc((size_t)n_mat, 1);
  if (!used) return -1.0;
  for (int64_t e = 0; e < ne; ++e)
    if (mat[e] >= 0) used[mat[e]] = 1;
  double dt = -1.0;
  for (int m = 0; m < n_mat; ++m) {
    if (!used[m]) continue;
    double kap, g, rho;
    if (material_moduli(table + 3 * m, &kap, &g, &rho)) { free(used); return -1.0; }
    double lmax = oracle_element_max_eig(kind, ds, kap, g, rho);
    double dtc = 2.0 / sqrt(lmax);
    if (dt < 0.0 || dtc < dt) dt = dtc;
  }
  free(used);
  return dt < 0.0 ? -1.0 : cfl_fraction * dt;
}

double oracle_ricker(double t, double f0, double t0) {
  double a = M_PI * M_PI * f0 * f0 * (t - t0) * (t - t0);
  return (1.0 - 2.0 * a) * exp(-a);
}

/* ---------- fixed nodes ---------------------------------------------------- */

/* fix_bottom: 0 none, 1 every node of the bottom plane k = 0, 2 the four
 * corner nodes of the bottom plane (Section 3 fixes the four bottom corner
 * points in x, y and z); massless nodes are always fixed. */
static char node_fixed(int fix_bottom, int nx, int ny, int64_t n, double mass) {
  const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
  const int64_t i = n % sx, j = (n / sx) % (ny + 1), k = n / sxy;
  if (mass == 0.0) return 1;
  if (k != 0) return 0;
  if (fix_bottom == 1) return 1;
  if (fix_bottom == 2) return (char)((i == 0 || i == nx) && (j == 0 || j == ny));
  return 0;
}

int oracle_run(int kind, int nx, int ny, int nz, double ds,
               const int32_t *mat, const double *table, int n_mat,
               int fix_bottom, double dt, int nsteps,
               int64_t src_node, const double *src_dir, double f0,
               double t0, double amp,
               int n_rec, const int64_t *rec_nodes,
               const double *u0, const double *um1,
               double *traces, double *u_out, double *um1_out) {
  if (check_mesh(nx, ny, nz, mat, n_mat) || !(dt > 0.0) || nsteps < 0) return -1;
  if (n_rec < 0 || (n_rec > 0 && (!rec_nodes || !traces))) return -1;
  int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  if (src_node >= nn) return -1;
  for (int r = 0; r < n_rec; ++r)
    if (rec_nodes[r] < 0 || rec_nodes[r] >= nn) return -1;
  double *mass = (double *)malloc(sizeof(double) * nn);
  double *u = (double *)malloc(sizeof(double) * 3 * nn);
  double *up = (double *)malloc(sizeof(double) * 3 * nn);
  double *un = (double *)malloc(sizeof(double) * 3 * nn);
  double *f = (double *)malloc(sizeof(double) * 3 * nn);
  char *fixed = (char *)malloc((size_t)nn);
  int rc = -1;
  if (!mass || !u || !up || !un || !f || !fixed) goto done;
  if (oracle_node_mass(kind, nx, ny, nz, ds, mat, table, n_mat, mass)) goto done;
  for (int64_t n = 0; n < nn; ++n) {
    fixed[n] = node_fixed(fix_bottom, nx, ny, n, mass[n]);
  }
  for (int64_t d = 0; d < 3 * nn; ++d) {
    u[d] = u0 ? u0[d] : 0.0;
    up[d] = um1 ? um1[d] : 0.0;
    if (fixed[d / 3]) u[d] = up[d] = 0.0;
  }
  for (int it = 0; it < nsteps; ++it) {
    if (oracle_ku(kind, nx, ny, nz, ds, mat, table, n_mat, 0, u, f)) goto done;
    double fsrc = src_node >= 0 ? amp * oracle_ricker(it * dt, f0, t0) : 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
#endif
    for (int64_t n = 0; n < nn; ++n)
      for (int c = 0; c < 3; ++c) {
        int64_t d = 3 * n + c;
        if (fixed[n]) { un[d] = 0.0; continue; }
        double F = (n == src_node) ? fsrc * src_dir[c] : 0.0;
        un[d] = 2.0 * u[d] - up[d] + dt * dt / mass[n] * (F - f[d]);
      }
    for (int r = 0; r < n_rec; ++r)
      for (int c = 0; c < 3; ++c)
        traces[((int64_t)it * n_rec + r) * 3 + c] = un[3 * rec_nodes[r] + c];
    double *t = up; up = u; u = un; un = t;
  }
  if (u_out) memcpy(u_out, u, sizeof(double) * 3 * nn);
  if (um1_out) memcpy(um1_out, up, sizeof(double) * 3 * nn);
  rc = 0;
done:
  free(mass); free(u); free(up); free(un); free(f); free(fixed);
  return rc;
}

/* ---------- central-difference run with Rayleigh damping ------------------ */

int oracle_run_damped(int kind, int nx, int ny, int nz, double ds,
                      const int32_t *mat, const double *table, int n_mat,
                      int fix_bottom, double dt, int nsteps,
                      int64_t src_node, const double *src_dir, double f0,
                      double t0, double amp, double alpha, double beta,
                      int n_rec, const int64_t *rec_nodes,
                      const double *u0, const double *um1,
                      double *traces, double *u_out, double *um1_out) {
  if (check_mesh(nx, ny, nz, mat, n_mat) || !(dt > 0.0) || nsteps < 0) return -1;
  if (!(alpha >= 0.0) || !(beta >= 0.0)) return -1;
  if (n_rec < 0 || (n_rec > 0 && (!rec_nodes || !traces))) return -1;
  int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  if (src_node >= nn) return -1;
  for (int r = 0; r < n_rec; ++r)
    if (rec_nodes[r] < 0 || rec_nodes[r] >= nn) return -1;
  double *mass = (double *)malloc(sizeof(double) * nn);
  double *u = (double *)malloc(sizeof(double) * 3 * nn);
  double *up = (double *)malloc(sizeof(double) * 3 * nn);
  double *un = (double *)malloc(sizeof(double) * 3 * nn);
  double *w = (double *)malloc(sizeof(double) * 3 * nn);
  double *f = (double *)malloc(sizeof(double) * 3 * nn);
  char *fixed = (char *)malloc((size_t)nn);
  const double a = 0.5 * alpha * dt, b = beta / dt;
  int rc = -1;
  if (!mass || !u || !up || !un || !w || !f || !fixed) goto done;
  if (oracle_node_mass(kind, nx, ny, nz, ds, mat, table, n_mat, mass)) goto done;
  for (int64_t n = 0; n < nn; ++n) {
    fixed[n] = node_fixed(fix_bottom, nx, ny, n, mass[n]);
  }
  for (int64_t d = 0; d < 3 * nn; ++d) {
    u[d] = u0 ? u0[d] : 0.0;
    up[d] = um1 ? um1[d] : 0.0;
    if (fixed[d / 3]) u[d] = up[d] = 0.0;
  }
  for (int it = 0; it < nsteps; ++it) {
    /* K acts on u plus beta times the backward velocity */
    for (int64_t d = 0; d < 3 * nn; ++d) w[d] = u[d] + b * (u[d] - up[d]);
    if (oracle_ku(kind, nx, ny, nz, ds, mat, table, n_mat, 0, w, f)) goto done;
    double fsrc = src_node >= 0 ? amp * oracle_ricker(it * dt, f0, t0) : 0.0;
    for (int64_t n = 0; n < nn; ++n)
      for (int c = 0; c < 3; ++c) {
        int64_t d = 3 * n + c;
        if (fixed[n]) { un[d] = 0.0; continue; }
        double F = (n == src_node) ? fsrc * src_dir[c] : 0.0;
        un[d] = (2.0 * u[d] - (1.0 - a) * up[d] + dt * dt / mass[n] * (F - f[d])) / (1.0 + a);
      }
    for (int r = 0; r < n_rec; ++r)
      for (int c = 0; c < 3; ++c)
        traces[((int64_t)it * n_rec + r) * 3 + c] = un[3 * rec_nodes[r] + c];
    double *t = up; up = u; u = un; un = t;
  }
  if (u_out) memcpy(u_out, u, sizeof(double) * 3 * nn);
  if (um1_out) memcpy(um1_out, up, sizeof(double) * 3 * nn);
  rc = 0;
done:
  free(mass); free(u); free(up); free(un); free(w); free(f); free(fixed);
  return rc;
}

/* ---------- adjoint-state gradient (plain loops, all states stored) ------ */

int oracle_misfit_gradient(int kind, int nx, int ny, int nz, double ds,
                           const int32_t *mat, const double *table, int n_mat,
                           int fix_bottom, double dt, int nsteps,
                           int64_t src_node, const double *src_dir, double f0,
                           double t0, double amp, int n_rec,
                           const int64_t *rec_nodes, const double *data,
                           double *grad, double *misfit) {
  if (check_mesh(nx, ny, nz, mat, n_mat) || nsteps < 1 || n_rec < 1 || !data || !grad) return -1;
  const int N = nsteps;
  int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1), ne = (int64_t)nx * ny * nz;
  size_t sz = 3 * (size_t)nn;
  double *U = (double *)calloc(sz * (size_t)(N + 1), sizeof(double)); /* u^0 .. u^N */
  double *tr = (double *)malloc(sizeof(double) * 3 * (size_t)n_rec * N);
  double *mass = (double *)malloc(sizeof(double) * nn);
  double *mu0 = (double *)calloc(sz, sizeof(double));  /* mu^{m+1} */
  double *mu1 = (double *)calloc(sz, sizeof(double));  /* mu^m */
  double *mu2 = (double *)calloc(sz, sizeof(double));  /* mu^{m-1} */
  double *Kmu = (double *)malloc(sizeof(double) * sz);
  double *g = (double *)malloc(sizeof(double) * sz);
  double *Kg = (double *)malloc(sizeof(double) * 576 * n_mat);
  char *fixed = (char *)malloc((size_t)nn);
  int rc = -1;
  if (!U || !tr || !mass || !mu0 || !mu1 || !mu2 || !Kmu || !g || !Kg || !fixed) goto done;
  if (oracle_node_mass(kind, nx, ny, nz, ds, mat, table, n_mat, mass)) goto done;
  for (int64_t n = 0; n < nn; ++n) {
    fixed[n] = node_fixed(fix_bottom, nx, ny, n, mass[n]);
  }
  /* forward: the same run as oracle_run, keeping every state */
  for (int it = 0; it < N; ++it) {
    double *u = U + sz * it, *un = U + sz * (it + 1);
    const double *up = it > 0 ? U + sz * (it - 1) : U;  /* u^{-1} = u^0 = 0 */
    if (oracle_ku(kind, nx, ny, nz, ds, mat, table, n_mat, 0, u, Kmu)) goto done;
    double fsrc = src_node >= 0 ? amp * oracle_ricker(it * dt, f0, t0) : 0.0;
    for (int64_t n = 0; n < nn; ++n)
      for (int c = 0; c < 3; ++c) {
        int64_t d = 3 * n + c;
        if (fixed[n]) { un[d] = 0.0; continue; }
        double F = (n == src_node) ? fsrc * src_dir[c] : 0.0;
        un[d] = 2.0 * u[d] - up[d] + dt * dt / mass[n] * (F - Kmu[d]);
      }
    for (int r = 0; r < n_rec; ++r)
      for (int c = 0; c < 3; ++c)
        tr[((int64_t)it * n_rec + r) * 3 + c] = un[3 * rec_nodes[r] + c];
  }
  double J = 0.0;
  for (int64_t q = 0; q < 3 * (int64_t)n_rec * N; ++q) J += 0.5 * (tr[q] - data[q]) * (tr[q] - data[q]);
  if (misfit) *misfit = J;
  /* dK_e/dG at fixed kappa for each material's element size (same for all) */
  if (oracle_element_stiffness(kind, ds, 0.0, 1.0, Kg)) goto done;
  for (int64_t e = 0; e < ne; ++e) grad[e] = 0.0;
  /* backward: m = N .. 1 produces mu^{m-1}; then the n = m-1 gradient term */
  for (int m = N; m >= 1; --m) {
    /* g = dJ/du^m: residual of trace row m-1 at the receiver nodes */
    for (size_t q = 0; q < sz; ++q) g[q] = 0.0;
    for (int r = 0; r < n_rec; ++r)
      for (int c = 0; c < 3; ++c) {
        int64_t q = ((int64_t)(m - 1) * n_rec + r) * 3 + c;
        g[3 * rec_nodes[r] + c] += tr[q] - data[q];
      }
    if (oracle_ku(kind, nx, ny, nz, ds, mat, table, n_mat, 0, mu1, Kmu)) goto done;
    for (int64_t n = 0; n < nn; ++n)
      for (int c = 0; c < 3; ++c) {
        int64_t d = 3 * n + c;
        mu2[d] = fixed[n] ? 0.0
                          : 2.0 * mu1[d] - mu0[d] - dt * dt / mass[n] * Kmu[d] - g[d] / mass[n];
      }
    /* dJ/dG_e += dt^2 mu^{m-1}_e . dK_e/dG u^{m-1}_e */
    const double *u = U + sz * (m - 1);
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
          if (mat[e] < 0) continue;
          double ue[24], me[24];
          for (int a = 0; a < 8; ++a) {
            int64_t nd = node_id(nx, ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
            for (int c = 0; c < 3; ++c) { ue[3 * a + c] = u[3 * nd + c]; me[3 * a + c] = mu2[3 * nd + c]; }
          }
          double acc = 0.0;
          for (int rr = 0; rr < 24; ++rr) {
            double kr = 0.0;
            for (int s2 = 0; s2 < 24; ++s2) kr += Kg[rr * 24 + s2] * ue[s2];
            acc += me[rr] * kr;
          }
          grad[e] += dt * dt * acc;
        }
    double *t = mu0; mu0 = mu1; mu1 = mu2; mu2 = t;
  }
  rc = 0;
done:
  free(U); free(tr); free(mass); free(mu0); free(mu1); free(mu2); free(Kmu); free(g); free(Kg);
  free(fixed);
  return rc;
}
