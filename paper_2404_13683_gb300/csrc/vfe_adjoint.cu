// vfe_adjoint.cu -- kernels of the adjoint-state gradient (the paper's
// internal-structure estimation use, Section 1).
//
// For the central-difference run R^n = u^{n+1} - 2u^n + u^{n-1} + dt^2 M^-1
// (K u^n - F^n) = 0 and the receiver misfit J = 1/2 sum_n |u^{n+1}(r) - d^n|^2,
// the multipliers obey the same leapfrog backward in time,
//   mu^{m-1} = 2 mu^m - mu^{m+1} - dt^2 M^-1 K mu^m - M^-1 dJ/du^m,
// and dJ/dG_e = dt^2 sum_n mu^n_e . (dK_e/dG) u^n_e at fixed kappa_e.  The
// leapfrog steps run in the ordinary step kernels (with the residual injected
// at the receivers); these kernels convert states and accumulate the sum.
#include "vfe_internal.h"

// fixed-point state (padded SoA, u = U 2^-F, F = persist[0] + extra) -> FP64 [nn][3]
__global__ void tc_state_to_f64_kernel(const int64_t *U, const int64_t *persist, int extra_shift,
                                       int nx, int ny, int64_t nn, int nxp, int64_t plane,
                                       int64_t comp, double *out) {
  const int F = (int)persist[0] + extra_shift;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nn;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = n % (nx + 1), j = (n / (nx + 1)) % (ny + 1),
                  k = n / ((int64_t)(nx + 1) * (ny + 1));
    const int64_t t = k * plane + j * nxp + i;
    for (int c = 0; c < 3; ++c) out[3 * n + c] = ldexp((double)U[c * comp + t], -F);
  }
}

// grad[e] += scale * mu_e . (dK_e/dG) u_e for every solid element, at fixed
// kappa_e (lambda = kappa - 2G/3, so dlambda/dG = -2/3).  Both voxel elements
// (Section 2) have entries K_(a,i),(b,j) = ds [lambda S_ij + G S_ji + G delta_ij
// sum_k S_kk] with S_kl(a,b) = 1/16 s^a_k s^b_l prod_{m not in {k,l}} (1 +
// alpha s^a_m s^b_m), where s^a in {-1,1}^3 are the local node signs and alpha
// = 3/4 (orthogonal element) or 1/3 (trilinear element).  Summing over the
// nodes first, the bilinear form needs only the 8-point Walsh-Hadamard
// coefficients W_v[i][T] = sum_a prod_{m in T} s^a_m v_(a,i) (T a subset of the
// axes, a bit mask) of mu_e and u_e:
//   16/ds mu.(dK/dG)u = -2/3 X + Y + D/3 + Z,
//   X = sum_{i!=j} W_mu[i][i] W_u[j][j] + alpha W_mu[i][ip] W_u[j][jp],
//   Y = sum_{i!=j} W_mu[i][j] W_u[j][i] + alpha W_mu[i][jp] W_u[j][ip],
//   D = sum_i W_mu[i][i] W_u[i][i] + alpha (W_mu[i][im] W_u[i][im] + W_mu[i][in]
//       W_u[i][in]) + alpha^2 W_mu[i][xyz] W_u[i][xyz],
//   Z = sum_i sum_T |T| alpha^(|T|-1) W_mu[i][T] W_u[i][T],
// (p the third axis of i != j; m, n the two axes other than i): about 60
// multiply-adds and 140 additions instead of the 600 multiply-adds of the dense
// 24x24 form.
__device__ __forceinline__ void wht8(double *v) {  // in place; index = T afterwards
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!((a >> m) & 1)) {
        const double lo = v[a], hi = v[a | (1 << m)];
        v[a] = hi + lo;           // the subsets without axis m
        v[a | (1 << m)] = hi - lo;  // with axis m: s = +1 on the upper node
      }
}

__global__ void __launch_bounds__(256) grad_g_kernel(int nx, int ny, int nz, const int32_t *mat,
                                                     double alpha, const double *u,
                                                     const double *mu, double scale,
                                                     double *grad) {
  const int64_t ne = (int64_t)nx * ny * nz;
  const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
  const double a2 = alpha * alpha;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (mat[e] < 0) continue;
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    double M[3][8], U[3][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t nb = (ex + (a & 1)) + sx * (ey + ((a >> 1) & 1)) + sxy * (ez + (a >> 2));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        M[c][a] = mu[3 * nb + c];
        U[c][a] = u[3 * nb + c];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      wht8(M[c]);
      wht8(U[c]);
    }
    double X = 0.0, Y = 0.0, D = 0.0, Z = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int bi = 1 << i;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (j == i) continue;
        const int bj = 1 << j, bp = 7 ^ bi ^ bj;
        X = fma(M[i][bi], U[j][bj], X);
        X = fma(alpha * M[i][bi | bp], U[j][bj | bp], X);
        Y = fma(M[i][bj], U[j][bi], Y);
        Y = fma(alpha * M[i][bj | bp], U[j][bi | bp], Y);
      }
      const int bm = 1 << ((i + 1) % 3), bn = 1 << ((i + 2) % 3);
      D = fma(M[i][bi], U[i][bi], D);
      D = fma(alpha * M[i][bi | bm], U[i][bi | bm], D);
      D = fma(alpha * M[i][bi | bn], U[i][bi | bn], D);
      D = fma(a2 * M[i][7], U[i][7], D);
#pragma unroll
      for (int T = 1; T < 8; ++T) {
        const int n = (T & 1) + ((T >> 1) & 1) + ((T >> 2) & 1);
        const double w = n == 1 ? 1.0 : (n == 2 ? 2.0 * alpha : 3.0 * a2);
        Z = fma(w * M[i][T], U[i][T], Z);
      }
    }
    grad[e] += scale * (Y + Z + (D - 2.0 * X) * (1.0 / 3.0));
  }
}

// The same sum on the tensor-core path, from the fixed-point states directly
// (u = U 2^-Fu, mu = Mu 2^-Fm, padded SoA layout) and in integer arithmetic:
// the orthogonal element's alpha = 3/4 makes 48 (16/ds) mu.(dK/dG)u an
// integer combination of the products W_mu[i][T] W_u[j][T'] (coefficients
// -32 and -24 for X, 48 and 36 for Y, 16, 12 and 9 for D, 48, 72 and 81 for
// Z).  The Walsh-Hadamard sums are exact in int64 on U >> 3 (|U| < 2^62);
// each state's 24 coefficients of the element are then cut to 31 bits below
// the largest of them (W >> s, one s per element and state), the 57 products
// of two such are split at bit 31 and the halves summed separately, so
// nothing overflows (57 x 81 x 2^31 < 2^44), and one FP64 conversion per
// element and step carries the result, 2^(6 + s_u + s_mu) 2^-(Fu + Fm) ds /
// (16 48) dt^2, into the gradient.  The cut costs at most 2^-30 of the
// element's largest coefficient, far below the accuracy the states carry.
__device__ __forceinline__ void wht8_i64(int64_t *v) {
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!((a >> m) & 1)) {
        const int64_t lo = v[a], hi = v[a | (1 << m)];
        v[a] = hi + lo;
        v[a | (1 << m)] = hi - lo;
      }
}

__global__ void __launch_bounds__(256) grad_g_tc_kernel(int nx, int ny, int nz, const int32_t *mat,
                                                        const int64_t *Uf, const int64_t *Fu,
                                                        const int64_t *Mu, const int64_t *Fm,
                                                        int nxp, int64_t plane, int64_t comp,
                                                        double scale, double *grad) {
  const int64_t ne = (int64_t)nx * ny * nz;
  const int fexp = 6 - (int)(*Fu) - (int)(*Fm);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (mat[e] < 0) continue;
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    int64_t wm[3][8], wu[3][8];
    uint64_t om = 0, ou = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t t = c * comp + (ez + (a >> 2)) * plane + (ey + ((a >> 1) & 1)) * nxp +
                          (ex + (a & 1));
        wm[c][a] = Mu[t] >> 3;
        wu[c][a] = Uf[t] >> 3;
      }
      wht8_i64(wm[c]);
      wht8_i64(wu[c]);
#pragma unroll
      for (int T = 0; T < 8; ++T) {
        om |= (uint64_t)(wm[c][T] ^ (wm[c][T] >> 63));
        ou |= (uint64_t)(wu[c][T] ^ (wu[c][T] >> 63));
      }
    }
    // |W| < 2^b: keep 31 bits below the top (W >> s lies in [-2^31, 2^31))
    const int sm = max(0, (64 - __clzll((long long)om)) - 31);
    const int su = max(0, (64 - __clzll((long long)ou)) - 31);
    int M[3][8], U[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int T = 0; T < 8; ++T) {
        M[c][T] = (int)(wm[c][T] >> sm);
        U[c][T] = (int)(wu[c][T] >> su);
      }
    int64_t hi = 0, lo = 0;
    auto term = [&](int coef, int a, int b) {
      const int64_t p = (int64_t)a * (int64_t)b;
      hi += (int64_t)coef * (p >> 31);
      lo += (int64_t)coef * (p & 0x7FFFFFFF);
    };
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int bi = 1 << i;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (j == i) continue;
        const int bj = 1 << j, bp = 7 ^ bi ^ bj;
        term(-32, M[i][bi], U[j][bj]);             // X
        term(-24, M[i][bi | bp], U[j][bj | bp]);
        term(48, M[i][bj], U[j][bi]);              // Y
        term(36, M[i][bj | bp], U[j][bi | bp]);
      }
      const int bm = 1 << ((i + 1) % 3), bn = 1 << ((i + 2) % 3);
      term(16, M[i][bi], U[i][bi]);                // D
      term(12, M[i][bi | bm], U[i][bi | bm]);
      term(12, M[i][bi | bn], U[i][bi | bn]);
      term(9, M[i][7], U[i][7]);
#pragma unroll
      for (int T = 1; T < 8; ++T) {                // Z
        const int n = (T & 1) + ((T >> 1) & 1) + ((T >> 2) & 1);
        term(n == 1 ? 48 : (n == 2 ? 72 : 81), M[i][T], U[i][T]);
      }
    }
    grad[e] += ldexp(scale * ((double)hi * 2147483648.0 + (double)lo), fexp + sm + su);
  }
}

cudaError_t grad_g_tc_accumulate(cudaStream_t s, int nx, int ny, int nz, const int32_t *mat,
                                 double ds, const int64_t *Uf, const int64_t *Fu,
                                 const int64_t *Mu, const int64_t *Fm, int nxp, int64_t plane,
                                 int64_t comp, double scale, double *grad) {
  const int64_t ne = (int64_t)nx * ny * nz;
  const int blocks = (int)((ne + 255) / 256 < 8192 ? (ne + 255) / 256 : 8192);
  grad_g_tc_kernel<<<blocks, 256, 0, s>>>(nx, ny, nz, mat, Uf, Fu, Mu, Fm, nxp, plane, comp,
                                          scale * ds / (16.0 * 48.0), grad);
  return cudaGetLastError();
}

cudaError_t tc_state_to_f64(cudaStream_t s, const int64_t *U, const int64_t *persist,
                            int extra_shift, int nx, int ny, int64_t nn, int nxp, int64_t plane,
                            int64_t comp, double *out) {
  const int blocks = (int)((nn + 255) / 256 < 4096 ? (nn + 255) / 256 : 4096);
  tc_state_to_f64_kernel<<<blocks, 256, 0, s>>>(U, persist, extra_shift, nx, ny, nn, nxp, plane,
                                                comp, out);
  return cudaGetLastError();
}

cudaError_t grad_g_accumulate(cudaStream_t s, int nx, int ny, int nz, const int32_t *mat,
                              double alpha, double ds, const double *u, const double *mu,
                              double scale, double *grad) {
  const int64_t ne = (int64_t)nx * ny * nz;
  const int blocks = (int)((ne + 255) / 256 < 8192 ? (ne + 255) / 256 : 8192);
  grad_g_kernel<<<blocks, 256, 0, s>>>(nx, ny, nz, mat, alpha, u, mu, scale * ds / 16.0, grad);
  return cudaGetLastError();
}
