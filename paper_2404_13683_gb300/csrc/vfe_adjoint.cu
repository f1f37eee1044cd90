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

// grad[e] += scale * mu_e^T Kg u_e for every solid element (Kg = dK_e/dG)
__global__ void __launch_bounds__(256) grad_g_kernel(int nx, int ny, int nz, const int32_t *mat,
                                                     const double *Kg, const double *u,
                                                     const double *mu, double scale,
                                                     double *grad) {
  __shared__ double sK[576];
  for (int i = threadIdx.x; i < 576; i += blockDim.x) sK[i] = Kg[i];
  __syncthreads();
  const int64_t ne = (int64_t)nx * ny * nz;
  const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (mat[e] < 0) continue;
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    double ue[24], me[24];
    for (int a = 0; a < 8; ++a) {
      const int64_t nb = (ex + (a & 1)) + sx * (ey + ((a >> 1) & 1)) + sxy * (ez + (a >> 2));
      for (int c = 0; c < 3; ++c) {
        ue[3 * a + c] = u[3 * nb + c];
        me[3 * a + c] = mu[3 * nb + c];
      }
    }
    double acc = 0.0;
    for (int r = 0; r < 24; ++r) {
      double kr = 0.0;
      for (int s = 0; s < 24; ++s) kr = fma(sK[r * 24 + s], ue[s], kr);
      acc = fma(me[r], kr, acc);
    }
    grad[e] += scale * acc;
  }
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
                              const double *Kg, const double *u, const double *mu, double scale,
                              double *grad) {
  const int64_t ne = (int64_t)nx * ny * nz;
  const int blocks = (int)((ne + 255) / 256 < 8192 ? (ne + 255) / 256 : 8192);
  grad_g_kernel<<<blocks, 256, 0, s>>>(nx, ny, nz, mat, Kg, u, mu, scale, grad);
  return cudaGetLastError();
}
