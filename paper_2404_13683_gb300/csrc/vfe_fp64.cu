// vfe_fp64.cu -- the plain FP64 CUDA-core path (baseline form).
//
// f = K u element by element in FP64 with the per-material 24x24 element
// matrices (Section 2: VFEM or OVFEM, Eq. OVFEMstiff), followed by the
// central-difference update with the diagonal mass (Eq. eqtimehistory).
// One thread per node gathers the rows of its (up to) eight elements, so the
// node sums need no atomics and the update is fused into the same pass.
// The path is FP64-bound (576 FMA per node), which is the point: it is the
// baseline the integer tensor-core path is measured against.  With Rayleigh
// damping the gather reads w^n = u^n + (beta/dt)(u^n - u^{n-1}) (kept as a
// state array, since u^{n-1} is overwritten in place) and the update divides
// by 1 + alpha dt / 2.
#include "vfe_internal.h"

struct F64StepParams {
  int64_t step;
  int64_t trace_row;
  int64_t inj_row;
  double src[3];
};

// persist[0] = step, [1] = trace rows, [2] = first step of the injection
// array (-1: none), [3] unused, [4] = first step of the explicit force series
// (-1: none), [5] unused
__global__ void f64_prologue_kernel(F64StepParams *p, int64_t *persist, TcSource sd, int have_src,
                                    int trace_on, int *status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t n = persist[0];
  F64StepParams q;
  q.step = n;
  q.trace_row = trace_on ? persist[1] : -1;
  q.inj_row = persist[2] >= 0 ? n - persist[2] : -1;
  // F^n = amp ricker(n dt) dir, or the caller's row of an explicit force series
  q.src[0] = q.src[1] = q.src[2] = 0.0;
  if (have_src && persist[4] >= 0 && sd.force) {
    const int64_t frow = n - persist[4];
    if (frow >= 0 && frow < sd.force_rows) {
      for (int c = 0; c < 3; ++c) q.src[c] = sd.force_scale * sd.force[3 * frow + c];
    } else {
      atomicOr(status, 8);  // a forced step beyond the supplied rows: no force
    }
  } else if (have_src) {
    const double fv = sd.amp_scale * ricker_wavelet((double)n * sd.dt, sd.f0, sd.t0);
    for (int c = 0; c < 3; ++c) q.src[c] = fv * sd.dir[c];
  }
  *p = q;
  persist[0] = n + 1;
  if (trace_on) persist[1] += 1;
}

template <int MODE>
__global__ void __launch_bounds__(256) f64_step_kernel(const F64Device d, const F64StepParams *pp) {
  extern __shared__ double sK[];
  // per-material element matrices, or Kk, Kg with per-element shear moduli
  const bool per_elem = d.elem_G != nullptr;
  const int nK = per_elem ? 2 * 576 : d.n_mat * 576;
  const double *Ksrc = per_elem ? d.Kkg : d.K;
  for (int i = threadIdx.x; i < nK; i += blockDim.x) sK[i] = Ksrc[i];
  __syncthreads();
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < d.nn;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int ni = (int)(n % sx), nj = (int)((n / sx) % (ny + 1)), nk = (int)(n / sxy);
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    const double *x = d.damped ? d.w : d.u;  // the vector K acts on
    for (int a = 0; a < 8; ++a) {
      const int ex = ni - (a & 1), ey = nj - ((a >> 1) & 1), ez = nk - (a >> 2);
      if (ex < 0 || ey < 0 || ez < 0 || ex >= nx || ey >= ny || ez >= nz) continue;
      const int64_t e = (int64_t)ex + (int64_t)nx * ((int64_t)ey + (int64_t)ny * ez);
      const int m = d.mat[e];
      if (m < 0) continue;
      if (per_elem) {  // kappa_m (Kk u_e) + G_e (Kg u_e)
        const double *Kk = sK + (3 * a) * 24, *Kg = sK + 576 + (3 * a) * 24;
        double g0 = 0.0, g1 = 0.0, g2 = 0.0, h0 = 0.0, h1 = 0.0, h2 = 0.0;
        for (int b = 0; b < 8; ++b) {
          const int64_t nb = (ex + (b & 1)) + sx * (ey + ((b >> 1) & 1)) + sxy * (ez + (b >> 2));
          const double u0 = x[3 * nb], u1 = x[3 * nb + 1], u2 = x[3 * nb + 2];
          const double *k0 = Kk + 3 * b, *k1 = Kk + 24 + 3 * b, *k2 = Kk + 48 + 3 * b;
          g0 = fma(k0[0], u0, fma(k0[1], u1, fma(k0[2], u2, g0)));
          g1 = fma(k1[0], u0, fma(k1[1], u1, fma(k1[2], u2, g1)));
          g2 = fma(k2[0], u0, fma(k2[1], u1, fma(k2[2], u2, g2)));
          const double *q0 = Kg + 3 * b, *q1 = Kg + 24 + 3 * b, *q2 = Kg + 48 + 3 * b;
          h0 = fma(q0[0], u0, fma(q0[1], u1, fma(q0[2], u2, h0)));
          h1 = fma(q1[0], u0, fma(q1[1], u1, fma(q1[2], u2, h1)));
          h2 = fma(q2[0], u0, fma(q2[1], u1, fma(q2[2], u2, h2)));
        }
        const double kap = d.kappa[m], G = d.elem_G[e];
        f0 = fma(kap, g0, fma(G, h0, f0));
        f1 = fma(kap, g1, fma(G, h1, f1));
        f2 = fma(kap, g2, fma(G, h2, f2));
        continue;
      }
      const double *K = sK + m * 576 + (3 * a) * 24;
      for (int b = 0; b < 8; ++b) {
        const int64_t nb = (ex + (b & 1)) + sx * (ey + ((b >> 1) & 1)) + sxy * (ez + (b >> 2));
        const double u0 = x[3 * nb], u1 = x[3 * nb + 1], u2 = x[3 * nb + 2];
        const double *k0 = K + 3 * b, *k1 = K + 24 + 3 * b, *k2 = K + 48 + 3 * b;
        f0 = fma(k0[0], u0, fma(k0[1], u1, fma(k0[2], u2, f0)));
        f1 = fma(k1[0], u0, fma(k1[1], u1, fma(k1[2], u2, f1)));
        f2 = fma(k2[0], u0, fma(k2[1], u1, fma(k2[2], u2, f2)));
      }
    }
    if (MODE == 1) {
      d.f_out[3 * n] = f0;
      d.f_out[3 * n + 1] = f1;
      d.f_out[3 * n + 2] = f2;
      continue;
    }
    const F64StepParams p = *pp;
    const double c = d.dt2_m[n];
    const bool src = (n == d.src_node);
    const double fv[3] = {f0, f1, f2};
    double un[3];
    for (int k = 0; k < 3; ++k) {
      const double F = src ? p.src[k] : 0.0;
      if (d.damped)
        un[k] = (2.0 * d.u[3 * n + k] - (1.0 - d.da) * d.u_prev[3 * n + k] + c * (F - fv[k])) /
                (1.0 + d.da);
      else
        un[k] = 2.0 * d.u[3 * n + k] - d.u_prev[3 * n + k] + c * (F - fv[k]);
    }
    if (p.inj_row >= 0)  // injected increments at receiver nodes (adjoint source)
      for (int r = 0; r < d.n_rec; ++r)
        if (d.recv_nodes[r] == n)
          for (int k = 0; k < 3; ++k) un[k] += d.inj[(p.inj_row * d.n_rec + r) * 3 + k];
    for (int k = 0; k < 3; ++k) {
      if (c == 0.0) un[k] = 0.0;
      if (d.damped) d.w_next[3 * n + k] = un[k] + d.db * (un[k] - d.u[3 * n + k]);
      d.u_next[3 * n + k] = un[k];
    }
    if (p.trace_row >= 0) {
      for (int r = 0; r < d.n_rec; ++r)
        if (d.recv_nodes[r] == n)
          for (int k = 0; k < 3; ++k) d.traces[(p.trace_row * d.n_rec + r) * 3 + k] = un[k];
    }
  }
}

cudaError_t f64_prepare() {
  const int smem = F64_MAX_MAT * 576 * (int)sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(f64_step_kernel<0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(f64_step_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem);
}

template <int MODE>
static cudaError_t f64_launch(cudaStream_t s, const F64Device &d, const F64StepParams *pp) {
  const int smem = (d.elem_G ? 2 : d.n_mat) * 576 * (int)sizeof(double);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (d.nn + 255) / 256;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (blocks < 1) blocks = 1;
  f64_step_kernel<MODE><<<(unsigned)blocks, 256, smem, s>>>(d, pp);
  return cudaGetLastError();
}

size_t f64_params_bytes() { return sizeof(F64StepParams); }

cudaError_t f64_launch_prologue(cudaStream_t s, void *params, int64_t *persist,
                                const TcSource &src, int have_src, int trace_on, int *status) {
  f64_prologue_kernel<<<1, 32, 0, s>>>(reinterpret_cast<F64StepParams *>(params), persist, src,
                                       have_src, trace_on, status);
  return cudaGetLastError();
}

cudaError_t f64_launch_step(cudaStream_t s, const F64Device &d, const void *params, int mode) {
  const F64StepParams *pp = reinterpret_cast<const F64StepParams *>(params);
  return mode == 1 ? f64_launch<1>(s, d, pp) : f64_launch<0>(s, d, pp);
}
