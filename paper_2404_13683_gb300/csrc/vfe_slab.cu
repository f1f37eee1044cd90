// vfe_slab.cu -- node-plane exchange for the z-slab decomposition of a mesh
// over several GPUs (the paper's closing remark that the method extends to
// many GPUs, Section 4).  A slab's step needs u^n on the node plane below and
// above its own planes; these kernels copy one node plane of the state out as
// FP64 and write a received FP64 plane into the state.  On the tensor-core
// path the state is the 64-bit fixed point U = u 2^F of the mesh (F in the
// persistent step record); a received plane is rounded into the receiver's
// own unit and its magnitudes are ORed into the bound records from which the
// next step picks its digit quantum (one word per 15x15 node column and one
// for the whole mesh), as the step kernels do for the planes they update.
#include "vfe_internal.h"

namespace {

// FP64 [(ny+1)(nx+1)][3] <- U plane k (padded SoA, unit 2^-F)
__global__ void pack_plane_tc_kernel(const int64_t *U, int nx, int ny, int nxp, int64_t plane,
                                     int64_t comp, int k, const int64_t *persist, double *out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t np = (int64_t)(nx + 1) * (ny + 1);
  if (n >= np) return;
  const int F = (int)persist[0];
  const int64_t i = n % (nx + 1), j = n / (nx + 1);
  const int64_t t = (int64_t)k * plane + j * nxp + i;
#pragma unroll
  for (int c = 0; c < 3; ++c) out[3 * n + c] = ldexp((double)U[c * comp + t], -F);
}

// U plane k <- round(in 2^F); |U| ORed into the column bounds and the global
// bound of the slot the next step reads
__global__ void unpack_plane_tc_kernel(int64_t *U, int nx, int ny, int nxp, int64_t plane,
                                       int64_t comp, int k, const int64_t *persist,
                                       const double *in, unsigned long long *slot, int tiles_x) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t np = (int64_t)(nx + 1) * (ny + 1);
  unsigned long long o = 0;
  if (n < np) {
    const int F = (int)persist[0];
    const int64_t i = n % (nx + 1), j = n / (nx + 1);
    const int64_t t = (int64_t)k * plane + j * nxp + i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t v = llrint(ldexp(in[3 * n + c], F));
      U[c * comp + t] = v;
      o |= (unsigned long long)(v < 0 ? -v : v);
    }
    if (o) atomicOr(&slot[1 + (j / TC_OWN) * tiles_x + (i / TC_OWN)], o);
  }
  for (int s = 16; s > 0; s >>= 1) o |= __shfl_xor_sync(0xffffffffu, o, s);
  if ((threadIdx.x & 31) == 0 && o) atomicOr(&slot[0], o);
}

}  // namespace

cudaError_t slab_pack_tc(cudaStream_t s, const int64_t *U, int nx, int ny, int nxp, int64_t plane,
                         int64_t comp, int k, const int64_t *persist, double *out) {
  const int64_t np = (int64_t)(nx + 1) * (ny + 1);
  pack_plane_tc_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(U, nx, ny, nxp, plane, comp, k,
                                                                    persist, out);
  return cudaGetLastError();
}

cudaError_t slab_unpack_tc(cudaStream_t s, int64_t *U, int nx, int ny, int nxp, int64_t plane,
                           int64_t comp, int k, const int64_t *persist, const double *in,
                           unsigned long long *slot, int tiles_x) {
  const int64_t np = (int64_t)(nx + 1) * (ny + 1);
  unpack_plane_tc_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(U, nx, ny, nxp, plane, comp,
                                                                      k, persist, in, slot,
                                                                      tiles_x);
  return cudaGetLastError();
}
