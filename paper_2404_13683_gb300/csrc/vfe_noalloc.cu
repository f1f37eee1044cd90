// vfe_noalloc.cu -- K u on the tensor-core path without any allocation.
//
// Some callers cannot allocate device memory: code that runs inside a host
// framework owning the whole device pool (allocation would fragment or exceed
// its budget), callers in real-time loops where cudaMalloc's implicit
// synchronisation is not allowed, and embedded uses that pre-budget every
// byte at start-up.  vfe_internal_force_noalloc gives them the K u product of
// the tensor-core path with every temporary in one fixed device array that
// this file declares statically, so the call performs no cudaMalloc,
// cudaFree or other allocating routine.
//
// The array is a file-scope __device__ variable: each GPU that loads the
// library holds VFE_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Host code cannot use the variable's name as a device address (it is a
// host-side stand-in), so the first call on each device, with that device
// current, asks cudaGetSymbolAddress for the real address and caches it.
// That first call should therefore happen before any stream capture.
//
// All calls share the one array and it keeps whatever the last call left in
// it: everything that must start at zero is cleared by each call, and calls
// whose work overlaps on a GPU (other threads, other streams) race on it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "vfe_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[VFE_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

int set_err(int code, const char *msg) {
  vfe_set_last_error(msg);
  return code;
}

// Layout of the array: [0, 256) header {max |u| bits, TcStepParams},
// then two int64 regions of 3*comp entries each (A, B).
constexpr size_t kHeader = 256;

__global__ void noalloc_maxabs_kernel(const double *u, int64_t n, unsigned long long *maxbits) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    // |u| as unsigned bits orders like the value for finite doubles
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(u[i]));
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(maxbits, m);
}

// u (FP64, [nn][3]) -> fixed point U = round(u 2^F) in the padded SoA layout,
// with F such that max|u| 2^F lies in [2^(TC_UNITS_BITS-1), 2^TC_UNITS_BITS);
// block 0 / thread 0 also writes the K u kernel's parameters.
__global__ void noalloc_to_fixed_kernel(const double *u, int nx, int ny, int64_t nn, int nxp,
                                        int64_t plane, int64_t comp,
                                        const unsigned long long *maxbits, int64_t *U,
                                        TcStepParams *params) {
  const double mx = __longlong_as_double((long long)*maxbits);
  const int F = mx > 0.0 ? (TC_UNITS_BITS - 1) - ilogb(mx) : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long top = mx > 0.0 ? llrint(ldexp(mx, F)) : 0;
    const int b = top ? 64 - __clzll(top) : 0;
    TcStepParams p;
    p.step = 0;
    p.trace_row = -1;
    p.dU_src[0] = p.dU_src[1] = p.dU_src[2] = 0;
    p.rs = 0;
    p.shq = b > TC_QBITS ? b - TC_QBITS : 0;
    p.R = 0;
    p.F = F;
    p.or_slot = 0;
    p.rs_prev = 0;
    *params = p;
  }
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nn;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = n % (nx + 1), j = (n / (nx + 1)) % (ny + 1), k = n / ((int64_t)(nx + 1) * (ny + 1));
    const int64_t t = k * plane + j * nxp + i;
    for (int c = 0; c < 3; ++c) U[c * comp + t] = llrint(ldexp(u[3 * n + c], F));
  }
}

// S (padded SoA, unit 2^(63 - e_ref + shq - F)) -> f FP64 [nn][3]
__global__ void noalloc_from_fixed_kernel(const int64_t *S, int nx, int ny, int64_t nn, int nxp,
                                          int64_t plane, int64_t comp, int e_ref,
                                          const TcStepParams *params, double *f) {
  const int ex = 63 - e_ref + params->shq - params->F;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nn;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = n % (nx + 1), j = (n / (nx + 1)) % (ny + 1), k = n / ((int64_t)(nx + 1) * (ny + 1));
    const int64_t t = k * plane + j * nxp + i;
    for (int c = 0; c < 3; ++c) f[3 * n + c] = ldexp((double)S[c * comp + t], ex);
  }
}

#define NA_TRY(expr)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      char m_[256];                                                                         \
      snprintf(m_, sizeof(m_), "%s failed: %s", #expr, cudaGetErrorString(e_));             \
      return set_err(VFE_ECUDA, m_);                                                        \
    }                                                                                       \
  } while (0)

// Puts the caller's current device back when the call returns.
struct DeviceRestore {
  int prev = -1;
  DeviceRestore() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~DeviceRestore() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// the device address of the array on the current device (set up once)
int scratch_address(int device, unsigned char **out) {
  if (device < 0 || device >= kMaxDevices) return set_err(VFE_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      char m[256];
      snprintf(m, sizeof(m), "cudaGetSymbolAddress of the no-alloc scratch failed: %s",
               cudaGetErrorString(e));
      return set_err(VFE_ECUDA, m);
    }
    g_scratch_ptr[device] = p;
  }
  *out = static_cast<unsigned char *>(g_scratch_ptr[device]);
  return VFE_OK;
}

}  // namespace

extern "C" {

int vfe_internal_force_noalloc(vfe_mesh *mesh, const double *u, double *f) {
  if (!mesh || !u || !f) return set_err(VFE_EINVAL, "NULL argument");
  VfeMeshView v;
  if (vfe_mesh_view(mesh, &v) != VFE_OK) return set_err(VFE_EINVAL, "bad mesh");
  if (!v.tc) return set_err(VFE_ESTATE, "the no-alloc K u needs a mesh on the tensor-core path");
  // a NaN or an infinity would make the fixed-point scale meaningless
  for (int64_t i = 0; i < 3 * v.nn; ++i)
    if (!std::isfinite(u[i])) return set_err(VFE_EINVAL, "u has non-finite values");
  const size_t region = sizeof(int64_t) * 3 * (size_t)v.comp;
  const size_t need = kHeader + 2 * region;
  if (need > (size_t)VFE_NOALLOC_SCRATCH_BYTES) {
    char m[256];
    snprintf(m, sizeof(m),
             "mesh needs %zu bytes of no-alloc scratch, more than the fixed %zu-byte array",
             need, (size_t)VFE_NOALLOC_SCRATCH_BYTES);
    return set_err(VFE_EINVAL, m);
  }
  DeviceRestore restore;
  NA_TRY(cudaSetDevice(v.device));
  unsigned char *base = nullptr;
  int rc = scratch_address(v.device, &base);
  if (rc != VFE_OK) return rc;
  unsigned long long *maxbits = reinterpret_cast<unsigned long long *>(base);
  TcStepParams *params = reinterpret_cast<TcStepParams *>(base + 64);
  int64_t *regA = reinterpret_cast<int64_t *>(base + kHeader);
  int64_t *regB = reinterpret_cast<int64_t *>(base + kHeader + region);
  cudaStream_t s = v.stream;
  const int64_t n3 = 3 * v.nn;

  // u -> region B (FP64 AoS); clear the max slot and region A (its padding is
  // the halo the K u kernel reads at the mesh edges)
  NA_TRY(cudaMemcpyAsync(regB, u, sizeof(double) * n3, cudaMemcpyHostToDevice, s));
  NA_TRY(cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), s));
  NA_TRY(cudaMemsetAsync(regA, 0, region, s));
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((n3 + threads - 1) / threads, 4096);
  noalloc_maxabs_kernel<<<blocks, threads, 0, s>>>(reinterpret_cast<const double *>(regB), n3,
                                                   maxbits);
  NA_TRY(cudaGetLastError());
  noalloc_to_fixed_kernel<<<blocks, threads, 0, s>>>(reinterpret_cast<const double *>(regB), v.nx,
                                                     v.ny, v.nn, v.nxp, v.plane, v.comp, maxbits,
                                                     regA, params);
  NA_TRY(cudaGetLastError());
  // K u of the fixed-point copy (region A) into region B, cleared first: the
  // kernels write every node that has a solid element, the rest stay zero
  CUtensorMap map, smap;
  if (vfe_encode_state_map(&map, regA, v) != CUDA_SUCCESS ||
      vfe_encode_state_map(&smap, regA, v, true) != CUDA_SUCCESS)
    return set_err(VFE_ECUDA, "cuTensorMapEncodeTiled failed for the no-alloc scratch");
  NA_TRY(cudaMemsetAsync(regB, 0, region, s));
  TcDevice d = v.dev;
  d.params = params;
  d.src_node = -1;
  d.n_rec = 0;
  d.S_out = regB;
  d.partials_out = nullptr;
  if (d.n_ctas > 0) NA_TRY(tc_launch_step(s, d, &map, TC_MODE_KU));
  if (v.stencil_on) {
    TcDevice ds = v.st;
    ds.params = params;
    ds.S_out = regB;
    ds.U_cur = regA;  // u^n for the per-node corrections
    NA_TRY(stencil_launch(s, ds, &smap, TC_MODE_KU));
    NA_TRY(stencil_fix(s, ds, TC_MODE_KU));
  }
  // S -> f (FP64 AoS) in region A, then to the caller
  noalloc_from_fixed_kernel<<<blocks, threads, 0, s>>>(regB, v.nx, v.ny, v.nn, v.nxp, v.plane,
                                                       v.comp, v.e_ref, params,
                                                       reinterpret_cast<double *>(regA));
  NA_TRY(cudaGetLastError());
  NA_TRY(cudaMemcpyAsync(f, regA, sizeof(double) * n3, cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaStreamSynchronize(s));
  // the kernel's status word: a bounded wait that gave up, or a failed
  // tensor-memory allocation, leaves f unwritten (read like vfe_internal_force)
  int st = 0;
  NA_TRY(cudaMemcpy(&st, v.dev.status, sizeof(int), cudaMemcpyDeviceToHost));
  char m[128];
  if (st & 1) {
    snprintf(m, sizeof(m), "a device-side wait timed out (status %d)", st);
    return set_err(VFE_ETIMEOUT, m);
  }
  if (st & 2) {
    snprintf(m, sizeof(m), "fixed-point shift out of range (status %d)", st);
    return set_err(VFE_ETIMEOUT, m);
  }
  if (st & 4) {
    snprintf(m, sizeof(m), "tensor-memory allocation failed (status %d)", st);
    return set_err(VFE_ECUDA, m);
  }
  if (st & 8) {
    snprintf(m, sizeof(m), "a forced step ran past the supplied force rows (status %d)", st);
    return set_err(VFE_ESTATE, m);
  }
  return VFE_OK;
}

}  // extern "C"
