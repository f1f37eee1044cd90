// vfe_stencil.cu -- tensor-core K u and central-difference step on the node
// planes whose surrounding elements all share one material.
//
// Method (arXiv 2404.13683, Section 2, Eq. GE:TC with Eqs. intscaling and
// int8comp1-int8comp2).  Where every element touching the nodes of a 15x15
// node column, on both sides of a node plane, has one material (kappa, G),
// the element products summed at a node are one 27-point integer stencil per
// part:
//     f(n) = ds (kappa/256 S^k q + G/384 (S^G q + 1024 q(n)))
// with S^k the node sum of K^kappa = 256/ds K_e(kappa=1, G=0) over the node's
// eight elements and S^G that of the paper's Kbar^G = 384/ds K_e(0, 1) - 128 I
// (the 128 I of eight elements is the 1024 q(n) term).  The inputs are the
// same integer split as the element path (q = floor(U / 2^shq), balanced
// 11-bit digits, exact in fp16); the tensor core forms the stencil sums per
// digit stage (fp32-exact: |partial sum| <= 3152 * 1024 < 2^22), and the
// epilogue recombines six words per node and stage -- the element path needs
// 48 per element -- before one material product per component.
//
// Operand layout.  An M row of an MMA is a pair of adjacent x-nodes (local
// x = 2p+1, 2p+2) of one node row; its K rows are the 4 x-shifts (local
// x = 2p .. 2p+3) x 3 components of one node row of one INPUT plane (12 of 16
// rows used).  A node row of a digit plane is one 256-byte block (8 pairs,
// MN-major core matrices: K groups at 128 B, the next node row at 256 B), so
// input row y + dy of all 128 output pairs (16 node rows x 8 pairs) is one
// descriptor.  Each MMA (M = 128, N = 48, K = 16) takes one input plane p,
// one digit stage and one dy, and its 48 columns are the contributions of
// that input to the three output planes p-1, p, p+1 (16 columns each: node
// of the pair x component x (P, Q), 8 per node).  The accumulators of a
// stage form a ring of three 16-column slots, output plane z in slot z mod 3:
// the B operand of input p starts at the rotation of its three blocks that
// puts each output in its slot, so every MMA writes all 48 columns of the
// ring and the z-sum of the stencil happens in TMEM.  A slot is read for
// plane z once input z+1 is in; before input z+2's MMAs add to it, an N = 16
// MMA without accumulation writes the magic bias 0x4B400000 (1.5 2^23) into
// it (constant K rows 12..15 of the digit block against a bias image), the
// start value for plane z+3; every accumulator word is then 0x4B400000 + the
// exact integer.  Per input plane: (1 + 3 dy) x STAGES MMAs, the dy ones
// reading their 4 KB of digits once for three outputs.
//
// A segment is a 15x15 node column (the element path's partition; the CTA
// computes 16x16 nodes and drops the 16th row and column) over two or more
// node planes.  A CTA marches up in z through its segments as one stream:
// TMA brings node planes (box 20 x 18 x 1 x 3 int64) into an 8-slot ring up
// to seven planes ahead, and the digits and MMAs of the next segment's first
// planes are made while the current one finishes, so a segment boundary
// costs no pipeline refill.  Per output plane the 8 epilogue warps read its
// TMEM slot, recombine and update the node plane while warps 8 and 13-15
// issue the MMAs of the next output's inputs (the digit stages shared out)
// and warps 9-12 digitise the inputs of the
// output after it (one CTA barrier per output plane).  Source and receiver
// planes, mesh faces and material interfaces are left to the element kernel
// (vfe_tc.cu).
#include <cuda_fp16.h>

#include <cstring>

#include "vfe_internal.h"
#include "vfe_tc_common.cuh"

using namespace vfe_tc;

namespace {

constexpr int kSX = ST_BOXX;                              // TMA box width (int64)
constexpr int kSY = ST_BOXY;                              // node rows 0..17
constexpr int kRowBytes = 256;                            // 8 pairs x 16 K rows x fp16
constexpr int kStageBytes = kSY * kRowBytes;              // 4608
constexpr int kDSlotBytes = TC_MAX_STAGES * kStageBytes;  // 23040
constexpr int kDSlots = 4;                                // digit planes L .. L+3
constexpr int kUBytes = 3 * kSY * kSX * 8;                // 8640
constexpr int kUStride = (kUBytes + 127) / 128 * 128;
constexpr int kUSlots = 8;
// B images: per (variant, dy) 16 K rows x 80 N columns (five 16-column
// blocks: outputs p-1, p, p+1, p-1, p), K-major core matrices with N groups
// at 128 B and K groups at 1280 B; variants: all outputs, none below (the
// second input plane of a segment), only above (the first)
constexpr int kBKStride = 10 * 128;
constexpr int kBImage = 2 * kBKStride;                    // 2560
constexpr int kBBytes = 9 * kBImage;
static_assert(kBBytes == ST_MASK_IDX_OFF, "the host's operand buffer: B images, then the correction table");
// the bias image: 16 K rows x 16 N columns, K rows 12..15 = 12288 (fp16),
// the rest zero; against the constant 256 in K rows 12..15 of every digit
// block it gives 4 x 256 x 12288 = 1.5 2^23 in each of the 16 columns
constexpr int kBiasBytes = 512;

constexpr int kOffD = 0;
constexpr int kOffU = kOffD + kDSlots * kDSlotBytes;
constexpr int kOffB = kOffU + kUSlots * kUStride;
constexpr int kOffBias = kOffB + kBBytes;
// the CTA's first kSegCap segments, staged once per launch: column and
// planes, and digit shift (32 bytes each); later segments are read from
// global memory where they are needed
constexpr int kSegCap = 256;
constexpr int kSegInfoBytes = 32;
constexpr int kOffSeg = kOffBias + kBiasBytes;
constexpr int kOffBar = kOffSeg + kSegCap * kSegInfoBytes;
constexpr int kOffMisc = kOffBar + 16 * 8;
// the material multipliers as 31-bit limbs {A1, A0, B1, B0}, per material
// index 0 .. TC_MAX_MAT (ST_NO_MAT: zero)
constexpr int kOffLimb = kOffMisc + 64;
constexpr int kSmemBytes = kOffLimb + (TC_MAX_MAT + 1) * 16;

static_assert(kOffU % 128 == 0 && kUStride % 128 == 0, "TMA destinations 128-byte aligned");
static_assert(kOffLimb % 16 == 0, "limb table alignment");
static_assert(kDSlotBytes % 256 == 0 && kOffB % 128 == 0 && kOffBias % 128 == 0 &&
                  kOffBar % 8 == 0,
              "alignment");
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
static_assert(kSmemBytes > 114 * 1024, "one CTA per SM (TMEM and the element kernel)");

constexpr int kThreads = 512;
constexpr int kTmemCols = 256;
constexpr int kRingCols = 48;                 // one stage: slots of planes z mod 3
constexpr int kTasks = kSY * 3 * 2;           // digitisation tasks per plane
constexpr int kEpiWarps = 8;                  // warps 0-7: epilogue (lane quarter x node)
// MMA issue: warps 8, 13, 14, 15 (ranks 0-3), stage s_lo + k from the warp
// of rank k mod 4; digitisation: warps 9-12, 27 tasks each (one warp per
// scheduler, none of them issuing MMAs)
constexpr int kMmaWarps = 4;
__device__ __forceinline__ int mma_rank_of(int warp) {
  return warp == 8 ? 0 : (warp >= 13 ? warp - 12 : -1);
}
constexpr int kDigit0 = 9 * 32;               // first digitising thread (warps 9-12)
constexpr int kDigitWarps = 4;
constexpr int kTasksPerWarp = 27;
static_assert(kDigitWarps * kTasksPerWarp == 18 * 3 * 2, "digitisation tasks per plane");
static_assert(kThreads - kDigit0 >= kTasks, "one task per digitising thread");

// kind::f16, D f32, A f16 MN-major, B f16 K-major, N = 48, M = 128
constexpr uint32_t kIdescN48 =
    (1u << 4) | (1u << 15) | ((uint32_t)(48 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
// the same with N = 16 (one ring slot)
constexpr uint32_t kIdescN16 =
    (1u << 4) | (1u << 15) | ((uint32_t)(16 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t kHalf256 = 0x5C005C00u;    // two fp16 256.0
constexpr uint32_t kHalf12288 = 0x72007200u;  // two fp16 12288.0

}  // namespace

// ---------------------------------------------------------------------------
// Per-node corrections.  The stencil kernel forms every node of its runs as
// if the eight elements around it were all of the node's reference material
// (node_mat; the material table's zero entry where the node has no solid
// element).  Where some of them are of another material, void or outside the
// mesh, one thread per such node (after the stencil kernel, on the same
// stream) forms, from the digit values q' the kernel used, the parts
// P_M = sum over the elements of octant mask M of their K^kappa rows at the
// node times q', Q_M the same with Kbar^G (the correction table's 3x3 blocks
// at the neighbour offsets the mask's elements reach; a neighbour outside
// the mesh holds zero, as in the kernel), and the identity term
// 128 |M| q'(n) of K^G', and exchanges the material of those elements:
//   dS = hi63(A_f P_M + B_f Q_M) + hi63(128 |M| q'(n) B_f) - (the same with A_r, B_r),
// f the elements' material (zero multipliers where absent), r the node's.
// The sum over the node's entries is added to S (K u) or its increment is
// taken off u^{n+1} with the update's own fixed-point arithmetic (time step),
// folding |u^{n+1}| into the column bounds again: within a few units of
// forming the corrected S at once.
// ---------------------------------------------------------------------------
// the corrections of the node whose first entry is fix[e0]; time step:
// returns the OR of |u^{n+1}| over its components and sets its column
template <int MODE>
__device__ __forceinline__ unsigned long long fix_node(const TcDevice &d, const TcStepParams &P,
                                                      int e0, int4 f, int &col) {
  const int16_t *mask_idx = reinterpret_cast<const int16_t *>(
      reinterpret_cast<const unsigned char *>(d.Bst) + ST_MASK_IDX_OFF);
  const int16_t *mask_rows = reinterpret_cast<const int16_t *>(
      reinterpret_cast<const unsigned char *>(d.Bst) + ST_MASK_ROW_OFF);
  const int64_t dbias = (1LL << 10) | (1LL << 21) | (1LL << 32) | (1LL << 43) | (1LL << 54);
  const int lo_bits = TC_DIGIT_BITS * (TC_MAX_STAGES - d.stages);
  const int64_t dbias_hi = (dbias >> lo_bits) << lo_bits;
  const int64_t *Un = d.U_cur;
  const int gi = f.x, gj = f.y, z = f.z;
  // the digit shift of the node's column, as the stencil kernel takes it
  int shq = P.shq;
  if (MODE == TC_MODE_STEP) {
    const int tx = gi / TC_OWN, ty = gj / TC_OWN;
    const unsigned long long *prev =
        d.or_slots + (size_t)((P.or_slot + 2) % 3) * (1 + d.tiles_x * d.tiles_y) + 1;
    unsigned long long o = 0;
    for (int dyc = -1; dyc <= 1; ++dyc)
      for (int dxc = -1; dxc <= 1; ++dxc) {
        const int cx = tx + dxc, cy = ty + dyc;
        if (cx >= 0 && cy >= 0 && cx < d.tiles_x && cy < d.tiles_y) o |= prev[cy * d.tiles_x + cx];
      }
    const int b = o ? 64 - __clzll((long long)o) : 0;
    shq = min(P.shq, max(0, b - TC_QBITS));
  }
  auto qprime = [&](int64_t u) -> int64_t {
    const int64_t v = (u >> shq) + dbias;
    return ((v >> lo_bits) << lo_bits) - dbias_hi;
  };
  const int64_t nidx = (int64_t)z * d.plane + (int64_t)gj * d.nxp + gi;
  int64_t qn[3];
  for (int c = 0; c < 3; ++c) qn[c] = qprime(Un[c * d.comp + nidx]);
  const TcMaterial mr = d.mats[(f.w >> 16) & 255];
  const int Ar1 = (int)(mr.A >> 31), Ar0 = (int)(mr.A & 0x7FFFFFFF);
  const int Br1 = (int)(mr.B >> 31), Br0 = (int)(mr.B & 0x7FFFFFFF);
  int64_t dS[3] = {0, 0, 0};
  for (int e = e0;;) {
    const int mask = f.w & 255;
    const int r0 = mask_idx[2 * mask], r1 = r0 + mask_idx[2 * mask + 1];
    int64_t pg[3] = {0, 0, 0}, qg[3] = {0, 0, 0};
    for (int r = r0; r < r1; ++r) {
      const int16_t *row = mask_rows + 20 * r;
      const int off = row[0];
      const int ni = gi + off % 3 - 1, nj = gj + (off / 3) % 3 - 1, nk = z + off / 9 - 1;
      if (ni < 0 || nj < 0 || nk < 0 || ni > d.nx || nj > d.ny || nk > d.nz) continue;
      const int64_t nb = (int64_t)nk * d.plane + (int64_t)nj * d.nxp + ni;
      int64_t q[3];
      for (int j = 0; j < 3; ++j) q[j] = qprime(Un[j * d.comp + nb]);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          pg[i] += (int64_t)row[1 + 3 * i + j] * q[j];
          qg[i] += (int64_t)row[10 + 3 * i + j] * q[j];
        }
    }
    const TcMaterial mf = d.mats[(f.w >> 8) & 255];
    const int Af1 = (int)(mf.A >> 31), Af0 = (int)(mf.A & 0x7FFFFFFF);
    const int Bf1 = (int)(mf.B >> 31), Bf0 = (int)(mf.B & 0x7FFFFFFF);
    const int64_t w = 128 * __popc(mask);
    for (int c = 0; c < 3; ++c)
      dS[c] += mul2_hi63(pg[c], qg[c], Af1, Af0, Bf1, Bf0) + mul_hi63(qn[c] * w, Bf1, Bf0) -
               mul2_hi63(pg[c], qg[c], Ar1, Ar0, Br1, Br0) - mul_hi63(qn[c] * w, Br1, Br0);
    if (++e >= d.n_fix) break;
    f = d.fix[e];
    if (!(f.w & ST_FIX_CONT)) break;
  }
  if (MODE == TC_MODE_KU) {
    for (int c = 0; c < 3; ++c) d.S_out[c * d.comp + nidx] += dS[c];
    return 0;
  }
  const int64_t cn = d.C[nidx];
  if (cn == 0) return 0;  // fixed or massless: left at zero
  const int Rseg = P.eCref + P.rs - shq - 63;
  const int C1 = (int)(cn >> 31), C0 = (int)(cn & 0x7FFFFFFF);
  unsigned long long orv = 0;
  for (int c = 0; c < 3; ++c) {
    int64_t du;
    if (Rseg >= 63) {
      const int64_t H = mul_hi63(dS[c], C1, C0);
      const int sh = Rseg - 63;
      du = sh == 0 ? H : (sh > 62 ? 0 : (H + ((int64_t)1 << (sh - 1))) >> sh);
    } else if (Rseg > 0) {
      du = mul_shr_round(dS[c], cn, Rseg);
    } else {
      const __int128 prod = (__int128)dS[c] * (__int128)cn;
      du = (int64_t)(prod << min(-Rseg, 63));
    }
    const int64_t un = d.U_next[c * d.comp + nidx] - du;
    d.U_next[c * d.comp + nidx] = un;
    orv |= (unsigned long long)(un ^ (un >> 63));
  }
  col = (gj / TC_OWN) * d.tiles_x + gi / TC_OWN;
  return orv;
}

template <int MODE>
__global__ void __launch_bounds__(256) stencil_fix_kernel(const TcDevice d) {
  const TcStepParams P = *d.params;
  const int lane = threadIdx.x & 31;
  // warp-uniform trips, so that the time step's bounds are OR-reduced per
  // warp before the atomics (one per warp for the global word, one per
  // group of lanes of one column for the column words)
  for (int w0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < d.n_fix;
       w0 += gridDim.x * blockDim.x) {
    const int e0 = w0 + lane;
    const int4 f = e0 < d.n_fix ? d.fix[e0] : make_int4(0, 0, 0, ST_FIX_CONT);
    int col = -1;
    // a continuation entry is handled with its node's first entry
    const unsigned long long orv = (f.w & ST_FIX_CONT) ? 0ull : fix_node<MODE>(d, P, e0, f, col);
    if (MODE == TC_MODE_STEP) {
      unsigned long long *cur = d.or_slots + (size_t)P.or_slot * (1 + d.tiles_x * d.tiles_y);
      const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)orv);
      const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(orv >> 32));
      if (lane == 0 && (lo | hi)) atomicOr(&cur[0], ((unsigned long long)hi << 32) | lo);
      const unsigned grp = __match_any_sync(0xffffffffu, col);
      const unsigned glo = __reduce_or_sync(grp, (unsigned)orv);
      const unsigned ghi = __reduce_or_sync(grp, (unsigned)(orv >> 32));
      if (col >= 0 && lane == __ffs(grp) - 1 && (glo | ghi))
        atomicOr(&cur[1 + col], ((unsigned long long)ghi << 32) | glo);
    }
  }
}

cudaError_t stencil_fix(cudaStream_t s, const TcDevice &d, int mode) {
  if (d.n_fix <= 0 || d.n_ctas <= 0) return cudaSuccess;
  const int blocks = (d.n_fix + 255) / 256 < 1024 ? (d.n_fix + 255) / 256 : 1024;
  if (mode == TC_MODE_STEP)
    stencil_fix_kernel<TC_MODE_STEP><<<blocks, 256, 0, s>>>(d);
  else if (mode == TC_MODE_KU)
    stencil_fix_kernel<TC_MODE_KU><<<blocks, 256, 0, s>>>(d);
  else
    return cudaSuccess;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// MODE: TC_MODE_STEP (time step), TC_MODE_KU (S of K u), TC_MODE_PARTIALS
// (per node: P, the stencil part of Q and q', 9 int64 in component-stride
// layout, for exact checks).  CTA b walks stencil segments seg_off[b] ..
// seg_off[b+1]-1; segment (tx, ty, z0, z1), each node with its material
// node_mat[].
// ---------------------------------------------------------------------------
template <int MODE, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    tc_stencil_kernel(const __grid_constant__ CUtensorMap tmap_u, const TcDevice d) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *digits = smem + kOffD;
  int64_t *uslot = reinterpret_cast<int64_t *>(smem + kOffU);
  unsigned char *bimg = smem + kOffB;
  unsigned char *bias_img = smem + kOffBias;
  int4 *seginfo = reinterpret_cast<int4 *>(smem + kOffSeg);  // 2 int4 per segment
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);  // 0..7 U slots, 8,9 TMEM bufs
  uint32_t *misc = reinterpret_cast<uint32_t *>(smem + kOffMisc);  // [0] tmem base, [1] abort, [2] copies issued
  int4 *limbs = reinterpret_cast<int4 *>(smem + kOffLimb);

  const int tid = threadIdx.x;
  const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0), lane = tid & 31;
  constexpr int s_lo = TC_MAX_STAGES - STAGES;
  static_assert(STAGES >= 1 && STAGES <= TC_MAX_STAGES, "stages");

  // epilogue threads (warps 0-7): TMEM lane quarter, pair row, node of the
  // pair (all three components)
  const bool epi = warp < kEpiWarps;
  const int quarter = warp & 3, jnode = (warp >> 2) & 1;
  const int mrow = 32 * quarter + lane;
  const int xl = 2 * (mrow & 7) + 1 + jnode;  // local node x, 1..16
  const int yl = (mrow >> 3) + 1;             // local node y, 1..16

  // ---- one-time setup ------------------------------------------------------
  if (tid == 0) {
    misc[1] = 0;
    misc[2] = 0;
    for (int i = 0; i < kUSlots; ++i) mbar_init(&bars[i], 1);
    mbar_init(&bars[8], STAGES < kMmaWarps ? STAGES : kMmaWarps);  // one commit per issuing warp
    mbar_init(&bars[9], STAGES < kMmaWarps ? STAGES : kMmaWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&misc[0])),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int i = tid; i < kBBytes / 16; i += kThreads)
    reinterpret_cast<uint4 *>(bimg)[i] = reinterpret_cast<const uint4 *>(d.Bst)[i];
  for (int i = tid; i <= TC_MAX_MAT; i += kThreads) {
    const TcMaterial mt = d.mats[i];
    limbs[i] = make_int4((int)(mt.A >> 31), (int)(mt.A & 0x7FFFFFFF), (int)(mt.B >> 31),
                         (int)(mt.B & 0x7FFFFFFF));
  }
  {  // the unused K rows 12..15 of every node row block: the constant 256,
     // which the stencil images meet with zeros and the bias image with
     // 12288 (the digitisers never write these rows)
    const int nrow = kDSlots * TC_MAX_STAGES * kSY;
    for (int i = tid; i < 4 * nrow; i += kThreads)
      *reinterpret_cast<uint4 *>(digits + (i >> 2) * kRowBytes + 128 + (4 + (i & 3)) * 16) =
          make_uint4(kHalf256, kHalf256, kHalf256, kHalf256);
    // bias image, K-major core matrices: N groups at 128 B, K groups at 256 B;
    // an N row holds 8 K values (16 bytes); K rows 12..15 are bytes 8..15 of
    // the N rows of K group 1
    for (int i = tid; i < kBiasBytes / 16; i += kThreads) {
      const bool hi = i >= 16;  // K group 1
      reinterpret_cast<uint4 *>(bias_img)[i] =
          hi ? make_uint4(0u, 0u, kHalf12288, kHalf12288) : make_uint4(0u, 0u, 0u, 0u);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = misc[0];
  // a time step follows the element kernel as a programmatic dependent: the
  // setup above overlaps its tail, the step parameters are read after it
  if constexpr (MODE == TC_MODE_STEP) asm volatile("griddepcontrol.wait;" ::: "memory");
  if ((tmem_base & 0xFFFFu) + kTmemCols > 512u) {  // cannot happen; fail loudly
    if (tid == 0) atomicOr(d.status, 4);
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(kTmemCols));
    return;
  }

  uint32_t mma_phase = 0;  // parity per MMA mbarrier (bits 0, 1)
  // MMA batches in flight (the same bookkeeping in every thread): on an
  // abort the CTA waits, bounded, for them and for its copies before freeing
  // TMEM
  uint32_t mma_out = 0;
  bool aborted = false;
  auto sync_abort = [&](bool ok) -> bool {
    if (!ok) atomicExch(&misc[1], 1u);
    __syncthreads();
    return misc[1] != 0;
  };
  const TcStepParams P = *d.params;
  const int64_t dbias = (1LL << 10) | (1LL << 21) | (1LL << 32) | (1LL << 43) | (1LL << 54);
  // digit planes keep only stages s_lo..4: q' = sum of those digits
  const int lo_bits = TC_DIGIT_BITS * s_lo;
  const int64_t dbias_hi = (dbias >> lo_bits) << lo_bits;
  const int sbeg = d.seg_off[blockIdx.x], send = d.seg_off[blockIdx.x + 1];

  // digit shift of a segment's column (Eq. intscaling): the previous step's
  // bound over the 3x3 columns around it, as in the element kernel
  auto seg_shq_global = [&](int4 seg) -> int {
    int shq = P.shq;
    if (MODE == TC_MODE_STEP) {
      const unsigned long long *prev =
          d.or_slots + (size_t)((P.or_slot + 2) % 3) * (1 + d.tiles_x * d.tiles_y) + 1;
      unsigned long long o = 0;
      for (int dyc = -1; dyc <= 1; ++dyc)
        for (int dxc = -1; dxc <= 1; ++dxc) {
          const int cx = seg.x + dxc, cy = seg.y + dyc;
          if (cx >= 0 && cy >= 0 && cx < d.tiles_x && cy < d.tiles_y) o |= prev[cy * d.tiles_x + cx];
        }
      const int b = o ? 64 - __clzll((long long)o) : 0;
      shq = min(P.shq, max(0, b - TC_QBITS));
    }
    return shq;
  };
  // segment table entry: {tx, ty, z0, z1}, {shq, -, -, -}
  auto seg_fill = [&](int sg, int4 *e) {
    const int4 s = d.segs[sg];
    e[0] = s;
    e[1] = make_int4(seg_shq_global(s), 0, 0, 0);
  };
  for (int i = tid; i < min(send - sbeg, kSegCap); i += kThreads) seg_fill(sbeg + i, seginfo + 2 * i);
  __syncthreads();
  auto seg_at = [&](int sg) -> int4 {
    return sg - sbeg < kSegCap ? seginfo[2 * (sg - sbeg)] : d.segs[sg];
  };
  auto seg_entry = [&](int sg, int4 &s, int &shq) {
    if (sg - sbeg < kSegCap) {
      s = seginfo[2 * (sg - sbeg)];
      shq = seginfo[2 * (sg - sbeg) + 1].x;
    } else {
      int4 e[2];
      seg_fill(sg, e);
      s = e[0];
      shq = e[1].x;
    }
  };

  // ---- the CTA's segments as streams ---------------------------------------
  // Segment s (column (tx, ty), owned node planes [z0, z1), z1 - z0 >= 2) has
  // the input planes z0-1 .. z1 and the outputs z0 .. z1-1.  Inputs are
  // numbered g over all of the CTA's segments, outputs o.  Input g goes to U
  // slot g mod 8 (copy completion: phase g/8 mod 2 of mbarrier g mod 8) and
  // digit slot g mod 4; output o accumulates in TMEM ring slot o mod 3, and
  // input plane p of a segment whose first output is o_s feeds the outputs
  // v - 1, v, v + 1 with v = o_s + p - z0.  While output o (input gin) is
  // finished, the copies run up to input gin + 7, the digits up to the last
  // input of output o + 2 and the MMAs (issued after the barrier) up to the
  // last input of output o + 1, across segment boundaries.  Slots stay
  // consistent: inputs below gin are done with (their U slots are free); the
  // MMAs of output o's inputs are complete when o is read, so the digits in
  // use are those of outputs o + 1 and o + 2, at most 4 inputs because every
  // segment has two outputs or more; ring slot o + 3 = o is restarted by a
  // bias MMA issued after the barrier that follows its read, and the zero
  // blocks of a segment's first two inputs land on slots already read.
  struct InCur {
    int sg, p, z1, ob, g;  // segment, plane, its z1, its first output index; input index
  };
  auto in_seek = [&](InCur &c, int sg, int ob) {
    c.sg = sg;
    c.ob = ob;
    if (sg < send) {
      const int4 s = seg_at(sg);
      c.p = s.z - 1;
      c.z1 = s.w;
    }
  };
  auto in_next = [&](InCur &c) {
    ++c.g;
    if (++c.p > c.z1) {
      const int4 s = seg_at(c.sg);
      in_seek(c, c.sg + 1, c.ob + (s.w - s.z));
    }
  };
  InCur lc, dc, mc;  // copy, digit and MMA cursors
  lc.g = dc.g = mc.g = 0;
  in_seek(lc, sbeg, 0);
  in_seek(dc, sbeg, 0);
  in_seek(mc, sbeg, 0);
  int d_shq = 0, d_xo = 0;  // digit cursor's column shift and box offset
  if (sbeg < send) {
    int4 s;
    seg_entry(sbeg, s, d_shq);
    d_xo = (TC_OWN * s.x - 1) & 1;
  }

  auto uslot_g = [&](int g) { return uslot + (g & 7) * (kUStride / 8); };
  auto dslot_g = [&](int g) { return digits + (g & 3) * kDSlotBytes; };

  // copies: thread kDigit0 alone issues them and keeps the cursor (the
  // teardown reads its count from shared memory)
  auto load_upto = [&](int gmax) {
    if (tid != kDigit0) return;
    while (lc.sg < send && lc.g <= gmax) {
      {
        const int4 s = seg_at(lc.sg);
        const int slot = lc.g & 7;
        mbar_expect_tx(&bars[slot], kUBytes);
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(uslot_g(lc.g))),
            "l"(&tmap_u), "r"(smem_u32(&bars[slot])), "r"((TC_OWN * s.x - 1) & ~1),
            "r"(TC_OWN * s.y - 1), "r"(lc.p), "r"(0)
            : "memory");
      }
      in_next(lc);
    }
    misc[2] = (uint32_t)lc.g;
  };
  // task t of an input plane: node row y, component c and x parity e
  // (t = (3 y + c) 2 + e) digitise the nine nodes x = e + 2 i, i = 0..8,
  // once, and write the 16-byte chunks of K rows k = 3 d + c for the
  // x-shifts d = e (nodes i = 0..7 for pairs 0..7) and d = e + 2 (nodes
  // i = 1..8) of every stage.  With the offset-binary bias dbias =
  // sum_s 1024 2^(11 s), digit s of q = floor(U / 2^shq) is
  // ((q + dbias) >> 11 s) & 2047 - 1024 (q + dbias is positive and below
  // 2^55 since |q| < 2^51); the float with bits 0x4B000000 | x is 2^23 + x,
  // so subtracting 2^23 + 1024 leaves the digit exactly.
  auto digitise_task = [&](int g, int xo, int shq, int t) {
    const int e = t & 1, c = (t >> 1) % 3, y = (t >> 1) / 3;
    const int64_t *src = uslot_g(g) + (c * kSY + y) * kSX + xo + e;
    unsigned char *row = dslot_g(g) + y * kRowBytes;
    unsigned char *dst0 = row + ((3 * e + c) >> 3) * 128 + ((3 * e + c) & 7) * 16;
    unsigned char *dst1 = row + ((3 * e + 6 + c) >> 3) * 128 + ((3 * e + 6 + c) & 7) * 16;
    uint64_t v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = (uint64_t)((src[2 * i] >> shq) + dbias);
#pragma unroll
    for (int s = s_lo; s < TC_MAX_STAGES; ++s) {
      float f[9];
#pragma unroll
      for (int i = 0; i < 9; ++i)
        f[i] = __int_as_float((int)(((uint32_t)(v[i] >> (TC_DIGIT_BITS * s)) & 2047u) |
                                    0x4B000000u)) - 8389632.0f;
      uint32_t w0[4], w1[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const __half2 h0 = __floats2half2_rn(f[2 * i], f[2 * i + 1]);
        const __half2 h1 = __floats2half2_rn(f[2 * i + 1], f[2 * i + 2]);
        w0[i] = *reinterpret_cast<const uint32_t *>(&h0);
        w1[i] = *reinterpret_cast<const uint32_t *>(&h1);
      }
      *reinterpret_cast<uint4 *>(dst0 + s * kStageBytes) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
      *reinterpret_cast<uint4 *>(dst1 + s * kStageBytes) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    }
  };
  // digits of the inputs up to gmax, by the threads from `first` on (they
  // alone keep the cursor), each waiting for its input's copy
  // (first = 0: every thread, tasks strided over the block; first = kDigit0:
  // warps 9-12, kTasksPerWarp tasks each)
  auto digitise_upto = [&](int gmax, int first) -> bool {
    bool ok = true;
    if (tid < first || (first > 0 && tid >= kDigit0 + 32 * kDigitWarps)) return ok;
    const int t_own = first > 0 ? (lane < kTasksPerWarp ? (warp - 9) * kTasksPerWarp + lane : -1)
                                : -1;
    while (dc.sg < send && dc.g <= gmax) {
      ok = mbar_wait(&bars[dc.g & 7], (uint32_t)(dc.g >> 3) & 1u) && ok;
      if (first > 0) {
        if (t_own >= 0) digitise_task(dc.g, d_xo, d_shq, t_own);
      } else {
        for (int t = tid; t < kTasks; t += kThreads) digitise_task(dc.g, d_xo, d_shq, t);
      }
      const int sg = dc.sg;
      in_next(dc);
      if (dc.sg != sg && dc.sg < send) {
        int4 s;
        seg_entry(dc.sg, s, d_shq);
        d_xo = (TC_OWN * s.x - 1) & 1;
      }
    }
    return ok;
  };
  // MMAs of the inputs up to gmax into the rings of every stage, stage
  // s_lo + k issued by the warp of rank k mod 4 (a tcgen05.mma occupies its
  // issuing warp for about a hundred cycles, so the stages are issued side by
  // side; each stage has its own accumulators, and MMAs of one thread run in
  // issue order).  Input plane p of a segment with first
  // output o_s (v = o_s + p - z0) uses B variant 0 (all outputs), 1 (none
  // below: p = z0) or 2 (only above: p = z0 - 1); the B start block
  // (1 - v) mod 3 of the five stored blocks puts output v + k into slot
  // (v + k) mod 3.  Input p is the first to reach output v + 1: per stage an
  // N = 16 MMA without accumulation first writes the magic bias 1.5 2^23
  // into that slot (the constant K rows of the digit block against the bias
  // image).  Then each issuing warp commits onto mbarrier 8 + (batch & 1),
  // which completes once all of them have and all their MMAs are done.  The
  // issuing warps alone keep the cursor; there is something to issue exactly
  // when the output the batch completes exists.
  const int mma_rank = mma_rank_of(warp);
  auto mma_upto = [&](int gmax, int batch) {
    if (mma_rank < 0 || mma_rank >= STAGES || !(mc.sg < send && mc.g <= gmax)) return;
    __syncwarp();
    tc_fence_after();
    while (mc.sg < send && mc.g <= gmax) {
      {
        const int z0 = seg_at(mc.sg).z;
        const int var = mc.p == z0 - 1 ? 2 : (mc.p == z0 ? 1 : 0);
        const int v = mc.ob + mc.p - z0;
        const int s0 = ((1 - v) % 3 + 3) % 3;
        const uint32_t bimg_base = smem_u32(bimg) + (uint32_t)(var * 3 * kBImage + s0 * 256);
        const uint32_t next_slot = (uint32_t)(16 * (((v + 1) % 3 + 3) % 3));
        const uint64_t bias_desc = make_sdesc(smem_u32(bias_img), 256, 128);
        const unsigned char *ds = dslot_g(mc.g);
        for (int st = s_lo + mma_rank; st < TC_MAX_STAGES; st += kMmaWarps) {
          const uint32_t dcol = tmem_base + (uint32_t)(st * kRingCols);
          mma_f16_elect(dcol + next_slot,
                        make_sdesc(smem_u32(ds + st * kStageBytes + kRowBytes), 128, 256),
                        bias_desc, kIdescN16, 0u);
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
            const uint32_t a = smem_u32(ds + st * kStageBytes + (1 + dy) * kRowBytes);
            mma_f16_elect(dcol, make_sdesc(a, 128, 256),
                          make_sdesc(bimg_base + (uint32_t)((dy + 1) * kBImage), kBKStride, 128),
                          kIdescN48, 1u);
          }
        }
      }
      in_next(mc);
    }
    mma_commit_elect(&bars[8 + (batch & 1)]);
  };
  // ---- output cursor and the epilogue's view of its segment ---------------
  int o = 0, osg = sbeg, oz = 0, oz1 = 0, gin = 1;  // output o: plane oz, input gin
  int gi = 0, gj = 0, e_xo = 0, e_shq = 0, Rseg = 0;
  bool own = false;
  auto out_seek = [&](int sg) {
    osg = sg;
    if (sg >= send) return;
    int4 s;
    int shq;
    seg_entry(sg, s, shq);
    oz = s.z;
    oz1 = s.w;
    if (!epi) return;
    const int X0 = TC_OWN * s.x - 1, Y0 = TC_OWN * s.y - 1;
    e_xo = X0 & 1;  // offset of the copied box, whose x start is even
    gi = X0 + xl;
    gj = Y0 + yl;
    own = epi && xl <= TC_OWN && yl <= TC_OWN && gi <= d.nx && gj <= d.ny;
    e_shq = shq;
    Rseg = P.eCref + P.rs - e_shq - 63;
  };
  // the node's reference material and the update's global operands
  // (u^{n-1} and the multiplier C of the node) are loaded one output ahead
  int64_t nx_uprev[3] = {0, 0, 0}, nx_cn = 0;
  int nx_mat = ST_NO_MAT;
  auto load_update_at = [&](int4 s, int z) {
    if (MODE != TC_MODE_PARTIALS && epi) {
      const int i = TC_OWN * s.x - 1 + xl, j = TC_OWN * s.y - 1 + yl;
      if (xl <= TC_OWN && yl <= TC_OWN && i <= d.nx && j <= d.ny) {
        const int64_t n = (int64_t)z * d.plane + (int64_t)j * d.nxp + i;
        nx_mat = d.node_mat[n];
        if (MODE == TC_MODE_STEP) {
          nx_cn = d.C[n];
#pragma unroll
          for (int c = 0; c < 3; ++c) nx_uprev[c] = d.U_prev[c * d.comp + n];
        }
      }
    }
  };
  unsigned long long or_seg = 0;

  // ---- prologue: copies of inputs 0..7, the digits of the inputs of outputs
  // 0 and 1 (every thread), the MMAs of output 0's inputs (batch 1)
  if (sbeg < send) {
    out_seek(sbeg);
    load_upto(gin + 6);
    const bool ok = digitise_upto(gin + (oz + 1 < oz1 ? 1 : 3) + 1, 0);
    fence_async_smem();
    tc_fence_before();
    if (sync_abort(ok)) {
      aborted = true;
    } else {
      mma_upto(gin + 1, 1);
      mma_out |= 1u << 1;
    }
    load_update_at(seg_at(sbeg), oz);
  }

  bool okp = true;
  while (!aborted && osg < send) {
    // (a) this output's update operands; the next output's are requested
    const int64_t nidx = (int64_t)oz * d.plane + (int64_t)gj * d.nxp + gi;
    const int64_t uprev[3] = {nx_uprev[0], nx_uprev[1], nx_uprev[2]};
    const int64_t cn = nx_cn;
    const int mcur = nx_mat;  // the node's reference material
    if (MODE != TC_MODE_PARTIALS && epi) {
      if (oz + 1 < oz1) {
        load_update_at(seg_at(osg), oz + 1);
      } else if (osg + 1 < send) {
        const int4 s = seg_at(osg + 1);
        load_update_at(s, s.z);
      }
    }
    // output o is complete once batch o+1 is in: read its ring slot
    const int bL = (o + 1) & 1;
    uint32_t w[TC_MAX_STAGES][8];
    if (epi) {
      __syncwarp();
      mma_out &= ~(1u << bL);
      const bool okm = mbar_wait(&bars[8 + bL], (mma_phase >> bL) & 1u);
      if (!okm) atomicExch(&misc[1], 1u);
      tc_fence_after();
      const uint32_t tb = tmem_base + ((uint32_t)(32 * quarter) << 16) +
                          (uint32_t)(16 * (o % 3) + 8 * jnode);
#pragma unroll
      for (int s = s_lo; s < TC_MAX_STAGES; ++s) tmem_ld8(tb + (uint32_t)(s * kRingCols), w[s]);
#pragma unroll
      for (int s = s_lo; s < TC_MAX_STAGES; ++s) tmem_wait_ld8(w[s]);
    }
    mma_phase ^= 1u << bL;
    // (b) TMEM reads done, digit writes visible to the tensor core
    tc_fence_before();
    fence_async_smem();
    if (sync_abort(okp)) {
      aborted = true;
      break;
    }
    // (c) warps 8, 13-15: the MMAs of output o+1's inputs (batch o+2);
    // thread kDigit0: copies; warps 9-12: the digits of output o+2's inputs; warps
    // 0-7: finish output o
    mma_upto(gin + (oz + 1 < oz1 ? 1 : 3) + 1, o + 2);
    if (oz + 1 < oz1 || osg + 1 < send) mma_out |= 1u << ((o + 2) & 1);  // output o+1 exists
    load_upto(gin + 7);
    okp = digitise_upto(gin + (oz + 2 < oz1 ? 2 : 4) + 1, kDigit0);
    if (epi) {
      // recombination (Horner over the stages), the node's own q' for the
      // 1024 q(n) term, and the material product; node columns 2 c + part
      uint64_t acc[6];
#pragma unroll
      for (int st = 0; st < TC_MAX_STAGES; ++st)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            const uint32_t x = st < s_lo ? (uint32_t)TC_MAGIC_BITS : w[st][2 * c + part];
            uint64_t &a = acc[3 * part + c];
            if (st == 0) recomb_stage<0>(a, x);
            else if (st == 1) recomb_stage<1>(a, x);
            else if (st == 2) recomb_stage<2>(a, x);
            else if (st == 3) recomb_stage<3>(a, x);
            else recomb_stage<4>(a, x);
          }
      // the copy of this output's plane completed before the digitising
      // warps read it; the test acquires that completion for these reads
      if (!mbar_test_wait(&bars[gin & 7], (uint32_t)(gin >> 3) & 1u)) atomicExch(&misc[1], 1u);
      const int64_t *ucur = uslot_g(gin);
      int64_t u0[3], qn[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        u0[c] = ucur[(c * kSY + yl) * kSX + xl + e_xo];
        const int64_t v = (u0[c] >> e_shq) + dbias;
        qn[c] = ((v >> lo_bits) << lo_bits) - dbias_hi;
      }
      if constexpr (MODE == TC_MODE_PARTIALS) {
        if (own) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            d.partials_out[c * d.comp + nidx] = recomb_finish(acc[c]);
            d.partials_out[(3 + c) * d.comp + nidx] = recomb_finish(acc[3 + c]);
            d.partials_out[(6 + c) * d.comp + nidx] = qn[c];
          }
        }
      } else {
        const int4 lm = limbs[mcur];
        const int A1 = lm.x, A0 = lm.y, B1 = lm.z, B0 = lm.w;
        int64_t S[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          S[c] = mul2_hi63(recomb_finish(acc[c]), recomb_finish(acc[3 + c]), A1, A0, B1, B0) +
                 mul_hi63(qn[c] * 1024, B1, B0);
        if (own && MODE == TC_MODE_KU) {
#pragma unroll
          for (int c = 0; c < 3; ++c) d.S_out[c * d.comp + nidx] = S[c];
        } else if (own) {
          // update of node (gi, gj, oz): the element kernel's fixed-point step
          const int C1 = (int)(cn >> 31), C0 = (int)(cn & 0x7FFFFFFF);
          const bool rescaled = (P.rs | P.rs_prev) != 0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            int64_t uc = u0[c], um = uprev[c];
            if (rescaled) {
              uc = shr_round(uc, P.rs);
              um = shr_round(um, P.rs + P.rs_prev);
            }
            int64_t du;
            if (Rseg >= 63) {
              const int64_t H = mul_hi63(S[c], C1, C0);
              const int sh = Rseg - 63;
              du = sh == 0 ? H : (sh > 62 ? 0 : (H + ((int64_t)1 << (sh - 1))) >> sh);
            } else if (Rseg > 0) {
              du = mul_shr_round(S[c], cn, Rseg);
            } else {
              const __int128 prod = (__int128)S[c] * (__int128)cn;
              du = (int64_t)(prod << min(-Rseg, 63));
            }
            int64_t un = 2 * uc - um - du;
            if (cn == 0) un = 0;  // fixed or massless node
            d.U_next[c * d.comp + nidx] = un;
            or_seg |= (unsigned long long)(un ^ (un >> 63)) | (unsigned long long)(uc ^ (uc >> 63));
          }
        }
      }
    }
    // (d) next output; leaving a segment: its column's bounds for the next step
    if (oz + 1 >= oz1) {
      if (MODE == TC_MODE_STEP && epi) {
        for (int sh = 16; sh > 0; sh >>= 1) or_seg |= __shfl_xor_sync(0xffffffffu, or_seg, sh);
        if (lane == 0 && or_seg) {
          const int4 s = seg_at(osg);
          unsigned long long *cur = d.or_slots + (size_t)P.or_slot * (1 + d.tiles_x * d.tiles_y);
          atomicOr(&cur[1 + s.y * d.tiles_x + s.x], or_seg);
          atomicOr(&cur[0], or_seg);
        }
      }
      or_seg = 0;
      out_seek(osg + 1);
      gin += 3;
    } else {
      ++oz;
      ++gin;
    }
    ++o;
  }

  // ---- teardown -------------------------------------------------------------
  if (aborted && tid == 0) {
    atomicOr(d.status, 1);
    // let the copies and MMAs still in flight land (each wait bounded): the
    // last copy into each U slot is among the last eight issued
    const int gl = (int)misc[2];
    for (int g = max(0, gl - kUSlots); g < gl; ++g)
      mbar_wait(&bars[g & 7], (uint32_t)(g >> 3) & 1u);
    for (int b = 0; b < 2; ++b)
      if (mma_out & (1u << b)) mbar_wait(&bars[8 + b], (mma_phase >> b) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols));
  }
}

template <int MODE, int S>
static cudaError_t st_set_attr() {
  return cudaFuncSetAttribute(tc_stencil_kernel<MODE, S>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

template <int MODE>
static cudaError_t st_set_attr_all() {
  cudaError_t e;
  if ((e = st_set_attr<MODE, 1>()) != cudaSuccess) return e;
  if ((e = st_set_attr<MODE, 2>()) != cudaSuccess) return e;
  if ((e = st_set_attr<MODE, 3>()) != cudaSuccess) return e;
  if ((e = st_set_attr<MODE, 4>()) != cudaSuccess) return e;
  return st_set_attr<MODE, 5>();
}

cudaError_t stencil_prepare() {
  cudaError_t e;
  if ((e = st_set_attr_all<TC_MODE_STEP>()) != cudaSuccess) return e;
  if ((e = st_set_attr_all<TC_MODE_KU>()) != cudaSuccess) return e;
  return st_set_attr_all<TC_MODE_PARTIALS>();
}

template <int MODE, int S>
static cudaError_t st_launch_one(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap,
                                 int n_ctas, bool pdl) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(n_ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = MODE == TC_MODE_STEP && pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, tc_stencil_kernel<MODE, S>, *tmap, d);
}

template <int MODE>
static cudaError_t st_launch_mode(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap,
                                  int stages, int n_ctas, bool pdl) {
  switch (stages) {
    case 1: return st_launch_one<MODE, 1>(s, d, tmap, n_ctas, pdl);
    case 2: return st_launch_one<MODE, 2>(s, d, tmap, n_ctas, pdl);
    case 3: return st_launch_one<MODE, 3>(s, d, tmap, n_ctas, pdl);
    case 4: return st_launch_one<MODE, 4>(s, d, tmap, n_ctas, pdl);
    default: return st_launch_one<MODE, 5>(s, d, tmap, n_ctas, pdl);
  }
}

// d.segs / d.seg_off / d.n_ctas describe the stencil segments;
// pdl: a time step is launched as a programmatic dependent of the kernel
// before it on the stream
cudaError_t stencil_launch_ex(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap, int mode,
                              bool pdl) {
  if (d.n_ctas <= 0) return cudaSuccess;
  switch (mode) {
    case TC_MODE_STEP: return st_launch_mode<TC_MODE_STEP>(s, d, tmap, d.stages, d.n_ctas, pdl);
    case TC_MODE_KU: return st_launch_mode<TC_MODE_KU>(s, d, tmap, d.stages, d.n_ctas, pdl);
    default: return st_launch_mode<TC_MODE_PARTIALS>(s, d, tmap, d.stages, d.n_ctas, pdl);
  }
}

cudaError_t stencil_launch(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap, int mode) {
  return stencil_launch_ex(s, d, tmap, mode, true);
}
