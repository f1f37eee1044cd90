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
// A CTA owns 15x15 node columns (the element path's partition) and computes
// 16x16 (the 16th row and column are dropped), marching up in z through its
// segment's planes: TMA brings node planes (box 20 x 18 x 1 x 3 int64) into an
// 8-slot ring six planes ahead; per plane L the 8 epilogue warps read the
// TMEM slot of plane L, recombine and update node plane L while
// warp 8 issues the MMAs of input plane L+2 and warps 9-15 digitise plane L+3
// (one CTA barrier per plane).  Source and receiver planes, mesh faces and
// material interfaces are left to the element kernel (vfe_tc.cu).
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
// the bias image: 16 K rows x 16 N columns, K rows 12..15 = 12288 (fp16),
// the rest zero; against the constant 256 in K rows 12..15 of every digit
// block it gives 4 x 256 x 12288 = 1.5 2^23 in each of the 16 columns
constexpr int kBiasBytes = 512;

constexpr int kOffD = 0;
constexpr int kOffU = kOffD + kDSlots * kDSlotBytes;
constexpr int kOffB = kOffU + kUSlots * kUStride;
constexpr int kOffBias = kOffB + kBBytes;
constexpr int kOffBar = kOffBias + kBiasBytes;
constexpr int kOffMisc = kOffBar + 16 * 8;
constexpr int kSmemBytes = kOffMisc + 64;

static_assert(kOffU % 128 == 0 && kUStride % 128 == 0, "TMA destinations 128-byte aligned");
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
constexpr int kMmaWarp = 8;                   // warp 8: MMA issue
constexpr int kDigit0 = 9 * 32;               // first digitising thread (warps 9-15)
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
// MODE: TC_MODE_STEP (time step), TC_MODE_KU (S of K u), TC_MODE_PARTIALS
// (per node: P, the stencil part of Q and q', 9 int64 in component-stride
// layout, for exact checks).  CTA b walks stencil segments seg_off[b] ..
// seg_off[b+1]-1; segment (tx, ty, z0, z1) with material seg_mat[].
// ---------------------------------------------------------------------------
template <int MODE, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    tc_stencil_kernel(const __grid_constant__ CUtensorMap tmap_u, const TcDevice d) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *digits = smem + kOffD;
  int64_t *uslot = reinterpret_cast<int64_t *>(smem + kOffU);
  unsigned char *bimg = smem + kOffB;
  unsigned char *bias_img = smem + kOffBias;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);  // 0..7 U slots, 8,9 TMEM bufs
  uint32_t *misc = reinterpret_cast<uint32_t *>(smem + kOffMisc);  // [0] tmem base, [1] abort

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
    for (int i = 0; i < kUSlots; ++i) mbar_init(&bars[i], 1);
    mbar_init(&bars[8], 1);
    mbar_init(&bars[9], 1);
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

  uint32_t uphase = 0;
  uint32_t mma_phase = 0;  // parity per MMA mbarrier (bits 0, 1)
  // copies and MMAs in flight (the same bookkeeping in every thread): on an
  // abort the CTA waits, bounded, for them before freeing TMEM
  uint32_t tma_out = 0, mma_out = 0;
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
  for (int sg = sbeg; sg < send && !aborted; ++sg) {
    const int4 seg = d.segs[sg];
    const TcMaterial mt = d.mats[d.seg_mat[sg]];
    const int A1 = (int)(mt.A >> 31), A0 = (int)(mt.A & 0x7FFFFFFF);
    const int B1 = (int)(mt.B >> 31), B0 = (int)(mt.B & 0x7FFFFFFF);
    const int X0 = TC_OWN * seg.x - 1, Y0 = TC_OWN * seg.y - 1;
    const int Z0 = seg.z, Z1 = seg.w;  // owned node planes [Z0, Z1), 1 <= Z0 < Z1 <= nz
    const int xbox = X0 & ~1, xo = X0 - xbox;
    const int gi = X0 + xl, gj = Y0 + yl;
    const bool own = epi && xl <= TC_OWN && yl <= TC_OWN && gi <= d.nx && gj <= d.ny;

    // digit shift of this column (Eq. intscaling): the previous step's bound
    // over the 3x3 columns around it, as in the element kernel
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
    const int Rseg = P.eCref + P.rs - shq - 63;
    unsigned long long or_seg = 0;

    auto issue_plane = [&](int p, int issuer) {
      tma_out |= 1u << (p & 7);
      if (tid == issuer) {
        const int s = p & 7;
        mbar_expect_tx(&bars[s], kUBytes);
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(uslot + s * (kUStride / 8))),
            "l"(&tmap_u), "r"(smem_u32(&bars[s])), "r"(xbox), "r"(Y0), "r"(p), "r"(0)
            : "memory");
      }
    };
    auto wait_plane = [&](int p, bool do_wait) -> bool {
      const int s = p & 7;
      const bool ok = do_wait ? mbar_wait(&bars[s], (uphase >> s) & 1u) : true;
      uphase ^= 1u << s;
      tma_out &= ~(1u << s);
      return ok;
    };
    auto uslot_of = [&](int p) { return uslot + (p & 7) * (kUStride / 8); };
    auto dslot_of = [&](int p) { return digits + (p & 3) * kDSlotBytes; };
    // task t of a plane: node row y, component c and x parity e
    // (t = (3 y + c) 2 + e) digitise the nine nodes x = e + 2 i, i = 0..8,
    // once, and write the 16-byte chunks of K rows k = 3 d + c for the
    // x-shifts d = e (nodes i = 0..7 for pairs 0..7) and d = e + 2 (nodes
    // i = 1..8) of every stage.  With the offset-binary bias dbias =
    // sum_s 1024 2^(11 s), digit s of q = floor(U / 2^shq) is
    // ((q + dbias) >> 11 s) & 2047 - 1024 (q + dbias is positive and below
    // 2^55 since |q| < 2^51); the float with bits 0x4B000000 | x is 2^23 + x,
    // so subtracting 2^23 + 1024 leaves the digit exactly.
    auto digitise_task = [&](int p, int t) {
      const int e = t & 1, c = (t >> 1) % 3, y = (t >> 1) / 3;
      const int64_t *src = uslot_of(p) + (c * kSY + y) * kSX + xo + e;
      unsigned char *row = dslot_of(p) + y * kRowBytes;
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
    // MMAs of input plane p (B variant v: 0 all outputs, 1 none below, 2 only
    // above) into the rings of every stage, all issued by warp 8 (an issuing
    // warp stalls while the tensor pipe drains, so no other work waits behind
    // it).  The B start block (1 - p) mod 3 of the five stored blocks puts
    // output z = p + o into slot z mod 3.  Input p is the first to reach
    // output p + 1: per stage, an N = 16 MMA without accumulation first
    // writes the magic bias 1.5 2^23 into that slot (the constant K rows of
    // the digit block against the bias image; the epilogue read the slot's
    // previous plane before the barrier that precedes this issue, and MMAs of
    // one thread run in issue order).  commit: one mbarrier arrival once
    // these and all earlier MMAs are done (batch b on mbarrier 8 + (b & 1)).
    auto issue_mma = [&](int p, int v, int commit_batch) {
      if (commit_batch >= 0) mma_out |= 1u << (commit_batch & 1);
      if (warp != kMmaWarp) return;
      __syncwarp();
      tc_fence_after();
      const int s0 = ((1 - p) % 3 + 3) % 3;
      const uint32_t bimg_base = smem_u32(bimg) + (uint32_t)(v * 3 * kBImage + s0 * 256);
      const uint32_t next_slot = (uint32_t)(16 * (((p + 1) % 3 + 3) % 3));
      const uint64_t bias_desc = make_sdesc(smem_u32(bias_img), 256, 128);
#pragma unroll 1
      for (int st = s_lo; st < TC_MAX_STAGES; ++st) {
        const uint32_t dcol = tmem_base + (uint32_t)(st * kRingCols);
        mma_f16_elect(dcol + next_slot,
                      make_sdesc(smem_u32(dslot_of(p) + st * kStageBytes + kRowBytes), 128, 256),
                      bias_desc, kIdescN16, 0u);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const uint32_t a = smem_u32(dslot_of(p) + st * kStageBytes + (1 + dy) * kRowBytes);
          mma_f16_elect(dcol, make_sdesc(a, 128, 256),
                        make_sdesc(bimg_base + (uint32_t)((dy + 1) * kBImage), kBKStride, 128),
                        kIdescN48, 1u);
        }
      }
      if (commit_batch >= 0) mma_commit_elect(&bars[8 + (commit_batch & 1)]);
    };
    // ---- segment prologue: TMA of planes Z0-1 .. Z0+5, digits of Z0-1 .. Z0+2,
    // the MMAs of inputs Z0-1, Z0, Z0+1 (batch Z0+1; their bias MMAs start
    // the slots of outputs Z0, Z0+1, Z0+2)
    for (int p = Z0 - 1; p <= min(Z0 + 5, Z1); ++p) issue_plane(p, 0);
    bool ok = true;
    for (int p = Z0 - 1; p <= min(Z0 + 2, Z1); ++p) ok = wait_plane(p, true) && ok;
    if (sync_abort(ok)) { aborted = true; break; }
    for (int p = Z0 - 1; p <= min(Z0 + 2, Z1); ++p)
      for (int t = tid; t < kTasks; t += kThreads) digitise_task(p, t);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    issue_mma(Z0 - 1, 2, -1);
    issue_mma(Z0, 1, -1);
    issue_mma(Z0 + 1, 0, Z0 + 1);  // Z0 + 1 <= Z1: a segment owns a plane

    // the update's global operands (u^{n-1} and the multiplier C of the
    // node) are loaded one plane ahead
    int64_t nx_uprev[3] = {0, 0, 0}, nx_cn = 0;
    auto load_update = [&](int L) {
      if (MODE == TC_MODE_STEP && own && L < Z1) {
        const int64_t n = (int64_t)L * d.plane + (int64_t)gj * d.nxp + gi;
        nx_cn = d.C[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) nx_uprev[c] = d.U_prev[c * d.comp + n];
      }
    };
    load_update(Z0);
    bool okp = true;
    for (int L = Z0; L < Z1; ++L) {
      // (a) this plane's update operands; the next plane's are requested
      const int64_t nidx = (int64_t)L * d.plane + (int64_t)gj * d.nxp + gi;
      const int64_t uprev[3] = {nx_uprev[0], nx_uprev[1], nx_uprev[2]};
      const int64_t cn = nx_cn;
      load_update(L + 1);
      // plane L is complete once batch L+1 (input L+1) is in: read its slot
      // (input L+2's bias MMA restarts it for plane L+3 after the barrier)
      const int bL = (L + 1) & 1;
      uint32_t w[TC_MAX_STAGES][8];
      if (epi) {
        __syncwarp();
        mma_out &= ~(1u << bL);
        const bool okm = mbar_wait(&bars[8 + bL], (mma_phase >> bL) & 1u);
        if (!okm) atomicExch(&misc[1], 1u);
        tc_fence_after();
        const uint32_t tb = tmem_base + ((uint32_t)(32 * quarter) << 16) +
                            (uint32_t)(16 * (L % 3) + 8 * jnode);
#pragma unroll
        for (int s = s_lo; s < TC_MAX_STAGES; ++s) tmem_ld8(tb + (uint32_t)(s * kRingCols), w[s]);
#pragma unroll
        for (int s = s_lo; s < TC_MAX_STAGES; ++s) tmem_wait_ld8(w[s]);
      }
      mma_phase ^= 1u << bL;
      // (b) TMEM reads done, digit writes visible to the tensor core
      tc_fence_before();
      fence_async_smem();
      if (sync_abort(okp)) { aborted = true; break; }
      if (L + 2 <= Z1) issue_mma(L + 2, 0, L + 2);

      // (c) second phase: warps 9-15 digitise plane L+3 (into the digit slot
      // of plane L-1, whose MMAs are done) and prefetch plane L+6 (into the U
      // slot of plane L-2); warps 0-7 finish plane L.  Every thread tracks
      // the U-slot phases.
      okp = true;
      if (L + 3 <= Z1) okp = wait_plane(L + 3, tid >= kDigit0);
      if (L + 6 <= Z1) issue_plane(L + 6, kDigit0);
      if (!epi) {  // warps 9-15: one digitisation chunk per thread (warp 8 issues MMAs)
        if (tid >= kDigit0 && L + 3 <= Z1)
          for (int t = tid - kDigit0; t < kTasks; t += kThreads - kDigit0) digitise_task(L + 3, t);
        continue;
      }
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
      // plane L's slot completed its phase before the digitising warps read
      // it; the test acquires that completion for these reads
      if (!mbar_test_wait(&bars[L & 7], ((uphase >> (L & 7)) & 1u) ^ 1u)) atomicExch(&misc[1], 1u);
      const int64_t *ucur = uslot_of(L);
      int64_t u0[3], qn[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        u0[c] = ucur[(c * kSY + yl) * kSX + xl + xo];
        const int64_t v = (u0[c] >> shq) + dbias;
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
        int64_t S[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          S[c] = mul2_hi63(recomb_finish(acc[c]), recomb_finish(acc[3 + c]), A1, A0, B1, B0) +
                 mul_hi63(qn[c] * 1024, B1, B0);
        if (own && MODE == TC_MODE_KU) {
#pragma unroll
          for (int c = 0; c < 3; ++c) d.S_out[c * d.comp + nidx] = S[c];
        } else if (own) {
          // update of node (gi, gj, L): the element kernel's fixed-point step
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
    if (MODE == TC_MODE_STEP) {  // per-column and global bounds for the next step
      for (int o = 16; o > 0; o >>= 1) or_seg |= __shfl_xor_sync(0xffffffffu, or_seg, o);
      if (lane == 0 && or_seg) {
        unsigned long long *cur = d.or_slots + (size_t)P.or_slot * (1 + d.tiles_x * d.tiles_y);
        atomicOr(&cur[1 + seg.y * d.tiles_x + seg.x], or_seg);
        atomicOr(&cur[0], or_seg);
      }
    }
    __syncthreads();  // the U and digit slots are reused by the next segment
  }

  // ---- teardown -------------------------------------------------------------
  if (aborted && tid == 0) {
    atomicOr(d.status, 1);
    // let the copies and MMAs still in flight land (each wait bounded)
    for (int s = 0; s < kUSlots; ++s)
      if (tma_out & (1u << s)) mbar_wait(&bars[s], (uphase >> s) & 1u);
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
                                 int n_ctas) {
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
  cfg.numAttrs = MODE == TC_MODE_STEP ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, tc_stencil_kernel<MODE, S>, *tmap, d);
}

template <int MODE>
static cudaError_t st_launch_mode(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap,
                                  int stages, int n_ctas) {
  switch (stages) {
    case 1: return st_launch_one<MODE, 1>(s, d, tmap, n_ctas);
    case 2: return st_launch_one<MODE, 2>(s, d, tmap, n_ctas);
    case 3: return st_launch_one<MODE, 3>(s, d, tmap, n_ctas);
    case 4: return st_launch_one<MODE, 4>(s, d, tmap, n_ctas);
    default: return st_launch_one<MODE, 5>(s, d, tmap, n_ctas);
  }
}

// d.segs / d.seg_off / d.seg_mat / d.n_ctas describe the stencil segments
cudaError_t stencil_launch(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap, int mode) {
  if (d.n_ctas <= 0) return cudaSuccess;
  switch (mode) {
    case TC_MODE_STEP: return st_launch_mode<TC_MODE_STEP>(s, d, tmap, d.stages, d.n_ctas);
    case TC_MODE_KU: return st_launch_mode<TC_MODE_KU>(s, d, tmap, d.stages, d.n_ctas);
    default: return st_launch_mode<TC_MODE_PARTIALS>(s, d, tmap, d.stages, d.n_ctas);
  }
}
