// vfe_tc.cu -- OVFEM K u and central-difference step on GB300 tensor cores.
//
// Method (arXiv 2404.13683, Section 2, Eq. GE:TC and Eqs. intscaling,
// int8comp1, int8comp2): the element product is split so that the tensor core
// only ever multiplies small integers, and the partial products are
// recombined exactly.  GB300 (sm_103a) has no tcgen05 kind::i8, so the
// integer digits are carried exactly in fp16 (|digit| <= 1024, base 2^11) on
// tcgen05.mma kind::f16 with fp32 accumulation; every partial sum stays below
// 2^22 in magnitude, so the fp32 accumulator holds it exactly.
//
//   * The per-material integer matrices are K^kappa = 256/ds K_e(kappa=1,G=0)
//     and K^G' = Kbar^G + 128 I = 384/ds K_e(kappa=0,G=1); stacking them as
//     48 outputs of one MMA gives P = K^kappa q_e and Q = K^G' q_e, and
//     K_e u_e = ds (kappa/256 P + G/384 Q) (Eq. GE:TC with the kappa and G
//     parts kept separate, so the digits are per node, not per element).
//   * Scaling (Eq. intscaling): one power-of-two shift per step puts every
//     node value below 2^51 (q = floor(U / 2^shq)).
//   * Hierarchical split (Eq. int8comp1): q = sum_s 2^(11 s) d_s with balanced
//     digits d_s in [-1024, 1023] (offset-binary extraction), fp16-exact.
//   * Recombination (Eq. int8comp2): sum_s 2^(11 s) D_s in int64.
//
// The state is a 64-bit fixed-point value u = U * 2^-F with a power-of-two
// scale F that a one-thread prologue adjusts every step (FP64 is ~40x slower
// than INT32 on GB300, so the per-element arithmetic is integer end to end).
//
// Tiling: a CTA owns 15 x 15 node columns in x-y and a chunk of node planes in
// z, computes the 16 x 16 elements per layer that touch them (one element of
// halo), and marches up in z.  TMA brings node planes into a ring of shared
// memory slots four planes ahead.  Per element layer L: two warps issue the
// MMAs of its two M = 128 tiles (2 x stages x 2 MMAs, M=128, N=48, K=16) on
// digit planes L and L+1, written beforehand in the MN-major operand layout
// the tensor core reads directly (no im2col); the 512 threads read their
// element's 48 x stages accumulators from TMEM, recombine, apply the element's
// material and reduce to nodes (warp shuffle in x, shared memory in y,
// registers in z).  After the one CTA barrier of the layer, half of the
// threads update node plane L while the other half digitises plane L+3.
#include <cuda_fp16.h>

#include <cstring>

#include "vfe_internal.h"
#include "vfe_tc_common.cuh"

using namespace vfe_tc;

namespace {

// --------------------------------------------------------------------------
// shared-memory map (bytes)
// --------------------------------------------------------------------------
constexpr int kBlockBytes = 128;                          // one 8x8 fp16 core matrix
constexpr int kStageBytes = TC_NODES * 2 * kBlockBytes;   // 17 rows x 2 x-chunks
constexpr int kDigitSlotBytes = TC_MAX_STAGES * kStageBytes;
constexpr int kDigitSlots = 3;
constexpr int kUSlotBytes = 3 * TC_NODES * TC_BOXX * 8;   // TMA box (18,17,1,3) int64
constexpr int kUSlotStride = (kUSlotBytes + 127) / 128 * 128;  // TMA smem dst: 128-B aligned
constexpr int kUSlots = 8;                                 // node planes L .. L+4 in use
constexpr int kBopBytes = TC_N * 32 * 2;
constexpr int kYbufBytes = 2 * 2 * TC_EX * TC_EX * 3 * 8;  // half x layer parity
constexpr int kCbufBytes = 2 * TC_EX * TC_EX * 3 * 8;     // z carry, double buffered

constexpr int kOffDigits = 0;
constexpr int kOffU = kOffDigits + kDigitSlots * kDigitSlotBytes;
constexpr int kOffBop = kOffU + kUSlots * kUSlotStride;
constexpr int kOffYbuf = kOffBop + kBopBytes;
constexpr int kOffCbuf = kOffYbuf + kYbufBytes;
constexpr int kOffMat = kOffCbuf + kCbufBytes;
constexpr int kOffRecv = kOffMat + TC_MAX_MAT * (int)sizeof(TcMaterial);
constexpr int kOffDev = kOffRecv + TC_MAX_REC_CTA * (int)sizeof(TcRecv);
constexpr int kOffBar = kOffDev + ((int)sizeof(TcDevice) + 15) / 16 * 16;
constexpr int kOffMisc = kOffBar + 16 * 8;
constexpr int kSmemUsed = kOffMisc + 64;
// padded so that only one CTA fits per SM (it allocates 512 TMEM columns)
constexpr int kSmemBytes = kSmemUsed > 120 * 1024 ? kSmemUsed : 120 * 1024;

static_assert(kOffU % 128 == 0 && kUSlotStride % 128 == 0, "TMA destinations are 128-byte aligned");
static_assert(kDigitSlotBytes % 128 == 0 && kStageBytes % 128 == 0, "operand blocks 128-byte aligned");
static_assert(kOffBop % 16 == 0 && kOffYbuf % 16 == 0 && kOffBar % 8 == 0, "alignment");
static_assert(kSmemUsed <= 227 * 1024, "shared memory budget");

constexpr int kTmemCols = 512;
constexpr int kTileCols = TC_MAX_STAGES * TC_N;            // 240 columns per M tile

// instruction descriptor, kind::f16: D f32, A f16 MN-major, B f16 K-major,
// N = 48, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (1u << 15) | (0u << 16) |
                            ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);


}  // namespace

// ---------------------------------------------------------------------------
// The fused kernel.  MODE: 0 = time step, 1 = K u only (writes S), 2 = exact
// partial products per element (diagnostic).
//
// Work: CTA b walks the segments seg_off[b] .. seg_off[b+1]-1; a segment is a
// 15x15 node column (tx, ty) and a range of owned node planes [z0, z1).  The
// host balances column-planes across CTAs, so every SM gets the same work.
// ---------------------------------------------------------------------------
template <int MODE, int STAGES, bool BATCHED, bool DAMPED>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_step_kernel(const __grid_constant__ CUtensorMap tmap_u, const TcDevice d0,
                   const TcBatch b) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *digits = smem + kOffDigits;
  int64_t *uslot = reinterpret_cast<int64_t *>(smem + kOffU);
  uint16_t *bop = reinterpret_cast<uint16_t *>(smem + kOffBop);
  int64_t *ybuf = reinterpret_cast<int64_t *>(smem + kOffYbuf);
  int64_t *cbuf = reinterpret_cast<int64_t *>(smem + kOffCbuf);
  TcMaterial *smat = reinterpret_cast<TcMaterial *>(smem + kOffMat);
  TcRecv *srecv = reinterpret_cast<TcRecv *>(smem + kOffRecv);
  TcDevice *sdev = reinterpret_cast<TcDevice *>(smem + kOffDev);  // batch: current mesh
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);  // 0..7: U slots, 8,9: MMA tiles
  uint32_t *misc = reinterpret_cast<uint32_t *>(smem + kOffMisc);  // [0] tmem base, [1] abort

  const int tid = threadIdx.x;
  // the warp index broadcast from lane 0 is provably warp-uniform, so TMEM
  // addresses and MMA descriptors derived from it live in uniform registers
  const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0), lane = tid & 31;
  // a single mesh reads its arguments straight from the kernel parameters
  constexpr bool batched = BATCHED;
  // with fewer stages the low digits are dropped (the top ones carry the value)
  constexpr int s_lo = TC_MAX_STAGES - STAGES;

  // thread <-> element: TMEM lane m of tile t holds element (m % 16, 8 t + m / 16);
  // warps 0-7 take the corner groups with dz = 0, warps 8-15 those with dz = 1
  const int half = warp >> 3;
  const int tile = (warp >> 2) & 1;
  const int m_row = ((warp & 3) << 5) + lane;
  const int ei = m_row & 15;
  const int ej = 8 * tile + (m_row >> 4);

  // ---- one-time setup ------------------------------------------------------
  if (tid == 0) {
    misc[1] = 0;
    for (int i = 0; i < kUSlots; ++i) mbar_init(&bars[i], 1);
    mbar_init(&bars[8], 4);
    mbar_init(&bars[9], 4);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&misc[0])),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const uint16_t *bop_src = batched ? b.devs[0].Bop : d0.Bop;  // the same for every mesh
  for (int i = tid; i < kBopBytes / 16; i += TC_THREADS)
    reinterpret_cast<uint4 *>(bop)[i] = reinterpret_cast<const uint4 *>(bop_src)[i];
  if (!batched)
    for (int i = tid; i < d0.n_mat; i += TC_THREADS) smat[i] = d0.mats[i];
  {  // magic rows (lines 6 and 7 of every block) of every digit slot and stage
    const uint32_t mg = (uint32_t)__half_as_ushort(__float2half(TC_MAGIC_A));
    const uint4 mv = make_uint4(mg | (mg << 16), mg | (mg << 16), mg | (mg << 16), mg | (mg << 16));
    const int nblocks = kDigitSlots * TC_MAX_STAGES * TC_NODES * 2;
    for (int i = tid; i < 2 * nblocks; i += TC_THREADS) {
      const int blk = i >> 1, line = 6 + (i & 1);
      *reinterpret_cast<uint4 *>(digits + blk * kBlockBytes + line * 16) = mv;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // all 512 columns are allocated, so the allocation starts at lane 0, column 0
  const uint32_t tmem_base = misc[0];
  if (tmem_base != 0u) {  // cannot happen; fail loudly rather than use wrong columns
    if (tid == 0) atomicOr(batched ? b.devs[0].status : d0.status, 4);
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(kTmemCols));
    return;
  }

  // a time step is launched as a programmatic dependent of its prologue: the
  // setup above overlaps the prologue, the step parameters are read after it
  if constexpr (MODE == TC_MODE_STEP) asm volatile("griddepcontrol.wait;" ::: "memory");

  uint32_t uphase = 0;   // parity bit per U slot
  uint32_t mma_phase = 0;
  bool aborted = false;
  const TcMaterial zero_mat = {0, 0, 0, 0};
  int cur_mesh = -1;

  auto sync_abort = [&](bool ok) -> bool {  // true if the CTA must stop
    if (!ok) atomicExch(&misc[1], 1u);
    __syncthreads();
    return misc[1] != 0;
  };

  const int sbeg = batched ? b.seg_off[blockIdx.x] : d0.seg_off[blockIdx.x];
  const int send = batched ? b.seg_off[blockIdx.x + 1] : d0.seg_off[blockIdx.x + 1];
  for (int sg = sbeg; sg < send && !aborted; ++sg) {
    // the mesh of this segment: arguments and materials in shared memory
    if (batched) {
      const int mesh = b.seg_mesh[sg];
      if (mesh != cur_mesh) {
        __syncthreads();  // the previous mesh's copies are no longer read
        if (tid == 0) *sdev = b.devs[mesh];
        __syncthreads();
        for (int i = tid; i < sdev->n_mat; i += TC_THREADS) smat[i] = sdev->mats[i];
        __syncthreads();
        cur_mesh = mesh;
      }
    }
    const TcDevice &d = batched ? *sdev : d0;
    const CUtensorMap *tmap = batched ? &b.maps[cur_mesh] : &tmap_u;
    const TcStepParams P = *d.params;
    const int4 seg = batched ? b.segs[sg] : d.segs[sg];
    const int X0 = TC_OWN * seg.x - 1;  // global x of local element/node column 0
    const int Y0 = TC_OWN * seg.y - 1;
    const int Z0 = seg.z, Z1 = seg.w;   // owned node planes [Z0, Z1)
    const int xbox = X0 & ~1;           // TMA x must be even (16-byte rule)
    const int xo = X0 - xbox;           // local node ni sits at box x = ni + xo
    const int gi = X0 + ei + 1, gj = Y0 + ej + 1;  // this thread's node (ei+1, ej+1)
    const bool own_xy = (ei < TC_OWN) && (ej < TC_OWN) && gi <= d.nx && gj <= d.ny;
    const bool updater = own_xy && half == 0;  // half 0 owns the node update
    const int gx = X0 + ei, gy = Y0 + ej;          // this thread's element column
    const bool elem_xy = gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;

    // receivers of this segment (the previous segment's reads are fenced by
    // the barriers of its last layer)
    int nrec = 0;
    if (MODE == TC_MODE_STEP && d.n_rec > 0 && (P.trace_row >= 0 || P.inj_row >= 0)) {
      const int32_t *roff = batched ? b.recv_off : d.recv_off;
      const TcRecv *rv = batched ? b.recv : d.recv;
      const int rbeg = roff[sg];
      nrec = min(roff[sg + 1] - rbeg, TC_MAX_REC_CTA);
      for (int i = tid; i < nrec; i += TC_THREADS) srecv[i] = rv[rbeg + i];
    }

    auto issue_plane = [&](int p, int issuer) {  // TMA of node plane p into U slot p & 7
      if (tid == issuer) {
        const int s = p & 7;
        mbar_expect_tx(&bars[s], kUSlotBytes);
        tma_load_u(uslot + s * (kUSlotStride / 8), tmap, &bars[s], xbox, Y0, p);
      }
    };
    // every thread tracks the phase of every U slot; only the threads that
    // read a plane's slot wait on it
    auto wait_plane = [&](int p, bool do_wait) -> bool {
      const int s = p & 7;
      const bool ok = do_wait ? mbar_wait(&bars[s], (uphase >> s) & 1u) : true;
      uphase ^= 1u << s;
      return ok;
    };
    // digitise node plane p into digit slot p mod 3.  One task per (node row,
    // node pair, component) shifts three node values once and writes, for
    // every stage, the 32-bit word of the pair in the dx = 0 line (nodes 2k,
    // 2k+1) and in the dx = 1 line (nodes 2k+1, 2k+2).  With the offset-binary
    // bias boff = sum_s 1024 2^(11 s), digit s of q = floor(U/2^shq) is
    // ((q + boff) >> 11 s) & 2047 - 1024; q + boff is positive and below 2^55
    // because |q| < 2^51.  The float of that digit is exact: the bits
    // 0x4B000000 | x are 2^23 + x, and subtracting 2^23 + 1024 leaves x - 1024.
    constexpr int ntask = TC_NODES * 8 * 3;
    // digit quantum of this segment (Eq. intscaling, per node column): the
    // step uses the max |u| over the 3x3 node columns around the segment's
    // column (its elements' nodes) from the previous step, never more than the
    // global shift; K u and the diagnostic modes use the global shift
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
    // S of this segment is in units 2^(63 - e_ref + shq) of the raw state
    const int Rseg = P.eCref + P.rs - shq - 63;
    const int64_t dbias = (1LL << 10) | (1LL << 21) | (1LL << 32) | (1LL << 43) | (1LL << 54);
    unsigned long long or_seg = 0;
    // task t's offsets in a U slot (int64 words) and in a digit slot (bytes)
    auto task_src = [&](int t) {
      return ((t >> 3) % 3 * TC_NODES + t / 24) * TC_BOXX + 2 * (t & 7) + xo;
    };
    auto task_dst = [&](int t) {
      return (t / 24 * 2 + ((t & 7) >> 2)) * kBlockBytes + (t >> 3) % 3 * 16 + (t & 3) * 4;
    };
    auto digitise_at = [&](const int64_t *src, unsigned char *dst) {
      uint64_t v[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) v[i] = (uint64_t)((src[i] >> shq) + dbias);
#pragma unroll
      for (int s = s_lo; s < TC_MAX_STAGES; ++s) {
        float f[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          f[i] = __int_as_float((int)(((uint32_t)(v[i] >> (TC_DIGIT_BITS * s)) & 2047u) |
                                      0x4B000000u)) - 8389632.0f;
        const __half2 lo = __floats2half2_rn(f[0], f[1]);
        const __half2 hi = __floats2half2_rn(f[1], f[2]);
        *reinterpret_cast<__half2 *>(dst + s * kStageBytes) = lo;
        *reinterpret_cast<__half2 *>(dst + s * kStageBytes + 48) = hi;
      }
    };
    auto uslot_of = [&](int p) { return uslot + (p & 7) * (kUSlotStride / 8); };
    auto dslot_of = [&](int p) {
      return digits + ((p % kDigitSlots + kDigitSlots) % kDigitSlots) * kDigitSlotBytes;
    };
    auto digitise_task = [&](int p, int t) {
      digitise_at(uslot_of(p) + task_src(t), dslot_of(p) + task_dst(t));
    };
    // the second half's phase-2 tasks: t0 = tid - 256 and, below 408, t1 = tid
    const int t0 = tid - TC_THREADS / 2;
    const bool has_t1 = tid < ntask;
    const int src0 = task_src(t0 < 0 ? 0 : t0), dst0 = task_dst(t0 < 0 ? 0 : t0);
    const int src1 = task_src(has_t1 ? tid : 0), dst1 = task_dst(has_t1 ? tid : 0);
    // the MMAs of element layer L read digit planes L and L+1.
    // A (MN-major): 8-element chunks at 128 B, K groups (dy) at 256 B; B (K-major):
    // 8-row N groups at 128 B, K groups at 6*128 B.  Descriptors differ only in
    // the start-address field (address >> 4, below 2^14 for shared memory), so
    // they are formed by adding offsets to one base descriptor.
    const uint64_t adesc0 = make_sdesc(smem_u32(digits), 2 * kBlockBytes, kBlockBytes);
    const uint64_t bdesc0 = make_sdesc(smem_u32(bop), 6 * kBlockBytes, kBlockBytes);
    // the eight warps of the second half issue (that half has slack after the
    // barrier): tile w & 1, stages with (s - s_lo) mod 4 = (w >> 1) & 3; each
    // commits its own MMAs to the tile's mbarrier (four arrivals)
    auto issue_mma = [&](int L) {
      const int iw = warp - TC_THREADS / 64;
      if (iw < 0 || iw >= 8) return;
      const int mt = iw & 1, part = iw >> 1;
      tc_fence_after();
      const int sl0 = ((L % kDigitSlots) + kDigitSlots) % kDigitSlots;
      const int sl1 = sl0 == kDigitSlots - 1 ? 0 : sl0 + 1;
      const uint64_t a0 = adesc0 + (uint64_t)((sl0 * kDigitSlotBytes + 16 * mt * kBlockBytes) >> 4);
      const uint64_t a1 = adesc0 + (uint64_t)((sl1 * kDigitSlotBytes + 16 * mt * kBlockBytes) >> 4);
      const uint32_t tcol = (uint32_t)(mt * kTileCols);
#pragma unroll
      for (int s = s_lo; s < TC_MAX_STAGES; ++s) {
        if (((s - s_lo) & 3) != part) continue;
        const uint64_t off = (uint64_t)((s * kStageBytes) >> 4);
        mma_f16_elect(tcol + (uint32_t)(s * TC_N), a0 + off, bdesc0, kIdesc, 0);
        mma_f16_elect(tcol + (uint32_t)(s * TC_N), a1 + off,
                      bdesc0 + (uint64_t)((2 * 6 * kBlockBytes) >> 4), kIdesc, 1);
      }
      mma_commit_elect(&bars[8 + mt]);
    };

    // ---- segment prologue: planes Z0-1 .. Z0+2 ----------------------------
    // (a segment owns at least one plane, so planes up to Z0+1 = Lfirst+2 exist)
    const int Lfirst = Z0 - 1, Llast = Z1 - 1;
    issue_plane(Lfirst, 0);
    issue_plane(Lfirst + 1, 0);
    issue_plane(Lfirst + 2, 0);
    if (Lfirst + 3 <= Llast + 1) issue_plane(Lfirst + 3, 0);
    bool ok = wait_plane(Lfirst, true);
    ok = wait_plane(Lfirst + 1, true) && ok;
    ok = wait_plane(Lfirst + 2, true) && ok;
    if (sync_abort(ok)) { aborted = true; break; }
    for (int t = tid; t < ntask; t += TC_THREADS) {
      digitise_task(Lfirst, t);
      digitise_task(Lfirst + 1, t);
      digitise_task(Lfirst + 2, t);
    }
    fence_async_smem();
    __syncthreads();
    issue_mma(Lfirst);

    // material id of this thread's element, loaded one layer ahead
    auto mat_at = [&](int L) -> int {
      return (elem_xy && L >= 0 && L < d.nz)
                 ? d.mat[(int64_t)gx + (int64_t)d.nx * ((int64_t)gy + (int64_t)d.ny * L)]
                 : -1;
    };
    // per-element shear multiplier (meshes with per-element G), one layer ahead
    auto elemB_at = [&](int L) -> int64_t {
      return (d.elem_B && elem_xy && L >= 0 && L < d.nz)
                 ? d.elem_B[(int64_t)gx + (int64_t)d.nx * ((int64_t)gy + (int64_t)d.ny * L)]
                 : 0;
    };
    int m_next = mat_at(Lfirst);
    int64_t b_next = elemB_at(Lfirst);
    bool okp = true;  // plane waits of the previous layer's second phase
    for (int L = Lfirst; L <= Llast; ++L) {
      const int m = m_next;
      m_next = mat_at(L + 1);
      const int64_t b_elem = b_next;
      b_next = elemB_at(L + 1);
      int64_t uprev[3] = {0, 0, 0}, cn = 0, ucur_g[3] = {0, 0, 0};
      const bool upd = (MODE == TC_MODE_STEP) && updater && L >= Z0;
      const int64_t nidx = (int64_t)L * d.plane + (int64_t)gj * d.nxp + gi;
      if (upd) {
        cn = d.C[nidx];
#pragma unroll
        for (int c = 0; c < 3; ++c) uprev[c] = d.U_prev[c * d.comp + nidx];
        if constexpr (DAMPED) {  // the U slots hold w^n: u^n of this node from memory
#pragma unroll
          for (int c = 0; c < 3; ++c) ucur_g[c] = d.U_cur[c * d.comp + nidx];
        }
      }

      // (b) wait for this warp's tile of MMA(L)
      const bool okm = mbar_wait(&bars[8 + tile], mma_phase);
      mma_phase ^= 1u;
      if (!okm) atomicExch(&misc[1], 1u);
      tc_fence_after();

      // (c) epilogue: per corner group (dy, dz), stages x 12 columns
      const TcMaterial mt = m >= 0 ? smat[m] : zero_mat;
      const int A1 = (int)(mt.A >> 31), A0 = (int)(mt.A & 0x7FFFFFFF);
      const int64_t mB = (d.elem_B && m >= 0) ? b_elem : mt.B;
      const int B1 = (int)(mB >> 31), B0 = (int)(mB & 0x7FFFFFFF);
      const uint32_t tbase =
          tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(tile * kTileCols);
      int64_t own[3] = {0, 0, 0};  // this half's (dy = 1) corner sums
      int64_t *yb_half = ybuf + (2 * half + (L & 1)) * (TC_EX * TC_EX * 3);
#pragma unroll
      for (int gg = 0; gg < 2; ++gg) {
        const int g = 2 * half + gg;
        // this group's 12 outputs (dx, part, component) are 12 contiguous
        // columns per stage, recombined in Horner order while the next stage's
        // words load (two buffers of 12 words)
        const int c0 = 24 * half + 12 * gg;  // 0, 12, 24, 36
        const bool first8 = gg == 0;  // c0 = 24 half + 12 gg is 0 mod 8 iff gg = 0
        const int dy = g & 1, dz = g >> 1;
        uint64_t acc[12];
        uint32_t wa[12], wb[12];
        static_assert(STAGES >= 1 && STAGES <= TC_MAX_STAGES, "stages");
        if constexpr (s_lo == 0) {  // otherwise the loop loads stage s_lo first
          tmem_ld12(tbase + (uint32_t)(s_lo * TC_N + c0), first8, wa);
          tmem_wait_ld12(wa);
        }
#pragma unroll
        for (int s = 0; s < TC_MAX_STAGES; ++s) {
          // the words of stage s are in wa (s - s_lo even) or wb (odd);
          // dropped low digits contribute magic-only words
          uint32_t *cur = ((s - s_lo) & 1) ? wb : wa;
          uint32_t *nxt = ((s - s_lo) & 1) ? wa : wb;
          if (s + 1 < TC_MAX_STAGES && s + 1 >= s_lo)
            tmem_ld12(tbase + (uint32_t)((s + 1) * TC_N + c0), first8, nxt);
#pragma unroll
          for (int i = 0; i < 12; ++i) {
            const uint32_t w = s < s_lo ? (uint32_t)TC_MAGIC_BITS : cur[i];
            if (s == 0) recomb_stage<0>(acc[i], w);
            else if (s == 1) recomb_stage<1>(acc[i], w);
            else if (s == 2) recomb_stage<2>(acc[i], w);
            else if (s == 3) recomb_stage<3>(acc[i], w);
            else recomb_stage<4>(acc[i], w);
          }
          if (s + 1 < TC_MAX_STAGES && s + 1 >= s_lo) tmem_wait_ld12(nxt);
        }
        int64_t f0[3], f1[3];
        if constexpr (MODE == TC_MODE_PARTIALS) {
          if (elem_xy && L >= 0 && L < d.nz) {
            const int64_t e = (int64_t)gx + (int64_t)d.nx * ((int64_t)gy + (int64_t)d.ny * L);
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
              const int a = dx + 2 * dy + 4 * dz;
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                d.partials_out[e * 48 + 3 * a + c] = recomb_finish(acc[6 * dx + c]);
                d.partials_out[e * 48 + 24 + 3 * a + c] = recomb_finish(acc[6 * dx + 3 + c]);
              }
            }
          }
        } else {
          // material: t = (P A + Q B) / 2^63 in the mesh-wide unit
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            f0[c] = mul2_hi63(recomb_finish(acc[c]), recomb_finish(acc[3 + c]), A1, A0, B1, B0);
            f1[c] = mul2_hi63(recomb_finish(acc[6 + c]), recomb_finish(acc[9 + c]), A1, A0, B1, B0);
          }
        }
        if constexpr (MODE != TC_MODE_PARTIALS) {
          // x reduction: node (ei+1) gets dx=1 of element ei and dx=0 of ei+1
          int64_t v[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int64_t nb = __shfl_down_sync(0xffffffffu, f0[c], 1);
            v[c] = f1[c] + nb;  // lane ei = 15 reads the next row: its node is not owned
          }
          if (dy == 0) {
            int64_t *yb = yb_half + (ej * TC_EX + ei) * 3;
#pragma unroll
            for (int c = 0; c < 3; ++c) yb[c] = v[c];
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) own[c] = v[c];
          }
        }
      }
      // (d) TMEM reads done; digit writes visible to the tensor core; MMA(L+1)
      tc_fence_before();
      fence_async_smem();
      if (sync_abort(okp)) { aborted = true; break; }
      if (L + 1 <= Llast) issue_mma(L + 1);

      // second phase: half 1 digitises plane L+3 (read by MMA(L+2)) and
      // prefetches plane L+4 while half 0 updates plane L.  Every thread keeps
      // the U-slot phase bookkeeping; only half 1 waits.
      okp = true;
      if (L + 3 <= Llast + 1) okp = wait_plane(L + 3, half == 1);
      if (L + 4 <= Llast + 1) issue_plane(L + 4, TC_THREADS / 2);
      if (half == 1 && L + 3 <= Llast + 1) {
        const int64_t *us = uslot_of(L + 3);
        unsigned char *ds = dslot_of(L + 3);
        digitise_at(us + src0, ds + dst0);
        if (has_t1) digitise_at(us + src1, ds + dst1);
      }
      if constexpr (MODE == TC_MODE_PARTIALS) continue;

      // (e) y reduction from the shared buffer.  Half 1 holds the forces of
      // layer L on plane L+1 and hands them to half 0 for the next layer through
      // the double-buffered carry; half 0 completes plane L.
      if (ej < TC_EX - 1) {
        const int64_t *yv = yb_half + ((ej + 1) * TC_EX + ei) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) own[c] += yv[c];
      }
      int64_t *cb_next = cbuf + ((L + 1) & 1) * (TC_EX * TC_EX * 3) + (ej * TC_EX + ei) * 3;
      const int64_t *cb_cur = cbuf + (L & 1) * (TC_EX * TC_EX * 3) + (ej * TC_EX + ei) * 3;
      if (half == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) cb_next[c] = own[c];
        continue;
      }
      int64_t S[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) S[c] = (L == Lfirst ? 0 : cb_cur[c]) + own[c];

      // (f) update / output of node (gi, gj, L)
      if (own_xy && L >= Z0) {
        if (MODE == TC_MODE_KU) {
#pragma unroll
          for (int c = 0; c < 3; ++c) d.S_out[c * d.comp + nidx] = S[c];
        } else if (MODE == TC_MODE_STEP) {
          // plane L's slot completed its phase before half 1 digitised it; the
          // test acquires that completion for these reads
          if (!mbar_test_wait(&bars[L & 7], ((uphase >> (L & 7)) & 1u) ^ 1u)) atomicExch(&misc[1], 1u);
          const int64_t *ucur = uslot + (L & 7) * (kUSlotStride / 8);
          const bool is_src = (nidx == d.src_node);
          // du = round(S C / 2^R): for R >= 63 (the usual case: C < 2^62 and
          // |S| < 2^63) from the high product floor(S C / 2^63), within a few
          // units of the 59-bit state; otherwise exactly in 128 bits
          const int C1 = (int)(cn >> 31), C0 = (int)(cn & 0x7FFFFFFF);
          const bool rescaled = (P.rs | P.rs_prev) != 0;
          int64_t unew[3], uold[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            int64_t u0 = DAMPED ? ucur_g[c] : ucur[(c * TC_NODES + ej + 1) * TC_BOXX + ei + 1 + xo];
            int64_t um = uprev[c];
            if (rescaled) {
              u0 = shr_round(u0, P.rs);
              um = shr_round(um, P.rs + P.rs_prev);
            }
            int64_t du;
            if (Rseg >= 63) {
              const int64_t H = mul_hi63(S[c], C1, C0);
              const int sh = Rseg - 63;
              du = sh == 0 ? H : (sh > 62 ? 0 : (H + ((int64_t)1 << (sh - 1))) >> sh);
            } else {
              if (Rseg > 0) {
                du = mul_shr_round(S[c], cn, Rseg);
              } else {  // the state is being scaled up: exact left shift
                const __int128 prod = (__int128)S[c] * (__int128)cn;
                du = (int64_t)(prod << min(-Rseg, 63));
              }
            }
            int64_t un;
            if constexpr (DAMPED) {  // 2 g u^n - (1 - a) g u^{n-1} - C S, rounded
              const int64_t t0 = (int64_t)(((__int128)u0 * d.dG + ((__int128)1 << 60)) >> 61);
              const int64_t t1 = (int64_t)(((__int128)um * d.dH + ((__int128)1 << 61)) >> 62);
              un = t0 - t1 - du;
            } else {
              un = 2 * u0 - um - du;
            }
            if (is_src) un += P.dU_src[c];
            unew[c] = un;
            uold[c] = u0;
          }
          // injected increments at receiver nodes (the adjoint's residual source)
          if (P.inj_row >= 0)
            for (int r = 0; r < nrec; ++r) {
              const TcRecv rv = srecv[r];
              if (rv.ei == ei && rv.ej == ej && rv.k == L) {
                const double *iv = d.inj + (P.inj_row * d.n_rec + rv.r) * 3;
#pragma unroll
                for (int c = 0; c < 3; ++c) unew[c] += llrint(ldexp(iv[c], P.F));
              }
            }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if (cn == 0) unew[c] = 0;  // fixed or massless node
            d.U_next[c * d.comp + nidx] = unew[c];
            if constexpr (DAMPED) {  // w^{n+1} = u^{n+1} + b (u^{n+1} - u^n), bounded too
              const int64_t wn =
                  unew[c] + (int64_t)(((__int128)(unew[c] - uold[c]) * d.dB + ((__int128)1 << 61)) >> 62);
              d.W_next[c * d.comp + nidx] = wn;
              or_seg |= (unsigned long long)(wn < 0 ? -wn : wn);
            }
            // the slot bounds u^{n+1} and u^n (both in the new units)
            or_seg |= (unsigned long long)(unew[c] ^ (unew[c] >> 63)) |
                      (unsigned long long)(uold[c] ^ (uold[c] >> 63));
          }
          if (P.trace_row >= 0)
            for (int r = 0; r < nrec; ++r) {
              const TcRecv rv = srecv[r];
              if (rv.ei == ei && rv.ej == ej && rv.k == L) {
                double *out = d.traces + (P.trace_row * d.n_rec + rv.r) * 3;
#pragma unroll
                for (int c = 0; c < 3; ++c) out[c] = ldexp((double)unew[c], -P.F);
              }
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
    __syncthreads();  // srecv and the U slots are reused by the next segment
  }

  // ---- teardown -------------------------------------------------------------
  if (aborted && tid == 0) atomicOr(batched ? b.devs[0].status : d0.status, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// per-step prologue: rescale decision, digit shift, source increment
// ---------------------------------------------------------------------------
// persist[0] = F of u^n, [1] = step, [2] = trace rows, [3] unused,
// [4] = eC + e_ref, [5] = shift of the last step
// (u^{n-1} has F + [5]), [6] = first step of the injection array (-1: none),
// [7] = first step of the explicit force series (-1: none)
// One mesh's prologue, run by a block (thread 0 does the scalar work).
__device__ void prologue_body(const TcPrologueArgs &A) {
  int64_t *persist = A.persist;
  unsigned long long *or_slots = A.or_slots;
  const int ncols = A.ncols;
  const int64_t n = persist[1];
  // clear the slot (global + per column) that the next step will OR into
  unsigned long long *next = or_slots + (size_t)((n + 1) % 3) * (1 + ncols);
  for (int i = threadIdx.x; i < 1 + ncols; i += blockDim.x) next[i] = 0;
  if (threadIdx.x != 0) return;
  const int F_old = (int)persist[0];
  const unsigned long long orp = or_slots[(size_t)((n + 2) % 3) * (1 + ncols)];
  // bit lengths of max|u^n|, max|u^{n-1}| (raw units) and of the source
  // increment at the old scale; 'valid' flags separate zero from tiny
  const int b = orp ? 64 - __clzll((long long)orp) : 0;
  double src[3] = {0.0, 0.0, 0.0};
  int bs = 0;
  bool bs_valid = false;
  if (A.have_src) {
    // F^n = amp ricker(n dt) dir, or the caller's row of an explicit force
    // series, scaled by dt^2 / m of the source node
    const int64_t frow = n - persist[7];
    if (persist[7] >= 0 && A.force) {
      if (frow >= 0 && frow < A.force_rows) {
        for (int c = 0; c < 3; ++c) src[c] = A.force_scale * A.force[3 * frow + c];
      } else {
        atomicOr(A.status, 8);  // a forced step beyond the supplied rows: no force
      }
    } else {
      const double fv = A.amp_scale * ricker_wavelet((double)n * A.dt, A.f0, A.t0);
      for (int c = 0; c < 3; ++c) src[c] = fv * A.dir[c];
    }
    double mx = 0.0;
    for (int c = 0; c < 3; ++c) mx = fmax(mx, fabs(src[c]));
    if (mx > 0.0) {
      bs = ilogb(mx) + F_old + 1;
      bs_valid = true;
    }
  }
  if (persist[6] >= 0 && A.inj) {  // injected increments count like the source
    const double *row = A.inj + (n - persist[6]) * A.n_inj;
    double mx = 0.0;
    for (int i = 0; i < A.n_inj; ++i) mx = fmax(mx, fabs(row[i]));
    if (mx > 0.0) {
      const int bi = ilogb(mx) + F_old + 1;
      bs = bs_valid ? max(bs, bi) : bi;
      bs_valid = true;
    }
  }
  int rs = 0;
  if (orp || bs_valid) {
    const int bb = orp ? (bs_valid ? max(b, bs) : b) : bs;
    rs = max(-200, min(200, bb - TC_UNITS_BITS));
  }
  const int F_new = F_old - rs;
  const int shq = max(0, b - TC_QBITS);
  const int R = (int)persist[4] + rs - shq - 63;
  TcStepParams p;
  p.step = n;
  p.trace_row = A.trace_on ? persist[2] : -1;
  p.inj_row = persist[6] >= 0 ? n - persist[6] : -1;
  for (int c = 0; c < 3; ++c) p.dU_src[c] = A.have_src ? llrint(ldexp(src[c], F_new)) : 0;
  p.rs = rs;
  p.shq = shq;
  p.R = R;
  p.F = F_new;
  p.or_slot = (int)(n % 3);
  p.rs_prev = (int)persist[5];
  p.eCref = (int)persist[4];
  p.pad = 0;
  if (F_new < -2000 || F_new > 2000) atomicOr(A.status, 2);
  *A.params = p;
  persist[0] = F_new;
  persist[5] = rs;
  persist[1] = n + 1;
  if (A.trace_on) persist[2] += 1;
}

// Each prologue lets its step kernel launch at once (that kernel waits for the
// prologue's results before reading them).
__global__ void tc_prologue_kernel(const TcPrologueArgs A) {
  asm volatile("griddepcontrol.launch_dependents;");
  prologue_body(A);
}

__global__ void tc_batch_prologue_kernel(const TcPrologueArgs *args) {
  asm volatile("griddepcontrol.launch_dependents;");
  prologue_body(args[blockIdx.x]);
}

int tc_smem_bytes() { return kSmemBytes; }

cudaError_t tc_launch_prologue_ex(cudaStream_t s, TcStepParams *params, int64_t *persist,
                                  const TcSource &src, unsigned long long *or_slots, int ncols,
                                  int have_src, int trace_on, int *status, const double *inj,
                                  int n_inj) {
  TcPrologueArgs A;
  A.params = params;
  A.persist = persist;
  A.or_slots = or_slots;
  A.status = status;
  A.amp_scale = src.amp_scale;
  A.dt = src.dt;
  A.f0 = src.f0;
  A.t0 = src.t0;
  for (int c = 0; c < 3; ++c) A.dir[c] = src.dir[c];
  A.ncols = ncols;
  A.have_src = have_src;
  A.trace_on = trace_on;
  A.n_inj = n_inj;
  A.inj = inj;
  A.force = src.force;
  A.force_scale = src.force_scale;
  A.force_rows = src.force_rows;
  tc_prologue_kernel<<<1, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t tc_launch_batch_prologue(cudaStream_t s, const TcPrologueArgs *args, int n_meshes) {
  tc_batch_prologue_kernel<<<n_meshes, 256, 0, s>>>(args);
  return cudaGetLastError();
}

template <int MODE, int S, bool BATCHED>
static cudaError_t set_attr() {
  return cudaFuncSetAttribute(tc_step_kernel<MODE, S, BATCHED, false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

template <int S>
static cudaError_t set_attr_damped() {
  return cudaFuncSetAttribute(tc_step_kernel<TC_MODE_STEP, S, false, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

template <int MODE, bool BATCHED>
static cudaError_t set_attr_all() {
  cudaError_t e;
  if ((e = set_attr<MODE, 1, BATCHED>()) != cudaSuccess) return e;
  if ((e = set_attr<MODE, 2, BATCHED>()) != cudaSuccess) return e;
  if ((e = set_attr<MODE, 3, BATCHED>()) != cudaSuccess) return e;
  if ((e = set_attr<MODE, 4, BATCHED>()) != cudaSuccess) return e;
  return set_attr<MODE, 5, BATCHED>();
}

cudaError_t tc_prepare() {
  cudaError_t e;
  if ((e = set_attr_all<TC_MODE_STEP, false>()) != cudaSuccess) return e;
  if ((e = set_attr_all<TC_MODE_STEP, true>()) != cudaSuccess) return e;
  if ((e = set_attr_all<TC_MODE_KU, false>()) != cudaSuccess) return e;
  if ((e = set_attr_all<TC_MODE_PARTIALS, false>()) != cudaSuccess) return e;
  for (cudaError_t (*f)() : {&set_attr_damped<1>, &set_attr_damped<2>, &set_attr_damped<3>,
                             &set_attr_damped<4>, &set_attr_damped<5>})
    if ((e = f()) != cudaSuccess) return e;
  return cudaSuccess;
}

template <int MODE, int S, bool BATCHED, bool DAMPED = false>
static cudaError_t launch_one(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap,
                              const TcBatch &b, int n_ctas) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(n_ctas);
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  // time steps follow their prologue as programmatic dependents
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = MODE == TC_MODE_STEP ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, tc_step_kernel<MODE, S, BATCHED, DAMPED>, *tmap, d, b);
}

template <int MODE, bool BATCHED, bool DAMPED = false>
static cudaError_t launch_mode(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap,
                               const TcBatch &b, int stages, int n_ctas) {
  switch (stages) {
    case 1: return launch_one<MODE, 1, BATCHED, DAMPED>(s, d, tmap, b, n_ctas);
    case 2: return launch_one<MODE, 2, BATCHED, DAMPED>(s, d, tmap, b, n_ctas);
    case 3: return launch_one<MODE, 3, BATCHED, DAMPED>(s, d, tmap, b, n_ctas);
    case 4: return launch_one<MODE, 4, BATCHED, DAMPED>(s, d, tmap, b, n_ctas);
    default: return launch_one<MODE, 5, BATCHED, DAMPED>(s, d, tmap, b, n_ctas);
  }
}

cudaError_t tc_launch_step(cudaStream_t s, const TcDevice &d, const CUtensorMap *tmap, int mode) {
  TcBatch none;
  memset(&none, 0, sizeof(none));
  switch (mode) {
    case TC_MODE_STEP:
      if (d.damped) return launch_mode<TC_MODE_STEP, false, true>(s, d, tmap, none, d.stages, d.n_ctas);
      return launch_mode<TC_MODE_STEP, false>(s, d, tmap, none, d.stages, d.n_ctas);
    case TC_MODE_KU: return launch_mode<TC_MODE_KU, false>(s, d, tmap, none, d.stages, d.n_ctas);
    default: return launch_mode<TC_MODE_PARTIALS, false>(s, d, tmap, none, d.stages, d.n_ctas);
  }
}

// All meshes of a batch in one launch (the tensor-map and device-struct
// arguments of the single-mesh form are unused placeholders here).
cudaError_t tc_launch_batch_step(cudaStream_t s, const TcBatch &b, int stages) {
  TcDevice none;
  memset(&none, 0, sizeof(none));
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  return launch_mode<TC_MODE_STEP, true>(s, none, &dummy, b, stages, b.n_ctas);
}
