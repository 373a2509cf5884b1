// Tensor-core fused pass (tcgen05 + TMA) for FP32 or bf16-stored D and compiled rank R <= 16.
//
// Same quantities as the SIMT pass (pass_impl.cuh): per entry of D, rebuild L_ij, take
// R_ij = D_ij - L_ij, the strict threshold S_ij = R_ij if |R_ij| > zeta_k (Eq. (10)),
// the residual sum over unthresholded entries (Eq. (11)) and Z = D - S_k; accumulate
// Y1 = Z V~ and Y2 = Z^T U~ (Section 2.1).  D is read once from HBM.
//
// Work decomposition.  D is cut into 128 x 64 tiles, and the tiles into row groups of
// different heights (one CTA per SM; the host's plan balances the tile counts): CTA (a, b)
// owns row group a's row tiles and the b-th range of column tiles, and walks them row tile by
// row tile.  Y1 for the current row tile and Y2 for every column tile of the CTA stay in
// tensor memory, so each CTA writes one Y1 partial per row (slice b) and, per column, the
// Z_hi and Z_lo parts of one Y2 partial (slices 2a, 2a + 1), added up chunk by chunk.
//
// Per tile (RK = 8 for R <= 8, RK = 16 for R <= 16: the operand image layout, tc_images.cuh):
//   TMA (warp 0)     : D tile (two 128 x 32 FP32 boxes, or one 128 x 64 bf16 box per part,
//                      128-byte swizzle) plus the operand images of V (tf32 hi/lo) and V~
//                      (bf16 hi/lo) -> stage s (5 stages for RK = 8, 4 for RK = 16); the W
//                      and U~ images once per 128-row block (double-buffered)
//   L MMAs (warp 1)  : L = W_hi V_hi^T + W_hi V_lo^T + W_lo V_hi^T, kind::tf32, M128 N64,
//                      3 (RK = 8) or 6 (RK = 16) k-steps of 8 over the [hi | lo] images
//                      (three-term split product: FP32-level accuracy of the K = r rebuild)
//   epilogue (16 warps, two groups of 8 on alternate tiles): L from TMEM, D from shared
//                      memory, threshold, residual, support count, Z split into bf16 hi + lo,
//                      written 128B-swizzled over the very bytes of D it came from, so a stage
//                      carries its own Z and no warp waits for another: FP32 D, box h (columns
//                      32h .. 32h+31) becomes [Z_hi | Z_lo] of those columns; bf16 D, Z_hi
//                      over the hi tile and Z_lo over the lo tile
//   Y1 MMAs (warp 2) : Y1 += [Z_hi | Z_lo] [V~_hi | V~_lo], kind::f16, M128 N(2 RK) K64 (x2)
//   Y2 MMAs (warp 3) : Y2 += [Z_hi^T ; Z_lo^T] [U~_hi | U~_lo], M128 (MN-major A) N(2 RK) K128;
//                      the stage is released when both have completed
// Each product has its own issuing thread: a tcgen05.mma of these small shapes costs about
// 40 cycles of tensor-pipe time but about 55 cycles of issue time on one thread, and a single
// issuer would also hold the Y products of tile t behind the TMA arrival of tile t + 1.
// The column halves of the N = 2 RK accumulators (hi and lo parts of V~, U~) and the two M
// halves of the Y2 accumulator (Z_hi, Z_lo) are added when the accumulators are drained.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "factor.cuh"
#include "tc_images.cuh"
#include "tc_util.cuh"

namespace rpca {

namespace {

using namespace tc;

constexpr int BM = img::BM, BN = img::BN;
constexpr int D_BYTES = BM * BN * 4;          // 32 KB: FP32 tile, or bf16 hi + lo tiles
constexpr int Z_BYTES = 2 * BM * BN * 2;      // hi + lo, 32 KB, in place of the D tile
constexpr int OFF_STAGE = 0;
constexpr int NBAR = 112;
constexpr int G2 = kTcY2Chunk;  // row tiles per Y2 accumulation chunk
constexpr int CT_BARS = 20;     // column tiles per CTA with their own Y2 chunk barriers
constexpr int EPI_WARPS = 16;
constexpr int THREADS = 128 + 32 * EPI_WARPS;  // warp 0 TMA, 1 L MMAs, 2 Y1 MMAs, 3 Y2 MMAs, 4..19 epilogue
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int TMEM_COLS = 512;
static_assert(Z_BYTES == D_BYTES, "Z replaces the D tile");

// Shared-memory and tensor-memory plan for image layout RK.
template <int RK>
struct Cfg {
  using Lay = img::Layout<RK>;
  static constexpr int NSTAGE = RK == 8 ? 5 : 4;
  static constexpr int VOP_BYTES = Lay::VOP_BYTES;    // 4 / 8 KB   [64 x 2RK] tf32
  static constexpr int VTOP_BYTES = Lay::VTOP_BYTES;  // 2 / 4 KB   [2RK x 64] bf16
  static constexpr int UTOP_BYTES = Lay::UTOP_BYTES;  // 4 / 8 KB   2 x [2RK x 64] bf16
  static constexpr int WOP_BYTES = Lay::WOP_BYTES;    // 8 / 16 KB  [128 x 2RK] tf32
  static constexpr int STAGE_BYTES = D_BYTES + VOP_BYTES + VTOP_BYTES;  // 38 / 44 KB
  static constexpr int OFF_W = NSTAGE * STAGE_BYTES;  // [2] W images
  static constexpr int OFF_U = OFF_W + 2 * WOP_BYTES;  // [2] U~ images
  static constexpr int OFF_BAR = OFF_U + 2 * UTOP_BYTES;
  static constexpr int SMEM_BYTES = OFF_BAR + NBAR * 8 + 256 + 1024;  // + alignment slack
  // W and V images: 64-byte rows with the 64-byte swizzle (RK = 8) or 128-byte rows with the
  // 128-byte swizzle; 8-row groups SBO apart; descriptor swizzle codes 4 and 2
  static constexpr uint32_t TF_SBO = 8 * Lay::ROW_BYTES, TF_SWZ = RK == 8 ? 4 : 2;
  static constexpr int NY = 2 * RK;                   // Y accumulator columns: hi and lo halves
  static constexpr int LK = RK == 8 ? 3 : 6;          // k-steps of the L product
  static constexpr int TM_Y1 = 2 * BN, TM_Y2 = TM_Y1 + 2 * NY;
  static constexpr int MAX_CT = (TMEM_COLS - TM_Y2) / NY;  // column tiles whose Y2 fits in TMEM
  static_assert(STAGE_BYTES % 1024 == 0 && OFF_W % 1024 == 0 && OFF_U % 1024 == 0 && WOP_BYTES % 1024 == 0 &&
                    UTOP_BYTES % 1024 == 0,
                "1024-byte aligned operands");
  static_assert((D_BYTES + VOP_BYTES) % 1024 == 0, "1024-byte aligned images");
  static_assert(SMEM_BYTES <= 232448, "shared memory");
  static_assert(NSTAGE <= 8, "barrier slots");
  static_assert(CT_BARS >= (RK == 8 ? 20 : 10), "Y2 chunk barriers for tc_max_col_tiles");
};

// barrier slots
enum {
  B_FULL = 0,      // [NSTAGE <= 8]
  B_EMPTY = 8,     // [NSTAGE]
  B_ZFULL = 16,    // [NSTAGE]
  B_LFULL = 24,    // [2]
  B_LEMPTY = 26,   // [2]
  B_WFULL = 28,    // [2] W and U~ images of a 128-row block
  B_WEMPTY = 30,   // [2] released by the last L and the last Y2 products of the block
  B_Y1FULL = 32,   // [2]
  B_Y1EMPTY = 34,  // [2]
  B_YFIN = 36,
  B_DRAIN = 37,
  B_LDRAIN = 70,
  B_Y1DRAIN = 71,
  B_Y2DONE = 72,   // [CT_BARS]: the MMAs of a non-final Y2 chunk of column tile ctl completed
  B_Y2FREE = 92    // [CT_BARS]: that chunk has been read out of tensor memory
};
static_assert(B_Y2FREE + CT_BARS <= NBAR, "barrier slots");

constexpr uint32_t kErrTimeout = 6;

template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

struct TcArgs {
  int m, n, R;
  int ncta, TR, TC;
  const int4* rect;
  const int4* ids;
  const uint8_t* wop;
  const uint8_t* vop;
  const uint8_t* vtop;
  const uint8_t* utop;
  const DevState* st;
  int* status;
  float* P1;
  float* P2;
  double* resP;
  unsigned long long* nnzP;
  unsigned* masks;
  long long mask_wr;
  unsigned* swords;
  int nw;
  int* emit_k;
  const float* tgram;
  int tnb, tw, tcta;
  float* tfac;
  unsigned long long* chgP;
};

// Variants of the epilogue: the plain pass; with the support bitmask of the learned schedule;
// with partially observed D (NaN entries unobserved).
enum { MODE_PLAIN = 0, MODE_MASK = 1, MODE_PARTIAL = 2 };

__device__ __forceinline__ void fail(const TcArgs& a, volatile int* abort_flag) {
  atomicCAS(a.status, 0, (int)kErrTimeout);
  *abort_flag = 1;
}

// Z layout in a stage (descriptor units of 16 bytes for the Y1 k-steps of 16 columns), and
// which column and which part (Z_hi or Z_lo) a row of the Y2 accumulator holds.  DM = 0: box h (16 KB) holds
// [Z_hi | Z_lo] of columns 32h .. 32h+31; DM = 1: Z_hi in the first 16 KB, Z_lo in the second.
template <int DM>
__device__ __forceinline__ uint64_t zhi_off(int k) {
  return DM == 0 ? (uint64_t)((k >> 1) * ((D_BYTES / 2) >> 4) + 2 * (k & 1)) : (uint64_t)(2 * k);
}
template <int DM>
__device__ __forceinline__ uint64_t zlo_off(int k) {
  return DM == 0 ? zhi_off<0>(k) + 4 : (uint64_t)(((Z_BYTES / 2) >> 4) + 2 * k);
}
template <int DM>
__device__ __forceinline__ int y2_row_col(int row) {
  return DM == 0 ? (row >> 6) * 32 + (row & 31) : (row & 63);
}
template <int DM>
__device__ __forceinline__ int y2_row_part(int row) {
  return DM == 0 ? ((row >> 5) & 1) : (row >> 6);
}

// NY consecutive accumulator columns of this warp's 32 lanes.
template <int NY>
__device__ __forceinline__ void tmem_ld_y(uint32_t taddr, uint32_t (&v)[NY]) {
  if constexpr (NY == 16)
    tmem_ld16(taddr, v);
  else
    tmem_ld32(taddr, v);
}

// DM = 0: D is FP32 (dmap, two 128 x 32 boxes per tile).  DM = 1: D is held as bf16 hi and
// lo parts (dmap = hi, dmap_lo = lo, one 128 x 64 box each); the lo part is read only once
// DevState.use_lo is set, and D = hi + lo (exact in FP32).  Either way the tile's D area is
// 32 KB and Z is written over it (where: zhi_off / zlo_off).  RK: operand image layout (8 or 16).
// MODE_MASK: also write the support as a bitmask, from which count_mask_changes takes the
// entries whose membership differs from the previous pass's (the learned schedule's
// support-change statistic).  Layout, tile-major so that a warp's 32 rows are 32 consecutive
// words: word
// ((rt TC + ct) 2 + h) 128 + row-in-tile holds columns 64 ct + 32 h .. + 31 of that row.
// MODE_PARTIAL: a NaN entry of D is unobserved: it is outside the support and the residual,
// and Z = L there; an observed entry outside the support gets Z = L + (D - L) / p (the step of
// the partially observed iteration, DevState.inv_p = 1 / p).
template <int DM, int RK, int MODE>
__global__ void __launch_bounds__(THREADS, 1) fused_pass_tc(const __grid_constant__ CUtensorMap dmap,
                                                            const __grid_constant__ CUtensorMap dmap_lo, TcArgs a) {
  using C = Cfg<RK>;
  constexpr bool MASK = MODE == MODE_MASK, PO = MODE == MODE_PARTIAL;
  constexpr int NSTAGE = C::NSTAGE, STAGE_BYTES = C::STAGE_BYTES, OFF_W = C::OFF_W, OFF_U = C::OFF_U;
  constexpr int OFF_BAR = C::OFF_BAR;
  constexpr int VOP_BYTES = C::VOP_BYTES, VTOP_BYTES = C::VTOP_BYTES, UTOP_BYTES = C::UTOP_BYTES;
  constexpr int WOP_BYTES = C::WOP_BYTES, NY = C::NY, TM_Y1 = C::TM_Y1, TM_Y2 = C::TM_Y2;
  if (a.st->done) return;
  const bool use_lo = DM == 1 && a.st->use_lo != 0;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ double red_res[EPI_WARPS];
  __shared__ unsigned long long red_nnz[EPI_WARPS];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cta = blockIdx.x;
  // this CTA's rectangle of tiles and its slices of the partial products (host plan)
  const int4 rc = a.rect[cta];
  const int4 id = a.ids[cta];
  const int bi = id.y, p2base = id.z;  // Y1 slice; Y2 slices of the row group (Z_hi, Z_lo parts)
  const int rt0 = rc.x, rt1 = rc.y, ct0 = rc.z, ct1 = rc.w;
  const int nrt = rt1 - rt0, nct = ct1 - ct0;
  const int ntiles = nrt * nct;
  // the host's partition keeps a CTA's column tiles within the tensor-memory and barrier
  // budget; refuse a launch that does not
  if (nct > C::MAX_CT || nct > CT_BARS) {
    if (tid == 0) atomicCAS(a.status, 0, 1);
    return;
  }

  // producer (thread 0): copies of tile t into stage t % NSTAGE, and the W and U~ images of
  // its 128-row block when t starts one; false if a wait gave up.  (Issuing the first tiles
  // before the block barrier, while the tensor memory is allocated, made the pass ~2 us slower
  // per launch, measured at 10^4 x 10^4.)
  int issued = 0, w_issued = 0;
  // D is read once per pass: its lines go first when L2 needs room, which keeps the operand
  // images, the partial products and the other kernels' code and data resident
  const uint64_t dpol = l2_evict_first_policy();
  auto issue = [&](int t) -> bool {
    const int rtl = t / nct, ctl = t % nct, s = t % NSTAGE;
    const int rt = rt0 + rtl, ct = ct0 + ctl;
    if (ctl == 0) {
      const int wb = rtl & 1;
      if (rtl >= 2 && !mbar_wait(&bar[B_WEMPTY + wb], ((rtl - 2) >> 1) & 1)) {
        fail(a, &abort_flag);
        return false;
      }
      mbar_arrive_expect_tx(&bar[B_WFULL + wb], WOP_BYTES + UTOP_BYTES);
      bulk_load(sm + OFF_W + wb * WOP_BYTES, a.wop + (size_t)rt * WOP_BYTES, WOP_BYTES, &bar[B_WFULL + wb]);
      bulk_load(sm + OFF_U + wb * UTOP_BYTES, a.utop + (size_t)rt * UTOP_BYTES, UTOP_BYTES, &bar[B_WFULL + wb]);
      w_issued = rtl + 1;
    }
    if (t >= NSTAGE && !mbar_wait(&bar[B_EMPTY + s], ((t - NSTAGE) / NSTAGE) & 1)) {
      fail(a, &abort_flag);
      return false;
    }
    uint8_t* st = sm + OFF_STAGE + s * STAGE_BYTES;
    if (DM == 0) {
      mbar_arrive_expect_tx(&bar[B_FULL + s], STAGE_BYTES);
      tma_load_2d_hint(st, &dmap, ct * BN, rt * BM, &bar[B_FULL + s], dpol);
      tma_load_2d_hint(st + D_BYTES / 2, &dmap, ct * BN + 32, rt * BM, &bar[B_FULL + s], dpol);
    } else {
      mbar_arrive_expect_tx(&bar[B_FULL + s], STAGE_BYTES - (use_lo ? 0 : D_BYTES / 2));
      tma_load_2d_hint(st, &dmap, ct * BN, rt * BM, &bar[B_FULL + s], dpol);
      if (use_lo) tma_load_2d_hint(st + D_BYTES / 2, &dmap_lo, ct * BN, rt * BM, &bar[B_FULL + s], dpol);
    }
    bulk_load(st + D_BYTES, a.vop + (size_t)ct * VOP_BYTES, VOP_BYTES, &bar[B_FULL + s]);
    bulk_load(st + D_BYTES + VOP_BYTES, a.vtop + (size_t)ct * VTOP_BYTES, VTOP_BYTES, &bar[B_FULL + s]);
    issued = t + 1;
    return true;
  };

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&bar[B_FULL + s], 1);
      mbar_init(&bar[B_EMPTY + s], 2);  // Y1 and Y2 issuers
      mbar_init(&bar[B_ZFULL + s], EPI_WARPS / 2);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar[B_LFULL + i], 1);
      mbar_init(&bar[B_LEMPTY + i], EPI_WARPS / 2);
      mbar_init(&bar[B_WFULL + i], 1);
      mbar_init(&bar[B_WEMPTY + i], 2);  // L and Y2 issuers
      mbar_init(&bar[B_Y1FULL + i], 1);
      mbar_init(&bar[B_Y1EMPTY + i], 4);
    }
    mbar_init(&bar[B_YFIN], 1);
    mbar_init(&bar[B_DRAIN], 1);
    mbar_init(&bar[B_LDRAIN], 1);
    mbar_init(&bar[B_Y1DRAIN], 1);
    for (int i = 0; i < CT_BARS; ++i) {
      mbar_init(&bar[B_Y2DONE + i], 1);
      mbar_init(&bar[B_Y2FREE + i], EPI_WARPS / 2);
    }
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (ntiles > 0 && warp == 0 && lane == 0) {
    // ------------------------------------------------------------------ producer
    for (int t = issued; t < ntiles && !abort_flag; ++t)
      if (!issue(t)) break;
    // wait (bounded) for this thread's copies still in flight before the CTA may exit: the
    // last NSTAGE stage loads and the last two W / U~ image loads (after an abort some of them
    // may never have been consumed)
    for (int t = (issued > NSTAGE ? issued - NSTAGE : 0); t < issued; ++t)
      mbar_wait(&bar[B_FULL + (t % NSTAGE)], (t / NSTAGE) & 1, 100000000ull);
    for (int i = (w_issued > 2 ? w_issued - 2 : 0); i < w_issued; ++i)
      mbar_wait(&bar[B_WFULL + (i & 1)], (i >> 1) & 1, 100000000ull);
  } else if (ntiles > 0 && warp == 1 && lane == 0) {
    // ------------------------------------------------------------------ L MMAs
    const uint32_t base = smem_u32(sm);
    const uint32_t idL = instr_desc(128, 64, 2, 2, false, false);
    const uint64_t dw0 = smem_desc(base + OFF_W, 16, C::TF_SBO, C::TF_SWZ);
    const uint64_t dv0 = smem_desc(base + OFF_STAGE + D_BYTES, 16, C::TF_SBO, C::TF_SWZ);
    int rtl = 0, ctl = 0;
    for (int t = 0; t < ntiles && !abort_flag; ++t, ctl = (ctl + 1 == nct) ? 0 : ctl + 1, rtl += (ctl == 0) ? 1 : 0) {
      const int s = t % NSTAGE, lb = t & 1, wb = rtl & 1;
      bool ok = true;
      if (ctl == 0) ok = ok && mbar_wait(&bar[B_WFULL + wb], (rtl >> 1) & 1);
      ok = ok && mbar_wait(&bar[B_FULL + s], (t / NSTAGE) & 1);
      if (t >= 2) ok = ok && mbar_wait(&bar[B_LEMPTY + lb], ((t - 2) >> 1) & 1);
      if (!ok) {
        fail(a, &abort_flag);
        break;
      }
      tc_fence_after();
      const uint64_t dw = dw0 + (uint64_t)(wb * (WOP_BYTES >> 4));
      const uint64_t dv = dv0 + (uint64_t)(s * (STAGE_BYTES >> 4));
      // k-steps of 8 tf32 (32 bytes = 2 descriptor units); each row is [hi | lo], the lo half
      // starting RK tf32 = RK / 4 units in
      constexpr int LO = RK / 4;
#pragma unroll
      for (int kb = 0; kb < RK / 8; ++kb) {
        mma_tf32(tmem + lb * BN, dw + 2 * kb, dv + 2 * kb, idL, kb > 0);            // W_hi V_hi
        mma_tf32(tmem + lb * BN, dw + 2 * kb, dv + LO + 2 * kb, idL, true);         // W_hi V_lo
        mma_tf32(tmem + lb * BN, dw + LO + 2 * kb, dv + 2 * kb, idL, true);         // W_lo V_hi
      }
      mma_commit(&bar[B_LFULL + lb]);
      if (ctl == nct - 1) mma_commit(&bar[B_WEMPTY + wb]);
    }
    mma_commit(&bar[B_LDRAIN]);
    mbar_wait(&bar[B_LDRAIN], 0, 100000000ull);
  } else if (ntiles > 0 && warp == 2 && lane == 0) {
    // ------------------------------------------------------------------ Y1 MMAs
    const uint32_t base = smem_u32(sm);
    const uint32_t idY1 = instr_desc(128, NY, 1, 1, false, false);
    const uint64_t dz0 = smem_desc(base + OFF_STAGE, 16, 1024);
    const uint64_t dvt0 = smem_desc(base + OFF_STAGE + D_BYTES + VOP_BYTES, 16, 1024);
    int rtl = 0, ctl = 0;
    for (int tp = 0; tp < ntiles && !abort_flag; ++tp, ctl = (ctl + 1 == nct) ? 0 : ctl + 1, rtl += (ctl == 0) ? 1 : 0) {
      const int s = tp % NSTAGE, yb = rtl & 1;
      bool ok = mbar_wait(&bar[B_ZFULL + s], (tp / NSTAGE) & 1);
      if (ok && ctl == 0 && rtl >= 2) ok = mbar_wait(&bar[B_Y1EMPTY + yb], ((rtl - 2) >> 1) & 1);
      if (!ok) {
        fail(a, &abort_flag);
        break;
      }
      tc_fence_after();
      const uint64_t so = (uint64_t)(s * (STAGE_BYTES >> 4));
      const uint64_t dz = dz0 + so, dvt = dvt0 + so;
      const uint32_t y1 = tmem + TM_Y1 + yb * NY;
      // k-step k: columns 16k .. 16k+15 of Z_hi and of Z_lo (32 bytes each)
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_f16(y1, dz + zhi_off<DM>(k), dvt + 2 * k, idY1, !(ctl == 0 && k == 0));
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_f16(y1, dz + zlo_off<DM>(k), dvt + 2 * k, idY1, true);
      mma_commit(&bar[B_EMPTY + s]);
      if (ctl == nct - 1) mma_commit(&bar[B_Y1FULL + yb]);
    }
    mma_commit(&bar[B_Y1DRAIN]);
    mbar_wait(&bar[B_Y1DRAIN], 0, 100000000ull);
  } else if (ntiles > 0 && warp == 3 && lane == 0) {
    // ------------------------------------------------------------------ Y2 MMAs
    const uint32_t base = smem_u32(sm);
    const uint32_t idY2 = instr_desc(128, NY, 1, 1, true, false);
    const uint64_t dzm0 = smem_desc(base + OFF_STAGE, Z_BYTES / 2, 1024);
    const uint64_t dut0 = smem_desc(base + OFF_U, 16, 1024);
    int rtl = 0, ctl = 0;
    for (int tp = 0; tp < ntiles && !abort_flag; ++tp, ctl = (ctl + 1 == nct) ? 0 : ctl + 1, rtl += (ctl == 0) ? 1 : 0) {
      const int s = tp % NSTAGE;
      // a Y2 accumulator restarts every G2 row tiles (the tensor-core accumulation of a long
      // chain of products drifts); the epilogue has read the previous chunk out first
      const bool restart = rtl % G2 == 0;
      const int wb = rtl & 1;
      bool ok = mbar_wait(&bar[B_ZFULL + s], (tp / NSTAGE) & 1);
      if (ok && ctl == 0) ok = mbar_wait(&bar[B_WFULL + wb], (rtl >> 1) & 1);  // U~ image of the block
      if (ok && restart && rtl > 0) ok = mbar_wait(&bar[B_Y2FREE + ctl], ((rtl / G2) - 1) & 1);
      if (!ok) {
        fail(a, &abort_flag);
        break;
      }
      tc_fence_after();
      const uint64_t so = (uint64_t)(s * (STAGE_BYTES >> 4));
      const uint64_t dzm = dzm0 + so, dut = dut0 + (uint64_t)(wb * (UTOP_BYTES >> 4));
      const uint32_t y2 = tmem + TM_Y2 + ctl * NY;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        mma_f16(y2, dzm + 128 * k, dut + (k >= 4 ? ((UTOP_BYTES / 2) >> 4) : 0) + 2 * (k & 3), idY2,
                !(restart && k == 0));
      mma_commit(&bar[B_EMPTY + s]);
      if (rtl % G2 == G2 - 1 && rtl != nrt - 1) mma_commit(&bar[B_Y2DONE + ctl]);
      if (ctl == nct - 1) mma_commit(&bar[B_WEMPTY + wb]);
    }
    mma_commit(&bar[B_YFIN]);
    mma_commit(&bar[B_DRAIN]);
    mbar_wait(&bar[B_DRAIN], 0, 100000000ull);  // all issued MMAs complete before TMEM is freed
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ epilogue
    // Two groups of 8 warps take alternate tiles (group grp: tiles grp, grp + 2, ...), so one
    // group loads while the other computes.  Warp (q, h) of a group: rows 32q .. 32q+31 (its
    // TMEM lane quarter), columns 32h .. 32h+31.
    const int e = warp - 4, grp = e >> 3, gq = e >> 2;
    const int q = warp & 3, h = (e >> 2) & 1;
    const int rowl = 32 * q + lane;
    const bool tcta = cta == a.tcta && a.tfac != nullptr;
    // this pass writes the support words of S_k when the update before it predicted that it is
    // the last one (FP32 D only)
    const bool emit = DM == 0 && !MASK && a.swords != nullptr && a.st->emit != 0;
    if (emit && cta == 0 && tid == 128) *a.emit_k = a.st->k;
    {
      // zero this CTA's columns of the group's two Y2 slices before the first add (the adds
      // come at least kTcY2Chunk row tiles later, after the barrier below)
      const int et = tid - 128, ncol = nct * BN;
      for (int e2 = et; e2 < 2 * ncol * (RK / 4); e2 += EPI_THREADS) {
        const int part = e2 / (ncol * (RK / 4)), rem = e2 % (ncol * (RK / 4));
        const int col = ct0 * BN + rem / (RK / 4);
        if (col < a.n)
          reinterpret_cast<float4*>(a.P2 + ((size_t)(p2base + part) * a.n + col) * RK)[rem % (RK / 4)] =
              make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (tcta) {
        // T factors for the update that follows, in the CTA with the fewest tiles while the
        // first tile is on its way: T_u and T_v (U~ = A~ T_u, V~ = B~ T_v, the orthonormal
        // bases of Section 2.1 by CholeskyQR) of the trimmed factors A~, B~ this pass reads,
        // from the Gram partials that the kernel which trimmed them left (per block of that
        // kernel).  Sums: warp e takes entries e, e + 16, ... of the two Gram matrices, each
        // lane the blocks lane, lane + 32, ... in order, then a fixed shuffle tree.
        const int w = a.tw, nb = a.tnb, ne = 2 * w * w;
        for (int q0 = e; q0 < ne; q0 += EPI_WARPS) {
          const int sd = q0 / (w * w), pe = q0 % (w * w);
          const float* src = a.tgram + (size_t)(6 + sd) * nb * 256 + pe;
          float v = 0.f;
          for (int b = lane; b < nb; b += 32) v += src[(size_t)b * 256];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) a.tfac[512 + q0] = v;  // the reduced Gram matrices, scratch
        }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_THREADS) : "memory");
      if (tcta && e < 2) {
        const int w = a.tw;
        float g[RK];
#pragma unroll
        for (int k = 0; k < RK; ++k) g[k] = (lane < w && k < w) ? a.tfac[512 + e * w * w + k * w + lane] : 0.f;
        fac::chol_cols<float, RK>(g, w, nullptr, a.tfac + e * 256);
      }
    }
    const float zeta = static_cast<float>(a.st->zeta);
    const float invp = PO ? static_cast<float>(a.st->inv_p) : 1.f;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    // residual: each tile's 32 squared terms of this thread are summed in a chain of their
    // own and only the tile sums (~40 per pass) are added up, so no FP32 chain is longer than
    // ~40 terms (one chain over the thousands of terms a thread sees per pass biased err_k by
    // up to ~1e-4 relative); the totals over threads are taken in FP64
    float res = 0.f;
    unsigned nnz = 0;
    // support bitmask of this pass (k even: buffer 0, odd: buffer 1; mask_wr words each, at
    // least TR TC 256); the entries that changed since the previous pass are counted from the
    // two buffers by a separate kernel (count_mask_changes)
    unsigned* mask_new = MASK ? a.masks + ((a.st->k & 1) ? a.mask_wr : 0) : nullptr;
    // the tile loop in two copies, without and with the support words, so that the plain
    // passes keep their registers
    auto tile_loop = [&](auto emit_c) {
      constexpr bool EMIT = decltype(emit_c)::value;
      for (int t = grp; t < ntiles && !abort_flag; t += 2) {
        const int rtl = t / nct, ctl = t % nct, s = t % NSTAGE, lb = t & 1, yb = rtl & 1;
        if (rtl % G2 == 0 && rtl > 0) {
          // chunk c - 1 of column tile ctl's Y2 accumulator is complete: read it out (hi + lo
          // column halves, this warp's half of the components) before this tile's products
          // restart the accumulator, and add it into the group's Y2 partial (slice p2base for the
          // Z_hi rows, p2base + 1 for the Z_lo rows; each (slice, column) belongs to this CTA
          // alone, zeroed before the first tile) with fire-and-forget vector atomic adds, so no
          // warp waits for the partial's previous value.  Consecutive chunks of a column tile are read
          // out at least kTcY2Chunk row tiles apart.
          const int c = rtl / G2;
          if (!mbar_wait(&bar[B_Y2DONE + ctl], (c - 1) & 1)) {
            fail(a, &abort_flag);
            break;
          }
          tc_fence_after();
          uint32_t yv[NY];
          tmem_ld_y<NY>(tmem + lane_base + TM_Y2 + ctl * NY, yv);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar[B_Y2FREE + ctl]);
          const int col = (ct0 + ctl) * BN + y2_row_col<DM>(rowl);
          if (col < a.n) {
            // components k = h RK/2 + j (register indices fixed at compile time), 4 per vector add
            float4* dst = reinterpret_cast<float4*>(a.P2 + ((size_t)(p2base + y2_row_part<DM>(rowl)) * a.n + col) * RK +
                                                    h * (RK / 2));
  #pragma unroll
            for (int j = 0; j < RK / 2; j += 4) {
              float v[4];
  #pragma unroll
              for (int u = 0; u < 4; ++u) {
                const uint32_t x = h ? yv[RK / 2 + j + u] : yv[j + u], y = h ? yv[RK + RK / 2 + j + u] : yv[RK + j + u];
                v[u] = __uint_as_float(x) + __uint_as_float(y);
              }
              atomicAdd(dst + j / 4, make_float4(v[0], v[1], v[2], v[3]));
            }
          }
        }
        if (!mbar_wait(&bar[B_LFULL + lb], (t >> 1) & 1) || !mbar_wait(&bar[B_FULL + s], (t / NSTAGE) & 1)) {
          fail(a, &abort_flag);
          break;
        }
        tc_fence_after();
        uint32_t lv[32];
        tmem_ld32(tmem + lane_base + lb * BN + 32 * h, lv);
        uint8_t* stg = sm + OFF_STAGE + s * STAGE_BYTES;
        float z[32];
        if (DM == 0) {
          const uint8_t* drow = stg + h * (D_BYTES / 2) + rowl * 128;
  #pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 d4 = *reinterpret_cast<const float4*>(drow + ((c ^ (rowl & 7)) << 4));
            z[4 * c + 0] = d4.x;
            z[4 * c + 1] = d4.y;
            z[4 * c + 2] = d4.z;
            z[4 * c + 3] = d4.w;
          }
        } else {
          // columns 32h .. 32h+31 of the bf16 row = 16-byte chunks 4h .. 4h+3 (8 values each)
          const uint8_t* hrow = stg + rowl * 128;
  #pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int off = (((4 * h + c) ^ (rowl & 7)) & 7) << 4;
            const uint4 hv = *reinterpret_cast<const uint4*>(hrow + off);
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
  #pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
              z[8 * c + 2 * e2] = __uint_as_float(hw[e2] << 16);
              z[8 * c + 2 * e2 + 1] = __uint_as_float(hw[e2] & 0xffff0000u);
            }
            if (use_lo) {
              const uint4 lv4 = *reinterpret_cast<const uint4*>(hrow + D_BYTES / 2 + off);
              const uint32_t lw[4] = {lv4.x, lv4.y, lv4.z, lv4.w};
  #pragma unroll
              for (int e2 = 0; e2 < 4; ++e2) {
                z[8 * c + 2 * e2] += __uint_as_float(lw[e2] << 16);
                z[8 * c + 2 * e2 + 1] += __uint_as_float(lw[e2] & 0xffff0000u);
              }
            }
          }
        }
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[B_LEMPTY + lb]);
        const float2 m1 = make_float2(-1.f, -1.f);
        float rq = 0.f;
        uint32_t bits = 0;
  #pragma unroll
        for (int c = 0; c < 32; c += 2) {
          const float2 l2 = make_float2(__uint_as_float(lv[c]), __uint_as_float(lv[c + 1]));
          const float2 r2 = __ffma2_rn(l2, m1, make_float2(z[c], z[c + 1]));  // D - L, exactly rounded
          const bool s0 = fabsf(r2.x) > zeta, s1 = fabsf(r2.y) > zeta;  // false for NaN
          if (PO) {
            const bool k0 = s0 || !(z[c] == z[c]), k1 = s1 || !(z[c + 1] == z[c + 1]);  // Z = L
            rq = k0 ? rq : fmaf(r2.x, r2.x, rq);
            rq = k1 ? rq : fmaf(r2.y, r2.y, rq);
            z[c] = k0 ? l2.x : fmaf(r2.x, invp, l2.x);
            z[c + 1] = k1 ? l2.y : fmaf(r2.y, invp, l2.y);
          } else {
            rq = s0 ? rq : fmaf(r2.x, r2.x, rq);
            rq = s1 ? rq : fmaf(r2.y, r2.y, rq);
            z[c] = s0 ? l2.x : z[c];
            z[c + 1] = s1 ? l2.y : z[c + 1];
          }
          if (MASK || EMIT)
            bits |= ((s0 ? 1u : 0u) << c) | ((s1 ? 1u : 0u) << (c + 1));
          else
            nnz += (s0 ? 1u : 0u) + (s1 ? 1u : 0u);
        }
        if (MASK || EMIT) nnz += __popc(bits);
        res += rq;
        const int erow = (rt0 + rtl) * BM + rowl;
        // the word's support bits, [word][row] layout: the lanes of a warp (consecutive rows)
        // write consecutive words
        if (EMIT && erow < a.m) a.swords[(size_t)(2 * (ct0 + ctl) + h) * a.m + erow] = bits;
        // Z -> bf16 hi/lo of row rowl, columns 32h .. 32h+31: FP32 D, logical 16-byte chunks
        // 0..3 (hi) and 4..7 (lo) of box h; bf16 D, chunks 4h .. 4h+3 of the hi and lo tiles
        uint8_t* zhi = DM == 0 ? stg + h * (D_BYTES / 2) : stg;
        uint8_t* zlo = DM == 0 ? zhi : stg + Z_BYTES / 2;
  #pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t hw[4], lw[4];
  #pragma unroll
          for (int e2 = 0; e2 < 4; ++e2) {
            const float2 zz = make_float2(z[8 * c + 2 * e2], z[8 * c + 2 * e2 + 1]);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(zz.x, zz.y);
            const float2 hf = __bfloat1622float2(hi);
            const float2 lf = __ffma2_rn(hf, make_float2(-1.f, -1.f), zz);  // z - hi, exact
            const __nv_bfloat162 lo = __floats2bfloat162_rn(lf.x, lf.y);
            hw[e2] = *reinterpret_cast<const uint32_t*>(&hi);
            lw[e2] = *reinterpret_cast<const uint32_t*>(&lo);
          }
          const int chi = DM == 0 ? c : 4 * h + c, clo = DM == 0 ? 4 + c : 4 * h + c;
          *reinterpret_cast<uint4*>(zhi + rowl * 128 + (((chi ^ (rowl & 7)) & 7) << 4)) =
              make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(zlo + rowl * 128 + (((clo ^ (rowl & 7)) & 7) << 4)) =
              make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[B_ZFULL + s]);
        if (MASK)  // tile-major; rows past m hold no support (their D reads as zero, L too)
          mask_new[(((long long)(rt0 + rtl) * a.TC + (ct0 + ctl)) * 2 + h) * BM + rowl] = bits;

        if (ctl == nct - 1 && h == 0) {
          // drain Y1 of this row tile
          if (!mbar_wait(&bar[B_Y1FULL + yb], (rtl >> 1) & 1)) {
            fail(a, &abort_flag);
            break;
          }
          tc_fence_after();
          uint32_t yv[NY];
          tmem_ld_y<NY>(tmem + lane_base + TM_Y1 + yb * NY, yv);
          tmem_wait_ld();
          const int row = (rt0 + rtl) * BM + rowl;
          if (row < a.m) {
  #pragma unroll
            for (int k = 0; k < RK; ++k)
              if (k < a.R)
                a.P1[((size_t)bi * a.m + row) * a.R + k] = __uint_as_float(yv[k]) + __uint_as_float(yv[RK + k]);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar[B_Y1EMPTY + yb]);
        }
      }
    };
    if (DM == 0 && !MASK && emit)
      tile_loop(BoolC<DM == 0 && !MASK>{});
    else
      tile_loop(BoolC<false>{});
    // drain Y2: the last chunk of every column tile is still in tensor memory; each warp takes
    // the column tiles ctl = g, g + 4, ...  (lane quarter q: accumulator rows 32q .. 32q+31) and
    // adds them into the group's Y2 partial as the read-outs above do
    if (ntiles > 0 && !abort_flag) {
      if (!mbar_wait(&bar[B_YFIN], 0)) {
        fail(a, &abort_flag);
      } else {
        tc_fence_after();
        const int col0 = y2_row_col<DM>(rowl);
        const int slice = p2base + y2_row_part<DM>(rowl);
        for (int ctl = gq; ctl < nct; ctl += EPI_WARPS / 4) {
          uint32_t yv[NY];
          tmem_ld_y<NY>(tmem + lane_base + TM_Y2 + ctl * NY, yv);
          tmem_wait_ld();
          const int col = (ct0 + ctl) * BN + col0;
          if (col < a.n) {
            float4* dst = reinterpret_cast<float4*>(a.P2 + ((size_t)slice * a.n + col) * RK);
#pragma unroll
            for (int k = 0; k < RK; k += 4)
              atomicAdd(dst + k / 4, make_float4(__uint_as_float(yv[k]) + __uint_as_float(yv[RK + k]),
                                                 __uint_as_float(yv[k + 1]) + __uint_as_float(yv[RK + k + 1]),
                                                 __uint_as_float(yv[k + 2]) + __uint_as_float(yv[RK + k + 2]),
                                                 __uint_as_float(yv[k + 3]) + __uint_as_float(yv[RK + k + 3])));
          }
        }
      }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(EPI_THREADS));
    // CTA totals of the residual and the support size
    double rd = (double)res;
    unsigned long long nz = nnz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rd += __shfl_xor_sync(0xffffffffu, rd, o);
      nz += __shfl_xor_sync(0xffffffffu, nz, o);
    }
    if (lane == 0) {
      red_res[warp - 4] = rd;
      red_nnz[warp - 4] = nz;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(EPI_THREADS));
    if (tid == 128) {
      double tr = 0.0;
      unsigned long long tz = 0;
      for (int w = 0; w < EPI_WARPS; ++w) {
        tr += red_res[w];
        tz += red_nnz[w];
      }
      a.resP[cta] = tr;
      a.nnzP[cta] = tz;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

static_assert(Cfg<8>::MAX_CT >= 20 && Cfg<16>::MAX_CT >= 10, "column tiles per CTA (tc_max_col_tiles)");

template <int DM, int RK, int MODE>
cudaError_t set_tc_smem() {
  return cudaFuncSetAttribute(fused_pass_tc<DM, RK, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Cfg<RK>::SMEM_BYTES);
}

template <int DM, int RK>
cudaError_t set_tc_smem_modes() {
  cudaError_t e = set_tc_smem<DM, RK, MODE_PLAIN>();
  if (e == cudaSuccess) e = set_tc_smem<DM, RK, MODE_MASK>();
  if (e == cudaSuccess) e = set_tc_smem<DM, RK, MODE_PARTIAL>();
  return e;
}

template <int DM, int RK>
cudaError_t launch_tc(const CUtensorMap& dmap, const CUtensorMap& lo, const TcArgs& a, int partial, cudaStream_t s) {
  if (a.masks)
    fused_pass_tc<DM, RK, MODE_MASK><<<a.ncta, THREADS, Cfg<RK>::SMEM_BYTES, s>>>(dmap, lo, a);
  else if (partial)
    fused_pass_tc<DM, RK, MODE_PARTIAL><<<a.ncta, THREADS, Cfg<RK>::SMEM_BYTES, s>>>(dmap, lo, a);
  else
    fused_pass_tc<DM, RK, MODE_PLAIN><<<a.ncta, THREADS, Cfg<RK>::SMEM_BYTES, s>>>(dmap, lo, a);
  return cudaGetLastError();
}

}  // namespace

bool tc_pass_supported(int R) { return R >= 1 && R <= 16; }

size_t tc_pass_smem() { return Cfg<8>::SMEM_BYTES; }

cudaError_t launch_fused_pass_tc(const CUtensorMap* dmap, const CUtensorMap* dmap_lo, int dm, const TcPassArgs& p,
                                 cudaStream_t s) {
  static unsigned long long attr_epoch = 0;
  if (attr_epoch != g_attr_epoch) {
    cudaError_t e = set_tc_smem_modes<0, 8>();
    if (e == cudaSuccess) e = set_tc_smem_modes<1, 8>();
    if (e == cudaSuccess) e = set_tc_smem_modes<0, 16>();
    if (e == cudaSuccess) e = set_tc_smem_modes<1, 16>();
    if (e != cudaSuccess) return e;
    attr_epoch = g_attr_epoch;
  }
  if (p.R < 1 || p.R > 16) return cudaErrorInvalidValue;
  TcArgs a;
  a.m = p.m;
  a.n = p.n;
  a.R = p.R;
  a.ncta = p.ncta;
  a.rect = p.rect;
  a.ids = p.ids;
  a.TR = p.TR;
  a.TC = p.TC;
  a.wop = p.wop;
  a.vop = p.vop;
  a.vtop = p.vtop;
  a.utop = p.utop;
  a.st = p.st;
  a.status = p.status;
  a.P1 = p.P1;
  a.P2 = p.P2;
  a.resP = p.resP;
  a.nnzP = p.nnzP;
  a.masks = p.masks;
  a.mask_wr = p.mask_wr;
  a.swords = p.swords;
  a.nw = p.nw;
  a.emit_k = p.emit_k;
  a.tgram = p.tgram;
  a.tnb = p.tnb;
  a.tw = p.tw;
  a.tcta = p.tcta;
  a.tfac = p.tfac;
  a.chgP = p.chgP;
  if (a.masks && (!a.chgP || a.mask_wr < 256ll * a.TR * a.TC || p.partial)) return cudaErrorInvalidValue;
  const CUtensorMap& lo = dm ? *dmap_lo : *dmap;
  const int po = p.partial;
  if (p.R <= 8) return dm == 0 ? launch_tc<0, 8>(*dmap, lo, a, po, s) : launch_tc<1, 8>(*dmap, lo, a, po, s);
  return dm == 0 ? launch_tc<0, 16>(*dmap, lo, a, po, s) : launch_tc<1, 16>(*dmap, lo, a, po, s);
}

}  // namespace rpca
