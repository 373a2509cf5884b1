// Internal declarations shared by the CUDA translation units of the AccAltProj library.
// Nothing here is part of the C ABI (include/rpca.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace rpca {

// Ranks with a compiled fused pass.  A rank r is run with the smallest entry >= r and
// zero-padded factors.
#define RPCA_FOR_EACH_R(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(14) X(16)
constexpr int kMaxR = 16;
inline int padded_rank(int r) {
  const int table[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 10, 12, 12, 14, 14, 16, 16};
  return (r >= 1 && r <= kMaxR) ? table[r - 1] : -1;
}

// Device-side state of one solve.  Lives in device memory; only `done`, `k` and `status`
// are read back by the host while iterating.
struct DevState {
  double zeta;           // threshold used by the next fused pass
  double normD2;         // ||D||_F^2
  double beta, gamma, tol, beta_init, mu_trim;
  double sigma[64];      // spectrum of the last small SVD (2r for M_k, b for init)
  double sigma_prev[64]; // previous spectrum (init convergence test)
  int k;                 // iteration index of the factors currently held
  int done;              // 1: converged or capped; passes and updates return at once
  int status;            // 0 or an rpca_status code raised on the device
  int conv;              // initialisation finished (both subspace iterations converged)
  int use_lo;            // bf16 split storage of D: the passes also read the lo part
  int emit;              // the next tensor-core pass writes its support words (predicted last)
  int emit_k;            // k of the last pass that wrote them (-1: none)
  int steps_run;         // initialisation steps that did work (profiling of the passes)
  double split_switch;   // bf16 split storage: set use_lo once err_k falls below this
  double inv_p;          // partial observation: m n / |observed entries| (1 otherwise)
  int max_iter;
  int zeta_mode;
  int trim;
  int init_phase;        // initialisation: 0 = sigma_1(D), 1 = top-r SVD of D - S_{-1}
  int init_step;         // Rayleigh-Ritz steps taken in the current phase
  unsigned bar_count;    // grid barrier
  unsigned bar_gen;
};

// One record per fused pass of Algorithm 1.
struct DevStats {
  double err, zeta, sigma1, sigma_r1, res2;
  long long nnz;
  int k, pad;
  // learned threshold schedule (zeta mode LEARNED; zero otherwise): zeta^plain_{k+1} of
  // Algorithm 1, the clamped network output g(s_k), the statistics s_k (mlp.cuh) and the
  // number of entries whose support membership changed since pass k - 1
  double zeta_next_plain, g;
  float feat[6];
  long long changes;
};

// Precision of the fused pass (what D is read as and what the m x n arithmetic uses).
enum PassPrec { PREC_F64 = 0, PREC_F32 = 1 };

// Geometry of one fused-pass work unit (a BH x BW block of D handled by one CTA).
struct PassGeom {
  int BH, BW;   // unit rows, unit columns
  int TM;       // rows per warp per row block
  int VW;       // columns per lane (one 16-byte vector of D)
  size_t smem;  // dynamic shared memory bytes
};
PassGeom pass_geometry(int prec, int R);

struct PassArgs {
  const void* D;
  long long ld;
  int m, n;
  const void* W;    // m x R, W = U_k Sigma_k (pass precision), row stride R
  const void* V;    // n x R, V_k
  const void* Ut;   // m x R, trimmed orthonormal U~_k
  const void* Vt;   // n x R, trimmed orthonormal V~_k
  const DevState* st;
  void* P1;         // [ceil(n/BW)][m][R] partial Z V~
  void* P2;         // [ceil(m/BH)][n][R] partial Z^T U~
  double* resP;     // per CTA: sum of R_ij^2 over the unthresholded entries
  unsigned long long* nnzP;  // per CTA: |supp(S)|
  int vec;          // 16-byte vector loads of D allowed
  // dm = 1: D holds bf16(D) (the hi part) and Dlo the lo part (null if none), both with rows
  // of ld elements, ld a multiple of 8; the pass reads D = hi (+ lo once DevState.use_lo).
  int dm;
  const void* Dlo;
  // support bitmasks (null unless the learned schedule needs the support change): two
  // buffers of m x mask_wr words (SIMT pass, row-major); pass k writes buffer k % 2 and
  // compares with the other
  unsigned* masks;
  long long mask_wr, mask_words;  // words per row, words per buffer
  unsigned long long* chgP;  // per CTA: entries whose support membership changed
  // partial observation: NaN entries of D are unobserved; the pass then takes
  // Z = L + (D - L - S) / p on observed entries and Z = L elsewhere (DevState.inv_p = 1 / p)
  int partial;
};

// Kernel attributes (the dynamic shared-memory limits) belong to a CUDA context: each launcher
// sets them again when this epoch changed, which rpca_create advances whenever it finds a new
// context (after a device reset, for example).
extern unsigned long long g_attr_epoch;

// Launches the fused pass for compiled rank R (must be an RPCA_FOR_EACH_R entry).
cudaError_t launch_fused_pass(int prec, int R, const PassArgs& a, cudaStream_t s);

// Tensor-core fused pass (FP32 or bf16-stored D, compiled rank R <= 16); see pass_tc.cu.
struct TcPassArgs {
  int m, n, R;
  int ncta;      // CTAs of the tile partition (TcPlan, below)
  const int4* rect;  // [ncta] tile rectangle of each CTA (device)
  const int4* ids;   // [ncta] {row group, index within the group, first Y2 slice of the group,
                     //  unused} (device)
  int TR, TC;    // 128-row and 64-column tile counts
  // operand images (tc_images.cuh) in the layout of tc_image_rank(R): per row tile W and
  // U~, per column tile V and V~
  const uint8_t* wop;
  const uint8_t* vop;
  const uint8_t* vtop;
  const uint8_t* utop;
  const DevState* st;
  int* status;
  float* P1;     // [Bmax][m][R]: slice = index of the CTA within its row group
  float* P2;     // [S2 = 2 A][n][RK]: per row group, the Z_hi and the Z_lo part of Z^T U~ over
                 // the group's rows (slices 2 a and 2 a + 1), rows padded to the image rank RK
                 // (tc_image_rank(R); the padding columns hold zeros)
  double* resP;  // [ncta]
  unsigned long long* nnzP;
  // support bitmasks as in PassArgs (null: not tracked), here two buffers of mask_wr words
  // each (>= TR TC 256, tile-major, see pass_tc.cu)
  unsigned* masks;
  long long mask_wr;
  unsigned long long* chgP;
  int partial;  // as in PassArgs (not together with masks)
  // support words of S_k (FP32 D only; null: never): when DevState.emit is set the pass
  // writes, per row and 32 columns, the bit mask of |D_ij - L_ij| > zeta_k ([word][row]
  // layout: word j (columns 32 j .. 32 j + 31) of row i at j m + i; nw = 2 TC words per row)
  // and *emit_k = k
  unsigned* swords;
  int nw;
  int* emit_k;
  // T factors for the update that follows (null: not computed), by CTA tcta: the Gram
  // partials of the trimmed factors (the small kernel's slots 6, 7: [slot][tnb blocks][256]
  // FP32, tw x tw) and the output [1024]: T_u, T_v (row-major, leading dimension tw) at 0 and
  // 256, the reduced Gram matrices (scratch) from 512
  const float* tgram;
  int tnb, tw, tcta;
  float* tfac;
};
// row tiles per Y2 accumulation chunk of the tensor-core pass
constexpr int kTcY2Chunk = 4;
// Tile partition of the tensor-core pass (api.cu, tc_plan): per CTA its rectangle of tiles
// {first row tile, end row tile, first column tile, end column tile} and its ids {row group a,
// index in the group (the m-slice of Y1 it writes), 2 a (its group's first n-slice of Y2),
// 0}; per row tile the number of Y1 slices its rows have.  S2 = 2 A Y2 slices in all.
struct TcPlan {
  int ncta = 0, A = 0, Bmax = 0, ct_max = 0, S2 = 0, T = 0;
  std::vector<int4> rect;
  std::vector<int4> ids;
  std::vector<int> p1_nsl;
  int min_cta = 0;  // a CTA with the fewest tiles
};
bool tc_pass_supported(int R);
// image layout (8 or 16) of the tensor-core pass for compiled rank R, and the most column
// tiles one CTA of that pass may own (its Y2 accumulators stay in tensor memory)
inline int tc_image_rank(int R) { return R <= 8 ? 8 : 16; }
inline int tc_max_col_tiles(int R) { return R <= 8 ? 20 : 10; }
size_t tc_pass_smem();
// dm = 0: FP32 D through dmap; dm = 1: bf16 hi (dmap) and lo (dmap_lo) parts of D.
cudaError_t launch_fused_pass_tc(const CUtensorMap* dmap, const CUtensorMap* dmap_lo, int dm, const TcPassArgs& p,
                                 cudaStream_t s);
// Sparse extraction (three kernels): per-row counts, exclusive scan, ordered write.
struct ExtractArgs {
  const void* D;
  long long ld;
  int m, n;
  const void* W;
  const void* V;
  const DevState* st;
  unsigned long long* rowcnt;  // m counts, then m+1 offsets (in place scan into rowoff)
  unsigned long long* rowoff;  // m+1
  long long* idx;
  double* val;
  int vec;
};
cudaError_t launch_extract_count(int prec, int R, const ExtractArgs& a, cudaStream_t s);
cudaError_t launch_extract_write(int prec, int R, const ExtractArgs& a, cudaStream_t s);

// The tall-skinny kernel (cooperative launch): reductions of the pass partials,
// CholeskyQR, the small SVD, the factor update, Trim and the pass-precision copies.
// Gram partials: kSmallSlots slots of 16 x 16 doubles per block.
constexpr int kSmallSlots = 8;
enum SmallMode { SM_UPDATE = 0, SM_PREPARE = 1, SM_RR = 2, SM_RAND = 3, SM_BASES = 4 };

struct SmallArgs {
  int mode;
  int m, n;
  int r;        // rank of the iteration (columns of U, V)
  int R;        // width of the pass arrays (compiled rank of the pass that ran)
  int b;        // width of the subspace-iteration bases in init (RR / RAND modes)
  int prec;
  int n_p1, n_p2, n_cta;  // partial slices and CTA count of the pass that ran
  const int* p1_nsl;      // tensor-core pass: Y1 slices of each 128-row tile (null: n_p1 everywhere)
  int emit_ok;            // SM_UPDATE: the iteration's pass can write the support words
  int R2;                 // row width of the Y2 partial slices (R; the image rank after a
                          // tensor-core pass)
  const float* tfac;      // SM_UPDATE after a tensor-core pass: T_u, T_v computed by that pass
                          // (TcPassArgs::tfac); null: the update computes them
  const void* P1;
  const void* P2;
  const double* resP;
  const unsigned long long* nnzP;
  const unsigned long long* chgP;  // per-CTA support changes (null: not tracked)
  const float* theta;              // learned schedule: network parameters (mlp.cuh)
  int depth;                       // learned schedule: unrolled depth K of the statistic (k+1)/K
  // Arrays below hold the kernel's working precision (double in FP64 mode, float in
  // FP32 mode).
  void* U; void* sig; void* V;         // factors of L_k (m x r, r, n x r)
  void* Ut; void* Vt;                  // bases (m x w, n x w), w = r or b
  void* Y1; void* Y2;                  // m x w, n x w
  void* part;                          // [kSmallSlots][grid][16*16] Gram partials (double)
  void* Wc; void* Vc; void* Utc; void* Vtc;  // pass-precision copies, width Rc
  int Rc;                              // width of the copies written for an init pass
  int Rit;                             // width of the copies written for an iteration pass
  DevState* st;
  DevStats* stats;
  double init_tol;
  unsigned long long seed;
  int init_max;       // RR: steps per phase at most (the last one is accepted as converged)
  // Operand images of the tensor-core pass (tc_images.cuh), written with the copies when the
  // pass that reads them is the tensor-core one: img_init for the width-Rc copies of the
  // initialisation (image set 0), img_iter for the width-Rit copies of the iteration (set 1);
  // img_rk[set] is the image layout (8 or 16) of that pass.
  uint8_t* wop[2];
  uint8_t* vop[2];
  uint8_t* vtop[2];
  uint8_t* utop[2];
  int img_rk[2];
  int img_init;
  int img_iter;
  // SM_BASES: outputs U~ (m x Rit), V~ (n x Rit) in the working precision
  void* out_ut;
  void* out_vt;
};
cudaError_t launch_small(const SmallArgs& a, int grid, cudaStream_t s);
// Runs the bounded-wait self-test kernels (small.cu) on the current device and returns the
// status each recorded (RPCA_ERR_TIMEOUT expected).
cudaError_t run_wait_selftest(int* mbar_status, int* grid_status);
int small_grid_size(int device);

cudaError_t launch_scan_rows(const unsigned long long* cnt, unsigned long long* off, int m, cudaStream_t s);
// Support of S_k from the support words of the tensor-core pass (TcPassArgs::swords): counts
// per row and per chunk of 32 words (cc[chunk][row]; rowcnt must be zero before), then (after
// the scan of rowcnt) the ordered write of indices and values S_ij = D_ij - L_ij.
constexpr int kWordChunk = 32;
// Support changes of the learned schedule after a tensor-core pass: chgP[b] for b < nblocks.
cudaError_t launch_count_mask_changes(const unsigned* masks, long long sz, long long nwords, const DevState* st,
                                      unsigned long long* chgP, int nblocks, cudaStream_t s);
cudaError_t launch_words_count(const unsigned* words, int nw, int m, unsigned* cc, unsigned long long* rowcnt,
                               cudaStream_t s);
cudaError_t launch_extract_words_f32(int R, const ExtractArgs& a, const unsigned* words, const unsigned* cc, int nw,
                                     cudaStream_t s);
cudaError_t launch_convert_f64_to_f32(const double* src, long long ld_src, float* dst, int m, int n,
                                      cudaStream_t s);
cudaError_t launch_convert_f32_to_f64(const float* src, long long ld_src, double* dst, int m, int n,
                                      cudaStream_t s);
// Number of entries of D (m x n, leading dimension ld, FP32 if f32 else FP64) that are not NaN,
// into *count (device).
cudaError_t launch_count_observed(const void* D, long long ld, int m, int n, bool f32, unsigned long long* count,
                                  cudaStream_t s);
// hi = bf16_rn(d), lo = bf16_rn(d - hi) into rows of ld_dst elements; lo may be null.
cudaError_t launch_convert_f32_to_bf16x2(const float* src, long long ld_src, void* hi, void* lo, long long ld_dst,
                                         int m, int n, cudaStream_t s);

}  // namespace rpca
