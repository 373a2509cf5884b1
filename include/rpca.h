/*
 * rpca.h -- C ABI of the GB300 AccAltProj library (robust PCA by accelerated alternating
 * projections, Cai, Cai & Wei, arXiv 1711.05519).
 *
 * Problem (Eq. (1)): split an m x n matrix D into L + S with rank(L) <= r and S sparse.
 * The library runs Algorithm 3 (initialisation) and Algorithm 1 (the iteration) on one
 * GPU.  Every m x n step happens in one fused streaming pass over D per iteration; the
 * O((m+n) r) steps (QR, 2r x 2r SVD, trim) run in small device kernels.
 *
 * Conventions for every call below:
 *   - Matrices are row-major.  D has leading dimension ld >= n (in elements).
 *   - Unless a name ends in _host, every pointer argument is a DEVICE pointer.
 *   - All device work is enqueued on the CUDA stream given to rpca_create (NULL = the
 *     legacy default stream).  Calls return after enqueueing, except where a host value
 *     is needed (stated per call).
 *   - No exception crosses the ABI.  A context is not thread-safe; separate contexts are.
 *   - Return values are rpca_status codes; rpca_status_string() names them.
 */
#ifndef RPCA_H
#define RPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RPCA_OK = 0,
  RPCA_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, unsupported rank or mode      */
  RPCA_ERR_CUDA = 2,          /* a CUDA runtime call failed                             */
  RPCA_ERR_NUMERICAL = 3,     /* NaN/Inf in D or in the factors                         */
  RPCA_ERR_CAPACITY = 4,      /* output buffer too small; required size is returned     */
  RPCA_ERR_NOT_CONVERGED = 5, /* max_iter reached; outputs are valid (last iterate)     */
  RPCA_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up                     */
  RPCA_ERR_STATE = 7          /* call out of order (e.g. iterate before init)           */
} rpca_status;

typedef enum { RPCA_DTYPE_F64 = 0, RPCA_DTYPE_F32 = 1 } rpca_dtype;

/* Arithmetic of the fused pass.
 *   FP64, FP32: D and the pass in that precision.
 *   BF16: the passes read D rounded to bf16 (a copy the context owns, 2 bytes per entry);
 *     the rest of the pass as in FP32.  The iteration then solves the problem for bf16(D):
 *     err_k measures against bf16(D), and once zeta_k falls below the rounding of D that
 *     rounding enters S, so err_k keeps falling while L_k stops improving at the part of the
 *     rounding the tangent space keeps (relative error of L about 1e-4 at n = 500 and 1e-5
 *     at n = 10^4 for r = 5).
 *   BF16_SPLIT: D is held as hi = bf16(D) and lo = bf16(D - hi) (4 bytes per entry); the
 *     passes read hi alone until err_k < split_switch and hi + lo (D to 2^-16 relative)
 *     after that, and only a pass that read hi + lo can end the run.
 * Both pass kinds read the bf16 storage.  The BF16 modes are not part of the method in the
 * paper (which states no precision): they apply its iteration to a quantised D and then to
 * D itself.  The sparse output is extracted from D in FP32. */
typedef enum {
  RPCA_PREC_FP64 = 0,
  RPCA_PREC_FP32 = 1,
  RPCA_PREC_BF16 = 2,
  RPCA_PREC_BF16_SPLIT = 3
} rpca_precision;

/* Threshold rule.  PAPER: zeta_{k+1} = beta (sigma_{r+1} + gamma^{k+1} sigma_1) of
 * P_T(D - S_k) (Algorithm 1).  SIMPLE: zeta_{k+1} = beta gamma^{k+1} sigma_1.
 * EXTERNAL: the caller sets zeta before each iteration with rpca_set_zeta.
 * LEARNED (not in the paper): zeta_{k+1} = zeta^plain_{k+1} exp(clamp(g(s_k), -log 4, log 4)),
 *   zeta^plain the PAPER rule and g a 6 -> 32 -> 32 -> 1 tanh network (FP32) on the statistics
 *   s_k = [log sigma_1, log(sigma_{r+1}/sigma_1), log err_k, fraction of the entries whose
 *   support membership changed since pass k - 1 (0 at k = 0), (k + 1) / K, log(zeta_k/sigma_1)]
 *   (FP32, arguments of the logarithms floored at 1e-37),
 *   evaluated on the device inside the iteration; parameters and K from rpca_set_schedule.
 *   The passes then also keep the support of the last two passes as bitmasks (2 m n / 8 bytes). */
typedef enum {
  RPCA_ZETA_PAPER = 0,
  RPCA_ZETA_SIMPLE = 1,
  RPCA_ZETA_EXTERNAL = 2,
  RPCA_ZETA_LEARNED = 3
} rpca_zeta_mode;

/* Number of FP32 parameters of the LEARNED threshold network, packed (row-major weight
 * matrices, output index first): W1 [32][6] | b1 [32] | W2 [32][32] | b2 [32] | w3 [32] | b3. */
#define RPCA_SCHEDULE_PARAMS 1313

typedef struct {
  double beta;       /* threshold parameter of Algorithm 1                               */
  double gamma;      /* convergence-rate parameter, 0 <= gamma < 1                        */
  double tol;        /* stop when err_k < tol (Eq. (11))                                  */
  double beta_init;  /* Algorithm 3 threshold parameter; 0 selects 2 beta (Section 3)     */
  double mu_trim;    /* incoherence level for Trim; 0 selects 2 beta sqrt(mn) / r         */
  int max_iter;      /* iteration cap; Section 3 uses 100                                 */
  int trim;          /* 1: Trim (Algorithm 2) before each projection; 0: skip it          */
  int precision;     /* rpca_precision                                                   */
  int zeta_mode;     /* rpca_zeta_mode                                                   */
  int init_max_passes; /* cap on D passes of each subspace iteration in rpca_init; 0=40   */
  double init_tol;   /* residual of the top Ritz triplets that ends a subspace iteration;
                        0 selects 1e-13 (FP64) / 1e-5 (FP32)                             */
  int pass_kind;     /* rpca_pass_kind: kernel of the fused pass                          */
  double split_switch; /* BF16_SPLIT: err_k level below which the passes read hi + lo; 0
                          selects 1e-2 (must lie above the bf16 floor of err_k)            */
  int observed;      /* rpca_observed: which entries of D are observed                    */
} rpca_params;

/* Observed entries.  ALL: the problem of the paper, every entry of D is observed.
 * NAN: robust PCA from a subset of the entries (the question the paper's closing section
 *   leaves open; not part of its method): an entry of D that is NaN is unobserved.  With
 *   P_Obs keeping the observed entries and p = |Obs| / (m n) (counted in rpca_init), every
 *   step of Algorithms 1-3 goes through P_Obs: the initialisation works on P_Obs(D) / p, the
 *   iteration takes L_{k+1} = H_r(P_T(L_k + P_Obs(D - L_k - S_k) / p)), S and err_k are
 *   taken on the observed entries only (err_k = ||P_Obs(D - L_k - S_k)|| / ||P_Obs(D)||).
 *   Not with zeta_mode LEARNED. */
typedef enum { RPCA_OBS_ALL = 0, RPCA_OBS_NAN = 1 } rpca_observed;

/* Kernel of the fused pass.  AUTO takes the tensor-core (tcgen05 + TMA) pass where it
 * applies (padded rank <= 16; FP32 with ld a multiple of 4 and D 16-byte aligned, or a BF16
 * mode) and the SIMT pass otherwise; SIMT and TENSOR force one (TENSOR falls back to SIMT
 * where it does not apply). */
typedef enum { RPCA_PASS_AUTO = 0, RPCA_PASS_SIMT = 1, RPCA_PASS_TENSOR = 2 } rpca_pass_kind;

typedef struct {
  int k;               /* iteration index of L_k, S_k                                     */
  double err;          /* err_k = ||D - L_k - S_k||_F / ||D||_F                           */
  double zeta;         /* zeta_k used for S_k                                            */
  double sigma1;       /* sigma_1 of P_T(D - S_k) (0 if the iteration stopped at k)       */
  double sigma_r1;     /* sigma_{r+1} of P_T(D - S_k)                                    */
  int64_t nnz;         /* |supp(S_k)|                                                    */
  double zeta_next_plain; /* zeta^plain_{k+1} of Algorithm 1 (0 if the iteration stopped)   */
  double g;            /* LEARNED: clamped network output g(s_k); zeta_{k+1} = plain e^g  */
  double features[6];  /* LEARNED: the statistics s_k the network read (0 otherwise)       */
  int64_t support_changes; /* LEARNED: entries whose support membership changed since k-1 */
} rpca_iter_stats;

typedef struct rpca_ctx rpca_ctx;

const char* rpca_status_string(int status);

/* Fills *p with the defaults above (beta = gamma = tol = 0 must still be set). */
int rpca_params_default(rpca_params* p);

/* Creates a context.  `stream` is a cudaStream_t (may be NULL).  The context owns its
 * device workspace; rpca_destroy frees it. */
int rpca_create(rpca_ctx** ctx, const rpca_params* params, void* stream);
void rpca_destroy(rpca_ctx* ctx);

/* Algorithm 3 (initialisation by two steps of AltProj).
 *   D: device, m x n, row-major with leading dimension ld, element type `dtype`.
 *   The context BORROWS D when dtype matches the precision (FP64/F64, FP32/F32): the
 *   caller keeps D alive and unchanged until rpca_destroy or the next rpca_init.  With
 *   an F64 input and FP32 precision the context keeps its own FP32 copy.  In the BF16 modes
 *   the context also keeps bf16 copies of D (hi, and lo for BF16_SPLIT; rows padded to a
 *   multiple of 8 entries), made here.
 *   r: target rank, 1 <= r <= 16, 2r <= min(m, n).
 * sigma_1(D) and the top-r SVD of D - S_{-1} are computed by block subspace iteration
 * with one fused pass over D per step.  Synchronises the stream once per pass. */
int rpca_init(rpca_ctx* ctx, const void* D, int64_t m, int64_t n, int64_t ld, int dtype, int r);

/* Runs up to n_iters iterations of Algorithm 1 (each: Trim, one fused pass giving S_k
 * and err_k, then the QR + 2r x 2r SVD route to L_{k+1} and zeta_{k+1}).  Stops early
 * when err_k < tol or k reaches max_iter.  `stats` (host, may be NULL) receives one
 * entry per pass run; *n_done (host, may be NULL) their number.  Returns RPCA_OK when
 * converged, RPCA_ERR_NOT_CONVERGED when n_iters passes ran without convergence (call
 * again to continue) or max_iter was hit.  Synchronises the stream at its end. */
int rpca_iterate(rpca_ctx* ctx, int n_iters, rpca_iter_stats* stats, int* n_done);

/* Reports the fused-pass kernel in use after rpca_init (host outputs): for the iterations
 * of Algorithm 1 and for the passes of the initialisation, RPCA_PASS_SIMT or
 * RPCA_PASS_TENSOR. */
int rpca_get_pass_kind(rpca_ctx* ctx, int* iteration_kind, int* init_kind);

/* Sets zeta_k for the next pass (zeta_mode EXTERNAL). */
int rpca_set_zeta(rpca_ctx* ctx, double zeta);

/* zeta_mode LEARNED: the network parameters (device, RPCA_SCHEDULE_PARAMS floats, copied into
 * the context) and the unrolled depth K of the statistic (k + 1) / K.  Must be called before
 * rpca_iterate (RPCA_ERR_STATE otherwise); RPCA_ERR_STATE in the other modes. */
int rpca_set_schedule(rpca_ctx* ctx, const float* theta, int depth);

/* Copies the four operands the next pass reads, into caller-owned device buffers of the
 * context's working precision (float in FP32 / BF16 modes, double in FP64): W = U_k Sigma_k
 * (m x R), V_k (n x R), and the trimmed orthonormal bases U~_k (m x R), V~_k (n x R) of
 * Section 2.1, row-major, zero-padded to the width R written to *width (host; the padded
 * rank, at most 16).  A checkpoint of the iterate in the form the pass uses; the learned
 * schedule trains on them.  Not part of the paper's method. */
int rpca_get_pass_operands(rpca_ctx* ctx, void* W, void* V, void* Ut, void* Vt, int* width);

/* Copies the current low-rank factors L_k = U diag(sigma) V^T into caller-owned device
 * buffers: U (m x r), sigma (r), V (n x r), all double, row-major. */
int rpca_get_lowrank(rpca_ctx* ctx, double* U, double* sigma, double* V);

/* Writes supp(S_k) = {(i,j) : |D_ij - L_k,ij| > zeta_k} (Eq. (10)) as linear indices
 * i*n + j in ascending order with the values S_ij = D_ij - L_k,ij, into caller-owned
 * device buffers idx (int64) and val (double).  If cap < nnz returns RPCA_ERR_CAPACITY
 * and writes only *nnz (host).  When the last fused pass computed S_k itself (a converged
 * FP32 solve on the tensor-core pass: the update before that pass predicts it to be the last
 * and the pass writes its support as bit masks), the support is read from those masks and
 * D only where S_k is nonzero; otherwise two passes over D count and write it.  The
 * support is then the pass's own (its count equals the iteration statistics' nnz), the
 * count is known on the host and the call returns with the writes queued on the context's
 * stream: idx and val are ready in stream order (synchronise that stream before reading them
 * from the host or from another stream).  Otherwise the call synchronises the stream (the
 * count decides the capacity check) and returns with the writes done. */
int rpca_get_sparse(rpca_ctx* ctx, int64_t* idx, double* val, int64_t cap, int64_t* nnz);

/* Bit of the checkpoint flags: the passes of a BF16_SPLIT solve read hi + lo. */
#define RPCA_STATE_READS_LO 1

/* Iteration state for a checkpoint: *k (host) = index of the iterate L_k the context holds,
 * *zeta (host) = the threshold zeta_k its next pass uses, *flags (host, may be NULL) = the
 * RPCA_STATE_* bits of the solve.  Synchronises the stream. */
int rpca_get_state(rpca_ctx* ctx, int* k, double* zeta, int* flags);

/* Resumes from a checkpoint of the factors (rpca_get_lowrank) and of rpca_get_state, e.g.
 * after the process that held them failed: U (m x r), sigma (r), V (n x r) are device FP64
 * arrays as rpca_get_lowrank writes them; k, zeta and flags as rpca_get_state returned them.
 * The context must have been initialised (rpca_init) on the same D, rank and precision; its
 * iterate is replaced, Trim and the bases for the next pass are recomputed (Algorithm 2), and
 * rpca_iterate continues from iteration k on the path the interrupted solve would have taken
 * (with RPCA_STATE_READS_LO a BF16_SPLIT solve keeps reading hi + lo).  Only the factors are
 * checkpointed, never an m x n array.  Not part of the paper's method.  Synchronises the
 * stream. */
int rpca_set_lowrank(rpca_ctx* ctx, const double* U, const double* sigma, const double* V, int k, double zeta,
                     int flags);

/* One call: init + iterate to tolerance + outputs.  D, U, sigma, V, s_idx, s_val are
 * device pointers; D is float32, m x n, leading dimension n; FP32 precision.  *nnz,
 * *iters, *err are host.  If s_cap < nnz the sparse part is not written and
 * RPCA_ERR_CAPACITY is returned with the other outputs valid. */
int rpca_solve(const float* D, int64_t m, int64_t n, int r, double beta, double gamma, double tol,
               double* U, double* sigma, double* V, int64_t* s_idx, double* s_val, int64_t s_cap,
               int64_t* nnz, int* iters, double* err);

/* As rpca_solve, with every array in HOST memory (D float32; outputs double/int64).  The
 * host-to-device copy of D and the device-to-host copies of the outputs are part of the
 * call.  The device buffers, stream and context it needs are kept between calls (one set per
 * process for the current device, grown when a call needs more) so that repeated calls do not
 * allocate; calls are serialised by a lock.  A CUDA error frees the set; so does
 * rpca_solve_host_release. */
int rpca_solve_host(const float* D, int64_t m, int64_t n, int r, double beta, double gamma,
                    double tol, double* U, double* sigma, double* V, int64_t* s_idx,
                    double* s_val, int64_t s_cap, int64_t* nnz, int* iters, double* err);

/* Frees the device buffers, stream and context kept by rpca_solve_host (the next call
 * allocates them again).  Not part of the paper's method. */
void rpca_solve_host_release(void);

/* Self-test of the bounded device-side waits, on the current device: a kernel waits for an
 * mbarrier phase that nothing completes (1 ms limit) and a kernel waits at a grid barrier that
 * one of its two blocks never reaches (1 s limit).  Each records RPCA_ERR_TIMEOUT instead of
 * hanging; *mbar_status and *grid_status (host) receive the recorded codes.  The context stays
 * usable.  Not part of the paper's method. */
int rpca_selftest_waits(int* mbar_status, int* grid_status);

/* ---------------------------------------------------------------------------------------
 * Learned threshold schedule: stateless pass and adjoint pass.
 *
 * Training a schedule zeta_k = f(statistics) through an unrolled AccAltProj needs the
 * derivative of one pass in zeta, which the hard threshold of Eq. (10) does not have.
 * These calls evaluate the pass with the soft gate g(R; zeta) = sigmoid((|R| - zeta) /
 * (tau zeta)), S = R g, Z = D - S (tau = 0 gives the hard threshold of Eq. (10)), and its
 * exact adjoint.  They allocate nothing and touch no context.
 *   D: device, m x n, leading dimension ld, dtype F32 or F64.  W = U Sigma (m x r),
 *   V (n x r), U~ (m x r), V~ (n x r): device, the same dtype, row-major.  r must be one
 *   of 1..8, 10, 12, 14, 16 (pad the factors with zero columns otherwise).
 *   zeta: device pointer to one double.
 * rpca_learn_pass writes Y1 = Z V~ (m x r), Y2 = Z^T U~ (n x r) and stats[0..2] (device
 * doubles): sum of (R - S)^2 over all entries, the hard support size |{|R| > zeta}|, and,
 * when mask_old is given, the number of entries whose hard support membership differs
 * from mask_old.  mask_new (optional) receives the hard support as a bitmask of
 * m * ceil(n/32) words (bit j%32 of word i*ceil(n/32) + j/32).
 * rpca_learn_pass_adjoint takes the cotangents Y1b (m x r), Y2b (n x r), resb of (Y1, Y2,
 * stats[0]) and writes the cotangents of U~ (Utb), V~ (Vtb), W (Wb), V (Vb) and of zeta
 * (*zetab, device).  Outputs are cleared by the call; sums use atomics, so results vary at
 * rounding level between runs.  Both calls enqueue on `stream` and return. */
int rpca_learn_pass(const void* D, int64_t m, int64_t n, int64_t ld, int dtype, int r, const void* W,
                    const void* V, const void* Ut, const void* Vt, const double* zeta, double tau,
                    void* Y1, void* Y2, double* stats, const uint32_t* mask_old, uint32_t* mask_new,
                    void* stream);
int rpca_learn_pass_adjoint(const void* D, int64_t m, int64_t n, int64_t ld, int dtype, int r,
                            const void* W, const void* V, const void* Ut, const void* Vt,
                            const double* zeta, double tau, const void* Y1b, const void* Y2b,
                            double resb, void* Utb, void* Vtb, void* Wb, void* Vb, double* zetab,
                            void* stream);

/* ---------------------------------------------------------------------------------------
 * Training the LEARNED threshold schedule (not part of the paper's method).  All device
 * pointers; all calls enqueue on `stream` and return.
 *
 * rpca_schedule_forward: for n statistic vectors feats (n x 6 float, the s_k of
 *   rpca_iter_stats.features) and plain thresholds plain (n double, zeta^plain_{k+1}),
 *   zeta[i] = plain[i] exp(clamp(g(feats[i]), -log 4, log 4)) (n double) and, if g is not
 *   NULL, the clamped g (n float): the same arithmetic as the LEARNED iteration.
 * rpca_schedule_backward: theta_bar (RPCA_SCHEDULE_PARAMS floats, overwritten) = gradient of
 *   sum_i zeta_bar[i] zeta[i] with respect to the parameters, by a hand-written backward pass
 *   of the network (zero through a saturated clamp); samples summed in order (deterministic).
 * rpca_adam_step: one Adam update (bias-corrected, step >= 1) of theta (count floats) from
 *   grad, with first / second moment buffers m1, m2 (count floats each, zero at step 1).
 * rpca_projection_loss: the training loss of iteration k,
 *   ||P_T Z - L*||_F^2 / ||L*||_F^2 with P_T Z = F G^T, F = [U~, Y1 - U~ C], G = [Y2, V~],
 *   C = U~^T Y1 (Eq. (6), from the pass products Y1 = Z V~ (m x R) and Y2 = Z^T U~ (n x R)
 *   of rpca_learn_pass; U~ (m x R), V~ (n x R) of the same dtype; only the first r columns
 *   are used), L* = P Q^T (P m x rp, Q n x rp, double, row-major), into *loss (device
 *   double), and its gradients Y1b (m x R), Y2b (n x R) with respect to Y1, Y2 (padding
 *   columns zero).  work: device doubles, 2 r (m + n).  r <= R <= 16, rp <= 16. */
int rpca_schedule_forward(const float* theta, const float* feats, const double* plain, int n, double* zeta, float* g,
                          void* stream);
int rpca_schedule_backward(const float* theta, const float* feats, const double* plain, const double* zeta_bar, int n,
                           float* theta_bar, void* stream);
int rpca_adam_step(float* theta, const float* grad, float* m1, float* m2, int count, int step, double lr, double beta1,
                   double beta2, double eps, void* stream);
int rpca_projection_loss(const void* Y1, const void* Y2, const void* Ut, const void* Vt, int64_t m, int64_t n, int R,
                         int r, int dtype, const double* P, const double* Q, int rp, double* loss, void* Y1b, void* Y2b,
                         double* work, void* stream);

/* Largest m accepted by rpca_get_sparse_noalloc. */
#define RPCA_NOALLOC_MAX_ROWS 65536

/* rpca_get_sparse without any device allocation (the paper has no counterpart; this is a
 * service of the library).  Some callers cannot call cudaMalloc: code that runs inside a
 * framework owning all device memory through its own caching pool (a raw cudaMalloc beside
 * the pool can fail or fragment what the pool has reserved), or code with a fixed
 * device-memory budget set at start-up.  This entry point writes the same support list as
 * rpca_get_sparse for the low-rank estimate L = U diag(sigma) V^T and threshold zeta:
 * linear indices i*n + j in ascending order of every entry with |D_ij - L_ij| > zeta, and
 * the values D_ij - L_ij, computed in FP32 as the FP32 pass does.
 *   D: device, float32, m x n, leading dimension ld.  U (m x r), sigma (r), V (n x r):
 *   device, double, row-major (as returned by rpca_get_lowrank).  idx, val: caller-owned
 *   device buffers of cap entries.  nnz: host.  stream: cudaStream_t (NULL allowed).
 * It allocates nothing: its per-row scratch lives in a static device array of
 * 2 * RPCA_NOALLOC_MAX_ROWS + 1 64-bit words (1 MiB) that every GPU loading the library
 * holds until the process exits.  m above RPCA_NOALLOC_MAX_ROWS returns
 * RPCA_ERR_INVALID_ARG; cap < nnz returns RPCA_ERR_CAPACITY with *nnz set.  Each call looks
 * up the scratch address in the current device's context (a host-side query).  All calls
 * share the scratch and each call rewrites what it reads, so calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the caller.  The call
 * blocks the host: it synchronises the stream twice (after the count, to read the total back,
 * and after the write). */
int rpca_get_sparse_noalloc(const float* D, int64_t m, int64_t n, int64_t ld, int r, const double* U,
                            const double* sigma, const double* V, double zeta, int64_t* idx,
                            double* val, int64_t cap, int64_t* nnz, void* stream);

/* Diagnostics.  on = 0 switches profiling off; on = 1 records CUDA events at the boundaries
 * of every kernel the context launches on its stream; on = k > 1 records them only around
 * every k-th fused-pass launch (the first, the (k+1)-th, ...), which keeps the events out of
 * most kernel boundaries; negative on is RPCA_ERR_INVALID_ARG.  rpca_get_profile (host
 * outputs, any may be NULL) returns, since profiling was last switched on: the summed device
 * time and the number of the timed fused-pass launches that did work, and the summed device
 * time of the other timed launches with the number of every other launch of the library
 * (timed or not, including passes that returned at once because the solve had already
 * converged), so that the two counts add up to all launches.  Synchronises the stream. */
int rpca_set_profiling(rpca_ctx* ctx, int on);
int rpca_get_profile(rpca_ctx* ctx, double* pass_ms, int64_t* pass_launches, double* other_ms,
                     int64_t* other_launches);

#ifdef __cplusplus
}
#endif
#endif /* RPCA_H */
