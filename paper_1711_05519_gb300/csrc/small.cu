// Tall-skinny kernel of the AccAltProj iteration and of the initialisation.
//
// One cooperative launch per call (one block per SM, all co-resident).  Rows of the m x w
// and n x w arrays are split into contiguous block ranges and every per-row step runs on
// the rows a block owns; phases that need a sum over all rows are separated by a bounded
// grid barrier.  Small matrices (w x w Gram matrices, their Cholesky factors, the
// 2r x 2r core M_k and its SVD) are computed redundantly, in the same order, by every
// block, so the only cross-block traffic is the per-block Gram partials.
//
// The per-row work runs in the working precision (double in FP64 mode, float in FP32 mode);
// the small steps of the iteration (Gram sums, Cholesky factors, the 2r x 2r SVD, sigma_1)
// run in double in every mode.  Sums run as pairwise trees, and Cholesky factorisations
// scale the Gram matrix to unit diagonal first.  The Q factor of the projected products is never formed: with
// (I - U~U~^T) Z V~ = W1 = Q1 R1 and Q1 = W1 T1 (T1 upper, T1 = R1^{-1} on the non-zero
// pivots), Eq. (9) becomes U_{k+1} = U~ U_M[:r, :r] + W1 (T1 U_M[r:, :r]).
//
// Modes:
//   SM_UPDATE : after a fused pass of Algorithm 1 (see mode_update): err_k (Eq. (11)) and the
//               stop test; the orthonormal bases U~, V~ of the trimmed factors the pass read;
//               Y1 = Z V~, Y2 = Z^T U~, the QR of their projections (Section 2.1) by Cholesky of
//               Gram matrices, M = [[C, R2^T], [R1, 0]] and its SVD, zeta_{k+1} (Algorithm 1),
//               the new factors (Eq. (9)), Trim (Algorithm 2) and the hand-over to the next pass.
//               One grid barrier (two in FP64 working precision).
//   SM_PREPARE: Trim and hand-over from the factors held (U, sigma, V).
//   SM_RR     : one step of block subspace iteration for Algorithm 3 (sigma_1(D), then the
//               top-r SVD of D - S_{-1}): Rayleigh-Ritz B = U~^T (Z V~), SVD(B), the Ritz
//               residuals, and the next bases orth(Z V~), orth(Z^T U~) by CholeskyQR2; after
//               the last step, Trim and the hand-over to the first pass of Algorithm 1.
//   SM_RAND   : random orthonormal starting bases for SM_RR.
//   SM_BASES  : the orthonormal bases U~, V~ of the next pass, for a caller.
// Where the next pass is the tensor-core one, the step that writes the pass copies also
// writes that pass's operand images (tc_images.cuh) for the rows it owns.
//
// The SVD is a one-sided Jacobi run by one warp with a column per lane, in single
// precision; in FP64 mode V is then re-orthonormalised in double and double-precision
// sweeps polish the result.  Double-precision operations are long-latency on this part, so
// the serial steps (factorisations, the SVD, the sums over blocks) keep them few and, where
// they remain, arranged as trees rather than chains.
#include <math.h>

#include "common.cuh"
#include "factor.cuh"
#include "mlp.cuh"
#include "tc_images.cuh"
#include "tc_util.cuh"

namespace rpca {

namespace {

using fac::rsqrt_d;

constexpr int ST = 256;             // threads per block
constexpr int MW = 16;              // max width of the tall-skinny arrays
constexpr int GSLOT = MW * MW;      // entries per Gram partial
constexpr int kErrTimeout = 6;
constexpr int kErrNumerical = 3;
constexpr unsigned FULL = 0xffffffffu;

template <typename T, int WM>
struct Smem {
  static constexpr int NM = 2 * WM;  // max order of the small SVD
  T red[ST];
  double dred[ST / 32];
  unsigned long long ured[2][ST / 32];
  T G[3][GSLOT];           // reduced Gram matrices (row-major, leading dimension w)
  T Rf[2][GSLOT];          // Cholesky factors (upper)
  T Tf[2][GSLOT];          // T factors: X T has orthonormal columns (upper)
  T C[GSLOT];              // U~^T Y1 (leading dimension r)
  T cm[WM * WM];           // C zero-padded to WM x WM
  T M[NM * NM];            // small SVD input (row-major, leading dimension NM, zero-padded)
  T UM[NM * NM];           // left singular vectors, column c at UM[c * NM + i], descending
  T VM[NM * NM];           // right singular vectors
  T sig[NM];               // singular values, descending
  T scal[4];
  T stage[2][ST * WM];     // rows staged for the Gram sums (row stride WM)
  T mat[2][2 * WM * WM];   // per side: rows 0..w-1 act on the basis, rows w..2w-1 on W
  T tm[2][WM * WM];        // T factors zero-padded to WM x WM
  T sv[2][MW];             // sigma_c, 1/sigma_c
  int pairs[32 * 32];      // Jacobi round-robin partner of each lane in each round
  int ok;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait.  Returns false (and leaves a TIMEOUT status) if
// another block failed to arrive within one second, so no block can spin forever.
template <typename S>
__device__ bool grid_barrier(DevState* st, S& sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &st->bar_gen;
    volatile int* status = &st->status;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&st->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer();
      while (*gen == g && *status == 0) {
        if (globaltimer() - t0 > 1000000000ull) {
          atomicCAS(&st->status, 0, kErrTimeout);
          break;
        }
      }
    }
    __threadfence();
    sh.ok = (*status == 0);
  }
  __syncthreads();
  return sh.ok != 0;
}

// The same barrier, with `idle` run by every thread but thread 0 while thread 0 waits for the
// other blocks (work that needs nothing from them).
template <typename S, typename F>
__device__ bool grid_barrier(DevState* st, S& sh, F idle) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &st->bar_gen;
    volatile int* status = &st->status;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&st->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer();
      while (*gen == g && *status == 0) {
        if (globaltimer() - t0 > 1000000000ull) {
          atomicCAS(&st->status, 0, kErrTimeout);
          break;
        }
      }
    }
    __threadfence();
    sh.ok = (*status == 0);
  } else {
    idle();
  }
  __syncthreads();
  return sh.ok != 0;
}

__device__ __forceinline__ void block_range(int rows, int& lo, int& hi) {
  const int chunk = (rows + gridDim.x - 1) / gridDim.x;
  lo = min(rows, (int)blockIdx.x * chunk);
  hi = min(rows, lo + chunk);
}

template <typename T>
__device__ __forceinline__ T* slot_ptr(void* part, int slot, int block) {
  return static_cast<T*>(part) + ((size_t)slot * gridDim.x + block) * GSLOT;
}

// Block-wide sums of v (double, summed in a fixed order: lanes by xor shuffles, then the
// warps' partials by halving) and of z (and of z2 when it is not null) in one round of the
// shared-memory reduction; every thread gets the totals.
template <typename S>
__device__ __noinline__ void block_sum_dz(double& v, unsigned long long& z, unsigned long long* z2, S& sh) {
  const int t = threadIdx.x;
  unsigned long long y = z2 ? *z2 : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(FULL, v, o);
    z += __shfl_xor_sync(FULL, z, o);
    y += __shfl_xor_sync(FULL, y, o);
  }
  __syncthreads();
  if ((t & 31) == 0) {
    sh.dred[t >> 5] = v;
    sh.ured[0][t >> 5] = z;
    sh.ured[1][t >> 5] = y;
  }
  __syncthreads();
  double w[ST / 32];
  unsigned long long sz = 0, sy = 0;
#pragma unroll
  for (int q = 0; q < ST / 32; ++q) {
    w[q] = sh.dred[q];
    sz += sh.ured[0][q];
    sy += sh.ured[1][q];
  }
#pragma unroll
  for (int h = ST / 64; h > 0; h >>= 1)
#pragma unroll
    for (int q = 0; q < h; ++q) w[q] += w[q + h];
  __syncthreads();
  v = w[0];
  z = sz;
  if (z2) *z2 = sy;
}

// Per-thread share of X^T Y over the staged rows (row stride WM): thread t takes entry
// p = t % P and rows l, l + nl, ... with l = t / P, nl = ST / P (P = wx * wy <= 256).
template <typename T, int WM>
__device__ __forceinline__ T gram_acc(const T* X, int wx, const T* Y, int wy, int nrows, T acc) {
  const int P = wx * wy, t = threadIdx.x, nl = ST / P, l = t / P;
  if (l < nl) {
    const int p = t % P, a = p / wy, b = p % wy;
    for (int i = l; i < nrows; i += nl) acc = fma(X[i * WM + a], Y[i * WM + b], acc);
  }
  return acc;
}

// Pairwise sum of K (a power of two) values, in a fixed order.
template <typename T, int K>
__device__ __forceinline__ T tree_sum(T (&v)[K]) {
#pragma unroll
  for (int h = K / 2; h > 0; h >>= 1)
#pragma unroll
    for (int u = 0; u < h; ++u) v[u] += v[u + h];
  return v[0];
}

// sh.red[j] <- sum over q < nparts of sh.red[q * cnt + j] (j < cnt), pairwise in a fixed
// order (a tree is shorter than a chain).  sh.red must be written and synchronised before
// the call.
template <typename S>
__device__ __noinline__ void tree_combine(int cnt, int nparts, S& sh) {
  const int t = threadIdx.x, q = t / cnt, j = t % cnt;
  int h = 1;
  while (h < nparts) h <<= 1;
  for (h >>= 1; h > 0; h >>= 1) {
    if (q < h && q + h < nparts) sh.red[q * cnt + j] += sh.red[(q + h) * cnt + j];
    __syncthreads();
  }
}

// Combines the per-thread shares of a P-entry Gram matrix into this block's partial.
template <typename T, typename S>
__device__ __noinline__ void gram_store(T acc, int P, void* part, int slot, S& sh) {
  const int t = threadIdx.x;
  sh.red[t] = acc;
  __syncthreads();
  tree_combine(P, ST / P, sh);
  if (t < P) slot_ptr<T>(part, slot, blockIdx.x)[t] = sh.red[t];
  __syncthreads();
}

// G + s * GSLOT <- sum over blocks of slot (slot0 + s), entries 0..P-1, for s < ns.  The
// summation order depends only on the grid size, so every block gets the same bits.
template <typename T, typename S>
__device__ __noinline__ void reduce_slots(const void* part, int slot0, int ns, int P, T* G, S& sh) {
  const int t = threadIdx.x, nb = gridDim.x, total = ns * P;
  const T* pb = static_cast<const T*>(part);
  for (int j0 = 0; j0 < total; j0 += ST) {
    const int cnt = min(ST, total - j0);
    const int nch = min(32, ST / cnt);
    const int c = t / cnt;
    T s = T(0);
    if (c < nch) {
      const int j = j0 + t % cnt;
      const T* base = pb + (size_t)(slot0 + j / P) * nb * GSLOT + (j % P);
      for (int b0 = c; b0 < nb; b0 += 16 * nch) {
        T v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int b = b0 + u * nch;
          v[u] = (b < nb) ? base[(size_t)b * GSLOT] : T(0);
        }
        s += tree_sum<T, 16>(v);
      }
    }
    sh.red[t] = s;
    __syncthreads();
    tree_combine(cnt, nch, sh);
    if (t < cnt) {
      const int j = j0 + t;
      G[(j / P) * GSLOT + (j % P)] = sh.red[t];
    }
    __syncthreads();
  }
}

// R (upper, R^T R = G) and T (X T = Q for X = Q R, upper) of a w x w Gram matrix G (w <= WM,
// row-major, leading dimension w) by one warp (fac::chol_cols).  A real call: the update runs
// it several times per launch from one copy of its code.
template <typename T, int WM>
__device__ __noinline__ void factor_warp(const T* G, int w, T* R, T* Tm) {
  const int l = threadIdx.x & 31;
  T g[WM];
#pragma unroll
  for (int k = 0; k < WM; ++k) g[k] = (l < w && k < w) ? G[k * w + l] : T(0);
  fac::chol_cols<T, WM>(g, w, R, Tm);
}

template <typename T, int WM>
__device__ __forceinline__ void factor_one(const T* G, int w, int s, Smem<T, WM>& sh) {
  factor_warp<T, WM>(G, w, sh.Rf[s], sh.Tf[s]);
}

// Both factors at once: warp 0 factors G[ga] into Rf[0]/Tf[0], warp 1 G[gb] into
// Rf[1]/Tf[1]; then the T factors are copied to sh.tm in the working precision.
template <typename T, int WM>
__device__ void factor_pair(int w, int ga, int gb, Smem<T, WM>& sh) {
  const int warp = threadIdx.x >> 5;
  if (warp == 0) factor_one<T, WM>(sh.G[ga], w, 0, sh);
  if (warp == 1) factor_one<T, WM>(sh.G[gb], w, 1, sh);
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * WM * WM; e += ST) {
    const int s = e / (WM * WM), q = (e / WM) % WM, c = e % WM;
    sh.tm[s][q * WM + c] = (q < w && c < w) ? sh.Tf[s][q * w + c] : T(0);
  }
  __syncthreads();
}

template <typename T, int WM>
__device__ __forceinline__ void zero_row(T (&x)[WM]) {
#pragma unroll
  for (int j = 0; j < WM; ++j) x[j] = T(0);
}

template <typename T, int WM>
__device__ __forceinline__ void load_row(const T* X, size_t i, int w, T (&x)[WM]) {
#pragma unroll
  for (int j = 0; j < WM; ++j) x[j] = (j < w) ? X[i * w + j] : T(0);
}

template <typename T, int WM>
__device__ __forceinline__ void store_row(T* X, size_t i, int w, const T (&x)[WM]) {
#pragma unroll
  for (int j = 0; j < WM; ++j)
    if (j < w) X[i * w + j] = x[j];
}

// Row i of a pass copy of width Rc <= WM: x zero-padded.
template <typename T, int WM>
__device__ __forceinline__ void store_copy(T* X, size_t i, int Rc, const T (&x)[WM]) {
#pragma unroll
  for (int j = 0; j < WM; ++j)
    if (j < Rc) X[i * Rc + j] = x[j];
}

template <typename T, int WM>
__device__ __forceinline__ void stage_row(T* S, int li, const T (&x)[WM]) {
#pragma unroll
  for (int j = 0; j < WM; ++j) S[li * WM + j] = x[j];
}

// y = x A for a WM x WM matrix A in shared memory (row-major, leading dimension WM).
template <typename T, int WM>
__device__ __forceinline__ void row_times(const T (&x)[WM], const T* A, T (&y)[WM]) {
#pragma unroll
  for (int c = 0; c < WM; ++c) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < WM; ++q) s = fma(x[q], A[q * WM + c], s);
    y[c] = s;
  }
}

// Round-robin pairing of N columns (N + 1 if N is odd) for the Jacobi sweeps: lane 0 stays,
// the others move one position per round; pairs[rd * 32 + lane] is the partner of `lane`
// in round rd (itself if it has none).  Written by one warp.
__device__ void jacobi_pairs(int N, int* pairs) {
  const int lane = threadIdx.x & 31;
  const int Np = N + (N & 1), L = Np - 1;
  for (int rd = 0; rd < L; ++rd) {
    int q = lane;
    if (lane < Np) {
      const int pos = (lane == 0) ? 0 : 1 + (lane - 1 + rd) % L;
      const int pp = Np - 1 - pos;
      q = (pp == 0) ? 0 : 1 + ((pp - 1 - rd) % L + L) % L;
    }
    pairs[rd * 32 + lane] = q;
  }
  __syncwarp();
}

// One-sided Jacobi by one warp: lane j < N holds column j of X in x[] and of V in v[]
// (entries >= N zero).  Both lanes of a pair compute the same rotation from the same
// numbers.  A pair rotates while gamma^2 > tol2 * alpha * beta; the sweeps stop when no
// pair rotated.  All partner values are exchanged before the arithmetic so the shuffles
// overlap (a single warp has nothing else to hide their latency).
template <typename U, int NM>
__device__ void jacobi_lanes(int N, U (&x)[NM], U (&v)[NM], U tol2, int max_sweeps, const int* pairs) {
  const int lane = threadIdx.x & 31;
  const int L = N + (N & 1) - 1;
  const U big = sizeof(U) == 4 ? U(1e18) : U(1e150);
  for (int sweep = 0; sweep < max_sweeps && L > 0; ++sweep) {
    bool rot = false;
    for (int rd = 0; rd < L; ++rd) {
      const int q = pairs[rd * 32 + lane];
      const bool low = lane < q;
      U xq[NM], vq[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) xq[i] = __shfl_sync(FULL, x[i], q);
#pragma unroll
      for (int i = 0; i < NM; ++i) vq[i] = __shfl_sync(FULL, v[i], q);
      U sa0 = U(0), sb0 = U(0), sg0 = U(0), sa1 = U(0), sb1 = U(0), sg1 = U(0);
#pragma unroll
      for (int i = 0; i < NM; i += 2) {
        const U a0 = low ? x[i] : xq[i], b0 = low ? xq[i] : x[i];
        sa0 = fma(a0, a0, sa0);
        sb0 = fma(b0, b0, sb0);
        sg0 = fma(a0, b0, sg0);
        const U a1 = low ? x[i + 1] : xq[i + 1], b1 = low ? xq[i + 1] : x[i + 1];
        sa1 = fma(a1, a1, sa1);
        sb1 = fma(b1, b1, sb1);
        sg1 = fma(a1, b1, sg1);
      }
      const U sa = sa0 + sa1, sb = sb0 + sb1, sg = sg0 + sg1;
      bool doit = (q != lane) && sg != U(0) && sg * sg > tol2 * sa * sb;
      if (doit) {
        U tt, c;
        if constexpr (sizeof(U) == 4) {
          // t = tan(theta) of the rotation with tan(2 theta) = 2 gamma / (beta - alpha), the
          // smaller root: t = sign(d) 2 gamma / (|d| + sqrt(d^2 + 4 gamma^2)), d = beta - alpha
          // (one square root and one division); c = 1 / sqrt(1 + t^2) from the hardware
          // estimate and one Newton step y <- y (3 - x y^2) / 2.  The operands are column sums of
          // a matrix scaled to max |M_ij| = 1, so d^2 + 4 gamma^2 cannot overflow.
          // t only has to zero gamma to a few ulps (the next sweep takes what is left), so the
          // square root and the division are the fast hardware approximations; c is refined
          // so that c^2 + s^2 = c^2 (1 + t^2) = 1 to rounding and the rotations stay orthogonal.
          const float d = sb - sa, g2 = 2.f * sg;
          const float e2 = fmaf(d, d, g2 * g2);
          if (e2 > 1e-36f) {  // else both columns are below 1e-18: left as they are
            const float h = e2 * rsqrtf(e2);
            tt = __fdividef(g2, fabsf(d) + h);
            tt = (d < 0.f) ? -tt : tt;
          } else {
            tt = 0.f;
          }
          const float x1 = fmaf(tt, tt, 1.f);
          const float y0 = rsqrtf(x1);
          c = y0 * fmaf(-0.5f * x1 * y0, y0, 1.5f);
        } else {
          const U z = (sb - sa) / (U(2) * sg);
          const U az = fabs(z);
          tt = (az > big) ? U(0.5) / az : U(1) / (az + sqrt(fma(z, z, U(1))));
          tt = (z < U(0)) ? -tt : tt;
          c = U(1) / sqrt(fma(tt, tt, U(1)));
        }
        const U sn = low ? -(c * tt) : (c * tt);  // low: c x - s xq; high: c x + s xq
        doit = tt != U(0);
        if (doit) {
#pragma unroll
          for (int i = 0; i < NM; ++i) {
            x[i] = fma(c, x[i], sn * xq[i]);
            v[i] = fma(c, v[i], sn * vq[i]);
          }
        }
      }
      rot = rot || doit;
    }
    if (!__any_sync(FULL, rot)) break;
  }
}

// Single-precision one-sided Jacobi on the columns of sc * M (N <= NJ <= NM) with V, in
// registers sized NJ; results returned zero-padded to NM.
template <int NJ, int NM, typename T>
__device__ __forceinline__ void jacobi_f32_sized(int N, const T* M, T sc, const int* pairs, float (&x)[NM],
                                                 float (&v)[NM], int max_sweeps = 12) {
  const int lane = threadIdx.x & 31;
  float xj[NJ], vj[NJ];
#pragma unroll
  for (int i = 0; i < NJ; ++i) {
    xj[i] = (lane < N && i < N) ? (float)(M[i * NM + lane] * sc) : 0.f;
    vj[i] = (lane < N && i == lane) ? 1.f : 0.f;
  }
  jacobi_lanes<float, NJ>(N, xj, vj, 1e-11f, max_sweeps, pairs);
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    x[i] = i < NJ ? xj[i < NJ ? i : 0] : 0.f;
    v[i] = i < NJ ? vj[i < NJ ? i : 0] : 0.f;
  }
}

// One-sided Jacobi with two lanes per column (N <= 16): lanes 2j and 2j + 1 hold rows
// 0 .. NH-1 and NH .. 2NH-1 of column j of X (x) and of V (v).  The sums alpha, beta, gamma
// of a pair are formed by halves and added across the two lanes (the same additions in both
// columns' lanes, so both take the same rotation); each lane exchanges and rotates NH entries
// instead of N.  Rotation as in jacobi_lanes (single precision).
template <int NH>
__device__ void jacobi_two_lane(int N, float (&x)[NH], float (&v)[NH], float tol2, int max_sweeps,
                                const int* pairs) {
  const int lane = threadIdx.x & 31, j = lane >> 1, hf = lane & 1;
  const int L = N + (N & 1) - 1;
  for (int sweep = 0; sweep < max_sweeps && L > 0; ++sweep) {
    bool rot = false;
    for (int rd = 0; rd < L; ++rd) {
      const int q = (j < 16) ? pairs[rd * 32 + j] : j;
      const bool low = j < q;
      const int pl = 2 * q + hf;
      float xq[NH], vq[NH];
#pragma unroll
      for (int i = 0; i < NH; ++i) xq[i] = __shfl_sync(FULL, x[i], pl);
#pragma unroll
      for (int i = 0; i < NH; ++i) vq[i] = __shfl_sync(FULL, v[i], pl);
      float sa = 0.f, sb = 0.f, sg = 0.f;
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        const float a = low ? x[i] : xq[i], b = low ? xq[i] : x[i];
        sa = fmaf(a, a, sa);
        sb = fmaf(b, b, sb);
        sg = fmaf(a, b, sg);
      }
      sa += __shfl_xor_sync(FULL, sa, 1);
      sb += __shfl_xor_sync(FULL, sb, 1);
      sg += __shfl_xor_sync(FULL, sg, 1);
      bool doit = (q != j) && j < N && sg != 0.f && sg * sg > tol2 * sa * sb;
      if (doit) {
        const float d = sb - sa, g2 = 2.f * sg;
        const float e2 = fmaf(d, d, g2 * g2);
        float tt = 0.f;
        if (e2 > 1e-36f) {
          const float h = e2 * rsqrtf(e2);
          tt = __fdividef(g2, fabsf(d) + h);
          tt = (d < 0.f) ? -tt : tt;
        }
        const float x1 = fmaf(tt, tt, 1.f);
        const float y0 = rsqrtf(x1);
        const float c = y0 * fmaf(-0.5f * x1 * y0, y0, 1.5f);
        const float sn = low ? -(c * tt) : (c * tt);
        doit = tt != 0.f;
        if (doit) {
#pragma unroll
          for (int i = 0; i < NH; ++i) {
            x[i] = fmaf(c, x[i], sn * xq[i]);
            v[i] = fmaf(c, v[i], sn * vq[i]);
          }
        }
      }
      rot = rot || doit;
    }
    if (!__any_sync(FULL, rot)) break;
  }
}

// small_svd for N <= 2 NH <= 16 in single precision on the two-lane layout; same outputs.
template <int NH, typename T, int WM>
__device__ __forceinline__ void small_svd_two_lane(int N, T mx, T sc, int max_sweeps, Smem<T, WM>& sh) {
  constexpr int NM = Smem<T, WM>::NM;
  const int lane = threadIdx.x & 31, j = lane >> 1, hf = lane & 1;
  float x[NH], v[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    const int row = hf * NH + i;
    x[i] = (j < N && row < N) ? (float)(sh.M[row * NM + j] * sc) : 0.f;
    v[i] = (j < N && row == j) ? 1.f : 0.f;
  }
  jacobi_two_lane<NH>(N, x, v, 1e-11f, max_sweeps, sh.pairs);
  float s2 = 0.f;
#pragma unroll
  for (int i = 0; i < NH; ++i) s2 = fmaf(x[i], x[i], s2);
  s2 += __shfl_xor_sync(FULL, s2, 1);
  const float sf = sqrtf(s2);
  const float inv = sf > 0.f ? 1.f / sf : 0.f;
  const T sg = (j < N) ? (T)(sf * (float)mx) : T(-1);
  int rank = 0;
  for (int i = 0; i < N; ++i) {
    const T si = __shfl_sync(FULL, sg, 2 * i);
    rank += (si > sg || (si == sg && i < j)) ? 1 : 0;
  }
  if (j < N) {
    if (hf == 0) sh.sig[rank] = sg;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const int row = hf * NH + i;
      if (row < NM) {
        sh.UM[rank * NM + row] = (row < N) ? (T)(x[i] * inv) : T(0);
        sh.VM[rank * NM + row] = (row < N) ? (T)v[i] : T(0);
      }
    }
  }
  __syncwarp();
}

// SVD of the N x N matrix in sh.M (N <= NM), by the one warp that calls it.
// On return sh.sig holds the singular values in descending order and sh.UM / sh.VM the
// matching left / right singular vectors (a zero singular value gives a zero left vector).
// Single-precision one-sided Jacobi on M scaled to max |M_ij| = 1 keeps the small singular
// values to high relative accuracy; in FP64 mode V is then re-orthonormalised in double
// and double-precision sweeps on M V polish the result.  pairs_ready: sh.pairs already holds
// jacobi_pairs(N).
template <typename T, int WM>
__device__ __noinline__ void small_svd(int N, Smem<T, WM>& sh, int max_sweeps = 12, bool pairs_ready = false) {
  constexpr int NM = Smem<T, WM>::NM;
  const int lane = threadIdx.x & 31;
  if (!pairs_ready) jacobi_pairs(N, sh.pairs);
  T mx = T(0);
  for (int e = lane; e < N * N; e += 32) mx = fmax(mx, fabs(sh.M[(e / N) * NM + (e % N)]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
  const T sc = mx > T(0) ? T(1) / mx : T(1);
  if constexpr (sizeof(T) == 4) {
    // two lanes per column up to N = 16 (half the exchanges and products per round)
    if (N <= 8) {
      small_svd_two_lane<4, T, WM>(N, mx, sc, max_sweeps, sh);
      return;
    } else if (N <= 10) {
      small_svd_two_lane<5, T, WM>(N, mx, sc, max_sweeps, sh);
      return;
    } else if (N <= 12) {
      small_svd_two_lane<6, T, WM>(N, mx, sc, max_sweeps, sh);
      return;
    } else if (N <= 16) {
      small_svd_two_lane<8, T, WM>(N, mx, sc, max_sweeps, sh);
      return;
    }
  }
  float xf[NM], vf[NM];
  // rotate until every pair of columns is orthogonal to ~3e-6, on registers sized to N
  // (the padding entries are zero and would only add exact zeros)
  if (N <= 8)
    jacobi_f32_sized<8, NM>(N, sh.M, sc, sh.pairs, xf, vf, max_sweeps);
  else if (N <= 10)
    jacobi_f32_sized<(NM < 10 ? NM : 10), NM>(N, sh.M, sc, sh.pairs, xf, vf, max_sweeps);
  else if (N <= 12)
    jacobi_f32_sized<(NM < 12 ? NM : 12), NM>(N, sh.M, sc, sh.pairs, xf, vf, max_sweeps);
  else if (N <= 16 || NM <= 16)
    jacobi_f32_sized<(NM < 16 ? NM : 16), NM>(N, sh.M, sc, sh.pairs, xf, vf, max_sweeps);
  else if (N <= 20)
    jacobi_f32_sized<(NM < 20 ? NM : 20), NM>(N, sh.M, sc, sh.pairs, xf, vf, max_sweeps);
  else if (N <= 24)
    jacobi_f32_sized<(NM < 24 ? NM : 24), NM>(N, sh.M, sc, sh.pairs, xf, vf, max_sweeps);
  else
    jacobi_f32_sized<NM, NM>(N, sh.M, sc, sh.pairs, xf, vf, max_sweeps);
  T sg;
  T y[NM], vd[NM];
  if (sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < NM; ++i) vd[i] = (T)vf[i];
    // V is orthogonal to single precision only: orthonormalise it in double (modified
    // Gram-Schmidt over the lanes) before the double-precision sweeps
    for (int j = 0; j < N; ++j) {
      T s2 = T(0);
#pragma unroll
      for (int i = 0; i < NM; ++i) s2 = fma(vd[i], vd[i], s2);
      if (lane == j) {
        const T inv = T(1) / sqrt(s2);
#pragma unroll
        for (int i = 0; i < NM; ++i) vd[i] *= inv;
      }
      T vj[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) vj[i] = __shfl_sync(FULL, vd[i], j);
      if (lane > j && lane < N) {
        T d = T(0);
#pragma unroll
        for (int i = 0; i < NM; ++i) d = fma(vd[i], vj[i], d);
#pragma unroll
        for (int i = 0; i < NM; ++i) vd[i] = fma(-d, vj[i], vd[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NM; ++k) s = fma(sh.M[i * NM + k], vd[k], s);
      y[i] = (lane < N) ? s : T(0);
    }
    jacobi_lanes<T, NM>(N, y, vd, T(1e-28), 8, sh.pairs);
    T s2 = T(0);
#pragma unroll
    for (int i = 0; i < NM; ++i) s2 = fma(y[i], y[i], s2);
    sg = (lane < N) ? sqrt(s2) : T(-1);
    const T inv = sg > T(0) ? T(1) / sg : T(0);
#pragma unroll
    for (int i = 0; i < NM; ++i) y[i] *= inv;
  } else {
    float s2 = 0.f;
#pragma unroll
    for (int i = 0; i < NM; ++i) s2 = fmaf(xf[i], xf[i], s2);
    const float sf = sqrtf(s2);
    const float inv = sf > 0.f ? 1.f / sf : 0.f;
    sg = (lane < N) ? (T)(sf * (float)mx) : T(-1);
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      y[i] = (T)(xf[i] * inv);
      vd[i] = (T)vf[i];
    }
  }
  int rank = 0;
  for (int i = 0; i < N; ++i) {
    const T si = __shfl_sync(FULL, sg, i);
    rank += (si > sg || (si == sg && i < lane)) ? 1 : 0;
  }
  if (lane < N) {
    sh.sig[rank] = sg;
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      sh.UM[rank * NM + i] = y[i];
      sh.VM[rank * NM + i] = vd[i];
    }
  }
  __syncwarp();
}

// Double-precision sweeps of one-sided Jacobi on nearly orthogonal columns (the refinement
// after the single-precision sweeps): the rotation angle is taken in single precision (near
// convergence only its relative accuracy matters for the quadratic convergence of Jacobi's
// method), the rotation itself is exactly orthogonal in double (c = 1/sqrt(1 + t^2) by
// rsqrt_d, s = c t) and applied in double.  Pairs rotate while gamma^2 > 1e-28 alpha beta.
template <int NM>
__device__ void jacobi_refine_d(int N, double (&x)[NM], double (&v)[NM], int max_sweeps, const int* pairs) {
  const int lane = threadIdx.x & 31;
  const int L = N + (N & 1) - 1;
  for (int sweep = 0; sweep < max_sweeps && L > 0; ++sweep) {
    bool rot = false;
    for (int rd = 0; rd < L; ++rd) {
      const int q = pairs[rd * 32 + lane];
      const bool low = lane < q;
      // partner values are fetched element by element (twice: for the sums and for the
      // rotation) so that only this lane's two columns stay in registers
      double sa = 0.0, sb = 0.0, sg = 0.0;
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        const double xq = __shfl_sync(FULL, x[i], q);
        const double a0 = low ? x[i] : xq, b0 = low ? xq : x[i];
        sa = fma(a0, a0, sa);
        sb = fma(b0, b0, sb);
        sg = fma(a0, b0, sg);
      }
      bool doit = (q != lane) && sg != 0.0 && sg * sg > 1e-28 * sa * sb;
      double c_rot = 1.0, s_rot = 0.0;
      if (doit) {
        // (sb - sa) / (2 sg) in single precision, both terms first scaled by the same power of
        // two so that neither underflows (columns of tiny norm have tiny sums)
        const double num = sb - sa, den = 2.0 * sg;
        int e;
        frexp(fmax(fabs(num), fabs(den)), &e);
        const float zf = (float)ldexp(num, -e) / (float)ldexp(den, -e);
        const float az = fabsf(zf);
        float tf = (az > 1e18f) ? 0.5f / az : 1.0f / (az + sqrtf(fmaf(zf, zf, 1.0f)));
        tf = (zf < 0.0f) ? -tf : tf;
        const double t = (double)tf;
        c_rot = rsqrt_d(fma(t, t, 1.0));
        s_rot = low ? -(c_rot * t) : (c_rot * t);
        doit = tf != 0.0f;
      }
      // every lane takes part in the shuffles; a lane that does not rotate keeps its columns
      const double cc = doit ? c_rot : 1.0, ss = doit ? s_rot : 0.0;
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        const double xq = __shfl_sync(FULL, x[i], q), vq = __shfl_sync(FULL, v[i], q);
        x[i] = fma(cc, x[i], ss * xq);
        v[i] = fma(cc, v[i], ss * vq);
      }
      rot = rot || doit;
    }
    if (!__any_sync(FULL, rot)) break;
  }
}

// Double-precision part of small_svd_d on registers sized NJ >= N: V from the single-precision
// sweeps (vf) re-orthonormalised in double (modified Gram-Schmidt), then double-precision
// sweeps on M V; results sorted by singular value into sh.sig, sh.UM, sh.VM.
template <int NJ, typename T, int WM>
__device__ __forceinline__ void svd_refine_sized(int N, const float* vf, Smem<T, WM>& sh) {
  constexpr int NM = Smem<T, WM>::NM;
  const int lane = threadIdx.x & 31;
  double vd[NJ], y[NJ];
#pragma unroll
  for (int i = 0; i < NJ; ++i) vd[i] = (double)vf[i];
  for (int j = 0; j < N; ++j) {
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < NJ; ++i) s2 = fma(vd[i], vd[i], s2);
    if (lane == j) {
      const double inv = rsqrt_d(s2);
#pragma unroll
      for (int i = 0; i < NJ; ++i) vd[i] *= inv;
    }
    double vj[NJ];
#pragma unroll
    for (int i = 0; i < NJ; ++i) vj[i] = __shfl_sync(FULL, vd[i], j);
    if (lane > j && lane < N) {
      double d = 0.0;
#pragma unroll
      for (int i = 0; i < NJ; ++i) d = fma(vd[i], vj[i], d);
#pragma unroll
      for (int i = 0; i < NJ; ++i) vd[i] = fma(-d, vj[i], vd[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < NJ; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NJ; ++k) acc = fma(sh.M[i * NM + k], vd[k], acc);
    y[i] = (lane < N && i < N) ? acc : 0.0;
  }
  jacobi_refine_d<NJ>(N, y, vd, 4, sh.pairs);
  double s2 = 0.0;
#pragma unroll
  for (int i = 0; i < NJ; ++i) s2 = fma(y[i], y[i], s2);
  const double inv = s2 > 0.0 ? rsqrt_d(s2) : 0.0;
  const double sg = (lane < N) ? s2 * inv : -1.0;
#pragma unroll
  for (int i = 0; i < NJ; ++i) y[i] *= inv;
  int rank = 0;
  for (int i = 0; i < N; ++i) {
    const double si = __shfl_sync(FULL, sg, i);
    rank += (si > sg || (si == sg && i < lane)) ? 1 : 0;
  }
  if (lane < N) {
    sh.sig[rank] = sg;
    for (int i = 0; i < NM; ++i) {
      sh.UM[rank * NM + i] = 0.0;
      sh.VM[rank * NM + i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < NJ; ++i) {
      sh.UM[rank * NM + i] = y[i];
      sh.VM[rank * NM + i] = vd[i];
    }
  }
  __syncwarp();
}

// SVD of the N x N matrix sh.M (N <= NM) by warp 0, double working precision: single-precision
// one-sided Jacobi on M scaled to max |M_ij| = 1, then the double-precision refinement above.
// On return sh.sig holds the singular values in descending order and sh.UM / sh.VM the
// matching left / right singular vectors (column c at [c * NM + i]; a zero singular value
// gives a zero left vector).  Measured on this part (10^4 x 10^4, r = 5): ~165 us, against
// ~20 us for the single-precision sweeps alone (small_svd), which the FP32 working precision
// keeps.
template <typename T, int WM>
__device__ void small_svd_d(int N, Smem<T, WM>& sh) {
  constexpr int NM = Smem<T, WM>::NM;
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  jacobi_pairs(N, sh.pairs);
  double mx = 0.0;
  for (int e = lane; e < N * N; e += 32) mx = fmax(mx, fabs(sh.M[(e / N) * NM + (e % N)]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
  const double sc = mx > 0.0 ? 1.0 / mx : 1.0;
  float xf[NM], vf[NM];
  if (N <= 8) {
    jacobi_f32_sized<8, NM>(N, sh.M, sc, sh.pairs, xf, vf);
    svd_refine_sized<8>(N, vf, sh);
  } else if (N <= 12) {
    jacobi_f32_sized<(NM < 12 ? NM : 12), NM>(N, sh.M, sc, sh.pairs, xf, vf);
    svd_refine_sized<(NM < 12 ? NM : 12)>(N, vf, sh);
  } else if (N <= 16 || NM <= 16) {
    jacobi_f32_sized<(NM < 16 ? NM : 16), NM>(N, sh.M, sc, sh.pairs, xf, vf);
    svd_refine_sized<(NM < 16 ? NM : 16)>(N, vf, sh);
  } else if (N <= 20) {
    jacobi_f32_sized<20, NM>(N, sh.M, sc, sh.pairs, xf, vf);
    svd_refine_sized<20>(N, vf, sh);
  } else {
    jacobi_f32_sized<NM, NM>(N, sh.M, sc, sh.pairs, xf, vf);
    svd_refine_sized<NM>(N, vf, sh);
  }
}

template <typename T, int WM>
__device__ void cta_totals(const SmallArgs& a, double& res2, unsigned long long& nnz, Smem<T, WM>& sh,
                           unsigned long long* changes = nullptr) {
  // every block sums the per-CTA totals in the same order
  const int t = threadIdx.x;
  double s = 0.0;
  unsigned long long z = 0, c2 = 0;
  for (int c = t; c < a.n_cta; c += ST) {
    s += a.resP[c];
    z += a.nnzP[c];
    if (changes && a.chgP) c2 += a.chgP[c];
  }
  block_sum_dz(s, z, changes ? &c2 : nullptr, sh);
  res2 = s;
  nnz = z;
  if (changes) *changes = a.chgP ? c2 : 0ull;
}

// Row i of Y (width w) <- fixed-order sum of the nsl pass partial slices (width R,
// slice stride `stride`).
template <typename T, int WM>
__device__ __forceinline__ void reduce_row(const T* __restrict__ Pp, int nsl, size_t stride, size_t i, int R, int w,
                                           T (&y)[WM]) {
  zero_row<T, WM>(y);
  const T* p = Pp + i * R;
  constexpr int UNR = (WM * sizeof(T) <= 32) ? 8 : 4;  // slices whose loads are issued together
  int q = 0;
  for (; q + UNR <= nsl; q += UNR) {
    T v[UNR][WM];
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int j = 0; j < WM; ++j) v[u][j] = (j < w) ? p[(size_t)(q + u) * stride + j] : T(0);
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int j = 0; j < WM; ++j) y[j] += v[u][j];
  }
  for (; q < nsl; ++q)
#pragma unroll
    for (int j = 0; j < WM; ++j) y[j] += (j < w) ? p[(size_t)q * stride + j] : T(0);
}

// Row i of the tensor-core operand images of image set `set` (0: the initialisation's pass,
// 1: the iteration's): side 0 gives rows of W (= f) and U~ (= q), side 1 rows of V (= f) and
// V~ (= q), in the layout of that pass (img_rk); entries past WM are zero.
template <int RK, typename T, int WM>
__device__ __forceinline__ void write_images_rk(const SmallArgs& a, int set, int side, int i, const T (&f)[WM],
                                                const T (&q)[WM]) {
  float fv[RK], qv[RK];
#pragma unroll
  for (int j = 0; j < RK; ++j) {
    fv[j] = j < WM ? (float)f[j < WM ? j : 0] : 0.f;
    qv[j] = j < WM ? (float)q[j < WM ? j : 0] : 0.f;
  }
  if (side == 0)
    img::write_row_images<RK>(i, fv, qv, a.wop[set], a.utop[set]);
  else
    img::write_col_images<RK>(i, fv, qv, a.vop[set], a.vtop[set]);
}

template <typename T, int WM>
__device__ __noinline__ void write_images(const SmallArgs& a, int set, int side, int i, const T (&f)[WM],
                                          const T (&q)[WM]) {
  if (a.img_rk[set] == 8)
    write_images_rk<8, T, WM>(a, set, side, i, f, q);
  else
    write_images_rk<16, T, WM>(a, set, side, i, f, q);
}

// ---------------------------------------------------------------------------------------
// Half-block steps: the m-side rows (side 0) and the n-side rows (side 1) are
// processed at once, side s by threads s HT .. s HT + HT - 1 with its own named barrier
// (1 + s) and its own staging rows, so neither side waits for the other.
constexpr int HT = ST / 2;

__device__ __forceinline__ void half_sync(int side) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + side), "r"(HT) : "memory");
}

// Entries p = tl and p = tl + HT (p < w^2) of X^T Y over nrows staged rows (row stride WM),
// each added by one thread in row order into acc[0], acc[1] (no cross-thread combination).
template <typename T, int WM>
__device__ __forceinline__ void gram_rows_h(const T* X, const T* Y, int w, int nrows, int tl, T (&acc)[2]) {
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int p = tl + e * HT;
    if (p < w * w) {
      const int ca = p / w, cb = p % w;
      T s = acc[e];
      for (int i = 0; i < nrows; ++i) s = fma(X[i * WM + ca], Y[i * WM + cb], s);
      acc[e] = s;
    }
  }
}

// This block's partial of the Gram matrix (entries as in gram_rows_h) into slot `slot`.
template <typename T>
__device__ __forceinline__ void gram_put_h(const T (&acc)[2], int w, void* part, int slot, int tl) {
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int p = tl + e * HT;
    if (p < w * w) slot_ptr<T>(part, slot, blockIdx.x)[p] = acc[e];
  }
}

// ---------------------------------------------------------------------------------------
// Trim (Algorithm 2) and the hand-over to the next pass.
//
// The pass of iteration k reads W = U_k Sigma_k, V_k and, in place of the orthonormal bases
// U~_k, V~_k of the footnote to Eq. (5), the trimmed factors A~_k, B~_k themselves, so its
// products are X1 = Z B~ and X2 = Z^T A~.  The update that follows takes U~ = A~ T_u and
// V~ = B~ T_v (one CholeskyQR each, T = R^-1 from the Gram matrices of A~, B~), and
// Y1 = Z V~ = X1 T_v, Y2 = Z^T U~ = X2 T_u.  The Gram partials of A~, B~ are written by the
// kernel that trims (slots 6, 7) and summed by the next kernel, so no grid barrier separates
// the trim from the orthonormalisation.

// Pass copies of row i for the next pass: W = f sigma (side 0) or V = f (side 1) and the
// trimmed row t (A~ or B~), zero-padded to width Rit, and (tensor-core pass) their images.
template <typename T, int WM>
__device__ __forceinline__ void hand_over_row(const SmallArgs& a, int side, int i, const T (&f)[WM], const T (&t)[WM],
                                              const T* sig) {
  T w[WM];
#pragma unroll
  for (int j = 0; j < WM; ++j) w[j] = side ? f[j] : f[j] * sig[j];
  store_copy<T, WM>(static_cast<T*>(side ? a.Vc : a.Wc), i, a.Rit, w);
  store_copy<T, WM>(static_cast<T*>(side ? a.Vtc : a.Utc), i, a.Rit, t);
  if constexpr (sizeof(T) == 4) {
    if (a.img_iter) write_images<T, WM>(a, 1, side, i, w, t);
  }
}

// Row f of U (side 0, cap sqrt(mu r / m)) or V (side 1, cap sqrt(mu r / n)) scaled by
// min(1, cap / ||f||) (Algorithm 2), or left as it is without trimming.
template <typename T, int WM>
__device__ __forceinline__ void trim_row(const T (&f)[WM], T cap, bool do_trim, T (&x)[WM]) {
  T nrm = T(0);
#pragma unroll
  for (int j = 0; j < WM; ++j) nrm = fma(f[j], f[j], nrm);
  nrm = sqrt(nrm);
  const T sc = (do_trim && nrm > cap) ? cap / nrm : T(1);
#pragma unroll
  for (int j = 0; j < WM; ++j) x[j] = f[j] * sc;
}

template <typename T>
__device__ __forceinline__ T trim_cap(const SmallArgs& a, int side) {
  return sqrt((T)a.st->mu_trim * (T)a.r / (T)(side ? a.n : a.m));
}

// Trim and hand-over of the factors held (U, V; sigma in sh.sv[0]) over the block's rows,
// with the Gram partials of A~, B~ into slots 6, 7.
template <typename T, int WM>
__device__ void trim_hand_over(const SmallArgs& a, Smem<T, WM>& sh) {
  const int r = a.r, t = threadIdx.x;
  const bool do_trim = a.st->trim != 0;
  const int side = t / HT, tl = t % HT;  // both sides at once on the two half blocks
  const int rows = side ? a.n : a.m;
  const T cap = trim_cap<T>(a, side);
  const T* F = static_cast<const T*>(side ? a.V : a.U);
  T* sx = sh.stage[side];
  int lo, hi;
  block_range(rows, lo, hi);
  T acc[2] = {T(0), T(0)};
  for (int c0 = lo; c0 < hi; c0 += HT) {
    const int i = c0 + tl;
    T x[WM];
    zero_row<T, WM>(x);
    if (i < hi) {
      T f[WM];
      load_row<T, WM>(F, i, r, f);
      trim_row<T, WM>(f, cap, do_trim, x);
      hand_over_row<T, WM>(a, side, i, f, x, sh.sv[0]);
    }
    stage_row<T, WM>(sx, tl, x);
    half_sync(side);
    gram_rows_h<T, WM>(sx, sx, r, min(HT, hi - c0), tl, acc);
    half_sync(side);
  }
  gram_put_h<T>(acc, r, a.part, 6 + side, tl);
}

// T_u, T_v of the trimmed factors the last pass read, from the Gram partials in slots 6, 7
// (every block sums them in the same order; one warp factors each), into sh.tm (zero-padded).
template <typename T, int WM>
__device__ void trimmed_t_factors(const SmallArgs& a, Smem<T, WM>& sh) {
  reduce_slots(a.part, 6, 2, a.r * a.r, &sh.G[0][0], sh);
  factor_pair<T, WM>(a.r, 0, 1, sh);
}

// ---------------------------------------------------------------------------------------
// One update of Algorithm 1 after the fused pass, in the working precision:
//   start: err_k, the stop test, T_u and T_v (above; after a tensor-core pass, which computes
//          them beside its tiles, only loaded)
//   A    : rows of Y1 = X1 T_v, U~ = A~ T_u, Y2 = X2 T_u, V~ = B~ T_v; partials of C = U~^T Y1
//   -- grid barrier --
//   A2   : W1 = Y1 - U~ C and W2 = Y2 - V~ C^T (the projections of Section 2.1) and their
//          Gram partials
//   -- grid barrier --
//   serial (every block, same order): R1, R2 by Cholesky (the QR of Section 2.1, with the Q
//          factors implicit), M = [[C, R2^T], [R1, 0]], its SVD, zeta_{k+1} (Algorithm 1)
//   B    : new factors by Eq. (9), U_{k+1} = U~ U_M[:r, :r] + W1 (T1 U_M[r:, :r]), Trim and
//          the hand-over to the next pass.
// Double-precision serial steps are long-latency on this part (measured at 10^4 x 10^4,
// r = 5: ~250 us per update with the Gram sums, Cholesky factors and the SVD refinement in
// double, against ~60 us in single precision), so only the FP64 working precision runs them
// in double.
template <typename T, int WM>
__device__ void mode_update(const SmallArgs& a, Smem<T, WM>& sh) {
  constexpr int NM = Smem<T, WM>::NM;
  DevState* st = a.st;
  const int m = a.m, n = a.n, r = a.r, t = threadIdx.x;
  T* Ut = static_cast<T*>(a.Ut);
  T* Vt = static_cast<T*>(a.Vt);
  T* Y1 = static_cast<T*>(a.Y1);
  T* Y2 = static_cast<T*>(a.Y2);
  const T* At = static_cast<const T*>(a.Utc);  // A~ and B~ as the pass read them (width Rit)
  const T* Bt = static_cast<const T*>(a.Vtc);
  // the first loads go out together: the T factors the tensor-core pass computed, the state
  // the stop test reads, and (in cta_totals) the pass's per-CTA totals
  constexpr int NTF = (2 * WM * WM + ST - 1) / ST;
  float tfv[NTF];
  if (a.tfac) {
#pragma unroll
    for (int i = 0; i < NTF; ++i) {
      const int e = t + i * ST, q = (e / WM) % WM, c = e % WM;
      tfv[i] = (e < 2 * WM * WM && q < r && c < r) ? a.tfac[(e / (WM * WM)) * 256 + q * r + c] : 0.f;
    }
  }
  const double normD2 = st->normD2, tol = st->tol;
  const int k = st->k, max_iter = st->max_iter;
  const bool hi_only = st->split_switch > 0 && !st->use_lo;
  double res2;
  unsigned long long nnz, changes;
  cta_totals(a, res2, nnz, sh, &changes);
  const double err = sqrt(res2 / normD2);
  if (blockIdx.x == 0 && t == 0) {
    DevStats& s = a.stats[k];
    s.err = err;
    s.zeta = st->zeta;
    s.res2 = res2;
    s.nnz = (long long)nnz;
    s.k = k;
    s.sigma1 = 0.0;
    s.sigma_r1 = 0.0;
    s.zeta_next_plain = 0.0;
    s.g = 0.0;
    for (int i = 0; i < mlp::IN; ++i) s.feat[i] = 0.f;
    s.changes = (k > 0 && a.chgP) ? (long long)changes : 0;
  }
  if (!(err == err) || isinf(err)) {
    if (blockIdx.x == 0 && t == 0) {
      atomicCAS(&st->status, 0, kErrNumerical);
      st->done = 1;
    }
    return;
  }
  // bf16 split storage of D: while the passes read only the hi part (hi_only), err_k measures
  // against bf16(D) and cannot end the run; the next pass reads hi + lo once err_k is below
  // the switch level (use_lo is written below, after grid barriers every CTA passes after the
  // read above)
  if ((err < tol && !hi_only) || k >= max_iter) {
    if (blockIdx.x == 0 && t == 0) st->done = 1;
    return;
  }
  if (a.tfac) {
#pragma unroll
    for (int i = 0; i < NTF; ++i) {
      const int e = t + i * ST;
      if (e < 2 * WM * WM) sh.tm[e / (WM * WM)][e % (WM * WM)] = (T)tfv[i];
    }
    __syncthreads();
  } else {
    trimmed_t_factors<T, WM>(a, sh);
  }

  // A: own rows of Y1, U~ (side 0) and Y2, V~ (side 1), both sides at once; partial of
  // C = U~^T Y1 (slot 0)
  {
    const int side = t / HT, tl = t % HT;
    const int rows = side ? n : m;
    const T* Pp = static_cast<const T*>(side ? a.P2 : a.P1);
    const int nsl_all = side ? a.n_p2 : a.n_p1;
    const T* F = side ? Bt : At;
    T* Yo = side ? Y2 : Y1;
    T* Bo = side ? Vt : Ut;
    T* sb = sh.stage[0];            // side 0: rows of U~ ...
    T* sy = sh.stage[0] + HT * WM;  // ... and of Y1
    int lo, hi;
    block_range(rows, lo, hi);
    T acc[2] = {T(0), T(0)};
    for (int c0 = lo; c0 < hi; c0 += HT) {
      const int i = c0 + tl;
      T y[WM], b[WM];
      zero_row<T, WM>(y);
      zero_row<T, WM>(b);
      if (i < hi) {
        T x[WM], f[WM];
        load_row<T, WM>(F, i, a.Rit, f);
        const int nsl = (!side && a.p1_nsl) ? a.p1_nsl[i >> 7] : nsl_all;
        const int Rw = side ? a.R2 : a.R;  // row width of the partial slices
        reduce_row<T, WM>(Pp, nsl, (size_t)rows * Rw, i, Rw, r, x);
        row_times<T, WM>(x, sh.tm[1 - side], y);  // X1 T_v, X2 T_u
        row_times<T, WM>(f, sh.tm[side], b);      // A~ T_u, B~ T_v
        store_row<T, WM>(Yo, i, r, y);
        store_row<T, WM>(Bo, i, r, b);
      }
      if (!side) {
        stage_row<T, WM>(sb, tl, b);
        stage_row<T, WM>(sy, tl, y);
        half_sync(0);
        gram_rows_h<T, WM>(sb, sy, r, min(HT, hi - c0), tl, acc);
        half_sync(0);
      }
    }
    if (!side) gram_put_h<T>(acc, r, a.part, 0, tl);
  }
  if (!grid_barrier(st, sh)) return;

  // A2: W1 = Y1 - U~ C, W2 = Y2 - V~ C^T (in place) and their Gram matrices (slots 1, 2)
  reduce_slots(a.part, 0, 1, r * r, sh.C, sh);
  for (int e = t; e < WM * WM; e += ST) {
    const int q = e / WM, c = e % WM;
    sh.cm[e] = (q < r && c < r) ? sh.C[q * r + c] : T(0);
  }
  __syncthreads();
  {
    const int side = t / HT, tl = t % HT;
    const int rows = side ? n : m;
    T* Y = side ? Y2 : Y1;
    const T* B = side ? Vt : Ut;
    T* sw = sh.stage[side];
    int lo, hi;
    block_range(rows, lo, hi);
    T acc[2] = {T(0), T(0)};
    for (int c0 = lo; c0 < hi; c0 += HT) {
      const int i = c0 + tl;
      T y[WM];
      zero_row<T, WM>(y);
      if (i < hi) {
        T b[WM];
        load_row<T, WM>(Y, i, r, y);
        load_row<T, WM>(B, i, r, b);
#pragma unroll
        for (int c = 0; c < WM; ++c) {
          T sacc = y[c];
#pragma unroll
          for (int q = 0; q < WM; ++q) sacc = fma(-b[q], side ? sh.cm[c * WM + q] : sh.cm[q * WM + c], sacc);
          y[c] = sacc;
        }
        store_row<T, WM>(Y, i, r, y);
      }
      stage_row<T, WM>(sw, tl, y);
      half_sync(side);
      gram_rows_h<T, WM>(sw, sw, r, min(HT, hi - c0), tl, acc);
      half_sync(side);
    }
    gram_put_h<T>(acc, r, a.part, 1 + side, tl);
  }
  // while thread 0 waits at the barrier, warp 1 runs the Cholesky factorisation on a stand-in
  // matrix: the code of this one-warp serial step is executed once per launch and would
  // otherwise be fetched while the whole grid waits for it (measured: the first factorisation
  // of a launch ~6 us, a second one ~1.6-2 us); its scratch (G[2], the factors) is rewritten
  // after the barrier.  (The same for one Jacobi sweep of the SVD cost more than it saved: its
  // cold run outlasts the barrier.)
  auto warm = [&]() {
    if constexpr (sizeof(T) == 4) {
      const int wp = t >> 5, lane = t & 31;
      if (wp == 1) {
        for (int e = lane; e < r * r; e += 32) sh.G[2][e] = (e / r == e % r) ? T(2) : T(1);
        __syncwarp();
        factor_warp<T, WM>(sh.G[2], r, sh.Rf[0], sh.Tf[0]);
      }
      if (wp == 2) jacobi_pairs(2 * r, sh.pairs);  // the pairing of the SVD below
    }
  };
  if (!grid_barrier(st, sh, warm)) return;

  // R1, R2; M = [[C, R2^T], [R1, 0]] and its SVD
  reduce_slots(a.part, 1, 2, r * r, &sh.G[0][0], sh);
  factor_pair<T, WM>(r, 0, 1, sh);
  const int N = 2 * r;
  for (int e = t; e < NM * NM; e += ST) {
    const int row = e / NM, col = e % NM;
    T v = T(0);
    if (row < r && col < r)
      v = sh.C[row * r + col];
    else if (row < r && col >= r && col < N)
      v = sh.Rf[1][(col - r) * r + row];  // R2^T
    else if (row >= r && row < N && col < r)
      v = sh.Rf[0][(row - r) * r + col];  // R1
    sh.M[e] = v;
  }
  __syncthreads();
  if constexpr (sizeof(T) == 8)
    small_svd_d<T, WM>(N, sh);
  else if (t < 32)
    small_svd<T, WM>(N, sh, 12, true);
  __syncthreads();
  // update matrices: side 0 acts on [U~ W1], side 1 on [V~ W2]; rows q < r take the top block
  // of U_M (V_M), rows r + q the bottom block premultiplied by T1 (T2)
  for (int e = t; e < 2 * 2 * WM * WM; e += ST) {
    const int side = e / (2 * WM * WM), rem = e % (2 * WM * WM), row = rem / WM, c = rem % WM;
    const T* Y = side ? sh.VM : sh.UM;
    T v = T(0);
    if (c < r) {
      if (row < r) {
        v = Y[c * NM + row];
      } else if (row < 2 * r) {
        const int q = row - r;
        for (int kk = q; kk < r; ++kk) v = fma(sh.Tf[side][q * r + kk], Y[c * NM + r + kk], v);
      }
    }
    sh.mat[side][rem] = v;
  }
  if (t < MW) sh.sv[0][t] = (t < r) ? (T)sh.sig[t] : T(0);
  __syncthreads();
  const double s1 = (double)sh.sig[0], sr1 = (double)sh.sig[r];
  if (t < r) static_cast<T*>(a.sig)[t] = (T)sh.sig[t];
  if (blockIdx.x == 0 && t >= ST - 32) {  // a warp with no rows when m, n <= 224 * grid
    const int lane = t & 31;
    const int k1 = k + 1;
    const double gamma = st->gamma, beta = st->beta;
    const int zmode = st->zeta_mode;
    double g = 1.0;  // gamma^(k+1) by repeated multiplication (k is small)
    for (int i = 0; i < k1; ++i) g *= gamma;
    const double plain = beta * (sr1 + g * s1);  // Algorithm 1
    double zeta_new = st->zeta;                   // EXTERNAL: the caller sets it
    if (zmode == 0) {
      zeta_new = plain;
    } else if (zmode == 1) {
      zeta_new = beta * g * s1;
    } else if (zmode == 3) {
      // learned schedule: zeta_{k+1} = zeta^plain_{k+1} exp(clamp(g(s_k))), the network run by
      // this warp on the statistics of this iteration (mlp.cuh)
      float f[mlp::IN], h1, h2;
      const double change = (k > 0 && a.chgP) ? (double)changes / ((double)m * (double)n) : 0.0;
      mlp::features(s1, sr1, err, change, k, a.depth, st->zeta, f);
      const float gc = mlp::clamp_g(mlp::forward_warp(a.theta, f, h1, h2));
      zeta_new = plain * (double)expf(gc);
      if (lane == 0) {
        for (int i = 0; i < mlp::IN; ++i) a.stats[k].feat[i] = f[i];
        a.stats[k].g = (double)gc;
      }
    }
    if (lane == 0) {
      st->zeta = zeta_new;
      a.stats[k].zeta_next_plain = plain;
      for (int i = 0; i < N; ++i) st->sigma[i] = (double)sh.sig[i];
      a.stats[k].sigma1 = s1;
      a.stats[k].sigma_r1 = sr1;
      if (hi_only && (err < st->split_switch || err < st->tol)) st->use_lo = 1;
      // the next pass writes the support words if it is likely the last one: err_{k+1}
      // predicted from the contraction of the last two passes below 2 tol, or k + 1 the cap
      const double prev = k > 0 ? a.stats[k - 1].err : 0.0;
      const double pred = (prev > err) ? err * (err / prev) : err;
      st->emit = (a.emit_ok && (k1 >= st->max_iter || pred < 2.0 * st->tol)) ? 1 : 0;
      st->k = k1;
    }
  }

  // B: new factors (Eq. (9)), Trim (Algorithm 2), hand-over; Gram partials of A~, B~ (both
  // sides at once)
  {
    const bool do_trim = st->trim != 0;
    const int side = t / HT, tl = t % HT;
    const int rows = side ? n : m;
    const T* B = side ? Vt : Ut;
    const T* W = side ? Y2 : Y1;
    T* F = static_cast<T*>(side ? a.V : a.U);
    const T* A = sh.mat[side];
    const T cap = trim_cap<T>(a, side);
    T* sx = sh.stage[side];
    int lo, hi;
    block_range(rows, lo, hi);
    T acc[2] = {T(0), T(0)};
    for (int c0 = lo; c0 < hi; c0 += HT) {
      const int i = c0 + tl;
      T x[WM];
      zero_row<T, WM>(x);
      if (i < hi) {
        T b[WM], w[WM], f[WM];
        load_row<T, WM>(B, i, r, b);
        load_row<T, WM>(W, i, r, w);
#pragma unroll
        for (int c = 0; c < WM; ++c) {
          T sacc = T(0);
#pragma unroll
          for (int q = 0; q < WM; ++q) sacc = fma(b[q], A[q * WM + c], fma(w[q], A[(r + q) * WM + c], sacc));
          f[c] = sacc;
        }
        store_row<T, WM>(F, i, r, f);
        trim_row<T, WM>(f, cap, do_trim, x);
        hand_over_row<T, WM>(a, side, i, f, x, sh.sv[0]);
      }
      stage_row<T, WM>(sx, tl, x);
      half_sync(side);
      gram_rows_h<T, WM>(sx, sx, r, min(HT, hi - c0), tl, acc);
      half_sync(side);
    }
    gram_put_h<T>(acc, r, a.part, 6 + side, tl);
  }
}

template <typename T, int WM>
__device__ void mode_prepare(const SmallArgs& a, Smem<T, WM>& sh) {
  if (threadIdx.x < MW) sh.sv[0][threadIdx.x] = (threadIdx.x < a.r) ? static_cast<const T*>(a.sig)[threadIdx.x] : T(0);
  __syncthreads();
  trim_hand_over<T, WM>(a, sh);
}

// The orthonormal bases U~ = A~ T_u and V~ = B~ T_v of the pass that comes next, into out_ut
// (m x Rit) and out_vt (n x Rit), zero-padded.
template <typename T, int WM>
__device__ void mode_bases(const SmallArgs& a, Smem<T, WM>& sh) {
  trimmed_t_factors<T, WM>(a, sh);
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? a.n : a.m;
    const T* F = static_cast<const T*>(side ? a.Vtc : a.Utc);
    T* O = static_cast<T*>(side ? a.out_vt : a.out_ut);
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + threadIdx.x; i < hi; i += ST) {
      T f[WM], b[WM];
      load_row<T, WM>(F, i, a.Rit, f);
      row_times<T, WM>(f, sh.tm[side], b);
      store_copy<T, WM>(O, i, a.Rit, b);
    }
  }
}

__device__ float gauss(unsigned long long seed, unsigned long long i) {
  auto mix = [](unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  };
  const unsigned long long a = mix(seed * 0x632be59bd9b4e019ull + 2 * i);
  const unsigned long long b = mix(seed * 0x632be59bd9b4e019ull + 2 * i + 1);
  const float u1 = ((a >> 40) + 1) * (1.0f / 16777217.0f);
  const float u2 = (b >> 40) * (1.0f / 16777216.0f);
  return sqrtf(-2.0f * logf(u1)) * cosf(6.2831853f * u2);
}

// Y1 <- Y1 T1, Y2 <- Y2 T2 on the own rows (T factors in sh.tm) and the Gram matrices of
// the results into slots s1, s1 + 1: the first pass of CholeskyQR2.
template <typename T, int WM>
__device__ void orth_first_pass(const SmallArgs& a, int w, int s1, Smem<T, WM>& sh) {
  const int t = threadIdx.x;
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? a.n : a.m;
    T* Y = static_cast<T*>(side ? a.Y2 : a.Y1);
    int lo, hi;
    block_range(rows, lo, hi);
    T acc = T(0);
    for (int c0 = lo; c0 < hi; c0 += ST) {
      const int i = c0 + t;
      T q[WM];
      zero_row<T, WM>(q);
      if (i < hi) {
        T y[WM];
        load_row<T, WM>(Y, i, w, y);
        row_times<T, WM>(y, sh.tm[side], q);
        store_row<T, WM>(Y, i, w, q);
      }
      stage_row<T, WM>(sh.stage[0], t, q);
      __syncthreads();
      acc = gram_acc<T, WM>(sh.stage[0], w, sh.stage[0], w, min(ST, hi - c0), acc);
      __syncthreads();
    }
    gram_store(acc, w * w, a.part, s1 + side, sh);
  }
}

// After a barrier: the second CholeskyQR pass from slots s1, s1 + 1, the new bases U~, V~
// (width w) and their pass copies (width Rc; W = V = 0 for the initialisation passes).
template <typename T, int WM>
__device__ void orth_second_pass(const SmallArgs& a, int w, int s1, Smem<T, WM>& sh) {
  const int t = threadIdx.x, Rc = a.Rc;
  reduce_slots(a.part, s1, 2, w * w, &sh.G[0][0], sh);
  factor_pair<T, WM>(w, 0, 1, sh);
  {
    const int side = t / HT, tl = t % HT;
    const int rows = side ? a.n : a.m;
    const T* Y = static_cast<const T*>(side ? a.Y2 : a.Y1);
    T* B = static_cast<T*>(side ? a.Vt : a.Ut);
    T* d0 = static_cast<T*>(side ? a.Vtc : a.Utc);
    T* d1 = static_cast<T*>(side ? a.Vc : a.Wc);
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + tl; i < hi; i += HT) {
      T y[WM], q[WM], z[WM];
      load_row<T, WM>(Y, i, w, y);
      row_times<T, WM>(y, sh.tm[side], q);
      store_row<T, WM>(B, i, w, q);
      zero_row<T, WM>(z);
      store_copy<T, WM>(d0, i, Rc, q);
      store_copy<T, WM>(d1, i, Rc, z);
      if constexpr (sizeof(T) == 4) {
        if (a.img_init) write_images<T, WM>(a, 0, side, i, z, q);
      }
    }
  }
}

template <typename T, int WM>
__device__ void mode_rand(const SmallArgs& a, Smem<T, WM>& sh) {
  const int w = a.b, t = threadIdx.x;
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? a.n : a.m;
    T* Y = static_cast<T*>(side ? a.Y2 : a.Y1);
    const unsigned long long seed = side ? (a.seed ^ 0x5bd1e995ull) : a.seed;
    int lo, hi;
    block_range(rows, lo, hi);
    T acc = T(0);
    for (int c0 = lo; c0 < hi; c0 += ST) {
      const int i = c0 + t;
      T y[WM];
#pragma unroll
      for (int j = 0; j < WM; ++j) y[j] = (i < hi && j < w) ? (T)gauss(seed, (unsigned long long)i * w + j) : T(0);
      if (i < hi) store_row<T, WM>(Y, i, w, y);
      stage_row<T, WM>(sh.stage[0], t, y);
      __syncthreads();
      acc = gram_acc<T, WM>(sh.stage[0], w, sh.stage[0], w, min(ST, hi - c0), acc);
      __syncthreads();
    }
    gram_store(acc, w * w, a.part, 1 + side, sh);
  }
  if (!grid_barrier(a.st, sh)) return;
  reduce_slots(a.part, 1, 2, w * w, &sh.G[0][0], sh);
  factor_pair<T, WM>(w, 0, 1, sh);
  orth_first_pass<T, WM>(a, w, 3, sh);
  if (!grid_barrier(a.st, sh)) return;
  orth_second_pass<T, WM>(a, w, 3, sh);
}

template <typename T, int WM>
__device__ void mode_rr(const SmallArgs& a, Smem<T, WM>& sh) {
  constexpr int NM = Smem<T, WM>::NM;
  DevState* st = a.st;
  const int m = a.m, n = a.n, w = a.b, r = a.r, t = threadIdx.x;
  const T* Ut = static_cast<const T*>(a.Ut);
  const T* Vt = static_cast<const T*>(a.Vt);
  T* Y1 = static_cast<T*>(a.Y1);
  T* Y2 = static_cast<T*>(a.Y2);
  // phase and step of the initialisation live on the device, so the host can queue steps
  // without waiting for each one (read here, before block 0 updates them at the end)
  const int phase = st->init_phase, step = st->init_step;
  const bool first = step == 0, force = step >= a.init_max - 1;
  if (blockIdx.x == 0 && t == 0) st->steps_run += 1;  // read by the host after every batch
  // the pass's totals are needed once: ||D||_F^2 from the first pass of the first phase
  // (L = 0 there); the branch is uniform over the block
  if (phase == 0 && first && blockIdx.x == 0) {
    double res2;
    unsigned long long nnz;
    cta_totals(a, res2, nnz, sh);
    if (t == 0) st->normD2 = res2;
  }

  // A: own rows of Y1 = Z V~, Y2 = Z^T U~ (both sides at once on the two half blocks);
  // partials of B = U~^T Y1 (slot 0), Y1^T Y1 (slot 1) and Y2^T Y2 (slot 2)
  {
    const int side = t / HT, tl = t % HT;
    const int rows = side ? n : m;
    T* sy = sh.stage[side];          // rows of Y1 / Y2
    T* su = sh.stage[0] + HT * WM;   // side 0: rows of U~
    int lo, hi;
    block_range(rows, lo, hi);
    T accB[2] = {T(0), T(0)}, accG[2] = {T(0), T(0)};
    for (int c0 = lo; c0 < hi; c0 += HT) {
      const int i = c0 + tl;
      T y[WM], u[WM];
      zero_row<T, WM>(y);
      zero_row<T, WM>(u);
      if (i < hi) {
        reduce_row<T, WM>(static_cast<const T*>(side ? a.P2 : a.P1),
                          side ? a.n_p2 : (a.p1_nsl ? a.p1_nsl[i >> 7] : a.n_p1),
                          (size_t)rows * (side ? a.R2 : a.R), i, side ? a.R2 : a.R, w, y);
        store_row<T, WM>(side ? Y2 : Y1, i, w, y);
        if (!side) load_row<T, WM>(Ut, i, w, u);
      }
      stage_row<T, WM>(sy, tl, y);
      if (!side) stage_row<T, WM>(su, tl, u);
      half_sync(side);
      const int nr = min(HT, hi - c0);
      if (!side) gram_rows_h<T, WM>(su, sy, w, nr, tl, accB);
      gram_rows_h<T, WM>(sy, sy, w, nr, tl, accG);
      half_sync(side);
    }
    if (!side) gram_put_h<T>(accB, w, a.part, 0, tl);
    gram_put_h<T>(accG, w, a.part, 1 + side, tl);
  }
  // while thread 0 waits: the pairing of the SVD below (warp 2)
  auto pairs = [&]() {
    if constexpr (sizeof(T) == 4) {
      if ((t >> 5) == 2) jacobi_pairs(w, sh.pairs);
    }
  };
  if (!grid_barrier(st, sh, pairs)) return;

  // B: SVD of B (warp 0) while warps 1, 2 factor Y1^T Y1 and Y2^T Y2; Ritz vectors,
  // residuals, first CholeskyQR pass of Y1, Y2
  reduce_slots(a.part, 0, 3, w * w, &sh.G[0][0], sh);  // G[0] = B, G[1], G[2] = Grams
  for (int e = t; e < NM * NM; e += ST) {
    const int row = e / NM, col = e % NM;
    sh.M[e] = (row < w && col < w) ? sh.G[0][row * w + col] : T(0);
  }
  __syncthreads();
  {
    const int warp = t >> 5;
    if (warp == 0) small_svd<T, WM>(w, sh, 12, sizeof(T) == 4);
    if (warp == 1) factor_one<T, WM>(sh.G[1], w, 0, sh);
    if (warp == 2) factor_one<T, WM>(sh.G[2], w, 1, sh);
  }
  __syncthreads();
  // mat[0] rows 0..w-1: U_B[:, :r]; mat[1]: V_B[:, :r]; tm: T1, T2
  for (int e = t; e < 2 * WM * WM; e += ST) {
    const int s = e / (WM * WM), q = (e / WM) % WM, c = e % WM;
    const T* Y = s ? sh.VM : sh.UM;
    sh.mat[s][q * WM + c] = (q < w && c < r) ? Y[c * NM + q] : T(0);
    sh.tm[s][q * WM + c] = (q < w && c < w) ? sh.Tf[s][q * w + c] : T(0);
  }
  if (t < MW) {
    const T sg = (t < r) ? sh.sig[t] : T(0);
    sh.sv[0][t] = sg;
    sh.sv[1][t] = sg > T(0) ? T(1) / sg : T(0);
  }
  __syncthreads();
  // Top Ritz triplets: u_c = U~ U_B[:, c], v_c = V~ V_B[:, c], sigma_c.  Their residuals
  // Z v_c - sigma_c u_c = Y1 V_B[:, c] - sigma_c u_c and Z^T u_c - sigma_c v_c =
  // Y2 U_B[:, c] - sigma_c v_c need no further pass over D; the sum of their squared
  // norms, each divided by sigma_c^2, decides convergence.
  const int nr = (phase == 0) ? 1 : r;
  T res = T(0);
  {
    const int side = t / HT, tl = t % HT;
    const int rows = side ? n : m;
    const T* B = side ? Vt : Ut;
    T* Y = side ? Y2 : Y1;
    T* F = static_cast<T*>(side ? a.V : a.U);
    const T* Mb = sh.mat[side];      // basis coefficients
    const T* My = sh.mat[1 - side];  // product coefficients
    T* sq = sh.stage[side];
    int lo, hi;
    block_range(rows, lo, hi);
    T acc[2] = {T(0), T(0)};
    for (int c0 = lo; c0 < hi; c0 += HT) {
      const int i = c0 + tl;
      T q[WM];
      zero_row<T, WM>(q);
      if (i < hi) {
        T b[WM], y[WM], f[WM], zy[WM];
        load_row<T, WM>(B, i, w, b);
        load_row<T, WM>(Y, i, w, y);
        row_times<T, WM>(b, Mb, f);
        row_times<T, WM>(y, My, zy);
        store_row<T, WM>(F, i, r, f);
#pragma unroll
        for (int c = 0; c < WM; ++c)
          if (c < nr) {
            const T d = fma(-sh.sv[0][c], f[c], zy[c]) * sh.sv[1][c];
            res = fma(d, d, res);
          }
        row_times<T, WM>(y, sh.tm[side], q);
        store_row<T, WM>(Y, i, w, q);
      }
      stage_row<T, WM>(sq, tl, q);
      half_sync(side);
      gram_rows_h<T, WM>(sq, sq, w, min(HT, hi - c0), tl, acc);
      half_sync(side);
    }
    gram_put_h<T>(acc, w, a.part, 3 + side, tl);
  }
  sh.red[t] = res;
  __syncthreads();
  tree_combine(1, ST, sh);
  if (t == 0) slot_ptr<T>(a.part, 5, blockIdx.x)[0] = sh.red[0];
  if (blockIdx.x == 0 && t < w) st->sigma[t] = (double)sh.sig[t];
  if (t < r) static_cast<T*>(a.sig)[t] = (T)sh.sig[t];
  if (!grid_barrier(st, sh)) return;

  // C: convergence; then either the bases for the next step or (top-r converged) Trim
  reduce_slots(a.part, 5, 1, 1, sh.scal, sh);
  const double crit = sqrt((double)sh.scal[0]);
  const double tol = (phase == 0) ? sqrt(a.init_tol) : a.init_tol;
  const int conv = (force || (!first && crit <= tol)) ? 1 : 0;
  if (blockIdx.x == 0 && t == 0) {
    if (!(crit == crit)) atomicCAS(&st->status, 0, kErrNumerical);
    st->sigma_prev[0] = crit;
    if (conv && phase == 0) {
      st->zeta = st->beta_init * (double)sh.sig[0];
      st->init_phase = 1;
      st->init_step = 0;
    } else if (conv && phase == 1) {
      // initialisation finished: the steps still queued behind this one return at once
      st->zeta = st->beta * (double)sh.sig[0];
      st->k = 0;
      st->conv = 1;
      st->done = 1;
    } else {
      st->init_step = step + 1;
    }
  }
  if (conv && phase == 1) {
    trim_hand_over<T, WM>(a, sh);
    return;
  }
  orth_second_pass<T, WM>(a, w, 3, sh);
}

// One kernel per mode: a launch then carries only the code of its own mode, which keeps its
// instruction footprint small (the serial steps run once per launch, so they mostly execute
// from a cold instruction cache).
template <typename T, int WM, int MODE>
__global__ void __launch_bounds__(ST, 1) small_kernel(SmallArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T, WM>& sh = *reinterpret_cast<Smem<T, WM>*>(smem_raw);
  if (MODE == SM_UPDATE || MODE == SM_RR) {
    if (a.st->done) return;
  }
  if (MODE == SM_UPDATE) mode_update<T, WM>(a, sh);
  if (MODE == SM_PREPARE) mode_prepare<T, WM>(a, sh);
  if (MODE == SM_RR) mode_rr<T, WM>(a, sh);
  if (MODE == SM_RAND) mode_rand<T, WM>(a, sh);
  if (MODE == SM_BASES) mode_bases<T, WM>(a, sh);
}

template <typename T, int WM, int MODE>
void set_smem_mode() {
  cudaFuncSetAttribute(small_kernel<T, WM, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(Smem<T, WM>));
}

template <typename T, int WM>
void set_smem() {
  set_smem_mode<T, WM, SM_UPDATE>();
  set_smem_mode<T, WM, SM_PREPARE>();
  set_smem_mode<T, WM, SM_RR>();
  set_smem_mode<T, WM, SM_RAND>();
  set_smem_mode<T, WM, SM_BASES>();
}

template <typename T, int WM, int MODE>
cudaError_t launch_mode(const SmallArgs& a, int grid, cudaStream_t s) {
  SmallArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)small_kernel<T, WM, MODE>, dim3(grid), dim3(ST), args,
                                     sizeof(Smem<T, WM>), s);
}

template <typename T, int WM>
cudaError_t launch_one(const SmallArgs& a, int grid, cudaStream_t s) {
  switch (a.mode) {
    case SM_UPDATE:
      return launch_mode<T, WM, SM_UPDATE>(a, grid, s);
    case SM_PREPARE:
      return launch_mode<T, WM, SM_PREPARE>(a, grid, s);
    case SM_RR:
      return launch_mode<T, WM, SM_RR>(a, grid, s);
    case SM_RAND:
      return launch_mode<T, WM, SM_RAND>(a, grid, s);
    case SM_BASES:
      return launch_mode<T, WM, SM_BASES>(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

// Self-test of the bounded waits: an mbarrier phase that nothing completes, waited for with a
// 1 ms limit, and a grid barrier that one of two blocks never reaches (1 s limit).  Both end
// with a TIMEOUT status and return; nothing else is in flight.
struct BarrierFlag {
  int ok;
};

__global__ void selftest_mbar_kernel(int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    *out = tc::mbar_wait(&bar, 0, 1000000ull) ? 0 : (int)kErrTimeout;
  }
}

__global__ void selftest_grid_kernel(DevState* st) {
  __shared__ BarrierFlag sh;
  if (blockIdx.x == 1) return;  // never arrives
  grid_barrier(st, sh);
}

}  // namespace

int small_grid_size(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  set_smem<float, 8>();
  set_smem<float, 16>();
  set_smem<double, 8>();
  set_smem<double, 16>();
  return sms;  // one block per SM keeps the barrier short
}

cudaError_t launch_small(const SmallArgs& a, int grid, cudaStream_t s) {
  const bool init = (a.mode == SM_RR || a.mode == SM_RAND);
  int need = a.r > a.Rit ? a.r : a.Rit;
  if (init) {
    need = need > a.b ? need : a.b;
    need = need > a.Rc ? need : a.Rc;
  }
  if (a.r < 1 || need > MW) return cudaErrorInvalidValue;
  const bool narrow = need <= 8;
  if (a.prec == PREC_F32) return narrow ? launch_one<float, 8>(a, grid, s) : launch_one<float, 16>(a, grid, s);
  return narrow ? launch_one<double, 8>(a, grid, s) : launch_one<double, 16>(a, grid, s);
}

cudaError_t run_wait_selftest(int* mbar_status, int* grid_status) {
  int* d_out = nullptr;
  DevState* st = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_out, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&st, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMemset(d_out, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(DevState));
  if (e == cudaSuccess) {
    selftest_mbar_kernel<<<1, 32>>>(d_out);
    selftest_grid_kernel<<<2, 32>>>(st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(mbar_status, d_out, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(grid_status, &st->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (d_out) cudaFree(d_out);
  if (st) cudaFree(st);
  return e;
}

}  // namespace rpca
