// Tall-skinny kernel of the AccAltProj iteration and of the initialisation.
//
// One cooperative launch per call (one block per SM, all co-resident).  Phases are
// separated by a bounded grid barrier.  Rows of the m x w and n x w arrays are split
// into contiguous block ranges; small matrices (w x w Gram and Cholesky factors, the
// 2r x 2r core M_k and its SVD) are computed redundantly by every block in shared memory,
// so the only cross-block traffic is the per-block Gram partials.
//
// The kernel is templated on the arithmetic of the per-row work: double in FP64 mode,
// float in FP32 mode.  GB300 runs FP64 at a small fraction of its FP32 rate, so the
// FP32 mode keeps FP64 for what needs it: the residual / support totals, the threshold,
// and the singular values of M_k (an FP32 Jacobi SVD refined in FP64: the columns of
// M_k V are formed in double and their norms taken as the singular values).
//
// Modes:
//   SM_UPDATE : after a fused pass of Algorithm 1.  Reduce the pass partials to
//               Y1 = Z V~ and Y2 = Z^T U~ and err_k (Eq. (11)); stop if err_k < tol;
//               otherwise C = U~^T Y1, QR of (I - U~U~^T) Z V~ = Y1 - U~ C and of
//               (I - V~V~^T) Z^T U~ = Y2 - V~ C^T (shifted CholeskyQR3), the 2r x 2r
//               M = [[C, R2^T], [R1, 0]] and its SVD (one-sided Jacobi), the new
//               factors by Eq. (9), zeta_{k+1} (Algorithm 1), then PREPARE.
//   SM_PREPARE: Trim (Algorithm 2) of U_k, V_k, orthonormal bases U~_k, V~_k of the
//               trimmed factors (CholeskyQR2; the footnote to Eq. (5) asks for a QR),
//               and the pass-precision copies W = U_k Sigma_k, V_k, U~_k, V~_k.
//   SM_RR     : one step of block subspace iteration for Algorithm 3 (sigma_1(D), then
//               the top-r SVD of D - S_{-1}): Rayleigh-Ritz B = U~^T (Z V~), SVD(B),
//               convergence test, new bases orth(Z V~), orth(Z^T U~).
//   SM_RAND   : random orthonormal starting bases for SM_RR.
#include <math.h>

#include "common.cuh"

namespace rpca {

namespace {

constexpr int ST = 512;     // threads per block
constexpr int MW = 16;      // max width of the tall-skinny arrays
constexpr int MN = 32;      // max order of the small SVD (2r)
constexpr int LD = MN + 1;  // leading dimension of the column-major SVD work arrays
constexpr int GSLOT = MW * MW;
constexpr int NSLOT = 4;    // Gram partial slots per block
constexpr int kErrTimeout = 6;
constexpr int kErrNumerical = 3;

template <typename T>
struct Smem {
  double red[ST];
  T G[2][GSLOT];       // reduced Gram matrices
  T Racc[2][GSLOT];    // accumulated R factors (upper)
  T Rstep[2][GSLOT];   // R factor of the current CholeskyQR pass
  T C[GSLOT];          // U~^T Y1
  T rinv[2][MW];       // reciprocals of the diagonal of Rstep
  T um[2][MN * MW];    // ordered top columns of U_M, V_M in the working precision
  T ub[MN * MW];       // Rayleigh-Ritz: U_B, V_B top columns, sigma, 1/sigma
  T vb[MN * MW];
  T sgs[MW];
  T invs[MW];
  double A[MN * LD];   // SVD: the matrix, then its rotated columns (U Sigma), column-major
  double Vm[MN * LD];  // SVD: right singular vectors
  float Af[MN * LD];   // FP32 Jacobi work
  float Vf[MN * LD];
  double UMs[MN * LD];  // scratch / ordered top columns of U_M, V_M in double
  double VMs[MN * MW];
  double sig[MN];
  int order[MN];
  int flag;
  int ok;
  double scal[8];
};

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait.  Returns false (and leaves a TIMEOUT status) if
// another block failed to arrive within one second, so no block can spin forever.
template <typename T>
__device__ bool grid_barrier(DevState* st, Smem<T>& sh) {
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

__device__ void block_range(int rows, int& lo, int& hi) {
  const int chunk = (rows + gridDim.x - 1) / gridDim.x;
  lo = min(rows, (int)blockIdx.x * chunk);
  hi = min(rows, lo + chunk);
}

// This block's part of X^T Y over its rows (X: rows x wx, Y: rows x wy, row-major with
// leading dimensions ldx, ldy) into part[blockIdx][slot][wx*wy].
template <typename T>
__device__ void gram_partial(const T* X, int ldx, int wx, const T* Y, int ldy, int wy, int rows, T* part, int slot,
                             Smem<T>& sh) {
  int lo, hi;
  block_range(rows, lo, hi);
  const int P = wx * wy;
  const int t = threadIdx.x;
  T* out = part + ((size_t)blockIdx.x * NSLOT + slot) * GSLOT;
  const int nl = ST / P;  // P <= 256
  const int p = t % P, l = t / P;
  T acc = T(0);
  if (l < nl) {
    const int a = p / wy, b = p % wy;
    for (int i = lo + l; i < hi; i += nl) acc = fma(X[(size_t)i * ldx + a], Y[(size_t)i * ldy + b], acc);
  }
  sh.red[t] = (double)acc;
  __syncthreads();
  if (t < P) {
    T s = T(0);
    for (int q = 0; q < nl; ++q) s += (T)sh.red[t + q * P];
    out[t] = s;
  }
  __syncthreads();
}

// Fixed-order sum over blocks of a partial slot into shared G (P <= 256).  Threads are
// split into (pair, block-chunk) groups with eight independent loads in flight.
template <typename T>
__device__ void gram_reduce(const T* part, int slot, int P, T* G, Smem<T>& sh) {
  const int t = threadIdx.x, nb = gridDim.x;
  const int nch = ST / P;
  const int p = t % P, c = t / P;
  T s = T(0);
  if (c < nch) {
    int b = c;
    for (; b + 7 * nch < nb; b += 8 * nch) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = part[((size_t)(b + u * nch) * NSLOT + slot) * GSLOT + p];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; b < nb; b += nch) s += part[((size_t)b * NSLOT + slot) * GSLOT + p];
  }
  sh.red[t] = (double)s;
  __syncthreads();
  if (t < P) {
    T acc = T(0);
    for (int q = 0; q < nch; ++q) acc += (T)sh.red[t + q * P];
    G[t] = acc;
  }
  __syncthreads();
}

// Upper Cholesky factor R (R^T R = G + shift I) of a w x w symmetric matrix, by one warp.
// A pivot that is not positive (rank deficiency) gives a zero row of R.
template <typename T>
__device__ void cholesky_warp(const T* G, int w, T shift, T* R) {
  const int l = threadIdx.x & 31;
  for (int j = 0; j < w; ++j)
    if (l < w) R[j * w + l] = (l >= j) ? G[j * w + l] + ((l == j) ? shift : T(0)) : T(0);
  __syncwarp();
  T scale = T(0);
  for (int j = 0; j < w; ++j) scale = fmax(scale, fabs(G[j * w + j]) + shift);
  const T tiny = sizeof(T) == 8 ? T(1e-30) : T(1e-12);
  for (int j = 0; j < w; ++j) {
    const T d = R[j * w + j];
    const bool good = d > T(0) && d > tiny * scale;
    const T rjj = good ? sqrt(d) : T(0);
    const T inv = good ? T(1) / rjj : T(0);
    __syncwarp();
    if (l >= j && l < w) R[j * w + l] = good ? ((l == j) ? rjj : R[j * w + l] * inv) : T(0);
    __syncwarp();
    if (l > j && l < w)
      for (int k = j + 1; k <= l; ++k) R[k * w + l] -= R[j * w + k] * R[j * w + l];
    __syncwarp();
  }
}

// Both sides at once: warp 0 factors G1, warp 1 factors G2 (if given).
template <typename T>
__device__ void cholesky_pair(const T* G1, int w1, T s1, T* R1, const T* G2, int w2, T s2, T* R2) {
  const int warp = threadIdx.x >> 5;
  if (warp == 0) cholesky_warp(G1, w1, s1, R1);
  if (warp == 1 && G2) cholesky_warp(G2, w2, s2, R2);
  __syncthreads();
}

// y (1 x w) <- y R^{-1} for upper R given the reciprocals of its diagonal (0 where the
// diagonal is 0, which gives a zero entry).
template <typename T>
__device__ __forceinline__ void trsv_row(T* y, const T* R, const T* rinv, int w) {
  for (int j = 0; j < w; ++j) {
    T s = y[j];
    for (int k = 0; k < j; ++k) s -= y[k] * R[k * w + j];
    y[j] = s * rinv[j];
  }
}

// Racc <- Rstep * Racc (both upper w x w), by the block.
template <typename T>
__device__ void upper_mul_acc(T* Racc, const T* Rstep, int w) {
  const int t = threadIdx.x;
  T v = T(0);
  if (t < w * w) {
    const int i = t / w, j = t % w;
    for (int k = i; k <= j; ++k) v += Rstep[i * w + k] * Racc[k * w + j];
  }
  __syncthreads();
  if (t < w * w) Racc[t] = v;
  __syncthreads();
}

// In-place QR of X1 (rows1 x w1) and X2 (rows2 x w2, may be null) by CholeskyQR, `passes`
// passes, the first with the shift of shifted CholeskyQR (Fukaya et al. 2020) when
// `shifted`.  Leaves the R factors in sh.Racc[0], sh.Racc[1].  When `first_reduced` the
// Gram matrices of the first pass are already in sh.G.  Returns false on a barrier
// failure.  `copy1`/`copy2` (may be null) receive a copy of the final Q.
template <typename T>
__device__ bool cholqr(T* X1, int rows1, int w1, T* X2, int rows2, int w2, int passes, bool shifted, T* part,
                       DevState* st, Smem<T>& sh, T* copy1, T* copy2, bool first_reduced = false) {
  const int t = threadIdx.x;
  for (int e = t; e < GSLOT; e += ST) {
    sh.Racc[0][e] = ((e / w1) == (e % w1) && e < w1 * w1) ? T(1) : T(0);
    sh.Racc[1][e] = (X2 && (e / w2) == (e % w2) && e < w2 * w2) ? T(1) : T(0);
  }
  if (!first_reduced) {
    gram_partial((const T*)X1, w1, w1, (const T*)X1, w1, w1, rows1, part, 0, sh);
    if (X2) gram_partial((const T*)X2, w2, w2, (const T*)X2, w2, w2, rows2, part, 1, sh);
  }
  __syncthreads();
  for (int ps = 0; ps < passes; ++ps) {
    if (!(first_reduced && ps == 0)) {
      if (!grid_barrier(st, sh)) return false;
      gram_reduce((const T*)part, 0, w1 * w1, sh.G[0], sh);
      if (X2) gram_reduce((const T*)part, 1, w2 * w2, sh.G[1], sh);
    }
    T sh1 = T(0), sh2 = T(0);
    if (shifted && ps == 0) {
      const T u = sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08);
      T tr1 = T(0), tr2 = T(0);
      for (int j = 0; j < w1; ++j) tr1 += sh.G[0][j * w1 + j];
      for (int j = 0; X2 && j < w2; ++j) tr2 += sh.G[1][j * w2 + j];
      sh1 = T(11) * (T(rows1) * w1 + T(w1) * (w1 + 1)) * u * tr1;
      sh2 = T(11) * (T(rows2) * w2 + T(w2) * (w2 + 1)) * u * tr2;
    }
    cholesky_pair(sh.G[0], w1, sh1, sh.Rstep[0], X2 ? sh.G[1] : nullptr, w2, sh2, sh.Rstep[1]);
    if (t < w1) sh.rinv[0][t] = sh.Rstep[0][t * w1 + t] != T(0) ? T(1) / sh.Rstep[0][t * w1 + t] : T(0);
    if (X2 && t >= 32 && t - 32 < w2) {
      const int j = t - 32;
      sh.rinv[1][j] = sh.Rstep[1][j * w2 + j] != T(0) ? T(1) / sh.Rstep[1][j * w2 + j] : T(0);
    }
    upper_mul_acc(sh.Racc[0], sh.Rstep[0], w1);
    if (X2) upper_mul_acc(sh.Racc[1], sh.Rstep[1], w2);
    const bool last = (ps == passes - 1);
    for (int side = 0; side < (X2 ? 2 : 1); ++side) {
      T* X = side ? X2 : X1;
      const int rows = side ? rows2 : rows1, w = side ? w2 : w1;
      T* cp = side ? copy2 : copy1;
      int lo, hi;
      block_range(rows, lo, hi);
      for (int i = lo + t; i < hi; i += ST) {
        T y[MW];
        for (int j = 0; j < w; ++j) y[j] = X[(size_t)i * w + j];
        trsv_row(y, sh.Rstep[side], sh.rinv[side], w);
        for (int j = 0; j < w; ++j) X[(size_t)i * w + j] = y[j];
        if (last && cp)
          for (int j = 0; j < w; ++j) cp[(size_t)i * w + j] = y[j];
      }
    }
    __syncthreads();
    if (!last) {
      gram_partial((const T*)X1, w1, w1, (const T*)X1, w1, w1, rows1, part, 0, sh);
      if (X2) gram_partial((const T*)X2, w2, w2, (const T*)X2, w2, w2, rows2, part, 1, sh);
    }
  }
  return true;
}

// One-sided Jacobi on the N x N column-major matrix X (leading dimension LD), with the
// right rotations accumulated in Vr (set to I here); N even, N <= 32; the warps that own
// a rotation pair synchronise on a named barrier.  The rotation angle is computed in
// single precision; c and s follow from it in the working precision, so each rotation is
// orthogonal to working precision.
template <typename U>
__device__ void jacobi_sweeps(int N, U* X, U* Vr, U tol2, int max_sweeps, int* flag) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int e = t; e < N * N; e += ST) {
    const int c = e / N, rw = e % N;
    Vr[c * LD + rw] = (c == rw) ? U(1) : U(0);
  }
  __syncthreads();
  const int half = N / 2;
  if (warp < half) {
    const int nthr = half * 32;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
      if (t == 0) *flag = 0;
      asm volatile("bar.sync 1, %0;" ::"r"(nthr));
      for (int round = 0; round < N - 1; ++round) {
        // round-robin pairing: position 0 fixed, positions 1..N-1 rotated by `round`
        int p = (warp == 0) ? 0 : 1 + (warp - 1 + round) % (N - 1);
        int q = 1 + (N - 2 - warp + round) % (N - 1);
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        const U ap = (lane < N) ? X[p * LD + lane] : U(0);
        const U aq = (lane < N) ? X[q * LD + lane] : U(0);
        const U alpha = wsum(ap * ap), beta = wsum(aq * aq), gam = wsum(ap * aq);
        if (gam != U(0) && gam * gam > tol2 * alpha * beta) {
          const float zf = (float)((beta - alpha) / (U(2) * gam));
          const float tf = (zf >= 0.f ? 1.f : -1.f) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.f)));
          const U tt = (U)tf;
          const U c = U(1) / sqrt(tt * tt + U(1)), s = c * tt;
          if (lane < N) {
            X[p * LD + lane] = c * ap - s * aq;
            X[q * LD + lane] = s * ap + c * aq;
            const U vp = Vr[p * LD + lane], vq = Vr[q * LD + lane];
            Vr[p * LD + lane] = c * vp - s * vq;
            Vr[q * LD + lane] = s * vp + c * vq;
          }
          if (lane == 0) *flag = 1;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nthr));
      }
      const int f = *flag;
      asm volatile("bar.sync 1, %0;" ::"r"(nthr));
      if (!f) break;
    }
  }
  __syncthreads();
}

// SVD of the N x N matrix held column-major (double) in sh.A.  On return sh.sig holds the
// singular values, sh.order their descending order, sh.A the columns M V (= U Sigma) and
// sh.Vm the right singular vectors, all in double.
template <typename T>
__device__ void small_svd(int N, Smem<T>& sh) {
  const int t = threadIdx.x;
  if (sizeof(T) == 8) {
    jacobi_sweeps<double>(N, sh.A, sh.Vm, 1e-30, 40, &sh.flag);
  } else {
    // FP32 Jacobi, then the columns M V are formed in double and their norms taken as
    // the singular values (exact up to the square of the FP32 orthogonality error).
    for (int e = t; e < N * N; e += ST) {
      const int c = e / N, rw = e % N;
      sh.Af[c * LD + rw] = (float)sh.A[c * LD + rw];
    }
    __syncthreads();
    jacobi_sweeps<float>(N, sh.Af, sh.Vf, 1e-13f, 30, &sh.flag);
    for (int e = t; e < N * N; e += ST) {
      const int c = e / N, rw = e % N;
      double s = 0.0;
      for (int q = 0; q < N; ++q) s += sh.A[q * LD + rw] * (double)sh.Vf[c * LD + q];
      sh.UMs[c * LD + rw] = s;  // scratch: column c of M V
    }
    __syncthreads();
    for (int e = t; e < N * N; e += ST) {
      const int c = e / N, rw = e % N;
      sh.A[c * LD + rw] = sh.UMs[c * LD + rw];
      sh.Vm[c * LD + rw] = (double)sh.Vf[c * LD + rw];
    }
    __syncthreads();
  }
  if (t < N) {
    double s = 0.0;
    for (int rw = 0; rw < N; ++rw) s += sh.A[t * LD + rw] * sh.A[t * LD + rw];
    sh.sig[t] = sqrt(s);
  }
  __syncthreads();
  if (t == 0) {
    for (int i = 0; i < N; ++i) sh.order[i] = i;
    for (int i = 1; i < N; ++i) {  // insertion sort, descending, stable
      const int x = sh.order[i];
      int j = i - 1;
      while (j >= 0 && sh.sig[sh.order[j]] < sh.sig[x]) {
        sh.order[j + 1] = sh.order[j];
        --j;
      }
      sh.order[j + 1] = x;
    }
  }
  __syncthreads();
}

// Trim (Algorithm 2) + orthonormal bases + pass-precision copies, from the master
// factors U (m x r), sig, V (n x r).
template <typename T>
__device__ bool prepare(const SmallArgs& a, Smem<T>& sh) {
  const int m = a.m, n = a.n, r = a.r, t = threadIdx.x;
  T* U = static_cast<T*>(a.U);
  T* V = static_cast<T*>(a.V);
  T* Ut = static_cast<T*>(a.Ut);
  T* Vt = static_cast<T*>(a.Vt);
  const T* sig = static_cast<const T*>(a.sig);
  T* part = static_cast<T*>(a.part);
  const double mu = a.st->mu_trim;
  const T cu = (T)sqrt(mu * r / m), cv = (T)sqrt(mu * r / n);
  int scaled = 0;
  for (int side = 0; side < 2; ++side) {
    const T* F = side ? V : U;
    T* Tt = side ? Vt : Ut;
    const int rows = side ? n : m;
    const T cap = side ? cv : cu;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      T nrm = T(0);
      for (int j = 0; j < r; ++j) nrm += F[(size_t)i * r + j] * F[(size_t)i * r + j];
      nrm = sqrt(nrm);
      const bool cut = a.st->trim && nrm > cap;
      scaled += cut ? 1 : 0;
      const T sc = cut ? cap / nrm : T(1);
      for (int j = 0; j < r; ++j) Tt[(size_t)i * r + j] = sc * F[(size_t)i * r + j];
    }
  }
  __syncthreads();
  if (a.st->trim) {
    // Orthonormal bases of the trimmed factors by CholeskyQR2.  When no row was scaled the
    // trimmed factors are U_k, V_k themselves and the QR is skipped.
    gram_partial((const T*)Ut, r, r, (const T*)Ut, r, r, m, part, 0, sh);
    gram_partial((const T*)Vt, r, r, (const T*)Vt, r, r, n, part, 1, sh);
    sh.red[t] = (double)scaled;
    __syncthreads();
    for (int h = ST / 2; h > 0; h >>= 1) {
      if (t < h) sh.red[t] += sh.red[t + h];
      __syncthreads();
    }
    if (t == 0) part[((size_t)blockIdx.x * NSLOT + 3) * GSLOT] = (T)sh.red[0];
    if (!grid_barrier(a.st, sh)) return false;
    double tot = 0.0;
    for (int b = t; b < (int)gridDim.x; b += ST) tot += (double)part[((size_t)b * NSLOT + 3) * GSLOT];
    __syncthreads();
    sh.red[t] = tot;
    __syncthreads();
    for (int h = ST / 2; h > 0; h >>= 1) {
      if (t < h) sh.red[t] += sh.red[t + h];
      __syncthreads();
    }
    const double any = sh.red[0];
    __syncthreads();
    if (any > 0.0) {
      gram_reduce((const T*)part, 0, r * r, sh.G[0], sh);
      gram_reduce((const T*)part, 1, r * r, sh.G[1], sh);
      if (!cholqr(Ut, m, r, Vt, n, r, 2, false, part, a.st, sh, (T*)nullptr, (T*)nullptr, true)) return false;
    }
  }
  // pass-precision copies, zero-padded to the compiled width of the iteration's pass
  const int Rc = a.Rit;
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    int lo, hi;
    block_range(rows, lo, hi);
    T* dst0 = static_cast<T*>(side ? a.Vc : a.Wc);
    T* dst1 = static_cast<T*>(side ? a.Vtc : a.Utc);
    const T* F = side ? V : U;
    const T* Tt = side ? Vt : Ut;
    for (int i = lo + t; i < hi; i += ST)
      for (int j = 0; j < Rc; ++j) {
        const size_t o = (size_t)i * Rc + j;
        dst0[o] = j < r ? (side ? F[(size_t)i * r + j] : F[(size_t)i * r + j] * sig[j]) : T(0);
        dst1[o] = j < r ? Tt[(size_t)i * r + j] : T(0);
      }
  }
  return true;
}

// Y1 (m x w), Y2 (n x w) <- fixed-order sums of the pass partials (width R), each block
// taking its own rows (block_range) so it can use them without a grid barrier.
template <typename T>
__device__ void reduce_side(const T* __restrict__ Pp, int nsl, int rows, int R, int w, T* __restrict__ Y) {
  int lo, hi;
  block_range(rows, lo, hi);
  const size_t stride = (size_t)rows * R;
  for (int e = threadIdx.x; e < (hi - lo) * w; e += ST) {
    const int i = lo + e / w, c = e % w;
    const T* p = Pp + (size_t)i * R + c;
    T s = T(0);
#pragma unroll 8
    for (int q = 0; q < nsl; ++q) s += p[q * stride];
    Y[(size_t)i * w + c] = s;
  }
}

template <typename T>
__device__ void reduce_partials(const SmallArgs& a, int w) {
  reduce_side(static_cast<const T*>(a.P1), a.n_p1, a.m, a.R, w, static_cast<T*>(a.Y1));
  reduce_side(static_cast<const T*>(a.P2), a.n_p2, a.n, a.R, w, static_cast<T*>(a.Y2));
  __syncthreads();
}

template <typename T>
__device__ void cta_totals(const SmallArgs& a, double& res2, unsigned long long& nnz, Smem<T>& sh) {
  // every block sums the per-CTA totals with the same fixed-shape tree
  const int t = threadIdx.x;
  double s = 0.0;
  unsigned long long z = 0;
  for (int c = t; c < a.n_cta; c += ST) {
    s += a.resP[c];
    z += a.nnzP[c];
  }
  sh.red[t] = s;
  __syncthreads();
  for (int h = ST / 2; h > 0; h >>= 1) {
    if (t < h) sh.red[t] += sh.red[t + h];
    __syncthreads();
  }
  res2 = sh.red[0];
  __syncthreads();
  sh.red[t] = __longlong_as_double((long long)z);
  __syncthreads();
  for (int h = ST / 2; h > 0; h >>= 1) {
    if (t < h)
      sh.red[t] = __longlong_as_double(__double_as_longlong(sh.red[t]) + __double_as_longlong(sh.red[t + h]));
    __syncthreads();
  }
  nnz = (unsigned long long)__double_as_longlong(sh.red[0]);
  __syncthreads();
}

template <typename T>
__device__ void mode_update(const SmallArgs& a, Smem<T>& sh) {
  DevState* st = a.st;
  const int m = a.m, n = a.n, r = a.r, t = threadIdx.x;
  T* U = static_cast<T*>(a.U);
  T* V = static_cast<T*>(a.V);
  T* Ut = static_cast<T*>(a.Ut);
  T* Vt = static_cast<T*>(a.Vt);
  T* Y1 = static_cast<T*>(a.Y1);
  T* Y2 = static_cast<T*>(a.Y2);
  T* part = static_cast<T*>(a.part);
  double res2;
  unsigned long long nnz;
  cta_totals(a, res2, nnz, sh);
  const double err = sqrt(res2 / st->normD2);
  const int k = st->k;
  if (blockIdx.x == 0 && t == 0) {
    DevStats& s = a.stats[k];
    s.err = err;
    s.zeta = st->zeta;
    s.res2 = res2;
    s.nnz = (long long)nnz;
    s.k = k;
    s.sigma1 = 0.0;
    s.sigma_r1 = 0.0;
  }
  if (!(err == err) || isinf(err)) {
    if (blockIdx.x == 0 && t == 0) {
      atomicCAS(&st->status, 0, kErrNumerical);
      st->done = 1;
    }
    return;
  }
  if (err < st->tol || k >= st->max_iter) {
    if (blockIdx.x == 0 && t == 0) st->done = 1;
    return;
  }
  reduce_partials<T>(a, r);  // this block's rows of Y1, Y2
  // C = U~^T Y1
  gram_partial((const T*)Ut, r, r, (const T*)Y1, r, r, m, part, 2, sh);
  if (!grid_barrier(st, sh)) return;
  gram_reduce((const T*)part, 2, r * r, sh.C, sh);
  // Y1 <- Y1 - U~ C ; Y2 <- Y2 - V~ C^T
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    T* Y = side ? Y2 : Y1;
    const T* B = side ? Vt : Ut;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      T bq[MW], y[MW];
      for (int q = 0; q < r; ++q) {
        bq[q] = B[(size_t)i * r + q];
        y[q] = Y[(size_t)i * r + q];
      }
      for (int c = 0; c < r; ++c) {
        T s = y[c];
        for (int q = 0; q < r; ++q) s -= bq[q] * (side ? sh.C[c * r + q] : sh.C[q * r + c]);
        Y[(size_t)i * r + c] = s;
      }
    }
  }
  __syncthreads();
  if (!cholqr(Y1, m, r, Y2, n, r, 3, true, part, st, sh, (T*)nullptr, (T*)nullptr)) return;
  // M = [[C, R2^T], [R1, 0]], column-major in sh.A (double)
  const int N = 2 * r;
  for (int e = t; e < N * N; e += ST) {
    const int row = e / N, col = e % N;
    T v = T(0);
    if (row < r && col < r)
      v = sh.C[row * r + col];
    else if (row < r && col >= r)
      v = sh.Racc[1][(col - r) * r + row];  // R2^T
    else if (row >= r && col < r)
      v = sh.Racc[0][(row - r) * r + col];  // R1
    sh.A[col * LD + row] = (double)v;
  }
  __syncthreads();
  small_svd(N, sh);
  const double s1 = sh.sig[sh.order[0]];
  const double sr1 = sh.sig[sh.order[r]];
  // new factors by Eq. (9): U <- [U~ Q1] U_M[:, :r], V <- [V~ Q2] V_M[:, :r]; the needed
  // columns of U_M and V_M (ordered by singular value) go to shared memory first
  for (int e = t; e < N * r; e += ST) {
    const int q = e / r, c = e % r, oc = sh.order[c];
    const double sg = sh.sig[oc];
    sh.um[0][e] = (T)(sg > 0.0 ? sh.A[oc * LD + q] / sg : 0.0);
    sh.um[1][e] = (T)sh.Vm[oc * LD + q];
  }
  __syncthreads();
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    const T* B = side ? Vt : Ut;
    const T* Q = side ? Y2 : Y1;
    T* F = side ? V : U;
    const T* MM = sh.um[side];
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      T bq[MW], qq[MW];
      for (int q = 0; q < r; ++q) {
        bq[q] = B[(size_t)i * r + q];
        qq[q] = Q[(size_t)i * r + q];
      }
      for (int c = 0; c < r; ++c) {
        T s = T(0);
        for (int q = 0; q < r; ++q) s += bq[q] * MM[q * r + c] + qq[q] * MM[(r + q) * r + c];
        F[(size_t)i * r + c] = s;
      }
    }
  }
  if (t < r) static_cast<T*>(a.sig)[t] = (T)sh.sig[sh.order[t]];
  __syncthreads();
  if (blockIdx.x == 0 && t == 0) {
    const int k1 = k + 1;
    double g = 1.0;  // gamma^(k+1) by repeated multiplication (k is small)
    for (int i = 0; i < k1; ++i) g *= st->gamma;
    if (st->zeta_mode == 0)
      st->zeta = st->beta * (sr1 + g * s1);
    else if (st->zeta_mode == 1)
      st->zeta = st->beta * g * s1;
    for (int i = 0; i < N; ++i) st->sigma[i] = sh.sig[sh.order[i]];
    a.stats[k].sigma1 = s1;
    a.stats[k].sigma_r1 = sr1;
    st->k = k1;
  }
  prepare(a, sh);
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

template <typename T>
__device__ void write_basis_copies(const SmallArgs& a, int w) {
  // U~, V~ (width w) -> pass copies of width Rc; W = 0, V = 0 (init passes use L = 0)
  const int t = threadIdx.x, Rc = a.Rc;
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? a.n : a.m;
    const T* B = static_cast<const T*>(side ? a.Vt : a.Ut);
    T* d0 = static_cast<T*>(side ? a.Vtc : a.Utc);
    T* d1 = static_cast<T*>(side ? a.Vc : a.Wc);
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST)
      for (int j = 0; j < Rc; ++j) {
        const size_t o = (size_t)i * Rc + j;
        d0[o] = j < w ? B[(size_t)i * w + j] : T(0);
        d1[o] = T(0);
      }
  }
}

template <typename T>
__device__ void mode_rand(const SmallArgs& a, Smem<T>& sh) {
  const int w = a.b;
  T* Y1 = static_cast<T*>(a.Y1);
  T* Y2 = static_cast<T*>(a.Y2);
  const size_t gt = (size_t)blockIdx.x * ST + threadIdx.x, gs = (size_t)gridDim.x * ST;
  for (size_t e = gt; e < (size_t)a.m * w; e += gs) Y1[e] = (T)gauss(a.seed, e);
  for (size_t e = gt; e < (size_t)a.n * w; e += gs) Y2[e] = (T)gauss(a.seed ^ 0x5bd1e995ull, e);
  if (!grid_barrier(a.st, sh)) return;
  if (!cholqr(Y1, a.m, w, Y2, a.n, w, 3, true, static_cast<T*>(a.part), a.st, sh, static_cast<T*>(a.Ut),
              static_cast<T*>(a.Vt)))
    return;
  write_basis_copies<T>(a, w);
}

template <typename T>
__device__ void mode_rr(const SmallArgs& a, Smem<T>& sh) {
  DevState* st = a.st;
  const int m = a.m, n = a.n, w = a.b, r = a.r, t = threadIdx.x;
  T* Ut = static_cast<T*>(a.Ut);
  T* Vt = static_cast<T*>(a.Vt);
  T* Y1 = static_cast<T*>(a.Y1);
  T* Y2 = static_cast<T*>(a.Y2);
  T* part = static_cast<T*>(a.part);
  double res2;
  unsigned long long nnz;
  cta_totals(a, res2, nnz, sh);
  if (a.init_phase == 0 && a.rr_first && blockIdx.x == 0 && t == 0) st->normD2 = res2;
  reduce_partials<T>(a, w);  // this block's rows of Y1, Y2
  gram_partial((const T*)Ut, w, w, (const T*)Y1, w, w, m, part, 2, sh);  // B = U~^T (Z V~)
  if (!grid_barrier(st, sh)) return;
  gram_reduce((const T*)part, 2, w * w, sh.C, sh);
  for (int e = t; e < w * w; e += ST) {
    const int row = e / w, col = e % w;
    sh.A[col * LD + row] = (double)sh.C[row * w + col];
  }
  __syncthreads();
  small_svd(w, sh);
  // Top Ritz triplets: u_c = U~ U_B[:, c], v_c = V~ V_B[:, c], sigma_c.  Their residuals
  // Z v_c - sigma_c u_c = Y1 V_B[:, c] - sigma_c u_c and Z^T u_c - sigma_c v_c =
  // Y2 U_B[:, c] - sigma_c v_c need no further pass over D; the sum of their squared
  // norms, each divided by sigma_c^2, decides convergence.
  for (int e = t; e < w * r; e += ST) {
    const int q = e / r, c = e % r, oc = sh.order[c];
    const double sg = sh.sig[oc];
    sh.ub[e] = (T)(sg > 0.0 ? sh.A[oc * LD + q] / sg : 0.0);
    sh.vb[e] = (T)sh.Vm[oc * LD + q];
    if (q == 0) {
      sh.sgs[c] = (T)sg;
      sh.invs[c] = (T)(sg > 0.0 ? 1.0 / sg : 0.0);
    }
  }
  __syncthreads();
  const int nr = (a.init_phase == 0) ? 1 : r;
  T acc = T(0);
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    const T* B = side ? Vt : Ut;
    const T* Y = side ? Y2 : Y1;
    T* F = static_cast<T*>(side ? a.V : a.U);
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      for (int c = 0; c < r; ++c) {
        T f = T(0), zy = T(0);
        for (int q = 0; q < w; ++q) {
          f += B[(size_t)i * w + q] * (side ? sh.vb[q * r + c] : sh.ub[q * r + c]);
          zy += Y[(size_t)i * w + q] * (side ? sh.ub[q * r + c] : sh.vb[q * r + c]);
        }
        F[(size_t)i * r + c] = f;
        if (c < nr) {
          const T d = (zy - sh.sgs[c] * f) * sh.invs[c];
          acc += d * d;
        }
      }
    }
  }
  sh.red[t] = (double)acc;
  __syncthreads();
  for (int h = ST / 2; h > 0; h >>= 1) {
    if (t < h) sh.red[t] += sh.red[t + h];
    __syncthreads();
  }
  if (t == 0) part[((size_t)blockIdx.x * NSLOT + 3) * GSLOT] = (T)sh.red[0];
  if (t < r) static_cast<T*>(a.sig)[t] = (T)sh.sig[sh.order[t]];
  if (!grid_barrier(st, sh)) return;
  if (t == 0) {
    double tot = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) tot += (double)part[((size_t)b * NSLOT + 3) * GSLOT];
    const double crit = sqrt(tot);
    if (!(crit == crit) && blockIdx.x == 0) atomicCAS(&st->status, 0, kErrNumerical);
    const double tol = (a.init_phase == 0) ? sqrt(a.init_tol) : a.init_tol;
    sh.flag = (a.rr_force || (!a.rr_first && crit <= tol)) ? 1 : 0;
    sh.scal[2] = crit;
  }
  __syncthreads();
  const int conv = sh.flag;
  if (blockIdx.x == 0 && t == 0) {
    for (int c = 0; c < w; ++c) st->sigma[c] = sh.sig[sh.order[c]];
    st->sigma_prev[0] = sh.scal[2];
    st->conv = conv;
    if (conv && a.init_phase == 0) st->zeta = st->beta_init * sh.sig[sh.order[0]];
    if (conv && a.init_phase == 1) {
      st->zeta = st->beta * sh.sig[sh.order[0]];
      st->k = 0;
    }
  }
  __syncthreads();
  if (conv && a.init_phase == 1) {
    prepare(a, sh);
    return;
  }
  // next bases: orth(Z V~) -> U~, orth(Z^T U~) -> V~
  if (!cholqr(Y1, m, w, Y2, n, w, 3, true, part, st, sh, Ut, Vt)) return;
  write_basis_copies<T>(a, w);
}

template <typename T>
__global__ void __launch_bounds__(ST, 1) small_kernel(SmallArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T>& sh = *reinterpret_cast<Smem<T>*>(smem_raw);
  if (a.mode == SM_UPDATE || a.mode == SM_RR) {
    if (a.st->done) return;
  }
  switch (a.mode) {
    case SM_UPDATE:
      mode_update<T>(a, sh);
      break;
    case SM_PREPARE:
      prepare<T>(a, sh);
      break;
    case SM_RR:
      mode_rr<T>(a, sh);
      break;
    case SM_RAND:
      mode_rand<T>(a, sh);
      break;
  }
}

}  // namespace

int small_grid_size(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaFuncSetAttribute(small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<float>));
  cudaFuncSetAttribute(small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>));
  return sms;  // one block per SM keeps the barrier short
}

cudaError_t launch_small(const SmallArgs& a, int grid, cudaStream_t s) {
  SmallArgs copy = a;
  void* args[] = {&copy};
  if (a.prec == PREC_F32)
    return cudaLaunchCooperativeKernel((const void*)small_kernel<float>, dim3(grid), dim3(ST), args,
                                       sizeof(Smem<float>), s);
  return cudaLaunchCooperativeKernel((const void*)small_kernel<double>, dim3(grid), dim3(ST), args,
                                     sizeof(Smem<double>), s);
}

}  // namespace rpca
