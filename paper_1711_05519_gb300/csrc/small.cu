// FP64 tall-skinny kernel of the AccAltProj iteration and of the initialisation.
//
// One cooperative launch per call (all blocks co-resident, one per SM).  Phases are
// separated by a bounded grid barrier; small matrices (r x r Gram factors, the 2r x 2r
// core M_k, its SVD) are computed redundantly by every block in shared memory, so the
// only cross-block traffic is the per-block Gram partials.
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
constexpr int GSLOT = MW * MW;
constexpr int NSLOT = 4;    // Gram partial slots per block
constexpr int kErrTimeout = 6;
constexpr int kErrNumerical = 3;

struct Smem {
  double red[ST];
  double G[NSLOT][GSLOT];      // reduced Gram matrices
  double Racc[2][GSLOT];       // accumulated R factors (upper)
  double Rstep[2][GSLOT];      // R factor of the current CholeskyQR pass
  double C[GSLOT];             // U~^T Y1
  double A[MN * (MN + 1)];     // SVD work, column-major, leading dimension MN+1
  double Vm[MN * (MN + 1)];    // accumulated right rotations
  double sig[MN];
  int order[MN];
  int flag;
  int ok;
  double scal[8];
};

__device__ __forceinline__ double wsum(double v) {
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
__device__ bool grid_barrier(DevState* st, Smem& sh) {
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
        __nanosleep(100);
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

// This block's part of X^T Y over rows [lo, hi) (X: rows x wx, Y: rows x wy, row-major
// with leading dimensions ldx, ldy) into part[blockIdx][slot][wx*wy].
__device__ void gram_partial(const double* X, int ldx, int wx, const double* Y, int ldy, int wy, int rows,
                             double* part, int slot, Smem& sh) {
  int lo, hi;
  block_range(rows, lo, hi);
  const int P = wx * wy;
  const int t = threadIdx.x;
  double* out = part + ((size_t)blockIdx.x * NSLOT + slot) * GSLOT;
  if (P >= ST / 2) {
    for (int p = t; p < P; p += ST) {
      const int a = p / wy, b = p % wy;
      double acc = 0.0;
      for (int i = lo; i < hi; ++i) acc = fma(X[(size_t)i * ldx + a], Y[(size_t)i * ldy + b], acc);
      out[p] = acc;
    }
    return;
  }
  const int nl = ST / P;
  const int p = t % P, l = t / P;
  double acc = 0.0;
  if (l < nl) {
    const int a = p / wy, b = p % wy;
    for (int i = lo + l; i < hi; i += nl) acc = fma(X[(size_t)i * ldx + a], Y[(size_t)i * ldy + b], acc);
  }
  sh.red[t] = acc;
  __syncthreads();
  if (t < P) {
    double s = 0.0;
    for (int q = 0; q < nl; ++q) s += sh.red[t + q * P];
    out[t] = s;
  }
  __syncthreads();
}

// Fixed-order sum over blocks of a partial slot into shared G.
__device__ void gram_reduce(const double* part, int slot, int P, double* G) {
  for (int p = threadIdx.x; p < P; p += ST) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += part[((size_t)b * NSLOT + slot) * GSLOT + p];
    G[p] = s;
  }
  __syncthreads();
}

// Upper Cholesky factor R (R^T R = G + shift I) of a w x w symmetric matrix, by warp 0.
// A pivot that is not positive (rank deficiency) gives a zero row of R.
__device__ void cholesky_upper(const double* G, int w, double shift, double* R, Smem& sh) {
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    // work in R: start from the upper triangle of G + shift I
    for (int j = 0; j < w; ++j)
      if (l < w) R[j * w + l] = (l >= j) ? G[j * w + l] + ((l == j) ? shift : 0.0) : 0.0;
    __syncwarp();
    double scale = 0.0;
    for (int j = 0; j < w; ++j) scale = fmax(scale, fabs(G[j * w + j]) + shift);
    for (int j = 0; j < w; ++j) {
      const double d = R[j * w + j];
      const bool good = d > 1e-300 && d > 1e-30 * scale;
      const double rjj = good ? sqrt(d) : 0.0;
      __syncwarp();
      if (l >= j && l < w) R[j * w + l] = good ? ((l == j) ? rjj : R[j * w + l] / rjj) : 0.0;
      __syncwarp();
      // Schur update of rows j+1.. : lane l owns column l
      if (l > j && l < w)
        for (int k = j + 1; k <= l; ++k) R[k * w + l] -= R[j * w + k] * R[j * w + l];
      __syncwarp();
    }
  }
  __syncthreads();
}

// y (1 x w) <- y R^{-1} for upper R; zero diagonal gives a zero entry.
__device__ __forceinline__ void trsv_row(double* y, const double* R, int w) {
  for (int j = 0; j < w; ++j) {
    double s = y[j];
    for (int k = 0; k < j; ++k) s -= y[k] * R[k * w + j];
    const double d = R[j * w + j];
    y[j] = (d != 0.0) ? s / d : 0.0;
  }
}

// Racc <- Rstep * Racc (both upper w x w), by the block.
__device__ void upper_mul_acc(double* Racc, const double* Rstep, int w, Smem& sh) {
  double* tmp = sh.red;  // w*w <= 256 <= ST
  const int t = threadIdx.x;
  if (t < w * w) {
    const int i = t / w, j = t % w;
    double s = 0.0;
    for (int k = i; k <= j; ++k) s += Rstep[i * w + k] * Racc[k * w + j];
    tmp[t] = (j >= i) ? s : 0.0;
  }
  __syncthreads();
  if (t < w * w) Racc[t] = tmp[t];
  __syncthreads();
}

// In-place QR of X1 (rows1 x w1) and X2 (rows2 x w2, may be null) by CholeskyQR, `passes`
// passes, the first with the shift of shifted CholeskyQR (Fukaya et al. 2020) when
// `shifted`.  Leaves the R factors in sh.Racc[0], sh.Racc[1].  Returns false on a barrier
// failure.  `copy1`/`copy2` (may be null) receive a copy of the final Q.
__device__ bool cholqr(double* X1, int rows1, int w1, double* X2, int rows2, int w2, int passes, bool shifted,
                       double* part, DevState* st, Smem& sh, double* copy1, double* copy2) {
  const int t = threadIdx.x;
  for (int e = t; e < GSLOT; e += ST) {
    sh.Racc[0][e] = ((e / w1) == (e % w1) && e < w1 * w1) ? 1.0 : 0.0;
    sh.Racc[1][e] = (X2 && (e / w2) == (e % w2) && e < w2 * w2) ? 1.0 : 0.0;
  }
  gram_partial(X1, w1, w1, X1, w1, w1, rows1, part, 0, sh);
  if (X2) gram_partial(X2, w2, w2, X2, w2, w2, rows2, part, 1, sh);
  for (int ps = 0; ps < passes; ++ps) {
    if (!grid_barrier(st, sh)) return false;
    gram_reduce(part, 0, w1 * w1, sh.G[0]);
    if (X2) gram_reduce(part, 1, w2 * w2, sh.G[1]);
    double sh1 = 0.0, sh2 = 0.0;
    if (shifted && ps == 0) {
      const double u = 1.1102230246251565e-16;
      double tr1 = 0.0, tr2 = 0.0;
      for (int j = 0; j < w1; ++j) tr1 += sh.G[0][j * w1 + j];
      for (int j = 0; X2 && j < w2; ++j) tr2 += sh.G[1][j * w2 + j];
      sh1 = 11.0 * ((double)rows1 * w1 + (double)w1 * (w1 + 1)) * u * tr1;
      sh2 = 11.0 * ((double)rows2 * w2 + (double)w2 * (w2 + 1)) * u * tr2;
    }
    cholesky_upper(sh.G[0], w1, sh1, sh.Rstep[0], sh);
    if (X2) cholesky_upper(sh.G[1], w2, sh2, sh.Rstep[1], sh);
    upper_mul_acc(sh.Racc[0], sh.Rstep[0], w1, sh);
    if (X2) upper_mul_acc(sh.Racc[1], sh.Rstep[1], w2, sh);
    const bool last = (ps == passes - 1);
    // apply R^{-1} row by row
    for (int side = 0; side < (X2 ? 2 : 1); ++side) {
      double* X = side ? X2 : X1;
      const int rows = side ? rows2 : rows1, w = side ? w2 : w1;
      double* cp = side ? copy2 : copy1;
      int lo, hi;
      block_range(rows, lo, hi);
      for (int i = lo + t; i < hi; i += ST) {
        double y[MW];
        for (int j = 0; j < w; ++j) y[j] = X[(size_t)i * w + j];
        trsv_row(y, sh.Rstep[side], w);
        for (int j = 0; j < w; ++j) X[(size_t)i * w + j] = y[j];
        if (last && cp)
          for (int j = 0; j < w; ++j) cp[(size_t)i * w + j] = y[j];
      }
    }
    __syncthreads();
    if (!last) {
      gram_partial(X1, w1, w1, X1, w1, w1, rows1, part, 0, sh);
      if (X2) gram_partial(X2, w2, w2, X2, w2, w2, rows2, part, 1, sh);
    }
  }
  return true;
}

// One-sided Jacobi SVD of the N x N matrix held column-major in sh.A (N even, N <= 32).
// On return sh.sig holds the column norms (singular values), sh.order their descending
// order, sh.A the rotated columns (U Sigma) and sh.Vm the right singular vectors.
__device__ void jacobi_svd(int N, Smem& sh) {
  constexpr int LD = MN + 1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int e = t; e < N * N; e += ST) {
    const int c = e / N, rw = e % N;
    sh.Vm[c * LD + rw] = (c == rw) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int half = N / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (t == 0) sh.flag = 0;
    __syncthreads();
    for (int round = 0; round < N - 1; ++round) {
      if (warp < half) {
        // round-robin pairing: position 0 fixed, positions 1..N-1 rotated by `round`
        auto pos = [&](int s) { return s == 0 ? 0 : 1 + (s - 1 + round) % (N - 1); };
        int p = pos(warp), q = pos(N - 1 - warp);
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        const double ap = (lane < N) ? sh.A[p * LD + lane] : 0.0;
        const double aq = (lane < N) ? sh.A[q * LD + lane] : 0.0;
        const double alpha = wsum(ap * ap), beta = wsum(aq * aq), gam = wsum(ap * aq);
        if (gam != 0.0 && fabs(gam) > 1e-15 * sqrt(alpha * beta)) {
          const double zeta = (beta - alpha) / (2.0 * gam);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
          if (lane < N) {
            sh.A[p * LD + lane] = c * ap - s * aq;
            sh.A[q * LD + lane] = s * ap + c * aq;
            const double vp = sh.Vm[p * LD + lane], vq = sh.Vm[q * LD + lane];
            sh.Vm[p * LD + lane] = c * vp - s * vq;
            sh.Vm[q * LD + lane] = s * vp + c * vq;
          }
          if (lane == 0) sh.flag = 1;
        }
      }
      __syncthreads();
    }
    const int f = sh.flag;
    __syncthreads();
    if (!f) break;
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

__device__ __forceinline__ void store_tc(void* dst, int prec, size_t idx, double v) {
  if (prec == PREC_F32)
    static_cast<float*>(dst)[idx] = static_cast<float>(v);
  else
    static_cast<double*>(dst)[idx] = v;
}

// Trim (Algorithm 2) + orthonormal bases + pass-precision copies, from the master
// factors U (m x r), sig, V (n x r).
__device__ bool prepare(const SmallArgs& a, Smem& sh) {
  const int m = a.m, n = a.n, r = a.r, t = threadIdx.x;
  const double mu = a.st->mu_trim;
  const double cu = sqrt(mu * r / m), cv = sqrt(mu * r / n);
  for (int side = 0; side < 2; ++side) {
    const double* F = side ? a.V : a.U;
    double* T = side ? a.Vt : a.Ut;
    const int rows = side ? n : m;
    const double cap = side ? cv : cu;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      double nrm = 0.0;
      for (int j = 0; j < r; ++j) nrm += F[(size_t)i * r + j] * F[(size_t)i * r + j];
      nrm = sqrt(nrm);
      const double sc = (a.st->trim && nrm > cap) ? cap / nrm : 1.0;
      for (int j = 0; j < r; ++j) T[(size_t)i * r + j] = sc * F[(size_t)i * r + j];
    }
  }
  __syncthreads();
  if (a.st->trim) {
    if (!cholqr(a.Ut, m, r, a.Vt, n, r, 2, false, a.part, a.st, sh, nullptr, nullptr)) return false;
  }
  // pass-precision copies, zero-padded to the compiled width of the iteration's pass
  const int Rc = a.Rit;
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      for (int j = 0; j < Rc; ++j) {
        const size_t o = (size_t)i * Rc + j;
        if (side == 0) {
          store_tc(a.Wc, a.prec, o, j < r ? a.U[(size_t)i * r + j] * a.sig[j] : 0.0);
          store_tc(a.Utc, a.prec, o, j < r ? a.Ut[(size_t)i * r + j] : 0.0);
        } else {
          store_tc(a.Vc, a.prec, o, j < r ? a.V[(size_t)i * r + j] : 0.0);
          store_tc(a.Vtc, a.prec, o, j < r ? a.Vt[(size_t)i * r + j] : 0.0);
        }
      }
    }
  }
  return true;
}

// Y1 (m x w), Y2 (n x w) <- fixed-order sums of the pass partials (width R).
__device__ void reduce_partials(const SmallArgs& a, int w) {
  const size_t gt = (size_t)blockIdx.x * ST + threadIdx.x, gs = (size_t)gridDim.x * ST;
  for (size_t e = gt; e < (size_t)a.m * w; e += gs) {
    const size_t i = e / w, c = e % w;
    double s = 0.0;
    for (int q = 0; q < a.n_p1; ++q) {
      const size_t o = ((size_t)q * a.m + i) * a.R + c;
      s += (a.prec == PREC_F32) ? (double)static_cast<const float*>(a.P1)[o] : static_cast<const double*>(a.P1)[o];
    }
    a.Y1[e] = s;
  }
  for (size_t e = gt; e < (size_t)a.n * w; e += gs) {
    const size_t j = e / w, c = e % w;
    double s = 0.0;
    for (int q = 0; q < a.n_p2; ++q) {
      const size_t o = ((size_t)q * a.n + j) * a.R + c;
      s += (a.prec == PREC_F32) ? (double)static_cast<const float*>(a.P2)[o] : static_cast<const double*>(a.P2)[o];
    }
    a.Y2[e] = s;
  }
}

__device__ void cta_totals(const SmallArgs& a, double& res2, unsigned long long& nnz, Smem& sh) {
  // every block sums the per-CTA totals in the same order
  if (threadIdx.x < 32) {
    double s = 0.0;
    unsigned long long z = 0;
    for (int c = threadIdx.x; c < a.n_cta; c += 32) {
      s += a.resP[c];
      z += a.nnzP[c];
    }
    // fixed-shape reduction across the warp
    s = wsum(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (threadIdx.x == 0) {
      sh.scal[0] = s;
      sh.scal[1] = __longlong_as_double((long long)z);
    }
  }
  __syncthreads();
  res2 = sh.scal[0];
  nnz = (unsigned long long)__double_as_longlong(sh.scal[1]);
  __syncthreads();
}

__device__ void mode_update(const SmallArgs& a, Smem& sh) {
  DevState* st = a.st;
  const int m = a.m, n = a.n, r = a.r, t = threadIdx.x;
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
  reduce_partials(a, r);
  if (!grid_barrier(st, sh)) return;
  // C = U~^T Y1
  gram_partial(a.Ut, r, r, a.Y1, r, r, m, a.part, 2, sh);
  if (!grid_barrier(st, sh)) return;
  gram_reduce(a.part, 2, r * r, sh.C);
  // Y1 <- Y1 - U~ C ; Y2 <- Y2 - V~ C^T
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    double* Y = side ? a.Y2 : a.Y1;
    const double* B = side ? a.Vt : a.Ut;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      double y[MW];
      for (int c = 0; c < r; ++c) {
        double s = Y[(size_t)i * r + c];
        for (int q = 0; q < r; ++q) s -= B[(size_t)i * r + q] * (side ? sh.C[c * r + q] : sh.C[q * r + c]);
        y[c] = s;
      }
      for (int c = 0; c < r; ++c) Y[(size_t)i * r + c] = y[c];
    }
  }
  __syncthreads();
  if (!cholqr(a.Y1, m, r, a.Y2, n, r, 3, true, a.part, st, sh, nullptr, nullptr)) return;
  // M = [[C, R2^T], [R1, 0]], column-major in sh.A
  constexpr int LD = MN + 1;
  const int N = 2 * r;
  for (int e = t; e < N * N; e += ST) {
    const int row = e / N, col = e % N;
    double v = 0.0;
    if (row < r && col < r)
      v = sh.C[row * r + col];
    else if (row < r && col >= r)
      v = sh.Racc[1][(col - r) * r + row];  // R2^T
    else if (row >= r && col < r)
      v = sh.Racc[0][(row - r) * r + col];  // R1
    sh.A[col * LD + row] = v;
  }
  __syncthreads();
  jacobi_svd(N, sh);
  const double s1 = sh.sig[sh.order[0]];
  const double sr1 = sh.sig[sh.order[r]];
  // new factors by Eq. (9): U <- [U~ Q1] U_M[:, :r], V <- [V~ Q2] V_M[:, :r]
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    const double* B = side ? a.Vt : a.Ut;
    const double* Q = side ? a.Y2 : a.Y1;
    double* F = side ? a.V : a.U;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      double out[MW];
      for (int c = 0; c < r; ++c) {
        const int oc = sh.order[c];
        const double sg = sh.sig[oc];
        double s = 0.0;
        for (int q = 0; q < r; ++q) {
          const double um = side ? sh.Vm[oc * LD + q] : (sg > 0.0 ? sh.A[oc * LD + q] / sg : 0.0);
          const double um2 = side ? sh.Vm[oc * LD + r + q] : (sg > 0.0 ? sh.A[oc * LD + r + q] / sg : 0.0);
          s += B[(size_t)i * r + q] * um + Q[(size_t)i * r + q] * um2;
        }
        out[c] = s;
      }
      for (int c = 0; c < r; ++c) F[(size_t)i * r + c] = out[c];
    }
  }
  if (t < r) a.sig[t] = sh.sig[sh.order[t]];
  __syncthreads();
  if (blockIdx.x == 0 && t == 0) {
    const int k1 = k + 1;
    const double g = pow(st->gamma, (double)k1);
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

__device__ double gauss(unsigned long long seed, unsigned long long i) {
  auto mix = [](unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  };
  const unsigned long long a = mix(seed * 0x632be59bd9b4e019ull + 2 * i);
  const unsigned long long b = mix(seed * 0x632be59bd9b4e019ull + 2 * i + 1);
  const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);
  const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

__device__ void write_basis_copies(const SmallArgs& a, int w) {
  // U~, V~ (FP64, width w) -> pass copies of width Rc; W = 0, V = 0 (init passes use L = 0)
  const int t = threadIdx.x, Rc = a.Rc;
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? a.n : a.m;
    const double* B = side ? a.Vt : a.Ut;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST)
      for (int j = 0; j < Rc; ++j) {
        const size_t o = (size_t)i * Rc + j;
        store_tc(side ? a.Vtc : a.Utc, a.prec, o, j < w ? B[(size_t)i * w + j] : 0.0);
        store_tc(side ? a.Vc : a.Wc, a.prec, o, 0.0);
      }
  }
}

__device__ void mode_rand(const SmallArgs& a, Smem& sh) {
  const int w = a.b;
  const size_t gt = (size_t)blockIdx.x * ST + threadIdx.x, gs = (size_t)gridDim.x * ST;
  for (size_t e = gt; e < (size_t)a.m * w; e += gs) a.Y1[e] = gauss(a.seed, e);
  for (size_t e = gt; e < (size_t)a.n * w; e += gs) a.Y2[e] = gauss(a.seed ^ 0x5bd1e995ull, e);
  if (!grid_barrier(a.st, sh)) return;
  if (!cholqr(a.Y1, a.m, w, a.Y2, a.n, w, 3, true, a.part, a.st, sh, a.Ut, a.Vt)) return;
  write_basis_copies(a, w);
}

__device__ void mode_rr(const SmallArgs& a, Smem& sh) {
  DevState* st = a.st;
  const int m = a.m, n = a.n, w = a.b, r = a.r, t = threadIdx.x;
  constexpr int LD = MN + 1;
  double res2;
  unsigned long long nnz;
  cta_totals(a, res2, nnz, sh);
  if (a.init_phase == 0 && a.rr_first && blockIdx.x == 0 && t == 0) st->normD2 = res2;
  reduce_partials(a, w);
  if (!grid_barrier(st, sh)) return;
  gram_partial(a.Ut, w, w, a.Y1, w, w, m, a.part, 2, sh);  // B = U~^T (Z V~)
  if (!grid_barrier(st, sh)) return;
  gram_reduce(a.part, 2, w * w, sh.C);
  for (int e = t; e < w * w; e += ST) {
    const int row = e / w, col = e % w;
    sh.A[col * LD + row] = sh.C[row * w + col];
  }
  __syncthreads();
  jacobi_svd(w, sh);
  // Top Ritz triplets: u_c = U~ U_B[:, c], v_c = V~ V_B[:, c], sigma_c.  Their residuals
  // Z v_c - sigma_c u_c = Y1 V_B[:, c] - sigma_c u_c and Z^T u_c - sigma_c v_c =
  // Y2 U_B[:, c] - sigma_c v_c need no further pass over D; the sum of their squared
  // norms, each divided by sigma_c^2, decides convergence.
  const int nr = (a.init_phase == 0) ? 1 : r;
  double acc = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int rows = side ? n : m;
    const double* B = side ? a.Vt : a.Ut;
    const double* Y = side ? a.Y2 : a.Y1;
    double* F = side ? a.V : a.U;
    int lo, hi;
    block_range(rows, lo, hi);
    for (int i = lo + t; i < hi; i += ST) {
      for (int c = 0; c < r; ++c) {
        const int oc = sh.order[c];
        const double sg = sh.sig[oc];
        const double inv = sg > 0.0 ? 1.0 / sg : 0.0;
        double f = 0.0, zy = 0.0;
        for (int q = 0; q < w; ++q) {
          const double ub = sh.A[oc * LD + q] * inv;  // U_B[q][c]
          const double vb = sh.Vm[oc * LD + q];       // V_B[q][c]
          f += B[(size_t)i * w + q] * (side ? vb : ub);
          zy += Y[(size_t)i * w + q] * (side ? ub : vb);
        }
        F[(size_t)i * r + c] = f;
        if (c < nr) {
          const double d = (zy - sg * f) * inv;
          acc += d * d;
        }
      }
    }
  }
  sh.red[t] = acc;
  __syncthreads();
  for (int h = ST / 2; h > 0; h >>= 1) {
    if (t < h) sh.red[t] += sh.red[t + h];
    __syncthreads();
  }
  if (t == 0) a.part[((size_t)blockIdx.x * NSLOT + 3) * GSLOT] = sh.red[0];
  if (t < r) a.sig[t] = sh.sig[sh.order[t]];
  if (!grid_barrier(st, sh)) return;
  if (t == 0) {
    double tot = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) tot += a.part[((size_t)b * NSLOT + 3) * GSLOT];
    const double crit = sqrt(tot);
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
  if (!cholqr(a.Y1, m, w, a.Y2, n, w, 3, true, a.part, st, sh, a.Ut, a.Vt)) return;
  write_basis_copies(a, w);
}

__global__ void __launch_bounds__(ST, 1) small_kernel(SmallArgs a) {
  __shared__ Smem sh;
  if (a.mode == SM_UPDATE || a.mode == SM_RR) {
    if (a.st->done) return;
  }
  switch (a.mode) {
    case SM_UPDATE:
      mode_update(a, sh);
      break;
    case SM_PREPARE:
      prepare(a, sh);
      break;
    case SM_RR:
      mode_rr(a, sh);
      break;
    case SM_RAND:
      mode_rand(a, sh);
      break;
  }
}

}  // namespace

int small_grid_size(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, small_kernel, ST, 0);
  if (occ < 1) occ = 1;
  return sms;  // one block per SM keeps the barrier short
}

cudaError_t launch_small(const SmallArgs& a, int grid, cudaStream_t s) {
  SmallArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)small_kernel, dim3(grid), dim3(ST), args, 0, s);
}

}  // namespace rpca
