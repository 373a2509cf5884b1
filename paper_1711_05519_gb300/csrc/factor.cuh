// Cholesky factor R (R^T R = G) and its inverse T = R^-1 (X T has orthonormal columns for
// X = Q R) of a small Gram matrix G = X^T X, by one warp in registers.  This is the QR step of
// Section 2.1 with the Q factor left implicit (CholeskyQR): the update kernel factors the Gram
// matrices of the projected products and of the trimmed factors, and the tensor-core pass
// factors the latter for the update that follows it.
#pragma once

#include <cuda_runtime.h>

namespace rpca {
namespace fac {

// 1 / sqrt(x) for x > 0 in double precision: the single-precision estimate refined by two
// Newton-Raphson steps y <- y (3 - x y^2) / 2 (each roughly doubles the correct bits).  Double
// square roots and divisions are long-latency on this part; this takes a few fused
// multiply-adds.  Arguments outside the single-precision range take the library routine.
__device__ __forceinline__ double rsqrt_d(double x) {
  if (!(x > 1e-36 && x < 1e36)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}
__device__ __forceinline__ float rsqrt_d(float x) { return 1.0f / sqrtf(x); }

// Lane l < w holds column l of the w x w Gram matrix G in g (g[k] = G_kl, zero past w; lanes
// l >= w hold zeros), w <= WM.  G is scaled to unit diagonal first, G^ = D^-1/2 G D^-1/2; a
// pivot of G^ at or below 1e-6 (float) or 1e-14 (double), a direction lost to rounding, gives a
// zero row of R and a zero column of T.  Then R = R^ D^1/2 and T = D^-1/2 R^-1, column l of
// R^-1 by back substitution in lane l (the entries of R^ it needs come from the other lanes by
// shuffles).  Writes R (if not null) and T row-major with leading dimension w, upper
// triangular.  All 32 lanes of the warp must call.
template <typename T, int WM>
__device__ __forceinline__ void chol_cols(const T (&g)[WM], int w, T* R, T* Tm) {
  constexpr unsigned FULLM = 0xffffffffu;
  const int l = threadIdx.x & 31;
  const T tiny = sizeof(T) == 4 ? T(1e-6) : T(1e-14);
  T gll = T(0);
#pragma unroll
  for (int k = 0; k < WM; ++k)
    if (k == l) gll = g[k];
  const T il = (l < w && gll > T(0)) ? rsqrt_d(gll) : T(0);
  const T dl = gll * il;
  T a[WM];  // column l of the working matrix
#pragma unroll
  for (int k = 0; k < WM; ++k) {
    const T ik = __shfl_sync(FULLM, il, k);
    a[k] = (l < w && k < w) ? g[k] * (ik * il) : T(0);
  }
  // right-looking Cholesky: step j fixes row j of R^ (a[j] of every lane becomes R^_jl)
  T pinv = T(0);  // this lane's 1 / R^_ll
#pragma unroll
  for (int j = 0; j < WM; ++j) {
    if (j < w) {
      const T d = __shfl_sync(FULLM, a[j], j);
      const bool good = d > tiny;
      const T inv = good ? rsqrt_d(d) : T(0);
      const T rjj = d * inv;
      if (l == j) pinv = inv;
      const T rjl = (l > j) ? a[j] * inv : ((l == j) ? rjj : T(0));
      a[j] = rjl;
#pragma unroll
      for (int k = j + 1; k < WM; ++k) {
        const T rjk = __shfl_sync(FULLM, rjl, k);
        a[k] = fma(-rjk, rjl, a[k]);
      }
    }
  }
  // column l of R^-1: t_i = (delta_il - sum_{k=i+1}^{l} R^_ik t_k) / R^_ii for i = l .. 0,
  // with R^_ik = a[i] of lane k
  const T rd = (l < w) ? pinv : T(0);
  T t[WM];
#pragma unroll
  for (int i = WM - 1; i >= 0; --i) {
    t[i] = T(0);
    if (i < w) {
      const T ri = __shfl_sync(FULLM, rd, i);
      T sacc = (i == l) ? T(1) : T(0);
#pragma unroll
      for (int k = i + 1; k < WM; ++k) {
        if (k < w) {
          const T rik = __shfl_sync(FULLM, a[i], k);
          if (k <= l) sacc = fma(-rik, t[k], sacc);
        }
      }
      t[i] = (i <= l) ? sacc * ri : T(0);
    }
  }
  // T = D^-1/2 R^-1 (row i scaled by 1 / d_i), R = R^ D^1/2 (column l scaled by d_l)
#pragma unroll
  for (int i = 0; i < WM; ++i) {
    const T ii = __shfl_sync(FULLM, il, i);
    if (l < w && i < w) {
      Tm[i * w + l] = t[i] * ii;
      if (R) R[i * w + l] = (i <= l) ? a[i] * dl : T(0);
    }
  }
  __syncwarp();
}

}  // namespace fac
}  // namespace rpca
