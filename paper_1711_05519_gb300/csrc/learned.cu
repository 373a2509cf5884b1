// Stateless pass and adjoint pass for the learned threshold schedule.
//
// The learned schedule runs AccAltProj unrolled for a fixed number of iterations and
// trains a small network that sets zeta_k from per-iteration statistics.  The hard
// threshold of Eq. (10) has zero derivative in zeta almost everywhere, so training uses a
// soft gate in its place:
//     g(R; zeta) = sigmoid((|R| - zeta) / (tau zeta)),   S = R g,   Z = D - S,
// which tends to the hard threshold as tau -> 0 (tau = 0 selects the hard threshold).
//
// Forward (rpca_learn_pass): per entry, L = W V^T (W = U Sigma), R = D - L, S, Z and
//   Y1 = Z V~, Y2 = Z^T U~, res2 = sum (R - S)^2, the hard support size and, with
//   bitmasks, the number of entries whose hard support membership changed.
// Adjoint (rpca_learn_pass_adjoint): given cotangents Y1b, Y2b, resb of the forward
//   outputs, the cotangents of U~, V~, W, V and zeta:
//     Zb   = Y1b V~^T + U~ Y2b^T
//     Rb   = -Zb (g + R g_R) + resb (2 R (1-g)^2 - 2 R^2 (1-g) g_R)
//     U~b  = Z Y2b,  V~b = Z^T Y1b,  Wb = -Rb V,  Vb = -Rb^T W
//     zetab = sum [ -Zb R g_zeta - resb 2 R^2 (1-g) g_zeta ]
//   with g_R = g(1-g) sign(R) / (tau zeta) and g_zeta = -g(1-g) |R| / (tau zeta^2).
//
// Work decomposition (both kernels): a CTA covers a 32-row x 32-column tile, lane = column,
// each warp four rows.  Column quantities are reduced over the CTA's rows in shared memory
// and row quantities over the warp's lanes by shuffles; tile results are added to the
// outputs with atomics (the outputs are cleared first), so summation order varies from run
// to run at rounding level.
#include "../../include/rpca.h"
#include "common.cuh"

namespace rpca {
namespace {

constexpr int TILE = 32, WARPS = 8, ROWS_PER_WARP = TILE / WARPS;

template <typename T>
__device__ __forceinline__ T sigm(T x) {
  return T(1) / (T(1) + exp(-x));
}

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct LearnArgs {
  const void* D;
  long long ld;
  int m, n, R;
  const void *W, *V, *Ut, *Vt;
  const double* zeta;
  double tau;
  // forward
  void *Y1, *Y2;
  double* stats;  // [0] res2, [1] hard support size, [2] support changes
  const unsigned* mask_old;
  unsigned* mask_new;
  // adjoint
  const void *Y1b, *Y2b;
  double resb;
  void *Utb, *Vtb, *Wb, *Vb;
  double* zetab;
};

template <typename T, int R, bool ADJ>
__global__ void __launch_bounds__(256) learn_pass_kernel(LearnArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row0 = blockIdx.y * TILE, col0 = blockIdx.x * TILE;
  const int j = col0 + lane;
  const bool jok = j < a.n;
  const T* D = static_cast<const T*>(a.D);
  const T* W = static_cast<const T*>(a.W);
  const T* V = static_cast<const T*>(a.V);
  const T* Ut = static_cast<const T*>(a.Ut);
  const T* Vt = static_cast<const T*>(a.Vt);
  const T* Y1b = static_cast<const T*>(a.Y1b);
  const T* Y2b = static_cast<const T*>(a.Y2b);
  const T zeta = (T)*a.zeta;
  const T tau = (T)a.tau;
  const bool soft = a.tau > 0.0;

  __shared__ T sW[TILE][R], sUt[TILE][R], sY1b[ADJ ? TILE : 1][R];
  __shared__ T colacc[WARPS][R][TILE];
  for (int e = threadIdx.x; e < TILE * R; e += 256) {
    const int rl = e / R, k = e % R, i = row0 + rl;
    sW[rl][k] = i < a.m ? W[(size_t)i * R + k] : T(0);
    sUt[rl][k] = i < a.m ? Ut[(size_t)i * R + k] : T(0);
    if (ADJ) sY1b[rl][k] = i < a.m ? Y1b[(size_t)i * R + k] : T(0);
  }
  T v[R], vt[R], y2b[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    v[k] = jok ? V[(size_t)j * R + k] : T(0);
    vt[k] = jok ? Vt[(size_t)j * R + k] : T(0);
    y2b[k] = (ADJ && jok) ? Y2b[(size_t)j * R + k] : T(0);
  }
  __syncthreads();

  T c0[R], c1[R];  // column accumulators: forward Y2 (c0); adjoint V~b (c0), Vb (c1)
#pragma unroll
  for (int k = 0; k < R; ++k) c0[k] = c1[k] = T(0);
  double res = 0.0, zb = 0.0;
  unsigned long long nnz = 0, chg = 0;
  const size_t words = ((size_t)a.n + 31) / 32;

  for (int t = 0; t < ROWS_PER_WARP; ++t) {
    const int rl = warp * ROWS_PER_WARP + t, i = row0 + rl;
    const bool iok = i < a.m;
    T l = T(0);
#pragma unroll
    for (int k = 0; k < R; ++k) l = fma(sW[rl][k], v[k], l);
    const T d = (iok && jok) ? D[(size_t)i * a.ld + j] : T(0);
    const T rr = d - l;
    const bool hard = (iok && jok) && fabs(rr) > zeta;
    T g, x = T(0);
    if (soft) {
      x = (fabs(rr) - zeta) / (tau * zeta);
      g = (iok && jok) ? sigm(x) : T(0);
    } else {
      g = hard ? T(1) : T(0);
    }
    const T z = d - rr * g;
    if (!ADJ) {
      res += (double)((rr - rr * g) * (rr - rr * g));
      const unsigned bal = __ballot_sync(0xffffffffu, hard);
      nnz += hard ? 1 : 0;
      if (a.mask_new && iok && lane == 0) {
        const size_t wi = (size_t)i * words + col0 / 32;
        if (a.mask_old) chg += __popc(bal ^ a.mask_old[wi]);
        a.mask_new[wi] = bal;
      }
      // Y1 row contribution (over this warp's 32 columns), Y2 column contribution
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const T y1 = wsum(z * vt[k]);
        if (lane == 0 && iok) atomicAdd(static_cast<T*>(a.Y1) + (size_t)i * R + k, y1);
        c0[k] = fma(z, sUt[rl][k], c0[k]);
      }
    } else {
      T zbar = T(0);
#pragma unroll
      for (int k = 0; k < R; ++k) zbar = fma(sY1b[rl][k], vt[k], fma(sUt[rl][k], y2b[k], zbar));
      T dgdR = T(0), dgdz = T(0);
      if (soft && iok && jok) {
        const T gp = g * (T(1) - g) / (tau * zeta);
        dgdR = (rr >= T(0) ? gp : -gp);
        dgdz = -gp * fabs(rr) / zeta;
      }
      const T omg = T(1) - g;
      const T rbar = -zbar * (g + rr * dgdR) + (T)a.resb * (T(2) * rr * omg * omg - T(2) * rr * rr * omg * dgdR);
      zb += (double)(-zbar * rr * dgdz - (T)a.resb * T(2) * rr * rr * omg * dgdz);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const T ub = wsum(z * y2b[k]);     // U~b_i = sum_j Z_ij Y2b_j
        const T wb = wsum(-rbar * v[k]);   // Wb_i  = -sum_j Rb_ij V_j
        if (lane == 0 && iok) {
          atomicAdd(static_cast<T*>(a.Utb) + (size_t)i * R + k, ub);
          atomicAdd(static_cast<T*>(a.Wb) + (size_t)i * R + k, wb);
        }
        c0[k] = fma(z, sY1b[rl][k], c0[k]);       // V~b_j = sum_i Z_ij Y1b_i
        c1[k] = fma(-rbar, sW[rl][k], c1[k]);     // Vb_j  = -sum_i Rb_ij W_i
      }
    }
  }
  // column accumulators: reduce over the warps, then one atomic per column
  for (int which = 0; which < (ADJ ? 2 : 1); ++which) {
#pragma unroll
    for (int k = 0; k < R; ++k) colacc[warp][k][lane] = which ? c1[k] : c0[k];
    __syncthreads();
    for (int e = threadIdx.x; e < R * TILE; e += 256) {
      const int k = e / TILE, cl = e % TILE, jj = col0 + cl;
      T s = T(0);
      for (int w = 0; w < WARPS; ++w) s += colacc[w][k][cl];
      if (jj < a.n) {
        T* dst = ADJ ? static_cast<T*>(which ? a.Vb : a.Vtb) : static_cast<T*>(a.Y2);
        atomicAdd(dst + (size_t)jj * R + k, s);
      }
    }
    __syncthreads();
  }
  // scalars
  if (!ADJ) {
    const double rs = wsum(res);
    unsigned long long nz = nnz, ch = chg;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nz += __shfl_xor_sync(0xffffffffu, nz, o);
      ch += __shfl_xor_sync(0xffffffffu, ch, o);
    }
    if (lane == 0) {
      atomicAdd(&a.stats[0], rs);
      atomicAdd(&a.stats[1], (double)nz);
      atomicAdd(&a.stats[2], (double)ch);
    }
  } else {
    const double z2 = wsum(zb);
    if (lane == 0) atomicAdd(a.zetab, z2);
  }
}

template <typename T, bool ADJ>
cudaError_t launch_learn(int R, const LearnArgs& a, cudaStream_t s) {
  dim3 grid((a.n + TILE - 1) / TILE, (a.m + TILE - 1) / TILE);
#define RPCA_CASE(RR)                                              \
  case RR:                                                         \
    learn_pass_kernel<T, RR, ADJ><<<grid, 256, 0, s>>>(a);         \
    return cudaGetLastError();
  switch (R) { RPCA_FOR_EACH_R(RPCA_CASE) }
#undef RPCA_CASE
  return cudaErrorInvalidValue;
}

bool learn_args_ok(const void* D, int64_t m, int64_t n, int64_t ld, int dtype, int r, const void* W, const void* V,
                   const void* Ut, const void* Vt, const double* zeta, double tau) {
  return D && W && V && Ut && Vt && zeta && m >= 1 && n >= 1 && ld >= n && r >= 1 && r <= kMaxR &&
         padded_rank(r) == r && (dtype == RPCA_DTYPE_F32 || dtype == RPCA_DTYPE_F64) && tau >= 0.0 &&
         m * n < (1ll << 40);
}

}  // namespace
}  // namespace rpca

using namespace rpca;

extern "C" int rpca_learn_pass(const void* D, int64_t m, int64_t n, int64_t ld, int dtype, int r, const void* W,
                               const void* V, const void* Ut, const void* Vt, const double* zeta, double tau, void* Y1,
                               void* Y2, double* stats, const uint32_t* mask_old, uint32_t* mask_new, void* stream) {
  if (!learn_args_ok(D, m, n, ld, dtype, r, W, V, Ut, Vt, zeta, tau) || !Y1 || !Y2 || !stats)
    return RPCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ts = dtype == RPCA_DTYPE_F32 ? 4 : 8;
  if (cudaMemsetAsync(Y1, 0, (size_t)m * r * ts, s) || cudaMemsetAsync(Y2, 0, (size_t)n * r * ts, s) ||
      cudaMemsetAsync(stats, 0, 4 * sizeof(double), s))
    return RPCA_ERR_CUDA;
  LearnArgs a = {};
  a.D = D;
  a.ld = ld;
  a.m = (int)m;
  a.n = (int)n;
  a.R = r;
  a.W = W;
  a.V = V;
  a.Ut = Ut;
  a.Vt = Vt;
  a.zeta = zeta;
  a.tau = tau;
  a.Y1 = Y1;
  a.Y2 = Y2;
  a.stats = stats;
  a.mask_old = mask_old;
  a.mask_new = mask_new;
  const cudaError_t e = dtype == RPCA_DTYPE_F32 ? launch_learn<float, false>(r, a, s) : launch_learn<double, false>(r, a, s);
  return e == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}

extern "C" int rpca_learn_pass_adjoint(const void* D, int64_t m, int64_t n, int64_t ld, int dtype, int r,
                                       const void* W, const void* V, const void* Ut, const void* Vt, const double* zeta,
                                       double tau, const void* Y1b, const void* Y2b, double resb, void* Utb, void* Vtb,
                                       void* Wb, void* Vb, double* zetab, void* stream) {
  if (!learn_args_ok(D, m, n, ld, dtype, r, W, V, Ut, Vt, zeta, tau) || !Y1b || !Y2b || !Utb || !Vtb || !Wb || !Vb ||
      !zetab)
    return RPCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ts = dtype == RPCA_DTYPE_F32 ? 4 : 8;
  if (cudaMemsetAsync(Utb, 0, (size_t)m * r * ts, s) || cudaMemsetAsync(Wb, 0, (size_t)m * r * ts, s) ||
      cudaMemsetAsync(Vtb, 0, (size_t)n * r * ts, s) || cudaMemsetAsync(Vb, 0, (size_t)n * r * ts, s) ||
      cudaMemsetAsync(zetab, 0, sizeof(double), s))
    return RPCA_ERR_CUDA;
  LearnArgs a = {};
  a.D = D;
  a.ld = ld;
  a.m = (int)m;
  a.n = (int)n;
  a.R = r;
  a.W = W;
  a.V = V;
  a.Ut = Ut;
  a.Vt = Vt;
  a.zeta = zeta;
  a.tau = tau;
  a.Y1b = Y1b;
  a.Y2b = Y2b;
  a.resb = resb;
  a.Utb = Utb;
  a.Vtb = Vtb;
  a.Wb = Wb;
  a.Vb = Vb;
  a.zetab = zetab;
  const cudaError_t e = dtype == RPCA_DTYPE_F32 ? launch_learn<float, true>(r, a, s) : launch_learn<double, true>(r, a, s);
  return e == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}
