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

// ---------------------------------------------------------------------------------------
// Threshold network of the learned schedule (mlp.cuh): batched forward, hand-written
// backward and the Adam update used to train it.
// ---------------------------------------------------------------------------------------
#include "mlp.cuh"

namespace rpca {
namespace {

// One warp per statistic vector: zeta_i = plain_i exp(clamp(g(s_i))).
__global__ void __launch_bounds__(32) schedule_forward_kernel(const float* __restrict__ theta,
                                                             const float* __restrict__ feats,
                                                             const double* __restrict__ plain, int n,
                                                             double* __restrict__ zeta, float* __restrict__ gout) {
  const int i = blockIdx.x;
  if (i >= n) return;
  float s[mlp::IN], h1, h2;
#pragma unroll
  for (int q = 0; q < mlp::IN; ++q) s[q] = feats[i * mlp::IN + q];
  const float gc = mlp::clamp_g(mlp::forward_warp(theta, s, h1, h2));
  if ((threadIdx.x & 31) == 0) {
    zeta[i] = plain[i] * (double)expf(gc);
    if (gout) gout[i] = gc;
  }
}

// Gradient of sum_i zeta_bar_i zeta_i with respect to the parameters, one warp, samples in
// order (deterministic).  Lane j owns hidden unit j of both layers: row j of W2 and of W1.
// Through the clamp the derivative is zero where the output is saturated; d zeta / d g = zeta.
__global__ void __launch_bounds__(32) schedule_backward_kernel(const float* __restrict__ theta,
                                                              const float* __restrict__ feats,
                                                              const double* __restrict__ plain,
                                                              const double* __restrict__ zeta_bar, int n,
                                                              float* __restrict__ grad) {
  using namespace mlp;
  const int j = threadIdx.x & 31;
  float gW1[IN], gW2[H], gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
#pragma unroll
  for (int q = 0; q < IN; ++q) gW1[q] = 0.f;
#pragma unroll
  for (int q = 0; q < H; ++q) gW2[q] = 0.f;
  for (int i = 0; i < n; ++i) {
    float s[IN], h1, h2;
#pragma unroll
    for (int q = 0; q < IN; ++q) s[q] = feats[i * IN + q];
    const float g = forward_warp(theta, s, h1, h2);
    const float gc = clamp_g(g);
    const double z = plain[i] * (double)expf(gc);
    const float dg = (g > -kLog4 && g < kLog4) ? (float)(zeta_bar[i] * z) : 0.f;
    gb3 += dg;
    gw3 = fmaf(dg, h2, gw3);
    const float dz2 = dg * theta[OFF_W3 + j] * (1.f - h2 * h2);
    gb2 += dz2;
#pragma unroll 8
    for (int q = 0; q < H; ++q) gW2[q] = fmaf(dz2, __shfl_sync(0xffffffffu, h1, q), gW2[q]);
    // dh1_j = sum_q W2[q][j] dz2_q
    float dh1 = 0.f;
#pragma unroll 8
    for (int q = 0; q < H; ++q) dh1 = fmaf(theta[OFF_W2 + q * H + j], __shfl_sync(0xffffffffu, dz2, q), dh1);
    const float dz1 = dh1 * (1.f - h1 * h1);
    gb1 += dz1;
#pragma unroll
    for (int q = 0; q < IN; ++q) gW1[q] = fmaf(dz1, s[q], gW1[q]);
  }
#pragma unroll
  for (int q = 0; q < IN; ++q) grad[OFF_W1 + j * IN + q] = gW1[q];
  grad[OFF_B1 + j] = gb1;
#pragma unroll
  for (int q = 0; q < H; ++q) grad[OFF_W2 + j * H + q] = gW2[q];
  grad[OFF_B2 + j] = gb2;
  grad[OFF_W3 + j] = gw3;
  if (j == 0) grad[OFF_B3] = gb3;
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m1,
                            float* __restrict__ m2, int count, double lr, double b1, double b2, double eps, double bc1,
                            double bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double g = grad[i];
  const double a = b1 * m1[i] + (1.0 - b1) * g;
  const double v = b2 * m2[i] + (1.0 - b2) * g * g;
  m1[i] = (float)a;
  m2[i] = (float)v;
  theta[i] = (float)(theta[i] - lr * (a / bc1) / (sqrt(v / bc2) + eps));
}

// ---------------------------------------------------------------------------------------
// Training loss of the learned schedule: with Y1 = Z V~ and Y2 = Z^T U~ from a pass,
// P_T Z = F G^T (Eq. (6)), F = [U~, Y1 - U~ C], G = [Y2, V~], C = U~^T Y1; the loss is
// ||F G^T - P Q^T||_F^2 / ||P Q^T||_F^2 and its gradient with respect to Y1 and Y2 (U~, V~,
// P, Q held fixed).  One block; every sum over rows is a fixed-order tree, so the result is
// deterministic.  Work: F (m x 2r), G (n x 2r) in double.
// ---------------------------------------------------------------------------------------
constexpr int LT = 1024;

// out[a * cy + b] = sum over rows of X(i, a) Y(i, b) for a < cx, b < cy; X, Y are callables.
template <typename FX, typename FY>
__device__ void block_gram(int rows, int cx, int cy, FX X, FY Y, double* out, double* red) {
  const int t = threadIdx.x, E = cx * cy;
  for (int e0 = 0; e0 < E; e0 += LT) {
    const int cnt = min(LT, E - e0), groups = LT / cnt;
    const int e = e0 + t % cnt, gidx = t / cnt;
    double acc = 0.0;
    if (gidx < groups) {
      const int a = e / cy, b = e % cy;
      for (int i = gidx; i < rows; i += groups) acc = fma(X(i, a), Y(i, b), acc);
    }
    red[t] = acc;
    __syncthreads();
    if (t < cnt) {
      double s = 0.0;
      for (int g = 0; g < groups; ++g) s += red[g * cnt + t];
      out[e0 + t] = s;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(LT) projection_loss_kernel(const T* __restrict__ Y1, const T* __restrict__ Y2,
                                                             const T* __restrict__ Ut, const T* __restrict__ Vt,
                                                             int m, int n, int R, int r, const double* __restrict__ P,
                                                             const double* __restrict__ Q, int rp, double* loss,
                                                             T* __restrict__ Y1b, T* __restrict__ Y2b,
                                                             double* __restrict__ F, double* __restrict__ G) {
  __shared__ double red[LT];
  __shared__ double C[16 * 16], A[32 * 32], B[32 * 32], Hq[16 * 32], E[32 * 16], PP[16 * 16], QQ[16 * 16], X[16 * 16];
  __shared__ double sc;
  const int t = threadIdx.x, w = 2 * r;
  // G = [Y2, V~]
  for (int e = t; e < n * w; e += LT) {
    const int j = e / w, a = e % w;
    G[e] = a < r ? (double)Y2[(size_t)j * R + a] : (double)Vt[(size_t)j * R + a - r];
  }
  __syncthreads();
  auto gG = [&](int i, int a) { return G[(size_t)i * w + a]; };
  auto gQ = [&](int i, int a) { return Q[(size_t)i * rp + a]; };
  auto gP = [&](int i, int a) { return P[(size_t)i * rp + a]; };
  auto gU = [&](int i, int a) { return (double)Ut[(size_t)i * R + a]; };
  auto gY1 = [&](int i, int a) { return (double)Y1[(size_t)i * R + a]; };
  block_gram(n, w, w, gG, gG, A, red);   // G^T G
  block_gram(n, rp, w, gQ, gG, Hq, red);  // Q^T G
  block_gram(n, rp, rp, gQ, gQ, QQ, red);
  block_gram(m, rp, rp, gP, gP, PP, red);
  block_gram(m, r, r, gU, gY1, C, red);   // C = U~^T Y1
  // F = [U~, Y1 - U~ C]
  for (int i = t; i < m; i += LT) {
    for (int a = 0; a < r; ++a) {
      double v = gY1(i, a);
      for (int q = 0; q < r; ++q) v = fma(-gU(i, q), C[q * r + a], v);
      F[(size_t)i * w + a] = gU(i, a);
      F[(size_t)i * w + r + a] = v;
    }
  }
  __syncthreads();
  auto gF = [&](int i, int a) { return F[(size_t)i * w + a]; };
  block_gram(m, w, w, gF, gF, B, red);    // F^T F
  block_gram(m, w, rp, gF, gP, E, red);   // F^T P
  if (t == 0) {
    double nl = 0.0, ab = 0.0, eh = 0.0;
    for (int a = 0; a < rp; ++a)
      for (int b = 0; b < rp; ++b) nl += PP[a * rp + b] * QQ[a * rp + b];
    for (int a = 0; a < w; ++a)
      for (int b = 0; b < w; ++b) ab += B[a * w + b] * A[a * w + b];
    for (int a = 0; a < w; ++a)
      for (int c = 0; c < rp; ++c) eh += E[a * rp + c] * Hq[c * w + a];
    *loss = (ab - 2.0 * eh + nl) / nl;
    sc = 2.0 / nl;
  }
  __syncthreads();
  const double s2 = sc;
  // Y2b = first r columns of dG = (2 / ||L*||^2) (G F^T F - Q (F^T P)^T)
  for (int e = t; e < n * R; e += LT) {
    const int j = e / R, a = e % R;
    double v = 0.0;
    if (a < r) {
      for (int b = 0; b < w; ++b) v = fma(G[(size_t)j * w + b], B[b * w + a], v);
      for (int c = 0; c < rp; ++c) v = fma(-Q[(size_t)j * rp + c], E[a * rp + c], v);
      v *= s2;
    }
    Y2b[e] = (T)v;
  }
  // dW1 = last r columns of dF = (2 / ||L*||^2) (F G^T G - P Q^T G), written row by row over
  // the W1 half of F (each row is read before it is overwritten)
  __syncthreads();
  for (int i = t; i < m; i += LT) {
    double d[16];
    for (int a = 0; a < r; ++a) {
      double v = 0.0;
      for (int b = 0; b < w; ++b) v = fma(F[(size_t)i * w + b], A[b * w + r + a], v);
      for (int c = 0; c < rp; ++c) v = fma(-P[(size_t)i * rp + c], Hq[c * w + r + a], v);
      d[a] = v * s2;
    }
    for (int a = 0; a < r; ++a) F[(size_t)i * w + r + a] = d[a];
  }
  __syncthreads();
  auto gD = [&](int i, int a) { return F[(size_t)i * w + r + a]; };
  block_gram(m, r, r, gU, gD, X, red);  // X = U~^T dW1
  // Y1b = (I - U~ U~^T) dW1
  for (int e = t; e < m * R; e += LT) {
    const int i = e / R, a = e % R;
    double v = 0.0;
    if (a < r) {
      v = F[(size_t)i * w + r + a];
      for (int q = 0; q < r; ++q) v = fma(-gU(i, q), X[q * r + a], v);
    }
    Y1b[e] = (T)v;
  }
}

}  // namespace
}  // namespace rpca

extern "C" int rpca_schedule_forward(const float* theta, const float* feats, const double* plain, int n, double* zeta,
                                     float* g, void* stream) {
  if (!theta || !feats || !plain || !zeta || n < 0) return RPCA_ERR_INVALID_ARG;
  if (n == 0) return RPCA_OK;
  rpca::schedule_forward_kernel<<<n, 32, 0, static_cast<cudaStream_t>(stream)>>>(theta, feats, plain, n, zeta, g);
  return cudaGetLastError() == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}

extern "C" int rpca_schedule_backward(const float* theta, const float* feats, const double* plain,
                                      const double* zeta_bar, int n, float* theta_bar, void* stream) {
  if (!theta || !feats || !plain || !zeta_bar || !theta_bar || n < 0) return RPCA_ERR_INVALID_ARG;
  rpca::schedule_backward_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(theta, feats, plain, zeta_bar, n,
                                                                                   theta_bar);
  return cudaGetLastError() == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}

extern "C" int rpca_adam_step(float* theta, const float* grad, float* m1, float* m2, int count, int step, double lr,
                              double beta1, double beta2, double eps, void* stream) {
  if (!theta || !grad || !m1 || !m2 || count < 0 || step < 1 || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return RPCA_ERR_INVALID_ARG;
  if (count == 0) return RPCA_OK;
  const double bc1 = 1.0 - pow(beta1, step), bc2 = 1.0 - pow(beta2, step);
  rpca::adam_kernel<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(theta, grad, m1, m2, count, lr,
                                                                                          beta1, beta2, eps, bc1, bc2);
  return cudaGetLastError() == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}

extern "C" int rpca_projection_loss(const void* Y1, const void* Y2, const void* Ut, const void* Vt, int64_t m, int64_t n,
                                    int R, int r, int dtype, const double* P, const double* Q, int rp, double* loss,
                                    void* Y1b, void* Y2b, double* work, void* stream) {
  if (!Y1 || !Y2 || !Ut || !Vt || !P || !Q || !loss || !Y1b || !Y2b || !work || m < 1 || n < 1 || r < 1 || r > R ||
      R > 16 || rp < 1 || rp > 16 || (dtype != RPCA_DTYPE_F32 && dtype != RPCA_DTYPE_F64) || m > (1 << 26) ||
      n > (1 << 26))
    return RPCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* F = work;
  double* G = work + (size_t)m * 2 * r;
  if (dtype == RPCA_DTYPE_F32)
    rpca::projection_loss_kernel<float><<<1, rpca::LT, 0, s>>>(
        static_cast<const float*>(Y1), static_cast<const float*>(Y2), static_cast<const float*>(Ut),
        static_cast<const float*>(Vt), (int)m, (int)n, R, r, P, Q, rp, loss, static_cast<float*>(Y1b),
        static_cast<float*>(Y2b), F, G);
  else
    rpca::projection_loss_kernel<double><<<1, rpca::LT, 0, s>>>(
        static_cast<const double*>(Y1), static_cast<const double*>(Y2), static_cast<const double*>(Ut),
        static_cast<const double*>(Vt), (int)m, (int)n, R, r, P, Q, rp, loss, static_cast<double*>(Y1b),
        static_cast<double*>(Y2b), F, G);
  return cudaGetLastError() == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}
