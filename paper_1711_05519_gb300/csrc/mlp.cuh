// The threshold network of the learned schedule: a 6 -> 32 -> 32 -> 1 perceptron with tanh
// hidden units, in FP32, evaluated by one warp (lane j = hidden unit j).
//
// It maps the statistics of iteration k,
//   s_k = [log sigma_1, log(sigma_{r+1} / sigma_1), log err_k, fraction of the support that
//          changed since pass k - 1, (k + 1) / K, log(zeta_k / sigma_1)]
// (sigma_i of P_T(D - S_k), i.e. of the core M_k of Section 2.1; K the unrolled depth of
// training), to a multiplier of the threshold rule of Algorithm 1:
//   zeta_{k+1} = zeta^plain_{k+1} exp(clamp(g(s_k), -log 4, log 4)),
//   zeta^plain_{k+1} = beta (sigma_{r+1} + gamma^{k+1} sigma_1).
// The network is not part of the paper's method; with a zero output layer it gives back the
// paper's rule.
//
// Parameters, packed FP32 (row-major weight matrices, output index first):
//   W1 [32][6] | b1 [32] | W2 [32][32] | b2 [32] | w3 [32] | b3 [1]      (1313 values)
#pragma once

#include <cuda_runtime.h>

namespace rpca {
namespace mlp {

constexpr int IN = 6, H = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
constexpr float kLog4 = 1.38629436111989061883f;

// Statistics of one iteration (see above): the ratios are formed in double, rounded to FP32
// and floored at 1e-37 (a zero singular value or residual), and the logarithms taken in FP32
// (double-precision logarithms are long-latency on this part, and the network reads FP32).
__device__ __forceinline__ float log_floor(double x) { return logf(fmaxf((float)x, 1e-37f)); }

__device__ __forceinline__ void features(double sigma1, double sigma_r1, double err, double change, int k, int depth,
                                         double zeta, float (&s)[IN]) {
  const double s1 = fmax(sigma1, 1e-300);
  s[0] = log_floor(s1);
  s[1] = log_floor(sigma_r1 / s1);
  s[2] = log_floor(err);
  s[3] = (float)change;
  s[4] = (float)(k + 1) / (float)(depth > 0 ? depth : 1);
  s[5] = log_floor(zeta / s1);
}

// Network output g(s) before the clamp, the same in all 32 lanes of the calling warp (all
// lanes must call).  h1, h2: this lane's hidden activations (for the backward pass).
__device__ __forceinline__ float forward_warp(const float* __restrict__ th, const float (&s)[IN], float& h1,
                                              float& h2) {
  const int j = threadIdx.x & 31;
  float a = th[OFF_B1 + j];
#pragma unroll
  for (int i = 0; i < IN; ++i) a = fmaf(th[OFF_W1 + j * IN + i], s[i], a);
  h1 = tanhf(a);
  float b = th[OFF_B2 + j];
#pragma unroll 8
  for (int i = 0; i < H; ++i) b = fmaf(th[OFF_W2 + j * H + i], __shfl_sync(0xffffffffu, h1, i), b);
  h2 = tanhf(b);
  float g = th[OFF_W3 + j] * h2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  return g + th[OFF_B3];
}

__device__ __forceinline__ float clamp_g(float g) { return fminf(fmaxf(g, -kLog4), kLog4); }

}  // namespace mlp
}  // namespace rpca
