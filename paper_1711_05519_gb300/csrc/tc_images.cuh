// Operand images of the tensor-core fused pass: the factors of L_k and the bases U~, V~ laid
// out per 128-row / 64-column tile exactly as the MMAs read them from shared memory
// (K-major, 128-byte swizzle), so the pass brings them in with plain bulk copies.
//
//   W image  (per 128 rows, 16 KB):  [W_hi W_hi W_lo 0]  tf32, W = U_k Sigma_k
//   V image  (per 64 columns, 8 KB): [V_hi V_lo V_hi 0]  tf32, so W V^T = W_hi V_hi^T +
//                                    W_hi V_lo^T + W_lo V_hi^T (FP32-level accuracy)
//   U~ image (per 128 rows, 4 KB):   [U~_hi | U~_lo]^T   bf16, two 64-row halves
//   V~ image (per 64 columns, 2 KB): [V~_hi | V~_lo]^T   bf16
// hi = round-to-nearest tf32 / bf16 of x, lo = the rounding of x - hi.  Ranks up to 8.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace rpca {
namespace img {

constexpr int BM = 128, BN = 64;
constexpr int WOP_BYTES = BM * 32 * 4;       // 16 KB [128 x 32] tf32
constexpr int VOP_BYTES = BN * 32 * 4;       // 8 KB  [64 x 32] tf32
constexpr int VTOP_BYTES = 16 * 64 * 2;      // 2 KB  [16 x 64] bf16
constexpr int UTOP_BYTES = 2 * 16 * 64 * 2;  // 4 KB  2 x [16 x 64] bf16

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of (row, byte_in_row) in a K-major tile with 128-byte rows and 128-byte swizzle.
__device__ __forceinline__ int sw128(int row, int byte_in_row) {
  return row * 128 + ((((byte_in_row >> 4) ^ (row & 7)) & 7) << 4) + (byte_in_row & 15);
}

// Row i of the W and U~ images from w[0..7] (row i of W = U Sigma) and u[0..7] (row i of U~),
// both zero beyond the rank.
__device__ __forceinline__ void write_row_images(int i, const float (&w)[8], const float (&u)[8], uint8_t* wop,
                                                 uint8_t* utop) {
  const int rt = i / BM, il = i % BM;
  float hi[8], lo[8];
  __nv_bfloat16 uh[8], ul[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    hi[k] = tf32_rna(w[k]);
    lo[k] = w[k] - hi[k];
    uh[k] = __float2bfloat16_rn(u[k]);
    ul[k] = __float2bfloat16_rn(u[k] - __bfloat162float(uh[k]));
  }
  float* wt = reinterpret_cast<float*>(wop + (size_t)rt * WOP_BYTES);
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    const float v = kk < 8 ? hi[kk] : kk < 16 ? hi[kk - 8] : kk < 24 ? lo[kk - 16] : 0.f;
    wt[sw128(il, 4 * kk) >> 2] = v;
  }
  __nv_bfloat16* ut = reinterpret_cast<__nv_bfloat16*>(utop + (size_t)rt * UTOP_BYTES);
  const int sub = il / 64, kl = il % 64;
#pragma unroll
  for (int nn = 0; nn < 16; ++nn) ut[(sub * 2048 + sw128(nn, 2 * kl)) >> 1] = nn < 8 ? uh[nn] : ul[nn - 8];
}

// Row j of the V and V~ images from v[0..7] (row j of V) and t[0..7] (row j of V~).
__device__ __forceinline__ void write_col_images(int j, const float (&v)[8], const float (&t)[8], uint8_t* vop,
                                                 uint8_t* vtop) {
  const int ct = j / BN, jl = j % BN;
  float hi[8], lo[8];
  __nv_bfloat16 vh[8], vl[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    hi[k] = tf32_rna(v[k]);
    lo[k] = v[k] - hi[k];
    vh[k] = __float2bfloat16_rn(t[k]);
    vl[k] = __float2bfloat16_rn(t[k] - __bfloat162float(vh[k]));
  }
  float* vt = reinterpret_cast<float*>(vop + (size_t)ct * VOP_BYTES);
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    const float x = kk < 8 ? hi[kk] : kk < 16 ? lo[kk - 8] : kk < 24 ? hi[kk - 16] : 0.f;
    vt[sw128(jl, 4 * kk) >> 2] = x;
  }
  __nv_bfloat16* tt = reinterpret_cast<__nv_bfloat16*>(vtop + (size_t)ct * VTOP_BYTES);
#pragma unroll
  for (int nn = 0; nn < 16; ++nn) tt[sw128(nn, 2 * jl) >> 1] = nn < 8 ? vh[nn] : vl[nn - 8];
}

}  // namespace img
}  // namespace rpca
