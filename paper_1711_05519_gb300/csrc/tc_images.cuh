// Operand images of the tensor-core fused pass: the factors of L_k and the bases U~, V~ laid
// out per 128-row / 64-column tile exactly as the MMAs read them from shared memory
// (K-major, swizzled), so the pass brings them in with plain bulk copies.  Two layouts, for
// padded ranks up to RK = 8 and up to RK = 16:
//
//   W image  (per 128 rows):   [W_hi | W_lo]  tf32, W = U_k Sigma_k; rows of 2 RK tf32
//                              (64-byte swizzle for RK = 8: 8 KB; 128-byte for RK = 16: 16 KB)
//   V image  (per 64 columns): [V_hi | V_lo]  tf32, same row format (4 KB / 8 KB)
//                              The pass forms W V^T = W_hi V_hi^T + W_hi V_lo^T + W_lo V_hi^T
//                              (FP32-level accuracy) by pointing the k-steps of its MMAs at
//                              the matching halves.
//   U~ image (per 128 rows, 2 x 2RK x 64 bf16): [U~_hi | U~_lo]^T, two 64-row halves
//   V~ image (per 64 columns, 2RK x 64 bf16):   [V~_hi | V~_lo]^T
// hi = round-to-nearest tf32 / bf16 of x, lo = the rounding of x - hi.  Entries past the
// rank are zero.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace rpca {
namespace img {

constexpr int BM = 128, BN = 64;

template <int RK>
struct Layout {
  static_assert(RK == 8 || RK == 16, "image ranks");
  static constexpr int ROW_BYTES = 2 * RK * 4;                      // [hi | lo] tf32: 64 / 128
  static constexpr int SWIZZLE = RK == 8 ? 64 : 128;                // bytes
  static constexpr int WOP_BYTES = BM * ROW_BYTES;                  // 8 / 16 KB
  static constexpr int VOP_BYTES = BN * ROW_BYTES;                  // 4 / 8 KB
  static constexpr int VTOP_BYTES = 2 * RK * BN * 2;                // 2 / 4 KB
  static constexpr int UTOP_BYTES = 2 * (2 * RK * 64 * 2);          // 4 / 8 KB
};
// buffer sizes that hold either layout
constexpr int WOP_MAX = Layout<16>::WOP_BYTES, VOP_MAX = Layout<16>::VOP_BYTES;
constexpr int VTOP_MAX = Layout<16>::VTOP_BYTES, UTOP_MAX = Layout<16>::UTOP_BYTES;

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of (row, byte_in_row) in a K-major tile with 128-byte rows and 128-byte swizzle
// (the 16-byte chunk index is XORed with address bits 7..9, i.e. with row mod 8).
__device__ __forceinline__ int sw128(int row, int byte_in_row) {
  return row * 128 + ((((byte_in_row >> 4) ^ (row & 7)) & 7) << 4) + (byte_in_row & 15);
}
// Same for 64-byte rows and 64-byte swizzle (chunk index XORed with address bits 7..8, i.e.
// with (row / 2) mod 4).
__device__ __forceinline__ int sw64(int row, int byte_in_row) {
  return row * 64 + ((((byte_in_row >> 4) ^ (row >> 1)) & 3) << 4) + (byte_in_row & 15);
}
template <int RK>
__device__ __forceinline__ int sw_tf32(int row, int k) {
  return RK == 8 ? sw64(row, 4 * k) : sw128(row, 4 * k);
}

// Row i of the W and U~ images from w[0..RK) (row i of W = U Sigma) and u[0..RK) (row i of U~).
template <int RK>
__device__ __forceinline__ void write_row_images(int i, const float (&w)[RK], const float (&u)[RK], uint8_t* wop,
                                                 uint8_t* utop) {
  using Lay = Layout<RK>;
  const int rt = i / BM, il = i % BM;
  float hi[RK], lo[RK];
  __nv_bfloat16 uh[RK], ul[RK];
#pragma unroll
  for (int k = 0; k < RK; ++k) {
    hi[k] = tf32_rna(w[k]);
    lo[k] = w[k] - hi[k];
    uh[k] = __float2bfloat16_rn(u[k]);
    ul[k] = __float2bfloat16_rn(u[k] - __bfloat162float(uh[k]));
  }
  uint8_t* wt = wop + (size_t)rt * Lay::WOP_BYTES;
#pragma unroll
  for (int k = 0; k < RK; ++k) {
    *reinterpret_cast<float*>(wt + sw_tf32<RK>(il, k)) = hi[k];
    *reinterpret_cast<float*>(wt + sw_tf32<RK>(il, RK + k)) = lo[k];
  }
  __nv_bfloat16* ut = reinterpret_cast<__nv_bfloat16*>(utop + (size_t)rt * Lay::UTOP_BYTES);
  const int sub = il / 64, kl = il % 64;
#pragma unroll
  for (int nn = 0; nn < 2 * RK; ++nn)
    ut[(sub * (2 * RK * 128) + sw128(nn, 2 * kl)) >> 1] = nn < RK ? uh[nn % RK] : ul[(nn - RK) % RK];
}

// Row j of the V and V~ images from v[0..RK) (row j of V) and t[0..RK) (row j of V~).
template <int RK>
__device__ __forceinline__ void write_col_images(int j, const float (&v)[RK], const float (&t)[RK], uint8_t* vop,
                                                 uint8_t* vtop) {
  using Lay = Layout<RK>;
  const int ct = j / BN, jl = j % BN;
  float hi[RK], lo[RK];
  __nv_bfloat16 vh[RK], vl[RK];
#pragma unroll
  for (int k = 0; k < RK; ++k) {
    hi[k] = tf32_rna(v[k]);
    lo[k] = v[k] - hi[k];
    vh[k] = __float2bfloat16_rn(t[k]);
    vl[k] = __float2bfloat16_rn(t[k] - __bfloat162float(vh[k]));
  }
  uint8_t* vt = vop + (size_t)ct * Lay::VOP_BYTES;
#pragma unroll
  for (int k = 0; k < RK; ++k) {
    *reinterpret_cast<float*>(vt + sw_tf32<RK>(jl, k)) = hi[k];
    *reinterpret_cast<float*>(vt + sw_tf32<RK>(jl, RK + k)) = lo[k];
  }
  __nv_bfloat16* tt = reinterpret_cast<__nv_bfloat16*>(vtop + (size_t)ct * Lay::VTOP_BYTES);
#pragma unroll
  for (int nn = 0; nn < 2 * RK; ++nn) tt[sw128(nn, 2 * jl) >> 1] = nn < RK ? vh[nn % RK] : vl[(nn - RK) % RK];
}

}  // namespace img
}  // namespace rpca
