// Fused streaming pass of one AccAltProj iteration (SIMT form), templated on the
// arithmetic type T (float or double) and the compiled rank R.
//
// For every entry of D (one read of D from HBM per iteration) the pass
//   rebuilds L_ij = sum_k W_ik V_jk                  (L_k = U_k Sigma_k V_k^T, W = U_k Sigma_k)
//   forms R_ij = D_ij - L_ij and the hard threshold S_ij = R_ij if |R_ij| > zeta_k
//                                                   (Eq. (10), strict inequality)
//   accumulates sum R_ij^2 over unthresholded entries (the numerator of err_k, Eq. (11))
//   forms Z_ij = D_ij - S_ij (= L_ij on the support, D_ij elsewhere)
//   accumulates Y1 = Z V~_k and Y2 = Z^T U~_k          (the two tall-skinny products of
//                                                   Section 2.1 feeding the QR route)
// so S_k, err_k and the products for L_{k+1} all come from the same read.
//
// Work decomposition: a CTA owns a BH x BW unit of D.  Its 8 warps sweep the unit in row
// blocks of 8*TM rows; within a row block each lane owns VW consecutive columns of a
// 32*VW-column sub-chunk (one 16-byte vector load per row).  Y1 for the warp's TM rows
// stays in registers across the whole unit width and is reduced across lanes once per
// row block; Y2 for the lane's columns is summed over the TM rows in registers and added
// into a per-warp shared-memory slot.  At the end of the unit the 8 slots are summed in
// a fixed order and written as the unit's partial.  Partials are reduced in FP64 by the
// tall-skinny kernel, so results do not depend on scheduling.
#pragma once

#include "common.cuh"

namespace rpca {

template <typename T, int R>
struct PassCfg;

template <int R>
struct PassCfg<float, R> {
  static constexpr int VW = 4;
  static constexpr int TM = (R <= 6) ? 8 : 4;
  static constexpr int BH = (R <= 8) ? 512 : 256;
  static constexpr int BW = (R <= 6) ? 512 : 256;
};

template <int R>
struct PassCfg<double, R> {
  static constexpr int VW = 2;
  static constexpr int TM = (R <= 6) ? 4 : 2;
  static constexpr int BH = (R <= 8) ? 256 : 128;
  static constexpr int BW = (R <= 6) ? 256 : 128;
};

template <typename T, int R>
struct PassLayout {
  using C = PassCfg<T, R>;
  static constexpr int WARPS = 8;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int SCW = 32 * C::VW;          // sub-chunk width
  static constexpr int NSC = C::BW / SCW;          // sub-chunks per unit
  static constexpr int NRB = C::BH / (WARPS * C::TM);  // row blocks per unit
  // shared memory: W, U~ rows [BH][R]; V, V~ columns [R][BW]; Y2 slots [WARPS][R][BW]
  static constexpr size_t SMEM = sizeof(T) * (size_t)R * (2 * C::BH + 2 * C::BW + WARPS * C::BW);
  static_assert(C::BH % (WARPS * C::TM) == 0, "row blocks");
  static_assert(C::BW % SCW == 0, "sub-chunks");
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// L_ij for one entry: fixed summation order k = 0..R-1 (the extraction kernels use the
// same order so that their threshold decisions agree with the pass).
template <typename T, int R>
__device__ __forceinline__ T rebuild(const T* w, const T* v) {
  T l = T(0);
#pragma unroll
  for (int k = 0; k < R; ++k) l = fma(w[k], v[k], l);
  return l;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

// Loads D[i][c .. c+VW) with zero fill past the matrix edge.
template <typename T, int VW>
__device__ __forceinline__ void load_row_vec(const T* __restrict__ D, long long ld, int m, int n, int i,
                                             int c, bool vec, T (&out)[VW]) {
  if (i < m && vec && c + VW <= n) {
    static_assert(sizeof(typename Vec16<T>::type) == VW * sizeof(T), "one 16-byte vector per lane");
    const typename Vec16<T>::type x =
        __ldcs(reinterpret_cast<const typename Vec16<T>::type*>(D + (long long)i * ld + c));
    const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int e = 0; e < VW; ++e) out[e] = xs[e];
  } else {
#pragma unroll
    for (int e = 0; e < VW; ++e)
      out[e] = (i < m && c + e < n) ? __ldcs(D + (long long)i * ld + c + e) : T(0);
  }
}

// bf16 storage of D: D[i][c .. c+4) = hi (+ lo when use_lo) with zero fill past the matrix
// edge; rows of ld elements, ld a multiple of 8 and c a multiple of 4 (8-byte loads).
__device__ __forceinline__ void load_row_bf16(const uint16_t* __restrict__ hi, const uint16_t* __restrict__ lo,
                                              bool use_lo, long long ld, int m, int n, int i, int c,
                                              float (&out)[4]) {
  const long long o = (long long)i * ld + c;
  if (i < m && c + 4 <= n) {
    const uint2 h = __ldcs(reinterpret_cast<const uint2*>(hi + o));
    out[0] = __uint_as_float(h.x << 16);
    out[1] = __uint_as_float(h.x & 0xffff0000u);
    out[2] = __uint_as_float(h.y << 16);
    out[3] = __uint_as_float(h.y & 0xffff0000u);
    if (use_lo) {
      const uint2 l = __ldcs(reinterpret_cast<const uint2*>(lo + o));
      out[0] += __uint_as_float(l.x << 16);
      out[1] += __uint_as_float(l.x & 0xffff0000u);
      out[2] += __uint_as_float(l.y << 16);
      out[3] += __uint_as_float(l.y & 0xffff0000u);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool in = i < m && c + e < n;
      float x = in ? __uint_as_float((uint32_t)hi[o + e] << 16) : 0.f;
      if (in && use_lo) x += __uint_as_float((uint32_t)lo[o + e] << 16);
      out[e] = x;
    }
  }
}

// DM = 0: D in the pass precision T; DM = 1 (T = float): bf16 storage of D (PassArgs.dm).
template <typename T, int R, int DM>
__global__ void __launch_bounds__(256, 1) fused_pass_kernel(PassArgs a) {
  using C = PassCfg<T, R>;
  using Lay = PassLayout<T, R>;
  constexpr int VW = C::VW, TM = C::TM, BH = C::BH, BW = C::BW;
  constexpr int WARPS = Lay::WARPS, SCW = Lay::SCW, NSC = Lay::NSC, NRB = Lay::NRB;
  if (a.st->done) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);   // [BH][R]
  T* sUt = sW + BH * R;                     // [BH][R]
  T* sV = sUt + BH * R;                     // [R][BW]
  T* sVt = sV + R * BW;                     // [R][BW]
  T* sY2 = sVt + R * BW;                    // [WARPS][R][BW]

  const T* __restrict__ D = static_cast<const T*>(a.D);
  const T* __restrict__ W = static_cast<const T*>(a.W);
  const T* __restrict__ V = static_cast<const T*>(a.V);
  const T* __restrict__ Ut = static_cast<const T*>(a.Ut);
  const T* __restrict__ Vt = static_cast<const T*>(a.Vt);
  const int m = a.m, n = a.n;
  const int row0 = blockIdx.y * BH, col0 = blockIdx.x * BW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int e = tid; e < BH * R; e += Lay::THREADS) {
    const int i = row0 + e / R;
    sW[e] = (i < m) ? W[(long long)row0 * R + e] : T(0);
    sUt[e] = (i < m) ? Ut[(long long)row0 * R + e] : T(0);
  }
  for (int e = tid; e < BW * R; e += Lay::THREADS) {
    const int cl = e / R, k = e % R, j = col0 + cl;
    sV[k * BW + cl] = (j < n) ? V[(long long)j * R + k] : T(0);
    sVt[k * BW + cl] = (j < n) ? Vt[(long long)j * R + k] : T(0);
  }
  for (int e = tid; e < WARPS * R * BW; e += Lay::THREADS) sY2[e] = T(0);
  __syncthreads();

  const T zeta = static_cast<T>(a.st->zeta);
  // partial observation: a NaN entry of D is unobserved (Z = L there, outside the support and
  // the residual); an observed entry outside the support gets Z = L + (D - L) / p
  const bool po = a.partial != 0;
  const T invp = static_cast<T>(a.st->inv_p);
  const bool vec = a.vec != 0;
  const bool use_lo = DM == 1 && a.Dlo != nullptr && a.st->use_lo != 0;
  // residual: the TM x VW terms of one sub-chunk are summed in T, the sub-chunk sums in
  // double (one FP32 chain over the ~10^3 terms a thread sees would bias err_k)
  double res = 0.0;
  unsigned nnz = 0, chg = 0;
  T* mySlot = sY2 + warp * R * BW;
  // support bitmasks (learned schedule): word (i, chunk, c) holds, in bit l, the entry of row
  // i at column chunk * SCW + l * VW + c; pass k writes buffer k % 2 and compares with the other
  const bool track = a.masks != nullptr;
  const long long mask_sz = a.mask_words;
  unsigned* mask_new = track ? a.masks + ((a.st->k & 1) ? mask_sz : 0) : nullptr;
  const unsigned* mask_old = track ? a.masks + ((a.st->k & 1) ? 0 : mask_sz) : nullptr;

  for (int rb = 0; rb < NRB; ++rb) {
    const int rl0 = rb * WARPS * TM + warp * TM;  // local row of this warp's first row
    T y1[TM][R];
#pragma unroll
    for (int t = 0; t < TM; ++t)
#pragma unroll
      for (int k = 0; k < R; ++k) y1[t][k] = T(0);

#pragma unroll 1
    for (int sc = 0; sc < NSC; ++sc) {
      const int cl = sc * SCW + lane * VW;  // local column of this lane's first column
      T d[TM][VW];
#pragma unroll
      for (int t = 0; t < TM; ++t) {
        if constexpr (DM == 1) {
          static_assert(VW == 4, "bf16 storage: four columns per lane");
          load_row_bf16(static_cast<const uint16_t*>(a.D), static_cast<const uint16_t*>(a.Dlo), use_lo, a.ld, m,
                        n, row0 + rl0 + t, col0 + cl, d[t]);
        } else {
          load_row_vec<T, VW>(D, a.ld, m, n, row0 + rl0 + t, col0 + cl, vec, d[t]);
        }
      }
      T v[VW][R], vt[VW][R], y2[VW][R];
#pragma unroll
      for (int k = 0; k < R; ++k)
#pragma unroll
        for (int c = 0; c < VW; ++c) {
          v[c][k] = sV[k * BW + cl + c];
          vt[c][k] = sVt[k * BW + cl + c];
          y2[c][k] = T(0);
        }
      T rsc = T(0);
      static_assert(TM * VW <= 32, "support bits of a sub-chunk fit one word");
      unsigned sb = 0;
#pragma unroll
      for (int t = 0; t < TM; ++t) {
        T w[R], ut[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
          w[k] = sW[(rl0 + t) * R + k];
          ut[k] = sUt[(rl0 + t) * R + k];
        }
#pragma unroll
        for (int c = 0; c < VW; ++c) {
          const T l = rebuild<T, R>(w, v[c]);
          const T rr = d[t][c] - l;
          const bool s = fabs(rr) > zeta;  // false for NaN
          const bool keep_l = s || (po && !(d[t][c] == d[t][c]));
          rsc = keep_l ? rsc : fma(rr, rr, rsc);
          nnz += s ? 1u : 0u;
          sb |= (s ? 1u : 0u) << (t * VW + c);
          const T z = keep_l ? l : (po ? fma(rr, invp, l) : d[t][c]);
#pragma unroll
          for (int k = 0; k < R; ++k) {
            y1[t][k] = fma(z, vt[c][k], y1[t][k]);
            y2[c][k] = fma(z, ut[k], y2[c][k]);
          }
        }
      }
      res += static_cast<double>(rsc);
      if (track) {
        const long long chunk = (col0 + sc * SCW) / SCW;
#pragma unroll
        for (int t = 0; t < TM; ++t)
#pragma unroll
          for (int c = 0; c < VW; ++c) {
            const unsigned w = __ballot_sync(0xffffffffu, (sb >> (t * VW + c)) & 1u);
            const int i = row0 + rl0 + t;
            if (lane == t * VW + c && i < m) {
              const long long wi = (long long)i * a.mask_wr + chunk * VW + c;
              const unsigned old = mask_old[wi];
              mask_new[wi] = w;
              chg += __popc(w ^ old);
            }
          }
      }
#pragma unroll
      for (int k = 0; k < R; ++k)
#pragma unroll
        for (int c = 0; c < VW; ++c) mySlot[k * BW + cl + c] += y2[c][k];
    }
    // Y1 partial of the warp's TM rows over the unit width.
#pragma unroll
    for (int t = 0; t < TM; ++t) {
      const int i = row0 + rl0 + t;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const T s = warp_sum(y1[t][k]);
        if (lane == 0 && i < m) static_cast<T*>(a.P1)[((long long)blockIdx.x * m + i) * R + k] = s;
      }
    }
  }
  __syncthreads();
  // Y2 partial of the unit: fixed-order sum of the per-warp slots.
  for (int e = tid; e < BW * R; e += Lay::THREADS) {
    const int cl = e / R, k = e % R, j = col0 + cl;
    T s = T(0);
#pragma unroll
    for (int w = 0; w < WARPS; ++w) s += sY2[(w * R + k) * BW + cl];
    if (j < n) static_cast<T*>(a.P2)[((long long)blockIdx.y * n + j) * R + k] = s;
  }
  // CTA totals of the residual and the support size.
  __shared__ double sres[8];
  __shared__ unsigned long long snnz[8], schg[8];
  double rd = warp_sum(res);
  unsigned long long nz = nnz, cz = chg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
    cz += __shfl_xor_sync(0xffffffffu, cz, o);
  }
  if (lane == 0) {
    sres[warp] = rd;
    snnz[warp] = nz;
    schg[warp] = cz;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    unsigned long long z = 0, cc = 0;
    for (int w = 0; w < WARPS; ++w) {
      t += sres[w];
      z += snnz[w];
      cc += schg[w];
    }
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    a.resP[cta] = t;
    a.nnzP[cta] = z;
    if (track) a.chgP[cta] = cc;
  }
}

template <typename T, int R, int DM>
cudaError_t launch_pass_dm(const PassArgs& a, cudaStream_t s) {
  using C = PassCfg<T, R>;
  using Lay = PassLayout<T, R>;
  static unsigned long long attr_epoch = 0;
  if (attr_epoch != g_attr_epoch) {
    cudaError_t e = cudaFuncSetAttribute(fused_pass_kernel<T, R, DM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Lay::SMEM);
    if (e != cudaSuccess) return e;
    attr_epoch = g_attr_epoch;
  }
  dim3 grid((a.n + C::BW - 1) / C::BW, (a.m + C::BH - 1) / C::BH);
  fused_pass_kernel<T, R, DM><<<grid, Lay::THREADS, Lay::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int R>
cudaError_t launch_pass_t(const PassArgs& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.dm == 1) return launch_pass_dm<T, R, 1>(a, s);
  }
  if (a.dm != 0) return cudaErrorInvalidValue;
  return launch_pass_dm<T, R, 0>(a, s);
}

// ---------------------------------------------------------------------------------------
// Sparse extraction: supp(S_k) and its values, in ascending linear index order.
// One warp per row, 32 columns per step; the decision uses rebuild<T,R> and the same
// comparison as the pass, so the support agrees with the pass's nnz.
// ---------------------------------------------------------------------------------------
template <typename T, int R, bool WRITE>
__global__ void __launch_bounds__(256) extract_kernel(ExtractArgs a) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= a.m) return;
  const T* __restrict__ D = static_cast<const T*>(a.D);
  const T* __restrict__ W = static_cast<const T*>(a.W);
  const T* __restrict__ V = static_cast<const T*>(a.V);
  const T zeta = static_cast<T>(a.st->zeta);
  T w[R];
#pragma unroll
  for (int k = 0; k < R; ++k) w[k] = W[(long long)row * R + k];
  unsigned long long base = WRITE ? a.rowoff[row] : 0ull;
  unsigned long long cnt = 0;
  for (int j0 = 0; j0 < a.n; j0 += 32) {
    const int j = j0 + lane;
    bool s = false;
    T rr = T(0);
    if (j < a.n) {
      T v[R];
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = V[(long long)j * R + k];
      const T l = rebuild<T, R>(w, v);
      rr = D[(long long)row * a.ld + j] - l;
      s = fabs(rr) > zeta;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, s);
    if (WRITE && s) {
      const unsigned long long pos = base + cnt + __popc(ballot & ((1u << lane) - 1u));
      a.idx[pos] = (long long)row * a.n + j;
      a.val[pos] = static_cast<double>(rr);
    }
    cnt += __popc(ballot);
  }
  if (!WRITE && lane == 0) a.rowcnt[row] = cnt;
}

// The ordered write from the support words of the tensor-core pass (the bit of column j of
// row i is set iff |D_ij - L_ij| > zeta_k in that pass; [word][row] layout).  One block per 32
// rows and chunk of kWordChunk words (1024 columns): the block stages the chunk's rows of V
// and its 32 x 32 words in shared memory (coalesced), then each warp takes 4 of the rows.  A
// row's chunk starts at the row's offset (rowoff) plus the counts of its earlier chunks (cc);
// the warp scans its words' bit counts and takes the chunk's entries in order, lane l the
// entries l, l + 32, ... (UNR per lane at once, so their loads of D are in flight together):
// the word by a binary search over the scan, the column by the rank of the bit, and
// S_ij = D_ij - L_ij rebuilt there (D is read only where a 32-byte sector holds a support
// entry).  Consecutive lanes write consecutive positions.
template <int R>
__global__ void __launch_bounds__(256) extract_words_kernel(ExtractArgs a, const unsigned* __restrict__ words,
                                                            const unsigned* __restrict__ cc, int nw) {
  constexpr int UNR = 4, RB = 32, COLS = 32 * kWordChunk;
  extern __shared__ float vs[];  // [COLS][R]: the chunk's rows of V
  __shared__ unsigned ws[kWordChunk][RB];
  __shared__ unsigned long long rbase[RB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nrb = (a.m + RB - 1) / RB;
  const int rb = blockIdx.x % nrb, ch = blockIdx.x / nrb;
  const int r0 = rb * RB, j0 = ch * kWordChunk, c0 = 32 * j0;
  const int ncols = min(COLS, a.n - c0);
  const float* __restrict__ D = static_cast<const float*>(a.D);
  const float* __restrict__ W = static_cast<const float*>(a.W);
  const float* __restrict__ V = static_cast<const float*>(a.V);
  for (int e = threadIdx.x; e < ncols * R; e += blockDim.x) vs[e] = V[(long long)c0 * R + e];
  for (int e = threadIdx.x; e < kWordChunk * RB; e += blockDim.x) {
    const int jj = e / RB, rr = e % RB;
    ws[jj][rr] = (j0 + jj < nw && r0 + rr < a.m) ? words[(size_t)(j0 + jj) * a.m + r0 + rr] : 0u;
  }
  if (threadIdx.x < RB) {
    const int row = r0 + threadIdx.x;
    unsigned long long b = 0;
    if (row < a.m) {
      b = a.rowoff[row];
      for (int c = 0; c < ch; ++c) b += cc[(size_t)c * a.m + row];
    }
    rbase[threadIdx.x] = b;
  }
  __syncthreads();
  for (int rr = warp; rr < RB; rr += 8) {
    const int row = r0 + rr;
    if (row >= a.m) break;
    const unsigned wd = ws[lane][rr];
    const unsigned c = __popc(wd);
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned excl = incl - c;
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    float w[R];
#pragma unroll
    for (int k = 0; k < R; ++k) w[k] = W[(long long)row * R + k];
    const unsigned long long base = rbase[rr];
    for (unsigned e0 = 0; e0 < total; e0 += 32 * UNR) {
      int col[UNR];
      float d[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const unsigned e = e0 + 32u * u + lane;
        // source lane: the number of lanes whose inclusive count is <= e
        int src = 0;
#pragma unroll
        for (int b = 16; b > 0; b >>= 1) {
          const unsigned t = __shfl_sync(0xffffffffu, incl, src + b - 1);
          if (t <= e) src += b;
        }
        unsigned wsrc = __shfl_sync(0xffffffffu, wd, src & 31);
        const unsigned es = __shfl_sync(0xffffffffu, excl, src & 31);
        col[u] = -1;
        if (e < total) {
          for (unsigned q = es; q < e; ++q) wsrc &= wsrc - 1u;  // drop the lower set bits
          col[u] = 32 * src + (__ffs(wsrc) - 1);               // column within the chunk
          d[u] = D[(long long)row * a.ld + c0 + col[u]];
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        if (col[u] >= 0) {
          float v[R];
#pragma unroll
          for (int k = 0; k < R; ++k) v[k] = vs[col[u] * R + k];
          const unsigned long long pos = base + e0 + 32u * u + lane;
          a.idx[pos] = (long long)row * a.n + c0 + col[u];
          a.val[pos] = static_cast<double>(d[u] - rebuild<float, R>(w, v));
        }
      }
    }
  }
}

template <int R>
cudaError_t launch_extract_words_t(const ExtractArgs& a, const unsigned* words, const unsigned* cc, int nw,
                                   cudaStream_t s) {
  const long long blocks = (long long)((a.m + 31) / 32) * ((nw + kWordChunk - 1) / kWordChunk);
  const int vbytes = 32 * kWordChunk * R * (int)sizeof(float);  // up to 64 KB
  cudaError_t e = cudaFuncSetAttribute(extract_words_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, vbytes);
  if (e != cudaSuccess) return e;
  extract_words_kernel<R><<<(unsigned)blocks, 256, vbytes, s>>>(a, words, cc, nw);
  return cudaGetLastError();
}

template <typename T, int R>
cudaError_t launch_extract_count_t(const ExtractArgs& a, cudaStream_t s) {
  extract_kernel<T, R, false><<<(a.m + 7) / 8, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int R>
cudaError_t launch_extract_write_t(const ExtractArgs& a, cudaStream_t s) {
  extract_kernel<T, R, true><<<(a.m + 7) / 8, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rpca
