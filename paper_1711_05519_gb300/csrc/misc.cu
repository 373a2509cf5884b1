// Small helper kernels: precision conversion of D and the row-offset scan of the sparse
// extraction.
#include <cuda_bf16.h>

#include "common.cuh"

namespace rpca {

namespace {

__global__ void convert_f64_f32(const double* __restrict__ src, long long ld, float* __restrict__ dst, int m,
                                int n) {
  const long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    dst[e] = static_cast<float>(src[i * ld + j]);
  }
}

__global__ void convert_f32_f64(const float* __restrict__ src, long long ld, double* __restrict__ dst, int m,
                                int n) {
  const long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    dst[e] = static_cast<double>(src[i * ld + j]);
  }
}

// bf16 split storage of FP32 D: hi = bf16_rn(d), lo = bf16_rn(d - hi) (d - hi is exact in
// FP32), rows of ld_dst elements; lo may be null.
__global__ void convert_f32_bf16x2(const float* __restrict__ src, long long ld, __nv_bfloat16* __restrict__ hi,
                                   __nv_bfloat16* __restrict__ lo, long long ld_dst, int m, int n) {
  const long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    const float d = src[i * ld + j];
    const __nv_bfloat16 h = __float2bfloat16_rn(d);
    hi[i * ld_dst + j] = h;
    if (lo) lo[i * ld_dst + j] = __float2bfloat16_rn(d - __bfloat162float(h));
  }
}

// Entries of D that are not NaN (partial observation: NaN marks an unobserved entry).
template <typename T>
__global__ void count_observed(const T* __restrict__ D, long long ld, int m, int n, unsigned long long* count) {
  const long long total = (long long)m * n;
  unsigned long long c = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const T d = D[(e / n) * ld + e % n];
    c += (d == d) ? 1ull : 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(count, c);
}

// Exclusive scan of m row counts into m+1 offsets, one block of 1024 threads.  Warp w owns
// the contiguous rows [w seg, (w + 1) seg) (seg a multiple of 32): it sums them with
// coalesced loads, the 32 warp totals are scanned by warp 0, and each warp then walks its
// rows 32 at a time with a shuffle scan.
__global__ void __launch_bounds__(1024) scan_rows(const unsigned long long* __restrict__ cnt,
                                                  unsigned long long* __restrict__ off, int m) {
  __shared__ unsigned long long wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int seg = ((m + 1023) / 1024) * 32;
  const int lo = min(m, w * seg), hi = min(m, lo + seg);
  unsigned long long s = 0;
  for (int i = lo + lane; i < hi; i += 32) s += cnt[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) wsum[w] = s;
  __syncthreads();
  if (w == 0) {
    unsigned long long v = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    wsum[lane] = v;  // inclusive
  }
  __syncthreads();
  unsigned long long base = (w == 0) ? 0ull : wsum[w - 1];
  for (int i0 = lo; i0 < hi; i0 += 32) {
    const int i = i0 + lane;
    const unsigned long long c = (i < hi) ? cnt[i] : 0ull;
    unsigned long long v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (i < hi) off[i] = base + v - c;
    base += __shfl_sync(0xffffffffu, v, 31);
  }
  if (threadIdx.x == 0) off[m] = wsum[31];
}

// Support counts per row and per chunk of kWordChunk words ([word][row] layout): one warp per
// 32 rows and one chunk, lane l the row r0 + l (coalesced), cc[chunk][row] and rowcnt[row] +=.
__global__ void __launch_bounds__(256) words_count(const unsigned* __restrict__ words, int nw, int m,
                                                   unsigned* __restrict__ cc, unsigned long long* __restrict__ rowcnt) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int nrb = (m + 31) / 32;
  const int rb = wid % nrb, ch = wid / nrb;
  const int row = rb * 32 + lane, j0 = ch * kWordChunk;
  if (j0 >= nw || row >= m) return;
  const int j1 = min(nw, j0 + kWordChunk);
  unsigned c = 0;
#pragma unroll 8
  for (int j = j0; j < j1; ++j) c += __popc(words[(size_t)j * m + row]);
  cc[(size_t)ch * m + row] = c;
  if (c) atomicAdd(rowcnt + row, (unsigned long long)c);
}
// Support changes between the learned schedule's two bitmask buffers (the one this pass
// wrote, by the parity of k, against the other): block b counts its share of the words into
// chgP[b] (a fixed split and a fixed-order tree, so the count per block is deterministic).
__global__ void __launch_bounds__(1024) count_mask_changes(const unsigned* __restrict__ masks, long long sz,
                                                           long long nwords, const DevState* st,
                                                           unsigned long long* __restrict__ chgP) {
  __shared__ unsigned part[32];
  if (st->done) return;
  const uint4* cur = reinterpret_cast<const uint4*>(masks + ((st->k & 1) ? sz : 0));
  const uint4* prev = reinterpret_cast<const uint4*>(masks + ((st->k & 1) ? 0 : sz));
  const long long nv = nwords / 4;  // nwords is a multiple of 256
  const long long chunk = (nv + gridDim.x - 1) / gridDim.x;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(nv, lo + chunk);
  unsigned c = 0;
#pragma unroll 4
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint4 a = cur[i], b = prev[i];
    c += __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 32; ++w) t += part[w];
    chgP[blockIdx.x] = t;
  }
}

}  // namespace

cudaError_t launch_count_mask_changes(const unsigned* masks, long long sz, long long nwords, const DevState* st,
                                      unsigned long long* chgP, int nblocks, cudaStream_t s) {
  count_mask_changes<<<nblocks, 1024, 0, s>>>(masks, sz, nwords, st, chgP);
  return cudaGetLastError();
}

cudaError_t launch_words_count(const unsigned* words, int nw, int m, unsigned* cc, unsigned long long* rowcnt,
                               cudaStream_t s) {
  const long long warps = (long long)((m + 31) / 32) * ((nw + kWordChunk - 1) / kWordChunk);
  words_count<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(words, nw, m, cc, rowcnt);
  return cudaGetLastError();
}

cudaError_t launch_scan_rows(const unsigned long long* cnt, unsigned long long* off, int m, cudaStream_t s) {
  scan_rows<<<1, 1024, 0, s>>>(cnt, off, m);
  return cudaGetLastError();
}

cudaError_t launch_count_observed(const void* D, long long ld, int m, int n, bool f32, unsigned long long* count,
                                  cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (f32)
    count_observed<float><<<1024, 256, 0, s>>>(static_cast<const float*>(D), ld, m, n, count);
  else
    count_observed<double><<<1024, 256, 0, s>>>(static_cast<const double*>(D), ld, m, n, count);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_to_f32(const double* src, long long ld, float* dst, int m, int n, cudaStream_t s) {
  convert_f64_f32<<<1024, 256, 0, s>>>(src, ld, dst, m, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_f32_to_f64(const float* src, long long ld, double* dst, int m, int n, cudaStream_t s) {
  convert_f32_f64<<<1024, 256, 0, s>>>(src, ld, dst, m, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_f32_to_bf16x2(const float* src, long long ld, void* hi, void* lo, long long ld_dst, int m,
                                         int n, cudaStream_t s) {
  convert_f32_bf16x2<<<1024, 256, 0, s>>>(src, ld, static_cast<__nv_bfloat16*>(hi), static_cast<__nv_bfloat16*>(lo),
                                          ld_dst, m, n);
  return cudaGetLastError();
}

}  // namespace rpca
