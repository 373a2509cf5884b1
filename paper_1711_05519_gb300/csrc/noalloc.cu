// Support extraction that allocates no device memory.
//
// rpca_get_sparse needs per-row counts and offsets; this entry point keeps them in a
// fixed-size static device array instead of memory allocated by the library, so it can be
// used by code that is not allowed to allocate device memory itself.  The arithmetic is
// the same as the extraction kernels of rpca_get_sparse (FP32 rebuild of L_ij from
// W = U diag(sigma) and V in the same summation order, strict threshold), so both give the
// same support and values.
#include "../../include/rpca.h"
#include "common.cuh"

namespace rpca {
namespace {

constexpr int kMaxRows = RPCA_NOALLOC_MAX_ROWS;

// Scratch shared by every call on a device: [0, m) row counts, [m, 2m+1) row offsets.
// Each call overwrites all 2m+1 entries it uses before reading them.
static __device__ __align__(256) unsigned long long g_rows[2 * kMaxRows + 1];

// Device address of g_rows in the current device's context.  In host code the symbol is only
// a stand-in, so the address is looked up, and it is looked up on every call: the lookup is a
// host-side query that allocates nothing, and a cached address would go stale if the caller
// reset the device (the module, and with it g_rows, is then loaded again, possibly elsewhere).
int scratch_address(unsigned long long** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_rows) != cudaSuccess || !p) return RPCA_ERR_CUDA;
  *out = static_cast<unsigned long long*>(p);
  return RPCA_OK;
}

// One warp per row; 32 columns per step.  WRITE = false counts, true writes.
template <bool WRITE>
__global__ void __launch_bounds__(256) extract_noalloc(const float* __restrict__ D, long long ld, int m, int n, int r,
                                                       const double* __restrict__ U, const double* __restrict__ sig,
                                                       const double* __restrict__ V, float zeta,
                                                       unsigned long long* __restrict__ rows, long long* __restrict__ idx,
                                                       double* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= m) return;
  float w[kMaxR];
#pragma unroll
  for (int k = 0; k < kMaxR; ++k) w[k] = (k < r) ? static_cast<float>(U[(long long)row * r + k] * sig[k]) : 0.f;
  const unsigned long long base = WRITE ? rows[m + row] : 0ull;
  unsigned long long cnt = 0;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    bool s = false;
    float rr = 0.f;
    if (j < n) {
      float l = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxR; ++k)
        if (k < r) l = fmaf(w[k], static_cast<float>(V[(long long)j * r + k]), l);
      rr = D[(long long)row * ld + j] - l;
      s = fabsf(rr) > zeta;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, s);
    if (WRITE && s) {
      const unsigned long long pos = base + cnt + __popc(ballot & ((1u << lane) - 1u));
      idx[pos] = (long long)row * n + j;
      val[pos] = static_cast<double>(rr);
    }
    cnt += __popc(ballot);
  }
  if (!WRITE && lane == 0) rows[row] = cnt;
}

}  // namespace
}  // namespace rpca

using namespace rpca;

extern "C" int rpca_get_sparse_noalloc(const float* D, int64_t m, int64_t n, int64_t ld, int r, const double* U,
                                       const double* sigma, const double* V, double zeta, int64_t* idx,
                                       double* val, int64_t cap, int64_t* nnz, void* stream) {
  if (!D || !U || !sigma || !V || !nnz || m < 1 || n < 1 || ld < n || r < 1 || r > kMaxR || cap < 0 ||
      (cap > 0 && (!idx || !val)) || !(zeta >= 0) || n > (1ll << 30))
    return RPCA_ERR_INVALID_ARG;
  if (m > kMaxRows) return RPCA_ERR_INVALID_ARG;  // the static scratch holds kMaxRows rows
  unsigned long long* rows = nullptr;
  int st = scratch_address(&rows);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((m + 7) / 8);
  extract_noalloc<false><<<blocks, 256, 0, s>>>(D, ld, (int)m, (int)n, r, U, sigma, V, static_cast<float>(zeta), rows,
                                                 nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return RPCA_ERR_CUDA;
  if (launch_scan_rows(rows, rows + m, (int)m, s) != cudaSuccess) return RPCA_ERR_CUDA;
  unsigned long long total = 0;
  if (cudaMemcpyAsync(&total, rows + 2 * m, sizeof(total), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RPCA_ERR_CUDA;
  *nnz = (int64_t)total;
  if ((int64_t)total > cap) return RPCA_ERR_CAPACITY;
  extract_noalloc<true><<<blocks, 256, 0, s>>>(D, ld, (int)m, (int)n, r, U, sigma, V, static_cast<float>(zeta), rows,
                                                (long long*)idx, val);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return RPCA_ERR_CUDA;
  return RPCA_OK;
}
