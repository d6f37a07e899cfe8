// hd_fft_fast.cuh -- per-length pass twiddle tables of the cluster kernels
// (DFT lengths {1, 3, 5, 9} x 2^a, a >= 4), run by cta_fft_struct<.., true>
// of hd_fft.cuh.
//
// Pass (R, Ns) of cta_fft_struct reads zeta_{Ns R}^{r jm} at
// (Ns - 1) + (r - 1) Ns + jm (r = 1..R-1, jm < Ns), contiguous in jm; the
// passes' offsets telescope to a total of n - 1 entries.
#pragma once
#include "hd_fft.cuh"

namespace hd {

// Pass radices of a length n = odd * 2^a, odd in {1, 3, 5, 9}, a >= 4, in the
// order cta_fft_struct runs them: radix 16 while 16 divides the power of two,
// then the rest of it (8/4/2) and the odd factor (3/5/9), as one composite
// pass where merged_tail allows, else as two passes.
__host__ __device__ __forceinline__ int fast_passes(int n, int* Rs) {
  int a2 = 0;
  while (a2 < 30 && ((n >> a2) & 1) == 0) ++a2;
  const int odd = n >> a2;
  const int rem2 = 1 << (a2 & 3);
  int k = 0;
  for (int i = 0; i < (a2 >> 2); ++i) Rs[k++] = 16;
  const int mt = merged_tail(rem2, odd);
  if (mt) {
    Rs[k++] = mt;
  } else {
    if (rem2 > 1) Rs[k++] = rem2;
    if (odd > 1) Rs[k++] = odd;
  }
  return k;
}

// 8-byte asynchronous global -> shared copy (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Per-length table (built once per length, FP64 on the device, see
// hd_tables_plan.cu): entries [0, n-1) are the per-pass twiddles; entries
// [n-1, 2n-1) are zeta_n^l.  Starts the copy of the first part into shared
// memory without waiting: every thread calls cp_async_wait_all() and the CTA
// synchronises before the first DFT reads it.
__device__ __forceinline__ void fill_pass_twiddles_async(float2* tws, int n, const float2* __restrict__ tabm) {
  for (int i = threadIdx.x; i < n - 1; i += blockDim.x) cp_async8(tws + i, tabm + i);
}

}  // namespace hd
