// hd_fft_fast.cuh -- inlined Stockham passes for the cluster kernels
// (DFT lengths {1, 3, 5, 9} x 2^a).
//
// Same arithmetic as hd_fft.cuh (Sec. 2 sign convention, radix-2/3/4/5/8/16
// butterflies), specialised for speed:
//   * element i of an array is stored at swz(i) = i ^ ((i >> 4) & 15) from the
//     array's start (arrays start on 16-element boundaries): a permutation
//     inside each aligned block of 16 float2 (128 bytes), so contiguous runs
//     stay in one 128-byte row and the stride-R stores of the first passes land
//     in distinct banks;
//   * twiddles come from a per-pass table in shared memory: pass (R, Ns) reads
//     zeta_{Ns R}^{r jm} at tws[(Ns - 1) + (r - 1) Ns + jm] (r = 1..R-1, jm < Ns),
//     contiguous in jm; the passes' offsets telescope to a total of n - 1;
//   * index splits use a float reciprocal with one integer correction (exact
//     below 2^17) instead of integer division (recomputed after the barrier:
//     keeping the addresses in registers costs more than the few instructions).
#pragma once
#include "hd_fft.cuh"

namespace hd {

// Largest radix of the power-of-two passes (16, or 8 to fit a pass in 64
// registers for 1024-thread blocks).
#ifndef HD_FAST_MAXR
#define HD_FAST_MAXR 16
#endif
constexpr int kFastMaxRadix = HD_FAST_MAXR;

// swz, swz_stride, DivF / fdiv: hd_fft.cuh.

// One Stockham pass of radix R on nbuf arrays of length n at base + a*stride
// (stride a multiple of 16, indices swizzled per array), twiddles tws (per-pass
// table).
template <int R, int SIGN, int PTS>
__device__ __forceinline__ void fstage(float2* base, int stride, int nbuf, int n, int Ns,
                                       const float2* __restrict__ tws) {
  constexpr int BPT = (PTS + R - 1) / R;
  const int nb = n / R;
  const DivF dnb = make_div(nb), dNs = make_div(Ns);
  const int total = nb * nbuf;
  const int T = blockDim.x;
  const float2* tw_pass = tws + (Ns - 1);
  float2 v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int idx = threadIdx.x + b * T;
    if (idx < total) {
      const int a = fdiv(idx, dnb);
      const int j = idx - a * nb;
      const int jm = j - fdiv(j, dNs) * Ns;
      const float2* x = base + a * stride;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = x[swz(j + r * nb)];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw_pass[(r - 1) * Ns + jm];
          if (SIGN < 0) w.y = -w.y;
          v[b][r] = cmul(v[b][r], w);
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int idx = threadIdx.x + b * T;
    if (idx < total) {
      const int a = fdiv(idx, dnb);
      const int j = idx - a * nb;
      const int jm = j - fdiv(j, dNs) * Ns;
      dft_reg<R, SIGN>(v[b]);
      float2* y = base + a * stride;
      const int o = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) y[swz(o + r * Ns)] = v[b][r];
    }
  }
  __syncthreads();
}

// Pass radices of a length n = odd * 2^a, odd in {1, 3, 5, 9}, in the order
// cta_fft_fast runs them: radix 16 while 16 divides the power of two, one
// radix-8/4/2 pass for the rest of it, then one radix-3/5/9 pass.
__host__ __device__ __forceinline__ int fast_passes(int n, int* Rs) {
  int a2 = 0;
  while (a2 < 30 && ((n >> a2) & 1) == 0) ++a2;
  const int odd = n >> a2;
  int k = 0;
  if (kFastMaxRadix == 8) {
    for (int i = 0; i < a2 / 3; ++i) Rs[k++] = 8;
    if (a2 % 3) Rs[k++] = 1 << (a2 % 3);
  } else {
    for (int i = 0; i < (a2 >> 2); ++i) Rs[k++] = 16;
    if (a2 & 3) Rs[k++] = 1 << (a2 & 3);
  }
  if (odd > 1) Rs[k++] = odd;
  return k;
}

// Per-length table (built once per length, FP64 on the device, see
// hd_tables_plan.cu): entries [0, n-1) are the per-pass twiddles
// zeta_{Ns R}^{r jm} at (Ns - 1) + (r - 1) Ns + jm; entries [n-1, 2n-1) are
// zeta_n^l.  Copy the first part into shared memory (coalesced; no barrier).
__device__ __forceinline__ void fill_pass_twiddles(float2* tws, int n, const float2* __restrict__ tabm) {
  for (int i = threadIdx.x; i < n - 1; i += blockDim.x) tws[i] = __ldg(tabm + i);
}

// Whole DFT of length n on nbuf arrays (base + a * stride, swizzled), in place,
// passes as fast_passes lists them.  (A loop over a runtime radix table
// makes the register allocator spill; this fixed sequence does not.)
// Requires nbuf * n <= PTS * T.
template <int SIGN, int PTS, int MAXR = kFastMaxRadix>
__device__ __forceinline__ void cta_fft_fast(float2* base, int stride, int nbuf, int n,
                                             const float2* __restrict__ tws) {
  const int a2 = __ffs(n) - 1;
  const int odd = n >> a2;
  int Ns = 1;
  if (MAXR == 8) {
    // radix-8 passes while 8 divides the power of two, then one radix-4/2 pass
    for (int i = 0; i < a2 / 3; ++i) {
      fstage<8, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
      Ns *= 8;
    }
    const int rem8 = a2 % 3;
    if (rem8 == 2) {
      fstage<4, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
      Ns *= 4;
    } else if (rem8 == 1) {
      fstage<2, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
      Ns *= 2;
    }
  } else {
    for (int i = 0; i < (a2 >> 2); ++i) {
      fstage<16, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
      Ns *= 16;
    }
  }
  const int rem = (MAXR == 8) ? 0 : (a2 & 3);
  if (rem == 3) {
    fstage<8, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
    Ns *= 8;
  } else if (rem == 2) {
    fstage<4, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
    Ns *= 4;
  } else if (rem == 1) {
    fstage<2, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
    Ns *= 2;
  }
  if (odd == 3) {
    fstage<3, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
    Ns *= 3;
  }
  if (odd == 9) {
    fstage<9, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
    Ns *= 9;
  }
  if (odd == 5) {
    fstage<5, SIGN, PTS>(base, stride, nbuf, n, Ns, tws);
    Ns *= 5;
  }
}

}  // namespace hd
