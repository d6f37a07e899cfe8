// hd_fft_fast.cuh -- inlined Stockham passes for the cluster kernels
// (DFT lengths {1, 3, 5, 9} x 2^a).
//
// Same arithmetic as hd_fft.cuh (Sec. 2 sign convention, radix-2/3/4/5/8/16
// butterflies), specialised for speed:
//   * shared-memory arrays use a padded layout, element i at i + i/16, so the
//     strided stores of the first passes (stride R elements) hit distinct
//     banks;
//   * the twiddles of the length-n DFT come from a table zeta_n^k in shared
//     memory (k < n);
//   * index splits use a float reciprocal with one integer correction instead
//     of integer division (exact for the index range used, < 2^17).
#pragma once
#include "hd_fft.cuh"

namespace hd {

__host__ __device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
// padded stride of an array of n elements, rounded to an even count (16 B)
__host__ __device__ __forceinline__ int pad_stride(int n) { return (pad16(n > 0 ? n - 1 : 0) + 2) & ~1; }

struct DivF {
  float rcp;
  int d;
};
__device__ __forceinline__ DivF make_div(int d) { return DivF{1.0f / (float)d, d}; }
__device__ __forceinline__ int fdiv(int n, DivF v) {
  int q = __float2int_rz(__fmul_rn((float)n, v.rcp));
  const int r = n - q * v.d;
  if (r < 0) --q;
  else if (r >= v.d) ++q;
  return q;
}

template <int R, int SIGN, int PTS>
__device__ __forceinline__ void fstage(float2* base, int stride, int nbuf, int n, int Ns,
                                       const float2* __restrict__ twn) {
  constexpr int BPT = (PTS + R - 1) / R;
  const int nb = n / R;
  const DivF dnb = make_div(nb), dNs = make_div(Ns);
  const int total = nb * nbuf;
  const int T = blockDim.x;
  const int twstep = n / (Ns * R);
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
      for (int r = 0; r < R; ++r) v[b][r] = x[pad16(j + r * nb)];
      if (Ns > 1) {
        const int e = jm * twstep;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = twn[r * e];
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
      float2* y = base + a * stride;
      dft_reg<R, SIGN>(v[b]);
      const int o = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) y[pad16(o + r * Ns)] = v[b][r];
    }
  }
  __syncthreads();
}

// Whole DFT of length n = odd * 2^a, odd in {1, 3, 5, 9}, on nbuf padded
// arrays (base + a * stride), in place; twn[k] = zeta_n^k in shared memory.
// Passes: radix 16 while 16 divides the power of two, one radix-8/4/2 pass for
// the rest of it, then radix 3, 3 x 3 or 5.  (A loop over a runtime radix
// table makes the register allocator spill; this fixed sequence does not.)
// Requires nbuf * n <= PTS * T.
template <int SIGN, int PTS>
__device__ __forceinline__ void cta_fft_fast(float2* base, int stride, int nbuf, int n,
                                             const float2* __restrict__ twn) {
  const int a2 = __ffs(n) - 1;  // power of two in n
  const int odd = n >> a2;
  int Ns = 1;
  for (int i = 0; i < (a2 >> 2); ++i) {
    fstage<16, SIGN, PTS>(base, stride, nbuf, n, Ns, twn);
    Ns *= 16;
  }
  const int rem = a2 & 3;
  if (rem == 3) {
    fstage<8, SIGN, PTS>(base, stride, nbuf, n, Ns, twn);
    Ns *= 8;
  } else if (rem == 2) {
    fstage<4, SIGN, PTS>(base, stride, nbuf, n, Ns, twn);
    Ns *= 4;
  } else if (rem == 1) {
    fstage<2, SIGN, PTS>(base, stride, nbuf, n, Ns, twn);
    Ns *= 2;
  }
  if (odd == 3 || odd == 9) {
    fstage<3, SIGN, PTS>(base, stride, nbuf, n, Ns, twn);
    Ns *= 3;
  }
  if (odd == 9) {
    fstage<3, SIGN, PTS>(base, stride, nbuf, n, Ns, twn);
    Ns *= 3;
  }
  if (odd == 5) {
    fstage<5, SIGN, PTS>(base, stride, nbuf, n, Ns, twn);
    Ns *= 5;
  }
}

}  // namespace hd
