// hd_fft.cuh -- CTA-level mixed-radix Stockham FFT in shared memory (sm_103a).
//
// Every residue transform of the hybrid method (Sec. 2, Eqs. forwardr and
// accumulator) needs DFTs of length m of data held on chip.  This header holds
// the building blocks: complex helpers, register butterflies of radix
// 2/3/4/5/8/16 plus a generic radix for any other prime factor, and a stage
// loop that runs a Stockham autosort pass in place (all loads of a stage go to
// registers, a barrier, then the stores), so no ping-pong buffer is needed.
//
// Sign convention (Sec. 2): zeta_N = exp(+2 pi i / N); SIGN = +1 computes
// sum_j x_j zeta_n^{jk} (the forward transform of the paper), SIGN = -1 the
// backward transform.  No scaling.
//
// Twiddles come from one table tw[k] = zeta_N^k (k < N) per padded length N,
// generated in FP64 and rounded once to FP32; a length-n DFT with n | N reads
// zeta_n^x = tw[x * (N / n)].
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hd_bfly.cuh"

namespace hd {

constexpr int kMaxStages = 24;

// Radix sequence of one DFT length; the product of radix[0..nst) equals n.
struct FftPlan {
  int n;
  int nst;
  int radix[kMaxStages];
};

// zeta_N^{SIGN * k} from the table (k already reduced into [0, N)).
template <int SIGN>
__device__ __forceinline__ float2 tw_get(const float2* __restrict__ tw, int k) {
  float2 w = __ldg(tw + k);
  if (SIGN < 0) w.y = -w.y;
  return w;
}

// ---------------------------------------------------------------------------
// One Stockham pass of radix R over `nbuf` arrays of length n, stored at
// base + a * stride (a < nbuf).  Butterfly j (< n/R) reads x[j + r n/R],
// multiplies by zeta_{Ns R}^{SIGN r (j mod Ns)}, transforms, and writes
// y[(j / Ns) Ns R + (j mod Ns) + r Ns].  In place: loads, barrier, stores.
// Requires nbuf * n <= PTS * blockDim.x (checked by the host planner).
// ---------------------------------------------------------------------------
template <int R, int SIGN, int PTS>
__device__ __forceinline__ void fft_stage(float2* base, int stride, int nbuf, int n, int Ns,
                                          const float2* __restrict__ tw, int twmul) {
  constexpr int BPT = (PTS + R - 1) / R;
  const int nb = n / R;
  const int total = nb * nbuf;
  const int T = blockDim.x;
  const int twstep = twmul * (n / (Ns * R));
  float2 v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int idx = threadIdx.x + b * T;
    if (idx < total) {
      const int a = idx / nb;
      const int j = idx - a * nb;
      const float2* x = base + (size_t)a * stride;
      const int jm = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = x[j + r * nb];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], tw_get<SIGN>(tw, r * jm * twstep));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int idx = threadIdx.x + b * T;
    if (idx < total) {
      const int a = idx / nb;
      const int j = idx - a * nb;
      float2* y = base + (size_t)a * stride;
      const int jm = j % Ns;
      dft_reg<R, SIGN>(v[b]);
      const int o = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) y[o + r * Ns] = v[b][r];
    }
  }
  __syncthreads();
}

// Generic radix (any R, used for prime factors other than 2, 3, 5): each
// thread computes whole output points as direct sums over the R inputs of
// its butterfly, keeps them in registers until the barrier, then stores.
template <int SIGN, int PTS>
__device__ __forceinline__ void fft_stage_generic(float2* base, int stride, int nbuf, int n, int R, int Ns,
                                                  const float2* __restrict__ tw, int twmul) {
  const int total = n * nbuf;
  const int T = blockDim.x;
  const int nb = n / R;
  const int step_tw = n / (Ns * R);  // zeta_{Ns R} = zeta_n^{step_tw}
  const int step_r = n / R;          // zeta_R = zeta_n^{step_r}
  float2 out[PTS];
#pragma unroll
  for (int k = 0; k < PTS; ++k) {
    const int o = threadIdx.x + k * T;
    if (o < total) {
      const int a = o / n;
      const int oo = o - a * n;
      const int jm = oo % Ns;
      const int r = (oo / Ns) % R;
      const int j = (oo / (Ns * R)) * Ns + jm;
      const float2* x = base + (size_t)a * stride;
      float2 acc = make_float2(0.f, 0.f);
      for (int r2 = 0; r2 < R; ++r2) {
        const int e = (r2 * jm * step_tw + ((r * r2) % R) * step_r) % n;
        const float2 w = tw_get<SIGN>(tw, e * twmul);
        const float2 xv = x[j + r2 * nb];
        acc.x = fmaf(xv.x, w.x, fmaf(-xv.y, w.y, acc.x));
        acc.y = fmaf(xv.x, w.y, fmaf(xv.y, w.x, acc.y));
      }
      out[k] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PTS; ++k) {
    const int o = threadIdx.x + k * T;
    if (o < total) {
      const int a = o / n;
      base[(size_t)a * stride + (o - a * n)] = out[k];
    }
  }
  __syncthreads();
}


// ---------------------------------------------------------------------------
// Split-precision radix-16 pass on tensor cores.
//
// The 16-point butterflies of a pass are a matrix product: with X the
// (butterflies x 16) matrix of twiddled inputs and W_kr = zeta_16^{SIGN r k},
// Y = X W.  In real form, [Re X, Im X] (16 x 32) times
//   B = [[Re W, Im W], [-Im W, Re W]]  (32 x 32)
// gives [Re Y, Im Y].  Each operand is split as x = x_hi + x_lo with
// x_hi = bf16(x), x_lo = bf16(x - x_hi); the product is accumulated in FP32 as
// hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-16 relative, is dropped).  One
// warp computes 16 butterflies (one m16n8k16 row tile) with 4 column tiles x
// 2 k-steps x 3 products = 24 mma.sync.  Fragment layouts are those of the
// PTX m16n8k16 bf16 shape (lane = 4 g + t): A rows g, g+8, cols 2t, 2t+1,
// 2t+8, 2t+9; B rows 2t, 2t+1, 2t+8, 2t+9, col g; C rows g, g+8, cols 2t, 2t+1.
// In place like fft_stage: all tiles are computed into registers, a barrier,
// then the stores.  Requires ceil(nbuf n / 256) <= 2 * (blockDim.x / 32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ void split_bf16(float x, float& h, float& l) {
  h = __bfloat162float(__float2bfloat16_rn(x));
  l = x - h;
}
__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B entry (row K of 32, col c of 32) of the real-form DFT-16 matrix.
template <int SIGN>
__device__ __forceinline__ float dft16_real_entry(int K, int c) {
  // cos / sin of 2 pi j / 16, j = 0..15
  const float C16[16] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f,
                         0.0f, -0.38268343236508977173f, -0.70710678118654752440f, -0.92387953251128675613f,
                         -1.0f, -0.92387953251128675613f, -0.70710678118654752440f, -0.38268343236508977173f,
                         0.0f, 0.38268343236508977173f, 0.70710678118654752440f, 0.92387953251128675613f};
  const int r = K & 15, k = c & 15;
  const int e = (r * k) & 15;
  const float cr = C16[e];
  const float si = SIGN * C16[(e + 12) & 15];  // sin(x) = cos(x - pi/2)
  if (c < 16) return (K < 16) ? cr : -si;      // Re Y: Re W from Re X, -Im W from Im X
  return (K < 16) ? si : cr;                   // Im Y: Im W from Re X, Re W from Im X
}

template <int SIGN, int PTS>
__device__ __forceinline__ void fft_stage_tc16(float2* base, int stride, int nbuf, int n, int Ns,
                                               const float2* __restrict__ tw, int twmul) {
  constexpr int TPW = 2;
  const int nb = n / 16;
  const int total = nb * nbuf;
  const int ntiles = (total + 15) >> 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int twstep = twmul * (n / (Ns * 16));
  const int rr[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  // constant B fragments, hi and lo parts
  uint32_t bh[4][2][2], bl[4][2][2];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int K0 = 16 * kk + 2 * t + 8 * hh, col = 8 * nt + g;
        float h0, l0, h1, l1;
        split_bf16(dft16_real_entry<SIGN>(K0, col), h0, l0);
        split_bf16(dft16_real_entry<SIGN>(K0 + 1, col), h1, l1);
        bh[nt][kk][hh] = pack_bf16x2(h0, h1);
        bl[nt][kk][hh] = pack_bf16x2(l0, l1);
      }
  float acc[TPW][4][4];
  int bid[TPW][2];
#pragma unroll
  for (int tt = 0; tt < TPW; ++tt) {
    const int tile = warp + tt * nwarps;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[tt][nt][e] = 0.f;
    bid[tt][0] = bid[tt][1] = -1;
    if (tile < ntiles) {
      float2 xv[2][4];
#pragma unroll
      for (int row = 0; row < 2; ++row) {
        const int b = tile * 16 + g + 8 * row;
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[row][i] = make_float2(0.f, 0.f);
        if (b < total) {
          bid[tt][row] = b;
          const int a = b / nb, j = b - a * nb, jm = j % Ns;
          const float2* x = base + (size_t)a * stride;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float2 v = x[j + rr[i] * nb];
            if (Ns > 1 && rr[i] > 0) v = cmul(v, tw_get<SIGN>(tw, rr[i] * jm * twstep));
            xv[row][i] = v;
          }
        }
      }
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        float h[2][4], l[2][4];
#pragma unroll
        for (int row = 0; row < 2; ++row)
#pragma unroll
          for (int i = 0; i < 4; ++i) split_bf16(kk ? xv[row][i].y : xv[row][i].x, h[row][i], l[row][i]);
        ah[kk][0] = pack_bf16x2(h[0][0], h[0][1]);
        ah[kk][1] = pack_bf16x2(h[1][0], h[1][1]);
        ah[kk][2] = pack_bf16x2(h[0][2], h[0][3]);
        ah[kk][3] = pack_bf16x2(h[1][2], h[1][3]);
        al[kk][0] = pack_bf16x2(l[0][0], l[0][1]);
        al[kk][1] = pack_bf16x2(l[1][0], l[1][1]);
        al[kk][2] = pack_bf16x2(l[0][2], l[0][3]);
        al[kk][3] = pack_bf16x2(l[1][2], l[1][3]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          mma_bf16_16816(acc[tt][nt], ah[kk], bh[nt][kk]);
          mma_bf16_16816(acc[tt][nt], ah[kk], bl[nt][kk]);
          mma_bf16_16816(acc[tt][nt], al[kk], bh[nt][kk]);
        }
    }
  }
  __syncthreads();
#pragma unroll
  for (int tt = 0; tt < TPW; ++tt)
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const int b = bid[tt][row];
      if (b >= 0) {
        const int a = b / nb, j = b - a * nb, jm = j % Ns;
        float2* y = base + (size_t)a * stride;
        const int o = (j - jm) * 16 + jm;
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int k = 2 * t + 8 * q2 + e;
            y[o + k * Ns] = make_float2(acc[tt][q2][2 * row + e], acc[tt][2 + q2][2 * row + e]);
          }
      }
    }
  __syncthreads();
}

// Whole DFT of length pl.n on nbuf arrays (base + a * stride), in place.
// TC: radix-16 passes on tensor cores (split_bf16 operands, fft_stage_tc16).
// Ends with a barrier; the caller must have synchronised before the call.
template <int SIGN, int PTS, bool TC = false>
__device__ __noinline__ void cta_fft(float2* base, int stride, int nbuf, const FftPlan& pl, const float2* __restrict__ tw,
                        int twmul) {
  const int n = pl.n;
  int Ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.radix[st];
    switch (R) {
      case 2: fft_stage<2, SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul); break;
      case 3: fft_stage<3, SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul); break;
      case 4: fft_stage<4, SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul); break;
      case 5: fft_stage<5, SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul); break;
      case 8: fft_stage<8, SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul); break;
      case 16:
        if (TC) fft_stage_tc16<SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul);
        else fft_stage<16, SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul);
        break;
      default: fft_stage_generic<SIGN, PTS>(base, stride, nbuf, n, R, Ns, tw, twmul); break;
    }
    Ns *= R;
  }
}


// ---------------------------------------------------------------------------
// Structured engine for ladder lengths n = odd * 2^a (a >= 4, odd in
// {1, 3, 5, 9}): the passes are a fixed, fully inlined sequence (radix 16
// while 16 divides the power of two, one radix-8/4/2 pass for the rest of it,
// then one radix-3/5/9 pass), so no runtime radix switch forces the register
// allocator to spill.  Arrays enter and leave in natural order; only between
// the first pass (Ns = 1, whose stores stride by 16) and the second pass are
// the values kept at swz(i) = i ^ ((i >> 4) & 15), a permutation inside each
// aligned block of 16 values that sends those stores to distinct banks.
// Index splits use a float reciprocal with one integer correction (exact for
// numerators below 2^17).  Twiddles: PASS_TW = false reads the zeta_N table
// `tw` as fft_stage does (zeta_m^x = tw[x * twmul]); PASS_TW = true reads a
// per-pass table (in shared memory) where pass (R, Ns) finds zeta_{Ns R}^{r jm}
// at tw[(Ns - 1) + (r - 1) Ns + jm] (r = 1..R-1, jm < Ns; the offsets of the
// passes telescope to a table of n - 1 entries, built by hd_tables_plan.cu in
// the pass order of cta_fft_struct).
// ---------------------------------------------------------------------------
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

__host__ __device__ __forceinline__ int swz(int k) { return k ^ ((k >> 4) & 15); }
// array stride: a whole number of 16-element blocks, so swz stays inside the array
__host__ __device__ __forceinline__ int swz_stride(int n) { return (n + 15) & ~15; }

// Radix of the last pass of cta_fft_struct when the leftover power of two
// rem2 (2, 4 or 8) and the odd factor (3, 5 or 9) are merged into one
// composite butterfly (at most 24 points), else 0 (separate passes).
__host__ __device__ constexpr int merged_tail(int rem2, int odd) {
  return (rem2 > 1 && odd > 1 && rem2 * odd <= 24) ? rem2 * odd : 0;
}

// Points cta_fft_struct<SIGN, PTS> can transform in one call with T threads
// for a struct_length n: every pass must hold its butterflies, ceil(PTS / R)
// per thread, so the capacity is the smallest ceil(PTS / R) R T over the
// passes (e.g. 32 T for n = 4096 at PTS = 24, whose passes are all radix 16).
__host__ __device__ inline int struct_capacity(int n, int PTS, int T) {
  int a2 = 0;
  while (a2 < 30 && ((n >> a2) & 1) == 0) ++a2;
  const int odd = n >> a2, rem2 = 1 << (a2 & 3);
  auto cap = [&](int R) { return ((PTS + R - 1) / R) * R * T; };
  int c = cap(16);
  const int mt = merged_tail(rem2, odd);
  if (mt) {
    c = c < cap(mt) ? c : cap(mt);
  } else {
    if (rem2 > 1) c = c < cap(rem2) ? c : cap(rem2);
    if (odd > 1) c = c < cap(odd) ? c : cap(odd);
  }
  return c;
}

// Lengths cta_fft_struct takes.
__host__ __device__ inline bool struct_length(int n) {
  if (n < 16) return false;
  int a2 = 0;
  while (((n >> a2) & 1) == 0) ++a2;
  const int odd = n >> a2;
  return a2 >= 4 && (odd == 1 || odd == 3 || odd == 5 || odd == 9);
}

// NN > 0: the transform length NN and the stride NSS of this pass are
// compile-time constants (n and Ns ignored), so the index divisions below
// become multiplies and shifts.
template <int R, int SIGN, int PTS, bool IN_SWZ, bool OUT_SWZ, bool PASS_TW, int NN = 0, int NSS = 1>
__device__ __forceinline__ void gstage(float2* base, int stride, int nbuf, int n, int Ns,
                                       const float2* __restrict__ tw, int twmul) {
  if constexpr (NN > 0) {
    n = NN;
    Ns = NSS;
  }
  constexpr int BPT = (PTS + R - 1) / R;
  const int nb = n / R;
  const DivF dnb = make_div(nb), dNs = make_div(Ns);
  const int total = nb * nbuf;
  const int T = blockDim.x;
  const int twstep = twmul * (n / (Ns * R));
  float2 v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int idx = threadIdx.x + b * T;
    if (idx < total) {
      const int a = NN > 0 ? idx / nb : fdiv(idx, dnb);
      const int j = idx - a * nb;
      const int jm = NN > 0 ? j % Ns : j - fdiv(j, dNs) * Ns;
      const float2* x = base + a * stride;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = x[IN_SWZ ? swz(j + r * nb) : j + r * nb];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w;
          if constexpr (PASS_TW) {
            w = tw[(Ns - 1) + (r - 1) * Ns + jm];
            if (SIGN < 0) w.y = -w.y;
          } else {
            w = tw_get<SIGN>(tw, r * jm * twstep);
          }
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
      const int a = NN > 0 ? idx / nb : fdiv(idx, dnb);
      const int j = idx - a * nb;
      const int jm = NN > 0 ? j % Ns : j - fdiv(j, dNs) * Ns;
      dft_reg<R, SIGN>(v[b]);
      float2* y = base + a * stride;
      const int o = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) y[OUT_SWZ ? swz(o + r * Ns) : o + r * Ns] = v[b][r];
    }
  }
  __syncthreads();
}

// The pass after the radix-16 ones: radix 8/4/2 for the rest of the power of
// two (rem = a mod 4), else the odd radix; IN_SWZ when it is the second pass.
template <int SIGN, int PTS, bool IN_SWZ, bool PASS_TW>
__device__ __forceinline__ void gstage_rem(float2* base, int stride, int nbuf, int n, int& Ns, int rem,
                                           const float2* __restrict__ tw, int twmul) {
  if (rem == 3) {
    gstage<8, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
    Ns *= 8;
  } else if (rem == 2) {
    gstage<4, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
    Ns *= 4;
  } else if (rem == 1) {
    gstage<2, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
    Ns *= 2;
  }
}
template <int SIGN, int PTS, bool IN_SWZ, bool PASS_TW>
__device__ __forceinline__ void gstage_odd(float2* base, int stride, int nbuf, int n, int Ns, int odd,
                                           const float2* __restrict__ tw, int twmul) {
  if (odd == 3) gstage<3, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
  else if (odd == 5) gstage<5, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
  else if (odd == 9) gstage<9, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
}

template <int SIGN, int PTS, bool IN_SWZ, bool PASS_TW>
__device__ __forceinline__ void gstage_merged(float2* base, int stride, int nbuf, int n, int Ns, int R,
                                              const float2* __restrict__ tw, int twmul) {
  switch (R) {
    case 6: gstage<6, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul); break;
    case 10: gstage<10, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul); break;
    case 12: gstage<12, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul); break;
    case 18: gstage<18, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul); break;
    case 20: gstage<20, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul); break;
    default: gstage<24, SIGN, PTS, IN_SWZ, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul); break;
  }
}

// Whole DFT of a struct_length n on nbuf arrays (base + a * stride), in place,
// natural order in and out: radix-16 passes, then the leftover power of two
// and the odd factor, merged into one composite pass where merged_tail allows.
// Requires nbuf * n <= PTS * blockDim.x.
template <int SIGN, int PTS, bool PASS_TW = false>
__device__ __forceinline__ void cta_fft_struct(float2* base, int stride, int nbuf, int n,
                                               const float2* __restrict__ tw, int twmul) {
  const int a2 = __ffs(n) - 1;
  const int odd = n >> a2;
  const int n16 = a2 >> 2, rem = a2 & 3;
  const int mt = merged_tail(1 << rem, odd);
  if (n == 16) {
    gstage<16, SIGN, PTS, false, false, PASS_TW>(base, stride, nbuf, n, 1, tw, twmul);
    return;
  }
  gstage<16, SIGN, PTS, false, true, PASS_TW>(base, stride, nbuf, n, 1, tw, twmul);
  int Ns = 16;
  if (n16 >= 2) {
    gstage<16, SIGN, PTS, true, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
    Ns *= 16;
    for (int i = 2; i < n16; ++i) {
      gstage<16, SIGN, PTS, false, false, PASS_TW>(base, stride, nbuf, n, Ns, tw, twmul);
      Ns *= 16;
    }
    if (mt) {
      gstage_merged<SIGN, PTS, false, PASS_TW>(base, stride, nbuf, n, Ns, mt, tw, twmul);
    } else {
      gstage_rem<SIGN, PTS, false, PASS_TW>(base, stride, nbuf, n, Ns, rem, tw, twmul);
      gstage_odd<SIGN, PTS, false, PASS_TW>(base, stride, nbuf, n, Ns, odd, tw, twmul);
    }
  } else if (rem) {
    if (mt) {
      gstage_merged<SIGN, PTS, true, PASS_TW>(base, stride, nbuf, n, Ns, mt, tw, twmul);
    } else {
      gstage_rem<SIGN, PTS, true, PASS_TW>(base, stride, nbuf, n, Ns, rem, tw, twmul);
      gstage_odd<SIGN, PTS, false, PASS_TW>(base, stride, nbuf, n, Ns, odd, tw, twmul);
    }
  } else {
    gstage_odd<SIGN, PTS, true, PASS_TW>(base, stride, nbuf, n, Ns, odd, tw, twmul);
  }
}

// The passes of cta_fft_struct for a compile-time length N (at most three
// radix-16 passes), same order, same swizzles, every trip count and divisor a
// constant.
template <int SIGN, int PTS, int N, int NS, bool IN_SWZ, bool PASS_TW>
__device__ __forceinline__ void struct_tail_k(float2* base, int stride, int nbuf, const float2* __restrict__ tw,
                                              int twmul) {
  constexpr int a2 = __builtin_ctz(N);
  constexpr int odd = N >> a2, rem = a2 & 3;
  constexpr int mt = merged_tail(1 << rem, odd);
  if constexpr (mt) {
    gstage<mt, SIGN, PTS, IN_SWZ, false, PASS_TW, N, NS>(base, stride, nbuf, N, NS, tw, twmul);
  } else {
    if constexpr (rem) gstage<(1 << rem), SIGN, PTS, IN_SWZ, false, PASS_TW, N, NS>(base, stride, nbuf, N, NS, tw, twmul);
    constexpr int NS2 = NS << rem;
    constexpr bool SW2 = rem ? false : IN_SWZ;
    if constexpr (odd > 1) gstage<odd, SIGN, PTS, SW2, false, PASS_TW, N, NS2>(base, stride, nbuf, N, NS2, tw, twmul);
  }
}

template <int SIGN, int PTS, int N, bool PASS_TW = false>
__device__ __forceinline__ void cta_fft_struct_k(float2* base, int stride, int nbuf, const float2* __restrict__ tw,
                                                 int twmul) {
  constexpr int a2 = __builtin_ctz(N);
  constexpr int n16 = a2 >> 2;
  static_assert(n16 >= 1 && n16 <= 3, "compile-time structured lengths: 16 <= N, at most three radix-16 passes");
  if constexpr (N == 16) {
    gstage<16, SIGN, PTS, false, false, PASS_TW, N, 1>(base, stride, nbuf, N, 1, tw, twmul);
  } else {
    gstage<16, SIGN, PTS, false, true, PASS_TW, N, 1>(base, stride, nbuf, N, 1, tw, twmul);
    if constexpr (n16 >= 2) {
      gstage<16, SIGN, PTS, true, false, PASS_TW, N, 16>(base, stride, nbuf, N, 16, tw, twmul);
      if constexpr (n16 >= 3) {
        gstage<16, SIGN, PTS, false, false, PASS_TW, N, 256>(base, stride, nbuf, N, 256, tw, twmul);
        struct_tail_k<SIGN, PTS, N, 4096, false, PASS_TW>(base, stride, nbuf, tw, twmul);
      } else {
        struct_tail_k<SIGN, PTS, N, 256, false, PASS_TW>(base, stride, nbuf, tw, twmul);
      }
    } else {
      struct_tail_k<SIGN, PTS, N, 16, true, PASS_TW>(base, stride, nbuf, tw, twmul);
    }
  }
}


// ---------------------------------------------------------------------------
// Out-of-place form of the structured engine: pass k reads one buffer and
// writes the other, so a pass needs one barrier (after its stores) and holds
// one butterfly at a time.  Same pass sequence, swizzle and twiddles as
// cta_fft_struct.
// ---------------------------------------------------------------------------
template <int R, int SIGN, bool IN_SWZ, bool OUT_SWZ, bool PASS_TW>
__device__ __forceinline__ void gstage_oop(const float2* __restrict__ in, float2* __restrict__ out, int stride,
                                           int nbuf, int n, int Ns, const float2* __restrict__ tw, int twmul) {
  const int nb = n / R;
  const DivF dnb = make_div(nb), dNs = make_div(Ns);
  const int total = nb * nbuf;
  const int twstep = twmul * (n / (Ns * R));
  constexpr int UNR = R <= 8 ? 2 : 1;  // two small butterflies in flight; one large one
#pragma unroll UNR
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int a = fdiv(idx, dnb);
    const int j = idx - a * nb;
    const int jm = j - fdiv(j, dNs) * Ns;
    const float2* x = in + a * stride;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[IN_SWZ ? swz(j + r * nb) : j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w;
        if constexpr (PASS_TW) {
          w = tw[(Ns - 1) + (r - 1) * Ns + jm];
          if (SIGN < 0) w.y = -w.y;
        } else {
          w = tw_get<SIGN>(tw, r * jm * twstep);
        }
        v[r] = cmul(v[r], w);
      }
    }
    dft_reg<R, SIGN>(v);
    float2* y = out + a * stride;
    const int o = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) y[OUT_SWZ ? swz(o + r * Ns) : o + r * Ns] = v[r];
  }
  __syncthreads();
}

template <int SIGN, bool IN_SWZ, bool PASS_TW>
__device__ __forceinline__ void gstage_oop_tail(const float2* in, float2* out, int stride, int nbuf, int n, int Ns,
                                                int R, const float2* __restrict__ tw, int twmul) {
  switch (R) {
    case 2: gstage_oop<2, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 3: gstage_oop<3, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 4: gstage_oop<4, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 5: gstage_oop<5, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 6: gstage_oop<6, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 8: gstage_oop<8, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 9: gstage_oop<9, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 10: gstage_oop<10, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 12: gstage_oop<12, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 18: gstage_oop<18, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    case 20: gstage_oop<20, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
    default: gstage_oop<24, SIGN, IN_SWZ, false, PASS_TW>(in, out, stride, nbuf, n, Ns, tw, twmul); break;
  }
}

// Whole DFT of a struct_length n on nbuf arrays (b0 + a * stride), using the
// arrays at b1 (same shape) as the other buffer; returns 0 if the result is in
// b0, 1 if in b1.  Ends with a barrier.
template <int SIGN, bool PASS_TW>
__device__ __forceinline__ int cta_fft_struct_oop(float2* b0, float2* b1, int stride, int nbuf, int n,
                                                  const float2* __restrict__ tw, int twmul) {
  const int a2 = __ffs(n) - 1;
  const int odd = n >> a2;
  const int n16 = a2 >> 2, rem = a2 & 3;
  const int rem2 = 1 << rem;
  const int mt = merged_tail(rem2, odd);
  // the passes after the radix-16 ones: one merged pass, or rem2 then odd
  const int t1 = mt ? mt : (rem2 > 1 ? rem2 : odd);
  const int t2 = mt ? 1 : (rem2 > 1 ? odd : 1);
  float2* cur = b0;
  float2* nxt = b1;
  int res = 0;
  auto flip = [&]() {
    float2* t = cur;
    cur = nxt;
    nxt = t;
    res ^= 1;
  };
  if (n == 16) {
    gstage_oop<16, SIGN, false, false, PASS_TW>(cur, nxt, stride, nbuf, n, 1, tw, twmul);
    flip();
    return res;
  }
  gstage_oop<16, SIGN, false, true, PASS_TW>(cur, nxt, stride, nbuf, n, 1, tw, twmul);
  flip();
  int Ns = 16;
  if (n16 >= 2) {
    gstage_oop<16, SIGN, true, false, PASS_TW>(cur, nxt, stride, nbuf, n, Ns, tw, twmul);
    flip();
    Ns *= 16;
    for (int i = 2; i < n16; ++i) {
      gstage_oop<16, SIGN, false, false, PASS_TW>(cur, nxt, stride, nbuf, n, Ns, tw, twmul);
      flip();
      Ns *= 16;
    }
    if (t1 > 1) {
      gstage_oop_tail<SIGN, false, PASS_TW>(cur, nxt, stride, nbuf, n, Ns, t1, tw, twmul);
      flip();
      Ns *= t1;
    }
  } else if (t1 > 1) {
    gstage_oop_tail<SIGN, true, PASS_TW>(cur, nxt, stride, nbuf, n, Ns, t1, tw, twmul);
    flip();
    Ns *= t1;
  }
  if (t2 > 1) {
    gstage_oop_tail<SIGN, false, PASS_TW>(cur, nxt, stride, nbuf, n, Ns, t2, tw, twmul);
    flip();
  }
  return res;
}

// Structured pass sequence with the radix-16 passes on tensor cores
// (fft_stage_tc16, split bf16 operands) and the leftover power of two and
// odd factor in FP32 (gstage), natural order throughout.  Requires
// nbuf * n <= 16 * blockDim.x (the tensor-core pass) and <= PTS * blockDim.x.
template <int SIGN, int PTS>
__device__ __forceinline__ void cta_fft_struct_tc(float2* base, int stride, int nbuf, int n,
                                                  const float2* __restrict__ tw, int twmul) {
  const int a2 = __ffs(n) - 1;
  const int odd = n >> a2;
  const int n16 = a2 >> 2, rem = a2 & 3;
  const int mt = merged_tail(1 << rem, odd);
  int Ns = 1;
  for (int i = 0; i < n16; ++i) {
    fft_stage_tc16<SIGN, PTS>(base, stride, nbuf, n, Ns, tw, twmul);
    Ns *= 16;
  }
  if (mt) {
    gstage_merged<SIGN, PTS, false, false>(base, stride, nbuf, n, Ns, mt, tw, twmul);
  } else {
    gstage_rem<SIGN, PTS, false, false>(base, stride, nbuf, n, Ns, rem, tw, twmul);
    gstage_odd<SIGN, PTS, false, false>(base, stride, nbuf, n, Ns, odd, tw, twmul);
  }
}

// DFT dispatch of the nD kernels: SE (struct_length lengths) inlines the
// structured engine (TC: with tensor-core radix-16 passes), otherwise the
// generic plan-driven cta_fft.
// NN > 0: the structured engine at the compile-time length NN (= pl.n).
template <int SIGN, int PTS, bool TC, bool SE, int NN = 0>
__device__ __forceinline__ void fft_sel(float2* base, int stride, int nbuf, const FftPlan& pl,
                                        const float2* __restrict__ tw, int twmul) {
  if constexpr (SE && !TC && NN > 0) cta_fft_struct_k<SIGN, PTS, NN>(base, stride, nbuf, tw, twmul);
  else if constexpr (SE && TC) cta_fft_struct_tc<SIGN, PTS>(base, stride, nbuf, pl.n, tw, twmul);
  else if constexpr (SE) cta_fft_struct<SIGN, PTS>(base, stride, nbuf, pl.n, tw, twmul);
  else cta_fft<SIGN, PTS, TC>(base, stride, nbuf, pl, tw, twmul);
}

}  // namespace hd
