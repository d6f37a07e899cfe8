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

namespace hd {

constexpr int kMaxStages = 24;

// Radix sequence of one DFT length; the product of radix[0..nst) equals n.
struct FftPlan {
  int n;
  int nst;
  int radix[kMaxStages];
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// i * sign * a
template <int SIGN>
__device__ __forceinline__ float2 cmul_i(float2 a) {
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// zeta_N^{SIGN * k} from the table (k already reduced into [0, N)).
template <int SIGN>
__device__ __forceinline__ float2 tw_get(const float2* __restrict__ tw, int k) {
  float2 w = __ldg(tw + k);
  if (SIGN < 0) w.y = -w.y;
  return w;
}

// ---------------------------------------------------------------------------
// register butterflies: y_k = sum_j a_j zeta_R^{SIGN jk}
// ---------------------------------------------------------------------------
template <int SIGN>
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
  float2 t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <int SIGN>
__device__ __forceinline__ void dft3(float2& a0, float2& a1, float2& a2) {
  const float c = -0.5f;
  const float s = 0.86602540378443864676f;  // sin(2 pi / 3)
  float2 t1 = cadd(a1, a2);
  float2 t2 = csub(a1, a2);
  float2 y0 = cadd(a0, t1);
  float2 b = make_float2(fmaf(c, t1.x, a0.x), fmaf(c, t1.y, a0.y));
  float2 rot = cscale(cmul_i<SIGN>(t2), s);
  a0 = y0;
  a1 = cadd(b, rot);
  a2 = csub(b, rot);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = cmul_i<SIGN>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

template <int SIGN>
__device__ __forceinline__ void dft5(float2& a0, float2& a1, float2& a2, float2& a3, float2& a4) {
  const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
  const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
  const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
  const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
  float2 p14 = cadd(a1, a4), m14 = csub(a1, a4);
  float2 p23 = cadd(a2, a3), m23 = csub(a2, a3);
  float2 y0 = cadd(a0, cadd(p14, p23));
  float2 b1 = make_float2(a0.x + c1 * p14.x + c2 * p23.x, a0.y + c1 * p14.y + c2 * p23.y);
  float2 b2 = make_float2(a0.x + c2 * p14.x + c1 * p23.x, a0.y + c2 * p14.y + c1 * p23.y);
  float2 r1 = cmul_i<SIGN>(make_float2(s1 * m14.x + s2 * m23.x, s1 * m14.y + s2 * m23.y));
  float2 r2 = cmul_i<SIGN>(make_float2(s2 * m14.x - s1 * m23.x, s2 * m14.y - s1 * m23.y));
  a0 = y0;
  a1 = cadd(b1, r1);
  a4 = csub(b1, r1);
  a2 = cadd(b2, r2);
  a3 = csub(b2, r2);
}

template <int SIGN>
__device__ __forceinline__ void dft8(float2* a) {
  const float r = 0.70710678118654752440f;
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<SIGN>(e0, e1, e2, e3);
  dft4<SIGN>(o0, o1, o2, o3);
  // o_k *= zeta_8^{SIGN k}
  o1 = make_float2(r * (o1.x - SIGN * o1.y), r * (o1.y + SIGN * o1.x));
  o2 = cmul_i<SIGN>(o2);
  o3 = make_float2(r * (-o3.x - SIGN * o3.y), r * (-o3.y + SIGN * o3.x));
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

template <int SIGN>
__device__ __forceinline__ void dft16(float2* a) {
  // cos(k pi / 8), sin(k pi / 8), k = 0..7
  const float C[8] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f,
                      0.0f, -0.38268343236508977173f, -0.70710678118654752440f, -0.92387953251128675613f};
  const float S[8] = {0.0f, 0.38268343236508977173f, 0.70710678118654752440f, 0.92387953251128675613f,
                      1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f};
  float2 e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = a[2 * k];
    o[k] = a[2 * k + 1];
  }
  dft8<SIGN>(e);
  dft8<SIGN>(o);
#pragma unroll
  for (int k = 1; k < 8; ++k) o[k] = cmul(o[k], make_float2(C[k], SIGN * S[k]));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = cadd(e[k], o[k]);
    a[k + 8] = csub(e[k], o[k]);
  }
}

// 9 points as 3 x 3: inner length-3 DFTs over n2 (n = n1 + 3 n2), twiddles
// zeta_9^{n1 k2}, outer length-3 DFTs over n1; output k = 3 k1 + k2.
template <int SIGN>
__device__ __forceinline__ void dft9(float2* a) {
  const float c1 = 0.76604444311897803520f, s1 = 0.64278760968653932632f;   // zeta_9^1
  const float c2 = 0.17364817766693034885f, s2 = 0.98480775301220805936f;   // zeta_9^2
  const float c4 = -0.93969262078590838405f, s4 = 0.34202014332566873304f;  // zeta_9^4
  float2 y[3][3];
#pragma unroll
  for (int n1 = 0; n1 < 3; ++n1) {
    y[n1][0] = a[n1];
    y[n1][1] = a[n1 + 3];
    y[n1][2] = a[n1 + 6];
    dft3<SIGN>(y[n1][0], y[n1][1], y[n1][2]);
  }
  y[1][1] = cmul(y[1][1], make_float2(c1, SIGN * s1));
  y[1][2] = cmul(y[1][2], make_float2(c2, SIGN * s2));
  y[2][1] = cmul(y[2][1], make_float2(c2, SIGN * s2));
  y[2][2] = cmul(y[2][2], make_float2(c4, SIGN * s4));
#pragma unroll
  for (int k2 = 0; k2 < 3; ++k2) {
    float2 z0 = y[0][k2], z1 = y[1][k2], z2 = y[2][k2];
    dft3<SIGN>(z0, z1, z2);
    a[k2] = z0;
    a[3 + k2] = z1;
    a[6 + k2] = z2;
  }
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2* v);

// zeta_R^e = (cos, sin)(2 pi e / R), e < R, for the composite radices below
// (FP32 roundings of the exact values).
template <int R>
__device__ __forceinline__ float2 unit_root(int e);
template <>
__device__ __forceinline__ float2 unit_root<6>(int e) {
  const float c[6] = {1.0f, 0.5f, -0.5f, -1.0f, -0.5f, 0.5f};
  const float s[6] = {0.0f, 0.866025404f, 0.866025404f, 0.0f, -0.866025404f, -0.866025404f};
  return make_float2(c[e], s[e]);
}
template <>
__device__ __forceinline__ float2 unit_root<10>(int e) {
  const float c[10] = {1.0f, 0.809016994f, 0.309016994f, -0.309016994f, -0.809016994f, -1.0f, -0.809016994f, -0.309016994f, 0.309016994f, 0.809016994f};
  const float s[10] = {0.0f, 0.587785252f, 0.951056516f, 0.951056516f, 0.587785252f, 0.0f, -0.587785252f, -0.951056516f, -0.951056516f, -0.587785252f};
  return make_float2(c[e], s[e]);
}
template <>
__device__ __forceinline__ float2 unit_root<12>(int e) {
  const float c[12] = {1.0f, 0.866025404f, 0.5f, 0.0f, -0.5f, -0.866025404f, -1.0f, -0.866025404f, -0.5f, 0.0f, 0.5f, 0.866025404f};
  const float s[12] = {0.0f, 0.5f, 0.866025404f, 1.0f, 0.866025404f, 0.5f, 0.0f, -0.5f, -0.866025404f, -1.0f, -0.866025404f, -0.5f};
  return make_float2(c[e], s[e]);
}
template <>
__device__ __forceinline__ float2 unit_root<18>(int e) {
  const float c[18] = {1.0f, 0.939692621f, 0.766044443f, 0.5f, 0.173648178f, -0.173648178f, -0.5f, -0.766044443f, -0.939692621f, -1.0f, -0.939692621f, -0.766044443f, -0.5f, -0.173648178f, 0.173648178f, 0.5f, 0.766044443f, 0.939692621f};
  const float s[18] = {0.0f, 0.342020143f, 0.64278761f, 0.866025404f, 0.984807753f, 0.984807753f, 0.866025404f, 0.64278761f, 0.342020143f, 0.0f, -0.342020143f, -0.64278761f, -0.866025404f, -0.984807753f, -0.984807753f, -0.866025404f, -0.64278761f, -0.342020143f};
  return make_float2(c[e], s[e]);
}
template <>
__device__ __forceinline__ float2 unit_root<20>(int e) {
  const float c[20] = {1.0f, 0.951056516f, 0.809016994f, 0.587785252f, 0.309016994f, 0.0f, -0.309016994f, -0.587785252f, -0.809016994f, -0.951056516f, -1.0f, -0.951056516f, -0.809016994f, -0.587785252f, -0.309016994f, 0.0f, 0.309016994f, 0.587785252f, 0.809016994f, 0.951056516f};
  const float s[20] = {0.0f, 0.309016994f, 0.587785252f, 0.809016994f, 0.951056516f, 1.0f, 0.951056516f, 0.809016994f, 0.587785252f, 0.309016994f, 0.0f, -0.309016994f, -0.587785252f, -0.809016994f, -0.951056516f, -1.0f, -0.951056516f, -0.809016994f, -0.587785252f, -0.309016994f};
  return make_float2(c[e], s[e]);
}
template <>
__device__ __forceinline__ float2 unit_root<24>(int e) {
  const float c[24] = {1.0f, 0.965925826f, 0.866025404f, 0.707106781f, 0.5f, 0.258819045f, 0.0f, -0.258819045f, -0.5f, -0.707106781f, -0.866025404f, -0.965925826f, -1.0f, -0.965925826f, -0.866025404f, -0.707106781f, -0.5f, -0.258819045f, 0.0f, 0.258819045f, 0.5f, 0.707106781f, 0.866025404f, 0.965925826f};
  const float s[24] = {0.0f, 0.258819045f, 0.5f, 0.707106781f, 0.866025404f, 0.965925826f, 1.0f, 0.965925826f, 0.866025404f, 0.707106781f, 0.5f, 0.258819045f, 0.0f, -0.258819045f, -0.5f, -0.707106781f, -0.866025404f, -0.965925826f, -1.0f, -0.965925826f, -0.866025404f, -0.707106781f, -0.5f, -0.258819045f};
  return make_float2(c[e], s[e]);
}

// Composite radix R = R1 R2 in registers: with n = n1 + R1 n2 and
// k = k2 + R2 k1, X_k = sum_{n1} zeta_{R1}^{n1 k1} zeta_R^{n1 k2}
// sum_{n2} x_n zeta_{R2}^{n2 k2} (length-R2 DFTs, twiddles, length-R1 DFTs).
template <int R1, int R2, int SIGN>
__device__ __forceinline__ void dft_comp(float2* v) {
  constexpr int R = R1 * R2;
  float2 t[R];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) {
    float2 a[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) a[n2] = v[n1 + R1 * n2];
    dft_reg<R2, SIGN>(a);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      if (n1 * k2 == 0) {
        t[n1 * R2 + k2] = a[k2];
      } else {
        float2 w = unit_root<R>(n1 * k2);
        if (SIGN < 0) w.y = -w.y;
        t[n1 * R2 + k2] = cmul(a[k2], w);
      }
    }
  }
#pragma unroll
  for (int k2 = 0; k2 < R2; ++k2) {
    float2 b[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) b[n1] = t[n1 * R2 + k2];
    dft_reg<R1, SIGN>(b);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k2 + R2 * k1] = b[k1];
  }
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R == 2) dft2<SIGN>(v[0], v[1]);
  else if constexpr (R == 3) dft3<SIGN>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<SIGN>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 5) dft5<SIGN>(v[0], v[1], v[2], v[3], v[4]);
  else if constexpr (R == 8) dft8<SIGN>(v);
  else if constexpr (R == 9) dft9<SIGN>(v);
  else if constexpr (R == 16) dft16<SIGN>(v);
  else if constexpr (R == 6) dft_comp<2, 3, SIGN>(v);
  else if constexpr (R == 10) dft_comp<2, 5, SIGN>(v);
  else if constexpr (R == 12) dft_comp<4, 3, SIGN>(v);
  else if constexpr (R == 18) dft_comp<2, 9, SIGN>(v);
  else if constexpr (R == 20) dft_comp<4, 5, SIGN>(v);
  else if constexpr (R == 24) dft_comp<8, 3, SIGN>(v);
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

template <int R, int SIGN, int PTS, bool IN_SWZ, bool OUT_SWZ, bool PASS_TW>
__device__ __forceinline__ void gstage(float2* base, int stride, int nbuf, int n, int Ns,
                                       const float2* __restrict__ tw, int twmul) {
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
      const int a = fdiv(idx, dnb);
      const int j = idx - a * nb;
      const int jm = j - fdiv(j, dNs) * Ns;
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
      const int a = fdiv(idx, dnb);
      const int j = idx - a * nb;
      const int jm = j - fdiv(j, dNs) * Ns;
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
template <int SIGN, int PTS, bool TC, bool SE>
__device__ __forceinline__ void fft_sel(float2* base, int stride, int nbuf, const FftPlan& pl,
                                        const float2* __restrict__ tw, int twmul) {
  if constexpr (SE && TC) cta_fft_struct_tc<SIGN, PTS>(base, stride, nbuf, pl.n, tw, twmul);
  else if constexpr (SE) cta_fft_struct<SIGN, PTS>(base, stride, nbuf, pl.n, tw, twmul);
  else cta_fft<SIGN, PTS, TC>(base, stride, nbuf, pl, tw, twmul);
}

}  // namespace hd
