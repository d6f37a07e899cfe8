// hd_bfly.cuh -- complex helpers and register butterflies (radix 2, 3, 4, 5,
// 8, 9, 16 and the composites 6, 10, 12, 18, 20, 24) shared by every DFT engine
// of the library.  Host and device: the cluster kernel's steps are also
// stepped on the host.
//
// Sign convention (Sec. 2): zeta_N = exp(+2 pi i / N); SIGN = +1 computes
// y_k = sum_j a_j zeta_R^{jk} (the forward transform of the paper), SIGN = -1
// the backward transform.  No scaling.
#pragma once
#include <cuda_runtime.h>

namespace hd {

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// i * sign * a
template <int SIGN>
__host__ __device__ __forceinline__ float2 cmul_i(float2 a) {
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// register butterflies: y_k = sum_j a_j zeta_R^{SIGN jk}
// ---------------------------------------------------------------------------
template <int SIGN>
__host__ __device__ __forceinline__ void dft2(float2& a0, float2& a1) {
  float2 t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <int SIGN>
__host__ __device__ __forceinline__ void dft3(float2& a0, float2& a1, float2& a2) {
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
__host__ __device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = cmul_i<SIGN>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

template <int SIGN>
__host__ __device__ __forceinline__ void dft5(float2& a0, float2& a1, float2& a2, float2& a3, float2& a4) {
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
__host__ __device__ __forceinline__ void dft8(float2* a) {
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
__host__ __device__ __forceinline__ void dft16(float2* a) {
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
__host__ __device__ __forceinline__ void dft9(float2* a) {
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
__host__ __device__ __forceinline__ void dft_reg(float2* v);

// zeta_R^e = (cos, sin)(2 pi e / R), e < R, for the composite radices below
// (FP32 roundings of the exact values).
template <int R>
__host__ __device__ __forceinline__ float2 unit_root(int e);
template <>
__host__ __device__ __forceinline__ float2 unit_root<6>(int e) {
  const float c[6] = {1.0f, 0.5f, -0.5f, -1.0f, -0.5f, 0.5f};
  const float s[6] = {0.0f, 0.866025404f, 0.866025404f, 0.0f, -0.866025404f, -0.866025404f};
  return make_float2(c[e], s[e]);
}
template <>
__host__ __device__ __forceinline__ float2 unit_root<10>(int e) {
  const float c[10] = {1.0f, 0.809016994f, 0.309016994f, -0.309016994f, -0.809016994f, -1.0f, -0.809016994f, -0.309016994f, 0.309016994f, 0.809016994f};
  const float s[10] = {0.0f, 0.587785252f, 0.951056516f, 0.951056516f, 0.587785252f, 0.0f, -0.587785252f, -0.951056516f, -0.951056516f, -0.587785252f};
  return make_float2(c[e], s[e]);
}
template <>
__host__ __device__ __forceinline__ float2 unit_root<12>(int e) {
  const float c[12] = {1.0f, 0.866025404f, 0.5f, 0.0f, -0.5f, -0.866025404f, -1.0f, -0.866025404f, -0.5f, 0.0f, 0.5f, 0.866025404f};
  const float s[12] = {0.0f, 0.5f, 0.866025404f, 1.0f, 0.866025404f, 0.5f, 0.0f, -0.5f, -0.866025404f, -1.0f, -0.866025404f, -0.5f};
  return make_float2(c[e], s[e]);
}
template <>
__host__ __device__ __forceinline__ float2 unit_root<18>(int e) {
  const float c[18] = {1.0f, 0.939692621f, 0.766044443f, 0.5f, 0.173648178f, -0.173648178f, -0.5f, -0.766044443f, -0.939692621f, -1.0f, -0.939692621f, -0.766044443f, -0.5f, -0.173648178f, 0.173648178f, 0.5f, 0.766044443f, 0.939692621f};
  const float s[18] = {0.0f, 0.342020143f, 0.64278761f, 0.866025404f, 0.984807753f, 0.984807753f, 0.866025404f, 0.64278761f, 0.342020143f, 0.0f, -0.342020143f, -0.64278761f, -0.866025404f, -0.984807753f, -0.984807753f, -0.866025404f, -0.64278761f, -0.342020143f};
  return make_float2(c[e], s[e]);
}
template <>
__host__ __device__ __forceinline__ float2 unit_root<20>(int e) {
  const float c[20] = {1.0f, 0.951056516f, 0.809016994f, 0.587785252f, 0.309016994f, 0.0f, -0.309016994f, -0.587785252f, -0.809016994f, -0.951056516f, -1.0f, -0.951056516f, -0.809016994f, -0.587785252f, -0.309016994f, 0.0f, 0.309016994f, 0.587785252f, 0.809016994f, 0.951056516f};
  const float s[20] = {0.0f, 0.309016994f, 0.587785252f, 0.809016994f, 0.951056516f, 1.0f, 0.951056516f, 0.809016994f, 0.587785252f, 0.309016994f, 0.0f, -0.309016994f, -0.587785252f, -0.809016994f, -0.951056516f, -1.0f, -0.951056516f, -0.809016994f, -0.587785252f, -0.309016994f};
  return make_float2(c[e], s[e]);
}
template <>
__host__ __device__ __forceinline__ float2 unit_root<24>(int e) {
  const float c[24] = {1.0f, 0.965925826f, 0.866025404f, 0.707106781f, 0.5f, 0.258819045f, 0.0f, -0.258819045f, -0.5f, -0.707106781f, -0.866025404f, -0.965925826f, -1.0f, -0.965925826f, -0.866025404f, -0.707106781f, -0.5f, -0.258819045f, 0.0f, 0.258819045f, 0.5f, 0.707106781f, 0.866025404f, 0.965925826f};
  const float s[24] = {0.0f, 0.258819045f, 0.5f, 0.707106781f, 0.866025404f, 0.965925826f, 1.0f, 0.965925826f, 0.866025404f, 0.707106781f, 0.5f, 0.258819045f, 0.0f, -0.258819045f, -0.5f, -0.707106781f, -0.866025404f, -0.965925826f, -1.0f, -0.965925826f, -0.866025404f, -0.707106781f, -0.5f, -0.258819045f};
  return make_float2(c[e], s[e]);
}

// Composite radix R = R1 R2 in registers: with n = n1 + R1 n2 and
// k = k2 + R2 k1, X_k = sum_{n1} zeta_{R1}^{n1 k1} zeta_R^{n1 k2}
// sum_{n2} x_n zeta_{R2}^{n2 k2} (length-R2 DFTs, twiddles, length-R1 DFTs).
template <int R1, int R2, int SIGN>
__host__ __device__ __forceinline__ void dft_comp(float2* v) {
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
__host__ __device__ __forceinline__ void dft_reg(float2* v) {
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


}  // namespace hd
