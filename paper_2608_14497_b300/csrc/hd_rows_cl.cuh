// hd_rows_cl.cuh -- the row pass of hybridRCM in 2D/3D (Sec. 5, operator C_1)
// on the compile-time DFT engine of the cluster kernel (hd_cl_kernel.cuh).
//
// After the outer passes every row of the outer spectra F and G (packed
// complex, length Lp) must be convolved along the row with the operator C_1,
// which couples row k1 with its conjugate partner row k1* (Eqs. RCM-ndim).
// One CTA takes a row pair: the hybrid transform of each row with q = 2
// residues of length M = 256 R3 >= Lp (p = 1: residue 0 is the DFT of the row,
// residue 1 the DFT of the row times zeta_{2M}^s, Eq. forwardr), C_1 on the
// digit-reversed spectra (residue 0: l pairs with (M - l) mod M; residue 1: l
// with M - 1 - l; the partner values come from the partner row, or from the
// same row when the row is its own partner), the backward transforms of the
// two products (Eq. accumulator), and h~_s = (w_0[s] + zeta_{2M}^{-s} w_1[s]) /
// (2M) written to the output rows (over F's rows, or a separate buffer of
// longer rows for outputs beyond L; Eq. accumulation).
//
// Shared arrays, M complex each, layout of hd_cl_kernel.cuh (phys): for a row
// pair [F row r0, F row r1, F partner r0, F partner r1, G row r0, G row r1,
// G partner r0, G partner r1]; for a row that is its own partner [F r0, F r1,
// G r0, G r1] (the one-CTA layout of the cluster kernel); pass twiddles behind.
#pragma once
#include "hd_cl_kernel.cuh"
#include "hd_nd_kernels.cuh"

namespace hd {
namespace rows {

using cl::phys;

template <int R3>
struct RowShape {
  static constexpr int M = 256 * R3;
  // threads per row pair: two warps for M = 256 (one warp would run 64 points
  // per thread per pass with only the 12 CTAs per SM that shared memory allows)
  static constexpr int T = R3 == 1 ? 64 : 32 * R3;
  static constexpr size_t SMEM = sizeof(float2) * (8 * (size_t)M + cl::Shape<R3>::TABS);
  // CTAs per SM the launch bounds ask registers for (what shared memory allows)
  static constexpr int MINB = R3 == 1 ? 10 : R3 == 2 ? 6 : R3 <= 4 ? 3 : 2;
};

template <int R3>
struct RowSteps {
  using K = cl::Steps<1, R3, false, RowShape<R3>::T>;
  static constexpr int M = K::M;
  static constexpr int T = K::T;

  // residues 0 and 1 of source row x (p = 1) into arrays a0, a0 + M, pairs of s
  static __device__ __forceinline__ void load_row(const float2* __restrict__ x, int Lp, float2* a0,
                                                  const float2* __restrict__ tw, int tid) {
#pragma unroll 2
    for (int k = tid; k < M / 2; k += T) {
      const int s = 2 * k;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (s + 1 < Lp) {
        v0 = x[s];
        v1 = x[s + 1];
      } else if (s < Lp) {
        v0 = x[s];
      }
      const float4 w = cl::ldg4(tw + s);  // zeta_{2M}^s, zeta_{2M}^{s+1}
      cl::sts4(a0 + phys(s), v0, v1);
      cl::sts4(a0 + M + phys(s), cmul(v0, make_float2(w.x, w.y)), cmul(v1, make_float2(w.z, w.w)));
    }
  }

  // load_row for NR rows at once, into the array pairs a0 + 2 M r: every
  // global load of the NR rows (and the twiddles) is issued before the first
  // shared store, so the CTA waits for one round of memory latency, not 2 NR.
  template <int NR>
  static __device__ __forceinline__ void load_rows(const float2* const (&x)[NR], int Lp, float2* a0,
                                                   const float2* __restrict__ tw, int tid) {
    constexpr int U = M / 2 / T;  // 4 for every R3
    float2 v[NR][U][2];
    float4 w[U];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int s = 2 * (tid + i * T);
      w[i] = cl::ldg4(tw + s);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        v[r][i][0] = s < Lp ? x[r][s] : make_float2(0.f, 0.f);
        v[r][i][1] = s + 1 < Lp ? x[r][s + 1] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int s = 2 * (tid + i * T);
        float2* a = a0 + 2 * M * r;
        cl::sts4(a + phys(s), v[r][i][0], v[r][i][1]);
        cl::sts4(a + M + phys(s), cmul(v[r][i][0], make_float2(w[i].x, w[i].y)),
                 cmul(v[r][i][1], make_float2(w[i].z, w[i].w)));
      }
  }

  // C_1 across a row pair: residue 0 with the (M - l) mod M pairing (one
  // position per task), residue 1 with M - 1 - p (pairs of positions).
  static __device__ __forceinline__ void product_pair(float2* arr, const float2* __restrict__ zt, float2 z1, int tid) {
    float2* Fr0 = arr;
    float2* Fr1 = arr + M;
    float2* Fp0 = arr + 2 * M;
    float2* Fp1 = arr + 3 * M;
    const float2* Gr0 = arr + 4 * M;
    const float2* Gr1 = arr + 5 * M;
    const float2* Gp0 = arr + 6 * M;
    const float2* Gp1 = arr + 7 * M;
    for (int p = tid; p < M; p += T) {
      const int l = cl::digit_freq(p, R3);
      const int ps = cl::digit_pos(l == 0 ? 0 : M - l, R3);
      float2 A = Fr0[phys(p)], Cs = Fp0[phys(ps)];
      K::rcm_pair(A, Gr0[phys(p)], Cs, Gp0[phys(ps)], K::rcm_factor(cl::ldg2(zt + p), make_float2(1.f, 0.f)), false);
      Fr0[phys(p)] = A;
      Fp0[phys(ps)] = Cs;
    }
#pragma unroll 2
    for (int k = tid; k < M / 2; k += T) {
      const int p = 2 * k, pp = M - 2 - p;
      float2 A0, A1, B0, B1, C0, C1, D0, D1;
      cl::lds4(Fr1 + phys(p), A0, A1);
      cl::lds4(Gr1 + phys(p), B0, B1);
      cl::lds4(Fp1 + phys(pp), C1, C0);
      cl::lds4(Gp1 + phys(pp), D1, D0);
      const float4 z = cl::ldg4(zt + p);
      K::rcm_pair(A0, B0, C0, D0, K::rcm_factor(make_float2(z.x, z.y), z1), false);
      K::rcm_pair(A1, B1, C1, D1, K::rcm_factor(make_float2(z.z, z.w), z1), false);
      cl::sts4(Fr1 + phys(p), A0, A1);
      cl::sts4(Fp1 + phys(pp), C1, C0);
    }
  }

  // h~_s = (w_0[s] + zeta_{2M}^{-s} w_1[s]) * scale and, for outputs beyond M,
  // h~_{M+s} = (w_0[s] - zeta_{2M}^{-s} w_1[s]) * scale (zeta_{2M}^{-M} = -1),
  // for positions < Kp, written to row x.
  static __device__ __forceinline__ void store_row(float2* __restrict__ x, int Kp, const float2* a0,
                                                   const float2* __restrict__ tw, float scale, int tid) {
#pragma unroll 2
    for (int k = tid; k < M / 2; k += T) {
      const int s = 2 * k;
      if (s >= Kp) continue;
      float2 w00, w01, w10, w11;
      cl::lds4(a0 + phys(s), w00, w01);
      cl::lds4(a0 + M + phys(s), w10, w11);
      const float4 w = cl::ldg4(tw + s);
      const float2 t0 = cmul(w10, make_float2(w.x, -w.y)), t1 = cmul(w11, make_float2(w.z, -w.w));
      x[s] = cscale(cadd(w00, t0), scale);
      if (s + 1 < Kp) x[s + 1] = cscale(cadd(w01, t1), scale);
      if (M + s < Kp) x[M + s] = cscale(csub(w00, t0), scale);
      if (M + s + 1 < Kp) x[M + s + 1] = cscale(csub(w01, t1), scale);
    }
  }
};

// One row pair per CTA (rows whose partner precedes them exit at once).
template <int R3>
__global__ void __launch_bounds__(RowShape<R3>::T, RowShape<R3>::MINB)
    k_rows_cl(float2* F, const float2* __restrict__ G, float2* O, RowGeom rg, float scale,
              const float2* __restrict__ tw, const float2* __restrict__ tab) {
  using S = RowSteps<R3>;
  using K = typename S::K;
  constexpr int M = S::M, T = S::T;
  const int row = blockIdx.x;
  const int prow = row_partner(row, rg);
  if (prow < row) return;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);
  float2* tws = arr + 8 * M;
  const int tid = threadIdx.x;
  for (int i = tid; i < cl::Shape<R3>::TABS / 2; i += T) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tws + 2 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(tab + 2 * i) : "memory");
  }
  const int Lp = rg.Lrow, Kp = rg.Kout;
  const float2* zt = tab + cl::Shape<R3>::TABZ;
  if (prow == row) {
    // the row is its own partner: the one-CTA convolution of the cluster kernel
    {
      const float2* const src[2] = {F + (int64_t)row * Lp, G + (int64_t)row * Lp};
      S::template load_rows<2>(src, Lp, arr, tw, tid);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    K::template pass1<1, 4, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass2<1, 4, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass3<1, 4>(arr, tid);
    __syncthreads();
    cl::CtaState x;
    x.arr = arr;
    x.c = 0;
    x.tw = tw;
    x.tab = tab;
    K::product(x, tid);
    __syncthreads();
    K::template pass3<-1, 2>(arr, tid);
    __syncthreads();
    K::template pass2<-1, 2, 1>(arr, tid, tws);
    __syncthreads();
    K::template pass1<-1, 2, 1>(arr, tid, tws);
    __syncthreads();
    S::store_row(O + (int64_t)row * Kp, Kp, arr, tw, scale, tid);
    return;
  }
  {
    const float2* const src[4] = {F + (int64_t)row * Lp, F + (int64_t)prow * Lp, G + (int64_t)row * Lp,
                                  G + (int64_t)prow * Lp};
    S::template load_rows<4>(src, Lp, arr, tw, tid);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  K::template pass1<1, 8, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass2<1, 8, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass3<1, 8>(arr, tid);
  __syncthreads();
  S::product_pair(arr, zt, cl::ldg2(tw + 1), tid);
  __syncthreads();
  K::template pass3<-1, 4>(arr, tid);
  __syncthreads();
  K::template pass2<-1, 4, 1>(arr, tid, tws);
  __syncthreads();
  K::template pass1<-1, 4, 1>(arr, tid, tws);
  __syncthreads();
  S::store_row(O + (int64_t)row * Kp, Kp, arr, tw, scale, tid);
  S::store_row(O + (int64_t)prow * Kp, Kp, arr + 2 * M, tw, scale, tid);
}

// ---------------------------------------------------------------------------
// Rows with one residue (q = 1): when M >= the real row length, the packed
// row's residue-0 transform alone dealiases (q m >= L), half the work of
// q = 2 (rows of L <= 256 with M = 256, e.g. 3D L = 256).  Arrays [F row,
// F partner, G row, G partner]; C_1 pairs frequency l of the row with
// (M - l) mod M of the partner (the residue-0 rule of Eq. Hr); a row that is
// its own partner pairs l with (M - l) mod M of itself.
// ---------------------------------------------------------------------------
template <int R3>
struct Row1Shape {
  static constexpr int M = 256 * R3;
  static constexpr size_t SMEM = sizeof(float2) * (4 * (size_t)M + cl::Shape<R3>::TABS);
  static constexpr int MINB = R3 == 1 ? 12 : R3 == 2 ? 8 : R3 <= 4 ? 4 : 2;
};

template <int R3>
__global__ void __launch_bounds__(RowShape<R3>::T, Row1Shape<R3>::MINB)
    k_rows_cl1(float2* F, const float2* __restrict__ G, float2* O, RowGeom rg, float scale,
               const float2* __restrict__ tab) {
  using S = RowSteps<R3>;
  using K = typename S::K;
  constexpr int M = S::M, T = S::T;
  constexpr int U = M / 2 / T;
  const int row = blockIdx.x;
  const int prow = row_partner(row, rg);
  if (prow < row) return;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);
  float2* tws = arr + 4 * M;
  const int tid = threadIdx.x;
  for (int i = tid; i < cl::Shape<R3>::TABS / 2; i += T) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tws + 2 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(tab + 2 * i) : "memory");
  }
  const int Lp = rg.Lrow, Kp = rg.Kout;
  const float2* zt = tab + cl::Shape<R3>::TABZ;
  const bool self = (prow == row);
  const int nr = self ? 2 : 4;
  {
    // all loads in flight first: rows [F row, F partner, G row, G partner] (self: [F, G])
    const float2* src[4] = {F + (int64_t)row * Lp, F + (int64_t)prow * Lp, G + (int64_t)row * Lp,
                            G + (int64_t)prow * Lp};
    if (self) src[1] = src[2];
    float2 v[4][U][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int s = 2 * (tid + i * T);
        const bool on = r < nr;
        v[r][i][0] = on && s < Lp ? src[r][s] : make_float2(0.f, 0.f);
        v[r][i][1] = on && s + 1 < Lp ? src[r][s + 1] : make_float2(0.f, 0.f);
      }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r < nr)
#pragma unroll
        for (int i = 0; i < U; ++i) cl::sts4(arr + r * M + phys(2 * (tid + i * T)), v[r][i][0], v[r][i][1]);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  if (self) {
    K::template pass1<1, 2, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass2<1, 2, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass3<1, 2>(arr, tid);
    __syncthreads();
    float2* Fa = arr;
    const float2* Ga = arr + M;
    for (int p = tid; p < M; p += T) {
      const int l = cl::digit_freq(p, R3);
      const int ls = (l == 0) ? 0 : M - l;
      if (l > ls) continue;
      const int ps = cl::digit_pos(ls, R3);
      float2 A = Fa[phys(p)], Ac = Fa[phys(ps)];
      const bool own = (ls == l);
      K::rcm_pair(A, Ga[phys(p)], Ac, Ga[phys(ps)], K::rcm_factor(cl::ldg2(zt + p), make_float2(1.f, 0.f)), own);
      Fa[phys(p)] = A;
      if (!own) Fa[phys(ps)] = Ac;
    }
    __syncthreads();
    K::template pass3<-1, 1>(arr, tid);
    __syncthreads();
    K::template pass2<-1, 1, 1>(arr, tid, tws);
    __syncthreads();
    K::template pass1<-1, 1, 1>(arr, tid, tws);
    __syncthreads();
  } else {
    K::template pass1<1, 4, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass2<1, 4, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass3<1, 4>(arr, tid);
    __syncthreads();
    float2* Fr = arr;
    float2* Fp = arr + M;
    const float2* Gr = arr + 2 * M;
    const float2* Gp = arr + 3 * M;
    for (int p = tid; p < M; p += T) {
      const int l = cl::digit_freq(p, R3);
      const int ps = cl::digit_pos(l == 0 ? 0 : M - l, R3);
      float2 A = Fr[phys(p)], Cs = Fp[phys(ps)];
      K::rcm_pair(A, Gr[phys(p)], Cs, Gp[phys(ps)], K::rcm_factor(cl::ldg2(zt + p), make_float2(1.f, 0.f)), false);
      Fr[phys(p)] = A;
      Fp[phys(ps)] = Cs;
    }
    __syncthreads();
    K::template pass3<-1, 2>(arr, tid);
    __syncthreads();
    K::template pass2<-1, 2, 1>(arr, tid, tws);
    __syncthreads();
    K::template pass1<-1, 2, 1>(arr, tid, tws);
    __syncthreads();
  }
  // h~_s = w_0[s] * scale, s < Kp <= M
  for (int r = 0; r < (self ? 1 : 2); ++r) {
    float2* x = O + (int64_t)(r ? prow : row) * Kp;
    const float2* a = arr + r * M;
    for (int k = tid; k < M / 2; k += T) {
      const int s = 2 * k;
      if (s >= Kp) continue;
      float2 w0, w1;
      cl::lds4(a + phys(s), w0, w1);
      x[s] = cscale(w0, scale);
      if (s + 1 < Kp) x[s + 1] = cscale(w1, scale);
    }
  }
}

template <int R3>
cudaError_t launch_rows1(unsigned grid, cudaStream_t st, float2* F, const float2* G, float2* O, RowGeom rg,
                         float scale, const float2* tab) {
  auto k = k_rows_cl1<R3>;
  cudaError_t e = smem_optin((const void*)k, Row1Shape<R3>::SMEM);
  if (e != cudaSuccess) return e;
  k<<<grid, RowShape<R3>::T, Row1Shape<R3>::SMEM, st>>>(F, G, O, rg, scale, tab);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The adjoint's row pass: C_1 applied to (U, G) and (U, F) for the row pair,
// with U = rev(grad_h)'s outer spectra transformed once and only read; the
// products replace G's and F's rows (outs bit 0: G, bit 1: F).  Arrays: for
// a row pair [U row, U partner, F row, F partner, G row, G partner] x {r0, r1};
// for a row that is its own partner [U, F, G] x {r0, r1}.
// ---------------------------------------------------------------------------
// B_k <- U_k B_k - alpha, B_k* <- U_k* B_k* - conj(alpha),
// alpha = (U_k - conj U_k*)(B_k - conj B_k*) Z.
__host__ __device__ __forceinline__ void dual_pair(float2 Uk, float2 Uc, float2& Bk, float2& Bc, float2 Z, bool self) {
  const float2 alpha = cmul(cmul(csub(Uk, cconj(Uc)), csub(Bk, cconj(Bc))), Z);
  const float2 h1 = csub(cmul(Uk, Bk), alpha);
  if (!self) Bc = csub(cmul(Uc, Bc), cconj(alpha));
  Bk = h1;
}

template <int R3>
struct RowAdjSteps {
  using K = cl::Steps<1, R3>;
  static constexpr int M = K::M;
  static constexpr int T = K::T;

  // arrays: U r0/r1 at u0, u0 + M; partner values at up0 (residue 0 at up0,
  // residue 1 at up0 + M); B arrays likewise at b0 / bp0.  `cross` marks a
  // row pair (partner arrays distinct); otherwise the row pairs with itself.
  static __device__ __forceinline__ void product(float2* arr, int u0, int up0, int nb, const int* b0, const int* bp0,
                                                 bool cross, const float2* __restrict__ zt, float2 z1, int tid) {
    // residue 0: l pairs with (M - l) mod M
    for (int p = tid; p < M; p += T) {
      const int l = cl::digit_freq(p, R3);
      const int ls = (l == 0) ? 0 : M - l;
      if (!cross && l > ls) continue;
      const bool self = !cross && ls == l;
      const int ps = cl::digit_pos(ls, R3);
      const float2 Uk = arr[u0 + phys(p)], Uc = arr[up0 + phys(ps)];
      const float2 Z = K::rcm_factor(cl::ldg2(zt + p), make_float2(1.f, 0.f));
      for (int i = 0; i < nb; ++i) {
        float2 Bk = arr[b0[i] + phys(p)], Bc = arr[bp0[i] + phys(ps)];
        dual_pair(Uk, Uc, Bk, Bc, Z, self);
        arr[b0[i] + phys(p)] = Bk;
        if (!self) arr[bp0[i] + phys(ps)] = Bc;
      }
    }
    // residue 1: position p pairs with M - 1 - p (pairs of positions per task)
    const int NT = cross ? M / 2 : M / 4;
    for (int k = tid; k < NT; k += T) {
      const int p = 2 * k, pp = M - 2 - p;
      float2 U0, U1, C0, C1;
      cl::lds4(arr + u0 + M + phys(p), U0, U1);
      cl::lds4(arr + up0 + M + phys(pp), C1, C0);
      const float4 z = cl::ldg4(zt + p);
      const float2 Z0 = K::rcm_factor(make_float2(z.x, z.y), z1), Z1 = K::rcm_factor(make_float2(z.z, z.w), z1);
      for (int i = 0; i < nb; ++i) {
        float2 B0, B1, D0, D1;
        cl::lds4(arr + b0[i] + M + phys(p), B0, B1);
        cl::lds4(arr + bp0[i] + M + phys(pp), D1, D0);
        dual_pair(U0, C0, B0, D0, Z0, false);
        dual_pair(U1, C1, B1, D1, Z1, false);
        cl::sts4(arr + b0[i] + M + phys(p), B0, B1);
        cl::sts4(arr + bp0[i] + M + phys(pp), D1, D0);
      }
    }
  }
};

template <int R3>
struct RowAdjShape {
  static constexpr size_t SMEM = sizeof(float2) * (12 * (size_t)(256 * R3) + cl::Shape<R3>::TABS);
  static constexpr int MINB = R3 == 1 ? 8 : R3 == 2 ? 4 : R3 <= 4 ? 2 : 1;
};

template <int R3>
__global__ void __launch_bounds__(RowShape<R3>::T, RowAdjShape<R3>::MINB)
    k_rows_adj_cl(float2* F, float2* G, const float2* __restrict__ U, RowGeom rg, float scale, int outs,
                  const float2* __restrict__ tw, const float2* __restrict__ tab) {
  using S = RowSteps<R3>;
  using A = RowAdjSteps<R3>;
  using K = typename S::K;
  constexpr int M = S::M, T = S::T;
  const int row = blockIdx.x;
  const int prow = row_partner(row, rg);
  if (prow < row) return;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);
  float2* tws = arr + 12 * M;
  const int tid = threadIdx.x;
  for (int i = tid; i < cl::Shape<R3>::TABS / 2; i += T) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tws + 2 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(tab + 2 * i) : "memory");
  }
  const int Lp = rg.Lrow;
  const float2* zt = tab + cl::Shape<R3>::TABZ;
  const float2 z1 = cl::ldg2(tw + 1);
  if (prow == row) {  // [U, F, G] x {r0, r1}
    {
      const float2* const src[3] = {U + (int64_t)row * Lp, F + (int64_t)row * Lp, G + (int64_t)row * Lp};
      S::template load_rows<3>(src, Lp, arr, tw, tid);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    K::template pass1<1, 6, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass2<1, 6, 2>(arr, tid, tws);
    __syncthreads();
    K::template pass3<1, 6>(arr, tid);
    __syncthreads();
    const int b0[2] = {2 * M, 4 * M};
    A::product(arr, 0, 0, 2, b0, b0, false, zt, z1, tid);
    __syncthreads();
    K::template pass3<-1, 4>(arr + 2 * M, tid);
    __syncthreads();
    K::template pass2<-1, 4, 1>(arr + 2 * M, tid, tws);
    __syncthreads();
    K::template pass1<-1, 4, 1>(arr + 2 * M, tid, tws);
    __syncthreads();
    if (outs & 1) S::store_row(G + (int64_t)row * Lp, Lp, arr + 4 * M, tw, scale, tid);
    if (outs & 2) S::store_row(F + (int64_t)row * Lp, Lp, arr + 2 * M, tw, scale, tid);
    return;
  }
  // [U row, U partner, F row, F partner, G row, G partner] x {r0, r1}
  {
    const float2* const src[6] = {U + (int64_t)row * Lp, U + (int64_t)prow * Lp, F + (int64_t)row * Lp,
                                  F + (int64_t)prow * Lp, G + (int64_t)row * Lp, G + (int64_t)prow * Lp};
    S::template load_rows<6>(src, Lp, arr, tw, tid);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  K::template pass1<1, 12, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass2<1, 12, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass3<1, 12>(arr, tid);
  __syncthreads();
  const int b0[2] = {4 * M, 8 * M}, bp0[2] = {6 * M, 10 * M};
  A::product(arr, 0, 2 * M, 2, b0, bp0, true, zt, z1, tid);
  __syncthreads();
  K::template pass3<-1, 8>(arr + 4 * M, tid);
  __syncthreads();
  K::template pass2<-1, 8, 1>(arr + 4 * M, tid, tws);
  __syncthreads();
  K::template pass1<-1, 8, 1>(arr + 4 * M, tid, tws);
  __syncthreads();
  if (outs & 1) {
    S::store_row(G + (int64_t)row * Lp, Lp, arr + 8 * M, tw, scale, tid);
    S::store_row(G + (int64_t)prow * Lp, Lp, arr + 10 * M, tw, scale, tid);
  }
  if (outs & 2) {
    S::store_row(F + (int64_t)row * Lp, Lp, arr + 4 * M, tw, scale, tid);
    S::store_row(F + (int64_t)prow * Lp, Lp, arr + 6 * M, tw, scale, tid);
  }
}

template <int R3>
cudaError_t launch_rows_adj(unsigned grid, cudaStream_t st, float2* F, float2* G, const float2* U, RowGeom rg,
                            float scale, int outs, const float2* tw, const float2* tab) {
  auto k = k_rows_adj_cl<R3>;
  cudaError_t e = smem_optin((const void*)k, RowAdjShape<R3>::SMEM);
  if (e != cudaSuccess) return e;
  k<<<grid, RowShape<R3>::T, RowAdjShape<R3>::SMEM, st>>>(F, G, U, rg, scale, outs, tw, tab);
  return cudaGetLastError();
}

template <int R3>
cudaError_t launch_rows(unsigned grid, cudaStream_t st, float2* F, const float2* G, float2* O, RowGeom rg, float scale,
                        const float2* tw, const float2* tab) {
  auto k = k_rows_cl<R3>;
  cudaError_t e = smem_optin((const void*)k, RowShape<R3>::SMEM);
  if (e != cudaSuccess) return e;
  k<<<grid, RowShape<R3>::T, RowShape<R3>::SMEM, st>>>(F, G, O, rg, scale, tw, tab);
  return cudaGetLastError();
}

}  // namespace rows
}  // namespace hd
