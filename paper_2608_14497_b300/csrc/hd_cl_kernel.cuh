// hd_cl_kernel.cuh -- hybridRCM 1D convolutions with the residues of one
// convolution spread over a thread-block cluster: the batched hot path and the
// default single 1D call.
//
// A convolution of real length L (packed length Lp = ceil(L/2), Eq.
// complexPacking) runs on a cluster of C CTAs (C in {1, 2, 4, 8}) with q = 2C
// residues of length M = 256 R3 (R3 in {1,2,3,4,5,6,8,9,10,12,16,18}), so the
// padded packed length is N = q M >= Lp' = L (p = ceil(Lp / M) <= C blocks).
// CTA c owns the conjugate residue pair {c, q - c} (CTA 0: the self-paired
// residues 0 and q/2), so the RCM operator in residue form (Eqs. Hr and
// Hr-conj) needs no data from other CTAs.  Steps:
//   phase 1  (Eq. forwardr, inner sum)  CTA c takes the slice
//            s in [c M/C, (c+1) M/C), reads the p packed inputs x~_{tM+s} of
//            f and of g once, forms sum_t zeta_q^{rt} x_t for every residue r
//            as two length-C DFTs (the inputs vanish for t >= C = q/2),
//            multiplies by zeta_N^{rs} and stores each value into the shared
//            memory of residue r's owner (16-byte distributed-shared-memory
//            stores of two consecutive s);
//   DFTs     length-M DFTs of the four owned arrays (F and G of both
//            residues) by in-place decimation in frequency: passes of radix
//            R3 (stride 256), 16 (stride 16), 16 (stride 1); the spectra end
//            in digit-reversed order, position p holding frequency
//            l = P^-1(p) = p/256 + R3 ((p/16) mod 16) + 16 R3 (p mod 16);
//   product  the RCM operator on the digit-reversed spectra (the partner of
//            position p in the other residue is M-1-p, because digit reversal
//            commutes with the complement l -> M-1-l);
//   inverse  length-M backward DFTs of the two products by in-place
//            decimation in time (the DIF passes transposed, conjugated), which
//            take the digit-reversed order back to natural order (Eq.
//            accumulator);
//   phase 3  (Eq. accumulation) CTA c gathers w_r[s] of every residue for its
//            slice from the owners, applies zeta_N^{-rs} and the backward
//            length-q sum over r for the p needed blocks (two length-C DFTs),
//            scales by 1/N and writes the unpacked real output.
// Inputs are read once and outputs written once: the HBM traffic is the 12
// bytes per real element of the problem plus the L2-resident twiddle tables.
//
// Shared memory: the four arrays F_a, F_b, G_a, G_b, M complex each, element i
// at phys(i) = i ^ (((i >> 4) & 7) << 1): rows of 16 elements whose 16-byte
// chunks are permuted by the row index, so every pass's 128-bit accesses are
// free of bank conflicts (checked by enumeration on the host); behind them the
// pass twiddles, copied from the per-length table while phase 1 runs.
//
// Every step is written as a function of (thread index, CTA state) so the
// same code can be stepped thread by thread on the host; on the device the
// steps are separated by CTA or cluster barriers.  The kernel is instantiated
// per (C, R3): every trip count, stride and table offset is a compile-time
// constant.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hd_bfly.cuh"

namespace hd {
namespace cl {

// ---------------------------------------------------------------------------
// storage, table layout, shapes
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int phys(int i) { return i ^ (((i >> 4) & 7) << 1); }

template <int R3>
struct Shape {
  static constexpr int M = 256 * R3;
  static constexpr int T = 32 * R3;          // threads per CTA
  // CTAs per SM the launch bounds ask registers for (what shared memory allows,
  // up to a register budget that avoids spills)
  static constexpr int MINB = R3 <= 2 ? 8 : R3 == 3 ? 6 : R3 == 4 ? 5 : R3 == 5 ? 4 : R3 == 6 ? 3 : R3 <= 10 ? 2 : 1;
  static constexpr int TAB1 = (R3 - 1) * 256;  // pass 1: zeta_M^{u j}, u = 1..R3-1, j < 256
  static constexpr int TAB2 = 240;           // pass 2: zeta_256^{u j}, u = 1..15, j < 16
  static constexpr int TABZ = TAB1 + TAB2;   // product table: zeta_M^{P^-1(p)}, p < M
  static constexpr int TABN = TABZ + M;      // entries of the per-length table
  static constexpr int TABS = TAB1 + TAB2;    // pass twiddles, copied to shared memory behind the arrays
  static constexpr size_t SMEM = sizeof(float2) * (4 * (size_t)M + TABS);
};

// Frequency held at position p of a digit-reversed length-M spectrum.
__host__ __device__ __forceinline__ int digit_freq(int p, int R3) {
  return (p >> 8) + R3 * ((p >> 4) & 15) + 16 * R3 * (p & 15);
}
// Position of frequency l (the inverse of digit_freq).
__host__ __device__ __forceinline__ int digit_pos(int l, int R3) {
  const int u1 = l % R3, rest = l / R3;
  return 256 * u1 + 16 * (rest & 15) + (rest >> 4);
}

// ---------------------------------------------------------------------------
// memory helpers (device instructions, or plain accesses when stepped on the host)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 ldg2(const float2* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}
__host__ __device__ __forceinline__ float4 ldg4(const float2* p) {
#ifdef __CUDA_ARCH__
  return __ldg(reinterpret_cast<const float4*>(p));
#else
  return *reinterpret_cast<const float4*>(p);
#endif
}
__host__ __device__ __forceinline__ float ldgf(const float* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}
__host__ __device__ __forceinline__ void lds4(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__host__ __device__ __forceinline__ void sts4(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}

// Address of a CTA's shared memory as seen from the cluster: a 32-bit
// shared::cluster address on the device, a host pointer when stepped on the host.
#ifdef __CUDA_ARCH__
typedef unsigned raddr_t;
#else
typedef char* raddr_t;
#endif
// 16-byte store into a cluster CTA's shared memory that, once written,
// completes 16 bytes of the transaction count of that CTA's mbarrier `bar`
// (st.async: no fence at the sender; the receiver waits on its own barrier).
__host__ __device__ __forceinline__ void rst4_async(raddr_t a, float2 v0, float2 v1, raddr_t bar) {
#ifdef __CUDA_ARCH__
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];\n" ::"r"(a),
               "f"(v0.x), "f"(v0.y), "f"(v1.x), "f"(v1.y), "r"(bar)
               : "memory");
#else
  (void)bar;
  *reinterpret_cast<float4*>(a) = make_float4(v0.x, v0.y, v1.x, v1.y);
#endif
}
// 8-byte form of rst4_async.
__host__ __device__ __forceinline__ void rst2_async(raddr_t a, float2 v, raddr_t bar) {
#ifdef __CUDA_ARCH__
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n" ::"r"(a),
               "f"(v.x), "f"(v.y), "r"(bar)
               : "memory");
#else
  (void)bar;
  *reinterpret_cast<float2*>(a) = v;
#endif
}

// zeta_32^e = (cos, sin)(2 pi e / 32) (the residue sums over the blocks t use
// zeta_{2C}^t = zeta_32^{16 t / C}), exact values rounded to FP32.
template <int SIGN>
__host__ __device__ __forceinline__ float2 root32(int e) {
  const float c[32] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                       0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                       0.19509032201612826785f, 0.0f, -0.19509032201612826785f, -0.38268343236508977173f,
                       -0.55557023301960222474f, -0.70710678118654752440f, -0.83146961230254523708f,
                       -0.92387953251128675613f, -0.98078528040323044913f, -1.0f, -0.98078528040323044913f,
                       -0.92387953251128675613f, -0.83146961230254523708f, -0.70710678118654752440f,
                       -0.55557023301960222474f, -0.38268343236508977173f, -0.19509032201612826785f, 0.0f,
                       0.19509032201612826785f, 0.38268343236508977173f, 0.55557023301960222474f,
                       0.70710678118654752440f, 0.83146961230254523708f, 0.92387953251128675613f,
                       0.98078528040323044913f};
  const int es = e & 31;
  return make_float2(c[es], SIGN * c[(es + 24) & 31]);  // sin x = cos(x - pi/2)
}

template <int SIGN, int CC>
__host__ __device__ __forceinline__ void dft_small(float2* v) {
  if constexpr (CC == 2) dft2<SIGN>(v[0], v[1]);
  else if constexpr (CC == 4) dft4<SIGN>(v[0], v[1], v[2], v[3]);
  else if constexpr (CC == 8) dft8<SIGN>(v);
  else if constexpr (CC == 16) dft16<SIGN>(v);
}

// zeta_N^{r s} for r < Q from the zeta_N table: up to four table reads
// (zeta^s, zeta^{4s}, zeta^{8s}, zeta^{16s}) and at most 27 complex products.
template <int Q>
__host__ __device__ __forceinline__ void residue_twiddles(const float2* tw, int s, float2* w) {
  w[0] = make_float2(1.f, 0.f);
  if constexpr (Q >= 2) w[1] = ldg2(tw + s);
  if constexpr (Q >= 4) {
    w[2] = cmul(w[1], w[1]);
    w[3] = cmul(w[2], w[1]);
  }
  if constexpr (Q >= 8) {
    w[4] = ldg2(tw + 4 * s);
#pragma unroll
    for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
  }
  if constexpr (Q >= 16) {
    w[8] = ldg2(tw + 8 * s);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
  }
  if constexpr (Q >= 32) {
    w[16] = ldg2(tw + 16 * s);
#pragma unroll
    for (int r = 17; r < 32; ++r) w[r] = cmul(w[16], w[r - 16]);
  }
}

// The same twiddles built one at a time from six bases (for q = 32 residues,
// where holding all of them would exhaust the registers): zeta_N^{r s} =
// w16^{b4} w8^{b3} w4^{b2} w1^{r mod 4} for r = 16 b4 + 8 b3 + 4 b2 + (r mod 4).
struct TwBases {
  float2 w1, w2, w3, w4, w8, w16;
};
__host__ __device__ __forceinline__ TwBases twiddle_bases(const float2* tw, int s) {
  TwBases b;
  b.w1 = ldg2(tw + s);
  b.w2 = cmul(b.w1, b.w1);
  b.w3 = cmul(b.w2, b.w1);
  b.w4 = ldg2(tw + 4 * s);
  b.w8 = ldg2(tw + 8 * s);
  b.w16 = ldg2(tw + 16 * s);
  return b;
}
__host__ __device__ __forceinline__ float2 twiddle_of(const TwBases& b, int r) {
  float2 t = make_float2(1.f, 0.f);
  bool one = true;
  const int lo = r & 3;
  if (lo) {
    t = lo == 1 ? b.w1 : lo == 2 ? b.w2 : b.w3;
    one = false;
  }
  if (r & 4) {
    t = one ? b.w4 : cmul(t, b.w4);
    one = false;
  }
  if (r & 8) {
    t = one ? b.w8 : cmul(t, b.w8);
    one = false;
  }
  if (r & 16) t = one ? b.w16 : cmul(t, b.w16);
  return t;
}

__host__ __device__ __forceinline__ int owner_of(int r, int C) { return r < C ? r : (r == C ? 0 : 2 * C - r); }
__host__ __device__ __forceinline__ int slot_of(int r, int C) { return r < C ? 0 : 1; }

// What one CTA needs for the exchange phases and the product.
struct CtaState {
  const float* f;
  const float* g;
  float* h;
  int64_t off;
  int L, Lp, p, c;        // real length, packed length, blocks, rank in the cluster
  int64_t off_in;         // offset of the item in the input arrays
  int Lin, pin;           // real length of the input arrays' item and the blocks read
  int Lout, pout;         // real length of the output (L <= Lout <= 2L - 1) and the blocks written
  bool in16, in8, out16;  // f + off and g + off 16- / 8-byte aligned; h + off 16-byte aligned
  const float2* tw;       // zeta_N^k, N = 2 C M
  const float2* tab;      // per-length table (Shape::TAB1 | TAB2 | product)
  float2* arr;            // this CTA's four arrays
  raddr_t rbase[16];      // every CTA's arrays, as seen from this CTA
  raddr_t rbar1[16];      // every CTA's phase-1 mbarrier (its four arrays received)
  raddr_t rbar3[16];      // every CTA's phase-3 mbarrier (its gather buffer received)
};

// ---------------------------------------------------------------------------
// the kernel's steps
// ---------------------------------------------------------------------------
// EXP: the explicit-padding baseline on the same engine: the input arrays are
// materialised zero-padded copies (real length 2L), every block t < q of them
// is read (no block is known to be zero) and the q-point sum over t is the
// full DFT, x_t and x_{t+C} combined before the two length-C DFTs.
// TT: threads that run the steps (the cluster kernel: Shape<R3>::T; the
// row-pair kernel of the nD path may give a short row more threads).
template <int C, int R3, bool EXP = false, int TT = Shape<R3>::T>
struct Steps {
  using S = Shape<R3>;
  static constexpr int M = S::M;
  static constexpr int T = TT;
  static constexpr int Q = 2 * C;
  static constexpr int SL = M / C;                  // slice of s per CTA
  static constexpr int SW1 = (C >= 16) ? 1 : 2;     // s per phase-1 task
  static constexpr int NT1 = 2 * SL / SW1;          // phase-1 tasks: {f, g} x s-pairs
  static constexpr int SW3 = (SL >= 2 * T) ? 2 : 1; // s per phase-3 task
  static constexpr int NT3 = SL / SW3;
  static constexpr int U1 = (NT1 + T - 1) / T;      // phase-1 tasks per thread
  static constexpr int NB = EXP ? 2 * C : C;        // blocks t read per s

  // ---- phase 1 ------------------------------------------------------------
  // Packed inputs x~_j, j = t M + s + w (w < 2), of array `which`; zero past Lp.
  static __host__ __device__ __forceinline__ void load_task(const CtaState& x, int task, float2 (&v)[NB][2]) {
    const int which = task / (SL / SW1);
    const int s = x.c * SL + (task - which * (SL / SW1)) * SW1;
    const float* src = (which ? x.g : x.f) + x.off_in;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int j = t * M + s;
      v[t][0] = v[t][1] = make_float2(0.f, 0.f);
      if (t < x.pin && SW1 == 1) {
        const int rem = x.Lin - 2 * j;
        if (rem >= 2 && x.in8) {
#ifdef __CUDA_ARCH__
          v[t][0] = __ldg(reinterpret_cast<const float2*>(src + 2 * j));
#else
          v[t][0] = *reinterpret_cast<const float2*>(src + 2 * j);
#endif
        } else {
          if (rem > 0) v[t][0].x = ldgf(src + 2 * j);
          if (rem > 1) v[t][0].y = ldgf(src + 2 * j + 1);
        }
      } else if (t < x.pin) {
        const int rem = x.Lin - 2 * j;  // real values left from 2j
        if (rem >= 4 && x.in16) {
#ifdef __CUDA_ARCH__
          const float4 a = __ldg(reinterpret_cast<const float4*>(src + 2 * j));
#else
          const float4 a = *reinterpret_cast<const float4*>(src + 2 * j);
#endif
          v[t][0] = make_float2(a.x, a.y);
          v[t][1] = make_float2(a.z, a.w);
        } else if (rem >= 4 && x.in8) {
#ifdef __CUDA_ARCH__
          const float2 a = __ldg(reinterpret_cast<const float2*>(src + 2 * j));
          const float2 b = __ldg(reinterpret_cast<const float2*>(src + 2 * j + 2));
#else
          const float2 a = *reinterpret_cast<const float2*>(src + 2 * j);
          const float2 b = *reinterpret_cast<const float2*>(src + 2 * j + 2);
#endif
          v[t][0] = a;
          v[t][1] = b;
        } else {
          if (rem > 0) v[t][0].x = ldgf(src + 2 * j);
          if (rem > 1) v[t][0].y = ldgf(src + 2 * j + 1);
          if (rem > 2) v[t][1].x = ldgf(src + 2 * j + 2);
          if (rem > 3) v[t][1].y = ldgf(src + 2 * j + 3);
        }
      }
    }
  }

  // Sum over t for every residue, pre-twiddle, store into the owners' arrays.
  // The sum over t: e_t = x_t (+ x_{t+C}), o_t = zeta_q^t (x_t (- x_{t+C})).
  static __host__ __device__ __forceinline__ void split_blocks(const float2 (&v)[NB][2], int w, float2* e, float2* o) {
#pragma unroll
    for (int t = 0; t < C; ++t) {
      const float2 a = EXP ? cadd(v[t][w], v[t + (EXP ? C : 0)][w]) : v[t][w];
      const float2 b = EXP ? csub(v[t][w], v[t + (EXP ? C : 0)][w]) : v[t][w];
      e[t] = a;
      o[t] = (t == 0) ? b : cmul(b, root32<1>(t * (16 / C)));  // zeta_q^t
    }
  }

  static __host__ __device__ __forceinline__ void scatter_task(const CtaState& x, int task, const float2 (&v)[NB][2]) {
    const int which = task / (SL / SW1);
    const int s = x.c * SL + (task - which * (SL / SW1)) * SW1;
    if constexpr (SW1 == 1) {
      // one s, every residue stored as soon as it is formed
      float2 e[C], o[C];
      split_blocks(v, 0, e, o);
      dft_small<1, C>(e);
      dft_small<1, C>(o);
      const TwBases tb = twiddle_bases(x.tw, s);
      const int ps = phys(s);
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const float2 a = (r & 1) ? o[r >> 1] : e[r >> 1];
        const int ow = owner_of(r, C), sl = slot_of(r, C);
        const int idx = (which * 2 + sl) * M + ps;
        rst2_async(x.rbase[ow] + (size_t)idx * sizeof(float2), r == 0 ? a : cmul(a, twiddle_of(tb, r)), x.rbar1[ow]);
      }
      return;
    }
    float2 y[2][Q];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      float2 e[C], o[C];
      split_blocks(v, w, e, o);
      dft_small<1, C>(e);
      dft_small<1, C>(o);
      float2 wr[Q];
      residue_twiddles<Q>(x.tw, s + w, wr);
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const float2 a = (r & 1) ? o[r >> 1] : e[r >> 1];
        y[w][r] = (r == 0) ? a : cmul(a, wr[r]);
      }
    }
    const int ps = phys(s);
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      const int ow = owner_of(r, C), sl = slot_of(r, C);
      const int idx = (which * 2 + sl) * M + ps;  // element index in the owner's arrays
      if constexpr (C == 1) sts4(x.arr + idx, y[0][r], y[1][r]);  // one CTA: its own arrays
      else rst4_async(x.rbase[ow] + (size_t)idx * sizeof(float2), y[0][r], y[1][r], x.rbar1[ow]);
    }
  }

  // ---- length-M DFTs: in-place DIF (forward) and DIT (backward) passes -----
  // Pass 1: radix R3, stride 256 (transform size M), twiddles zeta_M^{u j}
  // read from `tws` (the table's first TABS entries, in shared memory).
  // Task = (array, pair of adjacent j) for W = 2, (array, j) for W = 1.
  template <int SIGN, int NARR, int W>
  static __host__ __device__ __forceinline__ void pass1(float2* arr, int tid, const float2* tws) {
    if constexpr (R3 > 1) {
      constexpr int PER = 256 / W;
      constexpr int NT = NARR * PER;
#pragma unroll
      for (int k = 0; k < (NT + T - 1) / T; ++k) {
        const int task = tid + k * T;
        if (NT % T == 0 || task < NT) {
          const int a = task / PER;
          const int j = (task - a * PER) * W;
          float2* x = arr + a * M;
          float2 v[W][R3];
#pragma unroll
          for (int u = 0; u < R3; ++u) {
            if constexpr (W == 2) lds4(x + phys(j + 256 * u), v[0][u], v[1][u]);
            else v[0][u] = x[phys(j + 256 * u)];
          }
          if constexpr (SIGN < 0) {  // DIT: conjugate twiddles first
#pragma unroll
            for (int u = 1; u < R3; ++u) {
              if constexpr (W == 2) {
                const float4 t = *reinterpret_cast<const float4*>(tws + (u - 1) * 256 + j);
                v[0][u] = cmul(v[0][u], make_float2(t.x, -t.y));
                v[1][u] = cmul(v[1][u], make_float2(t.z, -t.w));
              } else {
                v[0][u] = cmul(v[0][u], cconj(tws[(u - 1) * 256 + j]));
              }
            }
          }
#pragma unroll
          for (int b = 0; b < W; ++b) dft_reg<R3, SIGN>(v[b]);
          if constexpr (SIGN > 0) {  // DIF: twiddles after the butterfly
#pragma unroll
            for (int u = 1; u < R3; ++u) {
              if constexpr (W == 2) {
                const float4 t = *reinterpret_cast<const float4*>(tws + (u - 1) * 256 + j);
                v[0][u] = cmul(v[0][u], make_float2(t.x, t.y));
                v[1][u] = cmul(v[1][u], make_float2(t.z, t.w));
              } else {
                v[0][u] = cmul(v[0][u], tws[(u - 1) * 256 + j]);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < R3; ++u) {
            if constexpr (W == 2) sts4(x + phys(j + 256 * u), v[0][u], v[1][u]);
            else x[phys(j + 256 * u)] = v[0][u];
          }
        }
      }
    }
  }

  // Pass 2: radix 16, stride 16, inside each of the R3 blocks of 256;
  // twiddles zeta_256^{u j}, j < 16.
  template <int SIGN, int NARR, int W>
  static __host__ __device__ __forceinline__ void pass2(float2* arr, int tid, const float2* tws) {
    constexpr int PER = 16 / W;          // tasks per block
    constexpr int NT = NARR * R3 * PER;
    const float2* t2 = tws + S::TAB1;
#pragma unroll
    for (int k = 0; k < (NT + T - 1) / T; ++k) {
      const int task = tid + k * T;
      if (NT % T == 0 || task < NT) {
        const int ab = task / PER;                    // array * R3 + block
        const int j = (task - ab * PER) * W;
        float2* x = arr + ab * 256;                   // arrays are R3 blocks of 256 back to back
        float2 v[W][16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          if constexpr (W == 2) lds4(x + phys(j + 16 * u), v[0][u], v[1][u]);
          else v[0][u] = x[phys(j + 16 * u)];
        }
        if constexpr (SIGN < 0) {
#pragma unroll
          for (int u = 1; u < 16; ++u) {
            if constexpr (W == 2) {
              const float4 t = *reinterpret_cast<const float4*>(t2 + (u - 1) * 16 + j);
              v[0][u] = cmul(v[0][u], make_float2(t.x, -t.y));
              v[1][u] = cmul(v[1][u], make_float2(t.z, -t.w));
            } else {
              v[0][u] = cmul(v[0][u], cconj(t2[(u - 1) * 16 + j]));
            }
          }
        }
#pragma unroll
        for (int b = 0; b < W; ++b) dft16<SIGN>(v[b]);
        if constexpr (SIGN > 0) {
#pragma unroll
          for (int u = 1; u < 16; ++u) {
            if constexpr (W == 2) {
              const float4 t = *reinterpret_cast<const float4*>(t2 + (u - 1) * 16 + j);
              v[0][u] = cmul(v[0][u], make_float2(t.x, t.y));
              v[1][u] = cmul(v[1][u], make_float2(t.z, t.w));
            } else {
              v[0][u] = cmul(v[0][u], t2[(u - 1) * 16 + j]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          if constexpr (W == 2) sts4(x + phys(j + 16 * u), v[0][u], v[1][u]);
          else x[phys(j + 16 * u)] = v[0][u];
        }
      }
    }
  }

  // Pass 3: radix 16, stride 1: each task one row of 16 consecutive elements
  // (eight 16-byte chunks, permuted by phys inside the row).  No twiddles.
  template <int SIGN, int NARR>
  static __host__ __device__ __forceinline__ void pass3(float2* arr, int tid) {
    constexpr int NT = NARR * M / 16;
#pragma unroll
    for (int k = 0; k < (NT + T - 1) / T; ++k) {
      const int row = tid + k * T;
      if (NT % T == 0 || row < NT) {
        float2* x = arr + row * 16;
        const int sw = (row & 7) << 1;
        float2 v[16];
#pragma unroll
        for (int c2 = 0; c2 < 16; c2 += 2) lds4(x + (c2 ^ sw), v[c2], v[c2 + 1]);
        dft16<SIGN>(v);
#pragma unroll
        for (int c2 = 0; c2 < 16; c2 += 2) sts4(x + (c2 ^ sw), v[c2], v[c2 + 1]);
      }
    }
  }

  // ---- RCM product on the digit-reversed spectra ---------------------------
  // (1 + zeta_N^k) / 4 with k = q l + r, l = P^-1(p): zeta_N^k = zeta_M^l zeta_N^r.
  static __host__ __device__ __forceinline__ float2 rcm_factor(float2 zl, float2 zr) {
    const float2 z = cmul(zl, zr);
    return make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
  }
  // H_k = A B - alpha, H_k* = Ac Bc - conj(alpha), alpha = (A - conj Ac)(B - conj Bc) Z.
  static __host__ __device__ __forceinline__ void rcm_pair(float2& A, float2 B, float2& Ac, float2 Bc, float2 Z,
                                                           bool self) {
    const float2 alpha = cmul(cmul(csub(A, cconj(Ac)), csub(B, cconj(Bc))), Z);
    const float2 h1 = csub(cmul(A, B), alpha);
    if (!self) Ac = csub(cmul(Ac, Bc), cconj(alpha));
    A = h1;
  }

  // Task k: a pair of positions (p, p+1) of slot a's arrays and their
  // partners (M-2-p, M-1-p) of slot b's arrays (residues c and q - c), or, for
  // CTA 0, residue q/2 (slot 1, partner M-1-p in the same array, p < M/2) and
  // residue 0 (slot 0, partner P((M - l) mod M), one position per task).
  static __host__ __device__ __forceinline__ void product(const CtaState& x, int tid) {
    float2* Fa = x.arr;
    float2* Fb = x.arr + M;
    float2* Ga = x.arr + 2 * M;
    float2* Gb = x.arr + 3 * M;
    const float2* zt = x.tab + S::TABZ;
    if (x.c > 0) {
      const float2 zr = ldg2(x.tw + x.c);  // zeta_N^c (residue c; residue q-c uses the conjugate pairing)
      constexpr int NT = M / 2;
#pragma unroll 2
      for (int task = tid; task < NT; task += T) {
        const int p = 2 * task, pp = M - 2 - p;
        float2 A0, A1, B0, B1, C0, C1, D0, D1;
        lds4(Fa + phys(p), A0, A1);
        lds4(Ga + phys(p), B0, B1);
        lds4(Fb + phys(pp), C1, C0);  // C0 pairs with A0 (position M-1-p), C1 with A1 (M-2-p)
        lds4(Gb + phys(pp), D1, D0);
        const float4 z = ldg4(zt + p);
        rcm_pair(A0, B0, C0, D0, rcm_factor(make_float2(z.x, z.y), zr), false);
        rcm_pair(A1, B1, C1, D1, rcm_factor(make_float2(z.z, z.w), zr), false);
        sts4(Fa + phys(p), A0, A1);
        sts4(Fb + phys(pp), C1, C0);
      }
    } else {
      // residue q/2 = C: zeta_N^C, partner M-1-p in the same arrays
      const float2 zc = ldg2(x.tw + C);
      constexpr int NTB = M / 4;
      for (int task = tid; task < NTB; task += T) {
        const int p = 2 * task, pp = M - 2 - p;
        float2 A0, A1, B0, B1, C0, C1, D0, D1;
        lds4(Fb + phys(p), A0, A1);
        lds4(Gb + phys(p), B0, B1);
        lds4(Fb + phys(pp), C1, C0);
        lds4(Gb + phys(pp), D1, D0);
        const float4 z = ldg4(zt + p);
        rcm_pair(A0, B0, C0, D0, rcm_factor(make_float2(z.x, z.y), zc), false);
        rcm_pair(A1, B1, C1, D1, rcm_factor(make_float2(z.z, z.w), zc), false);
        sts4(Fb + phys(p), A0, A1);
        sts4(Fb + phys(pp), C1, C0);
      }
      // residue 0: l pairs with (M - l) mod M; l = 0 and l = M/2 pair with themselves
      for (int p = tid; p < M; p += T) {
        const int l = digit_freq(p, R3);
        const int ls = (l == 0) ? 0 : M - l;
        if (l > ls) continue;
        const int ps = digit_pos(ls, R3);
        float2 A = Fa[phys(p)], B = Ga[phys(p)];
        float2 Ac = Fa[phys(ps)], Bc = Ga[phys(ps)];
        const bool self = (ls == l);
        rcm_pair(A, B, Ac, Bc, rcm_factor(ldg2(zt + p), make_float2(1.f, 0.f)), self);
        Fa[phys(p)] = A;
        if (!self) Fa[phys(ps)] = Ac;
      }
    }
  }

  // ---- phase 3 --------------------------------------------------------------
  // Each owner pushes w_r[s] of its two residues to the CTA whose slice holds
  // s, into that CTA's gather buffer (its G arrays, free after the product):
  // buffer index r SL + (s - d SL) for residue r and destination d = s / SL.
  // Task k of destination D: (slot, pair of s in D's slice), k < SL.
  template <int D>
  static __host__ __device__ __forceinline__ void push_task(const CtaState& x, int k) {
    const int slot = k / (SL / 2);
    const int sl = 2 * (k - slot * (SL / 2));
    const int s = D * SL + sl;
    const int r = slot ? (x.c == 0 ? C : Q - x.c) : x.c;
    float2 a0, a1;
    lds4(x.arr + slot * M + phys(s), a0, a1);
    rst4_async(x.rbase[D] + (size_t)(2 * M + r * SL + sl) * sizeof(float2), a0, a1, x.rbar3[D]);
  }
  template <int D = 0>
  static __host__ __device__ __forceinline__ void push_all(const CtaState& x, int tid) {
    if constexpr (D < C) {
#pragma unroll
      for (int k = tid; k < SL; k += T) push_task<D>(x, k);
      push_all<D + 1>(x, tid);
    }
  }

  // w_r[s] from the gather buffer (one CTA: from its own arrays), zeta_N^{-rs},
  // the backward sum over r for t < p, scale, unpacked stores.
  static __host__ __device__ __forceinline__ void gather_task(const CtaState& x, int task, float sc) {
    const int sl = task * SW3;
    const int s = x.c * SL + sl;
    const float2* buf = x.arr + 2 * M;
    if constexpr (Q >= 32) {
      static_assert(SW3 == 1, "q = 32 gathers one s per task");
      // residues read and twiddled one at a time into the two length-C sums
      const TwBases tb = twiddle_bases(x.tw, s);
      float2 e[C], o[C];
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const float2 y = buf[r * SL + sl];
        const float2 v = (r == 0) ? y : cmul(y, cconj(twiddle_of(tb, r)));
        if (r & 1) o[r >> 1] = v;
        else e[r >> 1] = v;
      }
      dft_small<-1, C>(e);
      dft_small<-1, C>(o);
      float* hi = x.h + x.off;
#pragma unroll
      for (int t = 0; t < C; ++t) {
        const float2 ov = (t == 0) ? o[0] : cmul(o[t], root32<-1>(t * (16 / C)));
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // blocks t and t + C (zeta_q^{-C} = -1)
          if (t + half * C < x.pout) {
            const float2 out = cscale(half ? csub(e[t], ov) : cadd(e[t], ov), sc);
            const int j = (t + half * C) * M + s;
            const int rem = x.Lout - 2 * j;
            if (rem > 0) hi[2 * j] = out.x;
            if (rem > 1) hi[2 * j + 1] = out.y;
          }
        }
      }
      return;
    }
    float2 y[SW3][Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      if constexpr (C == 1) {  // one CTA: residue r's result is its array r, in natural order
        static_assert(SW3 == 2, "one CTA gathers pairs of s");
        lds4(x.arr + r * M + phys(s), y[0][r], y[1][r]);
      } else if constexpr (SW3 == 2) {
        lds4(buf + r * SL + sl, y[0][r], y[1][r]);
      } else {
        y[0][r] = buf[r * SL + sl];
      }
    }
    float2 out[SW3][2 * C];  // blocks t < 2C; t >= C only for outputs beyond L
#pragma unroll
    for (int w = 0; w < SW3; ++w) {
      float2 wr[Q];
      residue_twiddles<Q>(x.tw, s + w, wr);
      float2 e[C], o[C];
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const float2 v = (r == 0) ? y[w][r] : cmul(y[w][r], cconj(wr[r]));
        if (r & 1) o[r >> 1] = v;
        else e[r >> 1] = v;
      }
      dft_small<-1, C>(e);
      dft_small<-1, C>(o);
#pragma unroll
      for (int t = 0; t < C; ++t) {
        const float2 ov = (t == 0) ? o[0] : cmul(o[t], root32<-1>(t * (16 / C)));
        out[w][t] = cscale(cadd(e[t], ov), sc);
        out[w][t + C] = cscale(csub(e[t], ov), sc);  // zeta_q^{-C t'} = (-1)^r
      }
    }
    float* hi = x.h + x.off;
#pragma unroll
    for (int t = 0; t < 2 * C; ++t) {
      if (t < x.pout) {
        const int j = t * M + s;
        const int rem = x.Lout - 2 * j;
        if constexpr (SW3 == 2) {
          if (rem >= 4 && x.out16) {
            *reinterpret_cast<float4*>(hi + 2 * j) = make_float4(out[0][t].x, out[0][t].y, out[1][t].x, out[1][t].y);
          } else {
            if (rem > 0) hi[2 * j] = out[0][t].x;
            if (rem > 1) hi[2 * j + 1] = out[0][t].y;
            if (rem > 2) hi[2 * j + 2] = out[1][t].x;
            if (rem > 3) hi[2 * j + 3] = out[1][t].y;
          }
        } else {
          if (rem > 0) hi[2 * j] = out[0][t].x;
          if (rem > 1) hi[2 * j + 1] = out[0][t].y;
        }
      }
    }
  }
};

}  // namespace cl
}  // namespace hd

namespace hd {
namespace cl {

// Entry i of the per-length table of Shape<R3> as the exact angle 2 pi num / den.
__host__ __device__ __forceinline__ void table_angle(int i, int R3, long long* num, long long* den) {
  const int M = 256 * R3, tab1 = (R3 - 1) * 256, tabz = tab1 + 240;
  if (i < tab1) {  // pass 1: zeta_M^{u j}
    const int u = i / 256 + 1, j = i % 256;
    *num = (long long)u * j;
    *den = M;
  } else if (i < tabz) {  // pass 2: zeta_256^{u j}
    const int k = i - tab1;
    const int u = k / 16 + 1, j = k % 16;
    *num = (long long)u * j;
    *den = 256;
  } else {  // product: zeta_M^{P^-1(p)}
    *num = digit_freq(i - tabz, R3);
    *den = M;
  }
}

}  // namespace cl
}  // namespace hd
