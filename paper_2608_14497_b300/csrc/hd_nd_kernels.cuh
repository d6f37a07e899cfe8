// hd_nd_kernels.cuh -- device kernels of the 2D/3D recursion (Sec. 5) and of
// the explicit baselines' row transforms, with the launch helpers of the
// per-family translation units (hd_nd_colf.cu, hd_nd_colb.cu, hd_nd_csf.cu,
// hd_nd_csb.cu, hd_nd_rows.cu, hd_nd_cconv.cu, hd_nd_rfft.cu): each of those
// instantiates one kernel family in its three DFT engines, so the families
// compile in parallel.  The host drivers are in hd_nd.cu.
//
// Layout of transformed outer dimensions: residue-major rows, index r m + l
// for the natural frequency k = q l + r.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "hd_conv1d.cuh"
#include "hd_internal.h"

namespace hd {

// ---------------------------------------------------------------------------
// shared device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int modmul(int a, int b, int N) { return (int)(((int64_t)a * b) % N); }

// Natural index of storage row r m + l is q l + r; its conjugate partner
// (M - k) mod M in storage form.
__device__ __forceinline__ int partner_row(int idx, int m, int q) {
  const int r = idx / m, l = idx - r * m;
  if (r == 0) return (l == 0) ? 0 : (m - l);
  return (q - r) * m + (m - 1 - l);
}

// Column geometry: the transformed dimension has stride B (elements) inside
// blocks of A; a CTA owns W consecutive columns b0..b0+W-1 of one block a.
struct ColGeom {
  int64_t A, B;   // outer block count, inner (contiguous) extent
  int W;          // columns per CTA
  int64_t Bp;     // packed last-dimension length inside B (real packing modes)
};

// Real offset of packed element (row j of block a, column b): the inner index
// b runs over (B / Bp) rows of Bp packed pairs, each row Lreal reals long.
__device__ __forceinline__ int64_t packed_offset(const ColGeom& cg, int64_t a, int64_t Lrows, int64_t j, int64_t b,
                                                 int Lreal, int64_t* c) {
  const int64_t sub = b / cg.Bp;
  *c = 2 * (b - sub * cg.Bp);
  return ((a * Lrows + j) * (cg.B / cg.Bp) + sub) * (int64_t)Lreal;
}

// Mirror image of packed element (row j of block a, column b) in a real array
// reversed on every axis inside its block: rows Lrows-1-j, sub-rows
// (B/Bp)-1-sub, reals Lreal-1-2c' and Lreal-2-2c' (the second absent when
// 2c'+1 >= Lreal).  Returns the real offset of the first; *second is -1 when
// there is none.  The adjoint reads rev(u) and writes rev(result) this way.
__device__ __forceinline__ int64_t packed_offset_rev(const ColGeom& cg, int64_t a, int64_t Lrows, int64_t j,
                                                     int64_t b, int Lreal, int64_t* second) {
  const int64_t nsub = cg.B / cg.Bp;
  const int64_t sub = b / cg.Bp;
  const int64_t c2 = 2 * (b - sub * cg.Bp);
  const int64_t base = ((a * Lrows + (Lrows - 1 - j)) * nsub + (nsub - 1 - sub)) * (int64_t)Lreal;
  *second = (c2 + 1 < Lreal) ? base + Lreal - 2 - c2 : -1;
  return base + Lreal - 1 - c2;
}

// Element loop in batches: for idx < total, v = f(idx) (global loads) then
// g(idx, v) (shared stores); the f of KT elements per thread are all issued
// before the first g, so a CTA waits for one round of memory latency per KT T
// elements instead of one per element.
template <int KT, typename V, typename LoadFn, typename StoreFn>
__device__ __forceinline__ void batched(int total, LoadFn f, StoreFn g) {
  const int T = blockDim.x;
  for (int base = 0; base < total; base += KT * T) {
    V v[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int idx = base + threadIdx.x + k * T;
      if (idx < total) v[k] = f(idx);
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int idx = base + threadIdx.x + k * T;
      if (idx < total) g(idx, v[k]);
    }
  }
}

// Column strips: the W columns b0..b0+W-1 (W a power of two <= 8) of n rows,
// moved between global memory and shared arrays s[w * ld + j].  Element
// id = tid + k T is row j = id / W, column w = id mod W, so a warp reads whole
// 32-byte sectors of consecutive columns; the loads of KT elements per thread
// are all issued before the first shared store (one round of memory latency
// per KT T elements, not one per element).
template <int KT, typename LoadFn>
__device__ __forceinline__ void strip_load(float2* s, int ld, int n, int W, LoadFn f) {
  const int T = blockDim.x, total = n * W;
  const int wl = __ffs(W) - 1;
  for (int base = 0; base < total; base += KT * T) {
    float2 v[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int id = base + threadIdx.x + k * T;
      v[k] = id < total ? f(id >> wl, id & (W - 1)) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int id = base + threadIdx.x + k * T;
      if (id < total) s[(id & (W - 1)) * ld + (id >> wl)] = v[k];
    }
  }
}

template <typename StoreFn>
__device__ __forceinline__ void strip_store(const float2* s, int ld, int n, int W, StoreFn g) {
  const int T = blockDim.x, total = n * W;
  const int wl = __ffs(W) - 1;
  for (int id = threadIdx.x; id < total; id += T) {
    const int j = id >> wl, w = id & (W - 1);
    g(j, w, s[w * ld + j]);
  }
}

// Input element loaders for the column passes.
enum : int { IN_COMPLEX = 0, IN_PACKED_REAL = 1, IN_PACKED_REAL_REV = 2 };
enum : int { OUT_COMPLEX = 0, OUT_UNPACK_REAL = 1, OUT_UNPACK_REAL_REV = 2 };

// ---------------------------------------------------------------------------
// k_col_fwd: complex hybrid forward transform along a strided dimension.
//   X: [A][Lin][B] complex (or real packed along B: element (j, b) =
//      (f[j][2b], f[j][2b+1]) with real row length Lreal), Y: [A][q m][B],
//   residue-major rows.  Eq. forwardr per column.
// ---------------------------------------------------------------------------
// Launch bounds of the column passes: the structured engine with 16 points
// per thread runs at most 256 threads and asks for 4 resident CTAs per SM (64
// registers), the other engines as before.
#ifndef HD_COL_MINB
#define HD_COL_MINB 4
#endif
template <int PTS, bool TC, bool SE>
struct ColBounds {
  static constexpr int T = (SE && !TC && PTS <= 16) ? 256 : (TC || SE) ? 512 : 1024;
  static constexpr int MINB = (SE && !TC && PTS <= 16) ? HD_COL_MINB : 1;
  static constexpr int KT = (SE && !TC) ? (PTS <= 16 ? 8 : 16) : 4;  // strip_load batch
};

// NN > 0: an instance for the residue length m = NN (the structured engine's
// passes and the strip index arithmetic with a compile-time length).
template <int PTS, bool TC, bool SE, int NN = 0>
__global__ void __launch_bounds__(ColBounds<PTS, TC, SE>::T, ColBounds<PTS, TC, SE>::MINB) k_col_fwd(const void* Xv, float2* Y, ColGeom cg,
                                                  int Lin, int m, int q, int p, int in_mode, int Lreal,
                                                  const float2* __restrict__ tw, FftPlan pl) {
  if constexpr (NN > 0) m = NN;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int W = cg.W;
  const int64_t ncolblk = (cg.B + W - 1) / W;
  const int64_t a = blockIdx.x / ncolblk;
  const int64_t b0 = (blockIdx.x - a * ncolblk) * W;
  const int N = q * m;
  const int T = blockDim.x, tid = threadIdx.x;
  const bool keep = (q > 1);  // several residues reuse the loaded columns
  float2* x = sm;                              // W x Lin (only if keep)
  float2* buf = keep ? sm + acc_slots(W * Lin) : sm;  // W x m
  // load columns (zero beyond the input)
  float2* dst = keep ? x : buf;
  const int ldst = keep ? Lin : m;
  strip_load<ColBounds<PTS, TC, SE>::KT>(dst, ldst, ldst, W, [&](int j, int w) -> float2 {
    const int64_t b = b0 + w;
    float2 v = make_float2(0.f, 0.f);
    if (j < Lin && b < cg.B) {
      const int64_t e = (a * Lin + j) * cg.B + b;
      if (in_mode == IN_COMPLEX) {
        v = __ldg(reinterpret_cast<const float2*>(Xv) + e);
      } else if (in_mode == IN_PACKED_REAL) {
        int64_t c;
        const float* fr = reinterpret_cast<const float*>(Xv) + packed_offset(cg, a, Lin, j, b, Lreal, &c);
        v = make_float2(__ldg(fr + c), (c + 1 < Lreal) ? __ldg(fr + c + 1) : 0.f);
      } else {
        int64_t second;
        const float* xr = reinterpret_cast<const float*>(Xv);
        const int64_t first = packed_offset_rev(cg, a, Lin, j, b, Lreal, &second);
        v = make_float2(__ldg(xr + first), second >= 0 ? __ldg(xr + second) : 0.f);
      }
    }
    return v;
  });
  __syncthreads();
  auto residue_pass = [&](int r) __attribute__((always_inline)) {
    if (keep) {
      for (int idx = tid; idx < W * m; idx += T) {
        const int w = idx / m, s = idx - w * m;
        float2 sum = make_float2(0.f, 0.f);
        int e = r * s;
        const int estep = r * m;
        for (int t = 0; t < p; ++t) {
          const int j = t * m + s;
          if (j >= Lin) break;
          sum = cadd(sum, cmul(x[w * Lin + j], tw_get<1>(tw, e)));
          e += estep;
          if (e >= N) e -= N;
        }
        buf[idx] = sum;
      }
      __syncthreads();
    }
    fft_sel<1, PTS, TC, SE, NN>(buf, m, W, pl, tw, q);
    strip_store(buf, m, m, W, [&](int l, int w, float2 v) {
      const int64_t b = b0 + w;
      if (b < cg.B) Y[(a * (int64_t)N + (int64_t)r * m + l) * cg.B + b] = v;
    });
    __syncthreads();
  };
  // SE: q <= 2, one inlined transform per residue (no loop around inlined FFTs)
  if constexpr (SE) {
    residue_pass(0);
    if (q > 1) residue_pass(1);
  } else {
    for (int r = 0; r < q; ++r) residue_pass(r);
  }
}

// ---------------------------------------------------------------------------
// k_col_bwd: complex hybrid backward transform along a strided dimension.
//   Y: [A][q m][B] residue-major; Z: [A][Lout][B] complex, or the unpacked
//   real array (element (j, b) -> h[j][2b], h[j][2b+1], real row length Lreal).
//   Eqs. accumulator and accumulation per column, scaled by `scale`.
// ---------------------------------------------------------------------------
template <int PTS, bool TC, bool SE, int NN = 0>
__global__ void __launch_bounds__(ColBounds<PTS, TC, SE>::T, ColBounds<PTS, TC, SE>::MINB) k_col_bwd(const float2* Y, void* Zv, ColGeom cg, int Lout, int m,
                                                  int q, int out_mode, int Lreal, float scale,
                                                  const float2* __restrict__ tw, FftPlan pl) {
  if constexpr (NN > 0) m = NN;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int W = cg.W;
  const int64_t ncolblk = (cg.B + W - 1) / W;
  const int64_t a = blockIdx.x / ncolblk;
  const int64_t b0 = (blockIdx.x - a * ncolblk) * W;
  const int N = q * m;
  const int T = blockDim.x, tid = threadIdx.x;
  const bool sep = (q > 1) || (Lout > m);
  float2* acc = sm;                                  // W x Lout (if sep)
  float2* buf = sep ? sm + acc_slots(W * Lout) : sm;  // W x m
  if (sep)
    for (int idx = tid; idx < W * Lout; idx += T) acc[idx] = make_float2(0.f, 0.f);
  auto residue_pass = [&](int r) __attribute__((always_inline)) {
    strip_load<ColBounds<PTS, TC, SE>::KT>(buf, m, m, W, [&](int l, int w) -> float2 {
      const int64_t b = b0 + w;
      return (b < cg.B) ? __ldg(Y + (a * (int64_t)N + (int64_t)r * m + l) * cg.B + b) : make_float2(0.f, 0.f);
    });
    __syncthreads();
    fft_sel<-1, PTS, TC, SE, NN>(buf, m, W, pl, tw, q);
    if (sep) {
      for (int idx = tid; idx < W * Lout; idx += T) {
        const int w = idx / Lout, j = idx - w * Lout;
        acc[idx] = cadd(acc[idx], cmul(buf[w * m + (j % m)], tw_get<-1>(tw, modmul(r, j, N))));
      }
      __syncthreads();
    }
  };
  if constexpr (SE) {
    residue_pass(0);
    if (q > 1) residue_pass(1);
  } else {
    for (int r = 0; r < q; ++r) residue_pass(r);
  }
  const float2* res = sep ? acc : buf;
  const int lres = sep ? Lout : m;
  strip_store(res, lres, Lout, W, [&](int j, int w, float2 u) {
    const int64_t b = b0 + w;
    if (b >= cg.B) return;
    const float2 v = cscale(u, scale);
    if (out_mode == OUT_COMPLEX) {
      reinterpret_cast<float2*>(Zv)[(a * Lout + j) * cg.B + b] = v;
    } else if (out_mode == OUT_UNPACK_REAL) {
      int64_t c;
      float* hr = reinterpret_cast<float*>(Zv) + packed_offset(cg, a, Lout, j, b, Lreal, &c);
      hr[c] = v.x;
      if (c + 1 < Lreal) hr[c + 1] = v.y;
    } else {
      int64_t second;
      float* zr = reinterpret_cast<float*>(Zv);
      const int64_t first = packed_offset_rev(cg, a, Lout, j, b, Lreal, &second);
      zr[first] = v.x;
      if (second >= 0) zr[second] = v.y;
    }
  });
}

// ---------------------------------------------------------------------------
// k_col_fwd_cs: real residues of Sec. 3.1 along the first dimension of a
// real array X [Lin][B] (B contiguous real).  Output rows (complex, per column):
//   residue 0:   l = 0..m/2  (m/2 + 1 rows; the columns are transformed two at
//                a time as the real and imaginary parts of one complex DFT)
//   residues 1..ceil(q/2)-1: m rows each (Eq. forwardr)
//   residue q/2 (q even):    m/2 rows (Eq. forwardq2)
// ---------------------------------------------------------------------------
// The combined CS+RCM form (Sec. 6.3) runs hybridCS's residues strictly
// between 0 and q/2 only (rows (r - 1) m + l); residues 0 and q/2 come from
// an implicitly packed convolution whose real result `add` ([addlen][B], the
// linear convolution along the first dimension of the arrays folded modulo
// `period` = 2m) is folded modulo `period` and added, times add_scale, in the
// last pass.
struct CsMid {
  int only;
  const float* add;
  int period, addlen;
  float add_scale;
};

__host__ __device__ __forceinline__ int cs_rows(int m, int q) {
  return (m / 2 + 1) + ((q + 1) / 2 - 1) * m + ((q % 2 == 0) ? m / 2 : 0);
}

template <int PTS, bool SE, int NN = 0>
__global__ void __launch_bounds__(ColBounds<PTS, false, SE>::T, ColBounds<PTS, false, SE>::MINB) k_col_fwd_cs(const float* __restrict__ X, float2* __restrict__ Y, int64_t B,
                                                     int W, int Lin, int m, int q, int p,
                                                     const float2* __restrict__ tw, FftPlan pl_m, FftPlan pl_h,
                                                     CsMid mid) {
  if constexpr (NN > 0) m = NN;  // instance for the residue length NN (and NN / 2)
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int64_t b0 = (int64_t)blockIdx.x * W;
  const int N = q * m;
  const int R = cs_rows(m, q);
  const int T = blockDim.x, tid = threadIdx.x;
  float* x = reinterpret_cast<float*>(sm);          // W x Lin real
  float2* buf = sm + acc_slots((W * Lin + 1) / 2);  // W x m complex
  batched<ColBounds<PTS, false, SE>::KT, float>(
      W * Lin,
      [&](int idx) {
        const int j = idx / W, w = idx - j * W;
        const int64_t b = b0 + w;
        return (b < B) ? __ldg(X + (int64_t)j * B + b) : 0.f;
      },
      [&](int idx, float v) {
        const int j = idx / W, w = idx - j * W;
        x[w * Lin + j] = v;
      });
  __syncthreads();
  auto store = [&](int row, int w, float2 v) {
    const int64_t b = b0 + w;
    if (b < B) Y[(int64_t)row * B + b] = v;
  };
  // residue 0: pairs of real columns as one complex column
  if (!mid.only) {
    const int npair = W / 2;
    for (int idx = tid; idx < npair * m; idx += T) {
      const int pw = idx / m, s = idx - pw * m;
      float x0 = 0.f, x1 = 0.f;
      for (int t = 0; t < p; ++t) {
        const int j = t * m + s;
        if (j >= Lin) break;
        x0 += x[(2 * pw) * Lin + j];
        x1 += x[(2 * pw + 1) * Lin + j];
      }
      buf[idx] = make_float2(x0, x1);
    }
    __syncthreads();
    fft_sel<1, PTS, false, SE, NN>(buf, m, npair, pl_m, tw, q);
    const int nh = m / 2 + 1;
    for (int idx = tid; idx < npair * nh; idx += T) {
      const int l = idx / npair, pw = idx - l * npair;
      const float2 z = buf[pw * m + l], zc = cconj(buf[pw * m + (l == 0 ? 0 : m - l)]);
      // X_w = (Z_l + conj Z_{m-l}) / 2, X_{w+1} = (Z_l - conj Z_{m-l}) / (2i)
      store(l, 2 * pw, cscale(cadd(z, zc), 0.5f));
      store(l, 2 * pw + 1, cscale(cmul_i<-1>(csub(z, zc)), 0.5f));
    }
    __syncthreads();
  }
  int row0 = mid.only ? 0 : m / 2 + 1;
  // SE: q = 2, so no residue lies strictly between 0 and q/2
  for (int r = 1; r < (SE ? 1 : (q + 1) / 2); ++r) {
    for (int idx = tid; idx < W * m; idx += T) {
      const int w = idx / m, s = idx - w * m;
      float2 sum = make_float2(0.f, 0.f);
      int e = r * s;
      for (int t = 0; t < p; ++t) {
        const int j = t * m + s;
        if (j >= Lin) break;
        const float2 z = tw_get<1>(tw, e);
        const float v = x[w * Lin + j];
        sum.x = fmaf(v, z.x, sum.x);
        sum.y = fmaf(v, z.y, sum.y);
        e += r * m;
        if (e >= N) e -= N;
      }
      buf[idx] = sum;
    }
    __syncthreads();
    fft_sel<1, PTS, false, SE, NN>(buf, m, W, pl_m, tw, q);
    for (int idx = tid; idx < W * m; idx += T) {
      const int l = idx / W, w = idx - l * W;
      store(row0 + l, w, buf[w * m + l]);
    }
    __syncthreads();
    row0 += m;
  }
  if (q % 2 == 0 && !mid.only) {
    const int e = m / 2, qh = q / 2;
    for (int idx = tid; idx < W * e; idx += T) {
      const int w = idx / e, bb = idx - w * e;
      float x0 = 0.f, x1 = 0.f;
      for (int t = 0; t < p; ++t) {
        const float sg = (t & 1) ? -1.f : 1.f;
        const int j = t * m + bb;
        if (j < Lin) x0 += sg * x[w * Lin + j];
        if (j + e < Lin) x1 += sg * x[w * Lin + j + e];
      }
      buf[idx] = cmul(make_float2(x0, x1), tw_get<1>(tw, bb * qh));
    }
    __syncthreads();
    fft_sel<1, PTS, false, SE, NN / 2>(buf, e, W, pl_h, tw, 2 * q);
    for (int idx = tid; idx < W * e; idx += T) {
      const int c = idx / W, w = idx - c * W;
      store(row0 + c, w, buf[w * e + c]);
    }
  }
  (void)R;
}

// k_col_bwd_cs: inverse of k_col_fwd_cs with Eq. real-accumulation; writes the
// first Lout rows of the real array Z [Lout][B], scaled.
template <int PTS, bool SE, int NN = 0>
__global__ void __launch_bounds__(ColBounds<PTS, false, SE>::T, ColBounds<PTS, false, SE>::MINB) k_col_bwd_cs(const float2* __restrict__ Y, float* __restrict__ Z, int64_t B,
                                                     int W, int Lout, int m, int q, float scale,
                                                     const float2* __restrict__ tw, FftPlan pl_m, FftPlan pl_h,
                                                     CsMid mid) {
  if constexpr (NN > 0) m = NN;  // instance for the residue length NN (and NN / 2)
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int64_t b0 = (int64_t)blockIdx.x * W;
  const int N = q * m;
  const int T = blockDim.x, tid = threadIdx.x;
  float* acc = reinterpret_cast<float*>(sm);          // W x Lout real
  float2* buf = sm + acc_slots((W * Lout + 1) / 2);  // W x m complex
  auto load = [&](int row, int w) -> float2 {
    const int64_t b = b0 + w;
    return (b < B) ? Y[(int64_t)row * B + b] : make_float2(0.f, 0.f);
  };
  for (int idx = tid; idx < W * Lout; idx += T) acc[idx] = 0.f;
  // residue 0: complex-to-real, two columns per complex DFT: Z_l = H_w[l] + i H_{w+1}[l]
  if (!mid.only) {
    const int npair = W / 2;
    const int nh = m / 2 + 1;
    batched<ColBounds<PTS, false, SE>::KT / 2, float2>(
        npair * m,
        [&](int idx) {
          const int l = idx / npair, pw = idx - l * npair;
          float2 a0, a1;
          if (l < nh) {
            a0 = load(l, 2 * pw);
            a1 = load(l, 2 * pw + 1);
          } else {
            a0 = cconj(load(m - l, 2 * pw));
            a1 = cconj(load(m - l, 2 * pw + 1));
          }
          return cadd(a0, cmul_i<1>(a1));
        },
        [&](int idx, float2 v) {
          const int l = idx / npair, pw = idx - l * npair;
          buf[pw * m + l] = v;
        });
    __syncthreads();
    fft_sel<-1, PTS, false, SE, NN>(buf, m, npair, pl_m, tw, q);
    for (int idx = tid; idx < W * Lout; idx += T) {
      const int w = idx / Lout, j = idx - w * Lout;
      const float2 v = buf[(w / 2) * m + (j % m)];
      acc[idx] += (w & 1) ? v.y : v.x;
    }
    __syncthreads();
  }
  int row0 = mid.only ? 0 : m / 2 + 1;
  for (int r = 1; r < (SE ? 1 : (q + 1) / 2); ++r) {
    batched<ColBounds<PTS, false, SE>::KT / 2, float2>(
        W * m, [&](int idx) { return load(row0 + idx / W, idx % W); },
        [&](int idx, float2 v) { buf[(idx % W) * m + idx / W] = v; });
    __syncthreads();
    fft_sel<-1, PTS, false, SE, NN>(buf, m, W, pl_m, tw, q);
    for (int idx = tid; idx < W * Lout; idx += T) {
      const int w = idx / Lout, j = idx - w * Lout;
      acc[idx] += 2.f * cmul(buf[w * m + (j % m)], tw_get<-1>(tw, modmul(r, j, N))).x;
    }
    __syncthreads();
    row0 += m;
  }
  if (q % 2 == 0 && !mid.only) {
    const int e = m / 2, qh = q / 2;
    batched<ColBounds<PTS, false, SE>::KT / 2, float2>(
        W * e, [&](int idx) { return load(row0 + idx / W, idx % W); },
        [&](int idx, float2 v) { buf[(idx % W) * e + idx / W] = v; });
    __syncthreads();
    fft_sel<-1, PTS, false, SE, NN / 2>(buf, e, W, pl_h, tw, 2 * q);
    for (int idx = tid; idx < W * Lout; idx += T) {
      const int w = idx / Lout, j = idx - w * Lout;
      const int t = j / m, s = j - t * m;
      const int bb = s < e ? s : s - e;
      const float2 v = cmul(buf[w * e + bb], tw_get<-1>(tw, bb * qh));
      const float val = 2.f * (s < e ? v.x : v.y);
      acc[idx] += (t & 1) ? -val : val;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < W * Lout; idx += T) {
    const int j = idx / W, w = idx - j * W;
    const int64_t b = b0 + w;
    if (b >= B) continue;
    float v = acc[w * Lout + j] * scale;
    if (mid.add) {  // residues 0 and q/2: the period-2m convolution (the linear one folded)
      const int s = j % mid.period;
      float a = mid.add[(int64_t)s * B + b];
      if (s + mid.period < mid.addlen) a += mid.add[(int64_t)(s + mid.period) * B + b];
      v += mid.add_scale * a;
    }
    Z[(int64_t)j * B + b] = v;
  }
}

// ---------------------------------------------------------------------------
// k_rows_rcm: one row of the outer spectra and its conjugate partner, a 1D
// hybrid convolution along the last dimension with the operator C_1 (Sec. 5):
//   H1_k = A_k B_k - 1/4 (A_k - conj C_k*)(B_k - conj D_k*)(1 + zeta_M^k),
//   H2_k* = C_k* D_k* - conj(...)   (A, B: rows of F, G; C, D: partner rows).
// Rows are complex of length Lrow (packed), in place over F's rows.  A row
// that is its own partner reduces to the 1D RCM of Eqs. Hr / Hr-conj.
// ---------------------------------------------------------------------------
struct RowGeom {
  int nrows;        // rows in the grid (every item of a batch)
  int Lrow;         // row length (complex)
  int m, q, p;      // hybrid parameters along the row
  int nd;           // number of outer dimensions (1 or 2)
  int om[2], oq[2]; // outer (m, q) per outer dimension
  int rpi;          // rows per item: rows pair only inside their own item
  int Kout;         // output row length (complex; >= Lrow for outputs beyond L)
};

__device__ __forceinline__ int row_partner(int row, const RowGeom& g) {
  const int item = row / g.rpi, r = row - item * g.rpi;
  if (g.nd == 1) return item * g.rpi + partner_row(r, g.om[0], g.oq[0]);
  const int M2 = g.om[1] * g.oq[1];
  const int r1 = r / M2, r2 = r - r1 * M2;
  return item * g.rpi + partner_row(r1, g.om[0], g.oq[0]) * M2 + partner_row(r2, g.om[1], g.oq[1]);
}

template <int PTS, bool TC, bool SE>
__global__ void __launch_bounds__((TC || SE) ? 512 : 1024) k_rows_rcm(float2* F, const float2* __restrict__ G, float2* O,
                                                   RowGeom rg, float scale, const float2* __restrict__ tw, FftPlan pl) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int row = blockIdx.x;
  const int prow = row_partner(row, rg);
  if (prow < row) return;
  const bool selfrow = (prow == row);
  const int T = blockDim.x, tid = threadIdx.x;
  const int Lr = rg.Lrow, Kr = rg.Kout, m = rg.m, q = rg.q, p = rg.p, N = q * m;
  const int nrow = selfrow ? 1 : 2;
  float2* acc = sm;                          // nrow x Kr (outputs)
  float2* buf = sm + acc_slots(nrow * Kr);   // arrays of m
  const float2* src[4] = {F + (int64_t)row * Lr, F + (int64_t)prow * Lr, G + (int64_t)row * Lr,
                          G + (int64_t)prow * Lr};
  for (int idx = tid; idx < nrow * Kr; idx += T) acc[idx] = make_float2(0.f, 0.f);
  __syncthreads();
  auto residue_pass = [&](int ra) __attribute__((always_inline)) {
    const int rb = (q - ra) % q;
    const bool selfres = (ra == rb);
    const int nres = selfres ? 1 : 2;
    // arrays: index = (which * nres + slot) with which in {A, C, B, D} (C, D only if !selfrow)
    const int nwhich = selfrow ? 2 : 4;
    const int narr = nwhich * nres;
    for (int idx = tid; idx < narr * m; idx += T) {
      const int arr = idx / m, s = idx - arr * m;
      const int which = arr / nres, slot = arr - which * nres;
      const int r = slot ? rb : ra;
      // which: selfrow {0: A(F row), 1: B(G row)}; else {0: A, 1: C, 2: B, 3: D}
      const float2* x = selfrow ? src[which == 0 ? 0 : 2] : src[which == 0 ? 0 : (which == 1 ? 1 : (which == 2 ? 2 : 3))];
      float2 sum = make_float2(0.f, 0.f);
      int e = r * s;
      for (int t = 0; t < p; ++t) {
        const int j = t * m + s;
        if (j >= Lr) break;
        sum = cadd(sum, cmul(x[j], tw_get<1>(tw, e)));
        e += r * m;
        if (e >= N) e -= N;
      }
      buf[idx] = sum;
    }
    __syncthreads();
    fft_sel<1, PTS, TC, SE>(buf, m, narr, pl, tw, q);
    // multiply
    auto arrp = [&](int which, int slot) { return buf + (size_t)(which * nres + slot) * m; };
    if (selfrow) {
      float2* F0 = arrp(0, 0);
      float2* Fb = arrp(0, selfres ? 0 : 1);
      float2* G0 = arrp(1, 0);
      float2* Gb = arrp(1, selfres ? 0 : 1);
      for (int l = tid; l < m; l += T) {
        int ls;
        if (selfres) {
          ls = (ra == 0) ? (l == 0 ? 0 : m - l) : (m - 1 - l);
          if (l > ls) continue;
        } else {
          ls = m - 1 - l;
        }
        const float2 A = F0[l], B = G0[l], Ac = Fb[ls], Bc = Gb[ls];
        const float2 z = tw_get<1>(tw, q * l + ra);
        const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
        const float2 alpha = cmul(cmul(csub(A, cconj(Ac)), csub(B, cconj(Bc))), Z);
        F0[l] = csub(cmul(A, B), alpha);
        if (!(selfres && ls == l)) Fb[ls] = csub(cmul(Ac, Bc), cconj(alpha));
      }
    } else {
      // every k of residue ra (and of rb when distinct) gives H1_k and H2_{k*}
      for (int idx = tid; idx < nres * m; idx += T) {
        const int slot = idx / m, l = idx - slot * m;
        const int r = slot ? rb : ra;
        const int pslot = selfres ? 0 : 1 - slot;
        const int ls = (r == 0) ? (l == 0 ? 0 : m - l) : (m - 1 - l);
        float2* Ar = arrp(0, slot);
        float2* Cr = arrp(1, pslot);
        const float2 A = Ar[l], B = arrp(2, slot)[l], Cs = Cr[ls], Ds = arrp(3, pslot)[ls];
        const float2 z = tw_get<1>(tw, q * l + r);
        const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
        const float2 alpha = cmul(cmul(csub(A, cconj(Cs)), csub(B, cconj(Ds))), Z);
        const float2 h1 = csub(cmul(A, B), alpha);
        const float2 h2 = csub(cmul(Cs, Ds), cconj(alpha));
        // in place: (slot, l) -> (pslot, ls) is a bijection, so every location
        // is read and written by exactly one iteration
        Ar[l] = h1;
        Cr[ls] = h2;
      }
    }
    __syncthreads();
    // inverse: A arrays (and C arrays) hold the products
    fft_sel<-1, PTS, TC, SE>(buf, m, selfrow ? nres : 2 * nres, pl, tw, q);
    for (int idx = tid; idx < nrow * Kr; idx += T) {
      const int rr = idx / Kr, j = idx - rr * Kr;
      const int s = j % m;
      float2 v = cmul(arrp(rr, 0)[s], tw_get<-1>(tw, modmul(ra, j, N)));
      if (!selfres) v = cadd(v, cmul(arrp(rr, 1)[s], tw_get<-1>(tw, modmul(rb, j, N))));
      acc[idx] = cadd(acc[idx], v);
    }
    __syncthreads();
  };
  // SE: q <= 2, residues 0 and 1 are each self-paired
  if constexpr (SE) {
    residue_pass(0);
    if (q > 1) residue_pass(1);
  } else {
    for (int ra = 0; ra <= q / 2; ++ra) residue_pass(ra);
  }
  for (int idx = tid; idx < nrow * Kr; idx += T) {
    const int rr = idx / Kr, j = idx - rr * Kr;
    O[(int64_t)(rr ? prow : row) * Kr + j] = cscale(acc[idx], scale);
  }
}

// ---------------------------------------------------------------------------
// k_rows_adj: the row pass of the adjoint.  For the row pair (row, prow) of
// the outer spectra of U = rev(grad_h), F and G it forms the row transforms of
// U once and applies the operator C_1 (Sec. 5) to (U, G) and to (U, F):
//   G rows <- C_1(U, G)  (outer spectra of rev(grad_f)),
//   F rows <- C_1(U, F)  (outer spectra of rev(grad_g)),
// in place; `outs` selects which of the two are written (bit 0: G, bit 1: F).
// Shared arrays per residue step: [U, F, G] x [row, partner] x [residues].
// ---------------------------------------------------------------------------
template <int PTS, bool SE>
__global__ void __launch_bounds__(SE ? 512 : 1024) k_rows_adj(float2* F, float2* G, const float2* __restrict__ U,
                                                              RowGeom rg, float scale, int outs,
                                                              const float2* __restrict__ tw, FftPlan pl) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int row = blockIdx.x;
  const int prow = row_partner(row, rg);
  if (prow < row) return;
  const bool selfrow = (prow == row);
  const int T = blockDim.x, tid = threadIdx.x;
  const int Lr = rg.Lrow, m = rg.m, q = rg.q, p = rg.p, N = q * m;
  const int nrow = selfrow ? 1 : 2;
  float2* acc = sm;                              // [output (0: G, 1: F)][nrow][Lr]
  float2* buf = sm + acc_slots(2 * nrow * Lr);   // arrays of m
  const float2* srcs[3] = {U, F, G};
  for (int idx = tid; idx < 2 * nrow * Lr; idx += T) acc[idx] = make_float2(0.f, 0.f);
  __syncthreads();
  auto residue_pass = [&](int ra) __attribute__((always_inline)) {
    const int rb = (q - ra) % q;
    const bool selfres = (ra == rb);
    const int nres = selfres ? 1 : 2;
    const int narr = 3 * nrow * nres;
    auto arr = [&](int which, int k, int slot) { return buf + (size_t)((which * nrow + k) * nres + slot) * m; };
    // Eq. forwardr, first half, for every (source, row, residue)
    for (int idx = tid; idx < narr * m; idx += T) {
      const int a = idx / m, s = idx - a * m;
      const int slot = a % nres, k = (a / nres) % nrow, which = a / (nres * nrow);
      const float2* x = srcs[which] + (int64_t)(k ? prow : row) * Lr;
      const int r = slot ? rb : ra;
      float2 sum = make_float2(0.f, 0.f);
      int e = r * s;
      for (int t = 0; t < p; ++t) {
        const int j = t * m + s;
        if (j >= Lr) break;
        sum = cadd(sum, cmul(x[j], tw_get<1>(tw, e)));
        e += r * m;
        if (e >= N) e -= N;
      }
      buf[idx] = sum;
    }
    __syncthreads();
    fft_sel<1, PTS, false, SE>(buf, m, narr, pl, tw, q);
    // C_1 on (U, G) and (U, F); U's transforms are only read
    if (selfrow) {
      const int sb = selfres ? 0 : 1;
      for (int l = tid; l < m; l += T) {
        int ls;
        if (selfres) {
          ls = (ra == 0) ? (l == 0 ? 0 : m - l) : (m - 1 - l);
          if (l > ls) continue;
        } else {
          ls = m - 1 - l;
        }
        const float2 Uk = arr(0, 0, 0)[l], Uc = arr(0, 0, sb)[ls];
        const float2 z = tw_get<1>(tw, q * l + ra);
        const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
        const float2 du = csub(Uk, cconj(Uc));
#pragma unroll
        for (int which = 1; which <= 2; ++which) {
          float2* Bl = arr(which, 0, 0);
          float2* Bs = arr(which, 0, sb);
          const float2 B = Bl[l], Bc = Bs[ls];
          const float2 alpha = cmul(cmul(du, csub(B, cconj(Bc))), Z);
          Bl[l] = csub(cmul(Uk, B), alpha);
          if (!(selfres && ls == l)) Bs[ls] = csub(cmul(Uc, Bc), cconj(alpha));
        }
      }
    } else {
      for (int idx = tid; idx < nres * m; idx += T) {
        const int slot = idx / m, l = idx - slot * m;
        const int r = slot ? rb : ra;
        const int pslot = selfres ? 0 : 1 - slot;
        const int ls = (r == 0) ? (l == 0 ? 0 : m - l) : (m - 1 - l);
        const float2 A = arr(0, 0, slot)[l], Cs = arr(0, 1, pslot)[ls];
        const float2 z = tw_get<1>(tw, q * l + r);
        const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
        const float2 du = csub(A, cconj(Cs));
#pragma unroll
        for (int which = 1; which <= 2; ++which) {
          float2* Br = arr(which, 0, slot);
          float2* Dr = arr(which, 1, pslot);
          const float2 B = Br[l], D = Dr[ls];
          const float2 alpha = cmul(cmul(du, csub(B, cconj(D))), Z);
          Br[l] = csub(cmul(A, B), alpha);
          Dr[ls] = csub(cmul(Cs, D), cconj(alpha));
        }
      }
    }
    __syncthreads();
    // inverse of the F and G arrays (contiguous after the U arrays)
    fft_sel<-1, PTS, false, SE>(arr(1, 0, 0), m, 2 * nrow * nres, pl, tw, q);
    for (int idx = tid; idx < 2 * nrow * Lr; idx += T) {
      const int o = idx / (nrow * Lr), rem = idx - o * nrow * Lr;
      const int rr = rem / Lr, j = rem - rr * Lr;
      const int which = o == 0 ? 2 : 1;
      const int s = j % m;
      float2 v = cmul(arr(which, rr, 0)[s], tw_get<-1>(tw, modmul(ra, j, N)));
      if (!selfres) v = cadd(v, cmul(arr(which, rr, 1)[s], tw_get<-1>(tw, modmul(rb, j, N))));
      acc[idx] = cadd(acc[idx], v);
    }
    __syncthreads();
  };
  if constexpr (SE) {
    residue_pass(0);
    if (q > 1) residue_pass(1);
  } else {
    for (int ra = 0; ra <= q / 2; ++ra) residue_pass(ra);
  }
  for (int idx = tid; idx < 2 * nrow * Lr; idx += T) {
    const int o = idx / (nrow * Lr), rem = idx - o * nrow * Lr;
    if (!((outs >> o) & 1)) continue;
    const int rr = rem / Lr, j = rem - rr * Lr;
    float2* dst = (o == 0 ? G : F) + (int64_t)(rr ? prow : row) * Lr;
    dst[j] = cscale(acc[idx], scale);
  }
}

// ---------------------------------------------------------------------------
// k_rows_cconv: complex hybrid convolution (Sec. 2) of each row of F with the
// same row of G along the last dimension, pointwise product, in place over F.
// ---------------------------------------------------------------------------
// NN > 0: an instance for the residue length m = NN (compile-time passes).
template <int PTS, bool SE, int NN = 0>
__global__ void __launch_bounds__(ColBounds<PTS, false, SE>::T, ColBounds<PTS, false, SE>::MINB) k_rows_cconv(float2* F, const float2* __restrict__ G, int Lr, int m, int q,
                                                     int p, float scale, const float2* __restrict__ tw, FftPlan pl) {
  if constexpr (NN > 0) m = NN;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int64_t row = blockIdx.x;
  const int T = blockDim.x, tid = threadIdx.x;
  const int N = q * m;
  float2* acc = sm;
  float2* buf = sm + acc_slots(Lr);
  const float2* src[2] = {F + row * Lr, G + row * Lr};
  for (int j = tid; j < Lr; j += T) acc[j] = make_float2(0.f, 0.f);
  __syncthreads();
  auto residue_pass = [&](int r) __attribute__((always_inline)) {
    batched<ColBounds<PTS, false, SE>::KT / 2, float2>(
        2 * m,
        [&](int idx) {
          const int arr = idx / m, s = idx - arr * m;
          const float2* x = src[arr];
          float2 sum = make_float2(0.f, 0.f);
          int e = r * s;
          for (int t = 0; t < p; ++t) {
            const int j = t * m + s;
            if (j >= Lr) break;
            sum = cadd(sum, cmul(x[j], tw_get<1>(tw, e)));
            e += r * m;
            if (e >= N) e -= N;
          }
          return sum;
        },
        [&](int idx, float2 v) { buf[idx] = v; });
    __syncthreads();
    fft_sel<1, PTS, false, SE, NN>(buf, m, 2, pl, tw, q);
    for (int l = tid; l < m; l += T) buf[l] = cmul(buf[l], buf[m + l]);
    __syncthreads();
    fft_sel<-1, PTS, false, SE, NN>(buf, m, 1, pl, tw, q);
    for (int j = tid; j < Lr; j += T) acc[j] = cadd(acc[j], cmul(buf[j % m], tw_get<-1>(tw, modmul(r, j, N))));
    __syncthreads();
  };
  if constexpr (SE) {
    residue_pass(0);
    if (q > 1) residue_pass(1);
  } else {
    for (int r = 0; r < q; ++r) residue_pass(r);
  }
  for (int j = tid; j < Lr; j += T) F[row * Lr + j] = cscale(acc[j], scale);
}

// Row DFTs along the last dimension of length n (complex).  Modes:
//   0 R2C  : src real row of 2n (padded), pack, DFT(+), unpack U -> n+1 bins
//   1 C2R  : src n+1 bins, U^{-1}, DFT(-), unpack to 2n reals, keep Lkeep,
//            scaled; rows with outer index beyond the crop are skipped
//   2 C2C  : src complex row of n, DFT(+), in place
//   3 C2RU : src complex row of n, DFT(-), unpack to reals, keep Lkeep, scaled
struct RowsIO {
  const void* src;
  void* dst;
  int64_t src_stride, dst_stride;  // elements (float for real, float2 for complex)
  int Lkeep;                       // real outputs kept per row (modes 1, 3)
  int64_t crop_rows_outer[2];      // outer extents of padded rows (M0, M1) ...
  int64_t keep_rows_outer[2];      // ... and of the kept rows (L0, L1)
  float scale;
};

template <int PTS, bool SE>
__global__ void __launch_bounds__(ColBounds<PTS, false, SE>::T, ColBounds<PTS, false, SE>::MINB) k_rows_fft(RowsIO io, int mode, int n, const float2* __restrict__ tw,
                                                   int twmul, FftPlan pl) {
  extern __shared__ float4 smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const int64_t row = blockIdx.x;
  const int T = blockDim.x, tid = threadIdx.x;
  // output row (modes 1, 3 crop the outer dimensions)
  int64_t orow = row;
  if (mode == 1 || mode == 3) {
    const int64_t M1 = io.crop_rows_outer[1];
    const int64_t a = row / M1, b = row - a * M1;
    if (a >= io.keep_rows_outer[0] || b >= io.keep_rows_outer[1]) return;
    orow = a * io.keep_rows_outer[1] + b;
  }
  // load
  auto put = [&](int j, float2 v) { buf[j] = v; };
  if (mode == 0) {
    const float* s = reinterpret_cast<const float*>(io.src) + row * io.src_stride;
    batched<ColBounds<PTS, false, SE>::KT, float2>(n, [&](int j) { return make_float2(s[2 * j], s[2 * j + 1]); }, put);
  } else if (mode == 1) {
    const float2* s = reinterpret_cast<const float2*>(io.src) + row * io.src_stride;
    // Eq. fourierPack: Z_k = 1/2 (H_k + conj H_{n-k}) + i/2 (H_k - conj H_{n-k}) zeta_{2n}^{-k}
    batched<ColBounds<PTS, false, SE>::KT / 2, float2>(
        n,
        [&](int k) {
          const float2 hk = s[k], hc = cconj(s[n - k]);
          const float2 w = tw_get<-1>(tw, k * twmul / 2);
          return cscale(cadd(cadd(hk, hc), cmul_i<1>(cmul(csub(hk, hc), w))), 0.5f);
        },
        put);
  } else {
    const float2* s = reinterpret_cast<const float2*>(io.src) + row * io.src_stride;
    batched<ColBounds<PTS, false, SE>::KT, float2>(n, [&](int j) { return s[j]; }, put);
  }
  __syncthreads();
  if (mode == 0 || mode == 2)
    fft_sel<1, PTS, false, SE>(buf, n, 1, pl, tw, twmul);
  else
    fft_sel<-1, PTS, false, SE>(buf, n, 1, pl, tw, twmul);
  if (mode == 0) {
    // Eq. fourierUnpack: F_k = 1/2 (Z_k + conj Z_{n-k}) - i/2 (Z_k - conj Z_{n-k}) zeta_{2n}^k, k = 0..n
    float2* d = reinterpret_cast<float2*>(io.dst) + row * io.dst_stride;
    for (int k = tid; k <= n; k += T) {
      const float2 zk = buf[k % n], zc = cconj(buf[(n - k) % n]);
      const float2 w = tw_get<1>(tw, (k % (2 * n)) * twmul / 2);
      d[k] = cscale(csub(cadd(zk, zc), cmul_i<1>(cmul(csub(zk, zc), w))), 0.5f);
    }
  } else if (mode == 2) {
    float2* d = reinterpret_cast<float2*>(io.dst) + row * io.dst_stride;
    for (int j = tid; j < n; j += T) d[j] = buf[j];
  } else {
    float* d = reinterpret_cast<float*>(io.dst) + orow * (int64_t)io.Lkeep;
    for (int j = tid; j < io.Lkeep; j += T) {
      const float2 v = buf[j >> 1];
      d[j] = ((j & 1) ? v.y : v.x) * io.scale;
    }
  }
}

// ---------------------------------------------------------------------------
// DFT engines and launches
// ---------------------------------------------------------------------------
// The structured engine (struct_length DFTs, kPtsSE points per thread, <= 512
// threads), the generic plan-driven engine (kPts points per thread, <= 1024
// threads), or the split-precision tensor-core passes (kPts, <= 512 threads).
constexpr int kPtsSE = 32;
// TCS: the structured sequence with tensor-core radix-16 passes (split bf16)
enum class Eng { GEN, SE, TC, TCS };
inline Eng pick_eng(bool tc, bool se_ok) {
  return tc ? (se_ok ? Eng::TCS : Eng::TC) : (se_ok ? Eng::SE : Eng::GEN);
}
// Points one CTA may transform at once.
inline int64_t max_points(Eng e) {
  return e == Eng::SE ? (int64_t)kPtsSE * 512 : (int64_t)kPts * ((e == Eng::TC || e == Eng::TCS) ? 512 : 1024);
}
inline int eng_threads(Eng e, int64_t points) {
  if (e == Eng::SE) return std::min(512, threads_for_points(points, 16));
  return threads_for_points(points, kPts);
}

template <class T>
struct nodeduce {
  using type = T;
};
// Launch kernel k with dynamic shared memory smem (raising its limit first).
template <typename... A>
cudaError_t launch_kernel(void (*k)(A...), unsigned grid, int T, size_t smem, cudaStream_t st,
                          typename nodeduce<A>::type... args) {
  {
    const cudaError_t e = smem_optin((const void*)k, smem);
    if (e != cudaSuccess) return e;
  }
  void* argv[] = {(void*)&args...};
  const cudaError_t e = cudaLaunchKernel((const void*)k, dim3(grid), dim3(T), argv, smem, st);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_col_fwd(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const void* X, float2* Y,
                           ColGeom cg, int Lin, int m, int q, int p, int in_mode, int Lreal, const float2* tw,
                           FftPlan pl);
cudaError_t launch_col_bwd(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const float2* Y, void* Z,
                           ColGeom cg, int Lout, int m, int q, int out_mode, int Lreal, float scale, const float2* tw,
                           FftPlan pl);
cudaError_t launch_col_fwd_cs(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const float* X, float2* Y,
                              int64_t B, int W, int Lin, int m, int q, int p, const float2* tw, FftPlan pl_m,
                              FftPlan pl_h, CsMid mid = CsMid{0, nullptr, 1, 0, 0.f});
cudaError_t launch_col_bwd_cs(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const float2* Y, float* Z,
                              int64_t B, int W, int Lout, int m, int q, float scale, const float2* tw, FftPlan pl_m,
                              FftPlan pl_h, CsMid mid = CsMid{0, nullptr, 1, 0, 0.f});
// O: output rows (rg.Kout per row); O = F (in place) when Kout = Lrow.
cudaError_t launch_rows_rcm(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, float2* F, const float2* G,
                            float2* O, RowGeom rg, float scale, const float2* tw, FftPlan pl);
// Row pass of hybridRCM on the compile-time engine (hd_nd_rowscl.cu): rows of
// residue length m = 256 R3 (rows_cl_length), q = 2.
bool rows_cl_length(int m);
cudaError_t launch_rows_cl(int m, unsigned grid, cudaStream_t st, float2* F, const float2* G, float2* O, RowGeom rg,
                           float scale, const float2* tw, const float2* tab);
// The one-residue row pass (q = 1, M >= the real row length).
cudaError_t launch_rows_cl1(int m, unsigned grid, cudaStream_t st, float2* F, const float2* G, float2* O, RowGeom rg,
                            float scale, const float2* tab);
cudaError_t launch_rows_adj_cl(int m, unsigned grid, cudaStream_t st, float2* F, float2* G, const float2* U,
                               RowGeom rg, float scale, int outs, const float2* tw, const float2* tab);
cudaError_t launch_rows_adj(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, float2* F, float2* G,
                            const float2* U, RowGeom rg, float scale, int outs, const float2* tw, FftPlan pl);
cudaError_t launch_rows_cconv(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, float2* F, const float2* G,
                              int Lr, int m, int q, int p, float scale, const float2* tw, FftPlan pl);
cudaError_t launch_rows_fft(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, RowsIO io, int mode, int n,
                            const float2* tw, int twmul, FftPlan pl);

}  // namespace hd
