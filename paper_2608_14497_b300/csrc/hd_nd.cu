// hd_nd.cu -- 2D/3D convolutions by the recursive decomposition of Sec. 5, and
// the explicit-padding baselines (Sec. 6) in 1D/2D/3D.
//
// hybridRCM (Sec. 5, Eqs. multidimComplexPacking and RCM-ndim, operator C_n):
//   pack along the last dimension; complex hybrid forward along every outer
//   (strided) dimension (k_col_fwd, Eq. forwardr per column); for every row of
//   the outer spectra and its conjugate partner (k1*, k2*) a fused 1D hybrid
//   convolution along the last dimension with the C_1 operator (k_rows_rcm);
//   complex hybrid backward along the outer dimensions, the last one unpacking
//   the real result (k_col_bwd).
// hybridCS (Sec. 5 with Sec. 3): the first dimension is transformed with the
//   real residues of Sec. 3.1 (k_col_fwd_cs / k_col_bwd_cs); the middle
//   dimension (3D) with complex hybrid dealiasing; every row along the last
//   dimension is a complex hybrid convolution with a pointwise product
//   (k_rows_cconv).
// explicit / explicitRCM: zero padding materialised to 2L per dimension in
//   scratch, full-length DFTs pass by pass (rows along the last dimension,
//   columns along the others), pointwise product or the RCM operator of
//   Eq. RCM-ndim, inverse, crop.
//
// Layout of transformed outer dimensions: residue-major rows, index r m + l
// for the natural frequency k = q l + r.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "hd_conv1d.cuh"
#include "hd_internal.h"
#include "hd_nd.cuh"

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

// Input element loaders for the column passes.
enum : int { IN_COMPLEX = 0, IN_PACKED_REAL = 1 };
enum : int { OUT_COMPLEX = 0, OUT_UNPACK_REAL = 1 };

// ---------------------------------------------------------------------------
// k_col_fwd: complex hybrid forward transform along a strided dimension.
//   X: [A][Lin][B] complex (or real packed along B: element (j, b) =
//      (f[j][2b], f[j][2b+1]) with real row length Lreal), Y: [A][q m][B],
//   residue-major rows.  Eq. forwardr per column.
// ---------------------------------------------------------------------------
template <int PTS, bool TC = false>
__global__ void __launch_bounds__(TC ? 512 : 1024) k_col_fwd(const void* Xv, float2* Y, ColGeom cg,
                                                  int Lin, int m, int q, int p, int in_mode, int Lreal,
                                                  const float2* __restrict__ tw, FftPlan pl) {
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
  for (int idx = tid; idx < W * ldst; idx += T) {
    const int j = idx / W, w = idx - j * W;
    const int64_t b = b0 + w;
    float2 v = make_float2(0.f, 0.f);
    if (j < Lin && b < cg.B) {
      const int64_t e = (a * Lin + j) * cg.B + b;
      if (in_mode == IN_COMPLEX) {
        v = reinterpret_cast<const float2*>(Xv)[e];
      } else {
        int64_t c;
        const float* fr = reinterpret_cast<const float*>(Xv) + packed_offset(cg, a, Lin, j, b, Lreal, &c);
        v = make_float2(fr[c], (c + 1 < Lreal) ? fr[c + 1] : 0.f);
      }
    }
    dst[w * ldst + j] = v;
  }
  __syncthreads();
  for (int r = 0; r < q; ++r) {
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
    cta_fft<1, PTS, TC>(buf, m, W, pl, tw, q);
    for (int idx = tid; idx < W * m; idx += T) {
      const int l = idx / W, w = idx - l * W;
      const int64_t b = b0 + w;
      if (b < cg.B) Y[(a * (int64_t)N + (int64_t)r * m + l) * cg.B + b] = buf[w * m + l];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_col_bwd: complex hybrid backward transform along a strided dimension.
//   Y: [A][q m][B] residue-major; Z: [A][Lout][B] complex, or the unpacked
//   real array (element (j, b) -> h[j][2b], h[j][2b+1], real row length Lreal).
//   Eqs. accumulator and accumulation per column, scaled by `scale`.
// ---------------------------------------------------------------------------
template <int PTS, bool TC = false>
__global__ void __launch_bounds__(TC ? 512 : 1024) k_col_bwd(const float2* Y, void* Zv, ColGeom cg, int Lout, int m,
                                                  int q, int out_mode, int Lreal, float scale,
                                                  const float2* __restrict__ tw, FftPlan pl) {
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
  for (int r = 0; r < q; ++r) {
    for (int idx = tid; idx < W * m; idx += T) {
      const int l = idx / W, w = idx - l * W;
      const int64_t b = b0 + w;
      buf[w * m + l] = (b < cg.B) ? Y[(a * (int64_t)N + (int64_t)r * m + l) * cg.B + b] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    cta_fft<-1, PTS, TC>(buf, m, W, pl, tw, q);
    if (sep) {
      for (int idx = tid; idx < W * Lout; idx += T) {
        const int w = idx / Lout, j = idx - w * Lout;
        acc[idx] = cadd(acc[idx], cmul(buf[w * m + (j % m)], tw_get<-1>(tw, modmul(r, j, N))));
      }
      __syncthreads();
    }
  }
  const float2* res = sep ? acc : buf;
  const int lres = sep ? Lout : m;
  for (int idx = tid; idx < W * Lout; idx += T) {
    const int j = idx / W, w = idx - j * W;
    const int64_t b = b0 + w;
    if (b >= cg.B) continue;
    const float2 v = cscale(res[w * lres + j], scale);
    if (out_mode == OUT_COMPLEX) {
      reinterpret_cast<float2*>(Zv)[(a * Lout + j) * cg.B + b] = v;
    } else {
      int64_t c;
      float* hr = reinterpret_cast<float*>(Zv) + packed_offset(cg, a, Lout, j, b, Lreal, &c);
      hr[c] = v.x;
      if (c + 1 < Lreal) hr[c + 1] = v.y;
    }
  }
}

// ---------------------------------------------------------------------------
// k_col_fwd_cs: real residues of Sec. 3.1 along the first dimension of a
// real array X [Lin][B] (B contiguous real).  Output rows (complex, per column):
//   residue 0:   l = 0..m/2  (m/2 + 1 rows; the columns are transformed two at
//                a time as the real and imaginary parts of one complex DFT)
//   residues 1..ceil(q/2)-1: m rows each (Eq. forwardr)
//   residue q/2 (q even):    m/2 rows (Eq. forwardq2)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int cs_rows(int m, int q) {
  return (m / 2 + 1) + ((q + 1) / 2 - 1) * m + ((q % 2 == 0) ? m / 2 : 0);
}

template <int PTS>
__global__ void __launch_bounds__(1024) k_col_fwd_cs(const float* __restrict__ X, float2* __restrict__ Y, int64_t B,
                                                     int W, int Lin, int m, int q, int p,
                                                     const float2* __restrict__ tw, FftPlan pl_m, FftPlan pl_h) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int64_t b0 = (int64_t)blockIdx.x * W;
  const int N = q * m;
  const int R = cs_rows(m, q);
  const int T = blockDim.x, tid = threadIdx.x;
  float* x = reinterpret_cast<float*>(sm);          // W x Lin real
  float2* buf = sm + acc_slots((W * Lin + 1) / 2);  // W x m complex
  for (int idx = tid; idx < W * Lin; idx += T) {
    const int j = idx / W, w = idx - j * W;
    const int64_t b = b0 + w;
    x[w * Lin + j] = (b < B) ? X[(int64_t)j * B + b] : 0.f;
  }
  __syncthreads();
  auto store = [&](int row, int w, float2 v) {
    const int64_t b = b0 + w;
    if (b < B) Y[(int64_t)row * B + b] = v;
  };
  // residue 0: pairs of real columns as one complex column
  {
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
    cta_fft<1, PTS>(buf, m, npair, pl_m, tw, q);
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
  int row0 = m / 2 + 1;
  for (int r = 1; r < (q + 1) / 2; ++r) {
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
    cta_fft<1, PTS>(buf, m, W, pl_m, tw, q);
    for (int idx = tid; idx < W * m; idx += T) {
      const int l = idx / W, w = idx - l * W;
      store(row0 + l, w, buf[w * m + l]);
    }
    __syncthreads();
    row0 += m;
  }
  if (q % 2 == 0) {
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
    cta_fft<1, PTS>(buf, e, W, pl_h, tw, 2 * q);
    for (int idx = tid; idx < W * e; idx += T) {
      const int c = idx / W, w = idx - c * W;
      store(row0 + c, w, buf[w * e + c]);
    }
  }
  (void)R;
}

// k_col_bwd_cs: inverse of k_col_fwd_cs with Eq. real-accumulation; writes the
// first Lout rows of the real array Z [Lout][B], scaled.
template <int PTS>
__global__ void __launch_bounds__(1024) k_col_bwd_cs(const float2* __restrict__ Y, float* __restrict__ Z, int64_t B,
                                                     int W, int Lout, int m, int q, float scale,
                                                     const float2* __restrict__ tw, FftPlan pl_m, FftPlan pl_h) {
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
  {
    const int npair = W / 2;
    const int nh = m / 2 + 1;
    for (int idx = tid; idx < npair * m; idx += T) {
      const int l = idx / npair, pw = idx - l * npair;
      float2 a0, a1;
      if (l < nh) {
        a0 = load(l, 2 * pw);
        a1 = load(l, 2 * pw + 1);
      } else {
        a0 = cconj(load(m - l, 2 * pw));
        a1 = cconj(load(m - l, 2 * pw + 1));
      }
      buf[pw * m + l] = cadd(a0, cmul_i<1>(a1));
    }
    __syncthreads();
    cta_fft<-1, PTS>(buf, m, npair, pl_m, tw, q);
    for (int idx = tid; idx < W * Lout; idx += T) {
      const int w = idx / Lout, j = idx - w * Lout;
      const float2 v = buf[(w / 2) * m + (j % m)];
      acc[idx] += (w & 1) ? v.y : v.x;
    }
    __syncthreads();
  }
  int row0 = m / 2 + 1;
  for (int r = 1; r < (q + 1) / 2; ++r) {
    for (int idx = tid; idx < W * m; idx += T) {
      const int l = idx / W, w = idx - l * W;
      buf[w * m + l] = load(row0 + l, w);
    }
    __syncthreads();
    cta_fft<-1, PTS>(buf, m, W, pl_m, tw, q);
    for (int idx = tid; idx < W * Lout; idx += T) {
      const int w = idx / Lout, j = idx - w * Lout;
      acc[idx] += 2.f * cmul(buf[w * m + (j % m)], tw_get<-1>(tw, modmul(r, j, N))).x;
    }
    __syncthreads();
    row0 += m;
  }
  if (q % 2 == 0) {
    const int e = m / 2, qh = q / 2;
    for (int idx = tid; idx < W * e; idx += T) {
      const int c = idx / W, w = idx - c * W;
      buf[w * e + c] = load(row0 + c, w);
    }
    __syncthreads();
    cta_fft<-1, PTS>(buf, e, W, pl_h, tw, 2 * q);
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
    if (b < B) Z[(int64_t)j * B + b] = acc[w * Lout + j] * scale;
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
  int nrows;        // rows in the grid
  int Lrow;         // row length (complex)
  int m, q, p;      // hybrid parameters along the row
  int nd;           // number of outer dimensions (1 or 2)
  int om[2], oq[2]; // outer (m, q) per outer dimension
};

__device__ __forceinline__ int row_partner(int row, const RowGeom& g) {
  if (g.nd == 1) return partner_row(row, g.om[0], g.oq[0]);
  const int M2 = g.om[1] * g.oq[1];
  const int r1 = row / M2, r2 = row - r1 * M2;
  return partner_row(r1, g.om[0], g.oq[0]) * M2 + partner_row(r2, g.om[1], g.oq[1]);
}

template <int PTS, bool TC = false>
__global__ void __launch_bounds__(TC ? 512 : 1024) k_rows_rcm(float2* F, const float2* __restrict__ G, RowGeom rg, float scale,
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
  float2* acc = sm;                          // nrow x Lr
  float2* buf = sm + acc_slots(nrow * Lr);   // arrays of m
  const float2* src[4] = {F + (int64_t)row * Lr, F + (int64_t)prow * Lr, G + (int64_t)row * Lr,
                          G + (int64_t)prow * Lr};
  for (int idx = tid; idx < nrow * Lr; idx += T) acc[idx] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int ra = 0; ra <= q / 2; ++ra) {
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
    cta_fft<1, PTS, TC>(buf, m, narr, pl, tw, q);
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
    if (selfrow) {
      cta_fft<-1, PTS, TC>(buf, m, nres, pl, tw, q);
    } else {
      cta_fft<-1, PTS, TC>(buf, m, 2 * nres, pl, tw, q);
    }
    for (int idx = tid; idx < nrow * Lr; idx += T) {
      const int rr = idx / Lr, j = idx - rr * Lr;
      const int s = j % m;
      float2 v = cmul(arrp(rr, 0)[s], tw_get<-1>(tw, modmul(ra, j, N)));
      if (!selfres) v = cadd(v, cmul(arrp(rr, 1)[s], tw_get<-1>(tw, modmul(rb, j, N))));
      acc[idx] = cadd(acc[idx], v);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nrow * Lr; idx += T) {
    const int rr = idx / Lr, j = idx - rr * Lr;
    F[(int64_t)(rr ? prow : row) * Lr + j] = cscale(acc[idx], scale);
  }
}

// ---------------------------------------------------------------------------
// k_rows_cconv: complex hybrid convolution (Sec. 2) of each row of F with the
// same row of G along the last dimension, pointwise product, in place over F.
// ---------------------------------------------------------------------------
template <int PTS>
__global__ void __launch_bounds__(1024) k_rows_cconv(float2* F, const float2* __restrict__ G, int Lr, int m, int q,
                                                     int p, float scale, const float2* __restrict__ tw, FftPlan pl) {
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
  for (int r = 0; r < q; ++r) {
    for (int idx = tid; idx < 2 * m; idx += T) {
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
      buf[idx] = sum;
    }
    __syncthreads();
    cta_fft<1, PTS>(buf, m, 2, pl, tw, q);
    for (int l = tid; l < m; l += T) buf[l] = cmul(buf[l], buf[m + l]);
    __syncthreads();
    cta_fft<-1, PTS>(buf, m, 1, pl, tw, q);
    for (int j = tid; j < Lr; j += T) acc[j] = cadd(acc[j], cmul(buf[j % m], tw_get<-1>(tw, modmul(r, j, N))));
    __syncthreads();
  }
  for (int j = tid; j < Lr; j += T) F[row * Lr + j] = cscale(acc[j], scale);
}

// ---------------------------------------------------------------------------
// explicit baselines
// ---------------------------------------------------------------------------
// Materialised zero padding: P[(2L)^d] real (mode 0), or packed complex with
// the last dimension of packed length Mp (mode 1).
__global__ void k_pad(const float* __restrict__ f, void* P, int d, int64_t L0, int64_t L1, int64_t L2, int64_t M0,
                      int64_t M1, int64_t M2, int mode) {
  // M*: padded extents of the output (complex extent for the last dim in mode 1)
  const int64_t tot = M0 * M1 * M2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / (M1 * M2), b = (i / M2) % M1, c = i % M2;
    if (mode == 0) {
      float v = 0.f;
      if (a < L0 && b < L1 && c < L2) v = f[(a * L1 + b) * L2 + c];
      reinterpret_cast<float*>(P)[i] = v;
    } else {
      float2 v = make_float2(0.f, 0.f);
      if (a < L0 && b < L1) {
        const int64_t c0 = 2 * c;
        if (c0 < L2) v.x = f[(a * L1 + b) * L2 + c0];
        if (c0 + 1 < L2) v.y = f[(a * L1 + b) * L2 + c0 + 1];
      }
      reinterpret_cast<float2*>(P)[i] = v;
    }
  }
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

template <int PTS>
__global__ void __launch_bounds__(1024) k_rows_fft(RowsIO io, int mode, int n, const float2* __restrict__ tw,
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
  if (mode == 0) {
    const float* s = reinterpret_cast<const float*>(io.src) + row * io.src_stride;
    for (int j = tid; j < n; j += T) buf[j] = make_float2(s[2 * j], s[2 * j + 1]);
  } else if (mode == 1) {
    const float2* s = reinterpret_cast<const float2*>(io.src) + row * io.src_stride;
    // Eq. fourierPack: Z_k = 1/2 (H_k + conj H_{n-k}) + i/2 (H_k - conj H_{n-k}) zeta_{2n}^{-k}
    for (int k = tid; k < n; k += T) {
      const float2 hk = s[k], hc = cconj(s[n - k]);
      const float2 w = tw_get<-1>(tw, k * twmul / 2);
      buf[k] = cscale(cadd(cadd(hk, hc), cmul_i<1>(cmul(csub(hk, hc), w))), 0.5f);
    }
  } else {
    const float2* s = reinterpret_cast<const float2*>(io.src) + row * io.src_stride;
    for (int j = tid; j < n; j += T) buf[j] = s[j];
  }
  __syncthreads();
  if (mode == 0 || mode == 2)
    cta_fft<1, PTS>(buf, n, 1, pl, tw, twmul);
  else
    cta_fft<-1, PTS>(buf, n, 1, pl, tw, twmul);
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

// Pointwise product S_f <- S_f . S_g.
__global__ void k_pointwise(float2* __restrict__ A, const float2* __restrict__ B, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    A[i] = cmul(A[i], B[i]);
}

// Eq. RCM-ndim on full spectra of extents (M0, M1, M2) (the last packed):
// each thread owns the pair {k, k*} with k <= k* (linear index), in place.
__global__ void k_rcm_nd(float2* __restrict__ A, const float2* __restrict__ B, int64_t M0, int64_t M1, int64_t M2,
                         const float2* __restrict__ tw, int twmul) {
  const int64_t tot = M0 * M1 * M2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / (M1 * M2), b = (i / M2) % M1, c = i % M2;
    const int64_t as = (M0 - a) % M0, bs = (M1 - b) % M1, cs = (M2 - c) % M2;
    const int64_t j = (as * M1 + bs) * M2 + cs;
    if (j < i) continue;
    const float2 Fa = A[i], Ga = B[i], Fc = A[j], Gc = B[j];
    const float2 z = tw_get<1>(tw, (int)(c * twmul));
    const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
    const float2 alpha = cmul(cmul(csub(Fa, cconj(Fc)), csub(Ga, cconj(Gc))), Z);
    A[i] = csub(cmul(Fa, Ga), alpha);
    if (j != i) A[j] = csub(cmul(Fc, Gc), cconj(alpha));
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t allow(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static int elementwise_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::min<int64_t>(b, 148 * 32);
}

// Choose W columns per CTA for a column pass: shared memory per column
// `per_col` bytes and points per column `pts`; W <= 8, W even if `even`.
static int choose_W(size_t per_col, int pts, int64_t B, size_t max_smem, bool even,
                    int64_t max_points = (int64_t)kPts * 1024) {
  int W = 8;
  while (W > 1 && ((size_t)W * per_col > max_smem || (int64_t)W * pts > max_points)) W >>= 1;
  if (even && W < 2) W = 2;
  if ((int64_t)W > B && !even) W = (int)std::max<int64_t>(1, B);
  return W;
}

struct ColPass {
  int m, q, p;
  const float2* tw;
  FftPlan pl;
};

// Points one CTA may transform at once: kPts per thread up to 1024 threads, or
// up to 512 threads for the tensor-core instantiation (128 registers).
static int64_t max_points(bool tc) { return (int64_t)kPts * (tc ? 512 : 1024); }

static hd_status col_fwd(hd_ctx* c, const void* X, int in_mode, int Lreal, float2* Y, int64_t A, int Lin, int64_t B,
                         const ColPass& cp, cudaStream_t st, int64_t Bp = 0, bool tc = false) {
  const bool keep = cp.q > 1;
  const size_t per_col = sizeof(float2) * ((keep ? (size_t)Lin : 0) + (size_t)cp.m) + 16;
  const int W = choose_W(per_col, cp.m, B, (size_t)c->max_smem, false, max_points(tc));
  ColGeom cg{A, B, W, Bp > 0 ? Bp : B};
  const size_t smem = sizeof(float2) * ((keep ? (size_t)acc_slots(W * Lin) : 0) + (size_t)W * cp.m);
  if (smem > (size_t)c->max_smem || (int64_t)W * cp.m > max_points(tc)) return HD_EUNSUPPORTED;
  const int T = threads_for_points((int64_t)W * cp.m, kPts);
  const int64_t grid = A * ((B + W - 1) / W);
  if (tc) {
    if (allow(k_col_fwd<kPts, true>, smem) != cudaSuccess) return HD_ECUDA;
    k_col_fwd<kPts, true><<<(unsigned)grid, T, smem, st>>>(X, Y, cg, Lin, cp.m, cp.q, cp.p, in_mode, Lreal, cp.tw,
                                                           cp.pl);
  } else {
    if (allow(k_col_fwd<kPts>, smem) != cudaSuccess) return HD_ECUDA;
    k_col_fwd<kPts><<<(unsigned)grid, T, smem, st>>>(X, Y, cg, Lin, cp.m, cp.q, cp.p, in_mode, Lreal, cp.tw, cp.pl);
  }
  return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ECUDA;
}

static hd_status col_bwd(hd_ctx* c, const float2* Y, void* Z, int out_mode, int Lreal, int64_t A, int Lout, int64_t B,
                         const ColPass& cp, float scale, cudaStream_t st, int64_t Bp = 0, bool tc = false) {
  const bool sep = cp.q > 1 || Lout > cp.m;
  const size_t per_col = sizeof(float2) * ((sep ? (size_t)Lout : 0) + (size_t)cp.m) + 16;
  const int W = choose_W(per_col, cp.m, B, (size_t)c->max_smem, false, max_points(tc));
  ColGeom cg{A, B, W, Bp > 0 ? Bp : B};
  const size_t smem = sizeof(float2) * ((sep ? (size_t)acc_slots(W * Lout) : 0) + (size_t)W * cp.m);
  if (smem > (size_t)c->max_smem || (int64_t)W * cp.m > max_points(tc)) return HD_EUNSUPPORTED;
  const int T = threads_for_points((int64_t)W * cp.m, kPts);
  const int64_t grid = A * ((B + W - 1) / W);
  if (tc) {
    if (allow(k_col_bwd<kPts, true>, smem) != cudaSuccess) return HD_ECUDA;
    k_col_bwd<kPts, true><<<(unsigned)grid, T, smem, st>>>(Y, Z, cg, Lout, cp.m, cp.q, out_mode, Lreal, scale, cp.tw,
                                                           cp.pl);
  } else {
    if (allow(k_col_bwd<kPts>, smem) != cudaSuccess) return HD_ECUDA;
    k_col_bwd<kPts><<<(unsigned)grid, T, smem, st>>>(Y, Z, cg, Lout, cp.m, cp.q, out_mode, Lreal, scale, cp.tw, cp.pl);
  }
  return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ECUDA;
}

// Hybrid parameters of an outer (complex) dimension of real length L.
static hd_status outer_params(hd_ctx* c, int64_t L, const hd_dim_params* prm, ColPass* cp, cudaStream_t st) {
  int64_t m, q;
  if (prm && prm->m > 0) {
    m = prm->m;
    q = prm->q > 0 ? prm->q : (2 * L - 1 + m - 1) / m;
    if (q * m < 2 * L - 1) return HD_EINVAL;
  } else {
    m = next_smooth(L);
    q = 2;
  }
  if (m > (int64_t)kPts * 1024) return HD_EUNSUPPORTED;
  cp->m = (int)m;
  cp->q = (int)q;
  cp->p = (int)((L + m - 1) / m);
  factor_radices((int)m, &cp->pl);
  hd_status terr = HD_OK;
  cp->tw = c->tables.get(q * m, st, &terr);
  return cp->tw ? HD_OK : terr;
}

// Parameters of the last (row) dimension for the RCM rows (packed, needs
// q m >= L) or CS rows (complex, needs q m >= 2L-1).
static hd_status row_params(hd_ctx* c, int64_t L, bool packed, const hd_dim_params* prm, ColPass* cp,
                            cudaStream_t st) {
  const int64_t Lr = packed ? (L + 1) / 2 : L;
  const int64_t need = packed ? L : 2 * L - 1;
  int64_t m, q;
  if (prm && prm->m > 0) {
    m = prm->m;
    q = prm->q > 0 ? prm->q : (need + m - 1) / m;
    if (q * m < need) return HD_EINVAL;
  } else {
    m = next_smooth(Lr);
    q = (need + m - 1) / m;
  }
  cp->m = (int)m;
  cp->q = (int)q;
  cp->p = (int)((Lr + m - 1) / m);
  factor_radices((int)m, &cp->pl);
  hd_status terr = HD_OK;
  cp->tw = c->tables.get(q * m, st, &terr);
  return cp->tw ? HD_OK : terr;
}

static hd_status hybrid_rcm_nd(hd_ctx* c, int d, const int64_t* L, const hd_dim_params* prm, const float* f,
                               const float* g, float* h, cudaStream_t st, bool tc = false) {
  // d = 2: [L0][L1]; d = 3: [L0][L1][L2]; the last dimension is packed
  const int64_t Ln = L[d - 1];
  const int64_t Lp = (Ln + 1) / 2;
  ColPass outer[2], row;
  for (int i = 0; i < d - 1; ++i) {
    hd_status s = outer_params(c, L[i], prm ? &prm[i] : nullptr, &outer[i], st);
    if (s != HD_OK) return s;
  }
  hd_status s = row_params(c, Ln, true, prm ? &prm[d - 1] : nullptr, &row, st);
  if (s != HD_OK) return s;
  const int64_t M0 = (int64_t)outer[0].q * outer[0].m;
  const int64_t M1 = d == 3 ? (int64_t)outer[1].q * outer[1].m : 1;
  // scratch: F, G spectra [M0][M1][Lp] plus (3D) the intermediate [M0][L1][Lp]
  const int64_t spec = M0 * M1 * Lp;
  const int64_t mid = d == 3 ? M0 * L[1] * Lp : 0;
  const size_t bytes = sizeof(float2) * (size_t)(2 * spec + 2 * mid);
  if (ensure_ws(c, bytes) != HD_OK) return HD_ENOMEM;
  float2* SF = reinterpret_cast<float2*>(c->ws);
  float2* SG = SF + spec;
  float2* TF = SG + spec;
  float2* TG = TF + mid;
  // forward along the outer dimensions
  if (d == 2) {
    s = col_fwd(c, f, IN_PACKED_REAL, (int)Ln, SF, 1, (int)L[0], Lp, outer[0], st, 0, tc);
    if (s == HD_OK) s = col_fwd(c, g, IN_PACKED_REAL, (int)Ln, SG, 1, (int)L[0], Lp, outer[0], st, 0, tc);
  } else {
    s = col_fwd(c, f, IN_PACKED_REAL, (int)Ln, TF, 1, (int)L[0], L[1] * Lp, outer[0], st, Lp, tc);
    if (s == HD_OK) s = col_fwd(c, g, IN_PACKED_REAL, (int)Ln, TG, 1, (int)L[0], L[1] * Lp, outer[0], st, Lp, tc);
    if (s == HD_OK) s = col_fwd(c, TF, IN_COMPLEX, 0, SF, M0, (int)L[1], Lp, outer[1], st, 0, tc);
    if (s == HD_OK) s = col_fwd(c, TG, IN_COMPLEX, 0, SG, M0, (int)L[1], Lp, outer[1], st, 0, tc);
  }
  if (s != HD_OK) return s;
  // rows: C_1 on each row pair
  RowGeom rg;
  std::memset(&rg, 0, sizeof(rg));
  rg.nrows = (int)(M0 * M1);
  rg.Lrow = (int)Lp;
  rg.m = row.m;
  rg.q = row.q;
  rg.p = row.p;
  rg.nd = d - 1;
  rg.om[0] = outer[0].m;
  rg.oq[0] = outer[0].q;
  if (d == 3) {
    rg.om[1] = outer[1].m;
    rg.oq[1] = outer[1].q;
  }
  const size_t smem = sizeof(float2) * ((size_t)acc_slots(2 * (int)Lp) + 8 * (size_t)row.m);
  if (smem > (size_t)c->max_smem || 8 * (int64_t)row.m > max_points(tc)) return HD_EUNSUPPORTED;
  const int T = threads_for_points(8 * (int64_t)row.m, kPts);
  if (tc) {
    if (allow(k_rows_rcm<kPts, true>, smem) != cudaSuccess) return HD_ECUDA;
    k_rows_rcm<kPts, true><<<rg.nrows, T, smem, st>>>(SF, SG, rg, 1.0f / (float)(row.q * row.m), row.tw, row.pl);
  } else {
    if (allow(k_rows_rcm<kPts>, smem) != cudaSuccess) return HD_ECUDA;
    k_rows_rcm<kPts><<<rg.nrows, T, smem, st>>>(SF, SG, rg, 1.0f / (float)(row.q * row.m), row.tw, row.pl);
  }
  if (cudaGetLastError() != cudaSuccess) return HD_ECUDA;
  // backward along the outer dimensions, unpacking at the end
  if (d == 2) {
    s = col_bwd(c, SF, h, OUT_UNPACK_REAL, (int)Ln, 1, (int)L[0], Lp, outer[0], 1.0f / (float)M0, st, 0, tc);
  } else {
    s = col_bwd(c, SF, TF, OUT_COMPLEX, 0, M0, (int)L[1], Lp, outer[1], 1.0f / (float)M1, st, 0, tc);
    if (s == HD_OK)
      s = col_bwd(c, TF, h, OUT_UNPACK_REAL, (int)Ln, 1, (int)L[0], L[1] * Lp, outer[0], 1.0f / (float)M0, st, Lp,
                  tc);
  }
  return s;
}

static hd_status hybrid_cs_nd(hd_ctx* c, int d, const int64_t* L, const hd_dim_params* prm, const float* f,
                              const float* g, float* h, cudaStream_t st) {
  // first dimension: real residues (CS); middle (3D): complex hybrid; rows: complex conv
  const int64_t B0 = d == 2 ? L[1] : L[1] * L[2];  // real columns of the first pass
  int64_t m0, q0;
  if (prm && prm[0].m > 0) {
    m0 = prm[0].m;
    q0 = prm[0].q > 0 ? prm[0].q : (2 * L[0] - 1 + m0 - 1) / m0;
    if (q0 * m0 < 2 * L[0] - 1 || (q0 % 2 == 0 && m0 % 2 == 1)) return HD_EINVAL;
  } else {
    m0 = next_smooth(L[0]);
    while (m0 % 2) m0 = next_smooth(m0 + 1);
    q0 = 2;
  }
  if (m0 % 2) return HD_EUNSUPPORTED;  // residue 0 pairs columns through an even-length real DFT
  const int p0 = (int)((L[0] + m0 - 1) / m0);
  FftPlan pm0, ph0;
  factor_radices((int)m0, &pm0);
  factor_radices((int)(m0 / 2), &ph0);
  hd_status terr = HD_OK;
  const float2* tw0 = c->tables.get(q0 * m0, st, &terr);
  if (!tw0) return terr;
  const int R0 = cs_rows((int)m0, (int)q0);
  ColPass mid, row;
  hd_status s = HD_OK;
  if (d == 3) {
    s = outer_params(c, L[1], prm ? &prm[1] : nullptr, &mid, st);
    if (s != HD_OK) return s;
  }
  s = row_params(c, L[d - 1], false, prm ? &prm[d - 1] : nullptr, &row, st);
  if (s != HD_OK) return s;
  const int64_t M1 = d == 3 ? (int64_t)mid.q * mid.m : 1;
  const int64_t Lr = L[d - 1];
  const int64_t rowsz = (d == 3 ? M1 : 1) * Lr;  // complex elements per first-dim row of the spectra
  const int64_t spec = (int64_t)R0 * rowsz;
  const int64_t tmp = d == 3 ? (int64_t)R0 * L[1] * Lr : 0;
  if (ensure_ws(c, sizeof(float2) * (size_t)(2 * spec + 2 * tmp)) != HD_OK) return HD_ENOMEM;
  float2* SF = reinterpret_cast<float2*>(c->ws);
  float2* SG = SF + spec;
  float2* TF = SG + spec;
  float2* TG = TF + tmp;
  // first dimension: real columns (W even)
  {
    const size_t per_col = sizeof(float) * (size_t)L[0] + sizeof(float2) * (size_t)m0 + 16;
    const int W = choose_W(per_col, (int)m0, B0, (size_t)c->max_smem, true);
    const size_t smem = sizeof(float2) * ((size_t)acc_slots((W * (int)L[0] + 1) / 2) + (size_t)W * m0);
    if (smem > (size_t)c->max_smem || (int64_t)W * m0 > (int64_t)kPts * 1024) return HD_EUNSUPPORTED;
    const int T = threads_for_points((int64_t)W * m0, kPts);
    const int64_t grid = (B0 + W - 1) / W;
    if (allow(k_col_fwd_cs<kPts>, smem) != cudaSuccess) return HD_ECUDA;
    float2* outF = d == 3 ? TF : SF;
    float2* outG = d == 3 ? TG : SG;
    k_col_fwd_cs<kPts><<<(unsigned)grid, T, smem, st>>>(f, outF, B0, W, (int)L[0], (int)m0, (int)q0, p0, tw0, pm0, ph0);
    k_col_fwd_cs<kPts><<<(unsigned)grid, T, smem, st>>>(g, outG, B0, W, (int)L[0], (int)m0, (int)q0, p0, tw0, pm0, ph0);
    if (cudaGetLastError() != cudaSuccess) return HD_ECUDA;
  }
  if (d == 3) {
    s = col_fwd(c, TF, IN_COMPLEX, 0, SF, R0, (int)L[1], Lr, mid, st);
    if (s == HD_OK) s = col_fwd(c, TG, IN_COMPLEX, 0, SG, R0, (int)L[1], Lr, mid, st);
    if (s != HD_OK) return s;
  }
  {
    const int64_t nrows = (int64_t)R0 * (d == 3 ? M1 : 1);
    const size_t smem = sizeof(float2) * ((size_t)acc_slots((int)Lr) + 2 * (size_t)row.m);
    if (smem > (size_t)c->max_smem || 2 * (int64_t)row.m > (int64_t)kPts * 1024) return HD_EUNSUPPORTED;
    const int T = threads_for_points(2 * (int64_t)row.m, kPts);
    if (allow(k_rows_cconv<kPts>, smem) != cudaSuccess) return HD_ECUDA;
    k_rows_cconv<kPts><<<(unsigned)nrows, T, smem, st>>>(SF, SG, (int)Lr, row.m, row.q, row.p,
                                                         1.0f / (float)(row.q * row.m), row.tw, row.pl);
    if (cudaGetLastError() != cudaSuccess) return HD_ECUDA;
  }
  if (d == 3) {
    s = col_bwd(c, SF, TF, OUT_COMPLEX, 0, R0, (int)L[1], Lr, mid, 1.0f / (float)M1, st);
    if (s != HD_OK) return s;
  }
  {
    const float2* src = d == 3 ? TF : SF;
    const size_t per_col = sizeof(float) * (size_t)L[0] + sizeof(float2) * (size_t)m0 + 16;
    const int W = choose_W(per_col, (int)m0, B0, (size_t)c->max_smem, true);
    const size_t smem = sizeof(float2) * ((size_t)acc_slots((W * (int)L[0] + 1) / 2) + (size_t)W * m0);
    if (smem > (size_t)c->max_smem) return HD_EUNSUPPORTED;
    const int T = threads_for_points((int64_t)W * m0, kPts);
    const int64_t grid = (B0 + W - 1) / W;
    if (allow(k_col_bwd_cs<kPts>, smem) != cudaSuccess) return HD_ECUDA;
    k_col_bwd_cs<kPts><<<(unsigned)grid, T, smem, st>>>(src, h, B0, W, (int)L[0], (int)m0, (int)q0,
                                                        1.0f / (float)(q0 * m0), tw0, pm0, ph0);
    if (cudaGetLastError() != cudaSuccess) return HD_ECUDA;
  }
  return HD_OK;
}

hd_status explicit_nd(hd_ctx* c, hd_algo algo, int d, const int64_t* Lin, const float* f, const float* g, float* h,
                      cudaStream_t st) {
  // padded extents: 2L per dimension (real); explicitRCM packs the last one to
  // an even packed length (Alg. 4 needs it even)
  // (each padded length is 2 x the next 2,3,5-smooth size >= L, so every DFT
  // length factors into the register radices; any length >= 2L-1 dealiases)
  int64_t L[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) L[3 - d + i] = Lin[i];
  const bool rcm = (algo == HD_EXPLICIT_RCM);
  const int64_t Mo0 = d >= 3 ? 2 * next_smooth(L[0]) : 1, Mo1 = d >= 2 ? 2 * next_smooth(L[1]) : 1;
  int64_t n = next_smooth(L[2]);  // complex length of the last-dim DFT (real padded length 2n)
  if (rcm)
    while (n % 2) n = next_smooth(n + 1);
  const int64_t rows = Mo0 * Mo1;
  if (n > (int64_t)kPts * 1024) return HD_EUNSUPPORTED;
  const int64_t bins = rcm ? n : n + 1;                 // complex per row after the last-dim pass
  const int64_t Preal = rows * 2 * n;                   // padded real elements per array
  const int64_t spec = rows * bins;
  if (ensure_ws(c, sizeof(float) * (size_t)(2 * Preal) + sizeof(float2) * (size_t)(2 * spec)) != HD_OK)
    return HD_ENOMEM;
  float* PF = reinterpret_cast<float*>(c->ws);
  float* PG = PF + Preal;
  float2* SF = reinterpret_cast<float2*>(PG + Preal);
  float2* SG = SF + spec;
  hd_status terr = HD_OK;
  // table for the last dimension: N = 2n (covers zeta_{2n} for U and zeta_n)
  const float2* twl = c->tables.get(2 * n, st, &terr);
  if (!twl) return terr;
  FftPlan pln;
  factor_radices((int)n, &pln);
  // 1) materialised zero padding
  {
    const int64_t tot = rows * (rcm ? n : 2 * n);
    k_pad<<<elementwise_blocks(tot), 256, 0, st>>>(f, PF, 3, L[0], L[1], L[2], Mo0, Mo1, rcm ? n : 2 * n, rcm ? 1 : 0);
    k_pad<<<elementwise_blocks(tot), 256, 0, st>>>(g, PG, 3, L[0], L[1], L[2], Mo0, Mo1, rcm ? n : 2 * n, rcm ? 1 : 0);
  }
  // 2) last dimension
  const int T = threads_for_points(n, kPts);
  const size_t smem = sizeof(float2) * (size_t)n;
  if (allow(k_rows_fft<kPts>, smem) != cudaSuccess) return HD_ECUDA;
  for (int a = 0; a < 2; ++a) {
    RowsIO io;
    std::memset(&io, 0, sizeof(io));
    io.src = a ? (const void*)PG : (const void*)PF;
    io.dst = a ? SG : SF;
    io.src_stride = rcm ? n : 2 * n;
    io.dst_stride = bins;
    k_rows_fft<kPts><<<(unsigned)rows, T, smem, st>>>(io, rcm ? 2 : 0, (int)n, twl, 2, pln);
  }
  if (cudaGetLastError() != cudaSuccess) return HD_ECUDA;
  // 3) outer dimensions: full-length complex DFTs (q = 1, m = 2L)
  ColPass cp[2];
  const int nouter = d - 1;
  for (int i = 0; i < nouter; ++i) {
    const int64_t Mi = (i == 0) ? (d == 3 ? Mo0 : Mo1) : Mo1;
    cp[i].m = (int)Mi;
    cp[i].q = 1;
    cp[i].p = 1;
    factor_radices((int)Mi, &cp[i].pl);
    cp[i].tw = c->tables.get(Mi, st, &terr);
    if (!cp[i].tw) return terr;
  }
  hd_status s = HD_OK;
  if (d == 2) {
    for (int a = 0; a < 2 && s == HD_OK; ++a) {
      float2* S = a ? SG : SF;
      s = col_fwd(c, S, IN_COMPLEX, 0, S, 1, (int)Mo1, bins, cp[0], st);
    }
  } else if (d == 3) {
    for (int a = 0; a < 2 && s == HD_OK; ++a) {
      float2* S = a ? SG : SF;
      s = col_fwd(c, S, IN_COMPLEX, 0, S, 1, (int)Mo0, Mo1 * bins, cp[0], st);
      if (s == HD_OK) s = col_fwd(c, S, IN_COMPLEX, 0, S, Mo0, (int)Mo1, bins, cp[1], st);
    }
  }
  if (s != HD_OK) return s;
  // 4) product
  if (rcm) {
    k_rcm_nd<<<elementwise_blocks(spec), 256, 0, st>>>(SF, SG, Mo0, Mo1, n, twl, 2);
  } else {
    k_pointwise<<<elementwise_blocks(spec), 256, 0, st>>>(SF, SG, spec);
  }
  // 5) outer inverse
  if (d == 2) {
    s = col_bwd(c, SF, SF, OUT_COMPLEX, 0, 1, (int)Mo1, bins, cp[0], 1.0f, st);
  } else if (d == 3) {
    s = col_bwd(c, SF, SF, OUT_COMPLEX, 0, Mo0, (int)Mo1, bins, cp[1], 1.0f, st);
    if (s == HD_OK) s = col_bwd(c, SF, SF, OUT_COMPLEX, 0, 1, (int)Mo0, Mo1 * bins, cp[0], 1.0f, st);
  }
  if (s != HD_OK) return s;
  // 6) last dimension inverse, unpack, crop, scale 1 / prod(M)
  {
    RowsIO io;
    std::memset(&io, 0, sizeof(io));
    io.src = SF;
    io.dst = h;
    io.src_stride = bins;
    io.Lkeep = (int)L[2];
    io.crop_rows_outer[0] = Mo0;
    io.crop_rows_outer[1] = Mo1;
    io.keep_rows_outer[0] = L[0];
    io.keep_rows_outer[1] = L[1];
    // the unnormalised inverse returns n Mo0 Mo1 times the convolution, for
    // both the real (pack after U^{-1}) and the packed (RCM) forms
    io.scale = (float)(1.0 / ((double)Mo0 * (double)Mo1 * (double)n));
    k_rows_fft<kPts><<<(unsigned)rows, T, smem, st>>>(io, rcm ? 3 : 1, (int)n, twl, 2, pln);
  }
  return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ECUDA;
}

}  // namespace hd

using namespace hd;

static hd_status conv_nd(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int d,
                         const int64_t* L, const hd_dim_params* prm, void* stream) {
  if (!c || !f || !g || !h) return HD_EINVAL;
  for (int i = 0; i < d; ++i)
    if (L[i] < 1 || L[i] > (1 << 20)) return L[i] < 1 ? HD_EINVAL : HD_EUNSUPPORTED;
  // split precision: the radix-16 passes of hybridRCM's 2D/3D kernels on tensor cores
  if (prec == HD_SPLIT_BF16 && algo != HD_HYBRID_RCM) return HD_EUNSUPPORTED;
  if (prec != HD_FP32 && prec != HD_SPLIT_BF16) return HD_EINVAL;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  switch (algo) {
    case HD_HYBRID_RCM: return hybrid_rcm_nd(c, d, L, prm, f, g, h, st, prec == HD_SPLIT_BF16);
    case HD_HYBRID_CS: return hybrid_cs_nd(c, d, L, prm, f, g, h, st);
    case HD_EXPLICIT:
    case HD_EXPLICIT_RCM: return explicit_nd(c, algo, d, L, f, g, h, st);
  }
  return HD_EINVAL;
}

extern "C" {
hd_status hd_conv2d(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int64_t L1,
                    int64_t L2, const hd_dim_params* prm, void* stream) {
  const int64_t L[2] = {L1, L2};
  return conv_nd(c, algo, prec, f, g, h, 2, L, prm, stream);
}
hd_status hd_conv3d(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int64_t L1,
                    int64_t L2, int64_t L3, const hd_dim_params* prm, void* stream) {
  const int64_t L[3] = {L1, L2, L3};
  return conv_nd(c, algo, prec, f, g, h, 3, L, prm, stream);
}
}
