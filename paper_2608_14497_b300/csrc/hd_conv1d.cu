// hd_conv1d.cu -- fused 1D real convolutions by hybrid dealiasing, one CTA per
// convolution, residues processed in sequence (Sec. 2.1, "one residue at a
// time").  Two algorithms:
//
//   k_rcm1d  hybridRCM (Sec. 4): the real input is read as its complex packing
//            (Eq. complexPacking), each residue pair {r, q-r} (r = 0 and
//            r = q/2 self-paired) is transformed (Eq. forwardr: fold over t
//            with zeta_N^{r(tm+s)}, then a length-m DFT), multiplied with the
//            RCM operator in residue form (Eqs. Hr and Hr-conj), transformed
//            back and accumulated with zeta_N^{-r j} (Eqs. accumulator and
//            accumulation); the output is the unpacked real array.
//   k_cs1d   hybridCS (Sec. 3): residue 0 by a real DFT (a packed complex DFT
//            of length m/2 with the unpack/pack formulas Eqs. fourierUnpack
//            and fourierPack, or a complex DFT when m is odd), residues
//            1..ceil(q/2)-1 by complex DFTs with 2 Re accumulation, residue
//            q/2 by the half-length packing of Eqs. forwardq2, wb and
//            accumulateq2; Eq. real-accumulation combines them.
//            RCM0 = true is the combined CS+RCM form of Sec. 6.3: residue 0
//            keeps the packed length-m/2 DFTs but multiplies the packed
//            spectra with the RCM operator (Eq. RCM of packed length m/2)
//            instead of unpacking, multiplying and packing again; residue
//            q/2 is already an implicitly packed half-length transform whose
//            even-index products need no partner (Eq. realq2symmetry), so
//            every residue is computed on its own.
//
// All arithmetic is FP32 with FP64-generated twiddle tables.  The accumulator
// lives in shared memory, or in a global scratch area when it does not fit
// (then it is private to the CTA; no atomics are needed).
#include <cuda_runtime.h>

#include <algorithm>

#include "hd_conv1d.cuh"

namespace hd {

// Exponent (a * b) mod N for a, b >= 0 with a*b < 2^63.
__device__ __forceinline__ int mulmod(int a, int b, int N) { return (int)(((int64_t)a * b) % N); }

template <int PTS>
__global__ void __launch_bounds__(1024) k_rcm1d(Launch1D la, const float* f, const float* g, float* h) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  __shared__ FftPlan s_pl;
  const Item1D it = la.items ? la.items[blockIdx.x] : la.one;
  if (threadIdx.x == 0) s_pl = la.plans ? la.plans[it.plan] : la.plan_m;
  const int T = blockDim.x, tid = threadIdx.x;
  const int L = it.L, m = it.m, q = it.q, p = it.p;
  const int N = q * m;
  const int Lp = (L + 1) >> 1;
  const int K = it.K > 0 ? it.K : L;  // real output length
  const int Kp = (K + 1) >> 1;
  const float* fi = f + it.off;
  const float* gi = g + it.off;
  float* hi = h + it.off;
  float2* acc = it.gacc ? reinterpret_cast<float2*>(it.gacc) : sm;
  float2* buf = it.gacc ? sm : sm + acc_slots(Kp);
  const float2* __restrict__ tw = it.tw;
  for (int j = tid; j < Kp; j += T) acc[j] = make_float2(0.f, 0.f);
  __syncthreads();

  for (int ra = 0; ra <= q / 2; ++ra) {
    const int rb = (q - ra) % q;
    const bool self = (ra == rb);
    const int nres = self ? 1 : 2;
    const int narr = 2 * nres;
    // Eq. forwardr, first half: y_s = sum_t zeta_N^{r(tm+s)} f~_{tm+s}.
    // Layout: self [F_ra, G_ra]; pair [F_ra, F_rb, G_ra, G_rb]; stride m.
    for (int idx = tid; idx < narr * m; idx += T) {
      const int arr = idx / m, s = idx - arr * m;
      const bool isG = self ? (arr == 1) : (arr >= 2);
      const int r = self ? ra : ((arr & 1) ? rb : ra);
      const float* x = isG ? gi : fi;
      float2 sum = make_float2(0.f, 0.f);
      int e = r * s;
      const int estep = r * m;
      for (int t = 0; t < p; ++t) {
        const int j = t * m + s;
        if (j >= Lp) break;
        const float2 v = make_float2(x[2 * j], (2 * j + 1 < L) ? x[2 * j + 1] : 0.f);
        const float2 w = tw_get<1>(tw, e);
        sum.x = fmaf(v.x, w.x, fmaf(-v.y, w.y, sum.x));
        sum.y = fmaf(v.x, w.y, fmaf(v.y, w.x, sum.y));
        e += estep;
        if (e >= N) e -= N;
      }
      buf[idx] = sum;
    }
    __syncthreads();
    // Eq. forwardr, second half: length-m DFTs (zeta_m = zeta_N^q).
    cta_fft<1, PTS>(buf, m, narr, s_pl, tw, q);
    // Eqs. Hr / Hr-conj: k = q l + ra pairs with k* = (N - k) mod N, i.e.
    // l* = (m - l) mod m for ra = 0, l* = m - 1 - l otherwise (residue rb).
    float2* F0 = buf;
    float2* Fb = self ? buf : buf + m;
    float2* G0 = self ? buf + m : buf + 2 * m;
    float2* Gb = self ? buf + m : buf + 3 * m;
    for (int l = tid; l < m; l += T) {
      int ls;
      if (self) {
        ls = (ra == 0) ? (l == 0 ? 0 : m - l) : (m - 1 - l);
        if (l > ls) continue;
      } else {
        ls = m - 1 - l;
      }
      const float2 A = F0[l], B = G0[l], Ac = Fb[ls], Bc = Gb[ls];
      const float2 z = tw_get<1>(tw, q * l + ra);
      const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);  // (1 + zeta_N^k)/4
      const float2 alpha = cmul(cmul(csub(A, cconj(Ac)), csub(B, cconj(Bc))), Z);
      F0[l] = csub(cmul(A, B), alpha);
      if (!(self && ls == l)) Fb[ls] = csub(cmul(Ac, Bc), cconj(alpha));
    }
    __syncthreads();
    // Eq. accumulator: backward length-m DFTs of the products ...
    cta_fft<-1, PTS>(buf, m, nres, s_pl, tw, q);
    // ... then h_{r, j} = zeta_N^{-r j} w_r[j mod m], summed (Eq. accumulation).
    for (int j = tid; j < Kp; j += T) {
      const int s = j % m;
      float2 v = cmul(F0[s], tw_get<-1>(tw, mulmod(ra, j, N)));
      if (!self) v = cadd(v, cmul(Fb[s], tw_get<-1>(tw, mulmod(rb, j, N))));
      acc[j] = cadd(acc[j], v);
    }
    __syncthreads();
  }
  const float sc = 1.0f / (float)N;
  for (int j = tid; j < Kp; j += T) {
    const float2 v = acc[j];
    hi[2 * j] = v.x * sc;
    if (2 * j + 1 < K) hi[2 * j + 1] = v.y * sc;
  }
}

// A length-n DFT of k_cs1d on nbuf arrays at stride n: the plan-driven engine,
// or with NN > 0 the structured engine at the compile-time length NN (the
// half-length DFTs of residues 0 and q/2 in an instance for one m; the
// length-m DFTs of the other residues stay on the plan-driven engine, which
// such an instance, launched for q = 2 only, never runs).
template <int SIGN, int PTS, int NN>
__device__ __forceinline__ void cs1d_fft(float2* buf, int n, int nbuf, const FftPlan& pl, const float2* tw,
                                         int twmul) {
  if constexpr (NN > 0) cta_fft_struct_k<SIGN, PTS, NN>(buf, NN, nbuf, tw, twmul);
  else cta_fft<SIGN, PTS>(buf, n, nbuf, pl, tw, twmul);
}

template <int PTS, bool RCM0, int NM = 0>
__global__ void __launch_bounds__(NM > 0 ? 512 : 1024) k_cs1d(Launch1D la, const float* f, const float* g, float* h) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  __shared__ FftPlan s_pm, s_ph;
  const Item1D it = la.items ? la.items[blockIdx.x] : la.one;
  if (threadIdx.x == 0) {
    s_pm = la.plans ? la.plans[it.plan] : la.plan_m;
    if (it.plan_half >= 0) s_ph = la.plans ? la.plans[it.plan_half] : la.plan_half;
  }
  const int T = blockDim.x, tid = threadIdx.x;
  const int L = it.L, m = NM > 0 ? NM : it.m, q = it.q, p = it.p;
  const int N = q * m;
  const int K = it.K > 0 ? it.K : L;  // real output length
  const float* fi = f + it.off;
  const float* gi = g + it.off;
  float* hi = h + it.off;
  float* acc = it.gacc ? reinterpret_cast<float*>(it.gacc) : reinterpret_cast<float*>(sm);
  float2* buf = it.gacc ? sm : sm + acc_slots((K + 1) >> 1);
  const float2* __restrict__ tw = it.tw;
  for (int j = tid; j < K; j += T) acc[j] = 0.f;
  __syncthreads();

  const int nlow = (q + 1) / 2;                 // residues 0 .. ceil(q/2)-1
  const int nres = nlow + ((q % 2 == 0) ? 1 : 0);  // plus q/2 when q is even
  for (int ri = 0; ri < nres; ++ri) {
    const int r = ri < nlow ? ri : q / 2;
    if (r == 0 && (m % 2 == 0)) {
      // Sec. 3.1.1: real fold x_s = sum_t f_{tm+s}; real DFT of length m by a
      // complex DFT of the packing z_j = x_{2j} + i x_{2j+1} (Eq. complexPacking).
      const int n2 = m >> 1;
      for (int idx = tid; idx < 2 * n2; idx += T) {
        const int arr = idx / n2, jj = idx - arr * n2;
        const float* x = arr ? gi : fi;
        float x0 = 0.f, x1 = 0.f;
        for (int t = 0; t < p; ++t) {
          const int j = t * m + 2 * jj;
          if (j < L) x0 += x[j];
          if (j + 1 < L) x1 += x[j + 1];
        }
        buf[idx] = make_float2(x0, x1);
      }
      __syncthreads();
      cs1d_fft<1, PTS, NM / 2>(buf, n2, 2, s_ph, tw, 2 * q);
      float2* Z = buf;
      float2* Y = buf + n2;
      if constexpr (RCM0) {
        // Eq. RCM on the packed spectra (packed length n2): for the pair
        // (k, kc = (n2 - k) mod n2), alpha = (Z_k - conj Z_kc)(Y_k - conj Y_kc)
        // (1 + zeta_n2^k) / 4, Z_k <- Z_k Y_k - alpha, Z_kc <- Z_kc Y_kc - conj alpha
        // (zeta_n2^k = zeta_m^{2k} = tw[2 k q]).
        for (int k = tid; k <= n2 / 2; k += T) {
          const int kc = (n2 - k) % n2;
          const float2 zk = Z[k], zc = Z[kc], yk = Y[k], yc = Y[kc];
          const float2 w = tw_get<1>(tw, 2 * k * q);
          const float2 fac = make_float2(0.25f * (1.f + w.x), 0.25f * w.y);
          const float2 alpha = cmul(cmul(csub(zk, cconj(zc)), csub(yk, cconj(yc))), fac);
          Z[k] = csub(cmul(zk, yk), alpha);
          if (kc != k) Z[kc] = csub(cmul(zc, yc), cconj(alpha));
        }
      } else {
      // Eq. fourierUnpack for F and G, pointwise product, Eq. fourierPack;
      // pairs (k, n2 - k) with Z_{n2} = Z_0 and zeta_m^k = tw[k q].
      for (int k = tid; k <= n2 / 2; k += T) {
        const int kc = n2 - k;
        const float2 zk = Z[k], zc = Z[kc % n2], yk = Y[k], yc = Y[kc % n2];
        const float2 wk = tw_get<1>(tw, k * q), wc = tw_get<1>(tw, kc * q);
        // X_k = 1/2 (Z_k + conj Z_kc) - i/2 (Z_k - conj Z_kc) zeta_m^k
        const float2 Xk = cscale(csub(cadd(zk, cconj(zc)), cmul_i<1>(cmul(csub(zk, cconj(zc)), wk))), 0.5f);
        const float2 Xc = cscale(csub(cadd(zc, cconj(zk)), cmul_i<1>(cmul(csub(zc, cconj(zk)), wc))), 0.5f);
        const float2 Gk = cscale(csub(cadd(yk, cconj(yc)), cmul_i<1>(cmul(csub(yk, cconj(yc)), wk))), 0.5f);
        const float2 Gc = cscale(csub(cadd(yc, cconj(yk)), cmul_i<1>(cmul(csub(yc, cconj(yk)), wc))), 0.5f);
        const float2 Hk = cmul(Xk, Gk), Hc = cmul(Xc, Gc);
        // Z'_k = 1/2 (H_k + conj H_kc) + i/2 (H_k - conj H_kc) zeta_m^{-k}
        Z[k] = cscale(cadd(cadd(Hk, cconj(Hc)), cmul_i<1>(cmul(csub(Hk, cconj(Hc)), cconj(wk)))), 0.5f);
        if (kc < n2 && kc != k)
          Z[kc] = cscale(cadd(cadd(Hc, cconj(Hk)), cmul_i<1>(cmul(csub(Hc, cconj(Hk)), cconj(wc)))), 0.5f);
      }
      }
      __syncthreads();
      cs1d_fft<-1, PTS, NM / 2>(buf, n2, 1, s_ph, tw, 2 * q);
      // h_0 = 2 unpack(z''), repeated for every block t (Sec. 3.1.1).
      for (int j = tid; j < K; j += T) {
        const int s = j % m;
        const float2 v = Z[s >> 1];
        acc[j] += 2.f * ((s & 1) ? v.y : v.x);
      }
      __syncthreads();
    } else if (r == 0) {
      // m odd (q odd): real fold as a complex DFT of length m.
      for (int idx = tid; idx < 2 * m; idx += T) {
        const int arr = idx / m, s = idx - arr * m;
        const float* x = arr ? gi : fi;
        float x0 = 0.f;
        for (int t = 0; t < p; ++t) {
          const int j = t * m + s;
          if (j < L) x0 += x[j];
        }
        buf[idx] = make_float2(x0, 0.f);
      }
      __syncthreads();
      cs1d_fft<1, PTS, 0>(buf, m, 2, s_pm, tw, q);
      for (int l = tid; l < m; l += T) buf[l] = cmul(buf[l], buf[m + l]);
      __syncthreads();
      cs1d_fft<-1, PTS, 0>(buf, m, 1, s_pm, tw, q);
      for (int j = tid; j < K; j += T) acc[j] += buf[j % m].x;
      __syncthreads();
    } else if (2 * r == q) {
      // Sec. 3.1.3: x_s = sum_t (-1)^t f_{tm+s}; W_b = zeta_2m^b (x_b + i x_{e+b})
      // (Eq. forwardq2), zeta_2m = zeta_N^{q/2}; DFT of length e = m/2.
      const int e = m >> 1;
      const int qh = q >> 1;
      for (int idx = tid; idx < 2 * e; idx += T) {
        const int arr = idx / e, b = idx - arr * e;
        const float* x = arr ? gi : fi;
        float x0 = 0.f, x1 = 0.f;
        for (int t = 0; t < p; ++t) {
          const float sg = (t & 1) ? -1.f : 1.f;
          const int j = t * m + b;
          if (j < L) x0 += sg * x[j];
          if (j + e < L) x1 += sg * x[j + e];
        }
        buf[idx] = cmul(make_float2(x0, x1), tw_get<1>(tw, b * qh));
      }
      __syncthreads();
      cs1d_fft<1, PTS, NM / 2>(buf, e, 2, s_ph, tw, 2 * q);
      for (int c = tid; c < e; c += T) buf[c] = cmul(buf[c], buf[e + c]);
      __syncthreads();
      cs1d_fft<-1, PTS, NM / 2>(buf, e, 1, s_ph, tw, 2 * q);
      // Eqs. wb / accumulateq2: w_b = zeta_2m^{-b} (...); (-1)^t 2Re w_b, (-1)^t 2Im w_b.
      for (int j = tid; j < K; j += T) {
        const int t = j / m, s = j - t * m;
        const int b = s < e ? s : s - e;
        const float2 w = cmul(buf[b], tw_get<-1>(tw, b * qh));
        float val = 2.f * (s < e ? w.x : w.y);
        acc[j] += (t & 1) ? -val : val;
      }
      __syncthreads();
    } else {
      // Sec. 3.1.2: complex residue, 2 Re of the contribution.
      for (int idx = tid; idx < 2 * m; idx += T) {
        const int arr = idx / m, s = idx - arr * m;
        const float* x = arr ? gi : fi;
        float2 sum = make_float2(0.f, 0.f);
        int ex = r * s;
        const int estep = r * m;
        for (int t = 0; t < p; ++t) {
          const int j = t * m + s;
          if (j >= L) break;
          const float2 w = tw_get<1>(tw, ex);
          sum.x = fmaf(x[j], w.x, sum.x);
          sum.y = fmaf(x[j], w.y, sum.y);
          ex += estep;
          if (ex >= N) ex -= N;
        }
        buf[idx] = sum;
      }
      __syncthreads();
      cs1d_fft<1, PTS, 0>(buf, m, 2, s_pm, tw, q);
      for (int l = tid; l < m; l += T) buf[l] = cmul(buf[l], buf[m + l]);
      __syncthreads();
      cs1d_fft<-1, PTS, 0>(buf, m, 1, s_pm, tw, q);
      for (int j = tid; j < K; j += T) {
        const float2 v = cmul(buf[j % m], tw_get<-1>(tw, mulmod(r, j, N)));
        acc[j] += 2.f * v.x;
      }
      __syncthreads();
    }
  }
  const float sc = 1.0f / (float)N;
  for (int j = tid; j < K; j += T) hi[j] = acc[j] * sc;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t rcm1d_smem_bytes(int L, int m, bool gacc) {
  return sizeof(float2) * ((gacc ? 0 : (size_t)acc_slots((L + 1) / 2)) + 4 * (size_t)m);
}

size_t cs1d_smem_bytes(int L, int m, bool gacc) {
  return sizeof(float2) * ((gacc ? 0 : (size_t)acc_slots((L + 1) / 2)) + 2 * (size_t)m);
}

int threads_for_points(int64_t points, int pts) {
  int64_t t = (points + pts - 1) / pts;
  int T = 64;
  while (T < t && T < 1024) T <<= 1;
  return T;
}

// Raise the kernel's dynamic shared-memory limit to what this launch needs.
template <typename K>
static cudaError_t allow_smem(K kernel, size_t smem) {
  return smem_optin((const void*)kernel, smem);
}

cudaError_t launch_rcm1d(const Launch1D& la, int nitems, int threads, size_t smem, const float* f, const float* g,
                         float* h, cudaStream_t st) {
  cudaError_t e = allow_smem(k_rcm1d<kPts>, smem);
  if (e != cudaSuccess) return e;
  k_rcm1d<kPts><<<nitems, threads, smem, st>>>(la, f, g, h);
  return cudaGetLastError();
}

cudaError_t launch_cs1d(const Launch1D& la, int nitems, int threads, size_t smem, const float* f, const float* g,
                        float* h, cudaStream_t st, bool rcm0) {
  auto k = rcm0 ? k_cs1d<kPts, true> : k_cs1d<kPts, false>;
  // single calls with q = 2 at the residue lengths of the usual sizes: the
  // compile-time instance (its DFTs of m / 2 on the structured engine, on two
  // arrays, so m points at kPts per thread: 256 to 512 threads, launch bound
  // 512 for the registers of the unrolled passes)
  if (!la.items && nitems == 1 && la.one.q == 2 && la.one.m <= 512 * kPts) {
    const int tq = std::max(256, la.one.m / kPts);
    switch (la.one.m) {
      case 1024: k = rcm0 ? k_cs1d<kPts, true, 1024> : k_cs1d<kPts, false, 1024>; break;
      case 2048: k = rcm0 ? k_cs1d<kPts, true, 2048> : k_cs1d<kPts, false, 2048>; break;
      case 3072: k = rcm0 ? k_cs1d<kPts, true, 3072> : k_cs1d<kPts, false, 3072>; break;
      case 4096: k = rcm0 ? k_cs1d<kPts, true, 4096> : k_cs1d<kPts, false, 4096>; break;
      case 8192: k = rcm0 ? k_cs1d<kPts, true, 8192> : k_cs1d<kPts, false, 8192>; break;
      default: break;
    }
    if (k != (rcm0 ? k_cs1d<kPts, true> : k_cs1d<kPts, false>)) threads = tq;
  }
  cudaError_t e = allow_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<nitems, threads, smem, st>>>(la, f, g, h);
  return cudaGetLastError();
}

}  // namespace hd
