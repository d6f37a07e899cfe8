// hd_cluster.cu -- hybridRCM 1D convolutions with the residues of one
// convolution spread over a thread-block cluster (the fast path of the batched
// and single 1D calls).
//
// A convolution of real length L (packed length Lp = ceil(L/2), Eq.
// complexPacking) is handled by C CTAs (C in {1, 2, 4, 8}) with q = 2C
// residues of length m (q m >= L, p = ceil(Lp/m) <= C).  CTA c owns the
// conjugate residue pair {c, q - c} (CTA 0 owns the self-paired residues 0 and
// q/2), so the RCM operator in residue form (Eqs. Hr and Hr-conj) needs no data
// from other CTAs.  The two sums over blocks that couple the residues run as
// exchanges through distributed shared memory:
//   phase 1  (Eq. forwardr, inner sum)  CTA c takes a slice of s, reads the p
//            inputs f~_{tm+s} of each s once, evaluates sum_t zeta_q^{rt} x_t
//            for every residue r with two length-C DFTs (the inputs vanish for
//            t >= q/2), multiplies by zeta_N^{rs}, and stores each value into
//            the shared memory of the residue's owner;
//   phase 2  length-m DFTs of the four owned arrays (F and G of both
//            residues), the RCM product, backward DFTs (Eq. accumulator);
//   phase 3  (Eq. accumulation) CTA c gathers w_r[s] of every residue for its
//            slice of s from the owners, applies zeta_N^{-rs} and the length-q
//            backward sum over r for the p needed blocks t (again two length-C
//            DFTs), scales by 1/N and writes the unpacked real outputs.
// Inputs are read once and outputs written once: the kernel's HBM traffic is
// the 12 bytes per real element of the problem plus twiddle tables.
//
// One launch covers a whole batch: clusters have 8 CTAs; a cluster processes a
// "unit" of 8/C convolutions of the same C (CTAs of different convolutions of a
// unit never exchange data; they only share the cluster barriers).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "hd_cluster.cuh"
#include "hd_fft_fast.cuh"

namespace cg = cooperative_groups;

namespace hd {

// length-C DFT (C in {1, 2, 4, 8}) of v[0..C), in place.
template <int SIGN>
__device__ __forceinline__ void dft_small(float2* v, int C) {
  if (C == 2) dft2<SIGN>(v[0], v[1]);
  else if (C == 4) dft4<SIGN>(v[0], v[1], v[2], v[3]);
  else if (C == 8) dft8<SIGN>(v);
}

__device__ __forceinline__ int res_owner(int r, int C) { return r < C ? r : (r == C ? 0 : 2 * C - r); }
__device__ __forceinline__ int res_slot(int r, int C) { return r < C ? 0 : 1; }

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads, 1)
    k_rcm1d_cluster(ClusterLaunch cl, const float* f, const float* g, float* h) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int T = blockDim.x, tid = threadIdx.x;
  const CUnit u = cl.units ? cl.units[blockIdx.x / kClusterCtas] : cl.one_unit;
  const int C = u.C;
  const int sub = crank / C, c = crank - sub * C;
  const bool active = sub < u.count;
  CItem it;
  if (active) it = cl.items ? cl.items[u.first + sub] : cl.one_item;
  const int m = active ? it.m : 1;
  const int q = 2 * C, N = q * m;
  const int Pm = pad_stride(m);
  float2* twn = sm;                          // zeta_m^k, k < m
  float2* arr = sm + ((m + 1) & ~1);         // F_a, F_b, G_a, G_b (stride Pm)
  if (active) {
    for (int k = tid; k < m; k += T) twn[k] = __ldg(it.tw + (size_t)k * q);
  }
  // every CTA of the cluster is running and has its tables before any
  // distributed-shared-memory traffic
  cluster.sync();

  const int L = active ? it.L : 0;
  const int Lp = (L + 1) >> 1;
  const int p = active ? it.p : 0;
  const int chunk = (m + C - 1) / C;
  const int s0 = c * chunk, s1 = min(m, s0 + chunk);
  const int rank0 = sub * C;
  const float2* __restrict__ tw = active ? it.tw : nullptr;

  // ---- phase 1: Eq. forwardr, sum over t and the pre-twiddle, scattered to owners
  if (active) {
    for (int which = 0; which < 2; ++which) {
      const float* x = (which ? g : f) + it.off;
      for (int s = s0 + tid; s < s1; s += T) {
        float2 e0[8], e1[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          float2 v = make_float2(0.f, 0.f);
          const int j = t * m + s;
          if (t < p && j < Lp) v = make_float2(x[2 * j], (2 * j + 1 < L) ? x[2 * j + 1] : 0.f);
          e0[t] = v;
          e1[t] = (t < C) ? cmul(v, __ldg(tw + (size_t)t * m)) : v;  // zeta_q^t x_t
        }
        dft_small<1>(e0, C);
        dft_small<1>(e1, C);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (r < q) {
            const float2 y = cmul((r & 1) ? e1[r >> 1] : e0[r >> 1], __ldg(tw + r * s));
            float2* dst = cluster.map_shared_rank(arr, rank0 + res_owner(r, C));
            dst[(which * 2 + res_slot(r, C)) * Pm + pad16(s)] = y;
          }
        }
      }
    }
  }
  cluster.sync();

  // ---- phase 2: DFTs of the owned residues, RCM product, backward DFTs
  if (active) {
    if (4 * m <= kClusterPts * T) {
      cta_fft_fast<1, kClusterPts>(arr, Pm, 4, m, twn);
    } else {
      cta_fft_fast<1, kClusterPts>(arr, Pm, 2, m, twn);
      cta_fft_fast<1, kClusterPts>(arr + 2 * Pm, Pm, 2, m, twn);
    }
    float2* Fa = arr;
    float2* Fb = arr + Pm;
    float2* Ga = arr + 2 * Pm;
    float2* Gb = arr + 3 * Pm;
    if (c == 0) {
      // residues 0 (l* = (m - l) mod m) and C = q/2 (l* = m - 1 - l), each self-paired
      for (int idx = tid; idx < 2 * m; idx += T) {
        const int slot = idx >= m ? 1 : 0;
        const int l = idx - slot * m;
        const int r = slot ? C : 0;
        const int ls = slot ? (m - 1 - l) : (l == 0 ? 0 : m - l);
        if (l > ls) continue;
        float2* F = slot ? Fb : Fa;
        float2* G = slot ? Gb : Ga;
        const float2 A = F[pad16(l)], B = G[pad16(l)], Ac = F[pad16(ls)], Bc = G[pad16(ls)];
        const float2 z = __ldg(tw + q * l + r);
        const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
        const float2 alpha = cmul(cmul(csub(A, cconj(Ac)), csub(B, cconj(Bc))), Z);
        F[pad16(l)] = csub(cmul(A, B), alpha);
        if (ls != l) F[pad16(ls)] = csub(cmul(Ac, Bc), cconj(alpha));
      }
    } else {
      const int ra = c;
      for (int l = tid; l < m; l += T) {
        const int ls = m - 1 - l;
        const float2 A = Fa[pad16(l)], B = Ga[pad16(l)], Ac = Fb[pad16(ls)], Bc = Gb[pad16(ls)];
        const float2 z = __ldg(tw + q * l + ra);
        const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
        const float2 alpha = cmul(cmul(csub(A, cconj(Ac)), csub(B, cconj(Bc))), Z);
        Fa[pad16(l)] = csub(cmul(A, B), alpha);
        Fb[pad16(ls)] = csub(cmul(Ac, Bc), cconj(alpha));
      }
    }
    __syncthreads();
    cta_fft_fast<-1, kClusterPts>(arr, Pm, 2, m, twn);
  }
  cluster.sync();

  // ---- phase 3: Eq. accumulation, gathered from the owners
  if (active) {
    const float sc = 1.0f / (float)N;
    float* hi = h + it.off;
    for (int s = s0 + tid; s < s1; s += T) {
      float2 e0[8], e1[8];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (r < q) {
          const float2* src = cluster.map_shared_rank(arr, rank0 + res_owner(r, C));
          const float2 w = cmul(src[res_slot(r, C) * Pm + pad16(s)], cconj(__ldg(tw + r * s)));
          if (r & 1) e1[r >> 1] = w;
          else e0[r >> 1] = w;
        }
      }
      dft_small<-1>(e0, C);
      dft_small<-1>(e1, C);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int j = t * m + s;
        if (t < p && j < Lp) {
          const float2 o = cadd(e0[t], cmul(e1[t], cconj(__ldg(tw + (size_t)t * m))));
          hi[2 * j] = o.x * sc;
          if (2 * j + 1 < L) hi[2 * j + 1] = o.y * sc;
        }
      }
    }
  }
  // no CTA leaves while others may still read its shared memory
  cluster.sync();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Candidate DFT lengths: {1, 3, 5, 9} x 2^a up to the cap (few distinct
// lengths, so twiddle tables are shared across a batch and stay in L2).
static const std::vector<int>& ladder() {
  static std::vector<int> v;
  if (v.empty()) {
    for (int base : {1, 3, 5, 9})
      for (int x = base; x <= kClusterMaxM; x *= 2) v.push_back(x);
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  return v;
}

bool cluster_params(int64_t L, int* C_out, int* m_out, int* p_out) {
  if (L < 1) return false;
  const int64_t Lp = (L + 1) / 2;
  for (int C = 1; C <= 8; C *= 2) {
    const int64_t need = (L + 2 * C - 1) / (2 * C);  // q m >= L, q = 2C
    for (int mm : ladder()) {
      if (mm >= need) {
        *C_out = C;
        *m_out = mm;
        *p_out = (int)((Lp + mm - 1) / mm);
        return true;
      }
    }
  }
  return false;
}

size_t cluster_smem_bytes(int m_max) {
  return sizeof(float2) * ((size_t)((m_max + 1) & ~1) + 4 * (size_t)pad_stride(m_max));
}

cudaError_t launch_rcm1d_cluster(const ClusterLaunch& cl, int nunits, size_t smem, const float* f, const float* g,
                                 float* h, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_rcm1d_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_rcm1d_cluster<<<nunits * kClusterCtas, kClusterThreads, smem, st>>>(cl, f, g, h);
  return cudaGetLastError();
}

int cluster_max_active(size_t smem) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(kClusterCtas * 64, 1, 1);
  cfg.blockDim = dim3(kClusterThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kClusterCtas;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaFuncSetAttribute(k_rcm1d_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_rcm1d_cluster, &cfg) != cudaSuccess) return -1;
  return n;
}

}  // namespace hd
