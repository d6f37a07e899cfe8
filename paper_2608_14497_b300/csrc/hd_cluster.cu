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
  const int Sm = swz_stride(m);
  float2* tws = sm;                 // per-pass twiddles of the length-m DFT (m - 1 entries)
  float2* arr = sm + swz_stride(m);  // F_a, F_b, G_a, G_b, each Sm long, swizzled
  const float2* __restrict__ tw = active ? it.tw : nullptr;  // zeta_N^k
  if (active) fill_pass_twiddles(tws, m, it.tabm);
  // every CTA of the cluster is running (and has its table) before any
  // distributed-shared-memory traffic
  cluster.sync();

  const int L = active ? it.L : 0;
  const int Lp = (L + 1) >> 1;
  const int p = active ? it.p : 0;
  const int chunk = (m + C - 1) / C;
  const int s0 = c * chunk, s1 = min(m, s0 + chunk);
  const int rank0 = sub * C;

  // zeta_N^{r s} for r < q from two table reads: zeta_N^{4a + b} s = w4^a w1^b
  auto residue_twiddles = [&](int s, float2* wr) {
    const float2 w1 = __ldg(tw + s);
    float2 p1[4], p4[4];
    p1[0] = make_float2(1.f, 0.f);
    p1[1] = w1;
    p1[2] = cmul(w1, w1);
    p1[3] = cmul(p1[2], w1);
    p4[0] = p1[0];
    if (q > 4) {
      const float2 w4 = __ldg(tw + 4 * s);
      p4[1] = w4;
      p4[2] = cmul(w4, w4);
      p4[3] = cmul(p4[2], w4);
    } else {
      p4[1] = p4[2] = p4[3] = p1[0];
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) wr[r] = (r < 4) ? p1[r] : cmul(p4[r >> 2], p1[r & 3]);
  };

  // ---- phase 1: Eq. forwardr, sum over t and the pre-twiddle, scattered to owners
  if (active) {
    for (int s = s0 + tid; s < s1; s += T) {
      float2 wr[16];
      residue_twiddles(s, wr);
      for (int which = 0; which < 2; ++which) {
        const float* x = (which ? g : f) + it.off;
        float2 e0[8], e1[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          float2 v = make_float2(0.f, 0.f);
          const int j = t * m + s;
          if (t < p && j < Lp) v = make_float2(x[2 * j], (2 * j + 1 < L) ? x[2 * j + 1] : 0.f);
          e0[t] = v;
          e1[t] = (t < C && t > 0) ? cmul(v, __ldg(tw + (size_t)t * m)) : v;  // zeta_q^t x_t
        }
        dft_small<1>(e0, C);
        dft_small<1>(e1, C);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (r < q) {
            const float2 y = cmul((r & 1) ? e1[r >> 1] : e0[r >> 1], wr[r]);
            float2* dst = cluster.map_shared_rank(arr, rank0 + res_owner(r, C));
            dst[(which * 2 + res_slot(r, C)) * Sm + swz(s)] = y;
          }
        }
      }
    }
  }
  cluster.sync();

  // ---- phase 2: DFTs of the owned residues, RCM product, backward DFTs
  if (active) {
    if (4 * m <= kClusterPts * T) {
      cta_fft_fast<1, kClusterPts>(arr, Sm, 4, m, tws);
    } else {
      cta_fft_fast<1, kClusterPts>(arr, Sm, 2, m, tws);
      cta_fft_fast<1, kClusterPts>(arr + 2 * Sm, Sm, 2, m, tws);
    }
    float2* Fa = arr;
    float2* Fb = arr + Sm;
    float2* Ga = arr + 2 * Sm;
    float2* Gb = arr + 3 * Sm;
    // c = 0: residues 0 (l* = (m - l) mod m) and C = q/2 (l* = m - 1 - l), each
    // self-paired; c > 0: residue c (l) with residue q - c (l* = m - 1 - l)
    const int npairs = (c == 0) ? 2 * m : m;
    for (int idx = tid; idx < npairs; idx += T) {
      const int slot = idx >= m ? 1 : 0;
      const int l = idx - slot * m;
      int r, ls;
      float2 *Fl, *Gl, *Fs, *Gs;
      if (c == 0) {
        r = slot ? C : 0;
        ls = slot ? (m - 1 - l) : (l == 0 ? 0 : m - l);
        if (l > ls) continue;
        Fl = Fs = slot ? Fb : Fa;
        Gl = Gs = slot ? Gb : Ga;
      } else {
        r = c;
        ls = m - 1 - l;
        Fl = Fa;
        Gl = Ga;
        Fs = Fb;
        Gs = Gb;
      }
      const int il = swz(l), is = swz(ls);
      const float2 A = Fl[il], B = Gl[il], Ac = Fs[is], Bc = Gs[is];
      // zeta_N^{q l + r} = zeta_m^l zeta_N^r
      const float2 z = cmul(__ldg(it.tabm + (m - 1) + l), __ldg(tw + r));
      const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);  // (1 + zeta_N^k) / 4
      const float2 alpha = cmul(cmul(csub(A, cconj(Ac)), csub(B, cconj(Bc))), Z);
      Fl[il] = csub(cmul(A, B), alpha);
      if (!(c == 0 && ls == l)) Fs[is] = csub(cmul(Ac, Bc), cconj(alpha));
    }
    __syncthreads();
    cta_fft_fast<-1, kClusterPts>(arr, Sm, 2, m, tws);
  }
  cluster.sync();

  // ---- phase 3: Eq. accumulation, gathered from the owners
  if (active) {
    const float sc = 1.0f / (float)N;
    float* hi = h + it.off;
    for (int s = s0 + tid; s < s1; s += T) {
      float2 wr[16];
      residue_twiddles(s, wr);
      float2 e0[8], e1[8];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (r < q) {
          const float2* src = cluster.map_shared_rank(arr, rank0 + res_owner(r, C));
          const float2 w = cmul(src[res_slot(r, C) * Sm + swz(s)], cconj(wr[r]));
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
          const float2 o = (t > 0) ? cadd(e0[t], cmul(e1[t], cconj(__ldg(tw + (size_t)t * m)))) : cadd(e0[0], e1[0]);
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

bool cluster_params(int64_t L, int* C_out, int* m_out, int* p_out, const ClusterTuning* tun) {
  if (L < 1) return false;
  const int64_t Lp = (L + 1) / 2;
  if (tun && tun->valid) {
    // cheapest measured candidate among the three shortest feasible lengths of each C
    double best = 1e300;
    int seen[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < tun->C.size(); ++i) {
      const int C = tun->C[i], mm = tun->m[i];
      const int ci = C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3;
      if ((int64_t)2 * C * mm < L || seen[ci] >= 3) continue;
      ++seen[ci];
      if (tun->us[i] < best) {
        best = tun->us[i];
        *C_out = C;
        *m_out = mm;
        *p_out = (int)((Lp + mm - 1) / mm);
      }
    }
    if (best < 1e300) return true;
  }
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

hd_status cluster_autotune(hd_ctx* c, ClusterTuning* out) {
  // candidates in increasing m per C (cluster_params relies on that order)
  std::vector<int> Cs, ms;
  for (int C = 1; C <= 8; C *= 2)
    for (int mm : ladder())
      if (mm >= 64) {
        Cs.push_back(C);
        ms.push_back(mm);
      }
  const int64_t budget = int64_t{1} << 22;  // real elements per timed batch
  float *f = nullptr, *g = nullptr, *h = nullptr;
  CUnit* d_units = nullptr;
  CItem* d_items = nullptr;
  hd_status st = HD_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&f, sizeof(float) * budget) != cudaSuccess || cudaMalloc(&g, sizeof(float) * budget) != cudaSuccess ||
      cudaMalloc(&h, sizeof(float) * budget) != cudaSuccess ||
      cudaMalloc(&d_units, sizeof(CUnit) * 4096) != cudaSuccess ||
      cudaMalloc(&d_items, sizeof(CItem) * 4096) != cudaSuccess) {
    st = HD_ENOMEM;
  }
  if (st == HD_OK) {
    cudaMemset(f, 0, sizeof(float) * budget);
    cudaMemset(g, 0, sizeof(float) * budget);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  out->C.clear();
  out->m.clear();
  out->us.clear();
  for (size_t i = 0; i < Cs.size() && st == HD_OK; ++i) {
    const int C = Cs[i], mm = ms[i];
    const int64_t L = (int64_t)2 * C * mm;
    const int per = kClusterCtas / C;
    int64_t K = budget / L;
    K = std::max<int64_t>(per, std::min<int64_t>(K, 4096));
    K = (K / per) * per;
    if (K * L > budget) continue;
    hd_status terr = HD_OK;
    const float2* tw = c->tables.get(L, 0, &terr);
    const float2* tabm = tw ? c->tables.get_pass_table(mm, 0, &terr) : nullptr;
    if (!tw || !tabm) {
      st = terr;
      break;
    }
    std::vector<CItem> items(K);
    std::vector<CUnit> units(K / per);
    for (int64_t k = 0; k < K; ++k) {
      std::memset(&items[k], 0, sizeof(CItem));
      items[k].off = k * L;
      items[k].L = (int32_t)L;
      items[k].m = mm;
      items[k].p = (int)(((L + 1) / 2 + mm - 1) / mm);
      items[k].C = C;
      items[k].tw = tw;
      items[k].tabm = tabm;
    }
    for (size_t u = 0; u < units.size(); ++u) {
      std::memset(&units[u], 0, sizeof(CUnit));
      units[u].first = (int)(u * per);
      units[u].count = per;
      units[u].C = C;
    }
    cudaMemcpy(d_items, items.data(), sizeof(CItem) * K, cudaMemcpyHostToDevice);
    cudaMemcpy(d_units, units.data(), sizeof(CUnit) * units.size(), cudaMemcpyHostToDevice);
    ClusterLaunch cl;
    std::memset(&cl, 0, sizeof(cl));
    cl.units = d_units;
    cl.items = d_items;
    const size_t smem = cluster_smem_bytes(mm);
    if (launch_rcm1d_cluster(cl, (int)units.size(), smem, f, g, h, 0) != cudaSuccess) {
      st = HD_ECUDA;
      break;
    }
    cudaEventRecord(e0, 0);
    for (int rep = 0; rep < 3; ++rep) launch_rcm1d_cluster(cl, (int)units.size(), smem, f, g, h, 0);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = HD_ECUDA;
      break;
    }
    float ms_el = 0.f;
    cudaEventElapsedTime(&ms_el, e0, e1);
    out->C.push_back(C);
    out->m.push_back(mm);
    out->us.push_back(1e3 * ms_el / (3.0 * (double)K));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(f);
  cudaFree(g);
  cudaFree(h);
  cudaFree(d_units);
  cudaFree(d_items);
  out->valid = (st == HD_OK) && !out->us.empty();
  return st;
}

size_t cluster_smem_bytes(int m_max) { return sizeof(float2) * 5 * (size_t)swz_stride(m_max); }

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
