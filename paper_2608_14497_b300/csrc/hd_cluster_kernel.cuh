// hd_cluster_kernel.cuh -- hybridRCM 1D convolutions with the residues of one
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
// The kernel is instantiated per C (cluster size C, one convolution per
// cluster; hd_cluster_c{1,2,4,8}.cu); a batch launches one instance per C in
// use, the launches running concurrently on separate streams (hd_batch.cu).
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "hd_cluster.cuh"
#include "hd_fft_fast.cuh"

namespace hd {
namespace cg = cooperative_groups;


__device__ __forceinline__ int res_owner(int r, int C) { return r < C ? r : (r == C ? 0 : 2 * C - r); }
__device__ __forceinline__ int res_slot(int r, int C) { return r < C ? 0 : 1; }

// Distributed shared memory through 32-bit shared::cluster addresses: the
// address of `local` (a shared::cta address) in the shared memory of CTA
// `rank` of the cluster, and 8-byte stores / loads there.
__device__ __forceinline__ unsigned map_rank_u32(unsigned local, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_f2(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float2 ld_cluster_f2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

// What the exchange phases of one CTA need.
struct XCtx {
  const float* f;
  const float* g;
  float* h;
  int64_t off;
  int L, Lp, m, p, Sm, s0, s1, rank0;
  unsigned arr_local;     // shared::cta address of this CTA's F_a
  const float2* tw;       // zeta_N^k, N = 2 C m
};

// zeta_N^{r s} for r < Q from two table reads: zeta_N^{(4a + b) s} = w4^a w1^b
template <int Q>
__device__ __forceinline__ void residue_twiddles_q(const float2* __restrict__ tw, int s, float2* wr) {
  const float2 w1 = __ldg(tw + s);
  float2 p1[4];
  p1[0] = make_float2(1.f, 0.f);
  p1[1] = w1;
  p1[2] = cmul(w1, w1);
  p1[3] = cmul(p1[2], w1);
  if constexpr (Q <= 4) {
#pragma unroll
    for (int r = 0; r < Q; ++r) wr[r] = p1[r];
  } else {
    const float2 w4 = __ldg(tw + 4 * s);
    float2 p4[4];
    p4[0] = p1[0];
    p4[1] = w4;
    p4[2] = cmul(w4, w4);
    p4[3] = cmul(p4[2], w4);
#pragma unroll
    for (int r = 0; r < Q; ++r) wr[r] = (r < 4) ? p1[r] : cmul(p4[r >> 2], p1[r & 3]);
  }
}

template <int SIGN, int CC>
__device__ __forceinline__ void dft_c(float2* v) {
  if constexpr (CC == 2) dft2<SIGN>(v[0], v[1]);
  else if constexpr (CC == 4) dft4<SIGN>(v[0], v[1], v[2], v[3]);
  else if constexpr (CC == 8) dft8<SIGN>(v);
}

// s values each thread keeps in flight in the exchange phases (their loads
// are all issued before any arithmetic): 8 / C, so p <= C inputs per array
// and s stay within 16 loads per array.
template <int CC>
constexpr int kSPerThread = CC >= 8 ? 1 : 8 / CC;

// Cluster barrier split in two: every CTA arrives when it starts (relaxed: no
// data is published) and waits only before its first store into another
// CTA's shared memory, so the wait overlaps the first input loads.
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory"); }
// Per-thread (non-aligned) arrive: a thread may arrive from divergent code.
__device__ __forceinline__ void cluster_arrive_thread() { asm volatile("barrier.cluster.arrive.relaxed;\n" ::: "memory"); }

// Phase 1 (Eq. forwardr, sum over t and the pre-twiddle) for C = CC: for each
// s of this CTA's slice, the p packed inputs f~_{tm+s} (t < p <= C; zero for
// C <= t < q) of f and of g, the q-point DFT over t as two length-C DFTs
// (even and odd residues), times zeta_N^{rs}, stored into residue r's owner.
// Both arrays' loads are issued before any arithmetic; zeta_N^{rs} is built
// per residue from zeta_N^{s} and zeta_N^{4s} (few registers held).  Ends the
// cluster barrier begun by cluster_arrive_relaxed().
template <int CC>
__device__ __forceinline__ void scatter_phase(const XCtx& x) {
  constexpr int Q = 2 * CC;
  constexpr int U = kSPerThread<CC>;
  const int T = blockDim.x;
  auto load = [&](int s, int which, float2* v) {
    const float* src = (which ? x.g : x.f) + x.off;
#pragma unroll
    for (int t = 0; t < CC; ++t) {
      const int j = t * x.m + s;
      v[t] = make_float2(0.f, 0.f);
      if (s < x.s1 && t < x.p && j < x.Lp)
        v[t] = make_float2(__ldg(src + 2 * j), (2 * j + 1 < x.L) ? __ldg(src + 2 * j + 1) : 0.f);
    }
  };
  float2 xv[U][2][CC];
  auto load_batch = [&](int sb) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      load(sb + u * T, 0, xv[u][0]);
      load(sb + u * T, 1, xv[u][1]);
    }
  };
  const int sb0 = x.s0 + (int)threadIdx.x;
  load_batch(sb0);
  cluster_wait();  // every CTA of the cluster is running
  for (int sb = sb0; sb < x.s1; sb += U * T) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = sb + u * T;
      if (s < x.s1) {
        // zeta_N^{rs} = (zeta_N^{4s})^{r >> 2} (zeta_N^s)^{r & 3}
        const float2 w1 = __ldg(x.tw + s);
        float2 p1[4], p4[4];
        p1[0] = make_float2(1.f, 0.f);
        p1[1] = w1;
        p1[2] = cmul(w1, w1);
        p1[3] = cmul(p1[2], w1);
        p4[0] = p1[0];
        if constexpr (Q > 4) {
          const float2 w4 = __ldg(x.tw + 4 * s);
          p4[1] = w4;
          p4[2] = cmul(w4, w4);
          p4[3] = cmul(p4[2], w4);
        }
#pragma unroll
        for (int which = 0; which < 2; ++which) {
          const float2* v = xv[u][which];
          float2 e0[CC], e1[CC];
#pragma unroll
          for (int t = 0; t < CC; ++t) {
            e0[t] = v[t];
            e1[t] = (t > 0) ? cmul(v[t], __ldg(x.tw + (size_t)t * x.m)) : v[t];  // zeta_q^t x_t
          }
          dft_c<1, CC>(e0);
          dft_c<1, CC>(e1);
          const unsigned loc = x.arr_local + (unsigned)((which * 2 * x.Sm + s) * sizeof(float2));
#pragma unroll
          for (int r = 0; r < Q; ++r) {
            const float2 wr = (r < 4) ? p1[r] : cmul(p4[r >> 2], p1[r & 3]);
            st_cluster_f2(map_rank_u32(loc + (unsigned)(res_slot(r, CC) * x.Sm * sizeof(float2)),
                                       (unsigned)(x.rank0 + res_owner(r, CC))),
                          cmul((r & 1) ? e1[r >> 1] : e0[r >> 1], wr));
          }
        }
      }
    }
    if (sb + U * T < x.s1) load_batch(sb + U * T);
  }
}

// Phase 3 (Eq. accumulation) for C = CC: w_r[s] of every residue from its
// owner, times zeta_N^{-rs}, the backward q-point sum over r for the p needed
// blocks t (two length-C DFTs), scaled by 1/N, unpacked to the real output.
// Each thread arrives at the final cluster barrier as soon as its last
// distributed-shared-memory value has been used, before its last output
// stores; the caller waits (no CTA may exit while others read its memory).
template <int CC>
__device__ __forceinline__ void gather_phase(const XCtx& x) {
  constexpr int Q = 2 * CC;
  constexpr int U = kSPerThread<CC>;
  const int T = blockDim.x;
  const float sc = 1.0f / (float)(Q * x.m);
  float* hi = x.h + x.off;
  bool arrived = false;
  for (int sb = x.s0 + (int)threadIdx.x; sb < x.s1; sb += U * T) {
    float2 yv[U][Q];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = sb + u * T;
      const unsigned loc = x.arr_local + (unsigned)(s * sizeof(float2));
#pragma unroll
      for (int r = 0; r < Q; ++r)
        yv[u][r] = (s < x.s1) ? ld_cluster_f2(map_rank_u32(loc + (unsigned)(res_slot(r, CC) * x.Sm * sizeof(float2)),
                                                           (unsigned)(x.rank0 + res_owner(r, CC))))
                              : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = sb + u * T;
      if (s < x.s1) {
        float2 wr[Q];
        residue_twiddles_q<Q>(x.tw, s, wr);
        float2 e0[CC], e1[CC];
#pragma unroll
        for (int r = 0; r < Q; ++r) {
          const float2 w = cmul(yv[u][r], cconj(wr[r]));
          if (r & 1) e1[r >> 1] = w;
          else e0[r >> 1] = w;
        }
        if (u == U - 1 && sb + U * T >= x.s1) {
          cluster_arrive_thread();  // every remote value of this thread is consumed
          arrived = true;
        }
        dft_c<-1, CC>(e0);
        dft_c<-1, CC>(e1);
#pragma unroll
        for (int t = 0; t < CC; ++t) {
          const int j = t * x.m + s;
          if (t < x.p && j < x.Lp) {
            const float2 o = (t > 0) ? cadd(e0[t], cmul(e1[t], cconj(__ldg(x.tw + (size_t)t * x.m)))) : cadd(e0[0], e1[0]);
            hi[2 * j] = o.x * sc;
            if (2 * j + 1 < x.L) hi[2 * j + 1] = o.y * sc;
          }
        }
      }
    }
  }
  if (!arrived) cluster_arrive_thread();
}

// One convolution per cluster of C CTAs (C = cluster size); CTA c of the
// cluster owns the residue pair {c, q - c}.
template <int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kClusterThreads, 1)
    k_rcm1d_cluster(ClusterLaunch cl, const float* f, const float* g, float* h) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const int T = blockDim.x, tid = threadIdx.x;
  const CItem it = cl.items ? cl.items[blockIdx.x / C] : cl.one_item;
  const int m = it.m;
  const int Sm = swz_stride(m);
  float2* tws = sm;                 // per-pass twiddles of the length-m DFT (m - 1 entries)
  float2* arr = sm + swz_stride(m);  // F_a, F_b, G_a, G_b, each Sm long, natural order
  const float2* __restrict__ tw = it.tw;  // zeta_N^k
  // the table copy overlaps phase 1 (waited for before the phase-2 barrier)
  fill_pass_twiddles_async(tws, m, it.tabm);
  // every CTA of the cluster must be running before any distributed-shared-
  // memory traffic: arrive now, wait in phase 1 after its first loads
  cluster_arrive_relaxed();

  const int L = it.L;
  const int Lp = (L + 1) >> 1;
  const int p = it.p;
  const int chunk = (m + C - 1) / C;
  const int s0 = c * chunk, s1 = min(m, s0 + chunk);
  const int rank0 = 0;
  XCtx xc;
  xc.f = f;
  xc.g = g;
  xc.h = h;
  xc.off = it.off;
  xc.L = L;
  xc.Lp = Lp;
  xc.m = m;
  xc.p = p;
  xc.Sm = Sm;
  xc.s0 = s0;
  xc.s1 = s1;
  xc.rank0 = rank0;
  xc.arr_local = (unsigned)__cvta_generic_to_shared(arr);
  xc.tw = tw;

  // ---- phase 1: Eq. forwardr, sum over t and the pre-twiddle, scattered to owners
  scatter_phase<C>(xc);  // completes the barrier begun above
  cp_async_wait_all();
  cluster.sync();

  // ---- phase 2: DFTs of the owned residues, RCM product, backward DFTs
  int bwd_res = 0;
  {
    if (4 * m <= struct_capacity(m, kClusterPts, T)) {
      cta_fft_struct<1, kClusterPts, true>(arr, Sm, 4, m, tws, 0);
    } else {
      cta_fft_struct<1, kClusterPts, true>(arr, Sm, 2, m, tws, 0);
      cta_fft_struct<1, kClusterPts, true>(arr + 2 * Sm, Sm, 2, m, tws, 0);
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
      const float2 A = Fl[l], B = Gl[l], Ac = Fs[ls], Bc = Gs[ls];
      // zeta_N^{q l + r} = zeta_m^l zeta_N^r
      const float2 z = cmul(__ldg(it.tabm + (m - 1) + l), __ldg(tw + r));
      const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);  // (1 + zeta_N^k) / 4
      const float2 alpha = cmul(cmul(csub(A, cconj(Ac)), csub(B, cconj(Bc))), Z);
      Fl[l] = csub(cmul(A, B), alpha);
      if (!(c == 0 && ls == l)) Fs[ls] = csub(cmul(Ac, Bc), cconj(alpha));
    }
    __syncthreads();
    // G_a, G_b are free after the product: the backward DFTs of F_a, F_b run
    // out of place between the two pairs of arrays (one barrier per pass)
    bwd_res = cta_fft_struct_oop<-1, true>(arr, arr + 2 * Sm, Sm, 2, m, tws, 0);
  }
  cluster.sync();
  xc.arr_local += (unsigned)(bwd_res * 2 * Sm * sizeof(float2));  // where the owners' results are

  // ---- phase 3: Eq. accumulation, gathered from the owners
  gather_phase<C>(xc);  // arrives at the final barrier
  // no CTA leaves while others may still read its shared memory
  cluster_wait();
}


// Launch of the C-CTA-cluster kernel over `nitems` convolutions.
template <int C>
cudaError_t launch_cluster_c(const ClusterLaunch& cl, int nitems, size_t smem, const float* f, const float* g,
                             float* h, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_rcm1d_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_rcm1d_cluster<C><<<nitems * C, kClusterThreads, smem, st>>>(cl, f, g, h);
  return cudaGetLastError();
}

}  // namespace hd
