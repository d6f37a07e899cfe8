// hd_cl_launch.cuh -- the cluster hybridRCM kernel (steps in hd_cl_kernel.cuh)
// and its launch, instantiated per (C, R3) by hd_cl_c{1,2,4,8}.cu.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "hd_cl_kernel.cuh"
#include "hd_cluster.cuh"

namespace hd {
namespace cl {
namespace cg = cooperative_groups;

__device__ __forceinline__ unsigned mapa_u32(unsigned local, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
// Cluster barrier halves: arrive (release, or relaxed when nothing is
// published) and wait (acquire); every thread executes each once per barrier.
__device__ __forceinline__ void arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void arrive_release() { asm volatile("barrier.cluster.arrive.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void wait_acquire() { asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory"); }

// mbarrier with one arrival (the thread that posts the expected byte count)
// and a transaction count completed by the senders' st.async stores.
__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// Wait for phase 0 of `bar`, bounded: the data of one cluster arrive within
// microseconds (the CTAs of a cluster are co-scheduled), so after kWaitCycles
// of SM clock (about 16 ms) the wait gives up, records HD_ETIMEOUT in the
// device error word and returns; once the word is set, later waits return at
// once, so a faulty launch ends quickly.  The results are then invalid; the
// host reads the word with hd_last_device_error.
constexpr long long kWaitCycles = 1LL << 25;
__device__ __forceinline__ void mbar_wait(unsigned bar, int* err) {
  if (err && *(volatile int*)err != 0) return;
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar)
        : "memory");
    if (done) return;
    if (clock64() - t0 > kWaitCycles) {
      if (err) atomicExch(err, (int)HD_ETIMEOUT);
      return;
    }
  }
}

// One convolution per cluster of C CTAs; CTA c owns the residue pair {c, q - c}.
// Data move between the CTAs only by st.async stores that complete on the
// receiver's mbarrier: phase 1 into the owners' four arrays (barrier 1, 32 M
// bytes per CTA), phase 3 into the gather buffers (barrier 3, 16 M bytes).
// The hardware cluster barrier is used twice: once at the start (every CTA
// is running and its mbarriers are initialised before any remote store) and
// once after the product (every CTA's G arrays, the gather buffers, are free).
// A single CTA (C = 1) works in its own shared memory only.
// EXP: the explicit-padding baseline (f and g are zero-padded copies, item at
// off_in, real length 2L).
template <int C, int R3, bool EXP>
__global__ void __launch_bounds__(Shape<R3>::T, Shape<R3>::MINB)
    k_rcm_cl(ClusterLaunch la, const float* f, const float* g, float* h) {
  using K = Steps<C, R3, EXP>;
  constexpr int T = K::T;
  constexpr int M = K::M;
  extern __shared__ float4 smem_raw[];
  __shared__ __align__(8) unsigned long long bars[2];
  float2* arr = reinterpret_cast<float2*>(smem_raw);
  float2* tws = arr + 4 * M;  // pass twiddles (Shape::TABS entries)
  const int tid = threadIdx.x;
  const unsigned bar1 = (unsigned)__cvta_generic_to_shared(&bars[0]);
  const unsigned bar3 = (unsigned)__cvta_generic_to_shared(&bars[1]);
  if (C > 1 && tid == 0) {
    mbar_init(bar1);
    mbar_init(bar3);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    mbar_expect(bar1, (unsigned)(sizeof(float2) * 4 * M));  // the four arrays
    mbar_expect(bar3, (unsigned)(sizeof(float2) * 2 * M));  // q slices of M / C
  }
  // every CTA of the cluster must be running, with its barriers initialised,
  // before the first remote store: arrive now, wait after the first loads
  if constexpr (C > 1) arrive_relaxed();
  CItem it = la.items ? la.items[blockIdx.x / C] : la.one_item;
  if (!la.items) {
    it.off += (int64_t)(blockIdx.x / C) * la.stride;
    it.off_in += (int64_t)(blockIdx.x / C) * (EXP ? 2 * la.stride : la.stride);
  }
  // copy the pass twiddles to shared memory while phase 1 runs; 16-byte chunks
  for (int i = tid; i < Shape<R3>::TABS / 2; i += T) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tws + 2 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(it.tabm + 2 * i) : "memory");
  }
  CtaState x;
  x.f = f;
  x.g = g;
  x.h = h;
  x.off = it.off;
  x.L = it.L;
  x.Lp = (it.L + 1) >> 1;
  x.p = it.p;
  x.c = (int)cg::this_cluster().block_rank();
  x.tw = it.tw;
  x.tab = it.tabm;
  x.arr = arr;
  x.off_in = EXP ? it.off_in : it.off;
  x.Lin = EXP ? 2 * it.L : it.L;
  x.pin = EXP ? (it.L + M - 1) / M : it.p;
  x.Lout = it.K > 0 ? it.K : it.L;
  x.pout = ((x.Lout + 1) / 2 + M - 1) / M;
  {
    const uintptr_t fa = (uintptr_t)(f + x.off_in), ga = (uintptr_t)(g + x.off_in), ha = (uintptr_t)(h + it.off);
    x.in16 = ((fa | ga) & 15) == 0;
    x.in8 = ((fa | ga) & 7) == 0;
    x.out16 = (ha & 15) == 0;
  }
  const unsigned local = (unsigned)__cvta_generic_to_shared(arr);
#pragma unroll
  for (int o = 0; o < C; ++o) {  // raddr_t: 32-bit shared::cluster addresses on the device
    x.rbase[o] = (raddr_t)(uintptr_t)mapa_u32(local, (unsigned)o);
    x.rbar1[o] = (raddr_t)(uintptr_t)mapa_u32(bar1, (unsigned)o);
    x.rbar3[o] = (raddr_t)(uintptr_t)mapa_u32(bar3, (unsigned)o);
  }

  static_assert(C <= 16, "clusters of at most 16 CTAs");
  // ---- phase 1 (Eq. forwardr, inner sum), pushed to the owners: every
  // task's loads in flight first (8 / C tasks of C blocks x 2 values)
  {
    float2 v[K::U1][K::NB][2];
#pragma unroll
    for (int u = 0; u < K::U1; ++u)
      if (K::NT1 % T == 0 || tid + u * T < K::NT1) K::load_task(x, tid + u * T, v[u]);
    if constexpr (C > 1) wait_acquire();
#pragma unroll
    for (int u = 0; u < K::U1; ++u)
      if (K::NT1 % T == 0 || tid + u * T < K::NT1) K::scatter_task(x, tid + u * T, v[u]);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();  // the twiddle copies of every thread are visible
  if constexpr (C > 1) mbar_wait(bar1, la.err);

  // ---- forward DFTs (DIF), RCM product, backward DFTs (DIT)
  K::template pass1<1, 4, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass2<1, 4, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass3<1, 4>(arr, tid);
  __syncthreads();
  K::product(x, tid);
  __syncthreads();
  if constexpr (C > 1) arrive_release();  // this CTA's G arrays (a gather buffer from now on) are free
  K::template pass3<-1, 2>(arr, tid);
  __syncthreads();
  K::template pass2<-1, 2, 1>(arr, tid, tws);
  __syncthreads();
  K::template pass1<-1, 2, 1>(arr, tid, tws);
  __syncthreads();
  if constexpr (C > 1) wait_acquire();  // every CTA's gather buffer is free

  // ---- phase 3 (Eq. accumulation): push w_r[s] to the slice owners, gather
  if constexpr (C > 1) {
    K::push_all(x, tid);
    mbar_wait(bar3, la.err);
  }
  const float sc = 1.0f / (float)(2 * C * M);
#pragma unroll 1
  for (int task = tid; task < K::NT3; task += T) K::gather_task(x, task, sc);
}

// Launch over `nitems` convolutions of the same (C, R3): grid nitems x C in
// clusters of C CTAs (the cluster size is a launch attribute; 16 is beyond the
// portable size and is allowed per kernel).
template <int C, int R3, bool EXP = false>
cudaError_t launch(const ClusterLaunch& la, int nitems, const float* f, const float* g, float* h, cudaStream_t st) {
  auto kern = k_rcm_cl<C, R3, EXP>;
  cudaError_t e = smem_optin((const void*)kern, Shape<R3>::SMEM);
  if (e != cudaSuccess) return e;
  if constexpr (C > 8) {
    static bool nonportable_set[64] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !nonportable_set[dev]) {
      e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) nonportable_set[dev] = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nitems * C), 1, 1);
  cfg.blockDim = dim3(Shape<R3>::T, 1, 1);
  cfg.dynamicSmemBytes = Shape<R3>::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, la, f, g, h);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace cl
}  // namespace hd
