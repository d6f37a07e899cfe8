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

// One convolution per cluster of C CTAs; CTA c owns the residue pair {c, q - c}.
template <int C, int R3>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(Shape<R3>::T, 1)
    k_rcm_cl(ClusterLaunch la, const float* f, const float* g, float* h) {
  using K = Steps<C, R3>;
  constexpr int T = K::T;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);
  const int tid = threadIdx.x;
  const CItem it = la.items ? la.items[blockIdx.x / C] : la.one_item;
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
  {
    const uintptr_t fa = (uintptr_t)(f + it.off), ga = (uintptr_t)(g + it.off), ha = (uintptr_t)(h + it.off);
    x.in16 = ((fa | ga) & 15) == 0;
    x.in8 = ((fa | ga) & 7) == 0;
    x.out16 = (ha & 15) == 0;
  }
  const unsigned local = (unsigned)__cvta_generic_to_shared(arr);
#pragma unroll
  for (int o = 0; o < C; ++o) x.rbase[o] = (raddr_t)(uintptr_t)mapa_u32(local, (unsigned)o);  // raddr_t: 32-bit on the device
  // every CTA of the cluster must be running before the first remote store:
  // arrive now, wait after the first loads are in flight
  arrive_relaxed();

  // ---- phase 1 (Eq. forwardr, inner sum), scattered to the owners
  {
    float2 v[C][2];
    if (tid < K::NT1) K::load_task(x, tid, v);
    wait_acquire();
#pragma unroll 1
    for (int task = tid; task < K::NT1; task += T) {
      K::scatter_task(x, task, v);
      if (task + T < K::NT1) K::load_task(x, task + T, v);
    }
  }
  arrive_release();
  wait_acquire();

  // ---- forward DFTs (DIF), RCM product, backward DFTs (DIT)
  K::template pass1<1, 4, 2>(arr, tid, x.tab);
  __syncthreads();
  K::template pass2<1, 4, 2>(arr, tid, x.tab);
  __syncthreads();
  K::template pass3<1, 4>(arr, tid);
  __syncthreads();
  K::product(x, tid);
  __syncthreads();
  K::template pass3<-1, 2>(arr, tid);
  __syncthreads();
  K::template pass2<-1, 2, 1>(arr, tid, x.tab);
  __syncthreads();
  K::template pass1<-1, 2, 1>(arr, tid, x.tab);
  arrive_release();
  wait_acquire();

  // ---- phase 3 (Eq. accumulation), gathered from the owners
  const float sc = 1.0f / (float)(2 * C * K::M);
#pragma unroll 1
  for (int task = tid; task < K::NT3; task += T) K::gather_task(x, task, sc);
  // no CTA leaves while others may still read its shared memory
  arrive_relaxed();
  wait_acquire();
}

// Launch over `nitems` convolutions of the same (C, R3): grid nitems x C.
template <int C, int R3>
cudaError_t launch(const ClusterLaunch& la, int nitems, const float* f, const float* g, float* h, cudaStream_t st) {
  const cudaError_t e = smem_optin((const void*)k_rcm_cl<C, R3>, Shape<R3>::SMEM);
  if (e != cudaSuccess) return e;
  k_rcm_cl<C, R3><<<nitems * C, Shape<R3>::T, Shape<R3>::SMEM, st>>>(la, f, g, h);
  return cudaGetLastError();
}

}  // namespace cl
}  // namespace hd
