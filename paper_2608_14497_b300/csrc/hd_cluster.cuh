// hd_cluster.cuh -- descriptors and host interface of the cluster hybridRCM
// kernel (hd_cl_kernel.cuh, hd_cl_launch.cuh).
#pragma once
#include <cuda_runtime.h>

#include "hd_conv1d.cuh"
#include "hd_internal.h"

namespace hd {

constexpr int kClusterCtas = 16;    // largest cluster (C = 16 CTAs, q = 32 residues)
constexpr int kClusterMaxM = 4608;  // largest residue DFT length (M = 256 R3, R3 <= 18)

// One convolution: q = 2C residues of length m = 256 R3, p = ceil(Lp/m) <= C.
struct CItem {
  int64_t off;
  int64_t off_in;  // explicit-padding baseline: offset of the item in the padded inputs
  int32_t L, m, p, C;
  int32_t K;           // real output length (L <= K <= 2L - 1; 0: K = L)
  int32_t pad_;
  const float2* tw;    // zeta_N^k, N = 2 C m
  const float2* tabm;  // per-length table of the kernel's passes and product (cl::Shape)
};

// Items of one launch (all of the same (C, m), one cluster each), or one item
// by value (items == nullptr) repeated at offsets one_item.off + i * stride
// (a batch of equal lengths).
struct ClusterLaunch {
  const CItem* items;
  CItem one_item;
  int64_t stride;
  int* err;  // device error word (bounded waits that gave up), or nullptr
};

// Whether the kernel is built for clusters of C CTAs with residue length m.
bool cluster_instance(int C, int m);
// (C, m, p) for a length: the measured cheapest built instance when `tun`
// holds an autotuner table, else the smallest cluster whose largest length
// suffices, with the smallest such length.
bool cluster_params(int64_t L, int* C, int* m, int* p, const ClusterTuning* tun = nullptr);
// (C, m, p) for one convolution per call (latency model; see hd_cluster.cu).
bool cluster_params_single(int64_t L, int* C, int* m, int* p);
// Time every built instance on synthetic batches (device scratch, ~50 MB).
hd_status cluster_autotune(hd_ctx* c, ClusterTuning* out);
// Launch over `nitems` convolutions of the same (C, m) (clusters of C CTAs);
// exp: the explicit-padding baseline (f, g zero-padded copies, C <= 8).
cudaError_t launch_rcm1d_cluster(const ClusterLaunch& cl, int C, int m, int nitems, const float* f,
                                 const float* g, float* h, cudaStream_t st, bool exp = false);
// Zero-padded copies of the items of f and g (item i: L_i values at off_i
// become 2 L_i values at off_in_i).
cudaError_t launch_pad_items(const CItem* items, int nitems, int Lmax, const float* f, const float* g, float* pf,
                             float* pg, cudaStream_t st);
cudaError_t launch_pad_one(int64_t L, int64_t batch, const float* f, const float* g, float* pf, float* pg,
                           cudaStream_t st);
// Per-cluster-size dispatch over R3 = m / 256 (hd_cl_c*.cu); cudaErrorInvalidValue
// for an instance that is not built.
#define HD_CL_LAUNCHER(name)                                                                                   \
  cudaError_t name(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h, \
                   cudaStream_t st);
HD_CL_LAUNCHER(launch_cl_c1)
HD_CL_LAUNCHER(launch_cl_c1b)
HD_CL_LAUNCHER(launch_cl_c2)
HD_CL_LAUNCHER(launch_cl_c4)
HD_CL_LAUNCHER(launch_cl_c4b)
HD_CL_LAUNCHER(launch_cl_c8)
HD_CL_LAUNCHER(launch_cl_c8b)
HD_CL_LAUNCHER(launch_cl_c16)
HD_CL_LAUNCHER(launch_clx_c1)
HD_CL_LAUNCHER(launch_clx_c1b)
HD_CL_LAUNCHER(launch_clx_c2)
HD_CL_LAUNCHER(launch_clx_c4)
HD_CL_LAUNCHER(launch_clx_c4b)
HD_CL_LAUNCHER(launch_clx_c8)
HD_CL_LAUNCHER(launch_clx_c8b)
#undef HD_CL_LAUNCHER

}  // namespace hd
