// hd_cluster.cuh -- descriptors of the cluster hybridRCM kernel.
#pragma once
#include <cuda_runtime.h>

#include "hd_conv1d.cuh"
#include "hd_internal.h"

namespace hd {

constexpr int kClusterCtas = 8;       // largest cluster (C = 8 CTAs, q = 16 residues)
constexpr int kClusterThreads = 512;  // threads per CTA
constexpr int kClusterPts = 24;       // FFT points per thread per pass
constexpr int kClusterMaxM = 4608;    // largest residue DFT length (shared memory)

// One convolution: q = 2C residues of length m, p = ceil(Lp/m) <= C.
struct CItem {
  int64_t off;
  int32_t L, m, p, C;
  int32_t plan;
  int32_t pad_;
  const float2* tw;    // zeta_N^k, N = 2 C m
  const float2* tabm;  // per-length table: pass twiddles, then zeta_m^l (hd_fft_fast.cuh)
};

// Items of one launch (all of the same C, one cluster each), or one item by
// value (items == nullptr).
struct ClusterLaunch {
  const CItem* items;
  CItem one_item;
};

// (C, m, p) for a length: the measured cheapest candidate when `tun` holds an
// autotuner table, else the smallest cluster whose largest ladder length
// suffices, with the smallest such length.
bool cluster_params(int64_t L, int* C, int* m, int* p, const ClusterTuning* tun = nullptr);
// Time every candidate on synthetic batches (device scratch, a few tens of MB).
hd_status cluster_autotune(hd_ctx* c, ClusterTuning* out);
size_t cluster_smem_bytes(int m_max);
// Launch over `nitems` convolutions of the same C (clusters of C CTAs).
cudaError_t launch_rcm1d_cluster(const ClusterLaunch& cl, int C, int nitems, size_t smem, const float* f,
                                 const float* g, float* h, cudaStream_t st);
cudaError_t launch_cluster_c1(const ClusterLaunch& cl, int nitems, size_t smem, const float* f, const float* g,
                              float* h, cudaStream_t st);
cudaError_t launch_cluster_c2(const ClusterLaunch& cl, int nitems, size_t smem, const float* f, const float* g,
                              float* h, cudaStream_t st);
cudaError_t launch_cluster_c4(const ClusterLaunch& cl, int nitems, size_t smem, const float* f, const float* g,
                              float* h, cudaStream_t st);
cudaError_t launch_cluster_c8(const ClusterLaunch& cl, int nitems, size_t smem, const float* f, const float* g,
                              float* h, cudaStream_t st);

}  // namespace hd
