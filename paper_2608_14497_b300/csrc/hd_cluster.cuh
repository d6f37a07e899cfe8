// hd_cluster.cuh -- descriptors of the cluster hybridRCM kernel.
#pragma once
#include <cuda_runtime.h>

#include "hd_conv1d.cuh"
#include "hd_internal.h"

namespace hd {

constexpr int kClusterCtas = 8;       // CTAs per cluster
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

// A cluster's work: `count` (<= 8/C) consecutive items starting at `first`.
struct CUnit {
  int32_t first, count, C, pad_;
};

struct ClusterLaunch {
  const CUnit* units;   // nullptr: one_unit / one_item / one_plan
  const CItem* items;
  const FftPlan* plans;
  CUnit one_unit;
  CItem one_item;
  FftPlan one_plan;
};

// (C, m, p) for a length: the measured cheapest candidate when `tun` holds an
// autotuner table, else the smallest cluster whose largest ladder length
// suffices, with the smallest such length.
bool cluster_params(int64_t L, int* C, int* m, int* p, const ClusterTuning* tun = nullptr);
// Time every candidate on synthetic batches (device scratch, a few tens of MB).
hd_status cluster_autotune(hd_ctx* c, ClusterTuning* out);
size_t cluster_smem_bytes(int m_max);
cudaError_t launch_rcm1d_cluster(const ClusterLaunch& cl, int nunits, size_t smem, const float* f, const float* g,
                                 float* h, cudaStream_t st);
int cluster_max_active(size_t smem);

}  // namespace hd
