// hd_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <vector>

#include "../../include/hdconv.h"
#include "hd_fft.cuh"

namespace hd {

// Per-item descriptor of a 1D convolution (one CTA, or one cluster, each).
struct Item1D {
  int64_t off;       // offset (in floats) of the item in f, g and h
  int32_t L;         // real length
  int32_t m, q, p;   // hybrid parameters (packed lengths for hybridRCM)
  int32_t plan;      // index of the length-m FFT plan
  int32_t plan_half; // index of the length-m/2 FFT plan (-1 if unused)
  int32_t K;         // real output length (L <= K <= 2L - 1; 0: K = L)
  const float2* tw;  // zeta_N^k table, N = q m
  void* gacc;        // accumulator in global memory, or nullptr for shared memory
};

// Host planner (hd_plan.cpp).
bool factor_radices(int n, FftPlan* out);  // false if n < 1
bool smooth235(int64_t n);
int64_t next_smooth(int64_t n);
int64_t ladder_ceil(int64_t n);  // smallest {1, 3, 5, 9} x 2^a >= n

// Twiddle tables: zeta_N^k, k < N, FP64 on the device, rounded to FP32.
// A table is built on the cache's own stream and is complete when get()
// returns (that stream is synchronised once per new table), so a call on any
// stream may read a cached table without an ordering hazard.  The stream
// argument is kept for the call sites; it does not order the build.
struct TableCache {
  std::map<int64_t, float2*> tabs;
  cudaStream_t build = nullptr;  // private non-blocking stream of the builds
  const float2* get(int64_t N, cudaStream_t st, hd_status* err);
  // per-length table of the cluster kernel, length n = 256 R3 (cl::Shape)
  const float2* get_pass_table(int n, cudaStream_t st, hd_status* err);
  cudaStream_t build_stream(hd_status* err);
  void clear();
};

// Autotuner result for the cluster hybridRCM kernel: measured microseconds
// per convolution for each candidate (C CTAs, residue DFT length m), timed at
// the largest length the candidate covers, L = 2 C m.
struct ClusterTuning {
  bool valid = false;
  std::vector<int> C, m;
  std::vector<double> us;
};

}  // namespace hd

struct hd_ctx {
  int device = 0;
  hd::TableCache tables;
  // reusable device scratch, grown on demand
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* ws2 = nullptr;  // the adjoint's reversed gradient and temporary
  size_t ws2_bytes = 0;
  // plan/item upload buffers for single calls
  void* meta = nullptr;
  size_t meta_bytes = 0;
  int* dev_err = nullptr;  // device error word (bounded waits, bad launches)
  hd::ClusterTuning tuning;  // filled on the first batched hybridRCM plan
  int max_smem = 0;        // opt-in shared memory per block
  int num_sms = 0;
  std::mutex mu;
};

namespace hd {
// Record the reason of a failed call for hd_last_error_string (per host
// thread) and return the status (HD_ECUDA for cuda_fail).
hd_status fail(hd_status s, const char* what);
hd_status cuda_fail(cudaError_t e, const char* where);
hd_status ensure_ws(hd_ctx* c, size_t bytes, cudaStream_t st);
// Dynamic shared-memory opt-in of a kernel, set once per device and size.
cudaError_t smem_optin(const void* fn, size_t smem);
hd_status ensure_ws2(hd_ctx* c, size_t bytes, cudaStream_t st);
hd_status ensure_meta(hd_ctx* c, size_t bytes);
}  // namespace hd
