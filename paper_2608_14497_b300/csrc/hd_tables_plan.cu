// hd_tables_plan.cu -- roots-of-unity tables (FP64 -> FP32) and FFT radix plans.
//
// Tables: tw[k] = zeta_N^k = exp(2 pi i k / N), k < N (Sec. 2 notation), for
// each padded length N = q m in use.  They are evaluated in FP64 on the GPU
// (sincospi of the exact rational 2k/N) and rounded once to FP32, so every
// twiddle the FP32 kernels use is correctly rounded to within 1 ulp.  One table
// serves all DFT lengths dividing N: zeta_n^x = tw[x N / n].
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "hd_cl_kernel.cuh"
#include "hd_internal.h"

namespace hd {

__global__ void k_roots_fp64(float2* __restrict__ tw, int64_t N) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    // 2k/N in [0, 2): reduce to [-1, 1] to keep the argument small
    double x = (2.0 * (double)k) / (double)N;
    if (x > 1.0) x -= 2.0;
    sincospi(x, &s, &c);
    tw[k] = make_float2((float)c, (float)s);
  }
}

// Per-length table of the cluster kernel for m = 256 R3 (layout cl::Shape in
// hd_cl_kernel.cuh): pass twiddles of the radix-R3 and radix-16 passes, then
// zeta_m^l for the digit-reversed positions; each entry evaluated in FP64 from
// its exact rational angle and rounded once.
__global__ void k_cl_table_fp64(float2* __restrict__ out, int R3, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    long long num, den;
    cl::table_angle(i, R3, &num, &den);
    double s, c;
    double x = (2.0 * (double)(num % den)) / (double)den;
    if (x > 1.0) x -= 2.0;
    sincospi(x, &s, &c);
    out[i] = make_float2((float)c, (float)s);
  }
}

cudaStream_t TableCache::build_stream(hd_status* err) {
  if (!build && cudaStreamCreateWithFlags(&build, cudaStreamNonBlocking) != cudaSuccess) {
    build = nullptr;
    *err = HD_ECUDA;
  }
  return build;
}

// Key space: padded lengths N > 0; per-length pass tables under -n.
const float2* TableCache::get_pass_table(int n, cudaStream_t /*st*/, hd_status* err) {
  auto it = tabs.find(-(int64_t)n);
  if (it != tabs.end()) return it->second;
  cudaStream_t bs = build_stream(err);
  if (!bs) return nullptr;
  if (n < 256 || n % 256) {
    *err = HD_EINVAL;
    return nullptr;
  }
  const int R3 = n / 256;
  const int entries = (R3 - 1) * 256 + 240 + n;  // cl::Shape<R3>::TABN
  float2* p = nullptr;
  if (cudaMalloc(&p, sizeof(float2) * (size_t)entries) != cudaSuccess) {
    *err = HD_ENOMEM;
    return nullptr;
  }
  k_cl_table_fp64<<<(entries + 255) / 256, 256, 0, bs>>>(p, R3, entries);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(bs) != cudaSuccess) {
    cudaFree(p);
    *err = HD_ECUDA;
    return nullptr;
  }
  tabs[-(int64_t)n] = p;
  return p;
}

const float2* TableCache::get(int64_t N, cudaStream_t /*st*/, hd_status* err) {
  auto it = tabs.find(N);
  if (it != tabs.end()) return it->second;
  cudaStream_t bs = build_stream(err);
  if (!bs) return nullptr;
  float2* p = nullptr;
  if (cudaMalloc(&p, sizeof(float2) * (size_t)N) != cudaSuccess) {
    *err = HD_ENOMEM;
    return nullptr;
  }
  int threads = 256;
  int64_t blocks64 = (N + threads - 1) / threads;
  int blocks = (int)(blocks64 < 4096 ? blocks64 : 4096);
  k_roots_fp64<<<blocks, threads, 0, bs>>>(p, N);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(bs) != cudaSuccess) {
    cudaFree(p);
    *err = HD_ECUDA;
    return nullptr;
  }
  tabs[N] = p;
  return p;
}

void TableCache::clear() {
  for (auto& kv : tabs) cudaFree(kv.second);
  tabs.clear();
  if (build) cudaStreamDestroy(build);
  build = nullptr;
}

// Radix sequence for a DFT of length n: radix 16, 8, 4, 2 for the power of
// two, then 5 and 3, then any remaining prime as a generic stage.
bool factor_radices(int n, FftPlan* out) {
  if (n < 1) return false;
  std::memset(out, 0, sizeof(*out));
  out->n = n;
  int v = n, k = 0;
  auto push = [&](int r) {
    if (k >= kMaxStages) return false;
    out->radix[k++] = r;
    return true;
  };
  while (v % 16 == 0) { if (!push(16)) return false; v /= 16; }
  if (v % 8 == 0) { if (!push(8)) return false; v /= 8; }
  if (v % 4 == 0) { if (!push(4)) return false; v /= 4; }
  if (v % 2 == 0) { if (!push(2)) return false; v /= 2; }
  while (v % 5 == 0) { if (!push(5)) return false; v /= 5; }
  while (v % 3 == 0) { if (!push(3)) return false; v /= 3; }
  for (int pr = 7; v > 1; pr += 2) {
    while (v % pr == 0) { if (!push(pr)) return false; v /= pr; }
    if ((int64_t)pr * pr > v && v > 1) { if (!push(v)) return false; v = 1; }
  }
  out->nst = k;
  return true;
}

bool smooth235(int64_t n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

int64_t next_smooth(int64_t n) {
  if (n < 1) n = 1;
  while (!smooth235(n)) ++n;
  return n;
}

// Smallest length {1, 3, 5, 9} x 2^a >= n: every such length factors into the
// register radices 16/8/4/2 and one of 3, 5, 9 (the structured FFT engine).
int64_t ladder_ceil(int64_t n) {
  if (n < 1) n = 1;
  int64_t best = INT64_MAX;
  for (int64_t base : {1, 3, 5, 9}) {
    int64_t x = base;
    while (x < n) x *= 2;
    best = std::min(best, x);
  }
  return best;
}

// Raise a kernel's dynamic shared-memory limit to at least `smem` on the
// current device, once: the limit is a per-device property of the function,
// so later launches of the same size skip the driver call.
cudaError_t smem_optin(const void* fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = set[{dev, fn}];
  if (cur >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) cur = smem;
  return e;
}

// Grow the context's scratch to `bytes`, stream-ordered on `st`: the old area
// is released after the work already queued on `st` and the new one is ready
// for what follows, with no device synchronisation.
hd_status ensure_ws(hd_ctx* c, size_t bytes, cudaStream_t st) {
  if (bytes <= c->ws_bytes) return HD_OK;
  if (c->ws) cudaFreeAsync(c->ws, st);
  c->ws = nullptr;
  c->ws_bytes = 0;
  if (cudaMallocAsync(&c->ws, bytes, st) != cudaSuccess) return HD_ENOMEM;
  c->ws_bytes = bytes;
  return HD_OK;
}

}  // namespace hd

namespace hd {
// Fill tw[0..N) with zeta_N^k on `st` (the same FP64 evaluation as the cache).
cudaError_t launch_roots_fp64(float2* tw, int64_t N, cudaStream_t st) {
  int threads = 256;
  int64_t blocks64 = (N + threads - 1) / threads;
  int blocks = (int)(blocks64 < 4096 ? blocks64 : 4096);
  k_roots_fp64<<<blocks, threads, 0, st>>>(tw, N);
  return cudaGetLastError();
}
}  // namespace hd
