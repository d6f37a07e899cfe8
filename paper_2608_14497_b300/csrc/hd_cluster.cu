// hd_cluster.cu -- host side of the cluster hybridRCM kernel (the fast path
// of the batched and single 1D calls; the kernel is in hd_cl_kernel.cuh and
// hd_cl_launch.cuh): the built instances (C, m), the parameter choice per
// length, the autotuner and the launch dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "hd_cluster.cuh"

namespace hd {

// Built instances: m = 256 R3.  One CTA covers L <= 2 m; a cluster of C CTAs
// covers L <= 2 C m.  Up to R3 = 10 two or more CTAs fit on an SM (shared
// memory 32 m + 8 (m - 16) bytes), so for long items the planner may trade a
// larger cluster for CTAs that overlap on the SMs; the autotuner decides.
static const int kR3One[] = {1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 16, 18};
static const int kR3Two[] = {10, 12, 16, 18};
static const int kR3Four[] = {5, 6, 8, 9, 10, 12, 16, 18};
static const int kR3Eight[] = {5, 6, 8, 9, 10, 12, 16, 18};
static const int kR3Sixteen[] = {5, 6, 8, 9};

template <size_t N>
static bool has(const int (&v)[N], int x) {
  return std::find(std::begin(v), std::end(v), x) != std::end(v);
}

bool cluster_instance(int C, int m) {
  if (m % 256) return false;
  const int R3 = m / 256;
  switch (C) {
    case 1: return has(kR3One, R3);
    case 2: return has(kR3Two, R3);
    case 4: return has(kR3Four, R3);
    case 8: return has(kR3Eight, R3);
    case 16: return has(kR3Sixteen, R3);
  }
  return false;
}

// Every built (C, m), in increasing m per C.
static std::vector<std::pair<int, int>> instances() {
  std::vector<std::pair<int, int>> v;
  for (int r : kR3One) v.push_back({1, 256 * r});
  for (int r : kR3Two) v.push_back({2, 256 * r});
  for (int r : kR3Four) v.push_back({4, 256 * r});
  for (int r : kR3Eight) v.push_back({8, 256 * r});
  for (int r : kR3Sixteen) v.push_back({16, 256 * r});
  return v;
}

bool cluster_params(int64_t L, int* C_out, int* m_out, int* p_out, const ClusterTuning* tun) {
  if (L < 1) return false;
  const int64_t Lp = (L + 1) / 2;
  if (tun && tun->valid) {
    // the cheapest measured instance whose padded length 2 C m covers L
    double best = 1e300;
    for (size_t i = 0; i < tun->C.size(); ++i) {
      const int C = tun->C[i], mm = tun->m[i];
      if ((int64_t)2 * C * mm < L || !cluster_instance(C, mm)) continue;
      if (tun->us[i] < best) {
        best = tun->us[i];
        *C_out = C;
        *m_out = mm;
        *p_out = (int)((Lp + mm - 1) / mm);
      }
    }
    if (best < 1e300) return true;
  }
  for (const auto& cm : instances()) {
    if ((int64_t)2 * cm.first * cm.second >= L) {
      *C_out = cm.first;
      *m_out = cm.second;
      *p_out = (int)((Lp + cm.second - 1) / cm.second);
      return true;
    }
  }
  return false;
}

// One convolution per call: the built instance with the smallest modelled time
// a_C + b_C m.  A call is one cluster, so its time is latency: a per-call cost
// a_C (launch, cluster set-up and the exchanges between the C CTAs) and a cost
// b_C per point of the C CTAs' m-point transforms, fitted to CUDA-graph
// timings of single calls on a B300 (L = 10^3 ... 65536; e.g. L = 16384:
// 18.9 us at (C, m) = (2, 4096), the first instance that fits, 11.0 us at
// (8, 1280)).  Small L stays on one CTA, whose a_1 has no exchange.
bool cluster_params_single(int64_t L, int* C_out, int* m_out, int* p_out) {
  if (L < 1) return false;
  struct Cost {
    int C;
    double a_us, b_us;
  };
  static const Cost model[] = {{1, 5.5, 1.5e-3}, {2, 5.3, 3.3e-3}, {4, 7.4, 2.1e-3}, {8, 6.8, 3.3e-3},
                               {16, 8.3, 2.9e-3}};
  const int64_t Lp = (L + 1) / 2;
  double best = 1e300;
  for (const auto& cm : instances()) {
    if ((int64_t)2 * cm.first * cm.second < L) continue;
    for (const Cost& k : model) {
      if (k.C != cm.first) continue;
      const double t = k.a_us + k.b_us * cm.second;
      if (t < best) {
        best = t;
        *C_out = cm.first;
        *m_out = cm.second;
        *p_out = (int)((Lp + cm.second - 1) / cm.second);
      }
    }
  }
  return best < 1e300;
}

hd_status cluster_autotune(hd_ctx* c, ClusterTuning* out) {
  const std::vector<std::pair<int, int>> cand = instances();
  const int64_t budget = int64_t{1} << 22;  // real elements per timed batch
  float *f = nullptr, *g = nullptr, *h = nullptr;
  CItem* d_items = nullptr;
  hd_status st = HD_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&f, sizeof(float) * budget) != cudaSuccess || cudaMalloc(&g, sizeof(float) * budget) != cudaSuccess ||
      cudaMalloc(&h, sizeof(float) * budget) != cudaSuccess ||
      cudaMalloc(&d_items, sizeof(CItem) * 16384) != cudaSuccess) {
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
  for (size_t i = 0; i < cand.size() && st == HD_OK; ++i) {
    const int C = cand[i].first, mm = cand[i].second;
    const int64_t L = (int64_t)2 * C * mm;
    const int64_t K = std::max<int64_t>(1, std::min<int64_t>(budget / L, 16384));
    hd_status terr = HD_OK;
    const float2* tw = c->tables.get(L, 0, &terr);
    const float2* tabm = tw ? c->tables.get_pass_table(mm, 0, &terr) : nullptr;
    if (!tw || !tabm) {
      st = terr;
      break;
    }
    std::vector<CItem> items(K);
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
    cudaMemcpy(d_items, items.data(), sizeof(CItem) * K, cudaMemcpyHostToDevice);
    ClusterLaunch cl;
    std::memset(&cl, 0, sizeof(cl));
    cl.items = d_items;
    cl.err = c->dev_err;
    if (launch_rcm1d_cluster(cl, C, mm, (int)K, f, g, h, 0) != cudaSuccess) {
      st = HD_ECUDA;
      break;
    }
    // best of three trials of two launches each (one noisy trial must not
    // steer the plan)
    float best_ms = 1e30f;
    for (int trial = 0; trial < 3 && st == HD_OK; ++trial) {
      cudaEventRecord(e0, 0);
      for (int rep = 0; rep < 2; ++rep) launch_rcm1d_cluster(cl, C, mm, (int)K, f, g, h, 0);
      cudaEventRecord(e1, 0);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = HD_ECUDA;
        break;
      }
      float ms_el = 0.f;
      cudaEventElapsedTime(&ms_el, e0, e1);
      best_ms = std::min(best_ms, ms_el);
    }
    if (st != HD_OK) break;
    out->C.push_back(C);
    out->m.push_back(mm);
    out->us.push_back(1e3 * best_ms / (2.0 * (double)K));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(f);
  cudaFree(g);
  cudaFree(h);
  cudaFree(d_items);
  out->valid = (st == HD_OK) && !out->us.empty();
  return st;
}

cudaError_t launch_rcm1d_cluster(const ClusterLaunch& cl, int C, int m, int nitems, const float* f, const float* g,
                                 float* h, cudaStream_t st, bool exp) {
  if (!cluster_instance(C, m) || nitems < 1) return cudaErrorInvalidValue;
  const int R3 = m / 256;
  if (exp) {
    switch (C) {
      case 1: return R3 <= 6 ? launch_clx_c1(R3, cl, nitems, f, g, h, st) : launch_clx_c1b(R3, cl, nitems, f, g, h, st);
      case 2: return launch_clx_c2(R3, cl, nitems, f, g, h, st);
      case 4: return R3 <= 9 ? launch_clx_c4(R3, cl, nitems, f, g, h, st) : launch_clx_c4b(R3, cl, nitems, f, g, h, st);
      case 8: return R3 <= 9 ? launch_clx_c8(R3, cl, nitems, f, g, h, st) : launch_clx_c8b(R3, cl, nitems, f, g, h, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (C) {
    case 1: return R3 <= 6 ? launch_cl_c1(R3, cl, nitems, f, g, h, st) : launch_cl_c1b(R3, cl, nitems, f, g, h, st);
    case 2: return launch_cl_c2(R3, cl, nitems, f, g, h, st);
    case 4: return R3 <= 9 ? launch_cl_c4(R3, cl, nitems, f, g, h, st) : launch_cl_c4b(R3, cl, nitems, f, g, h, st);
    case 8: return R3 <= 9 ? launch_cl_c8(R3, cl, nitems, f, g, h, st) : launch_cl_c8b(R3, cl, nitems, f, g, h, st);
    case 16: return launch_cl_c16(R3, cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}

// Zero-padded copies for the explicit-padding baseline: item i's L values at
// off become [values, L zeros] at off_in (grid: x over 2 Lmax, y over items).
__global__ void k_pad_items(const CItem* __restrict__ items, const float* __restrict__ f, const float* __restrict__ g,
                            float* __restrict__ pf, float* __restrict__ pg) {
  const CItem it = items[blockIdx.y];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 2 * (int64_t)it.L;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool in = k < it.L;
    pf[it.off_in + k] = in ? f[it.off + k] : 0.f;
    pg[it.off_in + k] = in ? g[it.off + k] : 0.f;
  }
}

__global__ void k_pad_one(int64_t L, int64_t total, const float* __restrict__ f, const float* __restrict__ g,
                          float* __restrict__ pf, float* __restrict__ pg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t item = i / (2 * L), k = i - item * 2 * L;
    const bool in = k < L;
    pf[i] = in ? f[item * L + k] : 0.f;
    pg[i] = in ? g[item * L + k] : 0.f;
  }
}

cudaError_t launch_pad_items(const CItem* items, int nitems, int Lmax, const float* f, const float* g, float* pf,
                             float* pg, cudaStream_t st) {
  const int bx = std::max(1, std::min(64, (2 * Lmax + 1023) / 1024));
  for (int first = 0; first < nitems; first += 65535) {
    const int n = std::min(65535, nitems - first);
    k_pad_items<<<dim3(bx, n), 256, 0, st>>>(items + first, f, g, pf, pg);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_pad_one(int64_t L, int64_t batch, const float* f, const float* g, float* pf, float* pg,
                           cudaStream_t st) {
  const int64_t total = 2 * L * batch;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
  k_pad_one<<<blocks, 256, 0, st>>>(L, total, f, g, pf, pg);
  return cudaGetLastError();
}

}  // namespace hd
