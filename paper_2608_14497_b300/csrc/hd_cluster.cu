// hd_cluster.cu -- host side of the cluster hybridRCM kernel (the fast path
// of the batched and single 1D calls; the kernel is in hd_cluster_kernel.cuh):
// the ladder of residue DFT lengths, the parameter choice per length, the
// autotuner and the launch dispatch over cluster sizes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "hd_cluster.cuh"

namespace hd {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Candidate DFT lengths: {1, 3, 5, 9} x 2^a with a >= 4 (the lengths of the
// structured engine, cta_fft_struct) up to the cap (few distinct lengths, so
// twiddle tables are shared across a batch and stay in L2).
static const std::vector<int>& ladder() {
  static std::vector<int> v;
  if (v.empty()) {
    for (int base : {1, 3, 5, 9})
      for (int x = 16 * base; x <= kClusterMaxM; x *= 2) v.push_back(x);
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
  CItem* d_items = nullptr;
  hd_status st = HD_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&f, sizeof(float) * budget) != cudaSuccess || cudaMalloc(&g, sizeof(float) * budget) != cudaSuccess ||
      cudaMalloc(&h, sizeof(float) * budget) != cudaSuccess ||
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
    const int64_t K = std::max<int64_t>(1, std::min<int64_t>(budget / L, 4096));
    if (K * L > budget) continue;
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
    const size_t smem = cluster_smem_bytes(mm);
    if (launch_rcm1d_cluster(cl, C, (int)K, smem, f, g, h, 0) != cudaSuccess) {
      st = HD_ECUDA;
      break;
    }
    // best of three trials of two launches each (one noisy trial must not
    // steer the plan)
    float best_ms = 1e30f;
    for (int trial = 0; trial < 3 && st == HD_OK; ++trial) {
      cudaEventRecord(e0, 0);
      for (int rep = 0; rep < 2; ++rep) launch_rcm1d_cluster(cl, C, (int)K, smem, f, g, h, 0);
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

size_t cluster_smem_bytes(int m_max) { return sizeof(float2) * 5 * (size_t)swz_stride(m_max); }

cudaError_t launch_rcm1d_cluster(const ClusterLaunch& cl, int C, int nitems, size_t smem, const float* f,
                                 const float* g, float* h, cudaStream_t st) {
  switch (C) {
    case 1: return launch_cluster_c1(cl, nitems, smem, f, g, h, st);
    case 2: return launch_cluster_c2(cl, nitems, smem, f, g, h, st);
    case 4: return launch_cluster_c4(cl, nitems, smem, f, g, h, st);
    case 8: return launch_cluster_c8(cl, nitems, smem, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hd
