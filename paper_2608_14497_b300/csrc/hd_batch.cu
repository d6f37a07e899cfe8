// hd_batch.cu -- batched 1D convolutions of uneven lengths.
//
// The plan is built once on the host: for every item the planner resolves the
// hybrid parameters (m, q) of Sec. 2 for its length (the role of the paper's
// empirical scan over m, Sec. 6), distinct DFT lengths share one radix plan,
// distinct padded lengths N = qm share one twiddle table, and items are grouped
// into one launch (block size and shared memory of the largest item), ordered
// longest first so the block scheduler balances the tail.  hybridRCM lengths
// the cluster kernel covers form one class per built instance (cluster size
// C, residue length m); the classes of one C run back to back on one stream,
// the streams of the different C concurrently, forked from the caller's
// stream and joined back (8-CTA clusters pack into the GPCs less densely than
// smaller ones, so the smaller clusters fill the SMs the C = 8 class cannot
// use; the C = 8 stream runs at the higher priority).  Everything the kernels read (item
// table, radix plans, tables, accumulator scratch) is uploaded or allocated
// here, so a launch of the plan performs no allocation and no host-to-device
// copy and can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "hd_cluster.cuh"
#include "hd_conv1d.cuh"
#include "hd_internal.h"

namespace hd {
struct LaunchClass {
  int first = 0, count = 0;  // range in the device item table
  int threads = 0;
  size_t smem = 0;
};
struct ClusterClass {
  int first = 0, count = 0;  // range in the device cluster item table
  int C = 0, m = 0;
  int stream = 0;            // index of the side stream (one per cluster size)
};
constexpr int kMaxClusterStreams = 5;  // C in {16, 8, 4, 2, 1}
}  // namespace hd

struct hd_batch_plan {
  hd_algo algo;
  int n = 0;
  int device = 0;
  hd::Item1D* d_items = nullptr;
  hd::FftPlan* d_plans = nullptr;
  void* d_acc = nullptr;
  std::vector<hd::LaunchClass> classes;
  int64_t total_len = 0;
  // cluster path (hybridRCM): one class per cluster size, concurrent streams
  hd::CItem* d_citems = nullptr;
  int64_t d_citems_count = 0;
  std::vector<hd::ClusterClass> cclasses;
  int nstreams = 0;
  cudaStream_t side[hd::kMaxClusterStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[hd::kMaxClusterStreams] = {};
  // explicit-padding baseline: zero-padded copies of f and g (item i at 2 off_i)
  bool exp = false;
  float* d_pad = nullptr;
  int64_t pad_floats = 0;  // per array
  int Lmax = 0;
};

using namespace hd;

extern "C" hd_status hd_batch_plan_create(hd_ctx* c, hd_algo algo, int32_t n, const int64_t* offsets,
                                          const int32_t* Ls, hd_batch_plan** out) {
  if (!c || !offsets || !Ls || !out || n < 1) return HD_EINVAL;
  if (algo != HD_HYBRID_RCM && algo != HD_HYBRID_CS && algo != HD_HYBRID_CSRCM && algo != HD_EXPLICIT_RCM)
    return HD_EUNSUPPORTED;
  const bool exp = (algo == HD_EXPLICIT_RCM);
  cudaSetDevice(c->device);
  struct HostItem {
    Item1D it;
    Params1D P;
    int64_t acc_bytes;
  };
  std::vector<HostItem> hs;
  hs.reserve(n);
  std::vector<FftPlan> plans;
  std::map<int, int> plan_of;
  auto plan_index = [&](int len) {
    auto f = plan_of.find(len);
    if (f != plan_of.end()) return f->second;
    FftPlan p;
    factor_radices(len, &p);
    plans.push_back(p);
    return plan_of[len] = (int)plans.size() - 1;
  };
  int64_t acc_total = 0;
  for (int i = 0; i < n; ++i)
    if (Ls[i] < 1 || offsets[i] < 0) return HD_EINVAL;
  // hybridRCM: every length the cluster kernel covers goes there
  std::vector<CItem> citems;
  std::vector<char> in_cluster(n, 0);
  if (algo == HD_HYBRID_RCM || exp) {
    // autotune the cluster kernel once per context (HD_AUTOTUNE=0 disables
    // it); the explicit-padding baseline takes the rule (no C = 16 instances)
    const char* at = getenv("HD_AUTOTUNE");
    if (!exp && !c->tuning.valid && !(at && at[0] == '0')) {
      hd_status ts = cluster_autotune(c, &c->tuning);
      if (ts != HD_OK) c->tuning.valid = false;
    }
    for (int i = 0; i < n; ++i) {
      int C, m, p;
      if (!cluster_params(Ls[i], &C, &m, &p, exp ? nullptr : &c->tuning) || (exp && C > 8)) {
        if (exp) return HD_EUNSUPPORTED;  // the explicit baseline covers L <= 73728
        continue;
      }
      hd_status terr = HD_OK;
      const float2* tw = c->tables.get((int64_t)2 * C * m, 0, &terr);
      if (!tw) return terr;
      CItem ci;
      std::memset(&ci, 0, sizeof(ci));
      ci.off = offsets[i];
      ci.off_in = 2 * offsets[i];
      ci.L = Ls[i];
      ci.m = m;
      ci.p = p;
      ci.C = C;
      ci.tw = tw;
      ci.tabm = c->tables.get_pass_table(m, 0, &terr);
      if (!ci.tabm) return terr;
      citems.push_back(ci);
      in_cluster[i] = 1;
    }
  }
  for (int i = 0; i < n; ++i) {
    if (in_cluster[i]) continue;
    Params1D P;
    hd_status s = (algo == HD_HYBRID_RCM) ? resolve_rcm1d(c, Ls[i], nullptr, &P) : resolve_cs1d(c, Ls[i], nullptr, &P);
    if (s != HD_OK) return s;
    hd_status terr = HD_OK;
    const float2* tw = c->tables.get((int64_t)P.q * P.m, 0, &terr);
    if (!tw) return terr;
    Item1D it;
    std::memset(&it, 0, sizeof(it));
    it.off = offsets[i];
    it.L = Ls[i];
    it.m = P.m;
    it.q = P.q;
    it.p = P.p;
    it.plan = plan_index(P.m);
    it.plan_half = (P.m % 2 == 0) ? plan_index(P.m / 2) : -1;
    it.tw = tw;
    int64_t accb = 0;
    if (P.gacc) {
      accb = (algo == HD_HYBRID_RCM) ? (int64_t)sizeof(float2) * ((Ls[i] + 1) / 2) : (int64_t)sizeof(float) * Ls[i];
      accb = (accb + 255) & ~(int64_t)255;
    }
    hs.push_back({it, P, accb});
    acc_total += accb;
  }
  const int ng = (int)hs.size();
  // Items the cluster kernel does not cover: one launch, longest first.
  std::stable_sort(hs.begin(), hs.end(), [](const HostItem& a, const HostItem& b) { return a.it.L > b.it.L; });
  hd_batch_plan* bp = new hd_batch_plan();
  bp->algo = algo;
  bp->exp = exp;
  bp->n = n;
  bp->device = c->device;
  if (acc_total > 0 && cudaMalloc(&bp->d_acc, acc_total) != cudaSuccess) {
    delete bp;
    return HD_ENOMEM;
  }
  int64_t acc_off = 0;
  std::vector<Item1D> items(ng);
  for (int i = 0; i < ng; ++i) {
    items[i] = hs[i].it;
    if (hs[i].acc_bytes) {
      items[i].gacc = (char*)bp->d_acc + acc_off;
      acc_off += hs[i].acc_bytes;
    }
    bp->total_len += hs[i].it.L;
    if (bp->classes.empty()) bp->classes.push_back(LaunchClass());
    LaunchClass& lc = bp->classes.back();
    lc.count++;
    lc.threads = std::max(lc.threads, hs[i].P.threads);
    lc.smem = std::max(lc.smem, hs[i].P.smem);
  }
  // cluster classes: by C (largest first), then m (largest first); lengths
  // descending within a class; one side stream per C
  if (!citems.empty()) {
    std::stable_sort(citems.begin(), citems.end(), [](const CItem& a, const CItem& b) {
      if (a.C != b.C) return a.C > b.C;
      if (a.m != b.m) return a.m > b.m;
      return a.L > b.L;
    });
    for (size_t i = 0; i < citems.size(); ++i) {
      if (bp->cclasses.empty() || bp->cclasses.back().C != citems[i].C || bp->cclasses.back().m != citems[i].m) {
        ClusterClass k;
        k.first = (int)i;
        k.C = citems[i].C;
        k.m = citems[i].m;
        k.stream = bp->cclasses.empty() ? 0
                   : bp->cclasses.back().stream + (bp->cclasses.back().C != citems[i].C ? 1 : 0);
        bp->cclasses.push_back(k);
      }
      ClusterClass& k = bp->cclasses.back();
      ++k.count;
      bp->total_len += citems[i].L;
    }
    bp->nstreams = bp->cclasses.back().stream + 1;
    if (exp) {
      int64_t extent = 0;
      for (const CItem& ci : citems) {
        extent = std::max<int64_t>(extent, ci.off + ci.L);
        bp->Lmax = std::max(bp->Lmax, ci.L);
      }
      bp->pad_floats = 2 * extent;
      if (cudaMalloc(&bp->d_pad, sizeof(float) * 2 * (size_t)bp->pad_floats) != cudaSuccess) {
        hd_batch_plan_destroy(bp);
        return HD_ENOMEM;
      }
    }
    if (cudaMalloc(&bp->d_citems, sizeof(CItem) * citems.size()) != cudaSuccess) {
      hd_batch_plan_destroy(bp);
      return HD_ENOMEM;
    }
    cudaMemcpy(bp->d_citems, citems.data(), sizeof(CItem) * citems.size(), cudaMemcpyHostToDevice);
    bp->d_citems_count = (int64_t)citems.size();
    if (bp->nstreams > 1) {
      int lo = 0, hi = 0;
      cudaDeviceGetStreamPriorityRange(&lo, &hi);
      bool ok = cudaEventCreateWithFlags(&bp->fork, cudaEventDisableTiming) == cudaSuccess;
      for (int k = 0; k < bp->nstreams && ok; ++k) {
        ok = cudaStreamCreateWithPriority(&bp->side[k], cudaStreamNonBlocking, k == 0 ? hi : lo) == cudaSuccess &&
             cudaEventCreateWithFlags(&bp->join[k], cudaEventDisableTiming) == cudaSuccess;
      }
      if (!ok) {
        hd_batch_plan_destroy(bp);
        return HD_ECUDA;
      }
    }
  }
  if ((ng > 0 && cudaMalloc(&bp->d_items, sizeof(Item1D) * ng) != cudaSuccess) ||
      cudaMalloc(&bp->d_plans, sizeof(FftPlan) * std::max<size_t>(1, plans.size())) != cudaSuccess) {
    hd_batch_plan_destroy(bp);
    return HD_ENOMEM;
  }
  if (ng > 0) cudaMemcpy(bp->d_items, items.data(), sizeof(Item1D) * ng, cudaMemcpyHostToDevice);
  if (!plans.empty()) cudaMemcpy(bp->d_plans, plans.data(), sizeof(FftPlan) * plans.size(), cudaMemcpyHostToDevice);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    hd_batch_plan_destroy(bp);
    return HD_ECUDA;
  }
  *out = bp;
  return HD_OK;
}

extern "C" hd_status hd_batch_plan_destroy(hd_batch_plan* bp) {
  if (!bp) return HD_OK;
  cudaSetDevice(bp->device);
  cudaDeviceSynchronize();
  if (bp->d_items) cudaFree(bp->d_items);
  if (bp->d_plans) cudaFree(bp->d_plans);
  if (bp->d_acc) cudaFree(bp->d_acc);
  if (bp->d_citems) cudaFree(bp->d_citems);
  if (bp->d_pad) cudaFree(bp->d_pad);
  for (int k = 0; k < kMaxClusterStreams; ++k) {
    if (bp->side[k]) cudaStreamDestroy(bp->side[k]);
    if (bp->join[k]) cudaEventDestroy(bp->join[k]);
  }
  if (bp->fork) cudaEventDestroy(bp->fork);
  delete bp;
  return HD_OK;
}

extern "C" hd_status hd_conv1d_batched(hd_ctx* c, const hd_batch_plan* bp, const float* f, const float* g, float* h,
                                       void* stream) {
  if (!c || !bp || !f || !g || !h) return HD_EINVAL;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int ncc = (int)bp->cclasses.size();
  if (bp->exp) {
    // explicit padding materialised in memory first
    float* pf = bp->d_pad;
    float* pg = bp->d_pad + bp->pad_floats;
    if (launch_pad_items(bp->d_citems, (int)bp->d_citems_count, bp->Lmax, f, g, pf, pg, st) != cudaSuccess)
      return HD_ECUDA;
    f = pf;
    g = pg;
  }
  if (bp->nstreams == 1) {
    for (int i = 0; i < ncc; ++i) {
      const ClusterClass& k = bp->cclasses[i];
      ClusterLaunch cl;
      std::memset(&cl, 0, sizeof(cl));
      cl.items = bp->d_citems + k.first;
      cl.err = c->dev_err;
      if (launch_rcm1d_cluster(cl, k.C, k.m, k.count, f, g, h, st, bp->exp) != cudaSuccess) return HD_ECUDA;
    }
  } else if (bp->nstreams > 1) {
    // fork: every cluster size on its own stream after the work already on
    // `st`; join back
    if (cudaEventRecord(bp->fork, st) != cudaSuccess) return HD_ECUDA;
    for (int s2 = 0; s2 < bp->nstreams; ++s2)
      if (cudaStreamWaitEvent(bp->side[s2], bp->fork, 0) != cudaSuccess) return HD_ECUDA;
    for (int i = 0; i < ncc; ++i) {
      const ClusterClass& k = bp->cclasses[i];
      ClusterLaunch cl;
      std::memset(&cl, 0, sizeof(cl));
      cl.items = bp->d_citems + k.first;
      cl.err = c->dev_err;
      if (launch_rcm1d_cluster(cl, k.C, k.m, k.count, f, g, h, bp->side[k.stream], bp->exp) != cudaSuccess) return HD_ECUDA;
    }
    for (int s2 = 0; s2 < bp->nstreams; ++s2)
      if (cudaEventRecord(bp->join[s2], bp->side[s2]) != cudaSuccess ||
          cudaStreamWaitEvent(st, bp->join[s2], 0) != cudaSuccess)
        return HD_ECUDA;
  }
  for (const LaunchClass& lc : bp->classes) {
    Launch1D la;
    std::memset(&la, 0, sizeof(la));
    la.items = bp->d_items + lc.first;
    la.plans = bp->d_plans;
    cudaError_t e = (bp->algo == HD_HYBRID_RCM) ? launch_rcm1d(la, lc.count, lc.threads, lc.smem, f, g, h, st)
                                                : launch_cs1d(la, lc.count, lc.threads, lc.smem, f, g, h, st,
                                                              bp->algo == HD_HYBRID_CSRCM);
    if (e != cudaSuccess) return HD_ECUDA;
  }
  return HD_OK;
}

extern "C" hd_status hd_batch_plan_launches(const hd_batch_plan* bp, int32_t* n) {
  if (!bp || !n) return HD_EINVAL;
  *n = (int32_t)(bp->cclasses.size() + bp->classes.size());
  return HD_OK;
}

extern "C" hd_status hd_tuning_table(hd_ctx* c, int32_t cap, int32_t* C, int32_t* m, double* us, int32_t* n) {
  if (!c || !n || cap < 0 || (cap > 0 && (!C || !m || !us))) return HD_EINVAL;
  const ClusterTuning& t = c->tuning;
  *n = t.valid ? (int32_t)t.us.size() : 0;
  for (int32_t i = 0; i < *n && i < cap; ++i) {
    C[i] = t.C[i];
    m[i] = t.m[i];
    us[i] = t.us[i];
  }
  return HD_OK;
}
