// hd_api.cu -- the C ABI of libhdconv.so (declared in include/hdconv.h):
// argument validation, the planner that picks the hybrid parameters (m, q) of
// Sec. 2 for a length, and dispatch to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "hd_cluster.cuh"
#include "hd_conv1d.cuh"
#include "hd_internal.h"
#include "hd_nd.cuh"

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace hd {
hd_status fail(hd_status s, const char* what) {
  g_last_error = what;
  return s;
}

hd_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return HD_ECUDA;
}
}  // namespace hd

namespace hd {

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// hybridCS in 1D without (m, q) from the caller: a single call (one
// convolution) runs the three-kernel path (App. A) from kCsSingleStaged on,
// its q residues on q/2 + 1 SMs instead of one CTA (L = 4096: 39 -> 10 us),
// and one CTA (q = 2) below; an equal-length batch always runs the three
// kernels over the whole batch (2048 items of L = 4096: 29 ms one CTA after
// another -> 1.0 ms).
constexpr int64_t kCsSingleStaged = 512;

static int64_t next_smooth_even(int64_t n) {
  int64_t m = next_smooth(n < 2 ? 2 : n);
  while (m % 2) m = next_smooth(m + 1);
  return m;
}

// hybridRCM: packed length Lp = ceil(L/2) must satisfy p m >= Lp (p =
// ceil(Lp/m)) and q m >= L (real padded length 2qm >= 2L-1).  The planner
// prefers p = 1, q = 2 (a single explicit block, residues 0 and 1, both
// self-paired) with the smallest 2,3,5-smooth m >= Lp; when 4m exceeds what one
// CTA transforms at once it lowers m and raises p and q.
hd_status resolve_rcm1d(hd_ctx* c, int64_t L, const hd_dim_params* prm, Params1D* out, int64_t K) {
  if (K <= 0) K = L;
  const int64_t Lp = ceil_div(L, 2);
  int64_t m, q;
  const int64_t mmax = (int64_t)kPts * 1024 / 4;
  if (prm && prm->m > 0) {
    m = prm->m;
    q = prm->q > 0 ? prm->q : ceil_div(L, m);
    if (q * m < L) return fail(HD_EINVAL, "hybridRCM needs q m >= L (packed)");
    if (m > mmax) return fail(HD_EUNSUPPORTED, "hybridRCM: m too large for one CTA (m <= 4096)");
  } else {
    m = next_smooth(Lp);
    q = 2;
    if (m > mmax) {
      for (int64_t k = 2;; ++k) {
        m = next_smooth(ceil_div(Lp, k));
        if (m <= mmax) break;
      }
      q = ceil_div(L, m);
    }
  }
  if (q * m > (int64_t)1 << 30) return fail(HD_EUNSUPPORTED, "padded length too large");
  out->m = (int)m;
  out->q = (int)q;
  out->p = (int)ceil_div(Lp, m);
  out->smem = rcm1d_smem_bytes((int)K, (int)m, false);
  out->gacc = out->smem > (size_t)c->max_smem;
  if (out->gacc) out->smem = rcm1d_smem_bytes((int)K, (int)m, true);
  if (out->smem > (size_t)c->max_smem) return fail(HD_EUNSUPPORTED, "hybridRCM: shared memory too small");
  out->threads = threads_for_points(4 * m, kPts);
  return HD_OK;
}

// hybridCS: real length L, q m >= 2L-1, m even when q is even (Sec. 3.1.3).
// The planner prefers q = 2 and the smallest even 2,3,5-smooth m >= L.
hd_status resolve_cs1d(hd_ctx* c, int64_t L, const hd_dim_params* prm, Params1D* out, int64_t K) {
  if (K <= 0) K = L;
  int64_t m, q;
  const int64_t mmax = (int64_t)kPts * 1024 / 2;
  if (prm && prm->m > 0) {
    m = prm->m;
    q = prm->q > 0 ? prm->q : ceil_div(2 * L - 1, m);
    if (q * m < 2 * L - 1) return fail(HD_EINVAL, "hybridCS needs q m >= 2L-1");
    if (q % 2 == 0 && m % 2 == 1) return fail(HD_EINVAL, "hybridCS needs m even when q is even");
    if (m > mmax) return fail(HD_EUNSUPPORTED, "hybridCS: m too large for one CTA (m <= 8192)");
  } else {
    m = next_smooth_even(L);
    q = 2;
    if (m > mmax) {
      for (int64_t k = 2;; ++k) {
        m = next_smooth_even(ceil_div(L, k));
        if (m <= mmax) break;
      }
      q = ceil_div(2 * L - 1, m);
      if (q % 2 == 1) ++q;  // keep q even so residue q/2 uses the half-length DFT
    }
  }
  if (q * m > (int64_t)1 << 30) return fail(HD_EUNSUPPORTED, "padded length too large");
  out->m = (int)m;
  out->q = (int)q;
  out->p = (int)ceil_div(L, m);
  out->smem = cs1d_smem_bytes((int)K, (int)m, false);
  out->gacc = out->smem > (size_t)c->max_smem;
  if (out->gacc) out->smem = cs1d_smem_bytes((int)K, (int)m, true);
  if (out->smem > (size_t)c->max_smem) return fail(HD_EUNSUPPORTED, "hybridCS: shared memory too small");
  out->threads = threads_for_points(2 * m, kPts);
  return HD_OK;
}

// hybridRCM with planner parameters: the cluster kernel, one item by value,
// repeated `batch` times at a stride of L floats.
static hd_status conv1d_rcm_cluster(hd_ctx* c, const float* f, const float* g, float* h, int64_t L, int C, int m,
                                    int p, cudaStream_t st, int64_t batch = 1, int64_t K = 0) {
  hd_status terr = HD_OK;
  const float2* tw = c->tables.get((int64_t)2 * C * m, st, &terr);
  if (!tw) return fail(terr, "twiddle table allocation failed");
  ClusterLaunch cl;
  std::memset(&cl, 0, sizeof(cl));
  cl.err = c->dev_err;
  cl.one_item.off = 0;
  cl.one_item.L = (int32_t)L;
  cl.one_item.m = m;
  cl.one_item.p = p;
  cl.one_item.C = C;
  cl.one_item.tw = tw;
  cl.one_item.tabm = c->tables.get_pass_table(m, st, &terr);
  if (!cl.one_item.tabm) return fail(terr, "pass table allocation failed");
  cl.one_item.K = (int32_t)K;
  cl.stride = L;
  if (K > 0 && K != L && batch > 1) return fail(HD_EINVAL, "batched calls return the first L outputs");
  cudaError_t e = launch_rcm1d_cluster(cl, C, m, (int)batch, f, g, h, st);
  if (e != cudaSuccess) return cuda_fail(e, "cluster launch");
  return HD_OK;
}

// The explicit-padding baseline on the same kernel: zero-padded copies of f
// and g (real length 2L per item, in scratch), every block read, the full
// q-point sums; `batch` items of length L back to back.
static hd_status conv1d_explicit_cluster(hd_ctx* c, const float* f, const float* g, float* h, int64_t L, int C, int m,
                                         int p, cudaStream_t st, int64_t batch = 1, int64_t K = 0) {
  hd_status terr = HD_OK;
  const float2* tw = c->tables.get((int64_t)2 * C * m, st, &terr);
  if (!tw) return fail(terr, "twiddle table allocation failed");
  const float2* tabm = c->tables.get_pass_table(m, st, &terr);
  if (!tabm) return fail(terr, "pass table allocation failed");
  if (ensure_ws(c, sizeof(float) * 4 * (size_t)L * (size_t)batch, st) != HD_OK)
    return fail(HD_ENOMEM, "workspace allocation failed");
  float* pf = reinterpret_cast<float*>(c->ws);
  float* pg = pf + 2 * L * batch;
  cudaError_t e = launch_pad_one(L, batch, f, g, pf, pg, st);
  if (e != cudaSuccess) return cuda_fail(e, "padding launch");
  ClusterLaunch cl;
  std::memset(&cl, 0, sizeof(cl));
  cl.err = c->dev_err;
  cl.one_item.L = (int32_t)L;
  cl.one_item.m = m;
  cl.one_item.p = p;
  cl.one_item.C = C;
  cl.one_item.tw = tw;
  cl.one_item.tabm = tabm;
  cl.one_item.K = (int32_t)K;
  cl.stride = L;
  if (K > 0 && K != L && batch > 1) return fail(HD_EINVAL, "batched calls return the first L outputs");
  e = launch_rcm1d_cluster(cl, C, m, (int)batch, pf, pg, h, st, true);
  if (e != cudaSuccess) return cuda_fail(e, "cluster launch");
  return HD_OK;
}

static hd_status conv1d_hybrid(hd_ctx* c, hd_algo algo, const float* f, const float* g, float* h, int64_t L,
                               const hd_dim_params* prm, cudaStream_t st, int64_t K) {
  if (algo == HD_HYBRID_RCM && !(prm && prm->m > 0)) {
    int C, m, p;
    if (cluster_params_single(L, &C, &m, &p)) return conv1d_rcm_cluster(c, f, g, h, L, C, m, p, st, 1, K);
    int M, q;
    if (staged_params(L, &M, &q)) return conv1d_staged(c, f, g, h, L, K, M, q, 1, st);
  }
  if (algo == HD_HYBRID_CS && !(prm && prm->m > 0) && L > kCsSingleStaged) {
    int M, q;
    if (staged_params(2 * L - 1, &M, &q)) return conv1d_staged(c, f, g, h, L, K, M, q, 1, st, true);
  }
  Params1D P;
  hd_status s = (algo == HD_HYBRID_RCM) ? resolve_rcm1d(c, L, prm, &P, K) : resolve_cs1d(c, L, prm, &P, K);
  if (s != HD_OK) return s;
  hd_status terr = HD_OK;
  const float2* tw = c->tables.get((int64_t)P.q * P.m, st, &terr);
  if (!tw) return fail(terr, "twiddle table allocation failed");
  Launch1D la;
  std::memset(&la, 0, sizeof(la));
  la.one.off = 0;
  la.one.L = (int32_t)L;
  la.one.m = P.m;
  la.one.q = P.q;
  la.one.p = P.p;
  la.one.plan = 0;
  la.one.plan_half = (P.m % 2 == 0) ? 1 : -1;
  la.one.K = (int32_t)K;
  la.one.tw = tw;
  factor_radices(P.m, &la.plan_m);
  if (P.m % 2 == 0) factor_radices(P.m / 2, &la.plan_half);
  if (P.gacc) {
    const size_t bytes = (algo == HD_HYBRID_RCM) ? sizeof(float2) * (size_t)ceil_div(K, 2) : sizeof(float) * (size_t)K;
    if (ensure_ws(c, bytes, st) != HD_OK) return fail(HD_ENOMEM, "workspace allocation failed");
    la.one.gacc = c->ws;
  }
  cudaError_t e = (algo == HD_HYBRID_RCM) ? launch_rcm1d(la, 1, P.threads, P.smem, f, g, h, st)
                                          : launch_cs1d(la, 1, P.threads, P.smem, f, g, h, st, algo == HD_HYBRID_CSRCM);
  if (e != cudaSuccess) return cuda_fail(e, "conv1d launch");
  return HD_OK;
}

}  // namespace hd

using namespace hd;

extern "C" {

const char* hd_strerror(hd_status s) {
  switch (s) {
    case HD_OK: return "ok";
    case HD_EINVAL: return "invalid argument";
    case HD_ENOMEM: return "out of memory";
    case HD_ECUDA: return "CUDA error";
    case HD_ETIMEOUT: return "device wait timed out";
    case HD_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* hd_last_error_string(void) { return g_last_error.c_str(); }

hd_status hd_create(hd_ctx** out, int device) {
  if (!out) return fail(HD_EINVAL, "null ctx pointer");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(HD_EINVAL, "no such device");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  hd_ctx* c = new hd_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  // keep a little room for the kernels' static shared memory (plans)
  c->max_smem -= 1024;
  e = cudaMalloc(&c->dev_err, sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc");
  }
  cudaMemset(c->dev_err, 0, sizeof(int));
  *out = c;
  return HD_OK;
}

hd_status hd_destroy(hd_ctx* c) {
  if (!c) return HD_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  c->tables.clear();
  if (c->ws) cudaFree(c->ws);
  if (c->ws2) cudaFree(c->ws2);
  if (c->dev_err) cudaFree(c->dev_err);
  delete c;
  return HD_OK;
}

hd_status hd_plan(hd_ctx* c, hd_algo algo, int64_t L, hd_dim_params* out) {
  if (!c || !out) return fail(HD_EINVAL, "null argument");
  if (L < 1) return fail(HD_EINVAL, "L < 1");
  Params1D P;
  hd_status s;
  switch (algo) {
    case HD_HYBRID_RCM: {
      int C, m, p;
      if (cluster_params_single(L, &C, &m, &p)) {
        out->m = m;
        out->q = 2 * C;
        return HD_OK;
      }
      int M, q;
      if (staged_params(L, &M, &q)) {
        out->m = M;
        out->q = q;
        return HD_OK;
      }
      s = resolve_rcm1d(c, L, nullptr, &P);
      break;
    }
    case HD_HYBRID_CS:
      if (L > kCsSingleStaged) {
        int M, q;
        if (staged_params(2 * L - 1, &M, &q)) {
          out->m = M;
          out->q = q;
          return HD_OK;
        }
      }
      s = resolve_cs1d(c, L, nullptr, &P);
      break;
    case HD_HYBRID_CSRCM: s = resolve_cs1d(c, L, nullptr, &P); break;
    default: return fail(HD_EINVAL, "hd_plan: hybrid algorithms only");
  }
  if (s != HD_OK) return s;
  out->m = P.m;
  out->q = P.q;
  return HD_OK;
}

hd_status hd_conv1d(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int64_t L,
                    const hd_dim_params* prm, void* stream) {
  return hd_conv_ext(c, algo, prec, 1, &L, nullptr, f, g, h, prm, stream);
}

hd_status hd_conv_batch(hd_ctx* c, hd_algo algo, hd_prec prec, int ndim, const int64_t* Ls, int32_t batch,
                        const float* f, const float* g, float* h, void* stream) {
  if (!c || !Ls || !f || !g || !h || ndim < 1 || ndim > 3 || batch < 1) return fail(HD_EINVAL, "null argument");
  int64_t n = 1;
  for (int i = 0; i < ndim; ++i) {
    if (Ls[i] < 1) return fail(HD_EINVAL, "L < 1");
    n *= Ls[i];
  }
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == HD_FP32 && algo == HD_HYBRID_RCM) {
    if (ndim >= 2) return conv_nd_batch_rcm(c, ndim, Ls, batch, f, g, h, st);
    // a batch whose clusters all fit in one wave is latency-bound like a single
    // call and takes the single-call choice (so each item equals its single-call
    // result bit for bit); larger batches take the throughput rule
    int C, m, p;
    bool cl = cluster_params_single(Ls[0], &C, &m, &p) && (int64_t)batch * C <= (int64_t)std::max(c->num_sms, 1);
    if (!cl) cl = batch < (1 << 24) && cluster_params(Ls[0], &C, &m, &p);
    if (cl) return conv1d_rcm_cluster(c, f, g, h, Ls[0], C, m, p, st, batch);
    int M, q;
    if (staged_params(Ls[0], &M, &q)) return conv1d_staged(c, f, g, h, Ls[0], Ls[0], M, q, batch, st);
  }
  if (prec == HD_FP32 && algo == HD_HYBRID_CS && ndim == 1) {
    int M, q;
    if (staged_params(2 * Ls[0] - 1, &M, &q))
      return conv1d_staged(c, f, g, h, Ls[0], Ls[0], M, q, batch, st, true);
  }
  if (prec == HD_FP32 && algo == HD_EXPLICIT_RCM && ndim == 1) {
    int C, m, p;
    if (batch < (1 << 24) && cluster_params(Ls[0], &C, &m, &p) && C <= 8)
      return conv1d_explicit_cluster(c, f, g, h, Ls[0], C, m, p, st, batch);
  }
  // every other case: one call per item
  for (int32_t b = 0; b < batch; ++b) {
    const int64_t o = (int64_t)b * n;
    hd_status s;
    if (ndim == 1) s = hd_conv1d(c, algo, prec, f + o, g + o, h + o, Ls[0], nullptr, stream);
    else if (ndim == 2) s = hd_conv2d(c, algo, prec, f + o, g + o, h + o, Ls[0], Ls[1], nullptr, stream);
    else s = hd_conv3d(c, algo, prec, f + o, g + o, h + o, Ls[0], Ls[1], Ls[2], nullptr, stream);
    if (s != HD_OK) return s;
  }
  return HD_OK;
}

hd_status hd_conv1d_staged(hd_ctx* c, hd_algo algo, int64_t L, int64_t K, int32_t M, int32_t q, int32_t batch,
                           const float* f, const float* g, float* h, void* stream) {
  if (!c || !f || !g || !h || batch < 1) return fail(HD_EINVAL, "staged path: null argument or batch < 1");
  if (algo != HD_HYBRID_RCM && algo != HD_HYBRID_CS) return fail(HD_EINVAL, "staged path: hybridRCM or hybridCS");
  const bool cs = (algo == HD_HYBRID_CS);
  if (L < 1 || L > ((int64_t)1 << 28)) return fail(HD_EINVAL, "staged path: L out of range");
  if (K == 0) K = L;
  if (K < L || K > 2 * L - 1) return fail(HD_EINVAL, "output extent K must satisfy L <= K <= 2L-1");
  const int64_t n_in = L * batch, n_out = K * batch;
  if (K != L && ((h < f + n_in && f < h + n_out) || (h < g + n_in && g < h + n_out)))
    return fail(HD_EINVAL, "h may alias f or g only when K = L");
  int Mx = M, qx = q;
  if (M == 0 && q == 0) {
    if (!staged_params(cs ? 2 * L - 1 : L, &Mx, &qx)) return fail(HD_EUNSUPPORTED, "staged path: L too large");
  } else if (M <= 0 || q <= 0) {
    return fail(HD_EINVAL, "staged path: give both M and q, or neither");
  }
  cudaSetDevice(c->device);
  return conv1d_staged(c, f, g, h, L, K, Mx, qx, batch, (cudaStream_t)stream, cs);
}

hd_status hd_conv1d_multi(hd_ctx* c, int32_t n, const float* const* x, const int64_t* L, int64_t K, int32_t M,
                          int32_t q, float* h, void* stream) {
  if (!c || !x || !L || !h) return fail(HD_EINVAL, "n-ary convolution: null argument");
  if (n < 2 || n > 16) return fail(HD_EINVAL, "n-ary convolution: 2 <= n <= 16 arrays");
  int64_t S = 1, Lmax = 0;
  for (int i = 0; i < n; ++i) {
    if (!x[i]) return fail(HD_EINVAL, "n-ary convolution: null array");
    if (L[i] < 1 || L[i] > ((int64_t)1 << 28)) return fail(HD_EINVAL, "n-ary convolution: L_i out of range");
    S += L[i] - 1;
    Lmax = L[i] > Lmax ? L[i] : Lmax;
  }
  if (K == 0) K = Lmax;
  if (K < 1 || K > S) return fail(HD_EINVAL, "n-ary convolution: K must satisfy 1 <= K <= sum L_i - n + 1");
  int Mx = M, qx = q;
  if (M == 0 && q == 0) {
    if (!staged_params((S + 1) / 2, &Mx, &qx)) return fail(HD_EUNSUPPORTED, "n-ary convolution: sum of lengths too large");
  } else if (M <= 0 || q <= 0) {
    return fail(HD_EINVAL, "n-ary convolution: give both M and q, or neither");
  }
  cudaSetDevice(c->device);
  return conv1d_multi(c, n, x, L, K, Mx, qx, h, (cudaStream_t)stream);
}

hd_status hd_conv_ext(hd_ctx* c, hd_algo algo, hd_prec prec, int ndim, const int64_t* L, const int64_t* K,
                      const float* f, const float* g, float* h, const hd_dim_params* prm, void* stream) {
  if (!c || !L || !f || !g || !h) return fail(HD_EINVAL, "null argument");
  if (ndim < 1 || ndim > 3) return fail(HD_EINVAL, "ndim must be 1, 2 or 3");
  int64_t Kx[3], n_in = 1, n_out = 1;
  bool full = false;
  for (int i = 0; i < ndim; ++i) {
    if (L[i] < 1) return fail(HD_EINVAL, "L < 1");
    Kx[i] = K ? K[i] : L[i];
    if (Kx[i] < L[i] || Kx[i] > 2 * L[i] - 1) return fail(HD_EINVAL, "output extent K must satisfy L <= K <= 2L-1");
    full = full || Kx[i] != L[i];
    n_in *= L[i];
    n_out *= Kx[i];
  }
  // a longer output is written while the inputs are still read
  if (full && ((h < f + n_in && f < h + n_out) || (h < g + n_in && g < h + n_out)))
    return fail(HD_EINVAL, "h may alias f or g only when K = L");
  if (prm)
    for (int i = 0; i < ndim; ++i)
      if (prm[i].m < 0 || prm[i].q < 0) return fail(HD_EINVAL, "negative m or q");
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (ndim > 1) return conv_nd_ext(c, algo, prec, f, g, h, ndim, L, Kx, prm, st);
  const int64_t L0 = L[0], K0 = Kx[0];
  if (L0 > ((int64_t)1 << 28)) return fail(HD_EUNSUPPORTED, "L too large");
  if (prec != HD_FP32) return fail(HD_EUNSUPPORTED, "1D path is FP32 only");
  switch (algo) {
    case HD_HYBRID_RCM:
    case HD_HYBRID_CS:
    case HD_HYBRID_CSRCM: return conv1d_hybrid(c, algo, f, g, h, L0, prm, st, K0);
    case HD_EXPLICIT_RCM: {
      int C, m, p;
      if (cluster_params(L0, &C, &m, &p) && C <= 8) return conv1d_explicit_cluster(c, f, g, h, L0, C, m, p, st, 1, K0);
      return explicit_nd(c, algo, 1, L, f, g, h, st, &K0);
    }
    case HD_EXPLICIT: return explicit_nd(c, algo, 1, L, f, g, h, st, &K0);
  }
  return fail(HD_EINVAL, "unknown algorithm");
}

hd_status hd_last_device_error(hd_ctx* c) {
  if (!c) return fail(HD_EINVAL, "null ctx");
  cudaSetDevice(c->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device");
  int w = 0;
  cudaMemcpy(&w, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemset(c->dev_err, 0, sizeof(int));
  return (hd_status)w;
}

}  // extern "C"
