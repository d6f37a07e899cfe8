// hd_noalloc.cu -- a 1D hybridRCM entry point that allocates no device memory.
//
// The paper has no counterpart: this exists for callers that are not allowed
// to allocate.  Every other entry point may grow the context's scratch or its
// twiddle-table cache with cudaMalloc on first use.  That is a problem for
// code that runs under an external memory budget or allocator (a framework
// that owns all device memory), for loops that must never block (cudaMalloc
// and cudaFree can synchronise the device), and for hosts that call in from a
// callback where allocation is forbidden.  This entry point keeps its scratch
// -- the twiddle table and the accumulator of the residue sums -- in one
// file-scope __device__ array that every GPU loading the library holds until
// the process exits, and it needs no context.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "hd_conv1d.cuh"
#include "hd_internal.h"

namespace hd {

cudaError_t launch_roots_fp64(float2* tw, int64_t N, cudaStream_t st);

constexpr int64_t kNoAllocTab = (int64_t{1} << 19) + 8192;  // twiddle entries (N = q m)
constexpr int64_t kNoAllocAcc = int64_t{1} << 18;           // accumulator entries (packed length)
constexpr int64_t kNoAllocMaxL = 2 * kNoAllocAcc;           // largest real length (524288)
constexpr int kNoAllocMaxDev = 64;

// 6.06 MB per device: [table | accumulator]
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocTab + kNoAllocAcc];

static std::mutex g_noalloc_mu;
static float2* g_noalloc_addr[kNoAllocMaxDev];

// Device address of the scratch array on the current device (looked up once
// per device; the array's name is only a host-side stand-in).
static hd_status noalloc_scratch(int dev, float2** out) {
  if (dev < 0 || dev >= kNoAllocMaxDev) return fail(HD_EUNSUPPORTED, "noalloc: device index beyond 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    float2* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetSymbolAddress");
    if (!p) return fail(HD_ECUDA, "noalloc: null scratch address");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return HD_OK;
}

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace hd

using namespace hd;

extern "C" hd_status hd_conv1d_rcm_noalloc(const float* f, const float* g, float* h, int64_t L,
                                           const hd_dim_params* prm, void* stream) {
  if (!f || !g || !h) return fail(HD_EINVAL, "noalloc: null array pointer");
  if (L < 1) return fail(HD_EINVAL, "noalloc: L < 1");
  if (L > kNoAllocMaxL) return fail(HD_EUNSUPPORTED, "noalloc: L beyond the static scratch (L <= 524288)");
  if (prm && (prm->m < 0 || prm->q < 0)) return fail(HD_EINVAL, "noalloc: negative m or q");
  int dev = 0;
  const cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return cuda_fail(de, "noalloc: cudaGetDevice");
  float2* scratch = nullptr;
  hd_status s = noalloc_scratch(dev, &scratch);
  if (s != HD_OK) return s;
  // parameters: the same rules as hd_conv1d for hybridRCM on one CTA
  const int64_t Lp = cdiv(L, 2);
  const int64_t mmax = (int64_t)kPts * 1024 / 4;
  int64_t m, q;
  if (prm && prm->m > 0) {
    m = prm->m;
    q = prm->q > 0 ? prm->q : cdiv(L, m);
    if (q * m < L) return fail(HD_EINVAL, "noalloc: hybridRCM needs q m >= L (packed)");
    if (m > mmax) return fail(HD_EUNSUPPORTED, "noalloc: m too large for one CTA (m <= 4096)");
  } else {
    m = next_smooth(Lp);
    q = 2;
    if (m > mmax) {
      for (int64_t k = 2;; ++k) {
        m = next_smooth(cdiv(Lp, k));
        if (m <= mmax) break;
      }
      q = cdiv(L, m);
    }
  }
  if (q * m > kNoAllocTab) return fail(HD_EUNSUPPORTED, "noalloc: q m beyond the static twiddle table (q m <= 532480)");
  int max_smem = 0;
  const cudaError_t ae = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ae != cudaSuccess) return cuda_fail(ae, "noalloc: cudaDeviceGetAttribute");
  const size_t smem = rcm1d_smem_bytes((int)L, (int)m, true);
  if (smem + 1024 > (size_t)max_smem) return fail(HD_EUNSUPPORTED, "noalloc: shared memory too small for m");
  cudaStream_t st = (cudaStream_t)stream;
  float2* tw = scratch;                // zeta_N^k, rewritten by every call
  float2* acc = scratch + kNoAllocTab; // zeroed by the kernel before use
  cudaError_t le = launch_roots_fp64(tw, q * m, st);
  if (le != cudaSuccess) return cuda_fail(le, "noalloc: table launch");
  Launch1D la;
  std::memset(&la, 0, sizeof(la));
  la.one.L = (int32_t)L;
  la.one.m = (int32_t)m;
  la.one.q = (int32_t)q;
  la.one.p = (int32_t)cdiv(Lp, m);
  la.one.plan = 0;
  la.one.plan_half = -1;
  la.one.tw = tw;
  la.one.gacc = acc;
  factor_radices((int)m, &la.plan_m);
  const int threads = threads_for_points(4 * m, kPts);
  le = launch_rcm1d(la, 1, threads, smem, f, g, h, st);
  if (le != cudaSuccess) return cuda_fail(le, "noalloc: convolution launch");
  return HD_OK;
}
