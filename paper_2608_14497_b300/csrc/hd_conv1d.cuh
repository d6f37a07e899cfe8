// hd_conv1d.cuh -- launch descriptors of the 1D kernels.
#pragma once
#include <cuda_runtime.h>

#include "hd_internal.h"

namespace hd {

// Points per thread of the shared-memory FFT passes (register budget).
constexpr int kPts = 16;

// Launch descriptor: either a device table of items (batched) or one item
// passed by value (single call, nothing uploaded).
struct Launch1D {
  const Item1D* items;  // nullptr: use `one`
  const FftPlan* plans; // nullptr: use plan_m / plan_half
  Item1D one;
  FftPlan plan_m;
  FftPlan plan_half;
};

// Shared-memory float2 slots taken by an accumulator of `nf2` float2 values,
// rounded to an even count so the buffers behind it stay 16-byte aligned.
__host__ __device__ __forceinline__ int acc_slots(int nf2) { return (nf2 + 1) & ~1; }

// Parameters of one 1D convolution, resolved against the kernel limits.
struct Params1D {
  int m = 0, q = 0, p = 0;
  bool gacc = false;  // accumulator in global scratch (does not fit on chip)
  int threads = 0;
  size_t smem = 0;
};

// K: real output length (0: K = L); it sizes the accumulator.
hd_status resolve_rcm1d(hd_ctx* c, int64_t L, const hd_dim_params* prm, Params1D* out, int64_t K = 0);
hd_status resolve_cs1d(hd_ctx* c, int64_t L, const hd_dim_params* prm, Params1D* out, int64_t K = 0);

size_t rcm1d_smem_bytes(int L, int m, bool gacc);
size_t cs1d_smem_bytes(int L, int m, bool gacc);
int threads_for_points(int64_t points, int pts);
cudaError_t launch_rcm1d(const Launch1D& la, int nitems, int threads, size_t smem, const float* f,
                         const float* g, float* h, cudaStream_t st);
// rcm0: the combined CS+RCM form (residue 0 by the RCM operator on packed spectra)
cudaError_t launch_cs1d(const Launch1D& la, int nitems, int threads, size_t smem, const float* f,
                        const float* g, float* h, cudaStream_t st, bool rcm0 = false);

// Three-kernel hybridRCM path (hd_staged.cu): planner (false beyond its range)
// and the call for `batch` items of L floats (h: K floats per item).
bool staged_params(int64_t L, int* M, int* q);
// cs: hybridCS (real residues; needs q M >= 2L - 1) instead of hybridRCM (q M >= L).
hd_status conv1d_staged(hd_ctx* c, const float* f, const float* g, float* h, int64_t L, int64_t K, int M, int q,
                        int64_t batch, cudaStream_t st, bool cs = false);
// n arrays x[i] of L[i] floats (2 <= n <= 16) through the same kernels.
hd_status conv1d_multi(hd_ctx* c, int n, const float* const* x, const int64_t* L, int64_t K, int M, int q,
                       float* h, cudaStream_t st);

}  // namespace hd
