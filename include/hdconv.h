/*
 * hdconv.h -- C ABI of libhdconv.so: dealiased linear convolutions of two
 * equal-size real FP32 arrays in 1D, 2D and 3D on one NVIDIA B300 (sm_103a),
 * by hybrid dealiasing (Murasko & Bowman, "Hybrid Dealiasing and Implicit
 * Packing for Real Convolutions").
 *
 * Problem (Sec. 2, statement before Eq. forwardr; Sec. 6): given real arrays
 * f and g of extent L per dimension, compute
 *       h_k = sum_j f_j g_{k-j},   0 <= k_i < L_i in every dimension,
 * i.e. the first L outputs per dimension of the linear convolution, which a
 * DFT method reproduces exactly (up to rounding) once every dimension is padded
 * to at least 2L-1.  Results are normalised (the 1/(qm) factor of
 * Eqs. accumulation and real-accumulation is applied inside the last pass).
 *
 * Algorithms (Sec. 6):
 *   HD_EXPLICIT      zero padding materialised to 2L per dimension, real DFT,
 *                    pointwise product, inverse, crop (the standard method).
 *   HD_EXPLICIT_RCM  explicit padding with implicit packing: pack, complex DFT
 *                    of half length, the RCM operator (Eq. RCM, Alg. 4),
 *                    inverse, unpack (Algs. 3 and 5).  In 1D (single calls
 *                    up to L = 73728, batches) it runs on the same cluster
 *                    kernel as hybridRCM, reading zero-padded copies of f and
 *                    g (real length 2L, materialised in scratch) block by
 *                    block with no block skipped.
 *   HD_HYBRID_CS     hybrid dealiasing with conjugate symmetries (Sec. 3).
 *   HD_HYBRID_RCM    hybrid dealiasing with implicit packing (Sec. 4).
 *   HD_HYBRID_CSRCM  the combination Sec. 6.3 proposes: the residues of
 *                    hybridCS, with residue 0 computed by implicit packing
 *                    (packed length-m/2 DFTs multiplied by the RCM operator,
 *                    Eq. RCM, with no unpack/pack step) and residue q/2 by
 *                    the implicitly packed half-length transform of Eqs.
 *                    forwardq2/accumulateq2, so every residue is computed on
 *                    its own (no r, q-r pairing).  1D (single calls,
 *                    hd_conv_ext, batched plans) and 2D/3D along the first
 *                    dimension (first L outputs): there residues 0 and q/2
 *                    run through the packed recursion of Sec. 5 and the
 *                    other residues through hybridCS's complex rows.
 *                    Parameters as HD_HYBRID_CS (q m >= 2L-1; m need not be
 *                    even in 2D/3D).
 *
 * Memory: every array argument of a compute call is a DEVICE pointer owned
 * by the caller (row-major, last dimension contiguous, FP32).  h may equal f
 * or g (in place, as the paper times it); partial overlap is not allowed.
 * Calls are asynchronous on the given CUDA stream (NULL = legacy default).
 * The context owns twiddle tables and scratch; the first call for a new size
 * allocates them (tables: cudaMalloc and a synchronisation of the context's
 * own table stream; scratch: stream-ordered cudaMallocAsync / cudaFreeAsync on
 * the call's stream, no device synchronisation), so capture a call in a CUDA
 * graph only after one uncaptured call of the same shape.
 * Tables are complete before the call that creates them returns, so any
 * stream may use them.  The scratch is one area per context: a context serves
 * one stream at a time (calls on different streams that overlap on the GPU
 * race on it); use one context per stream and per host thread.
 *
 * Errors: HD_EINVAL for invalid arguments (null pointer, L < 1, hybrid
 * parameters that do not dealias, see hd_dim_params), HD_EUNSUPPORTED for a
 * valid request this build cannot run (e.g. shared memory too small for the
 * requested m), HD_ECUDA when a CUDA call fails (the message is kept and can be
 * read with hd_last_error_string), HD_ENOMEM when an allocation fails.
 * Nothing is launched when an error is returned before launch.
 */
#ifndef HDCONV_H
#define HDCONV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hd_ctx hd_ctx;
typedef struct hd_batch_plan hd_batch_plan;

typedef enum {
  HD_OK = 0,
  HD_EINVAL = 1,
  HD_ENOMEM = 2,
  HD_ECUDA = 3,
  HD_ETIMEOUT = 4,
  HD_EUNSUPPORTED = 5
} hd_status;

typedef enum {
  HD_EXPLICIT = 0,
  HD_EXPLICIT_RCM = 1,
  HD_HYBRID_CS = 2,
  HD_HYBRID_RCM = 3,
  HD_HYBRID_CSRCM = 4 /* combined CS+RCM: see the algorithm list above */
} hd_algo;

/* Arithmetic of the DFT stages.  HD_FP32 everywhere; HD_SPLIT_BF16 runs the
 * radix-16 stages of the 2D/3D hybridRCM path on tensor cores with hi/lo
 * bfloat16 operands and FP32 accumulation (returns HD_EUNSUPPORTED where not
 * available).  HD_SPLIT_FP16 (hi/lo half precision) is declared for the same
 * stage and always returns HD_EUNSUPPORTED: the spectra of the 2D/3D
 * configurations exceed half precision's range (max 65504) before the
 * normalisation, and the bfloat16 split already meets the 5e-5 bar. */
typedef enum { HD_FP32 = 0, HD_SPLIT_BF16 = 1, HD_SPLIT_FP16 = 2 } hd_prec;

/* Hybrid parameters of one dimension (Sec. 2: p = ceil(L/m), q = ceil(M/m)).
 * m = 0 lets the planner choose (m, q).  For HD_HYBRID_CS the data are real
 * of length L and q m >= 2L-1 is required, with m even when q is even
 * (Sec. 3.1.3).  For HD_HYBRID_RCM the packed dimension (the last one) has
 * length ceil(L/2) and needs q m >= L; outer dimensions of a 2D/3D call are
 * complex and need q m >= 2L-1.  Explicit algorithms ignore the parameters. */
typedef struct {
  int32_t m;
  int32_t q;
} hd_dim_params;

/* Context on a CUDA device (the device becomes current for each call). */
hd_status hd_create(hd_ctx** ctx, int device);
hd_status hd_destroy(hd_ctx* ctx);

/* 1D: f, g, h hold L floats.  prm may be NULL (planner). */
hd_status hd_conv1d(hd_ctx* ctx, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h,
                    int64_t L, const hd_dim_params* prm, void* stream);

/* 2D: L1 x L2 (L2 contiguous).  prm: 2 entries or NULL. */
hd_status hd_conv2d(hd_ctx* ctx, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h,
                    int64_t L1, int64_t L2, const hd_dim_params* prm, void* stream);

/* 3D: L1 x L2 x L3 (L3 contiguous).  prm: 3 entries or NULL. */
hd_status hd_conv3d(hd_ctx* ctx, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h,
                    int64_t L1, int64_t L2, int64_t L3, const hd_dim_params* prm, void* stream);

/* Convolution with output extents K[0..ndim) (Sec. 2: any padding of at least
 * 2L-1 per dimension dealiases every output of the linear convolution, so the
 * same transforms yield h_k for 0 <= k_i < K_i, L_i <= K_i <= 2L_i - 1; K_i =
 * 2L_i - 1 is the full linear convolution).  h holds prod(K) floats, row-major
 * with extents K; K == NULL means K = L (hd_conv1d/2d/3d are this call).  h
 * may alias f or g only when K = L.  Supported: every algorithm in 1D;
 * hybridRCM, explicit and explicitRCM in 2D/3D (hybridCS in 2D/3D:
 * HD_EUNSUPPORTED unless K = L).  HD_EINVAL for K outside [L, 2L-1]. */
hd_status hd_conv_ext(hd_ctx* ctx, hd_algo algo, hd_prec prec, int ndim, const int64_t* L, const int64_t* K,
                      const float* f, const float* g, float* h, const hd_dim_params* prm, void* stream);

/* `batch` independent convolutions of equal extents Ls[0..ndim) stored back to
 * back in f, g and h (item b at offset b * prod(Ls)); the same convolutions as
 * one hd_conv1d/2d/3d call per item (bit for bit where both take the same
 * kernels).  hybridRCM in FP32 runs the whole batch in one pass sequence (1D:
 * one cluster launch; 2D/3D: every outer pass and the row pass over all items
 * at once, Sec. 5); hybridCS in 1D runs the three kernels of
 * hd_conv1d_staged over the whole batch; explicitRCM in 1D one cluster
 * launch; other cases run item by item.  Errors as hd_conv1d. */
hd_status hd_conv_batch(hd_ctx* ctx, hd_algo algo, hd_prec prec, int ndim, const int64_t* Ls, int32_t batch,
                        const float* f, const float* g, float* h, void* stream);

/* 1D hybrid convolution through three kernels, for long lengths (the block
 * sums of Eq. forwardr and the accumulation of Eqs. accumulation /
 * real-accumulation as q-point DFTs over the blocks: the inner loop of App. A
 * and of the complex case it cites): for q residues of length M, stage A
 * transforms f and g over the blocks for every s < M, stage B (one CTA per
 * residue pair for hybridRCM, per residue r <= q/2 for hybridCS) runs the
 * length-M DFTs, the product (RCM, Eqs. Hr/Hr-conj; or pointwise) and the
 * backward DFTs, stage C transforms back over the residues and unpacks
 * (hybridRCM) or takes the real part (hybridCS, Eq. real-accumulation).
 * hd_conv1d, hd_conv_ext and hd_conv_batch take this path when prm is NULL
 * for hybridRCM lengths beyond the cluster kernel (L > 73728) and for hybridCS
 * from L = 513 in single calls (hd_conv1d, hd_conv_ext: the q/2 + 1 residue
 * CTAs beat one CTA's latency) and for every L in hd_conv_batch (one pass
 * sequence over the batch); this call runs it for any L.
 *   algo: HD_HYBRID_RCM (needs q M >= L) or HD_HYBRID_CS (needs q M >= 2L-1).
 *   `batch` items of L floats back to back in f and g, of K floats in h
 *   (K = 0 means K = L; L <= K <= 2L-1).  M in {512, 1024, 2048, 4096,
 *   4608}, q even, 2 <= q <= 1024; M = q = 0 lets the planner choose.
 * Scratch: 24 q M bytes per item (hybridRCM), 12 (q + 2) M (hybridCS); batches
 * run in chunks of at most 1 GiB.  h may alias f or g only when K = L.
 * Errors as hd_conv1d. */
hd_status hd_conv1d_staged(hd_ctx* ctx, hd_algo algo, int64_t L, int64_t K, int32_t M, int32_t q, int32_t batch,
                           const float* f, const float* g, float* h, void* stream);

/* Convolution of n real 1D arrays of possibly different lengths on the same
 * three kernels: h_k = (x^1 * x^2 * ... * x^n)_k for 0 <= k < K.
 * n >= 3 is the implicitly packed convolution of more than two arrays
 * (Sec. 4.1: R^1 = F^1, R^j = R^{j-1} RCM F^j by Eqs. Akn, Rnk and RnMk);
 * unequal lengths (e.g. a long signal and a short kernel) follow Sec. 7: each
 * array is folded over its own number of blocks p_i = ceil(ceil(L_i/2) / M),
 * with M and q shared, so no array is padded to another's length.
 *   x: HOST array of n DEVICE pointers, x[i] holding L[i] floats; L: host
 *   array of n lengths (1 <= L_i <= 2^28); 2 <= n <= 16.
 *   K: output length, 1 <= K <= S = sum L_i - n + 1 (S is the whole linear
 *   convolution); K = 0 means max L_i.
 *   M in {512, 1024, 2048, 4096, 4608}, q even, 2 <= q <= 1024, 2 q M >= S;
 *   M = q = 0 lets the planner choose (HD_EUNSUPPORTED when S > 2 x 1024 x
 *   4608).
 *   h: DEVICE buffer of K floats; it may alias any input (every input is read
 *   by the first kernel, h is written by the last).
 * Scratch: 8 (n + 1) q M bytes.  Errors as hd_conv1d. */
hd_status hd_conv1d_multi(hd_ctx* ctx, int32_t n, const float* const* x, const int64_t* L, int64_t K, int32_t M,
                          int32_t q, float* h, void* stream);

/* Batched 1D convolutions of uneven lengths.  A plan is built on the host
 * from HOST arrays: item i occupies floats [offsets[i], offsets[i] + L[i]) of
 * f, g and h (items must not overlap).  The planner picks (m, q) per length
 * and uploads the item table; hd_conv1d_batched then enqueues a fixed set of
 * launches with no allocation and no host-to-device copy, so it can be
 * captured in a CUDA graph.  The plan must outlive every launch that uses it.
 * algo: HD_HYBRID_RCM, HD_HYBRID_CS, or HD_EXPLICIT_RCM (the explicit-padding
 * baseline: the plan holds zero-padded copies of the items, 16 bytes per
 * real input element, written by each call; lengths up to 73728, else
 * HD_EUNSUPPORTED). */
hd_status hd_batch_plan_create(hd_ctx* ctx, hd_algo algo, int32_t n, const int64_t* offsets, const int32_t* L,
                               hd_batch_plan** plan);
hd_status hd_batch_plan_destroy(hd_batch_plan* plan);
hd_status hd_conv1d_batched(hd_ctx* ctx, const hd_batch_plan* plan, const float* f, const float* g, float* h,
                            void* stream);
/* Number of kernel launches one hd_conv1d_batched call of the plan enqueues
 * (hybridRCM: one per cluster size in use, launched concurrently on streams
 * forked from and joined back to `stream`; plus one for lengths outside the
 * cluster kernel's range).  EINVAL on NULL arguments. */
hd_status hd_batch_plan_launches(const hd_batch_plan* plan, int32_t* n);

/* Adjoint of h = conv(f, g) (first L outputs per dimension) for `batch`
 * independent problems of extents Ls[0..ndim) stored back to back: given
 * grad_h, grad_f[j] = sum_k grad_h[k] g[k-j] and grad_g[j] = sum_k grad_h[k]
 * f[k-j], computed as rev(conv(rev(grad_h), g)) on every axis (the adjoint of
 * a truncated convolution is a reversed truncated convolution; the paper has
 * no adjoint, this follows from the definition).  grad_f or grad_g may be
 * NULL to skip it; neither may overlap grad_h, f, g or the other gradient
 * (HD_EINVAL).  hybridRCM in 2D/3D runs one fused pass sequence for the whole
 * batch: the reversal is folded into the first pass's loads and the last
 * pass's stores, and the transforms of rev(grad_h) are formed once for both
 * gradients; other cases reverse the batch in one launch per array and
 * convolve with hd_conv_batch.  Scratch grows stream-ordered on `stream`. */
hd_status hd_conv_adjoint(hd_ctx* ctx, hd_algo algo, int ndim, const int64_t* Ls, int32_t batch,
                          const float* grad_h, const float* f, const float* g, float* grad_f, float* grad_g,
                          void* stream);

/* The planner's (m, q) for one dimension of real length L and `algo`, as a
 * single hd_conv1d call uses it.  HD_HYBRID_RCM reports packed lengths: up to
 * L = 73728 the cluster instance (m, q = 2C) with the smallest modelled
 * latency for one convolution per call (a per-call cost for each cluster size
 * C plus a per-point cost of the m-point transforms, fitted to B300 timings;
 * batched plans choose by measured throughput instead); beyond, the (M, q) of
 * the three-kernel path of hd_conv1d_staged. */
hd_status hd_plan(hd_ctx* ctx, hd_algo algo, int64_t L, hd_dim_params* out);

/* The batched planner's autotuner table (filled by the first hybridRCM batch
 * plan of the context unless the environment sets HD_AUTOTUNE=0): for each
 * candidate i < *n (at most cap are copied), a cluster of C[i] CTAs with
 * residue DFT length m[i] took us[i] microseconds per convolution of length
 * 2 C[i] m[i].  The planner picks, per length, the cheapest candidate among
 * the three shortest feasible DFT lengths of each cluster size (the role of
 * the paper's empirical parameter scan, Sec. 6).  *n = 0 before tuning. */
hd_status hd_tuning_table(hd_ctx* ctx, int32_t cap, int32_t* C, int32_t* m, double* us, int32_t* n);

/* hybridRCM in 1D without any device allocation (no counterpart in the paper).
 * For callers that may not allocate: code running under an external memory
 * budget or allocator, loops that must not block (cudaMalloc / cudaFree can
 * synchronise the device), or hosts calling from a context where allocation
 * is forbidden.  Same arguments and results as hd_conv1d(HD_HYBRID_RCM, FP32)
 * except that it takes no context and always runs the one-CTA kernel with its
 * accumulator in global memory.  Scratch (the twiddle table and the
 * accumulator, 6.06 MB) is a file-scope device array that every GPU loading
 * the library holds until the process exits.  Limits: 1 <= L <= 524288, the
 * DFT length m <= 4096 and q m <= 532480; larger requests return
 * HD_EUNSUPPORTED.  Runs on the current device and `stream`.  The first call
 * on a device looks up the array's device address (set-up, no allocation):
 * make that first call before any stream capture.  All calls share the one
 * array, so calls that overlap on the GPU (different streams, or concurrent
 * host threads) race and give wrong results: serialise them.  Each call
 * rewrites the table and zeroes the accumulator before use. */
hd_status hd_conv1d_rcm_noalloc(const float* f, const float* g, float* h, int64_t L, const hd_dim_params* prm,
                                void* stream);

/* Status of device-side checks since the last call (bounded waits that gave
 * up report HD_ETIMEOUT); reading it synchronises the context's device and
 * clears the word. */
hd_status hd_last_device_error(hd_ctx* ctx);

const char* hd_strerror(hd_status s);
const char* hd_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* HDCONV_H */
