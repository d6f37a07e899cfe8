// hd_staged.cu -- hybridRCM in 1D through three kernels (the many-block path):
// the form of Sec. 2 for lengths whose q residues do not fit one cluster of
// CTAs (L > 73728), or for any length when called with explicit (M, q).
//
// With q residues of length M (N = q M >= L) and p = ceil(Lp / M) <= q/2
// blocks of the packed input (Lp = ceil(L/2), Eq. complexPacking):
//   stage A  for every s < M and both inputs, the q-point DFT over the blocks
//            t of x~_{tM+s} (the inner sums of Eq. forwardr for every residue
//            r at once: the pre-processing FFT over blocks of App. A, which
//            replaces p q direct multiply-adds by an FFT when p is large),
//            times zeta_N^{rs}, written as Y_r[s];
//   stage B  for every residue pair {c, q-c} (c = 0: the self-paired residues
//            0 and q/2), the length-M DFTs of Y_r (Eq. forwardr), the RCM
//            product (Eqs. Hr and Hr-conj) and the backward DFTs (Eq.
//            accumulator), written as w_r[s];
//   stage C  for every s, zeta_N^{-rs} w_r[s] and the backward q-point DFT
//            over r (Eq. accumulation, the post-processing FFT of App. A),
//            scaled by 1/N and unpacked to the real output of K samples.
// Stages A and C run their q-point DFTs on the CTA-level Stockham engine
// (hd_fft.cuh) over W consecutive s per CTA, so that each global access
// covers W consecutive complex values; stage B runs the compile-time engine of
// the cluster kernel (hd_cl_kernel.cuh) with one CTA per residue pair.  The
// intermediates Y_f, Y_g and w (24 N bytes per item) live in the context's
// workspace; batches run in chunks whose workspace stays under 1 GiB.
//
// The same three kernels convolve n >= 2 arrays x^1..x^n of different
// lengths L_i (Sec. 4.1, convolutions of more than two arrays: R^1 = F^1,
// R^j = R^{j-1} RCM F^j by Eqs. Akn, Rnk and RnMk, which are the binary RCM
// product with R^{j-1} in place of F; Sec. 7, arrays of different sizes:
// every array is folded over its own p_i = ceil(ceil(L_i/2) / M) blocks with
// the shared (M, q)).  The convolution has S = sum L_i - n + 1 samples, so
// 2 q M >= S dealiases every output.  Stage A transforms every array, stage B
// multiplies the n spectra of a residue pair one after the other, stage C is
// unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "hd_cl_kernel.cuh"
#include "hd_conv1d.cuh"
#include "hd_fft.cuh"
#include "hd_internal.h"

namespace hd {
namespace staged {

constexpr int kThreads = 256;                  // stages A and C
constexpr int kPoints = kThreads * kPts;       // q-point DFT points per CTA (W q <= kPoints)
constexpr int kMaxQ = 1024;
constexpr int kR3[] = {2, 4, 8, 16, 18};       // stage-B residue lengths M = 256 R3
constexpr int kLo = 64;                        // stage-B twiddles: zeta_N^{rs} = hi_r[s / 64] lo_r[s mod 64]
#ifndef HD_STAGED_MINB
#define HD_STAGED_MINB 4
#endif
constexpr int kMinB = HD_STAGED_MINB;          // resident CTAs per SM of stages A and C (structured engine)

constexpr int kMaxIn = 16;                     // arrays of one n-ary convolution

struct Geo {
  int M, q;          // residue length, residues
  int W, ldb;        // s per CTA in stages A and C (a power of two), shared-memory stride of one s
  int N;             // q M
  int K;             // real output length
  int nin;           // arrays convolved (2 for f * g)
  int rows;          // residues stored per array: q (hybridRCM), q/2 + 1 (hybridCS, Hermitian in r)
  int64_t out_stride;  // floats between items of h
};

// The input arrays: x[i] holds items of L[i] floats back to back (batches of
// the binary equal-length case); p[i] = ceil(ceil(L[i]/2) / M) blocks.
struct Inputs {
  const float* x[kMaxIn];
  int L[kMaxIn];
  int p[kMaxIn];
};

// The q-point DFTs of stages A and C on W arrays at stride ldb with the
// zeta_q table: the structured engine (inlined passes) for its lengths, else
// the plan-driven one.
template <int SIGN, bool SE>
__device__ __forceinline__ void q_dft(float2* buf, const Geo& G, const FftPlan& pq, const float2* __restrict__ tq) {
  if constexpr (SE) cta_fft_struct<SIGN, kPts>(buf, G.ldb, G.W, G.q, tq, 1);
  else cta_fft<SIGN, kPts>(buf, G.ldb, G.W, pq, tq, 1);
}

__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Programmatic dependent launch between the stages: a stage lets the next one
// be scheduled once all of its CTAs are running (launch_dependents), and the
// next stage does its set-up (tables) before it waits for the previous grid to
// complete and flush its writes (wait).  The wait returns when the previous
// grid ends; it is not a spin on memory.  It takes the pointer to the previous
// grid's output through the asm and hands it back: the loads through that
// pointer then depend on the wait, whereas a const __restrict__ pointer that
// only sits behind a "memory" clobber lets the compiler hoist unconditional
// loads above the wait and read the output before it is written.
__device__ __forceinline__ void allow_next_stage() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename T>
__device__ __forceinline__ T* after_prev_stage(T* p) {
  asm volatile("griddepcontrol.wait;" : "+l"(p) : : "memory");
  return p;
}

// Stages A and C move the W x q tile of a CTA between global memory (W
// consecutive s of each row t or r: contiguous) and shared memory (one array
// of q per s) in tasks of V consecutive s of one row: task id = tid + k
// kThreads covers row id mod q and the s chunk id / q, so consecutive lanes
// take consecutive rows (conflict-free shared accesses at any stride) and
// each lane moves V complex values with 16-byte accesses.  Every load of a
// loop is issued before the first store.

// Stage A: grid (M / W, n inputs, items).  Y[item][i][r M + s] =
// sum_{t < p_i} zeta_q^{rt} x~^i_{tM+s}: the q-point DFT over the blocks; the
// pre-twiddle zeta_N^{rs} of Eq. forwardr is applied in stage B.
// CS: real unpacked input (hybridCS, Sec. 3 with App. A), x_t[s] = f_{tM+s};
// the DFT over t of real data is Hermitian in r, so rows r <= q/2 are kept.
template <bool SE, int V, bool CS>
__global__ void __launch_bounds__(kThreads, SE ? kMinB : 1) k_stage_a(const __grid_constant__ Inputs in, float2* __restrict__ Y, Geo G,
                                                       const float2* __restrict__ tq, FftPlan pq) {
  constexpr int KT = kPts / V;  // tasks per thread (W q <= kPts kThreads)
  extern __shared__ float4 smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);  // buf[w ldb + t]
  allow_next_stage();
  const int which = blockIdx.y;
  const int Li = in.L[which], pi = in.p[which];
  const float* __restrict__ x = in.x[which] + (int64_t)blockIdx.z * Li;
  const int s0 = blockIdx.x * G.W;
  const int q = G.q, M = G.M, ldb = G.ldb, nt = G.q * (G.W / V);
  const DivF dq = make_div(q);
  const bool vec = aligned16(x);
  float2 v[KT][V];
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = threadIdx.x + k * kThreads;
    const int wc = fdiv(id, dq), t = id - wc * q;
#pragma unroll
    for (int i = 0; i < V; ++i) v[k][i] = make_float2(0.f, 0.f);
    if (CS && id < nt && t < pi) {
      const int j0 = t * M + s0 + wc * V;  // real index of the task's first value
      const float* src = x + j0;
      if (vec && j0 + V <= Li) {
#pragma unroll
        for (int i = 0; i < V; i += 4) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(src) + i / 4);
          v[k][i].x = a.x;
          v[k][i + 1].x = a.y;
          v[k][i + 2].x = a.z;
          v[k][i + 3].x = a.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (j0 + i < Li) v[k][i].x = __ldg(src + i);
      }
    } else if (!CS && id < nt && t < pi) {
      const int j0 = t * M + s0 + wc * V;  // packed index of the task's first value
      const float* src = x + 2 * j0;
      if (vec && 2 * (j0 + V) <= Li) {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(src) + i / 2);
          v[k][i] = make_float2(a.x, a.y);
          v[k][i + 1] = make_float2(a.z, a.w);
        }
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) {
          const int e = 2 * (j0 + i);
          if (e < Li) v[k][i].x = __ldg(src + 2 * i);
          if (e + 1 < Li) v[k][i].y = __ldg(src + 2 * i + 1);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = threadIdx.x + k * kThreads;
    const int wc = fdiv(id, dq), t = id - wc * q;
    if (id < nt) {
#pragma unroll
      for (int i = 0; i < V; ++i) buf[(wc * V + i) * ldb + t] = v[k][i];
    }
  }
  __syncthreads();
  q_dft<1, SE>(buf, G, pq, tq);
  float2* Yw = Y + ((int64_t)blockIdx.z * G.nin + which) * G.rows * M;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = threadIdx.x + k * kThreads;
    const int wc = fdiv(id, dq), r = id - wc * q;
    if (id < nt && r < G.rows) {
      float4* dst = reinterpret_cast<float4*>(Yw + r * M + s0 + wc * V);
#pragma unroll
      for (int i = 0; i < V; i += 2) {
        const float2 a = buf[(wc * V + i) * ldb + r], b = buf[(wc * V + i + 1) * ldb + r];
        dst[i / 2] = make_float4(a.x, a.y, b.x, b.y);
      }
    }
  }
}

// Stage C: grid (M / W, items).  h~_{tM+s} = (1/N) sum_r zeta_q^{-rt} w'_r[s]
// for the K output samples, where w'_r[s] = zeta_N^{-rs} w_r[s] comes from
// stage B (same task mapping as stage A).
// CS: rows r > q/2 are the conjugates of rows q - r (Eq. hrHerm), and the
// output is the real part, one real sample per (t, s) (Eq. real-accumulation).
template <bool SE, int V, bool CS>
__global__ void __launch_bounds__(kThreads, SE ? kMinB : 1) k_stage_c(const float2* __restrict__ Wr, float* __restrict__ h, Geo G,
                                                       const float2* __restrict__ tq, FftPlan pq) {
  constexpr int KT = kPts / V;
  extern __shared__ float4 smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const int s0 = blockIdx.x * G.W;
  const int q = G.q, M = G.M, ldb = G.ldb, nt = G.q * (G.W / V);
  const DivF dq = make_div(q);
  const float2* Wi = after_prev_stage(Wr) + (int64_t)blockIdx.z * G.rows * M;
  float2 v[KT][V];
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = threadIdx.x + k * kThreads;
    const int wc = fdiv(id, dq), r = id - wc * q;
    if (id < nt) {
      const bool mirror = CS && r >= G.rows;  // r > q/2: conj of row q - r
      const float4* src = reinterpret_cast<const float4*>(Wi + (mirror ? q - r : r) * M + s0 + wc * V);
#pragma unroll
      for (int i = 0; i < V; i += 2) {
        const float4 a = src[i / 2];
        v[k][i] = make_float2(a.x, mirror ? -a.y : a.y);
        v[k][i + 1] = make_float2(a.z, mirror ? -a.w : a.w);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = threadIdx.x + k * kThreads;
    const int wc = fdiv(id, dq), r = id - wc * q;
    if (id < nt) {
#pragma unroll
      for (int i = 0; i < V; ++i) buf[(wc * V + i) * ldb + r] = v[k][i];
    }
  }
  __syncthreads();
  q_dft<-1, SE>(buf, G, pq, tq);
  const float sc = 1.0f / (float)G.N;
  float* hi = h + blockIdx.z * G.out_stride;
  const bool vec = aligned16(hi);
  if constexpr (CS) {
    const int pout = (G.K + M - 1) / M;  // <= q since K <= N
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int id = threadIdx.x + k * kThreads;
      const int wc = fdiv(id, dq), t = id - wc * q;
      if (id < nt && t < pout) {
        const int j0 = t * M + s0 + wc * V;
        float* dst = hi + j0;
        if (vec && j0 + V <= G.K) {
#pragma unroll
          for (int i = 0; i < V; i += 4)
            reinterpret_cast<float4*>(dst)[i / 4] =
                make_float4(buf[(wc * V + i) * ldb + t].x * sc, buf[(wc * V + i + 1) * ldb + t].x * sc,
                            buf[(wc * V + i + 2) * ldb + t].x * sc, buf[(wc * V + i + 3) * ldb + t].x * sc);
        } else {
#pragma unroll
          for (int i = 0; i < V; ++i)
            if (j0 + i < G.K) dst[i] = buf[(wc * V + i) * ldb + t].x * sc;
        }
      }
    }
    return;
  }
  const int Kp = (G.K + 1) >> 1;
  const int pout = (Kp + M - 1) / M;  // <= q since K <= 2L - 1 < 2N
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = threadIdx.x + k * kThreads;
    const int wc = fdiv(id, dq), t = id - wc * q;
    if (id < nt && t < pout) {
      const int j0 = t * M + s0 + wc * V;
      float* dst = hi + 2 * j0;
      if (vec && 2 * (j0 + V) <= G.K) {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
          const float2 a = buf[(wc * V + i) * ldb + t], b = buf[(wc * V + i + 1) * ldb + t];
          reinterpret_cast<float4*>(dst)[i / 2] = make_float4(a.x * sc, a.y * sc, b.x * sc, b.y * sc);
        }
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) {
          const int e = 2 * (j0 + i);
          const float2 a = buf[(wc * V + i) * ldb + t];
          if (e < G.K) dst[2 * i] = a.x * sc;
          if (e + 1 < G.K) dst[2 * i + 1] = a.y * sc;
        }
      }
    }
  }
}

// Stages A and C for q = 256 R3 (R3 in {1, 2, 4}) on the compile-time engine
// of the cluster kernel (hd_cl_kernel.cuh): W = 16 / R3 arrays of q per CTA
// (4096 points), 256 threads, the in-place DIF passes (stage A, output in
// digit-reversed order: position p holds r = digit_freq(p)) and DIT passes
// (stage C, input placed at digit_pos(r), output in natural order), pass
// twiddles in shared memory.  Every trip count and stride is a compile-time
// constant, which the plan-driven and structured engines above are not.
template <int R3>
struct QEng {
  static constexpr int Q = 256 * R3;
  static constexpr int W = 16 / R3;    // s per CTA
  static constexpr int T = kThreads;
  using K = cl::Steps<1, R3, false, T>;
  static constexpr int TABS = cl::Shape<R3>::TABS;
  static constexpr size_t SMEM = sizeof(float2) * ((size_t)W * Q + TABS);
  static constexpr int V = W >= 8 ? 8 : 4;  // s per task
  static constexpr int KT = W * Q / V / T;  // tasks per thread (exact)
};

template <int R3>
__device__ __forceinline__ void qeng_tables(float2* tws, const float2* __restrict__ tab, int tid) {
  for (int i = tid; i < QEng<R3>::TABS / 2; i += QEng<R3>::T) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tws + 2 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(tab + 2 * i) : "memory");
  }
}

#ifndef HD_STAGE_AQ_MINB
#define HD_STAGE_AQ_MINB 2  // 117 registers, no spills (4: 64 registers, 340 B of spills, 7% slower)
#endif
template <int R3, bool CS>
__global__ void __launch_bounds__(kThreads, HD_STAGE_AQ_MINB) k_stage_a_q(const __grid_constant__ Inputs in, float2* __restrict__ Y, Geo G,
                                                            const float2* __restrict__ tab) {
  using E = QEng<R3>;
  using K = typename E::K;
  constexpr int Q = E::Q, W = E::W, V = E::V, KT = E::KT;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);  // W arrays of Q (row t at cl::phys(t))
  float2* tws = arr + W * Q;
  const int tid = threadIdx.x;
  allow_next_stage();
  qeng_tables<R3>(tws, tab, tid);
  const int which = blockIdx.y;
  const int Li = in.L[which], pi = in.p[which];
  const float* __restrict__ x = in.x[which] + (int64_t)blockIdx.z * Li;
  const int s0 = blockIdx.x * W, M = G.M;
  const bool vec = aligned16(x);
  float2 v[KT][V];
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = tid + k * E::T;
    const int wc = id / Q, t = id % Q;  // consecutive lanes: consecutive blocks t
#pragma unroll
    for (int i = 0; i < V; ++i) v[k][i] = make_float2(0.f, 0.f);
    if (t < pi) {
      const int j0 = t * M + s0 + wc * V;
      if constexpr (CS) {
        const float* src = x + j0;
        if (vec && j0 + V <= Li) {
#pragma unroll
          for (int i = 0; i < V; i += 4) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(src) + i / 4);
            v[k][i].x = a.x;
            v[k][i + 1].x = a.y;
            v[k][i + 2].x = a.z;
            v[k][i + 3].x = a.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < V; ++i)
            if (j0 + i < Li) v[k][i].x = __ldg(src + i);
        }
      } else {
        const float* src = x + 2 * j0;
        if (vec && 2 * (j0 + V) <= Li) {
#pragma unroll
          for (int i = 0; i < V; i += 2) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(src) + i / 2);
            v[k][i] = make_float2(a.x, a.y);
            v[k][i + 1] = make_float2(a.z, a.w);
          }
        } else {
#pragma unroll
          for (int i = 0; i < V; ++i) {
            const int e = 2 * (j0 + i);
            if (e < Li) v[k][i].x = __ldg(src + 2 * i);
            if (e + 1 < Li) v[k][i].y = __ldg(src + 2 * i + 1);
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = tid + k * E::T;
    const int wc = id / Q, t = id % Q;
#pragma unroll
    for (int i = 0; i < V; ++i) arr[(wc * V + i) * Q + cl::phys(t)] = v[k][i];
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  K::template pass1<1, W, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass2<1, W, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass3<1, W>(arr, tid);
  __syncthreads();
  float2* Yw = Y + ((int64_t)blockIdx.z * G.nin + which) * G.rows * M;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = tid + k * E::T;
    const int wc = id / Q, r = id % Q;
    if (r < G.rows) {
      const int pr = cl::phys(cl::digit_pos(r, R3));
      float4* dst = reinterpret_cast<float4*>(Yw + r * M + s0 + wc * V);
#pragma unroll
      for (int i = 0; i < V; i += 2) {
        const float2 a = arr[(wc * V + i) * Q + pr], b = arr[(wc * V + i + 1) * Q + pr];
        dst[i / 2] = make_float4(a.x, a.y, b.x, b.y);
      }
    }
  }
}

template <int R3, bool CS>
__global__ void __launch_bounds__(kThreads, 4) k_stage_c_q(const float2* __restrict__ Wr, float* __restrict__ h,
                                                            Geo G, const float2* __restrict__ tab) {
  using E = QEng<R3>;
  using K = typename E::K;
  constexpr int Q = E::Q, W = E::W, V = E::V, KT = E::KT;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);
  float2* tws = arr + W * Q;
  const int tid = threadIdx.x;
  qeng_tables<R3>(tws, tab, tid);
  const int s0 = blockIdx.x * W, M = G.M;
  const float2* Wi = after_prev_stage(Wr) + (int64_t)blockIdx.z * G.rows * M;
  float2 v[KT][V];
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = tid + k * E::T;
    const int wc = id / Q, r = id % Q;
    const bool mirror = CS && r >= G.rows;  // r > q/2: conj of row q - r
    const float4* src = reinterpret_cast<const float4*>(Wi + (mirror ? Q - r : r) * M + s0 + wc * V);
#pragma unroll
    for (int i = 0; i < V; i += 2) {
      const float4 a = src[i / 2];
      v[k][i] = make_float2(a.x, mirror ? -a.y : a.y);
      v[k][i + 1] = make_float2(a.z, mirror ? -a.w : a.w);
    }
  }
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = tid + k * E::T;
    const int wc = id / Q, r = id % Q;
    const int pr = cl::phys(cl::digit_pos(r, R3));
#pragma unroll
    for (int i = 0; i < V; ++i) arr[(wc * V + i) * Q + pr] = v[k][i];
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  K::template pass3<-1, W>(arr, tid);
  __syncthreads();
  K::template pass2<-1, W, 1>(arr, tid, tws);
  __syncthreads();
  K::template pass1<-1, W, 1>(arr, tid, tws);
  __syncthreads();
  const float sc = 1.0f / (float)G.N;
  float* hi = h + blockIdx.z * G.out_stride;
  const bool vec = aligned16(hi);
  const int Kp = CS ? G.K : (G.K + 1) >> 1;  // output positions j = t M + s (packed pairs for RCM)
  const int pout = (Kp + M - 1) / M;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int id = tid + k * E::T;
    const int wc = id / Q, t = id % Q;
    if (t >= pout) continue;
    const int j0 = t * M + s0 + wc * V;
    const int pt = cl::phys(t);
    if constexpr (CS) {
      float* dst = hi + j0;
      if (vec && j0 + V <= G.K) {
#pragma unroll
        for (int i = 0; i < V; i += 4)
          reinterpret_cast<float4*>(dst)[i / 4] =
              make_float4(arr[(wc * V + i) * Q + pt].x * sc, arr[(wc * V + i + 1) * Q + pt].x * sc,
                          arr[(wc * V + i + 2) * Q + pt].x * sc, arr[(wc * V + i + 3) * Q + pt].x * sc);
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (j0 + i < G.K) dst[i] = arr[(wc * V + i) * Q + pt].x * sc;
      }
    } else {
      float* dst = hi + 2 * j0;
      if (vec && 2 * (j0 + V) <= G.K) {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
          const float2 a = arr[(wc * V + i) * Q + pt], b = arr[(wc * V + i + 1) * Q + pt];
          reinterpret_cast<float4*>(dst)[i / 2] = make_float4(a.x * sc, a.y * sc, b.x * sc, b.y * sc);
        }
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) {
          const int e = 2 * (j0 + i);
          const float2 a = arr[(wc * V + i) * Q + pt];
          if (e < G.K) dst[2 * i] = a.x * sc;
          if (e + 1 < G.K) dst[2 * i + 1] = a.y * sc;
        }
      }
    }
  }
}

// Stage B: grid (q/2, items); CTA c holds residues c and q - c (c = 0:
// residues 0 and q/2) of both inputs in the four arrays [F_a, F_b, G_a, G_b]
// of the compile-time engine, in the same layout as one CTA of the cluster
// kernel with C = q/2.  It applies the pre-twiddle zeta_N^{rs} of Eq.
// forwardr on the way in and the post-twiddle zeta_N^{-rs} of Eq.
// accumulation on the way out, from two small tables per residue in shared
// memory (zeta_N^{rs} = zeta_N^{64 r (s / 64)} zeta_N^{r (s mod 64)}, both
// entries rounded once from FP64), and writes w'_c and w'_{q-c}.
template <int R3>
struct StageB {
  static constexpr int M = cl::Shape<R3>::M;
  static constexpr int NX = kLo + M / kLo;  // split-twiddle entries per residue
  static constexpr size_t SMEM = cl::Shape<R3>::SMEM + sizeof(float2) * 2 * NX;
};

template <int R3>
__device__ __forceinline__ float2 split_tw(const float2* tx, int s) {
  return cmul(tx[kLo + s / kLo], tx[s % kLo]);
}

// NA arrays of residues (c, rb, c, rb, ...) from Y into consecutive slots of
// the engine's layout, times zeta_N^{rs}: all loads are issued before the
// first store (SYNC: a barrier between them, for the twiddle tables).
template <int R3, int NA, bool SYNC, bool PAIRS = true>
__device__ __forceinline__ void load_twiddled(float2* dst, const float2* const (&src)[NA], const float2* tx, int tid) {
  constexpr int M = cl::Shape<R3>::M, T = cl::Shape<R3>::T, NX = StageB<R3>::NX;
  constexpr int U = M / 2 / T;  // 4
  float4 v[NA][U];
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int i = 0; i < U; ++i) v[a][i] = cl::ldg4(src[a] + 2 * (tid + i * T));
  if constexpr (SYNC) __syncthreads();
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int s = 2 * (tid + i * T);
      const float2* t = tx + (PAIRS ? (a & 1) * NX : 0);  // PAIRS: slots alternate residues c, rb
      cl::sts4(dst + a * M + cl::phys(s), cmul(make_float2(v[a][i].x, v[a][i].y), split_tw<R3>(t, s)),
               cmul(make_float2(v[a][i].z, v[a][i].w), split_tw<R3>(t, s + 1)));
    }
}

// The RCM product of one residue pair on the digit-reversed spectra in the
// slots [R_a, R_b, X_a, X_b]: R <- R RCM X (Eqs. Hr and Hr-conj; with R^{j-1}
// and F^j, Eqs. Akn, Rnk and RnMk).  Residue c at position p pairs with
// residue q - c at position M-1-p; for c = 0, residue q/2 pairs p with M-1-p
// of itself and residue 0 pairs frequency l with (M - l) mod M.
template <int R3>
__device__ __forceinline__ void pair_product(float2* arr, int c, int q, const float2* __restrict__ tw,
                                             const float2* __restrict__ zt, int tid) {
  using K = cl::Steps<1, R3>;
  constexpr int M = cl::Shape<R3>::M, T = cl::Shape<R3>::T;
  float2* Fa = arr;
  float2* Fb = arr + M;
  float2* Ga = arr + 2 * M;
  float2* Gb = arr + 3 * M;
  if (c > 0) {
    const float2 zr = __ldg(tw + c);
    for (int k = tid; k < M / 2; k += T) {
      const int p = 2 * k, pp = M - 2 - p;
      float2 A0, A1, B0, B1, C0, C1, D0, D1;
      cl::lds4(Fa + cl::phys(p), A0, A1);
      cl::lds4(Ga + cl::phys(p), B0, B1);
      cl::lds4(Fb + cl::phys(pp), C1, C0);
      cl::lds4(Gb + cl::phys(pp), D1, D0);
      const float4 z = cl::ldg4(zt + p);
      K::rcm_pair(A0, B0, C0, D0, K::rcm_factor(make_float2(z.x, z.y), zr), false);
      K::rcm_pair(A1, B1, C1, D1, K::rcm_factor(make_float2(z.z, z.w), zr), false);
      cl::sts4(Fa + cl::phys(p), A0, A1);
      cl::sts4(Fb + cl::phys(pp), C1, C0);
    }
  } else {
    const float2 zc = __ldg(tw + q / 2);
    for (int k = tid; k < M / 4; k += T) {
      const int p = 2 * k, pp = M - 2 - p;
      float2 A0, A1, B0, B1, C0, C1, D0, D1;
      cl::lds4(Fb + cl::phys(p), A0, A1);
      cl::lds4(Gb + cl::phys(p), B0, B1);
      cl::lds4(Fb + cl::phys(pp), C1, C0);
      cl::lds4(Gb + cl::phys(pp), D1, D0);
      const float4 z = cl::ldg4(zt + p);
      K::rcm_pair(A0, B0, C0, D0, K::rcm_factor(make_float2(z.x, z.y), zc), false);
      K::rcm_pair(A1, B1, C1, D1, K::rcm_factor(make_float2(z.z, z.w), zc), false);
      cl::sts4(Fb + cl::phys(p), A0, A1);
      cl::sts4(Fb + cl::phys(pp), C1, C0);
    }
    for (int p = tid; p < M; p += T) {
      const int l = cl::digit_freq(p, R3);
      const int ls = (l == 0) ? 0 : M - l;
      if (l > ls) continue;
      const int ps = cl::digit_pos(ls, R3);
      float2 A = Fa[cl::phys(p)], B = Ga[cl::phys(p)];
      float2 Ac = Fa[cl::phys(ps)], Bc = Ga[cl::phys(ps)];
      const bool self = (ls == l);
      K::rcm_pair(A, B, Ac, Bc, K::rcm_factor(cl::ldg2(zt + p), make_float2(1.f, 0.f)), self);
      Fa[cl::phys(p)] = A;
      if (!self) Fa[cl::phys(ps)] = Ac;
    }
  }
}

template <int R3>
__global__ void __launch_bounds__(cl::Shape<R3>::T, cl::Shape<R3>::MINB)
    k_stage_b(const float2* __restrict__ Y, float2* __restrict__ Wr, Geo G, const float2* __restrict__ tw,
              const float2* __restrict__ tab) {
  using K = cl::Steps<1, R3>;
  using S = cl::Shape<R3>;
  constexpr int M = S::M, T = S::T, NX = StageB<R3>::NX;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);
  float2* tws = arr + 4 * M;
  float2* tx = tws + S::TABS;  // [lo_a | hi_a | lo_b | hi_b]
  const int tid = threadIdx.x;
  const int c = blockIdx.x, q = G.q;
  const int rb = (c == 0) ? q / 2 : q - c;
  const float2* zt = tab + S::TABZ;  // zeta_M^{P^-1(p)}
  for (int i = tid; i < S::TABS / 2; i += T) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tws + 2 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(tab + 2 * i) : "memory");
  }
  for (int i = tid; i < 2 * NX; i += T) {
    const int rr = i < NX ? c : rb, u = i < NX ? i : i - NX;
    tx[i] = __ldg(tw + (u < kLo ? rr * u : rr * kLo * (u - kLo)));  // < r M <= N
  }
  allow_next_stage();
  const float2* Y0 = after_prev_stage(Y) + (int64_t)blockIdx.z * G.nin * G.N;
  float2* Wi = Wr + (int64_t)blockIdx.z * G.N;
  {
    const float2* const src[4] = {Y0 + c * M, Y0 + rb * M, Y0 + G.N + c * M, Y0 + G.N + rb * M};
    load_twiddled<R3, 4, true>(arr, src, tx, tid);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  K::template pass1<1, 4, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass2<1, 4, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass3<1, 4>(arr, tid);
  __syncthreads();
  pair_product<R3>(arr, c, q, tw, zt, tid);
  // arrays 3..n: R^j = R^{j-1} RCM F^j with F^j in the second pair of slots
  for (int i = 2; i < G.nin; ++i) {
    __syncthreads();
    const float2* Yi = Y0 + (int64_t)i * G.N;
    const float2* const src[2] = {Yi + c * M, Yi + rb * M};
    load_twiddled<R3, 2, false>(arr + 2 * M, src, tx, tid);
    __syncthreads();
    K::template pass1<1, 2, 2>(arr + 2 * M, tid, tws);
    __syncthreads();
    K::template pass2<1, 2, 2>(arr + 2 * M, tid, tws);
    __syncthreads();
    K::template pass3<1, 2>(arr + 2 * M, tid);
    __syncthreads();
    pair_product<R3>(arr, c, q, tw, zt, tid);
  }
  __syncthreads();
  K::template pass3<-1, 2>(arr, tid);
  __syncthreads();
  K::template pass2<-1, 2, 1>(arr, tid, tws);
  __syncthreads();
  K::template pass1<-1, 2, 1>(arr, tid, tws);
  __syncthreads();
  for (int k = tid; k < M / 2; k += T) {
    const int s = 2 * k;
    float2 a0, a1, b0, b1;
    cl::lds4(arr + cl::phys(s), a0, a1);
    cl::lds4(arr + M + cl::phys(s), b0, b1);
    a0 = cmul(a0, cconj(split_tw<R3>(tx, s)));
    a1 = cmul(a1, cconj(split_tw<R3>(tx, s + 1)));
    b0 = cmul(b0, cconj(split_tw<R3>(tx + NX, s)));
    b1 = cmul(b1, cconj(split_tw<R3>(tx + NX, s + 1)));
    *reinterpret_cast<float4*>(Wi + c * M + s) = make_float4(a0.x, a0.y, a1.x, a1.y);
    *reinterpret_cast<float4*>(Wi + rb * M + s) = make_float4(b0.x, b0.y, b1.x, b1.y);
  }
}

// Launch of a stage that may start while the previous one drains (its
// kernel waits for the previous grid before reading the previous output).
template <typename... KArgs, typename... Args>
static cudaError_t launch_after(void (*k)(KArgs...), dim3 grid, unsigned threads, size_t smem, cudaStream_t st,
                                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <int R3>
static cudaError_t launch_b(dim3 grid, cudaStream_t st, const float2* Y, float2* Wr, const Geo& G, const float2* tw,
                            const float2* tab) {
  auto k = k_stage_b<R3>;
  cudaError_t e = smem_optin((const void*)k, StageB<R3>::SMEM);
  if (e != cudaSuccess) return e;
  return launch_after(k, grid, cl::Shape<R3>::T, StageB<R3>::SMEM, st, Y, Wr, G, tw, tab);
}

static cudaError_t launch_b_any(int R3, dim3 grid, cudaStream_t st, const float2* Y, float2* Wr, const Geo& G,
                                const float2* tw, const float2* tab) {
  switch (R3) {
    case 2: return launch_b<2>(grid, st, Y, Wr, G, tw, tab);
    case 4: return launch_b<4>(grid, st, Y, Wr, G, tw, tab);
    case 8: return launch_b<8>(grid, st, Y, Wr, G, tw, tab);
    case 16: return launch_b<16>(grid, st, Y, Wr, G, tw, tab);
    case 18: return launch_b<18>(grid, st, Y, Wr, G, tw, tab);
  }
  return cudaErrorInvalidValue;
}

// Stage B of hybridCS: grid (q/2 + 1, items); CTA r holds residue r of f and
// g (the complex residue transform of Sec. 3.1.2, used here for every
// r <= q/2, as the paper's own code does for the v = 0 case of App. A):
// pre-twiddle zeta_N^{rs}, length-M DFTs, pointwise product (both spectra in
// the same digit-reversed order), backward DFT, post-twiddle; writes w'_r.
template <int R3>
struct StageBcs {
  static constexpr int M = cl::Shape<R3>::M;
  static constexpr size_t SMEM = sizeof(float2) * (2 * (size_t)M + cl::Shape<R3>::TABS + StageB<R3>::NX);
};

template <int R3>
__global__ void __launch_bounds__(cl::Shape<R3>::T, cl::Shape<R3>::MINB)
    k_stage_b_cs(const float2* __restrict__ Y, float2* __restrict__ Wr, Geo G, const float2* __restrict__ tw,
                 const float2* __restrict__ tab) {
  using K = cl::Steps<1, R3>;
  using S = cl::Shape<R3>;
  constexpr int M = S::M, T = S::T, NX = StageB<R3>::NX;
  extern __shared__ float4 smem_raw[];
  float2* arr = reinterpret_cast<float2*>(smem_raw);  // [F, G]
  float2* tws = arr + 2 * M;
  float2* tx = tws + S::TABS;  // [lo_r | hi_r]
  const int tid = threadIdx.x;
  const int r = blockIdx.x;
  for (int i = tid; i < S::TABS / 2; i += T) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tws + 2 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(tab + 2 * i) : "memory");
  }
  for (int i = tid; i < NX; i += T) tx[i] = __ldg(tw + (i < kLo ? r * i : r * kLo * (i - kLo)));  // < r M < N
  allow_next_stage();
  const int64_t astride = (int64_t)G.rows * M;
  const float2* Y0 = after_prev_stage(Y) + (int64_t)blockIdx.z * G.nin * astride;
  float2* Wi = Wr + (int64_t)blockIdx.z * astride;
  {
    const float2* const src[2] = {Y0 + r * M, Y0 + astride + r * M};
    load_twiddled<R3, 2, true, false>(arr, src, tx, tid);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  K::template pass1<1, 2, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass2<1, 2, 2>(arr, tid, tws);
  __syncthreads();
  K::template pass3<1, 2>(arr, tid);
  __syncthreads();
  for (int k = tid; k < M / 2; k += T) {
    const int p = cl::phys(2 * k);
    float2 a0, a1, b0, b1;
    cl::lds4(arr + p, a0, a1);
    cl::lds4(arr + M + p, b0, b1);
    cl::sts4(arr + p, cmul(a0, b0), cmul(a1, b1));
  }
  __syncthreads();
  K::template pass3<-1, 1>(arr, tid);
  __syncthreads();
  K::template pass2<-1, 1, 1>(arr, tid, tws);
  __syncthreads();
  K::template pass1<-1, 1, 1>(arr, tid, tws);
  __syncthreads();
  for (int k = tid; k < M / 2; k += T) {
    const int s = 2 * k;
    float2 a0, a1;
    cl::lds4(arr + cl::phys(s), a0, a1);
    a0 = cmul(a0, cconj(split_tw<R3>(tx, s)));
    a1 = cmul(a1, cconj(split_tw<R3>(tx, s + 1)));
    *reinterpret_cast<float4*>(Wi + r * M + s) = make_float4(a0.x, a0.y, a1.x, a1.y);
  }
}

template <int R3>
static cudaError_t launch_b_cs(dim3 grid, cudaStream_t st, const float2* Y, float2* Wr, const Geo& G,
                               const float2* tw, const float2* tab) {
  auto k = k_stage_b_cs<R3>;
  cudaError_t e = smem_optin((const void*)k, StageBcs<R3>::SMEM);
  if (e != cudaSuccess) return e;
  return launch_after(k, grid, cl::Shape<R3>::T, StageBcs<R3>::SMEM, st, Y, Wr, G, tw, tab);
}

static cudaError_t launch_b_cs_any(int R3, dim3 grid, cudaStream_t st, const float2* Y, float2* Wr, const Geo& G,
                                   const float2* tw, const float2* tab) {
  switch (R3) {
    case 2: return launch_b_cs<2>(grid, st, Y, Wr, G, tw, tab);
    case 4: return launch_b_cs<4>(grid, st, Y, Wr, G, tw, tab);
    case 8: return launch_b_cs<8>(grid, st, Y, Wr, G, tw, tab);
    case 16: return launch_b_cs<16>(grid, st, Y, Wr, G, tw, tab);
    case 18: return launch_b_cs<18>(grid, st, Y, Wr, G, tw, tab);
  }
  return cudaErrorInvalidValue;
}

static bool stage_b_length(int M) {
  for (int r : kR3)
    if (256 * r == M) return true;
  return false;
}

// Largest power of two W <= min(kPoints / q, 256): the s per CTA of stages A and C.
static int s_per_cta(int q) {
  int w = 1;
  while (2 * w * q <= kPoints && 2 * w <= 256) w *= 2;
  return w;
}

}  // namespace staged

// Planner of the three-kernel path for a needed padded length n (hybridRCM:
// q M >= L packed; hybridCS: q M >= 2L - 1 real), from CUDA-graph timings of
// single calls.  Up to n = 16384 (single hybridCS calls of L <= 8192), q = 4
// and the smallest M >= n / 4: a few long residues, 1.7-2x faster than
// M = 512 with q up to 32; up to n = 32768, (M, q) = (4096, 8) (L = 9000:
// 19.3 -> 14.5 us).  Beyond, q is one of 256, 512, 1024 (stages A and C on
// the compile-time engine) and M = 256 R3 (R3 in {2, 4, 8, 16, 18}) with the
// smallest N = q M >= n, the largest M among equal N (fewer, longer stage-B
// transforms measured faster); below n = 2^17 that is (512, 256), 13-14 us
// flat, where the q lengths {1, 3, 5, 9} x 2^a took 13-21 us (hybridRCM
// L = 80000: 16.2 -> 13.5 us).  False if n > 1024 x 4608.
bool staged_params(int64_t n, int* M, int* q) {
  if (n <= 4 * 4096) {
    *q = 4;
    *M = 512;
    while (4 * (int64_t)*M < n) *M *= 2;
    return true;
  }
  if (n <= 8 * 4096) {
    *q = 8;
    *M = 4096;
    return true;
  }
  int64_t bestN = 0;
  for (int qq : {256, 512, 1024})
    for (int r : staged::kR3) {
      const int64_t mm = 256 * r, N = qq * mm;
      if (N < n) continue;
      if (bestN == 0 || N < bestN || (N == bestN && mm > *M)) {
        bestN = N;
        *M = (int)mm;
        *q = qq;
      }
    }
  return bestN > 0;
}

namespace staged {

// The three stages for `batch` items (n arrays each, item b of array i at
// in.x[i] + b L_i, output item b at h + b K); S = sum L_i - n + 1 <= 2 q M.
// Stages A and C on the compile-time engine when q = 256 R3, R3 in {1, 2, 4}.
static bool qeng_length(int q) { return q == 256 || q == 512 || q == 1024; }

template <int R3>
static cudaError_t launch_a_q(bool cs, unsigned gx, unsigned gy, unsigned gz, cudaStream_t st, const Inputs& in,
                              float2* Y, const Geo& G, const float2* tabq) {
  auto k = cs ? k_stage_a_q<R3, true> : k_stage_a_q<R3, false>;
  cudaError_t e = smem_optin((const void*)k, QEng<R3>::SMEM);
  if (e != cudaSuccess) return e;
  k<<<dim3(gx, gy, gz), kThreads, QEng<R3>::SMEM, st>>>(in, Y, G, tabq);
  return cudaGetLastError();
}

template <int R3>
static cudaError_t launch_c_q(bool cs, unsigned gx, unsigned gz, cudaStream_t st, const float2* Wr, float* h,
                              const Geo& G, const float2* tabq) {
  auto k = cs ? k_stage_c_q<R3, true> : k_stage_c_q<R3, false>;
  cudaError_t e = smem_optin((const void*)k, QEng<R3>::SMEM);
  if (e != cudaSuccess) return e;
  return launch_after(k, dim3(gx, 1, gz), kThreads, QEng<R3>::SMEM, st, Wr, h, G, tabq);
}

static cudaError_t launch_a_q_any(int q, bool cs, unsigned gy, unsigned gz, cudaStream_t st, const Inputs& in,
                                  float2* Y, const Geo& G, const float2* tabq) {
  switch (q) {
    case 256: return launch_a_q<1>(cs, G.M / QEng<1>::W, gy, gz, st, in, Y, G, tabq);
    case 512: return launch_a_q<2>(cs, G.M / QEng<2>::W, gy, gz, st, in, Y, G, tabq);
    case 1024: return launch_a_q<4>(cs, G.M / QEng<4>::W, gy, gz, st, in, Y, G, tabq);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t launch_c_q_any(int q, bool cs, unsigned gz, cudaStream_t st, const float2* Wr, float* h,
                                  const Geo& G, const float2* tabq) {
  switch (q) {
    case 256: return launch_c_q<1>(cs, G.M / QEng<1>::W, gz, st, Wr, h, G, tabq);
    case 512: return launch_c_q<2>(cs, G.M / QEng<2>::W, gz, st, Wr, h, G, tabq);
    case 1024: return launch_c_q<4>(cs, G.M / QEng<4>::W, gz, st, Wr, h, G, tabq);
  }
  return cudaErrorInvalidValue;
}

// cs: hybridCS (real residues, q M >= S) instead of hybridRCM (packed, 2 q M >= S).
static hd_status run(hd_ctx* c, Inputs in, int nin, float* h, int64_t K, int M, int q, int64_t batch,
                     cudaStream_t st, bool cs = false) {
  int64_t S = 1;
  for (int i = 0; i < nin; ++i) S += in.L[i] - 1;
  if (!stage_b_length(M)) return fail(HD_EINVAL, "staged path: M must be 512, 1024, 2048, 4096 or 4608");
  if (q < 2 || q % 2 || q > kMaxQ) return fail(HD_EINVAL, "staged path: q must be even, 2 <= q <= 1024");
  if (cs && (int64_t)q * M < S) return fail(HD_EINVAL, "staged hybridCS needs q M >= 2L - 1");
  if (!cs && 2 * (int64_t)q * M < S)
    return fail(HD_EINVAL, "staged path needs 2 q M >= sum L_i - n + 1 (q M >= L for two arrays of length L)");
  Geo G;
  G.M = M;
  G.q = q;
  G.N = q * M;
  G.W = s_per_cta(q);  // >= 4 for q <= 1024
  const bool se = struct_length(q);
  const bool v8 = G.W >= 8;
  G.ldb = q;  // the structured engine keeps its swizzle inside whole 16-element blocks of each array
  G.K = (int)K;
  G.nin = nin;
  G.rows = cs ? q / 2 + 1 : q;
  G.out_stride = K;
  for (int i = 0; i < nin; ++i)
    in.p[i] = (int)(((cs ? (int64_t)in.L[i] : (int64_t)(in.L[i] + 1) / 2) + M - 1) / M);
  hd_status terr = HD_OK;
  const float2* tw = c->tables.get(G.N, st, &terr);
  if (!tw) return fail(terr, "twiddle table allocation failed");
  const float2* tab = c->tables.get_pass_table(M, st, &terr);
  if (!tab) return fail(terr, "pass table allocation failed");
  const float2* tq = c->tables.get(q, st, &terr);
  if (!tq) return fail(terr, "twiddle table allocation failed");
  const bool qe = qeng_length(q);
  const float2* tabq = qe ? c->tables.get_pass_table(q, st, &terr) : nullptr;
  if (qe && !tabq) return fail(terr, "pass table allocation failed");
  FftPlan pq;
  if (!factor_radices(q, &pq)) return fail(HD_EINVAL, "bad residue count");
  const size_t per_item = sizeof(float2) * (size_t)(nin + 1) * (size_t)G.rows * M;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(batch, 65535),
                                                                 ((int64_t)1 << 30) / (int64_t)per_item));
  if (ensure_ws(c, per_item * (size_t)chunk, st) != HD_OK) return fail(HD_ENOMEM, "workspace allocation failed");
  float2* Y = reinterpret_cast<float2*>(c->ws);  // [item][array][N]
  const size_t smem_ac = sizeof(float2) * (size_t)G.W * G.ldb;
  auto ka = cs ? (se ? (v8 ? k_stage_a<true, 8, true> : k_stage_a<true, 4, true>)
                     : (v8 ? k_stage_a<false, 8, true> : k_stage_a<false, 4, true>))
               : (se ? (v8 ? k_stage_a<true, 8, false> : k_stage_a<true, 4, false>)
                     : (v8 ? k_stage_a<false, 8, false> : k_stage_a<false, 4, false>));
  auto kc = cs ? (se ? (v8 ? k_stage_c<true, 8, true> : k_stage_c<true, 4, true>)
                     : (v8 ? k_stage_c<false, 8, true> : k_stage_c<false, 4, true>))
               : (se ? (v8 ? k_stage_c<true, 8, false> : k_stage_c<true, 4, false>)
                     : (v8 ? k_stage_c<false, 8, false> : k_stage_c<false, 4, false>));
  cudaError_t e = smem_optin((const void*)ka, smem_ac);
  if (e == cudaSuccess) e = smem_optin((const void*)kc, smem_ac);
  if (e != cudaSuccess) return cuda_fail(e, "shared memory opt-in");
  for (int64_t b0 = 0; b0 < batch; b0 += chunk) {
    const unsigned nb = (unsigned)std::min(chunk, batch - b0);
    float2* Wr = Y + (int64_t)nin * nb * G.rows * M;  // [item][rows][M]
    Inputs ic = in;
    for (int i = 0; i < nin; ++i) ic.x[i] = in.x[i] + b0 * in.L[i];
    float* hi = h + b0 * K;
    if (qe) {
      e = launch_a_q_any(q, cs, (unsigned)nin, nb, st, ic, Y, G, tabq);
    } else {
      ka<<<dim3(M / G.W, nin, nb), kThreads, smem_ac, st>>>(ic, Y, G, tq, pq);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "staged path: stage A launch");
    e = cs ? launch_b_cs_any(M / 256, dim3(q / 2 + 1, 1, nb), st, Y, Wr, G, tw, tab)
           : launch_b_any(M / 256, dim3(q / 2, 1, nb), st, Y, Wr, G, tw, tab);
    if (e != cudaSuccess) return cuda_fail(e, "staged path: stage B launch");
    e = qe ? launch_c_q_any(q, cs, nb, st, Wr, hi, G, tabq)
           : launch_after(kc, dim3(M / G.W, 1, nb), kThreads, smem_ac, st, (const float2*)Wr, hi, G, tq, pq);
    if (e != cudaSuccess) return cuda_fail(e, "staged path: stage C launch");
  }
  return HD_OK;
}

}  // namespace staged

hd_status conv1d_staged(hd_ctx* c, const float* f, const float* g, float* h, int64_t L, int64_t K, int M, int q,
                        int64_t batch, cudaStream_t st, bool cs) {
  staged::Inputs in = {};
  in.x[0] = f;
  in.x[1] = g;
  in.L[0] = in.L[1] = (int)L;
  return staged::run(c, in, 2, h, K > 0 ? K : L, M, q, batch, st, cs);
}

hd_status conv1d_multi(hd_ctx* c, int n, const float* const* x, const int64_t* L, int64_t K, int M, int q,
                       float* h, cudaStream_t st) {
  if (n < 2 || n > staged::kMaxIn) return fail(HD_EINVAL, "n-ary convolution: 2 <= n <= 16 arrays");
  staged::Inputs in = {};
  for (int i = 0; i < n; ++i) {
    in.x[i] = x[i];
    in.L[i] = (int)L[i];
  }
  return staged::run(c, in, n, h, K, M, q, 1, st);
}

}  // namespace hd
