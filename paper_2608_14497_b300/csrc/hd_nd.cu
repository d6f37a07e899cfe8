// hd_nd.cu -- 2D/3D convolutions by the recursive decomposition of Sec. 5, and
// the explicit-padding baselines (Sec. 6) in 1D/2D/3D.
//
// hybridRCM (Sec. 5, Eqs. multidimComplexPacking and RCM-ndim, operator C_n):
//   pack along the last dimension; complex hybrid forward along every outer
//   (strided) dimension (k_col_fwd, Eq. forwardr per column); for every row of
//   the outer spectra and its conjugate partner (k1*, k2*) a fused 1D hybrid
//   convolution along the last dimension with the C_1 operator (k_rows_rcm);
//   complex hybrid backward along the outer dimensions, the last one unpacking
//   the real result (k_col_bwd).
// hybridCS (Sec. 5 with Sec. 3): the first dimension is transformed with the
//   real residues of Sec. 3.1 (k_col_fwd_cs / k_col_bwd_cs); the middle
//   dimension (3D) with complex hybrid dealiasing; every row along the last
//   dimension is a complex hybrid convolution with a pointwise product
//   (k_rows_cconv).
// explicit / explicitRCM: zero padding materialised to 2L per dimension in
//   scratch, full-length DFTs pass by pass (rows along the last dimension,
//   columns along the others), pointwise product or the RCM operator of
//   Eq. RCM-ndim, inverse, crop.
//
// Layout of transformed outer dimensions: residue-major rows, index r m + l
// for the natural frequency k = q l + r.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "hd_nd.cuh"
#include "hd_nd_kernels.cuh"

namespace hd {

// ---------------------------------------------------------------------------
// explicit baselines
// ---------------------------------------------------------------------------
// Materialised zero padding: P[(2L)^d] real (mode 0), or packed complex with
// the last dimension of packed length Mp (mode 1).
__global__ void k_pad(const float* __restrict__ f, void* P, int d, int64_t L0, int64_t L1, int64_t L2, int64_t M0,
                      int64_t M1, int64_t M2, int mode) {
  // M*: padded extents of the output (complex extent for the last dim in mode 1)
  const int64_t tot = M0 * M1 * M2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / (M1 * M2), b = (i / M2) % M1, c = i % M2;
    if (mode == 0) {
      float v = 0.f;
      if (a < L0 && b < L1 && c < L2) v = f[(a * L1 + b) * L2 + c];
      reinterpret_cast<float*>(P)[i] = v;
    } else {
      float2 v = make_float2(0.f, 0.f);
      if (a < L0 && b < L1) {
        const int64_t c0 = 2 * c;
        if (c0 < L2) v.x = f[(a * L1 + b) * L2 + c0];
        if (c0 + 1 < L2) v.y = f[(a * L1 + b) * L2 + c0 + 1];
      }
      reinterpret_cast<float2*>(P)[i] = v;
    }
  }
}

// Pointwise product S_f <- S_f . S_g.
__global__ void k_pointwise(float2* __restrict__ A, const float2* __restrict__ B, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    A[i] = cmul(A[i], B[i]);
}

// Eq. RCM-ndim on full spectra of extents (M0, M1, M2) (the last packed):
// each thread owns the pair {k, k*} with k <= k* (linear index), in place.
__global__ void k_rcm_nd(float2* __restrict__ A, const float2* __restrict__ B, int64_t M0, int64_t M1, int64_t M2,
                         const float2* __restrict__ tw, int twmul) {
  const int64_t tot = M0 * M1 * M2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / (M1 * M2), b = (i / M2) % M1, c = i % M2;
    const int64_t as = (M0 - a) % M0, bs = (M1 - b) % M1, cs = (M2 - c) % M2;
    const int64_t j = (as * M1 + bs) * M2 + cs;
    if (j < i) continue;
    const float2 Fa = A[i], Ga = B[i], Fc = A[j], Gc = B[j];
    const float2 z = tw_get<1>(tw, (int)(c * twmul));
    const float2 Z = make_float2(0.25f * (1.f + z.x), 0.25f * z.y);
    const float2 alpha = cmul(cmul(csub(Fa, cconj(Fc)), csub(Ga, cconj(Gc))), Z);
    A[i] = csub(cmul(Fa, Ga), alpha);
    if (j != i) A[j] = csub(cmul(Fc, Gc), cconj(alpha));
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
#define HD_TRY(call)                                    \
  do {                                                  \
    if ((call) != cudaSuccess) return HD_ECUDA;         \
  } while (0)

static int elementwise_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::min<int64_t>(b, 148 * 32);
}

// Choose W columns per CTA for a column pass over A blocks of B columns:
// shared memory per column `per_col` bytes and points per column `pts`;
// W a power of two <= 8 (the strip loops of the complex passes split the
// element index with a shift and a mask), W even if `even`; no wider than B
// (the largest power of two <= B) unless `even`; then halved while the grid is
// under two CTAs per SM (wide column groups on few SMs leave most of the GPU
// idle).
int choose_W(size_t per_col, int pts, int64_t A, int64_t B, size_t max_smem, bool even, int64_t max_pts,
             int num_sms) {
  int W = 8;
  while (W > 1 && ((size_t)W * per_col > max_smem || (int64_t)W * pts > max_pts)) W >>= 1;
  if (even && W < 2) W = 2;
  while (!even && W > 1 && (int64_t)W > B) W >>= 1;
  const int wmin = even ? 2 : 1;
  while (W > wmin && A * ((B + W - 1) / W) < 2 * (int64_t)std::max(num_sms, 1)) W >>= 1;
  return W;
}

struct ColPass {
  int m, q, p;
  const float2* tw;
  FftPlan pl;
};

static hd_status col_fwd(hd_ctx* c, const void* X, int in_mode, int Lreal, float2* Y, int64_t A, int Lin, int64_t B,
                         const ColPass& cp, cudaStream_t st, int64_t Bp = 0, bool tc = false) {
  const bool keep = cp.q > 1;
  const Eng eng = pick_eng(tc, struct_length(cp.m) && cp.q <= 2);
  const size_t per_col = sizeof(float2) * ((keep ? (size_t)Lin : 0) + (size_t)cp.m) + 16;
  const int W = choose_W(per_col, cp.m, A, B, (size_t)c->max_smem, false, max_points(eng), c->num_sms);
  if (W < 1 || (W & (W - 1))) return fail(HD_EUNSUPPORTED, "column pass: strip width not a power of two");
  ColGeom cg{A, B, W, Bp > 0 ? Bp : B};
  const size_t smem = sizeof(float2) * ((keep ? (size_t)acc_slots(W * Lin) : 0) + (size_t)W * cp.m);
  if (smem > (size_t)c->max_smem || (int64_t)W * cp.m > max_points(eng)) return HD_EUNSUPPORTED;
  const int T = eng_threads(eng, (int64_t)W * cp.m);
  const unsigned grid = (unsigned)(A * ((B + W - 1) / W));
  HD_TRY(launch_col_fwd(eng, grid, T, smem, st, X, Y, cg, Lin, cp.m, cp.q, cp.p, in_mode, Lreal, cp.tw, cp.pl));
  return HD_OK;
}

static hd_status col_bwd(hd_ctx* c, const float2* Y, void* Z, int out_mode, int Lreal, int64_t A, int Lout, int64_t B,
                         const ColPass& cp, float scale, cudaStream_t st, int64_t Bp = 0, bool tc = false) {
  const bool sep = cp.q > 1 || Lout > cp.m;
  const Eng eng = pick_eng(tc, struct_length(cp.m) && cp.q <= 2);
  const size_t per_col = sizeof(float2) * ((sep ? (size_t)Lout : 0) + (size_t)cp.m) + 16;
  const int W = choose_W(per_col, cp.m, A, B, (size_t)c->max_smem, false, max_points(eng), c->num_sms);
  if (W < 1 || (W & (W - 1))) return fail(HD_EUNSUPPORTED, "column pass: strip width not a power of two");
  ColGeom cg{A, B, W, Bp > 0 ? Bp : B};
  const size_t smem = sizeof(float2) * ((sep ? (size_t)acc_slots(W * Lout) : 0) + (size_t)W * cp.m);
  if (smem > (size_t)c->max_smem || (int64_t)W * cp.m > max_points(eng)) return HD_EUNSUPPORTED;
  const int T = eng_threads(eng, (int64_t)W * cp.m);
  const unsigned grid = (unsigned)(A * ((B + W - 1) / W));
  HD_TRY(launch_col_bwd(eng, grid, T, smem, st, Y, Z, cg, Lout, cp.m, cp.q, out_mode, Lreal, scale, cp.tw, cp.pl));
  return HD_OK;
}

// Hybrid parameters of an outer (complex) dimension of real length L.
static hd_status outer_params(hd_ctx* c, int64_t L, const hd_dim_params* prm, ColPass* cp, cudaStream_t st) {
  int64_t m, q;
  if (prm && prm->m > 0) {
    m = prm->m;
    q = prm->q > 0 ? prm->q : (2 * L - 1 + m - 1) / m;
    if (q * m < 2 * L - 1) return HD_EINVAL;
  } else {
    m = ladder_ceil(L);
    q = 2;
  }
  if (m > (int64_t)kPts * 1024) return HD_EUNSUPPORTED;
  cp->m = (int)m;
  cp->q = (int)q;
  cp->p = (int)((L + m - 1) / m);
  factor_radices((int)m, &cp->pl);
  hd_status terr = HD_OK;
  cp->tw = c->tables.get(q * m, st, &terr);
  return cp->tw ? HD_OK : terr;
}

// Parameters of the last (row) dimension for the RCM rows (packed, needs
// q m >= L) or CS rows (complex, needs q m >= 2L-1).
static hd_status row_params(hd_ctx* c, int64_t L, bool packed, const hd_dim_params* prm, ColPass* cp,
                            cudaStream_t st, bool cl_rows = false, bool q1 = false) {
  const int64_t Lr = packed ? (L + 1) / 2 : L;
  const int64_t need = packed ? L : 2 * L - 1;
  int64_t m, q;
  if (prm && prm->m > 0) {
    m = prm->m;
    q = prm->q > 0 ? prm->q : (need + m - 1) / m;
    if (q * m < need) return HD_EINVAL;
  } else {
    m = ladder_ceil(Lr);
    q = (need + m - 1) / m;
    if (packed && cl_rows && Lr > 64) {
      // the row-pair kernel on the compile-time engine: q = 2, m = 256 R3 >= Lp
      for (int R3 : {1, 2, 3, 4, 5, 6, 8})
        if (256 * R3 >= Lr) {
          m = 256 * R3;
          q = 2;
          break;
        }
      // one residue (q = 1) when some 256 R3 >= L gives a shorter padded row
      if (q1)
        for (int R3 : {1, 2, 3, 4, 5, 6, 8})
          if (256 * R3 >= L) {
            if (256 * R3 < q * m) {
              m = 256 * R3;
              q = 1;
            }
            break;
          }
    }
  }
  cp->m = (int)m;
  cp->q = (int)q;
  cp->p = (int)((Lr + m - 1) / m);
  factor_radices((int)m, &cp->pl);
  hd_status terr = HD_OK;
  cp->tw = c->tables.get(q * m, st, &terr);
  return cp->tw ? HD_OK : terr;
}

// Outer and row parameters of a hybridRCM 2D/3D convolution.
struct RcmNdPlan {
  ColPass outer[2], row;
  int64_t Lp, M0, M1;
};
static hd_status rcm_nd_plan(hd_ctx* c, int d, const int64_t* L, const hd_dim_params* prm, RcmNdPlan* P,
                             cudaStream_t st, bool cl_rows = false, bool q1 = false) {
  P->Lp = (L[d - 1] + 1) / 2;
  for (int i = 0; i < d - 1; ++i) {
    hd_status s = outer_params(c, L[i], prm ? &prm[i] : nullptr, &P->outer[i], st);
    if (s != HD_OK) return s;
  }
  hd_status s = row_params(c, L[d - 1], true, prm ? &prm[d - 1] : nullptr, &P->row, st, cl_rows, q1);
  if (s != HD_OK) return s;
  P->M0 = (int64_t)P->outer[0].q * P->outer[0].m;
  P->M1 = d == 3 ? (int64_t)P->outer[1].q * P->outer[1].m : 1;
  return HD_OK;
}

// Forward outer passes of one real array (batch items back to back, each
// [L0][L1] or [L0][L1][L2]) into its outer spectra S = [batch][M0][M1][Lp];
// T is the 3D intermediate [batch][M0][L1][Lp].
static hd_status rcm_nd_forward(hd_ctx* c, int d, const int64_t* L, int64_t batch, const RcmNdPlan& P,
                                const float* x, int in_mode, float2* S, float2* T, cudaStream_t st, bool tc) {
  const int Ln = (int)L[d - 1];
  if (d == 2) return col_fwd(c, x, in_mode, Ln, S, batch, (int)L[0], P.Lp, P.outer[0], st, 0, tc);
  hd_status s = col_fwd(c, x, in_mode, Ln, T, batch, (int)L[0], L[1] * P.Lp, P.outer[0], st, P.Lp, tc);
  if (s == HD_OK) s = col_fwd(c, T, IN_COMPLEX, 0, S, batch * P.M0, (int)L[1], P.Lp, P.outer[1], st, 0, tc);
  return s;
}

// Backward outer passes from the outer spectra S to the real result.
// Backward outer passes from the outer spectra S (rows of Kp = ceil(K_last/2)
// packed values) to the real result of extents K (K = L: the first L
// outputs per dimension).
static hd_status rcm_nd_backward(hd_ctx* c, int d, const int64_t* K, int64_t batch, const RcmNdPlan& P,
                                 const float2* S, float2* T, float* z, int out_mode, cudaStream_t st, bool tc) {
  const int Kn = (int)K[d - 1];
  const int64_t Kp = (K[d - 1] + 1) / 2;
  if (d == 2)
    return col_bwd(c, S, z, out_mode, Kn, batch, (int)K[0], Kp, P.outer[0], 1.0f / (float)P.M0, st, 0, tc);
  hd_status s =
      col_bwd(c, S, T, OUT_COMPLEX, 0, batch * P.M0, (int)K[1], Kp, P.outer[1], 1.0f / (float)P.M1, st, 0, tc);
  if (s == HD_OK)
    s = col_bwd(c, T, z, out_mode, Kn, batch, (int)K[0], K[1] * Kp, P.outer[0], 1.0f / (float)P.M0, st, Kp, tc);
  return s;
}

static RowGeom rcm_row_geom(int d, int64_t batch, const RcmNdPlan& P, int64_t Kp = 0) {
  RowGeom rg;
  std::memset(&rg, 0, sizeof(rg));
  rg.rpi = (int)(P.M0 * P.M1);
  rg.nrows = (int)(batch * P.M0 * P.M1);
  rg.Lrow = (int)P.Lp;
  rg.Kout = (int)(Kp > 0 ? Kp : P.Lp);
  rg.m = P.row.m;
  rg.q = P.row.q;
  rg.p = P.row.p;
  rg.nd = d - 1;
  rg.om[0] = P.outer[0].m;
  rg.oq[0] = P.outer[0].q;
  if (d == 3) {
    rg.om[1] = P.outer[1].m;
    rg.oq[1] = P.outer[1].q;
  }
  return rg;
}

// hybridRCM in 2D/3D (Sec. 5) for `batch` problems stored back to back: outer
// forward passes of f and g, C_1 on every row pair, outer backward passes.
// K: output extents (nullptr: K = L; the first L outputs per dimension).
static hd_status hybrid_rcm_nd(hd_ctx* c, int d, const int64_t* L, const hd_dim_params* prm, const float* f,
                               const float* g, float* h, cudaStream_t st, bool tc = false, int64_t batch = 1,
                               const int64_t* K = nullptr) {
  if (!K) K = L;
  RcmNdPlan P;
  hd_status s = rcm_nd_plan(c, d, L, prm, &P, st, !tc, !tc);
  if (s != HD_OK) return s;
  const int64_t Kp = (K[d - 1] + 1) / 2;
  const bool ext = Kp != P.Lp;  // longer rows: the row pass writes a separate buffer
  // scratch: F, G spectra [batch][M0][M1][Lp], the row pass's output [..][Kp]
  // when K > L, and (3D) the intermediates [batch][M0][max(L1, K1)][max(Lp, Kp)]
  const int64_t spec = batch * P.M0 * P.M1 * P.Lp;
  const int64_t out = ext ? batch * P.M0 * P.M1 * Kp : 0;
  const int64_t mid = d == 3 ? batch * P.M0 * std::max(L[1], K[1]) * std::max(P.Lp, Kp) : 0;
  if (ensure_ws(c, sizeof(float2) * (size_t)(2 * spec + out + 2 * mid), st) != HD_OK) return HD_ENOMEM;
  float2* SF = reinterpret_cast<float2*>(c->ws);
  float2* SG = SF + spec;
  float2* SO = ext ? SG + spec : SF;
  float2* TF = SG + spec + out;
  float2* TG = TF + mid;
  s = rcm_nd_forward(c, d, L, batch, P, f, IN_PACKED_REAL, SF, TF, st, tc);
  if (s == HD_OK) s = rcm_nd_forward(c, d, L, batch, P, g, IN_PACKED_REAL, SG, TG, st, tc);
  if (s != HD_OK) return s;
  // rows: C_1 on each row pair; arrays per residue step: {A, C, B, D} x (1 or
  // 2 residues); with q <= 2 every residue is its own partner, so 4
  const RowGeom rg = rcm_row_geom(d, batch, P, Kp);
  if (!tc && P.row.q <= 2 && rows_cl_length(P.row.m) && (P.row.q == 2 || 2 * Kp <= 2 * P.row.m)) {
    hd_status terr = HD_OK;
    const float2* tab = c->tables.get_pass_table(P.row.m, st, &terr);
    if (!tab) return terr;
    if (P.row.q == 1)
      HD_TRY(launch_rows_cl1(P.row.m, (unsigned)rg.nrows, st, SF, SG, SO, rg, 1.0f / (float)P.row.m, tab));
    else
      HD_TRY(launch_rows_cl(P.row.m, (unsigned)rg.nrows, st, SF, SG, SO, rg, 1.0f / (float)(P.row.q * P.row.m),
                            P.row.tw, tab));
    return rcm_nd_backward(c, d, K, batch, P, SO, TF, h, OUT_UNPACK_REAL, st, tc);
  }
  const int narr = P.row.q <= 2 ? 4 : 8;
  const Eng reng = pick_eng(tc, struct_length(P.row.m) && P.row.q <= 2);
  const size_t smem = sizeof(float2) * ((size_t)acc_slots(2 * (int)Kp) + narr * (size_t)P.row.m);
  if (smem > (size_t)c->max_smem || narr * (int64_t)P.row.m > max_points(reng)) return HD_EUNSUPPORTED;
  const int T = eng_threads(reng, narr * (int64_t)P.row.m);
  HD_TRY(launch_rows_rcm(reng, (unsigned)rg.nrows, T, smem, st, SF, SG, SO, rg, 1.0f / (float)(P.row.q * P.row.m),
                         P.row.tw, P.row.pl));
  return rcm_nd_backward(c, d, K, batch, P, SO, TF, h, OUT_UNPACK_REAL, st, tc);
}

// The adjoint of hybridRCM 2D/3D for `batch` problems: U = outer spectra of
// rev(grad_h) (the reversal folded into the first pass's loads), F and G the
// outer spectra of f and g; one row pass forms U's row transforms once and
// applies C_1 to (U, G) and (U, F); the backward passes write grad_f =
// rev(conv(rev(grad_h), g)) and grad_g = rev(conv(rev(grad_h), f)), the
// reversal folded into the last pass's stores.  Nothing is stored from the
// forward call.
hd_status adjoint_rcm_nd(hd_ctx* c, int d, const int64_t* L, int64_t batch, const float* u, const float* f,
                         const float* g, float* gf, float* gg, cudaStream_t st) {
  RcmNdPlan P;
  hd_status s = rcm_nd_plan(c, d, L, nullptr, &P, st, true);
  if (s != HD_OK) return s;
  const int64_t spec = batch * P.M0 * P.M1 * P.Lp;
  const int64_t mid = d == 3 ? batch * P.M0 * L[1] * P.Lp : 0;
  if (ensure_ws(c, sizeof(float2) * (size_t)(3 * spec + mid), st) != HD_OK) return HD_ENOMEM;
  float2* SU = reinterpret_cast<float2*>(c->ws);
  float2* SF = SU + spec;
  float2* SG = SF + spec;
  float2* TM = SG + spec;  // 3D intermediate, reused by every pass
  // Both gradients: SG <- g, SF <- f.  One gradient: its source (g for
  // grad_f, f for grad_g) goes to SG, SF aliases SG and only G is written.
  const bool both = gf && gg;
  s = rcm_nd_forward(c, d, L, batch, P, u, IN_PACKED_REAL_REV, SU, TM, st, false);
  if (s == HD_OK) s = rcm_nd_forward(c, d, L, batch, P, gf ? g : f, IN_PACKED_REAL, SG, TM, st, false);
  if (s == HD_OK && both) s = rcm_nd_forward(c, d, L, batch, P, f, IN_PACKED_REAL, SF, TM, st, false);
  if (!both) SF = SG;
  if (s != HD_OK) return s;
  const RowGeom rg = rcm_row_geom(d, batch, P);
  const int outs = both ? 3 : 1;
  if (P.row.q == 2 && rows_cl_length(P.row.m)) {
    hd_status terr = HD_OK;
    const float2* tab = c->tables.get_pass_table(P.row.m, st, &terr);
    if (!tab) return terr;
    HD_TRY(launch_rows_adj_cl(P.row.m, (unsigned)rg.nrows, st, SF, SG, SU, rg, 1.0f / (float)(P.row.q * P.row.m),
                              outs, P.row.tw, tab));
  } else {
  const int narr = P.row.q <= 2 ? 6 : 12;  // {U, F, G} x {row, partner} x residues
  const Eng reng = pick_eng(false, struct_length(P.row.m) && P.row.q <= 2);
  const size_t smem = sizeof(float2) * ((size_t)acc_slots(4 * (int)P.Lp) + narr * (size_t)P.row.m);
  if (smem > (size_t)c->max_smem || narr * (int64_t)P.row.m > max_points(reng)) return HD_EUNSUPPORTED;
  const int T = eng_threads(reng, narr * (int64_t)P.row.m);
  HD_TRY(launch_rows_adj(reng, (unsigned)rg.nrows, T, smem, st, SF, SG, SU, rg, 1.0f / (float)(P.row.q * P.row.m),
                         outs, P.row.tw, P.row.pl));
  }
  if (gf) s = rcm_nd_backward(c, d, L, batch, P, SG, TM, gf, OUT_UNPACK_REAL_REV, st, false);
  if (s == HD_OK && gg) s = rcm_nd_backward(c, d, L, batch, P, both ? SF : SG, TM, gg, OUT_UNPACK_REAL_REV, st, false);
  return s;
}

// mid: the combined CS+RCM form (hybrid_csrcm_nd) — only the residues strictly
// between 0 and q0/2 of the first dimension, plus the period-2m0 convolution of
// residues 0 and q0/2 added in the last pass; (m0, q0) then come from the caller.
static hd_status hybrid_cs_nd(hd_ctx* c, int d, const int64_t* L, const hd_dim_params* prm, const float* f,
                              const float* g, float* h, cudaStream_t st, const CsMid* only_mid = nullptr) {
  // first dimension: real residues (CS); middle (3D): complex hybrid; rows: complex conv
  const int64_t B0 = d == 2 ? L[1] : L[1] * L[2];  // real columns of the first pass
  int64_t m0, q0;
  if (prm && prm[0].m > 0) {
    m0 = prm[0].m;
    q0 = prm[0].q > 0 ? prm[0].q : (2 * L[0] - 1 + m0 - 1) / m0;
    if (q0 * m0 < 2 * L[0] - 1 || (!only_mid && q0 % 2 == 0 && m0 % 2 == 1)) return HD_EINVAL;
  } else {
    m0 = ladder_ceil(L[0]);
    while (m0 % 2) m0 = ladder_ceil(m0 + 1);
    q0 = 2;
  }
  const CsMid md = only_mid ? *only_mid : CsMid{0, nullptr, 1, 0, 0.f};
  // residue 0 pairs columns through an even-length real DFT (not run in the mid form)
  if (m0 % 2 && !md.only) return HD_EUNSUPPORTED;
  const int p0 = (int)((L[0] + m0 - 1) / m0);
  FftPlan pm0, ph0;
  factor_radices((int)m0, &pm0);
  factor_radices((int)std::max<int64_t>(1, m0 / 2), &ph0);
  hd_status terr = HD_OK;
  const float2* tw0 = c->tables.get(q0 * m0, st, &terr);
  if (!tw0) return terr;
  const int R0 = md.only ? (int)(((q0 + 1) / 2 - 1) * m0) : cs_rows((int)m0, (int)q0);
  ColPass mid, row;
  hd_status s = HD_OK;
  if (d == 3) {
    s = outer_params(c, L[1], prm ? &prm[1] : nullptr, &mid, st);
    if (s != HD_OK) return s;
  }
  s = row_params(c, L[d - 1], false, prm ? &prm[d - 1] : nullptr, &row, st);
  if (s != HD_OK) return s;
  const int64_t M1 = d == 3 ? (int64_t)mid.q * mid.m : 1;
  const int64_t Lr = L[d - 1];
  const int64_t rowsz = (d == 3 ? M1 : 1) * Lr;  // complex elements per first-dim row of the spectra
  const int64_t spec = (int64_t)R0 * rowsz;
  const int64_t tmp = d == 3 ? (int64_t)R0 * L[1] * Lr : 0;
  if (ensure_ws(c, sizeof(float2) * (size_t)(2 * spec + 2 * tmp), st) != HD_OK) return HD_ENOMEM;
  float2* SF = reinterpret_cast<float2*>(c->ws);
  float2* SG = SF + spec;
  float2* TF = SG + spec;
  float2* TG = TF + tmp;
  // first dimension: real columns (W even); the structured engine needs both
  // the length-m residue-0 DFT and the length-m/2 residue-q/2 DFT on the ladder
  const Eng eng0 = pick_eng(false, q0 == 2 && struct_length((int)m0) && struct_length((int)(m0 / 2)));
  const size_t per_col0 = sizeof(float) * (size_t)L[0] + sizeof(float2) * (size_t)m0 + 16;
  const int W0 = choose_W(per_col0, (int)m0, 1, B0, (size_t)c->max_smem, true, max_points(eng0), c->num_sms);
  const size_t smem0 = sizeof(float2) * ((size_t)acc_slots((W0 * (int)L[0] + 1) / 2) + (size_t)W0 * m0);
  if (smem0 > (size_t)c->max_smem || (int64_t)W0 * m0 > max_points(eng0)) return HD_EUNSUPPORTED;
  const int T0 = eng_threads(eng0, (int64_t)W0 * m0);
  const unsigned grid0 = (unsigned)((B0 + W0 - 1) / W0);
  {
    float2* outF = d == 3 ? TF : SF;
    float2* outG = d == 3 ? TG : SG;
    HD_TRY(launch_col_fwd_cs(eng0, grid0, T0, smem0, st, f, outF, B0, W0, (int)L[0], (int)m0, (int)q0, p0, tw0, pm0,
               ph0, md));
    HD_TRY(launch_col_fwd_cs(eng0, grid0, T0, smem0, st, g, outG, B0, W0, (int)L[0], (int)m0, (int)q0, p0, tw0, pm0,
               ph0, md));
  }
  if (d == 3) {
    s = col_fwd(c, TF, IN_COMPLEX, 0, SF, R0, (int)L[1], Lr, mid, st);
    if (s == HD_OK) s = col_fwd(c, TG, IN_COMPLEX, 0, SG, R0, (int)L[1], Lr, mid, st);
    if (s != HD_OK) return s;
  }
  {
    const int64_t nrows = (int64_t)R0 * (d == 3 ? M1 : 1);
    const Eng reng = pick_eng(false, struct_length(row.m) && row.q <= 2);
    const size_t smem = sizeof(float2) * ((size_t)acc_slots((int)Lr) + 2 * (size_t)row.m);
    if (smem > (size_t)c->max_smem || 2 * (int64_t)row.m > max_points(reng)) return HD_EUNSUPPORTED;
    const int T = eng_threads(reng, 2 * (int64_t)row.m);
    HD_TRY(launch_rows_cconv(reng, (unsigned)nrows, T, smem, st, SF, SG, (int)Lr, row.m, row.q, row.p,
               1.0f / (float)(row.q * row.m), row.tw, row.pl));
  }
  if (d == 3) {
    s = col_bwd(c, SF, TF, OUT_COMPLEX, 0, R0, (int)L[1], Lr, mid, 1.0f / (float)M1, st);
    if (s != HD_OK) return s;
  }
  {
    const float2* src = d == 3 ? TF : SF;
    HD_TRY(launch_col_bwd_cs(eng0, grid0, T0, smem0, st, src, h, B0, W0, (int)L[0], (int)m0, (int)q0,
               1.0f / (float)(q0 * m0), tw0, pm0, ph0, md));
  }
  return HD_OK;
}

// Fold modulo P along the first dimension: out[s][b] = sum_t in[t P + s][b], s < P.
__global__ void k_fold_first(const float* __restrict__ in, float* __restrict__ out, int64_t L0, int64_t P, int64_t B) {
  const int64_t total = P * B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / B, b = i - s * B;
    float acc = 0.f;
    for (int64_t j = s; j < L0; j += P) acc += in[j * B + b];
    out[i] = acc;
  }
}

// The combined CS+RCM algorithm in 2D/3D (Sec. 6.3): hybridCS along the first
// dimension with (m0, q0), q0 m0 >= 2 L0 - 1.  For even q0, residues 0 and
// q0/2 of that dimension together are the convolution of period P = 2 m0 (in
// the first dimension; linear, truncated, in the others) of the arrays folded
// modulo 2 m0: even frequencies of the length-2m0 transform are residue 0, odd
// ones residue q0/2 (Eq. resq2 with the blocks t split by parity); for odd q0,
// residue 0 alone is the period-m0 convolution of the arrays folded modulo m0
// (Sec. 3.1.1).  That part is computed by implicit packing, the hybridRCM
// recursion (packed rows, C_1 within each residue), as the linear convolution
// of the folded arrays (first-dimension extent 2P - 1) folded back;
// residues 1..ceil(q0/2)-1 run through hybridCS's complex path, and the last
// pass adds (2 / q0, or 1 / q0 for odd q0) times the period-P result.  With
// q0 = 2 there is no other residue and the arrays need no folding: the call is
// the hybridRCM recursion with (m0, 2) along the first dimension.
static hd_status hybrid_csrcm_nd(hd_ctx* c, int d, const int64_t* L, const hd_dim_params* prm, const float* f,
                                 const float* g, float* h, cudaStream_t st) {
  int64_t m0, q0;
  if (prm && prm[0].m > 0) {
    m0 = prm[0].m;
    q0 = prm[0].q > 0 ? prm[0].q : (2 * L[0] - 1 + m0 - 1) / m0;
    if (q0 * m0 < 2 * L[0] - 1) return fail(HD_EINVAL, "hybridCSRCM needs q m >= 2L-1 in the first dimension");
  } else {
    m0 = ladder_ceil(L[0]);
    q0 = 2;
  }
  hd_dim_params pr[3] = {};
  for (int i = 1; i < d; ++i) pr[i] = prm ? prm[i] : hd_dim_params{0, 0};
  if (q0 <= 2) {
    pr[0] = hd_dim_params{(int32_t)m0, 2};
    const bool user = prm != nullptr;
    return hybrid_rcm_nd(c, d, L, user ? pr : nullptr, f, g, h, st, false, 1, L);
  }
  // q0 even: residues 0 and q0/2 (period 2 m0); q0 odd: residue 0 alone (period m0)
  const bool even = q0 % 2 == 0;
  const int64_t P = even ? 2 * m0 : m0;
  const int64_t B = d == 2 ? L[1] : L[1] * L[2];
  const int64_t Lf[3] = {P, L[1], d == 3 ? L[2] : 1};
  const int64_t Kf[3] = {2 * P - 1, L[1], d == 3 ? L[2] : 1};
  // scratch: the two folded arrays and the linear convolution of period extent
  const size_t nfold = (size_t)(P * B), nlin = (size_t)((2 * P - 1) * B);
  float* tmp = nullptr;
  if (cudaMallocAsync(&tmp, sizeof(float) * (2 * nfold + nlin), st) != cudaSuccess)
    return fail(HD_ENOMEM, "hybridCSRCM scratch");
  float* ff = tmp;
  float* fg = tmp + nfold;
  float* lin = tmp + 2 * nfold;
  const int blocks = (int)std::min<int64_t>((int64_t)(nfold + 255) / 256, 148 * 32);
  k_fold_first<<<blocks, 256, 0, st>>>(f, ff, L[0], P, B);
  k_fold_first<<<blocks, 256, 0, st>>>(g, fg, L[0], P, B);
  hd_status s = HD_OK;
  if (cudaGetLastError() != cudaSuccess) s = fail(HD_ECUDA, "hybridCSRCM fold launch");
  if (s == HD_OK) {
    hd_dim_params pf[3] = {hd_dim_params{(int32_t)m0, even ? 4 : 2}, pr[1], pr[2]};  // q m >= 2 P - 1
    s = hybrid_rcm_nd(c, d, Lf, prm ? pf : nullptr, ff, fg, lin, st, false, 1, Kf);
  }
  if (s == HD_OK) {
    const CsMid mid{1, lin, (int)P, (int)(2 * P - 1), (even ? 2.0f : 1.0f) / (float)q0};
    hd_dim_params pc[3] = {hd_dim_params{(int32_t)m0, (int32_t)q0}, pr[1], pr[2]};
    s = hybrid_cs_nd(c, d, L, pc, f, g, h, st, &mid);
    if (s != HD_OK) fail(s, "hybridCSRCM: the middle residues");
  }
  cudaFreeAsync(tmp, st);
  return s;
}

hd_status explicit_nd(hd_ctx* c, hd_algo algo, int d, const int64_t* Lin, const float* f, const float* g, float* h,
                      cudaStream_t st, const int64_t* Kin) {
  // padded extents: 2L per dimension (real); explicitRCM packs the last one to
  // an even packed length (Alg. 4 needs it even)
  // (each padded length is 2 x the smallest length {1, 3, 5, 9} x 2^a >= L, so
  // every DFT runs on the structured engine; any length >= 2L-1 dealiases)
  int64_t L[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) L[3 - d + i] = Lin[i];
  const bool rcm = (algo == HD_EXPLICIT_RCM);
  const int64_t Mo0 = d >= 3 ? 2 * ladder_ceil(L[0]) : 1, Mo1 = d >= 2 ? 2 * ladder_ceil(L[1]) : 1;
  int64_t n = ladder_ceil(L[2]);  // complex length of the last-dim DFT (real padded length 2n)
  if (rcm)
    while (n % 2) n = ladder_ceil(n + 1);
  const int64_t rows = Mo0 * Mo1;
  if (n > (int64_t)kPts * 1024) return HD_EUNSUPPORTED;
  const int64_t bins = rcm ? n : n + 1;                 // complex per row after the last-dim pass
  const int64_t Preal = rows * 2 * n;                   // padded real elements per array
  const int64_t spec = rows * bins;
  if (ensure_ws(c, sizeof(float) * (size_t)(2 * Preal) + sizeof(float2) * (size_t)(2 * spec), st) != HD_OK)
    return HD_ENOMEM;
  float* PF = reinterpret_cast<float*>(c->ws);
  float* PG = PF + Preal;
  float2* SF = reinterpret_cast<float2*>(PG + Preal);
  float2* SG = SF + spec;
  hd_status terr = HD_OK;
  // table for the last dimension: N = 2n (covers zeta_{2n} for U and zeta_n)
  const float2* twl = c->tables.get(2 * n, st, &terr);
  if (!twl) return terr;
  FftPlan pln;
  factor_radices((int)n, &pln);
  // 1) materialised zero padding
  {
    const int64_t tot = rows * (rcm ? n : 2 * n);
    k_pad<<<elementwise_blocks(tot), 256, 0, st>>>(f, PF, 3, L[0], L[1], L[2], Mo0, Mo1, rcm ? n : 2 * n, rcm ? 1 : 0);
    k_pad<<<elementwise_blocks(tot), 256, 0, st>>>(g, PG, 3, L[0], L[1], L[2], Mo0, Mo1, rcm ? n : 2 * n, rcm ? 1 : 0);
  }
  // 2) last dimension
  const Eng reng = pick_eng(false, struct_length((int)n));
  const int T = eng_threads(reng, n);
  const size_t smem = sizeof(float2) * (size_t)n;
  for (int a = 0; a < 2; ++a) {
    RowsIO io;
    std::memset(&io, 0, sizeof(io));
    io.src = a ? (const void*)PG : (const void*)PF;
    io.dst = a ? SG : SF;
    io.src_stride = rcm ? n : 2 * n;
    io.dst_stride = bins;
    HD_TRY(launch_rows_fft(reng, (unsigned)rows, T, smem, st, io, rcm ? 2 : 0, (int)n, twl, 2, pln));
  }
  // 3) outer dimensions: full-length complex DFTs (q = 1, m = 2L)
  ColPass cp[2];
  const int nouter = d - 1;
  for (int i = 0; i < nouter; ++i) {
    const int64_t Mi = (i == 0) ? (d == 3 ? Mo0 : Mo1) : Mo1;
    cp[i].m = (int)Mi;
    cp[i].q = 1;
    cp[i].p = 1;
    factor_radices((int)Mi, &cp[i].pl);
    cp[i].tw = c->tables.get(Mi, st, &terr);
    if (!cp[i].tw) return terr;
  }
  hd_status s = HD_OK;
  if (d == 2) {
    for (int a = 0; a < 2 && s == HD_OK; ++a) {
      float2* S = a ? SG : SF;
      s = col_fwd(c, S, IN_COMPLEX, 0, S, 1, (int)Mo1, bins, cp[0], st);
    }
  } else if (d == 3) {
    for (int a = 0; a < 2 && s == HD_OK; ++a) {
      float2* S = a ? SG : SF;
      s = col_fwd(c, S, IN_COMPLEX, 0, S, 1, (int)Mo0, Mo1 * bins, cp[0], st);
      if (s == HD_OK) s = col_fwd(c, S, IN_COMPLEX, 0, S, Mo0, (int)Mo1, bins, cp[1], st);
    }
  }
  if (s != HD_OK) return s;
  // 4) product
  if (rcm) {
    k_rcm_nd<<<elementwise_blocks(spec), 256, 0, st>>>(SF, SG, Mo0, Mo1, n, twl, 2);
  } else {
    k_pointwise<<<elementwise_blocks(spec), 256, 0, st>>>(SF, SG, spec);
  }
  // 5) outer inverse
  if (d == 2) {
    s = col_bwd(c, SF, SF, OUT_COMPLEX, 0, 1, (int)Mo1, bins, cp[0], 1.0f, st);
  } else if (d == 3) {
    s = col_bwd(c, SF, SF, OUT_COMPLEX, 0, Mo0, (int)Mo1, bins, cp[1], 1.0f, st);
    if (s == HD_OK) s = col_bwd(c, SF, SF, OUT_COMPLEX, 0, 1, (int)Mo0, Mo1 * bins, cp[0], 1.0f, st);
  }
  if (s != HD_OK) return s;
  // 6) last dimension inverse, unpack, crop, scale 1 / prod(M)
  {
    RowsIO io;
    std::memset(&io, 0, sizeof(io));
    io.src = SF;
    io.dst = h;
    io.src_stride = bins;
    // outputs kept per dimension: K (default L), 2L-1 at most, within the padded 2 ladder(L)
    int64_t K[3] = {1, 1, 1};
    for (int i = 0; i < d; ++i) K[3 - d + i] = Kin ? Kin[i] : Lin[i];
    io.Lkeep = (int)K[2];
    io.crop_rows_outer[0] = Mo0;
    io.crop_rows_outer[1] = Mo1;
    io.keep_rows_outer[0] = K[0];
    io.keep_rows_outer[1] = K[1];
    // the unnormalised inverse returns n Mo0 Mo1 times the convolution, for
    // both the real (pack after U^{-1}) and the packed (RCM) forms
    io.scale = (float)(1.0 / ((double)Mo0 * (double)Mo1 * (double)n));
    HD_TRY(launch_rows_fft(reng, (unsigned)rows, T, smem, st, io, rcm ? 3 : 1, (int)n, twl, 2, pln));
  }
  return HD_OK;
}

}  // namespace hd

using namespace hd;

namespace hd {
// hybridRCM 2D/3D over a batch of equal-size problems (one pass sequence).
hd_status conv_nd_batch_rcm(hd_ctx* c, int d, const int64_t* L, int64_t batch, const float* f, const float* g,
                            float* h, cudaStream_t st) {
  return hybrid_rcm_nd(c, d, L, nullptr, f, g, h, st, false, batch);
}
}  // namespace hd

namespace hd {
// 2D/3D with output extents K (validated by the caller: L <= K <= 2L-1).
hd_status conv_nd_ext(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int d,
                      const int64_t* L, const int64_t* K, const hd_dim_params* prm, cudaStream_t st) {
  for (int i = 0; i < d; ++i)
    if (L[i] > (1 << 20)) return fail(HD_EUNSUPPORTED, "L too large");
  bool full = false;
  for (int i = 0; i < d; ++i) full = full || K[i] != L[i];
  // split precision: the radix-16 passes of hybridRCM's 2D/3D kernels on tensor cores
  if (prec == HD_SPLIT_BF16 && algo != HD_HYBRID_RCM) return fail(HD_EUNSUPPORTED, "split precision: hybridRCM only");
  if (prec == HD_SPLIT_FP16) return fail(HD_EUNSUPPORTED, "split precision: bfloat16 only (half precision range)");
  if (prec != HD_FP32 && prec != HD_SPLIT_BF16) return fail(HD_EINVAL, "unknown precision");
  switch (algo) {
    case HD_HYBRID_RCM: return hybrid_rcm_nd(c, d, L, prm, f, g, h, st, prec == HD_SPLIT_BF16, 1, K);
    case HD_HYBRID_CS:
      if (full) return fail(HD_EUNSUPPORTED, "hybridCS in 2D/3D returns the first L outputs only");
      return hybrid_cs_nd(c, d, L, prm, f, g, h, st);
    case HD_EXPLICIT:
    case HD_EXPLICIT_RCM: return explicit_nd(c, algo, d, L, f, g, h, st, K);
    case HD_HYBRID_CSRCM:
      if (full) return fail(HD_EUNSUPPORTED, "hybridCSRCM in 2D/3D returns the first L outputs only");
      if (prec != HD_FP32) return fail(HD_EUNSUPPORTED, "hybridCSRCM: FP32 only");
      return hybrid_csrcm_nd(c, d, L, prm, f, g, h, st);
  }
  return fail(HD_EINVAL, "unknown algorithm");
}
}  // namespace hd

extern "C" {
hd_status hd_conv2d(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int64_t L1,
                    int64_t L2, const hd_dim_params* prm, void* stream) {
  const int64_t L[2] = {L1, L2};
  return hd_conv_ext(c, algo, prec, 2, L, nullptr, f, g, h, prm, stream);
}
hd_status hd_conv3d(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int64_t L1,
                    int64_t L2, int64_t L3, const hd_dim_params* prm, void* stream) {
  const int64_t L[3] = {L1, L2, L3};
  return hd_conv_ext(c, algo, prec, 3, L, nullptr, f, g, h, prm, stream);
}
}
