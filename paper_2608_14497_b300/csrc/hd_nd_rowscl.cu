// hd_nd_rowscl.cu -- instances of the row-pair kernel of hybridRCM in 2D/3D on
// the compile-time DFT engine (hd_rows_cl.cuh), residue lengths 256 R3, and
// of the adjoint's row pass.
#include "hd_rows_cl.cuh"

namespace hd {

bool rows_cl_length(int m) {
  if (m % 256) return false;
  const int R3 = m / 256;
  return R3 == 1 || R3 == 2 || R3 == 3 || R3 == 4 || R3 == 5 || R3 == 6 || R3 == 8;
}

cudaError_t launch_rows_cl(int m, unsigned grid, cudaStream_t st, float2* F, const float2* G, float2* O, RowGeom rg,
                           float scale, const float2* tw, const float2* tab) {
  switch (m / 256) {
    case 1: return rows::launch_rows<1>(grid, st, F, G, O, rg, scale, tw, tab);
    case 2: return rows::launch_rows<2>(grid, st, F, G, O, rg, scale, tw, tab);
    case 3: return rows::launch_rows<3>(grid, st, F, G, O, rg, scale, tw, tab);
    case 4: return rows::launch_rows<4>(grid, st, F, G, O, rg, scale, tw, tab);
    case 5: return rows::launch_rows<5>(grid, st, F, G, O, rg, scale, tw, tab);
    case 6: return rows::launch_rows<6>(grid, st, F, G, O, rg, scale, tw, tab);
    case 8: return rows::launch_rows<8>(grid, st, F, G, O, rg, scale, tw, tab);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rows_cl1(int m, unsigned grid, cudaStream_t st, float2* F, const float2* G, float2* O, RowGeom rg,
                            float scale, const float2* tab) {
  switch (m / 256) {
    case 1: return rows::launch_rows1<1>(grid, st, F, G, O, rg, scale, tab);
    case 2: return rows::launch_rows1<2>(grid, st, F, G, O, rg, scale, tab);
    case 3: return rows::launch_rows1<3>(grid, st, F, G, O, rg, scale, tab);
    case 4: return rows::launch_rows1<4>(grid, st, F, G, O, rg, scale, tab);
    case 5: return rows::launch_rows1<5>(grid, st, F, G, O, rg, scale, tab);
    case 6: return rows::launch_rows1<6>(grid, st, F, G, O, rg, scale, tab);
    case 8: return rows::launch_rows1<8>(grid, st, F, G, O, rg, scale, tab);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rows_adj_cl(int m, unsigned grid, cudaStream_t st, float2* F, float2* G, const float2* U,
                               RowGeom rg, float scale, int outs, const float2* tw, const float2* tab) {
  switch (m / 256) {
    case 1: return rows::launch_rows_adj<1>(grid, st, F, G, U, rg, scale, outs, tw, tab);
    case 2: return rows::launch_rows_adj<2>(grid, st, F, G, U, rg, scale, outs, tw, tab);
    case 3: return rows::launch_rows_adj<3>(grid, st, F, G, U, rg, scale, outs, tw, tab);
    case 4: return rows::launch_rows_adj<4>(grid, st, F, G, U, rg, scale, outs, tw, tab);
    case 5: return rows::launch_rows_adj<5>(grid, st, F, G, U, rg, scale, outs, tw, tab);
    case 6: return rows::launch_rows_adj<6>(grid, st, F, G, U, rg, scale, outs, tw, tab);
    case 8: return rows::launch_rows_adj<8>(grid, st, F, G, U, rg, scale, outs, tw, tab);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hd
