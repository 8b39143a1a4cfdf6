// bdct.cuh -- block-transform tape codec (tape type 9).
//
// Beyond the paper (Sec. 4 names JPEG-like compression of the boundary tape
// as future work): every face component [v][u] of a tape sample is cut into
// 8 x 8 blocks (cells past the face edge repeat the last row / column), each
// block goes through the orthonormal 2D DCT-II, and the first K coefficients
// in diagonal order (u + v ascending, then v ascending) are kept as int8
// codes round(C / s) with one float32 scale s = max(max|C| / 127, 2^-126) per
// block (1 for an all-zero block).  Everything runs in float32 in a fixed
// order (fmaf over the block's cells row by row, then over the kept
// coefficients in order) so that an independent implementation gives the
// same codes and values bit for bit.
//
// Sample layout: int8 codes [face][comp][block][K] padded to 16 bytes, then
// float32 scales [face][comp][block]; blocks row-major over (bv, bu).
#pragma once

#include "fdtd_internal.cuh"

namespace fdtd {

constexpr int kTapeBdct = 9;
constexpr int kBdctDefaultCoeffs = 10;   // the diagonals u + v <= 3

struct BdctLayout {
  int K;                 // coefficients kept per block
  int nbu[6], nbv[6];    // blocks per face along u and v
  int bstart[7];         // first block of each face (two components each)
  long long code_bytes;  // codes of one sample, padded to 16 bytes
  long long sample_bytes;
};

// Basis table: beta[i * 64 + y * 8 + x] = float(d_u[x] d_v[y]) for the i-th
// coefficient (u, v) in diagonal order, d_u[x] = c_u cos((2x + 1) u pi / 16),
// c_0 = sqrt(1/8), c_u = 1/2; computed in double on the host.
void bdct_basis_host(float* beta);
// (u, v) of the i-th coefficient in diagonal order.
void bdct_order_host(int i, int* u, int* v);
BdctLayout bdct_layout(const Faces& fc, int K);

// Upload the basis table to the device once per device (host-synchronous;
// call outside stream capture).
cudaError_t bdct_ensure_basis();

cudaError_t launch_record_bdct(const float* FH, const float* FE, Geo g, const Faces& fc,
                               const BdctLayout& bl, void* tape_sample, cudaStream_t s);
cudaError_t launch_restore_seed_bdct(float* F, float* L, Geo g, const Faces& fc,
                                     const BdctLayout& bl, const void* tape, long long stride,
                                     const Interp& ip, const Det& det, const Det& det2,
                                     const double* seeds, cudaStream_t s);
cudaError_t launch_bdct_encode(const float* in, int nu, int nv, int K, signed char* codes,
                               float* scales, cudaStream_t s);
cudaError_t launch_bdct_decode(const signed char* codes, const float* scales, int nu, int nv,
                               int K, float* out, cudaStream_t s);

}  // namespace fdtd
