// kernels_bdct.cu -- block-transform tape codec (tape type 9): record,
// restore and raw-plane entry points.  The codec is defined in bdct.cuh.
//
// Record: one warp per (face, component, 8 x 8 block): the lanes stage the
// block's 64 values in shared memory (x faces are strided in memory, but a
// sample is recorded only every k steps and covers the surface only), lane i
// forms coefficient i (and i + 32) as the codec's sequential fmaf chain over
// the 64 cells, the block's absmax is a warp max (exact in any order), and
// each lane quantises its own coefficients.  Restore: one thread per recorded
// value, decoding its block's K codes for each of the (up to four) time
// samples of the interpolation; the basis values of a warp's 32 cells lie in
// one 32-byte sector per coefficient.
#include <math.h>

#include <mutex>

#include "bdct.cuh"
#include "tape_common.cuh"

namespace fdtd {

static constexpr int BDCT_THREADS = 256;
static constexpr float kBdctMinScale = 1.17549435e-38f;   // 2^-126

__device__ float g_bdct_beta[64 * 64];
__device__ float g_bdct_beta_t[64 * 64];   // transposed: [cell][coefficient]

// ------------------------------------------------------------ host side ---
void bdct_order_host(int i, int* u, int* v) {
  // diagonal s = u + v ascending, then v ascending within the diagonal
  int n = 0;
  for (int s = 0; s <= 14; ++s)
    for (int vv = 0; vv <= s; ++vv) {
      const int uu = s - vv;
      if (uu > 7 || vv > 7) continue;
      if (n == i) {
        *u = uu;
        *v = vv;
        return;
      }
      ++n;
    }
  *u = *v = 0;
}

void bdct_basis_host(float* beta) {
  const double pi = 3.14159265358979323846;
  double d[8][8];
  for (int u = 0; u < 8; ++u)
    for (int x = 0; x < 8; ++x)
      d[u][x] = (u == 0 ? sqrt(1.0 / 8.0) : 0.5) * cos((2 * x + 1) * u * pi / 16.0);
  for (int i = 0; i < 64; ++i) {
    int u, v;
    bdct_order_host(i, &u, &v);
    for (int y = 0; y < 8; ++y)
      for (int x = 0; x < 8; ++x) beta[i * 64 + y * 8 + x] = (float)(d[u][x] * d[v][y]);
  }
}

BdctLayout bdct_layout(const Faces& fc, int K) {
  BdctLayout bl;
  bl.K = K;
  bl.bstart[0] = 0;
  for (int f = 0; f < 6; ++f) {
    bl.nbu[f] = (fc.f[f].nu + 7) / 8;
    bl.nbv[f] = (fc.f[f].nv + 7) / 8;
    bl.bstart[f + 1] = bl.bstart[f] + 2 * bl.nbu[f] * bl.nbv[f];
  }
  const long long nb = bl.bstart[6];
  bl.code_bytes = (nb * K + 15) / 16 * 16;
  bl.sample_bytes = (bl.code_bytes + nb * 4 + 15) / 16 * 16;
  return bl;
}

cudaError_t bdct_ensure_basis() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  float beta[64 * 64], beta_t[64 * 64];
  bdct_basis_host(beta);
  for (int i = 0; i < 64; ++i)
    for (int t = 0; t < 64; ++t) beta_t[t * 64 + i] = beta[i * 64 + t];
  if ((e = cudaMemcpyToSymbol(g_bdct_beta, beta, sizeof beta))) return e;
  if ((e = cudaMemcpyToSymbol(g_bdct_beta_t, beta_t, sizeof beta_t))) return e;
  done[dev] = true;
  return cudaSuccess;
}

// ---------------------------------------------------------- device side ---
// Quantise one block with a warp: X (64 values, row-major, shared memory,
// visible to the warp) -> K codes and the scale.  Lane i owns coefficients i
// and i + 32.
__device__ __forceinline__ void bdct_encode_block_warp(const float* X, int K, int lane,
                                                       signed char* __restrict__ codes,
                                                       float* __restrict__ scale) {
  float c[2] = {0.f, 0.f};
  float amax = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < K) {
      float acc = 0.f;
#pragma unroll 8
      for (int t = 0; t < 64; ++t) acc = __fmaf_rn(X[t], __ldg(g_bdct_beta_t + t * 64 + i), acc);
      c[h] = acc;
      amax = fmaxf(amax, fabsf(acc));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const float s = amax > 0.f ? fmaxf(__fdiv_rn(amax, 127.0f), kBdctMinScale) : 1.0f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < K) {
      const float q = fminf(fmaxf(rintf(__fdiv_rn(c[h], s)), -127.f), 127.f);
      codes[i] = (signed char)(int)q;
    }
  }
  if (lane == 0) *scale = s;
}

// Value of cell t (y * 8 + x) of a block from its K codes and scale.
__device__ __forceinline__ float bdct_decode_cell(const signed char* __restrict__ codes, float s,
                                                  int K, int t) {
  float acc = 0.f;
  for (int i = 0; i < K; ++i)
    acc = __fmaf_rn((float)codes[i], __ldg(g_bdct_beta + i * 64 + t), acc);
  return __fmul_rn(acc, s);
}

static constexpr int BDCT_WARPS = BDCT_THREADS / 32;

__global__ void __launch_bounds__(BDCT_THREADS) k_record_bdct(const float* __restrict__ FH,
                                                              const float* __restrict__ FE, Geo g,
                                                              const __grid_constant__ Faces fc,
                                                              const __grid_constant__ BdctLayout bl,
                                                              unsigned char* __restrict__ sample) {
  __shared__ float Xs[BDCT_WARPS][64];
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
  const int b = blockIdx.x * BDCT_WARPS + wv;
  if (b >= bl.bstart[6]) return;   // whole warps
  int f = 0;
#pragma unroll
  for (int t = 1; t < 6; ++t) f += b >= bl.bstart[t];
  const FaceDesc& fd = fc.f[f];
  const int nb = bl.nbu[f] * bl.nbv[f];
  const int rb = b - bl.bstart[f];
  const int comp_t = rb >= nb;
  const int blk = rb - comp_t * nb;
  const int bv = blk / bl.nbu[f], bu = blk - bv * bl.nbu[f];
  const float* __restrict__ F = (f & 1) ? FE : FH;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h, y = t >> 3, x = t & 7;
    const int v = min(bv * 8 + y, fd.nv - 1), u = min(bu * 8 + x, fd.nu - 1);
    int comp;
    const long long q = face_value_cell(g, fd, (comp_t * fd.nv + v) * fd.nu + u, &comp);
    Xs[wv][t] = F[comp * g.nc + q];
  }
  __syncwarp();
  bdct_encode_block_warp(Xs[wv], bl.K, lane,
                         reinterpret_cast<signed char*>(sample) + (long long)b * bl.K,
                         reinterpret_cast<float*>(sample + bl.code_bytes) + b);
}

cudaError_t launch_record_bdct(const float* FH, const float* FE, Geo g, const Faces& fc,
                               const BdctLayout& bl, void* tape_sample, cudaStream_t s) {
  const int nb = bl.bstart[6];
  if (nb == 0) return cudaSuccess;
  k_record_bdct<<<(nb + BDCT_WARPS - 1) / BDCT_WARPS, BDCT_THREADS, 0, s>>>(
      FH, FE, g, fc, bl, reinterpret_cast<unsigned char*>(tape_sample));
  return cudaGetLastError();
}

// Restore: value r of the sample (as in the other tape types) is
// sum_m w[m] * decode(sample slot[m]); then the detector blocks seed the
// adjoint.
__global__ void __launch_bounds__(BDCT_THREADS) k_restore_seed_bdct(
    float* __restrict__ F, float* __restrict__ L, Geo g, const __grid_constant__ Faces fc,
    const __grid_constant__ BdctLayout bl, const unsigned char* __restrict__ tape,
    long long stride, const __grid_constant__ Interp ip, Det det, Det det2,
    const double* __restrict__ seeds, int face_blocks, int det_blocks) {
  if ((int)blockIdx.x < face_blocks) {
    const int r = blockIdx.x * BDCT_THREADS + threadIdx.x;
    if (r >= fc.start[6]) return;
    int f = 0;
#pragma unroll
    for (int t = 1; t < 6; ++t) f += r >= fc.start[t];
    const FaceDesc& fd = fc.f[f];
    const int rr = r - fc.start[f];
    const int row = rr / fd.nu, u = rr - row * fd.nu;
    const int comp_t = row >= fd.nv, v = row - comp_t * fd.nv;
    const int bu = u >> 3, bv = v >> 3;
    const int b = bl.bstart[f] + comp_t * bl.nbu[f] * bl.nbv[f] + bv * bl.nbu[f] + bu;
    const int t = (v & 7) * 8 + (u & 7);
    const int fld = f & 1;  // 0: Ht on low faces, 1: E on high faces
    float val = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int s = ip.slot[fld][m];
      if (s >= 0) {
        const unsigned char* smp = tape + (long long)s * stride;
        const float sc = __ldg(reinterpret_cast<const float*>(smp + bl.code_bytes) + b);
        const float x =
            bdct_decode_cell(reinterpret_cast<const signed char*>(smp) + (long long)b * bl.K, sc,
                             bl.K, t);
        val += ip.w[fld][m] * x;
      }
    }
    int comp;
    const long long q = face_value_cell(g, fd, rr, &comp);
    F[comp * g.nc + q] = val;
    return;
  }
  seed_detectors(F, L, g, det, det2, seeds, blockIdx.x - face_blocks, det_blocks);
}

cudaError_t launch_restore_seed_bdct(float* F, float* L, Geo g, const Faces& fc,
                                     const BdctLayout& bl, const void* tape, long long stride,
                                     const Interp& ip, const Det& det, const Det& det2,
                                     const double* seeds, cudaStream_t s) {
  const int face_blocks = (fc.start[6] + BDCT_THREADS - 1) / BDCT_THREADS;
  int dmax = det.kind ? (det.u1 - det.u0) * (det.v1 - det.v0) : 0;
  if (det2.kind) dmax = max(dmax, (det2.u1 - det2.u0) * (det2.v1 - det2.v0));
  const int det_blocks = (dmax + BDCT_THREADS - 1) / BDCT_THREADS;
  const int blocks = face_blocks + (det2.kind ? 2 : 1) * det_blocks;
  if (blocks == 0) return cudaSuccess;
  k_restore_seed_bdct<<<blocks, BDCT_THREADS, 0, s>>>(
      F, L, g, fc, bl, reinterpret_cast<const unsigned char*>(tape), stride, ip, det, det2, seeds,
      face_blocks, det_blocks);
  return cudaGetLastError();
}

// ------------------------------------------------------ raw plane codec ---
__global__ void __launch_bounds__(BDCT_THREADS) k_bdct_encode(const float* __restrict__ in, int nu,
                                                              int nv, int K,
                                                              signed char* __restrict__ codes,
                                                              float* __restrict__ scales) {
  __shared__ float Xs[BDCT_WARPS][64];
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
  const int nbu = (nu + 7) / 8, nbv = (nv + 7) / 8;
  const int b = blockIdx.x * BDCT_WARPS + wv;
  if (b >= nbu * nbv) return;   // whole warps
  const int bv = b / nbu, bu = b - bv * nbu;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h, y = t >> 3, x = t & 7;
    const int v = min(bv * 8 + y, nv - 1), u = min(bu * 8 + x, nu - 1);
    Xs[wv][t] = in[(long long)v * nu + u];
  }
  __syncwarp();
  bdct_encode_block_warp(Xs[wv], K, lane, codes + (long long)b * K, scales + b);
}

__global__ void __launch_bounds__(BDCT_THREADS) k_bdct_decode(const signed char* __restrict__ codes,
                                                              const float* __restrict__ scales,
                                                              int nu, int nv, int K,
                                                              float* __restrict__ out) {
  const long long r = blockIdx.x * (long long)BDCT_THREADS + threadIdx.x;
  if (r >= (long long)nu * nv) return;
  const int v = (int)(r / nu), u = (int)(r - (long long)v * nu);
  const int nbu = (nu + 7) / 8;
  const int b = (v >> 3) * nbu + (u >> 3);
  out[r] = bdct_decode_cell(codes + (long long)b * K, __ldg(scales + b), K, (v & 7) * 8 + (u & 7));
}

cudaError_t launch_bdct_encode(const float* in, int nu, int nv, int K, signed char* codes,
                               float* scales, cudaStream_t s) {
  const long long nb = (long long)((nu + 7) / 8) * ((nv + 7) / 8);
  k_bdct_encode<<<(unsigned)((nb + BDCT_WARPS - 1) / BDCT_WARPS), BDCT_THREADS, 0, s>>>(
      in, nu, nv, K, codes, scales);
  return cudaGetLastError();
}

cudaError_t launch_bdct_decode(const signed char* codes, const float* scales, int nu, int nv,
                               int K, float* out, cudaStream_t s) {
  const long long n = (long long)nu * nv;
  k_bdct_decode<<<(unsigned)((n + BDCT_THREADS - 1) / BDCT_THREADS), BDCT_THREADS, 0, s>>>(
      codes, scales, nu, nv, K, out);
  return cudaGetLastError();
}

}  // namespace fdtd
