// fdtd_internal.cuh -- device data layout and helpers shared by the kernels.
//
// Layout in HBM (all float32 unless noted, x fastest, rows padded to px):
//   fields   F[6][nz][ny][px]       Ex Ey Ez Hx Hy Hz   (E, Ht = eta0 H)
//   cb       [nz][ny][px]           S / eps_r
//   psi set  per axis [4][nz][ny][px] (convolutional-PML auxiliaries; only the
//            cells of each axis' absorbing slabs are ever read or written, the
//            full-grid layout lets the TMA stage them with the field boxes);
//            the two-cells-per-thread kernels use the compact PsiLayout below
//   profiles [3 axes][6][nmax]      b_E a_E 1/kappa_E b_H a_H 1/kappa_H
// psi components per axis slab (curl term, sign):
//   x: 0 (Hy, -dEz/dx) 1 (Hz, +dEy/dx) 2 (Ey, -dHz/dx) 3 (Ez, +dHy/dx)
//   y: 0 (Hx, +dEz/dy) 1 (Hz, -dEx/dy) 2 (Ex, +dHz/dy) 3 (Ez, -dHx/dy)
//   z: 0 (Hx, -dEy/dz) 1 (Hy, +dEx/dz) 2 (Ex, -dHy/dz) 3 (Ey, +dHx/dz)
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

enum { PR_BE = 0, PR_AE = 1, PR_KE = 2, PR_BH = 3, PR_AH = 4, PR_KH = 5 };
enum { ERR_EPS = 1u, ERR_NONFINITE = 2u, ERR_TIMEOUT = 4u, ERR_LAUNCH = 8u, ERR_BOUNDS = 16u };

struct Geo {
  int nx, ny, nz, px, P, nmax;
  long long plane;  // ny * px
  long long nc;     // nz * plane (one component)
  float S;
  const float* prof;
};

// Source region: plane normal `axis` at `index`, cells (u,v) in [u0,u1)x[v0,v1),
// weights w[(v-v0)*(u1-u0) + (u-u0)] for field component `comp`.
struct Src {
  int kind, comp, axis, index, u0, u1, v0, v1;
  const float* w;
};

struct Det {
  int kind, axis, index, u0, u1, v0, v1;
};

struct FaceDesc {
  int axis, ua, va, nu, nv, layer;
  int comp0, comp1;          // field component index (0..5) of the two tangential values
  long long off;             // element offset of the face inside one tape sample
};

struct Faces {
  FaceDesc f[6];
  int start[7];              // prefix sums of the value counts (2 nu nv)
};

struct Interp {
  int slot[2][4];            // tape slot per term (-1: unused)
  float w[2][4];
};

__device__ __forceinline__ float prof(const Geo& g, int axis, int which, int i) {
  return __ldg(g.prof + ((long long)(axis * 6 + which)) * g.nmax + i);
}

__device__ __forceinline__ bool in_slab(int pos, int n, int P) { return pos < P || pos >= n - P; }

// psi component c (0..3) of axis a at cell (i, j, k): full-grid layout.
__device__ __forceinline__ long long psi_at(const Geo& g, int a, int c, int i, int j, int k) {
  return (long long)(a * 4 + c) * g.nc + (long long)k * g.plane + (long long)j * g.px + i;
}
__device__ __forceinline__ long long psi_x(const Geo& g, int c, int i, int j, int k) {
  return psi_at(g, 0, c, i, j, k);
}
__device__ __forceinline__ long long psi_y(const Geo& g, int c, int i, int j, int k) {
  return psi_at(g, 1, c, i, j, k);
}
__device__ __forceinline__ long long psi_z(const Geo& g, int c, int i, int j, int k) {
  return psi_at(g, 2, c, i, j, k);
}

// Layout of one CPML auxiliary set for the two-cells-per-thread kernels: per
// axis a (x, y, z) one array of four components [4][d2][d1][d0] that holds
// either the whole grid (full layout, d0 = px, d1 = ny, d2 = nz) or only the
// cells of that axis' two slabs (compact layout: the axis coordinate c maps
// to c below hs and to c - shift from hs on, which packs the high slab right
// after the low one).
struct PsiAxis {
  long long off;   // element offset of the axis array within the set
  long long cs;    // elements per component (d0 d1 d2)
  long long ps;    // elements per plane (d0 d1)
  int d0, d1, d2;  // array extents along x (row pitch), y, z
  int e0;          // cells along x (<= d0; the rest of a row is padding)
  int hs, shift;   // coordinate mapping along the axis
};
struct PsiLayout {
  PsiAxis ax[3];
  long long total;  // elements of the set
};

// Exact reversal: the field increment d rounded to the grid of multiples of
// 2^-xq.  Fields that start on the grid (zero) and move by grid increments
// stay on it, and while |field| < 2^(24-xq) the float32 sum of two grid
// values is exact, so the reverse step (field - the same increment) restores
// the previous value bit for bit.  Scaling by a power of two is exact.
__device__ __forceinline__ float grid_inc(float d, int xq, float xs, float xi) {
  return xq ? __fmul_rn(rintf(__fmul_rn(d, xs)), xi) : d;
}

__device__ __forceinline__ int psi_map(const PsiAxis& A, int c) {
  return c >= A.hs ? c - A.shift : c;
}

// Element index of component c of axis a's auxiliary at cell (x, y, z).
template <int AX>
__device__ __forceinline__ long long psi_ix(const PsiLayout& L, int c, int x, int y, int z) {
  const PsiAxis& A = L.ax[AX];
  const int xx = AX == 0 ? psi_map(A, x) : x;
  const int yy = AX == 1 ? psi_map(A, y) : y;
  const int zz = AX == 2 ? psi_map(A, z) : z;
  return A.off + c * A.cs + zz * A.ps + (yy * A.d0 + xx);
}

// Plane membership: p = (i, j, k); (u, v) = the two other axes in increasing order.
__device__ __forceinline__ bool on_plane(int axis, int index, int u0, int u1, int v0, int v1, int i,
                                         int j, int k, int* u, int* v) {
  int p0 = axis == 0 ? i : (axis == 1 ? j : k);
  if (p0 != index) return false;
  int uu = axis == 0 ? j : i;
  int vv = axis == 2 ? j : k;
  *u = uu;
  *v = vv;
  return uu >= u0 && uu < u1 && vv >= v0 && vv < v1;
}

// ---------------------------------------------------------------- codec ----
// Tape element types: 0 f32, 1 bf16, 2 f16, 3 e4m3 (OCP e4m3fn), 4..8 the
// software-coded 8-bit formats below.  Encoding is round-to-nearest-even with
// saturation to the largest finite value.
template <int DT> struct Code;
template <> struct Code<0> {
  typedef float T;
  static constexpr float fmax = 3.4028234663852886e38f;
  __device__ static T enc(float x) { return x; }
  __device__ static float dec(T c) { return c; }
};
template <> struct Code<1> {
  typedef __nv_bfloat16 T;
  static constexpr float fmax = 3.3895313892515355e38f;
  __device__ static T enc(float x) { return __float2bfloat16_rn(x); }
  __device__ static float dec(T c) { return __bfloat162float(c); }
};
template <> struct Code<2> {
  typedef __half T;
  static constexpr float fmax = 65504.0f;
  __device__ static T enc(float x) { return __float2half_rn(fminf(fmaxf(x, -65504.0f), 65504.0f)); }
  __device__ static float dec(T c) { return __half2float(c); }
};
template <> struct Code<3> {
  typedef __nv_fp8_storage_t T;
  static constexpr float fmax = 448.0f;
  __device__ static T enc(float x) { return __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3); }
  __device__ static float dec(T c) {
    __half_raw h = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
    return __half2float(__half(h));
  }
};

// Software codec of the 8-bit formats compared in Sec. 4 (Fig. 3) that have
// no hardware conversion: M stored mantissa bits, exponent bias BIAS, IEEE =
// the all-ones exponent encodes infinities / NaNs (else "fnuz": one NaN code
// 0x80, every other code finite, no negative zero).  Encoding saturates to
// FMAX and rounds to nearest, ties to even: below the smallest normal 2^(1-B)
// the value is an integer multiple of 2^(1-B-M) (exact power-of-two scaling,
// then a round-to-nearest-even integer conversion); above it the FP32 bit
// pattern (exponent and mantissa as one integer) is rounded at bit 23-M, a
// mantissa carry moving into the exponent, and re-biased.
__device__ __forceinline__ float pow2f(int e) {   // 2^e for normal-range e
  return __uint_as_float((uint32_t)(127 + e) << 23);
}
template <int M, int BIAS, bool IEEE>
__device__ __forceinline__ uint8_t soft8_enc(float x, float fmax) {
  const uint32_t sgn = (__float_as_uint(x) >> 24) & 0x80u;
  const float a = fminf(fabsf(x), fmax);
  uint32_t code;
  if (a < pow2f(1 - BIAS)) {
    code = __float2uint_rn(a * pow2f(BIAS + M - 1));
  } else {
    uint32_t u = __float_as_uint(a);
    constexpr int sh = 23 - M;
    u += (1u << (sh - 1)) - 1u + ((u >> sh) & 1u);
    code = (u >> sh) - ((uint32_t)(127 - BIAS) << M);
  }
  if (code == 0 && !IEEE) return 0;   // unsigned zero
  return (uint8_t)(code | sgn);
}
template <int E, int M, int BIAS, bool IEEE>
__device__ __forceinline__ float soft8_dec(uint8_t c) {
  const uint32_t mag = c & 0x7fu;
  const uint32_t ef = mag >> M, mf = mag & ((1u << M) - 1u);
  float v;
  if (ef == 0) v = (float)mf * pow2f(1 - BIAS - M);
  else v = __uint_as_float(((ef + 127u - BIAS) << 23) | (mf << (23 - M)));
  if (IEEE && ef == (1u << E) - 1u) v = mf ? __uint_as_float(0x7fc00000u) : __uint_as_float(0x7f800000u);
  if (!IEEE && c == 0x80u) return __uint_as_float(0x7fc00000u);
  return (c & 0x80u) ? -v : v;
}
template <int E, int M, int BIAS, bool IEEE, int FMAX_NUM, int FMAX_DEN>
struct Soft8 {
  typedef uint8_t T;
  static constexpr float fmax = (float)FMAX_NUM / (float)FMAX_DEN;
  __device__ static T enc(float x) { return soft8_enc<M, BIAS, IEEE>(x, fmax); }
  __device__ static float dec(T c) { return soft8_dec<E, M, BIAS, IEEE>(c); }
};
template <> struct Code<4> : Soft8<4, 3, 11, false, 30, 1> {};     // e4m3b11fnuz, max 30
template <> struct Code<5> : Soft8<5, 2, 16, false, 57344, 1> {};  // e5m2fnuz, max 57344
template <> struct Code<6> : Soft8<4, 3, 8, false, 240, 1> {};     // e4m3fnuz, max 240
template <> struct Code<7> : Soft8<4, 3, 7, true, 240, 1> {};      // e4m3 (IEEE-like), max 240
template <> struct Code<8> : Soft8<3, 4, 3, true, 31, 2> {};       // e3m4 (IEEE-like), max 15.5

constexpr int kTapeDtypes = 9;
inline int code_bytes(int dt) { return dt == 0 ? 4 : (dt <= 2 ? 2 : 1); }

// Units (32 x 8 tile, z chunk) of the staged kernels: ntx x nty tiles and nzc
// chunks.  [px0, px1) x [py0, py1) x [pz0, pz1): the units holding interior
// cells; [ix0, ix1) x [iy0, iy1) x [iz0, iz1): the units whose every cell
// and every neighbour one cell away (x in [x0-1, x0+32], y in [y0-1, y0+8],
// z in [k0-1, k1]) lies in the interior, i.e. without a CPML term.  The
// other units split into z-only units (tiles inside [ix0, ix1) x [iy0, iy1),
// chunks outside [iz0, iz1)) and ring units (every other tile, every chunk).
struct RevUnits {
  int ntx, nty, nzc;
  int px0, px1, py0, py1, pz0, pz1;
  int ix0, ix1, iy0, iy1, iz0, iz1;
};

// The chunk of z-only unit c (grid z index): below [iz0, iz1), then above.
__host__ __device__ inline int zonly_chunk(const RevUnits& U, int c) {
  return c < U.iz0 ? c : U.iz1 + (c - U.iz0);
}

__host__ __device__ inline long long ring_tiles(const RevUnits& U) {
  return (long long)U.ntx * U.nty - (long long)(U.ix1 - U.ix0) * (U.iy1 - U.iy0);
}

// Ring unit u: chunk u / ring_tiles, then the tile: rows below [iy0, iy1),
// rows above, then the left and right columns of the rows in between.
__host__ __device__ inline void ring_unit(const RevUnits& U, long long u, int* tx, int* ty, int* cz) {
  const long long ring = ring_tiles(U);
  *cz = (int)(u / ring);
  long long r = u % ring;
  const long long below = (long long)U.ntx * U.iy0;
  if (r < below) {
    *ty = (int)(r / U.ntx);
    *tx = (int)(r % U.ntx);
    return;
  }
  r -= below;
  const long long above = (long long)U.ntx * (U.nty - U.iy1);
  if (r < above) {
    *ty = U.iy1 + (int)(r / U.ntx);
    *tx = (int)(r % U.ntx);
    return;
  }
  r -= above;
  const int w = U.ix0 + (U.ntx - U.ix1);
  *ty = U.iy0 + (int)(r / w);
  const int c = (int)(r % w);
  *tx = c < U.ix0 ? c : U.ix1 + (c - U.ix0);
}

// ------------------------------------------------------------ launchers ----
// Implemented in kernels_step.cu / kernels_tape.cu; return cudaGetLastError().
// Tensor maps of the plane-staging kernels for a tw x ty tile: wide
// (tw+4) x (ty+1) boxes (own and one neighbour side), own tw x ty boxes;
// Q* view the per-axis auxiliary arrays of `pl` (4 components each): x own
// and (tw+4) x ty boxes, y own and tw x (ty+1) boxes, z own boxes.
struct alignas(64) LagMaps {
  CUtensorMap Fw, Fo, Lw, Lo, cbw, cbo, Qxo, Qxw, Qyo, Qyw, Qzo;
};
struct StepArgs {
  Geo g;
  float* F;        // fields
  float* cb;
  float* psiA;     // psi set read (and written in place by the forward)
  float* psiB;     // psi set written (ping-pong)
  float* L;        // adjoint fields (6 components, same layout as F)
  float* Fn;       // fused steps: fields written (the other buffer of a ping-pong pair);
                   // the forward half-steps write here when set, else in place
  float* Ln;       // fused reverse step: adjoint fields written
  float* Fm;       // two-step forward: the intermediate time level (frame of the deep box)
  double* gacc;    // FP64 design-box accumulator [dz][dy][dx]
  int dlo[3], dhi[3];
  Src src;
  Det det;
  double* obj;     // per-step objective slot
  float jn;        // J waveform value of this step
  int zchunk;
  int zc0, zc1;     // two-cells-per-thread kernels: z chunks [zc0, zc1) of this launch (zc1 = 0: to the last)
  int zcs;          // two-step forward: planes per z chunk of U (the split half-steps' chunks)
  int t0x, t0y;     // fused reverse step: first tile of a launch along x and y
  int umode;        // forward half-steps (32 x 8 tiles): 0 every unit of the grid (offset
                    // by zc0), 1 the z-only units of U, 2 the ring units of U
  RevUnits U;
  // batched designs (the BM kernel instantiations): CTA b runs unit bunits[b]
  // = (design, tile x, tile y, z chunk) of design bargs[design] (that
  // design's own arguments for this step) with the tensor maps bmaps[bmap]
  const int4* bunits;
  const StepArgs* bargs;
  const LagMaps* bmaps;
  int bmap;
  int bcount;       // units of a batched launch (its CTAs)
  int tile_y;
  int stages;      // ring stages of the one-plane kernels (2, 3 or 4)
  int pdl;         // launch the two-cells-per-thread kernels as programmatic dependents
  int prefetch;    // two-cells-per-thread kernels: warm L2 with the plane after the one staged
  int tile_x;      // two-cells-per-thread kernels: tile width (32 or 40 cells)
  PsiLayout pl;    // layout of the auxiliary sets the two-cells-per-thread kernels use
  int xq;          // exact reversal: increments rounded to multiples of 2^-xq (0 = off)
  float xs, xi;    // 2^xq, 2^-xq
  unsigned* err;   // device error word (ERR_*)
};

cudaError_t launch_prep(const float* eps, float* cb, Geo g, unsigned* err, cudaStream_t s);
// Plain-load half-steps (kernel 0, the independent cross-check of the staged
// kernels): one cell per thread, every neighbour read from global memory.
cudaError_t launch_fwd_h(const StepArgs& a, cudaStream_t s);
cudaError_t launch_fwd_e(const StepArgs& a, cudaStream_t s);
cudaError_t launch_rev_e(const StepArgs& a, cudaStream_t s);
cudaError_t launch_rev_h(const StepArgs& a, cudaStream_t s);

// Fwide (optional): the field buffer of the wide boxes Fw (the forward E
// half-step of a fused forward reads Ht^{n+1/2} from the buffer being written).
cudaError_t encode_lag_maps(const float* F, const float* L, const float* cb, const float* psiA,
                            const Geo& g, int ty, int tw, const PsiLayout& pl, LagMaps* m,
                            const float* Fwide = nullptr);
// Staged half-steps, two x-cells per thread (kernel 5; tile height >= 2).
// which: 0 forward H, 1 forward E, 2 reverse E phase, 3 reverse H phase.
cudaError_t launch_lag2(int which, const LagMaps& m, const StepArgs& a, cudaStream_t s);
// The fused steps (kernels_rev_fused.cu, kernels_fwd_fused.cu): tensor maps
// of 32 x 8 tiles over the current field, adjoint and auxiliary buffers
// (boxes: F40 / cb40 / L40 (TW+8) x (TY+2), F36 / cb36 / L36 (TW+4) x
// (TY+1), cb32 TW x TY, Qx40
// (TW+8) x (TY+1), Qy36 (TW+4) x (TY+2), Qz36 (TW+4) x (TY+1), Qxw (TW+4) x
// TY, Qyw TW x (TY+1), Qzo TW x TY).
struct alignas(64) RevMaps {
  CUtensorMap F40, F36, cb36, cb40, cb32, L40, L36, Qx40, Qy36, Qz36, Qxw, Qyw, Qzo;
};
cudaError_t encode_rev_maps(const float* F, const float* L, const float* cb, const float* psiA,
                            const Geo& g, const PsiLayout& pl, RevMaps* m);
// Tiles (32 x 8) and z chunks of the three launches of a fused reverse step:
// the primal one covers the tiles [px0, px1) x [py0, py1) and chunks
// [pz0, pz1) holding interior cells; the adjoint one without CPML terms the
// box [ix0, ix1) x [iy0, iy1) x [iz0, iz1) of units whose every evaluated
// term lies in the interior; the adjoint one with CPML every other unit of
// the ntx x nty x nzc grid.
RevUnits rev_units(const Geo& g, int zchunk);
// The CPML units split into z-only units (tiles inside [ix0, ix1) x
// [iy0, iy1), chunks outside [iz0, iz1)) and ring units (every other tile,
// every chunk); the launches' unit enumerations, for the host and tests.
void rev_zonly_unit(const RevUnits& U, int bx, int by, int bz, int* tx, int* ty, int* cz);
void rev_ring_unit(const RevUnits& U, long long u, int* tx, int* ty, int* cz);
long long rev_ring_tiles(const RevUnits& U);
// which: 0 primal (E^n, Ht^{n-1/2}, dL/dcb), 1 adjoint over the CPML-free
// units, 2 adjoint over the z-only units, 3 adjoint over the ring units.
// Reads a.F, a.L, a.psiA; writes a.Fn, a.Ln, a.psiB, a.gacc.
cudaError_t launch_rev_fused(int which, const RevMaps& m, const StepArgs& a, const RevUnits& U,
                             cudaStream_t s);
// The fused forward step (kernels_fwd_fused.cu) over the units [ix0, ix1) x
// [iy0, iy1) x [iz0, iz1) of U (none may hold a source or detector cell):
// reads a.F (E^n, Ht^{n-1/2}) and cb, writes a.Fn (E^{n+1}, Ht^{n+1/2}).
cudaError_t launch_fwd_fused(const RevMaps& m, const StepArgs& a, const RevUnits& U,
                             cudaStream_t s);
// Two forward time steps per pass (kernels_fwd_2step.cu): tensor maps over
// the fields (boxes 40 x 12, 3 components) and cb (40 x 10).
struct alignas(64) Fwd2Maps {
  CUtensorMap F4012, cb40;
};
cudaError_t encode_fwd2_maps(const float* F, const float* cb, const Geo& g, Fwd2Maps* m);
// The deep units of a grid for split z chunks of zcs planes: the tiles and
// full chunks ([ix0, ix1) x [iy0, iy1) x [iz0, iz1) of the ntx x nty x nzc
// grid of rev_units) on whose cells and two-cell halo a two-step pass
// evaluates no CPML term; the other units are U's z-only and ring units.
RevUnits deep_units(const Geo& g, int zcs);
// Steps n and n + 1 over the deep units U (chunks of a.zchunk planes, U's
// chunks of a.zcs planes; none may come within two cells of a source or
// detector cell): reads a.F (E^n, Ht^{n-1/2}) and cb, writes a.Fn (E^{n+2},
// Ht^{n+3/2}) and, on the one-cell frame of the deep box, a.Fm (E^{n+1},
// Ht^{n+1/2}).
cudaError_t launch_fwd_2step(const Fwd2Maps& m, const StepArgs& a, const RevUnits& U,
                             cudaStream_t s);
cudaError_t launch_finalize(const double* gacc, const float* cb, Geo g, const int* dlo,
                            const int* dhi, double scale, float* out, unsigned* err,
                            cudaStream_t s);
cudaError_t launch_gather(const float* F, Geo g, float* out, cudaStream_t s);
// One CTA waits (bounded by `limit` cycles) on an mbarrier nothing completes.
cudaError_t launch_wait_selftest(long long limit, unsigned* flag, cudaStream_t s);
// Objective of one detector plane for one step, added to *out (FP64).
cudaError_t launch_monitor(const float* F, Geo g, const Det& d, double* out, cudaStream_t s);
// FH holds Ht^{n+1/2} (low faces), FE holds E^n (high faces).
cudaError_t launch_record(int dtype, int scaled, const float* FH, const float* FE, Geo g,
                          const Faces& fc, void* tape_sample, float* scale_slot, cudaStream_t s);
// Seeds: det gets seeds[0], det2 (kind 0 = none) seeds[1] (device FP64).
cudaError_t launch_restore_seed(int dtype, float* F, float* L, Geo g, const Faces& fc,
                                const void* tape, long long sample_stride, const float* scales,
                                const Interp& ip, const Det& det, const Det& det2,
                                const double* seeds, cudaStream_t s);
// Batched designs: the record (unscaled formats) and restore launches of
// several designs in one launch, one job per design (lists in device memory).
struct RecordJob {
  const float* FH;
  const float* FE;
  Geo g;
  Faces fc;
  void* sample;
  float* scale_slot;
};
struct RestoreJob {
  float* F;
  float* L;
  Geo g;
  Faces fc;
  const void* tape;
  long long stride;
  const float* scales;
  Interp ip;
  Det det, det2;
  const double* seeds;
  int face_blocks, det_blocks;
};
cudaError_t launch_record_batch(int dtype, const RecordJob* jobs, int njobs, int max_blocks,
                                cudaStream_t s);
cudaError_t launch_restore_seed_batch(int dtype, const RestoreJob* jobs, int njobs,
                                      int max_blocks, cudaStream_t s);
void restore_blocks(const Faces& fc, const Det& det, const Det& det2, int* face_blocks,
                    int* det_blocks);
int record_flat_blocks(const Faces& fc);
cudaError_t launch_encode(int dtype, int scaled, const float* in, size_t n, void* code,
                          float* scale, cudaStream_t s);
cudaError_t launch_decode(int dtype, const void* code, size_t n, const float* scale, float* out,
                          cudaStream_t s);

}  // namespace fdtd
