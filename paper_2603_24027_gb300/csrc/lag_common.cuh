// lag_common.cuh -- pieces shared by the one-plane-per-iteration kernels
// (one and two x-cells per thread): CPML helpers, the plane ring, box
// geometry and the shared-memory stage layout of each half-step.
#pragma once

#include "fdtd_internal.cuh"
#include "tma.cuh"

namespace fdtd {

namespace lag {

constexpr int r128(int b) { return (b + 127) / 128 * 128; }

__device__ __forceinline__ float cpml_s(float d, float psi_old, float* pout, long long pi, float b,
                                        float a, float kv) {
  float s = __fmaf_rn(b, psi_old, __fmul_rn(a, d));
  pout[pi] = s;
  return __fmaf_rn(kv, d, s);
}

__device__ __forceinline__ float adj_s(float v, float lpsi, float* pout, long long pi, bool own,
                                       float b, float a, float kv) {
  float mu = lpsi + v;
  if (own) pout[pi] = b * mu;
  return kv * v + a * mu;
}

__device__ __forceinline__ float src_wt(const Src& s, int i, int j, int k) {
  int u, v;
  if (s.kind == 0 || !on_plane(s.axis, s.index, s.u0, s.u1, s.v0, s.v1, i, j, k, &u, &v))
    return 0.f;
  return __ldg(s.w + (long long)(v - s.v0) * (s.u1 - s.u0) + (u - s.u0));
}

__device__ __forceinline__ bool tile_in_slab(int lo, int hi_incl, int n, int P) {
  return lo < P || hi_incl >= n - P;
}

// Ring over planes p0..p1 (see kernels_split_tma.cu): plane p in stage
// (p - p0) % S, barrier parity ((p - p0) / S) & 1.  Here every plane is read
// in exactly one iteration, after which its stage is re-armed for p + S.
template <int S>
struct Ring {
  unsigned char* base;
  uint64_t* bars;
  int stage_bytes, p0, p1;
  __device__ unsigned char* at(int p) const { return base + ((p - p0) % S) * stage_bytes; }
  __device__ uint64_t* bar(int p) const { return &bars[(p - p0) % S]; }
  __device__ bool wait(int p) const {
    return mbar_wait(bar(p), ((p - p0) / S) & 1, kWaitCycles);
  }
};

template <int S>
__device__ __forceinline__ Ring<S> ring_setup(unsigned char* dsm, int stage_bytes, int p0, int p1) {
  Ring<S> r;
  r.base = dsm;
  r.bars = reinterpret_cast<uint64_t*>(dsm + S * stage_bytes);
  r.stage_bytes = stage_bytes;
  r.p0 = p0;
  r.p1 = p1;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&r.bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  return r;
}

template <int S>
__device__ void ring_drain(const Ring<S>& r, int p_waited, unsigned* err) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomicOr(err, ERR_TIMEOUT);
    for (int p = p_waited; p <= r.p1 && p < p_waited + S; ++p) r.wait(p);
  }
}

// Box geometry of a TW x TY tile: "lo" boxes start at (x0-4, y0-1) and cover
// own, -x, -y; "hi" boxes start at (x0, y0) and cover own, +x, +y.  Both are
// (TW+4) x (TY+1).
template <int TY, int TW = 32>
struct G {
  static constexpr int W = TW + 4, R = TY + 1, P = W * R;   // wide box plane
  static constexpr int OP = TW * TY;                         // own box plane
  static constexpr int XP = W * TY;                          // (TW+4) x TY psi box (x neighbour)
  static constexpr int YP = TW * (TY + 1);                   // TW x (TY+1) psi box (y neighbour)
};

}  // namespace lag

using namespace lag;

// Stage layouts (byte offsets of each box in one ring stage).
// Forward H half-step: E hi box, Ht own, psi_H own boxes of the three axes.
template <int TY, int S, int TW = 32>
struct LFH {
  typedef G<TY, TW> g_;
  static constexpr int E = 0;                                  // E hi box, 3 comps
  static constexpr int H = r128(3 * g_::P * 4);                // H own
  static constexpr int PX = H + r128(3 * g_::OP * 4);          // psi_H own x/y/z, 2 comps
  static constexpr int PY = PX + r128(2 * g_::OP * 4);
  static constexpr int PZ = PY + r128(2 * g_::OP * 4);
  static constexpr int STAGE = PZ + r128(2 * g_::OP * 4);
  static int smem() { return S * STAGE + 8 * S; }
};

// Forward E half-step: Ht lo box, E and cb own, psi_E own boxes; a small
// tail holds the per-warp objective partial sums.
template <int TY, int S, int TW = 32>
struct LFE {
  typedef G<TY, TW> g_;
  static constexpr int H = 0;                                  // Ht lo box
  static constexpr int E = r128(3 * g_::P * 4);                // E own
  static constexpr int CB = E + r128(3 * g_::OP * 4);          // cb own
  static constexpr int PX = CB + r128(g_::OP * 4);             // psi_E own x/y/z
  static constexpr int PY = PX + r128(2 * g_::OP * 4);
  static constexpr int PZ = PY + r128(2 * g_::OP * 4);
  static constexpr int STAGE = PZ + r128(2 * g_::OP * 4);
  static int smem() { return S * STAGE + 8 * S + 256; }
};

// Reverse E phase: Ht lo box, E own, cb and lam_E hi boxes, lam_H own,
// lam_psi_E boxes that reach the +x / +y neighbour.
template <int TY, int S, int TW = 32>
struct LRE {
  typedef G<TY, TW> g_;
  static constexpr int H = 0;                                  // Ht lo box
  static constexpr int E = r128(3 * g_::P * 4);                // E own
  static constexpr int CB = E + r128(3 * g_::OP * 4);          // cb hi box
  static constexpr int LE = CB + r128(g_::P * 4);              // lam_E hi box
  static constexpr int LH = LE + r128(3 * g_::P * 4);          // lam_H own
  static constexpr int PX = LH + r128(3 * g_::OP * 4);         // lam_psi_E x: 36 x TY at (x0, y0)
  static constexpr int PY = PX + r128(2 * g_::XP * 4);         // lam_psi_E y: 32 x (TY+1) at (x0, y0)
  static constexpr int PZ = PY + r128(2 * g_::YP * 4);         // lam_psi_E z: own
  static constexpr int STAGE = PZ + r128(2 * g_::OP * 4);
  static int smem() { return S * STAGE + 8 * S; }
};

// Reverse H phase: E hi box, Ht own, lam_H lo box, lam_E own, lam_psi_H
// boxes that reach the -x / -y neighbour.
template <int TY, int S, int TW = 32>
struct LRH {
  typedef G<TY, TW> g_;
  static constexpr int E = 0;                                  // E hi box
  static constexpr int H = r128(3 * g_::P * 4);                // Ht own
  static constexpr int LH = H + r128(3 * g_::OP * 4);          // lam_H lo box
  static constexpr int LE = LH + r128(3 * g_::P * 4);          // lam_E own
  static constexpr int PX = LE + r128(3 * g_::OP * 4);         // lam_psi_H x: 36 x TY at (x0-4, y0)
  static constexpr int PY = PX + r128(2 * g_::XP * 4);         // lam_psi_H y: 32 x (TY+1) at (x0, y0-1)
  static constexpr int PZ = PY + r128(2 * g_::YP * 4);         // lam_psi_H z: own
  static constexpr int STAGE = PZ + r128(2 * g_::OP * 4);
  static int smem() { return S * STAGE + 8 * S; }
};

}  // namespace fdtd
