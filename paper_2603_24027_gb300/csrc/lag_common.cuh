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

// Helpers of the two-cells-per-thread kernels (kernels_lag2.cu and the fused
// reverse step, kernels_rev_fused.cu).
namespace lag2 {

__device__ __forceinline__ float2 ld2(const float* b, int i) {
  return *reinterpret_cast<const float2*>(b + i);
}

// Store the pair (u, v) at element offset q (q even, 8-byte aligned because
// the row pitch is a multiple of 8): one 8-byte store when both cells are
// written, else the flagged one.
__device__ __forceinline__ void st2(float* p, long long q, float u, float v, bool f0, bool f1) {
  if (f0 && f1) {
    *reinterpret_cast<float2*>(p + q) = make_float2(u, v);
  } else {
    if (f0) p[q] = u;
    if (f1) p[q + 1] = v;
  }
}

#ifdef FDTD_BOUNDS_CHECK
// Bounds-checked test build: a store must land in the fields, the adjoint
// fields or one of the two auxiliary sets of the launch, else it is skipped
// and the error word records ERR_BOUNDS.
__device__ __forceinline__ bool in_buf(const float* p, const float* base, long long n) {
  return base && p >= base && p < base + n;
}
__device__ __forceinline__ bool store_ok(const StepArgs& a, const float* p) {
  const long long n6 = 6 * a.g.nc;
  if (in_buf(p, a.F, n6) || in_buf(p, a.L, n6) || in_buf(p, a.Fn, n6) || in_buf(p, a.Ln, n6) ||
      in_buf(p, a.Fm, n6) ||
      in_buf(p, a.psiA, a.pl.total) || in_buf(p, a.psiB, a.pl.total))
    return true;
  atomicOr(a.err, ERR_BOUNDS);
  return false;
}
#define ST2(p, q, u, v, f0, f1) \
  st2(p, q, u, v, (f0) && store_ok(a, (p) + (q)), (f1) && store_ok(a, (p) + (q) + 1))
#else
#define ST2(p, q, u, v, f0, f1) st2(p, q, u, v, f0, f1)
#endif

// Forward CPML recursion of one derivative d (Eq. 5 form): the updated psi
// goes to *s, the stretched derivative is returned.
__device__ __forceinline__ float cpml(float d, float psi_old, float b, float a, float kv, float* s) {
  const float t = __fmaf_rn(b, psi_old, __fmul_rn(a, d));
  *s = t;
  return __fmaf_rn(kv, d, t);
}

// Adjoint of the recursion: returns the curl term with the CPML response;
// the adjoint auxiliary for the next (earlier) step goes to *out.
__device__ __forceinline__ float adj(float v, float lpsi, float b, float a, float kv, float* out) {
  const float mu = lpsi + v;
  *out = b * mu;
  return kv * v + a * mu;
}

// Programmatic dependent launch: wait until the previous kernel in the stream
// has completed and its writes are visible (nothing before this point reads
// or writes data another kernel touches), then allow the next kernel's CTAs
// to start their own prologue as this grid's CTAs retire.  Without a
// programmatic dependency both are no-ops.
__device__ __forceinline__ void pdl_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Stage plane p: boxes(p, f) calls f(stage offset, tensor map, x, y, z,
// component, bytes) for every box the kernel needs of plane p (z is p, or its
// row in a compact auxiliary array).  The barrier expects the sum of the
// boxes' bytes, then every box is loaded; with prefetch, plane p + 1's boxes
// are also warmed in L2 so that their own load, one iteration later, finds
// them closer (only planes inside [0, nz) and the ring).
template <class Boxes>
__device__ __forceinline__ void stage_plane(const Boxes& boxes, int p, unsigned char* st,
                                            uint64_t* bar, bool prefetch_next) {
  // The CTA's generic-proxy reads of the stage's previous plane (ordered
  // before this point by the caller's __syncthreads) must also be ordered
  // before the async-proxy (TMA) writes that refill it: a barrier alone does
  // not order the two proxies.
  fence_proxy_async_smem();
  uint32_t bytes = 0;
  boxes(p, [&](int, const CUtensorMap*, int, int, int, int, uint32_t b) { bytes += b; });
  mbar_expect_tx(bar, bytes);
  boxes(p, [&](int off, const CUtensorMap* mp, int x, int y, int z, int c, uint32_t) {
    tma_load_4d(st + off, mp, bar, x, y, z, c);
  });
  if (prefetch_next)
    boxes(p + 1, [&](int, const CUtensorMap* mp, int x, int y, int z, int c, uint32_t) {
      tma_prefetch_l2_4d(mp, x, y, z, c);
    });
}

// Start coordinates of a tile's boxes in the per-axis auxiliary arrays: a
// tile whose boxes reach the mapped (high) part of the axis uses the mapped
// start, so that its slab cells land where the array holds them (its other
// cells are not slab cells and never read their auxiliaries).  TW + 4 / TY + 1
// cover the widest box of any kernel.
template <int TW, int TY>
__device__ __forceinline__ void psi_box_starts(const PsiLayout& pl, int x0, int y0, int* qx0,
                                               int* qy0) {
  const PsiAxis& X = pl.ax[0];
  const PsiAxis& Yy = pl.ax[1];
  *qx0 = x0 + TW + 4 > X.hs ? x0 - X.shift : x0;
  *qy0 = y0 + TY + 1 > Yy.hs ? y0 - Yy.shift : y0;
}

// A field increment of the leapfrog; EX (exact reversal) rounds it to the
// grid of multiples of 2^-xq (see grid_inc), compiled in only where used.
template <bool EX>
__device__ __forceinline__ float inc_of(float d, const StepArgs& a) {
  return EX ? grid_inc(d, 1, a.xs, a.xi) : d;
}

// Resident CTAs per SM the register allocation must allow for the default
// 32 x 8 tiles with two stages: eight for the forward half-steps (what their
// shared memory allows), five for the reverse phases (idem); other shapes
// leave the allocation to the compiler.
template <int TY, int S, int TW>
constexpr int min_ctas(bool fwd) {
  return (TY == 8 && S == 2 && TW == 32) ? (fwd ? 8 : 5) : 1;
}

template <int S>
__device__ __forceinline__ uint64_t* ring_init(unsigned char* dsm, int stage_bytes) {
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + S * stage_bytes);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  return bars;
}

// A wait for plane p (stage stg, parity par) gave up: record the timeout and
// wait, bounded, for the copies still in flight (planes p .. min(p1, p+S-1))
// so that no copy lands in shared memory after the CTA has left.
template <int S>
__device__ void ring_abort(uint64_t* bars, int stg, uint32_t par, int p, int p1, unsigned* err) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomicOr(err, ERR_TIMEOUT);
    for (int i = 0; i < S && p + i <= p1; ++i) {
      int s = stg + i;
      uint32_t ph = par;
      if (s >= S) {
        s -= S;
        ph ^= 1u;
      }
      mbar_wait(&bars[s], ph, kWaitCycles);
    }
  }
}

}  // namespace lag2


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
